// fd_mixed.cu -- the persistent launch of a mixed batch: every trajectory of
// the batch's plain single-precision on-chip contexts with N = 16, 32 or 64
// (any flow type, forcing, viscosity and step) goes into one work list that
// one launch of fv_mixed_rollout_kernel works through, instead of one kernel
// per context. Used by fd_batch_run.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "fd_ctx.h"
#include "fv_fused.cuh"

using namespace ldfv;

bool fd_mixed_eligible(const fd_ctx* c) {
  const int n = c->grid.nx;
  return !c->lrn && !c->gen && !c->big && c->grid.dtype == FD_F32 && c->grid.ny == n && (n == 16 || n == 32 || n == 64) &&
         c->n_stream == 0 && c->n_onchip == c->grid.batch && (c->opts.deriv_order == 2 || c->opts.deriv_order == 4);
}

void fd_mixed_items(const fd_ctx* c, const void* u0, void* u_final, int n_steps, std::vector<MixedItem>& out) {
  FvArgs a = c->base;
  a.u_in = u0;
  a.u_out = u_final;
  a.traj = nullptr;
  a.n_steps = n_steps;
  a.save_every = 0;
  a.traj_batch = 0;
  for (int t = 0; t < c->grid.batch; ++t) out.push_back(MixedItem{a, t, c->logn});
}

// the largest trajectories first: the launch's tail is then made of short items
void fd_mixed_order(std::vector<MixedItem>& items) {
  std::stable_sort(items.begin(), items.end(), [](const MixedItem& x, const MixedItem& y) {
    return (double)x.a.n_steps * (1 << (2 * x.logn)) > (double)y.a.n_steps * (1 << (2 * y.logn));
  });
}

namespace {

template <int DORD>
int& grid_of() {
  static int grid = 0;  // CTAs resident at once (set by prepare_dord)
  return grid;
}

template <int DORD>
cudaError_t prepare_dord() {
  int& grid = grid_of<DORD>();
  cudaError_t e = cudaSuccess;
  if (grid == 0) {
    const int smem = (int)mixed_smem<float>();
    e = cudaFuncSetAttribute(fv_mixed_rollout_kernel<DORD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fv_mixed_rollout_kernel<DORD>, kMixedNT, smem);
    if (e != cudaSuccess) return e;
    // tensor memory: at most 512 / kMixedTmemCols CTAs of this kernel per SM
    per_sm = std::min(per_sm, 512 / kMixedTmemCols);
    grid = std::max(1, per_sm * sms);
  }
  return e;
}

template <int DORD>
cudaError_t launch_dord(const MixedItem* d_items, int n, unsigned* d_counter, cudaStream_t st) {
  const int grid = grid_of<DORD>();
  if (grid == 0) return cudaErrorNotReady;  // fd_mixed_prepare was not called
  const int g = std::min(grid, n);
  fv_mixed_rollout_kernel<DORD><<<g, kMixedNT, mixed_smem<float>(), st>>>(d_items, n, d_counter);
  return cudaGetLastError();
}

}  // namespace

// sets the kernel attributes and sizes the grid; call outside stream capture
cudaError_t fd_mixed_prepare(int dord) { return dord == 2 ? prepare_dord<2>() : prepare_dord<4>(); }

cudaError_t fd_mixed_launch(const MixedItem* d_items, int n, unsigned* d_counter, int dord, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  return dord == 2 ? launch_dord<2>(d_items, n, d_counter, st) : launch_dord<4>(d_items, n, d_counter, st);
}
