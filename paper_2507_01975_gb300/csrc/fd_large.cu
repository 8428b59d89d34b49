// fd_large.cu -- plain FV rollouts on grids that stream through HBM (N = 512 ..
// 2048, or any N >= 32 on request): workspace, the 17-launch step, and its
// replay as a CUDA graph.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fv_large.cuh"

using namespace ldfv;

namespace {

// the three projection kernels of one stage, instantiated per grid size
template <int LOGN>
cudaError_t projection(const LargeArgs& a, int B, cudaStream_t st) {
  using R = RowCfg<LOGN>;
  using C = ColCfg<LOGN>;
  const dim3 grow(R::N / R::RG, B);
  const dim3 gcol((R::N / 2 + 1 + C::C - 1) / C::C, B);
  cudaError_t e = launch_pdl(large_rows_fwd_kernel<LOGN>, grow, dim3(R::NT), R::SMEM, st, a);
  if (e == cudaSuccess) e = launch_pdl(large_cols_kernel<LOGN>, gcol, dim3(C::NT), C::SMEM, st, a);
  if (e == cudaSuccess) e = launch_pdl(large_rows_inv_kernel<LOGN>, grow, dim3(R::NT), R::SMEM, st, a);
  return e;
}

template <int LOGN>
cudaError_t prepare_projection() {
  cudaError_t e = cudaFuncSetAttribute(large_rows_fwd_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)RowCfg<LOGN>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(large_cols_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ColCfg<LOGN>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(large_rows_inv_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)RowCfg<LOGN>::SMEM);
  return e;
}

cudaError_t dispatch_projection(int logn, const LargeArgs* a, int B, cudaStream_t st) {
  switch (logn) {
#define LDFV_PROJ(L) \
  case L:            \
    return a ? projection<L>(*a, B, st) : prepare_projection<L>();
    LDFV_PROJ(5)
    LDFV_PROJ(6)
    LDFV_PROJ(7)
    LDFV_PROJ(8)
    LDFV_PROJ(9)
    LDFV_PROJ(10)
    LDFV_PROJ(11)
#undef LDFV_PROJ
    default:
      return cudaErrorInvalidValue;
  }
}

LargeArgs base_args(fd_ctx* c) {
  LargeArgs a;
  std::memset(&a, 0, sizeof a);
  const FvArgs& f = c->base;
  LargeState& S = *c->big;
  a.un = S.un;
  a.acc = S.acc;
  a.spec = reinterpret_cast<float2*>(S.spec);
  a.pout = S.p;
  a.flow = c->grid.flow;
  a.forcing = c->forcing.kind;
  a.dt = (float)f.dt;
  a.nu = (float)f.nu;
  a.idx = (float)f.idx;
  a.idy = (float)f.idy;
  a.drag = (float)f.drag;
  a.inv_nn = (float)f.inv_nn;
  a.tw = reinterpret_cast<const float2*>(f.tw);
  a.symx = reinterpret_cast<const float*>(f.symx);
  a.symy = reinterpret_cast<const float*>(f.symy);
  a.frc = reinterpret_cast<const float*>(f.frc);
  return a;
}

// one time step u_n (S.un) -> u_{n+1} (S.un): 17 launches (Navier-Stokes), 5 (Burgers)
cudaError_t large_step(fd_ctx* c, cudaStream_t st) {
  LargeState& S = *c->big;
  const int n = c->grid.nx, logn = c->logn, B = c->grid.batch;
  LargeArgs a = base_args(c);
  float* wsb[2] = {S.wsA, S.wsB};
  const int tx = n >= 64 ? 64 : 32;  // stage tile width
  const dim3 gst(n / tx, n / kLTY, B);
  cudaError_t e = cudaSuccess;
  // Burgers has no pressure: the stages chain without projections
  const bool ns = c->grid.flow == FD_NAVIER_STOKES;
  for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
    a.stage = s;
    a.x = s == 0 ? S.un : wsb[(s - 1) & 1];
    a.p = (s == 0 || !ns) ? nullptr : S.p;
    a.ws = wsb[s & 1];
    if (tx == 64) {
      e = c->opts.deriv_order == 4 ? launch_pdl(large_stage_kernel<4, 64>, gst, dim3(256), 0, st, a, logn)
                                   : launch_pdl(large_stage_kernel<2, 64>, gst, dim3(256), 0, st, a, logn);
    } else {
      e = c->opts.deriv_order == 4 ? launch_pdl(large_stage_kernel<4, 32>, gst, dim3(128), 0, st, a, logn)
                                   : launch_pdl(large_stage_kernel<2, 32>, gst, dim3(128), 0, st, a, logn);
    }
    if (ns && e == cudaSuccess) e = dispatch_projection(logn, &a, B, st);
  }
  if (e == cudaSuccess) {
    a.ws = wsb[1];
    a.uout = S.un;
    if (!ns) a.pout = nullptr;
    const size_t quads = (size_t)B * n * n / 4;
    const int blocks = (int)((quads + 255) / 256 < 8192 ? (quads + 255) / 256 : 8192);
    e = launch_pdl(large_final_kernel, dim3(blocks), dim3(256), 0, st, a, logn, B);
  }
  return e;
}

}  // namespace

bool fd_large_supported(int dtype, int n) { return dtype == FD_F32 && n >= 32 && n <= 2048; }

fd_status fd_large_init(fd_ctx* c) {
  LargeState* S = new (std::nothrow) LargeState();
  if (!S) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: out of host memory");
  c->big = S;
  const size_t n = c->grid.nx, B = c->grid.batch;
  const size_t state = B * 2 * n * n * sizeof(float);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&S->un, state);
  alloc((void**)&S->acc, state);
  alloc((void**)&S->wsA, state);
  alloc((void**)&S->wsB, state);
  alloc((void**)&S->p, B * n * n * sizeof(float));
  alloc(&S->spec, B * (n / kLRB) * (n / 2 + 1) * kLRB * 8);
  if (e == cudaSuccess) e = dispatch_projection(c->logn, nullptr, 0, nullptr);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: streaming workspace: %s", cudaGetErrorString(e));
  return FD_OK;
}

void fd_large_free(fd_ctx* c) {
  LargeState* S = c->big;
  if (!S) return;
  if (S->graph) cudaGraphExecDestroy(S->graph);
  if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
  void* ps[] = {S->un, S->acc, S->wsA, S->wsB, S->p, S->spec};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete S;
  c->big = nullptr;
}

fd_status fd_large_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                           cudaStream_t st, bool allow_graph) {
  LargeState& S = *c->big;
  const size_t bytes = fd_state_bytes(c->grid);
  cudaError_t e = cudaMemcpyAsync(S.un, u0, bytes, cudaMemcpyDeviceToDevice, st);
  int launches = 0;
  const bool use_graph = allow_graph && save_every == 0;
  if (e == cudaSuccess && use_graph && n_steps > 0 && !S.graph) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = large_step(c, S.cap_stream);
      cudaError_t e2 = cudaStreamEndCapture(S.cap_stream, &g);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S.graph, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  int snap = 0;
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    if (use_graph) {
      e = cudaGraphLaunch(S.graph, st);
    } else {
      e = large_step(c, st);
      if (e == cudaSuccess && traj && save_every > 0 && (k + 1) % save_every == 0) {
        const size_t stride = S.snap_stride ? S.snap_stride : bytes;
        e = cudaMemcpyAsync(static_cast<char*>(traj) + (size_t)snap * stride, S.un, bytes, cudaMemcpyDeviceToDevice,
                            st);
        ++snap;
      }
    }
    launches += c->grid.flow == FD_NAVIER_STOKES ? 17 : 5;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, S.un, bytes, cudaMemcpyDeviceToDevice, st);
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout (streaming path): %s", cudaGetErrorString(e));
  return FD_OK;
}
