// fd_guard.cu -- learned rollout with the plain FV step as its fallback.
//
// The learned module only adds learnable parts to the FV module; with them
// removed the step is the traditional solver (Sec. 3.4: O = O_P alone; the
// "DNS" rows of the Sec. 4 ablation). fd_rollout_guarded advances a batch in
// chunks: every chunk runs both the learned rollout and the plain rollout from
// the same chunk-start state, then one kernel per trajectory keeps the learned
// result while it is finite and switches the trajectory to the plain result
// for good once a learned chunk of it produced a NaN or Inf. The plain chunk
// costs about a hundredth of the learned one (no network), so running it for
// the whole batch keeps the call free of host synchronisation.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/fd.h"
#include "fd_ctx.h"

fd_status fd_rollout_impl(fd_ctx* c, const void* u0, void* traj, void* u_final, int32_t n_steps, int32_t save_every,
                          void* stream, bool allow_graph);

namespace {

// One CTA per trajectory: out[b] = learned[b] unless learned[b] holds a
// non-finite value or the trajectory fell back in an earlier chunk, in which
// case out[b] = plain[b]; fell[b] records the first step of the chunk where
// the trajectory fell back (-1 = never).
__global__ void __launch_bounds__(256) guard_select_kernel(const float* __restrict__ learned,
                                                           const float* __restrict__ plain, float* __restrict__ out,
                                                           int32_t* __restrict__ fell, long long per_traj,
                                                           int32_t step0) {
  const int b = blockIdx.x;
  const long long base = (long long)b * per_traj;
  const int before = fell[b];
  int bad = 0;
  for (long long i = threadIdx.x; i < per_traj; i += blockDim.x) bad |= isfinite(learned[base + i]) ? 0 : 1;
  bad = __syncthreads_or(bad);
  const bool use_plain = before >= 0 || bad;
  if (threadIdx.x == 0 && before < 0 && bad) fell[b] = step0;
  const float* src = use_plain ? plain : learned;
  for (long long i = threadIdx.x; i < per_traj; i += blockDim.x) out[base + i] = src[base + i];
}

}  // namespace

extern "C" {

fd_status fd_rollout_guarded(fd_ctx* c, const void* u0, void* u_final, int32_t n_steps, int32_t chunk,
                             int32_t* fell_back, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_rollout_guarded: null context");
  c->launches = 0;
  if (!u0 || !u_final || !fell_back) return fd_set_error(c, FD_EINVAL, "fd_rollout_guarded: null pointer");
  if (!c->lrn)
    return fd_set_error(c, FD_EUNSUPPORTED, c->glrn ? "fd_rollout_guarded: built for the tensor-core learned path (32^2, 64^2)"
                                                    : "fd_rollout_guarded: needs a learned context");
  if (n_steps < 0) return fd_set_error(c, FD_EINVAL, "fd_rollout_guarded: n_steps must be >= 0");
  const int kc = c->opts.k_c;
  if (chunk <= 0) chunk = kc > 0 ? kc : 8;
  if (kc > 0 && chunk % kc != 0)
    return fd_set_error(c, FD_EINVAL, "fd_rollout_guarded: chunk must be a multiple of k_c (%d)", kc);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = fd_state_bytes(c->grid);
  const long long per_traj = (long long)(bytes / sizeof(float)) / c->grid.batch;
  if (!c->fallback) {
    fd_options o = c->opts;
    o.learned = 0;
    o.k_c = 0;
    o.fno_layers = o.fno_modes = o.fno_width = 0;
    o.tc_fno_layers = o.tc_fno_modes = o.tc_fno_width = 0;
    o.ablation = 0;
    o.path = 0;
    fd_ctx* p = nullptr;
    fd_status s = fd_init(&c->grid, c->nu, c->dt, &c->forcing, &o, &p);
    if (s != FD_OK) return fd_set_error(c, s, "fd_rollout_guarded: plain solver: %s", fd_last_error(nullptr));
    c->fallback = p;
  }
  if (!c->d_guard) {
    cudaError_t e = cudaMalloc(&c->d_guard, 3 * bytes);
    if (e != cudaSuccess) {
      c->d_guard = nullptr;
      return fd_set_error(c, FD_ENOMEM, "fd_rollout_guarded: cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  float* cur = static_cast<float*>(c->d_guard);
  float* lout = cur + bytes / sizeof(float);
  float* pout = lout + bytes / sizeof(float);
  cudaError_t e = cudaMemsetAsync(fell_back, 0xff, (size_t)c->grid.batch * sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cur, u0, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout_guarded: %s", cudaGetErrorString(e));
  int launches = 0;
  for (int done = 0; done < n_steps; done += chunk) {
    const int len = n_steps - done < chunk ? n_steps - done : chunk;
    fd_status s = fd_rollout_impl(c, cur, nullptr, lout, len, 0, stream, true);
    if (s != FD_OK) return s;
    launches += c->launches;
    s = fd_rollout_impl(c->fallback, cur, nullptr, pout, len, 0, stream, true);
    if (s != FD_OK) return fd_set_error(c, s, "fd_rollout_guarded: plain chunk: %s", fd_last_error(c->fallback));
    launches += fd_last_launch_count(c->fallback);
    guard_select_kernel<<<c->grid.batch, 256, 0, st>>>(lout, pout, cur, fell_back, per_traj, done);
    ++launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout_guarded: select: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(u_final, cur, bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout_guarded: %s", cudaGetErrorString(e));
  c->launches = launches;
  return FD_OK;
}

}  // extern "C"
