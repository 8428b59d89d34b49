// fd_generic.cu -- plain FV for Burgers' equation on any grid: non-power-of-two
// and rectangular nx x ny (App. C.1 Burgers on [0, 1]^2 at 100^2 and 25^2,
// Table S2), FP32 or FP64.
//
// Burgers has no pressure projection, so a step needs no FFT: four launches of
// generic_stage_kernel per RK4 step (App. B.5), each thread forming the
// tendency of a strip of 4 cells of one row with the same flux-block
// arithmetic as the other paths (strip_tendency: face values of the eight
// operator instances, flux assembly and divergence, the Burgers correction,
// forcing) from a 5 x 8 window gathered with periodic wrap, then the RK
// combination. The last strip of a row is ragged when 4 does not divide nx.
// A step is captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fv_common.cuh"

using namespace ldfv;

namespace {

template <typename T>
struct GenArgs {
  const T* w;    // stage state [batch][2][ny][nx]
  const T* un;   // state at the start of the step
  T* acc;        // RK4 accumulator
  T* wout;       // next stage state (stage 3: the new state)
  const T* frc;  // [ny] forcing amplitude at the u-face rows
  int nx, ny, stage, forced;
  T dt, nu, idx, idy, drag;
};

template <typename T, int DORD>
__global__ void __launch_bounds__(256) generic_stage_kernel(const GenArgs<T> a) {
  const int strips = (a.nx + 3) >> 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= strips * a.ny) return;
  const int row = q / strips, col0 = (q - row * strips) * 4;
  const size_t NN = (size_t)a.nx * a.ny;
  const T* wu = a.w + (size_t)blockIdx.y * 2 * NN;
  const T* wv = wu + NN;
  T u[5][8], v[5][8];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int j = (row - 2 + r + a.ny) % a.ny;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int i = (col0 - 2 + c + a.nx) % a.nx;
      u[r][c] = wu[(size_t)j * a.nx + i];
      v[r][c] = wv[(size_t)j * a.nx + i];
    }
  }
  T tu[4], tv[4];
  strip_tendency<T, DORD>(u, v, a.idx, a.idy, a.nu, true, a.forced != 0, a.frc[row], a.drag, tu, tv);
  const T h6 = a.dt / (T)6, h3 = a.dt / (T)3, h2 = a.dt * (T)0.5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = col0 + k;
    if (i >= a.nx) break;
    const size_t e = (size_t)blockIdx.y * 2 * NN + (size_t)row * a.nx + i;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const size_t ef = e + f * NN;
      const T r = f == 0 ? tu[k] : tv[k];
      switch (a.stage) {
        case 0: {
          const T un = a.un[ef];
          a.acc[ef] = un + h6 * r;
          a.wout[ef] = un + h2 * r;
          break;
        }
        case 1:
          a.acc[ef] += h3 * r;
          a.wout[ef] = a.un[ef] + h2 * r;
          break;
        case 2:
          a.acc[ef] += h3 * r;
          a.wout[ef] = a.un[ef] + a.dt * r;
          break;
        default:
          a.wout[ef] = a.acc[ef] + h6 * r;
      }
    }
  }
}

template <typename T>
cudaError_t generic_step(fd_ctx* c, cudaStream_t st) {
  GenericState& S = *c->gen;
  const fd_grid& g = c->grid;
  GenArgs<T> a;
  a.un = static_cast<const T*>(S.un);
  a.acc = static_cast<T*>(S.acc);
  a.frc = static_cast<const T*>(S.frc);
  a.nx = g.nx;
  a.ny = g.ny;
  a.forced = c->forcing.kind;
  a.dt = (T)c->dt;
  a.nu = (T)c->nu;
  a.idx = (T)(g.nx / g.lx);
  a.idy = (T)(g.ny / g.ly);
  a.drag = (T)(c->forcing.kind == 1 ? c->forcing.drag : 0.0);
  const int strips = (g.nx + 3) / 4;
  const dim3 grid((unsigned)(((size_t)strips * g.ny + 255) / 256), (unsigned)g.batch);
  T* const stage_out[4] = {static_cast<T*>(S.wa), static_cast<T*>(S.wb), static_cast<T*>(S.wa), static_cast<T*>(S.un)};
  const T* const stage_in[4] = {static_cast<const T*>(S.un), static_cast<const T*>(S.wa),
                                static_cast<const T*>(S.wb), static_cast<const T*>(S.wa)};
  for (int s = 0; s < 4; ++s) {
    a.stage = s;
    a.w = stage_in[s];
    a.wout = stage_out[s];
    if (c->opts.deriv_order == 4)
      generic_stage_kernel<T, 4><<<grid, 256, 0, st>>>(a);
    else
      generic_stage_kernel<T, 2><<<grid, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t generic_step_any(fd_ctx* c, cudaStream_t st) {
  return c->grid.dtype == FD_F64 ? generic_step<double>(c, st) : generic_step<float>(c, st);
}

}  // namespace

bool fd_generic_wanted(const fd_grid& g, int path) {
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  return g.flow == FD_BURGERS && (path == 3 || !pow2(g.nx) || !pow2(g.ny) || g.nx != g.ny);
}

fd_status fd_generic_init(fd_ctx* c) {
  GenericState* S = new (std::nothrow) GenericState();
  if (!S) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: out of host memory");
  c->gen = S;
  const fd_grid& g = c->grid;
  const size_t bytes = fd_state_bytes(g);
  const size_t es = g.dtype == FD_F64 ? sizeof(double) : sizeof(float);
  cudaError_t e = cudaSuccess;
  void** bufs[4] = {&S->un, &S->wa, &S->wb, &S->acc};
  for (void** p : bufs)
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&S->frc, (size_t)g.ny * es);
  if (e == cudaSuccess) {
    // f_x = amp sin(k y) at the u-face rows y = (j + 1/2) dy (App. C.1 forced flow)
    const double dy = g.ly / g.ny;
    if (g.dtype == FD_F64) {
      std::vector<double> f(g.ny);
      for (int j = 0; j < g.ny; ++j)
        f[j] = c->forcing.kind == 1 ? c->forcing.amp * std::sin(c->forcing.k * (j + 0.5) * dy) : 0.0;
      e = cudaMemcpy(S->frc, f.data(), g.ny * es, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> f(g.ny);
      for (int j = 0; j < g.ny; ++j)
        f[j] = c->forcing.kind == 1 ? (float)(c->forcing.amp * std::sin(c->forcing.k * (j + 0.5) * dy)) : 0.0f;
      e = cudaMemcpy(S->frc, f.data(), g.ny * es, cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: generic-grid workspace: %s", cudaGetErrorString(e));
  return FD_OK;
}

void fd_generic_free(fd_ctx* c) {
  GenericState* S = c->gen;
  if (!S) return;
  if (S->graph) cudaGraphExecDestroy(S->graph);
  if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
  void* ps[] = {S->un, S->wa, S->wb, S->acc, S->frc};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete S;
  c->gen = nullptr;
}

fd_status fd_generic_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                             cudaStream_t st, bool allow_graph) {
  GenericState& S = *c->gen;
  const size_t bytes = fd_state_bytes(c->grid);
  cudaError_t e = cudaMemcpyAsync(S.un, u0, bytes, cudaMemcpyDeviceToDevice, st);
  const bool use_graph = allow_graph && save_every == 0;
  if (e == cudaSuccess && use_graph && n_steps > 0 && !S.graph) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = generic_step_any(c, S.cap_stream);
      const cudaError_t e2 = cudaStreamEndCapture(S.cap_stream, &g);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S.graph, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  int snap = 0;
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    e = use_graph ? cudaGraphLaunch(S.graph, st) : generic_step_any(c, st);
    if (e == cudaSuccess && traj && save_every > 0 && (k + 1) % save_every == 0) {
      e = cudaMemcpyAsync(static_cast<char*>(traj) + (size_t)snap * bytes, S.un, bytes, cudaMemcpyDeviceToDevice, st);
      ++snap;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, S.un, bytes, cudaMemcpyDeviceToDevice, st);
  c->launches = 4 * n_steps;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout (generic grid): %s", cudaGetErrorString(e));
  return FD_OK;
}
