// fd_generic.cu -- plain FV on grids the other paths do not take: Burgers on
// any nx x ny (non-power-of-two and rectangular; App. C.1 Burgers on [0, 1]^2
// at 100^2 and 25^2, Table S2), FP32 or FP64, and Navier-Stokes on rectangular
// power-of-two grids (the shear-flow grids of Table 4, 128 x 64 and larger), FP32.
//
// A step is four launches of generic_stage_kernel (App. B.5), each thread
// forming the tendency of a strip of 4 cells of one row with the same
// flux-block arithmetic as the other paths (strip_tendency: face values of the
// eight operator instances, flux assembly and divergence, the Burgers
// correction, forcing) from a 5 x 8 window gathered with periodic wrap, then
// the RK combination; the last strip of a row is ragged when 4 does not divide
// nx. For Navier-Stokes every stage result is projected (Sec. 3.6, App. B.3-B.4):
// the divergence D2 w* and forward complex FFTs along x (one kernel), forward
// FFTs along y, division by the symbol of D2 G2 (or the continuous one),
// inverse FFTs along y (one kernel), inverse FFTs along x giving p, and
// w = w* - G2 p; the FFTs are the register-resident Stockham transforms of
// fv_fft.cuh (complex transforms of the real divergence; the rectangular
// grid rules out the square real-FFT layouts of the streaming path). A step
// is captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fv_common.cuh"
#include "fv_fft.cuh"

using namespace ldfv;

namespace {

template <typename T>
struct GenArgs {
  const T* w;    // stage state [batch][2][ny][nx]
  const T* un;   // state at the start of the step
  T* acc;        // RK4 accumulator
  T* wout;       // next stage state (stage 3: the new state)
  const T* frc;  // [ny] forcing amplitude at the u-face rows
  int nx, ny, stage, forced, burgers;
  T dt, nu, idx, idy, drag;
  // passive scalar (fd_rollout_scalar): stage scalar, scalar at the step start,
  // accumulator, next stage scalar [batch][ny][nx]; sw == null: no scalar
  const T* sw;
  const T* sn;
  T* sacc;
  T* sout;
  T diff;
};

// RK4 combination of one value (App. B.5): stage 0 starts the accumulator,
// stages 1 and 2 add to it, stage 3 finishes the step
template <typename T>
__device__ __forceinline__ void rk_combine(int stage, T r, T dt, const T* un, T* acc, T* out, size_t e) {
  const T h6 = dt / (T)6, h3 = dt / (T)3, h2 = dt * (T)0.5;
  switch (stage) {
    case 0: {
      const T u0 = un[e];
      acc[e] = u0 + h6 * r;
      out[e] = u0 + h2 * r;
      break;
    }
    case 1:
      acc[e] += h3 * r;
      out[e] = un[e] + h2 * r;
      break;
    case 2:
      acc[e] += h3 * r;
      out[e] = un[e] + dt * r;
      break;
    default:
      out[e] = acc[e] + h6 * r;
  }
}

// tendency of the passive scalar (shear flow, App. C.1) for the strip's 4
// cells: -div(u s_f - D grad_f s) with the face value and face derivative of s
// from the physics kernels along x at the u-faces and along y at the v-faces;
// s[r][c] = s(row - 2 + r, col - 2 + c), u / v the velocity windows of the strip
template <typename T, int DORD>
__device__ __forceinline__ void strip_scalar(const T (&s)[5][8], const T (&u)[5][8], const T (&v)[5][8], T idx,
                                             T idy, T D, T (&q)[4]) {
  constexpr T d0 = DORD == 4 ? (T)(1.0 / 24.0) : (T)0;
  constexpr T d1 = DORD == 4 ? (T)(-27.0 / 24.0) : (T)-1;
  constexpr T d2 = DORD == 4 ? (T)(27.0 / 24.0) : (T)1;
  constexpr T d3 = DORD == 4 ? (T)(-1.0 / 24.0) : (T)0;
  auto der = [&](T f0, T f1, T f2, T f3, T ih) { return (d0 * f0 + d1 * f1 + d2 * f2 + d3 * f3) * ih; };
  const T h = (T)0.5;
  T Fx[5];  // x-fluxes through the u-faces c = 2 .. 6 of row 2
#pragma unroll
  for (int c = 2; c <= 6; ++c)
    Fx[c - 2] = u[2][c] * h * (s[2][c - 1] + s[2][c]) - D * der(s[2][c - 2], s[2][c - 1], s[2][c], s[2][c + 1], idx);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = k + 2;
    const T Fs = v[2][c] * h * (s[1][c] + s[2][c]) - D * der(s[0][c], s[1][c], s[2][c], s[3][c], idy);
    const T Fn = v[3][c] * h * (s[2][c] + s[3][c]) - D * der(s[1][c], s[2][c], s[3][c], s[4][c], idy);
    q[k] = -(Fx[k + 1] - Fx[k]) * idx - (Fn - Fs) * idy;
  }
}

template <typename T, int DORD>
__global__ void __launch_bounds__(256) generic_stage_kernel(const GenArgs<T> a) {
  const int strips = (a.nx + 3) >> 2;
  const int sid = blockIdx.x * blockDim.x + threadIdx.x;  // strip index
  if (sid >= strips * a.ny) return;
  const int row = sid / strips, col0 = (sid - row * strips) * 4;
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
  strip_tendency<T, DORD>(u, v, a.idx, a.idy, a.nu, a.burgers != 0, a.forced != 0, a.frc[row], a.drag, tu, tv);
  T sq[4] = {};
  if (a.sw) {
    const T* sb = a.sw + (size_t)blockIdx.y * NN;
    T s[5][8];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int j = (row - 2 + r + a.ny) % a.ny;
#pragma unroll
      for (int c = 0; c < 8; ++c) s[r][c] = sb[(size_t)j * a.nx + (col0 - 2 + c + a.nx) % a.nx];
    }
    strip_scalar<T, DORD>(s, u, v, a.idx, a.idy, a.diff, sq);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = col0 + k;
    if (i >= a.nx) break;
    const size_t e = (size_t)blockIdx.y * 2 * NN + (size_t)row * a.nx + i;
    rk_combine<T>(a.stage, tu[k], a.dt, a.un, a.acc, a.wout, e);
    rk_combine<T>(a.stage, tv[k], a.dt, a.un, a.acc, a.wout, e + NN);
    if (a.sw) rk_combine<T>(a.stage, sq[k], a.dt, a.sn, a.sacc, a.sout, (size_t)blockIdx.y * NN + (size_t)row * a.nx + i);
  }
}

// ---- projection of a rectangular power-of-two grid (FP32) -----------------
// F transforms of L = 2^LOGL points per CTA, L / 16 threads each; every
// exchange is a CTA-wide barrier (all transforms of a CTA move in lockstep)
template <int LOGL>
struct AxCfg {
  static constexpr int L = 1 << LOGL, T = L / kFP;
  static constexpr int F = 4096 / L < 1 ? 1 : (4096 / L > 16 ? 16 : 4096 / L);
  static constexpr int NT = F * T;
  static constexpr size_t SMEM = ((size_t)F * SPlan<LOGL>::BUF + SPlan<LOGL>::TW) * sizeof(float2);
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
};

// rows: z = D2 w (real), forward FFT along x; Z[b][j][kx]
template <int LOGL>
__global__ void __launch_bounds__(AxCfg<LOGL>::NT) gproj_rows_fwd_kernel(const float* w, float2* Z, int ny,
                                                                        int ntr, const float2* twx, float idx,
                                                                        float idy) {
  using C = AxCfg<LOGL>;
  using SP = SPlan<LOGL>;
  constexpr int L = C::L, T = C::T;
  extern __shared__ __align__(16) float2 gsm[];
  float2* tws = gsm + C::F * SP::BUF;
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int tr = blockIdx.x * C::F + f;
  build_pass_twiddles<LOGL>(tws, twx);
  float2 z[kFP];
  const bool live = tr < ntr;
  const int b = live ? tr / ny : 0, j = live ? tr % ny : 0;
  const size_t NN = (size_t)L * ny;
  const float* u = w + (size_t)b * 2 * NN;
  const float* v = u + NN;
  const int jn = j + 1 == ny ? 0 : j + 1;
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const int i = t + m * T, in = (i + 1) & (L - 1);
    const float d = live ? (u[(size_t)j * L + in] - u[(size_t)j * L + i]) * idx +
                               (v[(size_t)jn * L + i] - v[(size_t)j * L + i]) * idy
                         : 0.0f;
    z[m] = make_float2(d, 0.0f);
  }
  __syncthreads();
  const TransformSync sync{0, C::NT};
  fft_forward<LOGL>(z, gsm + f * SP::BUF, tws, t, sync);
  if (live) {
#pragma unroll
    for (int s = 0; s < SP::SL; ++s)
#pragma unroll
      for (int r = 0; r < SP::RL; ++r) Z[(size_t)tr * L + t + s * T + r * SP::NSL] = z[s + SP::SL * r];
  }
}

// columns: forward FFT along y, divide by the symbol (zero mode dropped),
// inverse FFT along y; consecutive transforms are consecutive columns, so the
// F transforms of a CTA read F adjacent complex values per row
template <int LOGL>
__global__ void __launch_bounds__(AxCfg<LOGL>::NT) gproj_cols_kernel(float2* Z, int nx, int ncols,
                                                                    const float2* twy, const float* symx,
                                                                    const float* symy) {
  using C = AxCfg<LOGL>;
  using SP = SPlan<LOGL>;
  constexpr int L = C::L, T = C::T;
  extern __shared__ __align__(16) float2 gsm[];
  float2* tws = gsm + C::F * SP::BUF;
  const int f = threadIdx.x % C::F, t = threadIdx.x / C::F;
  const int col = blockIdx.x * C::F + f;
  build_pass_twiddles<LOGL>(tws, twy);
  const bool live = col < ncols;
  const int b = live ? col / nx : 0, i = live ? col % nx : 0;
  float2* base = Z + (size_t)b * L * nx + i;
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = live ? base[(size_t)(t + m * T) * nx] : make_float2(0.0f, 0.0f);
  __syncthreads();
  const TransformSync sync{0, C::NT};
  float2* buf = gsm + f * SP::BUF;
  fft_forward<LOGL>(z, buf, tws, t, sync);
  // register m holds point t + m T, the inverse transform's input order
  const float sx = live ? symx[i] : 1.0f;
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const float sy = sx + symy[t + m * T];
    const float inv = sy != 0.0f ? 1.0f / sy : 0.0f;
    z[m] = make_float2(z[m].x * inv, z[m].y * inv);
  }
  fft_inverse<LOGL>(z, buf, tws, t, sync);
  if (live) {
#pragma unroll
    for (int s = 0; s < SP::SL; ++s)
#pragma unroll
      for (int r = 0; r < SP::RL; ++r) base[(size_t)(t + s * T + r * SP::NSL) * nx] = z[s + SP::SL * r];
  }
}

// rows: inverse FFT along x, p = Re / (nx ny)
template <int LOGL>
__global__ void __launch_bounds__(AxCfg<LOGL>::NT) gproj_rows_inv_kernel(const float2* Z, float* p, int ntr,
                                                                        const float2* twx, float scale) {
  using C = AxCfg<LOGL>;
  using SP = SPlan<LOGL>;
  constexpr int L = C::L, T = C::T;
  extern __shared__ __align__(16) float2 gsm[];
  float2* tws = gsm + C::F * SP::BUF;
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int tr = blockIdx.x * C::F + f;
  build_pass_twiddles<LOGL>(tws, twx);
  const bool live = tr < ntr;
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = live ? Z[(size_t)tr * L + t + m * T] : make_float2(0.0f, 0.0f);
  __syncthreads();
  const TransformSync sync{0, C::NT};
  fft_inverse<LOGL>(z, gsm + f * SP::BUF, tws, t, sync);
  if (live) {
#pragma unroll
    for (int s = 0; s < SP::SL; ++s)
#pragma unroll
      for (int r = 0; r < SP::RL; ++r) p[(size_t)tr * L + t + s * T + r * SP::NSL] = z[s + SP::SL * r].x * scale;
  }
}

// w = w* - G2 p (differences of adjacent pressures)
__global__ void __launch_bounds__(256) gproj_grad_kernel(float* w, const float* p, int nx, int ny, int batch,
                                                         float idx, float idy) {
  const size_t NN = (size_t)nx * ny;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)batch * NN) return;
  const size_t b = e / NN, c = e - b * NN;
  const int j = (int)(c / nx), i = (int)(c - (size_t)j * nx);
  const float* pb = p + b * NN;
  const float pc = pb[c];
  w[b * 2 * NN + c] -= (pc - pb[(size_t)j * nx + (i == 0 ? nx - 1 : i - 1)]) * idx;
  w[b * 2 * NN + NN + c] -= (pc - pb[(size_t)(j == 0 ? ny - 1 : j - 1) * nx + i]) * idy;
}

template <int LOGL>
cudaError_t launch_rows_fwd(const float* w, float2* Z, int ny, int ntr, const float2* tw, float idx, float idy,
                            cudaStream_t st) {
  using C = AxCfg<LOGL>;
  gproj_rows_fwd_kernel<LOGL><<<(ntr + C::F - 1) / C::F, C::NT, C::SMEM, st>>>(w, Z, ny, ntr, tw, idx, idy);
  return cudaGetLastError();
}
template <int LOGL>
cudaError_t launch_cols(float2* Z, int nx, int ncols, const float2* tw, const float* sx, const float* sy,
                        cudaStream_t st) {
  using C = AxCfg<LOGL>;
  gproj_cols_kernel<LOGL><<<(ncols + C::F - 1) / C::F, C::NT, C::SMEM, st>>>(Z, nx, ncols, tw, sx, sy);
  return cudaGetLastError();
}
template <int LOGL>
cudaError_t launch_rows_inv(const float2* Z, float* p, int ntr, const float2* tw, float scale, cudaStream_t st) {
  using C = AxCfg<LOGL>;
  gproj_rows_inv_kernel<LOGL><<<(ntr + C::F - 1) / C::F, C::NT, C::SMEM, st>>>(Z, p, ntr, tw, scale);
  return cudaGetLastError();
}

// kernel attributes (outside any stream capture): the 2048-point transforms
// need more than the default 48 KB of dynamic shared memory
template <int LOGL>
cudaError_t prepare_axis() {
  using C = AxCfg<LOGL>;
  cudaError_t e = cudaFuncSetAttribute(gproj_rows_fwd_kernel<LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gproj_cols_kernel<LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gproj_rows_inv_kernel<LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  return e;
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// projection of the FP32 state w [batch][2][ny][nx] in place
cudaError_t generic_project(fd_ctx* c, float* w, cudaStream_t st) {
  GenericState& S = *c->gen;
  const fd_grid& g = c->grid;
  const int ntr = g.batch * g.ny, ncols = g.batch * g.nx;
  const float idx = (float)(g.nx / g.lx), idy = (float)(g.ny / g.ly);
  float2* Z = static_cast<float2*>(S.z);
  float* p = static_cast<float*>(S.p);
  const float2* twx = static_cast<const float2*>(S.twx);
  const float2* twy = static_cast<const float2*>(S.twy);
  const float* sx = static_cast<const float*>(S.symx);
  const float* sy = static_cast<const float*>(S.symy);
  cudaError_t e;
  switch (ilog2(g.nx)) {
    case 5: e = launch_rows_fwd<5>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
    case 6: e = launch_rows_fwd<6>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
    case 7: e = launch_rows_fwd<7>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
    case 8: e = launch_rows_fwd<8>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
    case 9: e = launch_rows_fwd<9>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
    case 10: e = launch_rows_fwd<10>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
    default: e = launch_rows_fwd<11>(w, Z, g.ny, ntr, twx, idx, idy, st); break;
  }
  if (e != cudaSuccess) return e;
  switch (ilog2(g.ny)) {
    case 5: e = launch_cols<5>(Z, g.nx, ncols, twy, sx, sy, st); break;
    case 6: e = launch_cols<6>(Z, g.nx, ncols, twy, sx, sy, st); break;
    case 7: e = launch_cols<7>(Z, g.nx, ncols, twy, sx, sy, st); break;
    case 8: e = launch_cols<8>(Z, g.nx, ncols, twy, sx, sy, st); break;
    case 9: e = launch_cols<9>(Z, g.nx, ncols, twy, sx, sy, st); break;
    case 10: e = launch_cols<10>(Z, g.nx, ncols, twy, sx, sy, st); break;
    default: e = launch_cols<11>(Z, g.nx, ncols, twy, sx, sy, st); break;
  }
  if (e != cudaSuccess) return e;
  const float scale = 1.0f / ((float)g.nx * (float)g.ny);
  switch (ilog2(g.nx)) {
    case 5: e = launch_rows_inv<5>(Z, p, ntr, twx, scale, st); break;
    case 6: e = launch_rows_inv<6>(Z, p, ntr, twx, scale, st); break;
    case 7: e = launch_rows_inv<7>(Z, p, ntr, twx, scale, st); break;
    case 8: e = launch_rows_inv<8>(Z, p, ntr, twx, scale, st); break;
    case 9: e = launch_rows_inv<9>(Z, p, ntr, twx, scale, st); break;
    case 10: e = launch_rows_inv<10>(Z, p, ntr, twx, scale, st); break;
    default: e = launch_rows_inv<11>(Z, p, ntr, twx, scale, st); break;
  }
  if (e != cudaSuccess) return e;
  const size_t cells = (size_t)g.batch * g.nx * g.ny;
  gproj_grad_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(w, p, g.nx, g.ny, g.batch, idx, idy);
  return cudaGetLastError();
}

// one step; with_scalar: the passive scalar with diffusivity diff advances
// alongside (buffers S.sn, S.sa, S.sb, S.sacc)
template <typename T>
cudaError_t generic_step(fd_ctx* c, cudaStream_t st, bool with_scalar = false, double diff = 0.0) {
  GenericState& S = *c->gen;
  const fd_grid& g = c->grid;
  GenArgs<T> a;
  a.sw = nullptr;
  a.sn = static_cast<const T*>(S.sn);
  a.sacc = static_cast<T*>(S.sacc);
  a.diff = (T)diff;
  T* const s_out[4] = {static_cast<T*>(S.sa), static_cast<T*>(S.sb), static_cast<T*>(S.sa), static_cast<T*>(S.sn)};
  const T* const s_in[4] = {static_cast<const T*>(S.sn), static_cast<const T*>(S.sa), static_cast<const T*>(S.sb),
                            static_cast<const T*>(S.sa)};
  a.un = static_cast<const T*>(S.un);
  a.acc = static_cast<T*>(S.acc);
  a.frc = static_cast<const T*>(S.frc);
  a.nx = g.nx;
  a.ny = g.ny;
  a.forced = c->forcing.kind;
  a.burgers = g.flow == FD_BURGERS;
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
    if (with_scalar) {
      a.sw = s_in[s];
      a.sout = s_out[s];
    }
    if (c->opts.deriv_order == 4)
      generic_stage_kernel<T, 4><<<grid, 256, 0, st>>>(a);
    else
      generic_stage_kernel<T, 2><<<grid, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && g.flow == FD_NAVIER_STOKES) {
      if constexpr (sizeof(T) == 4) e = generic_project(c, reinterpret_cast<float*>(stage_out[s]), st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t generic_step_any(fd_ctx* c, cudaStream_t st, bool with_scalar = false, double diff = 0.0) {
  return c->grid.dtype == FD_F64 ? generic_step<double>(c, st, with_scalar, diff)
                                 : generic_step<float>(c, st, with_scalar, diff);
}

}  // namespace

// Burgers on a non-power-of-two or rectangular grid, Navier-Stokes on a
// rectangular power-of-two grid, or either flow with path 3
bool fd_generic_wanted(const fd_grid& g, int path) {
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (g.flow == FD_BURGERS) return path == 3 || !pow2(g.nx) || !pow2(g.ny) || g.nx != g.ny;
  return pow2(g.nx) && pow2(g.ny) && (path == 3 || g.nx != g.ny);
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
  if (e == cudaSuccess && g.flow == FD_NAVIER_STOKES) {
    // projection workspace and tables: complex spectrum, pressure, twiddles
    // exp(-2 pi i m / L) (m < L/2) of both axes, the Poisson symbol per axis
    const size_t cells = (size_t)g.batch * g.nx * g.ny;
    e = cudaMalloc(&S->z, cells * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&S->p, cells * sizeof(float));
    const double pi = 3.14159265358979323846;
    auto twiddles = [&](void** dst, int L) {
      std::vector<float2> tw(L / 2);
      for (int m = 0; m < L / 2; ++m) tw[m] = make_float2((float)std::cos(2 * pi * m / L), (float)-std::sin(2 * pi * m / L));
      if (e == cudaSuccess) e = cudaMalloc(dst, tw.size() * sizeof(float2));
      if (e == cudaSuccess) e = cudaMemcpy(*dst, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    };
    auto symbol = [&](void** dst, int L, double len) {
      const double h = len / L;
      std::vector<float> sy(L);
      for (int k = 0; k < L; ++k) {
        const int ks = k <= L / 2 ? k : k - L;  // signed frequency
        const double sn = std::sin(pi * k / L), eta = 2 * pi * ks / len;
        sy[k] = (float)(c->opts.poisson_symbol == 0 ? -(4.0 / (h * h)) * sn * sn : -eta * eta);
      }
      if (e == cudaSuccess) e = cudaMalloc(dst, L * sizeof(float));
      if (e == cudaSuccess) e = cudaMemcpy(*dst, sy.data(), L * sizeof(float), cudaMemcpyHostToDevice);
    };
    if (e == cudaSuccess && (g.nx == 2048 || g.ny == 2048)) e = prepare_axis<11>();
    twiddles(&S->twx, g.nx);
    twiddles(&S->twy, g.ny);
    symbol(&S->symx, g.nx, g.lx);
    symbol(&S->symy, g.ny, g.ly);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: generic-grid workspace: %s", cudaGetErrorString(e));
  return FD_OK;
}

void fd_generic_free(fd_ctx* c) {
  GenericState* S = c->gen;
  if (!S) return;
  if (S->graph) cudaGraphExecDestroy(S->graph);
  if (S->sgraph) cudaGraphExecDestroy(S->sgraph);
  if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
  void* ps[] = {S->un, S->wa, S->wb, S->acc, S->frc, S->z, S->p, S->twx, S->twy, S->symx, S->symy,
                S->sn, S->sa, S->sb, S->sacc};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete S;
  c->gen = nullptr;
}

cudaError_t fd_generic_project(fd_ctx* c, float* w, cudaStream_t st) { return generic_project(c, w, st); }

fd_status fd_generic_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                             cudaStream_t st, bool allow_graph) {
  if (c->glrn) return fd_glearned_rollout(c, u0, traj, u_final, n_steps, save_every, st, allow_graph);
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
  c->launches = (c->grid.flow == FD_NAVIER_STOKES ? 4 * 5 : 4) * n_steps;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout (generic grid): %s", cudaGetErrorString(e));
  return FD_OK;
}

extern "C" {

fd_status fd_rollout_scalar(fd_ctx* c, double diffusivity, const void* u0, const void* s0, void* u_final,
                            void* s_final, int32_t n_steps, void* stream) {
  return fd_rollout_scalar_impl(c, diffusivity, u0, s0, u_final, s_final, n_steps, static_cast<cudaStream_t>(stream),
                                nullptr, nullptr);
}

}  // extern "C"

fd_status fd_rollout_scalar_impl(fd_ctx* c, double diffusivity, const void* u0, const void* s0, void* u_final,
                                 void* s_final, int n_steps, cudaStream_t st, void* traj_u, void* traj_s) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_rollout_scalar: null context");
  c->launches = 0;
  if (!c->gen)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_rollout_scalar: the passive scalar runs on the generic-grid path (path 3)");
  if (!u0 || !s0 || !u_final || !s_final) return fd_set_error(c, FD_EINVAL, "fd_rollout_scalar: null pointer");
  if (n_steps < 0) return fd_set_error(c, FD_EINVAL, "fd_rollout_scalar: n_steps must be >= 0");
  if (!(diffusivity >= 0) || !std::isfinite(diffusivity))
    return fd_set_error(c, FD_EINVAL, "fd_rollout_scalar: the diffusivity must be >= 0");
  if (c->glrn) return fd_glearned_rollout_scalar(c, diffusivity, u0, s0, u_final, s_final, n_steps, st, traj_u, traj_s);
  GenericState& S = *c->gen;
  const fd_grid& g = c->grid;
  const size_t sbytes = (size_t)g.batch * g.nx * g.ny * (g.dtype == FD_F64 ? sizeof(double) : sizeof(float));
  cudaError_t e = cudaSuccess;
  if (!S.sn) {  // scalar buffers, allocated by the first call (all four or none)
    void** bufs[4] = {&S.sn, &S.sa, &S.sb, &S.sacc};
    for (void** p : bufs)
      if (e == cudaSuccess) e = cudaMalloc(p, sbytes);
    if (e != cudaSuccess) {
      for (void** p : bufs) {
        if (*p) cudaFree(*p);
        *p = nullptr;
      }
      return fd_set_error(c, FD_ENOMEM, "fd_rollout_scalar: cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  const size_t bytes = fd_state_bytes(g);
  e = cudaMemcpyAsync(S.un, u0, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.sn, s0, sbytes, cudaMemcpyDeviceToDevice, st);
  // one step is captured as a graph and replayed; the diffusivity is a kernel
  // argument, so a call with another one recaptures it
  if (e == cudaSuccess && n_steps > 0 && (!S.sgraph || S.sgraph_diff != diffusivity)) {
    if (S.sgraph) {
      // an earlier replay may sit on any stream: wait for the device before the
      // graph is destroyed (a rare event: only a new diffusivity recaptures)
      e = cudaDeviceSynchronize();
      if (e == cudaSuccess) e = cudaGraphExecDestroy(S.sgraph);
      S.sgraph = nullptr;
    }
    cudaGraph_t gr = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = generic_step_any(c, S.cap_stream, true, diffusivity);
      const cudaError_t e2 = cudaStreamEndCapture(S.cap_stream, &gr);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S.sgraph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    S.sgraph_diff = e == cudaSuccess ? diffusivity : -1.0;
  }
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    e = cudaGraphLaunch(S.sgraph, st);
    if (e == cudaSuccess && traj_u) {
      e = cudaMemcpyAsync(static_cast<char*>(traj_u) + (size_t)k * bytes, S.un, bytes, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char*>(traj_s) + (size_t)k * sbytes, S.sn, sbytes, cudaMemcpyDeviceToDevice, st);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, S.un, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s_final, S.sn, sbytes, cudaMemcpyDeviceToDevice, st);
  c->launches = (g.flow == FD_NAVIER_STOKES ? 4 * 5 : 4) * n_steps;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout_scalar: %s", cudaGetErrorString(e));
  return FD_OK;
}
