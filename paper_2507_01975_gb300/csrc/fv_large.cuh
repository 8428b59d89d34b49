// fv_large.cuh -- the plain FV step for large grids (N = 512 .. 2048) that do
// not fit on chip: the state streams through HBM once per kernel.
//
// One RK4 stage (App. B.5) is four kernels:
//   stage     tiles of 64 x 16 cells with a 2-cell halo in shared memory:
//             w = x - G2 p (the projection of the previous stage, applied on
//             the fly), the eight physics face operators (Sec. 3.4, App. B.2),
//             the flux assembly and source terms, the RK combination with u_n
//             and the accumulator -> w* and acc;
//   rows_fwd  divergence D2 w* (two-point, Sec. 3.6) of 8 rows, real-to-complex
//             row FFTs (two real rows per complex transform), half spectra
//             written as one contiguous block per group of 8 rows:
//             spec[b][y / 8][kx][y % 8];
//   cols      column FFTs, multiplication by 1 / symbol(D2 G2) (zero mode 0,
//             App. B.3-B.4), inverse column FFTs;
//   rows_inv  complex-to-real inverse row FFTs -> pressure p.
// A final kernel forms u_{n+1} = w*_4 - G2 p_4. The FFTs are register-resident
// Stockham transforms: N/16 threads per transform hold 16 points each, a pass
// is one radix-16 (or the remaining radix-2/4/8) butterfly per thread in
// registers, and the points go through shared memory only between passes
// (two exchanges for N = 2048); input and output are in natural order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fv_common.cuh"

namespace ldfv {

struct LargeArgs {
  const float* x;     // stage: source of w (u_n at stage 0, w* of the previous stage after)
  const float* p;     // stage: pressure of the previous stage's projection, or null (stage 0)
  const float* un;    // state at the start of the step
  float* acc;         // RK accumulator
  float* ws;          // stage: w* output; rows_fwd input; final input
  float2* spec;       // [batch][N/8][N/2 + 1][8] complex half spectra (8-row groups)
  float* pout;        // rows_inv output; final input
  float* uout;        // final output
  int stage, flow, forcing;
  float dt, nu, idx, idy, drag, inv_nn;
  const float2* tw;   // [N/2]: exp(-2 pi i m / N)
  const float* symx;  // [N/2 + 2]
  const float* symy;  // [N]
  const float* frc;   // [N]
};

constexpr int kLTY = 16;             // stage tile rows (cells)
constexpr int kLRB = 8;              // rows per block of the half-spectrum layout
constexpr int kFP = 16;              // FFT points per thread (a power of two, 4 .. 16)
constexpr int kFPL = kFP == 16 ? 4 : kFP == 8 ? 3 : 2;  // log2 kFP
constexpr int kFMB = kFP == 16 ? 2 : 3;                  // CTAs per SM the FFT kernels are built for

__device__ __forceinline__ float2 c2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c2mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c2negi(float2 a) { return make_float2(a.y, -a.x); }  // -i a
__device__ __forceinline__ float2 c2conj(float2 a) { return make_float2(a.x, -a.y); }

// ---- register-resident Stockham FFT -------------------------------------------
// A transform of N = 2^LOGN points is done by T = N / P threads holding P =
// kFP points each. Pass p has radix R_p (P, P, ..., then the remaining power
// of two) and stride NS_p = R_0 ... R_{p-1}. Butterfly q of the pass takes the
// points q + r N / R (r < R), which thread t = q mod T holds in registers
// s + (P/R) r (s = q / T) when every thread holds the points t + m T (m < P); it
// multiplies point r by exp(-2 pi i (q mod NS) r / (NS R)), transforms the R
// points and sends output r to position (q / NS) NS R + (q mod NS) + r NS
// (Stockham autosort: after the last pass the order is natural). Between
// passes the points go through a padded shared-memory buffer and come back
// in the "points t + m T" pattern.
template <int LOGN>
struct SPlan {
  static constexpr int N = 1 << LOGN, T = N / kFP;
  static constexpr int NP = (LOGN + kFPL - 1) / kFPL;  // passes
  static constexpr int radix(int p) { return p < LOGN / kFPL ? kFP : (1 << (LOGN % kFPL)); }
  static constexpr int ns(int p) { return p == 0 ? 1 : ns(p - 1) * radix(p - 1); }
  // per-pass twiddle tables [R][NS] for passes 1 .. NP-1, stored one after another
  static constexpr int tw_off(int p) { return p <= 1 ? 0 : tw_off(p - 1) + ns(p - 1) * radix(p - 1); }
  static constexpr int TW = NP > 1 ? tw_off(NP) : 0;
  // after the last pass register s + SL r of thread t holds X[t + s T + r NSL]
  static constexpr int RL = radix(NP - 1), SL = kFP / RL, NSL = ns(NP - 1);
  static constexpr int BUF = N + N / 16 + 4;  // padded buffer of one transform (float2)
};

__device__ __forceinline__ int fpad(int p) { return p + (p >> 4); }

// twiddles of passes 1 .. NP-1 from the table tw[m] = exp(-2 pi i m / N), m < N/2
template <int LOGN>
__device__ void build_pass_twiddles(float2* tws, const float2* tw) {
  using SP = SPlan<LOGN>;
  constexpr int N = SP::N;
#pragma unroll
  for (int p = 1; p < SP::NP; ++p) {
    const int R = SP::radix(p), NS = SP::ns(p), off = SP::tw_off(p);
    for (int e = threadIdx.x; e < R * NS; e += blockDim.x) {
      const int r = e / NS, j = e % NS;
      const int m = j * r * (N / (NS * R));
      tws[off + e] = m < N / 2 ? tw[m] : make_float2(-tw[m - N / 2].x, -tw[m - N / 2].y);
    }
  }
}

// forward DFT of R points in registers, natural order in and out
template <int R>
__device__ __forceinline__ void dft(float2* v);
template <>
__device__ __forceinline__ void dft<1>(float2*) {}
template <>
__device__ __forceinline__ void dft<2>(float2* v) {
  const float2 a = v[0], b = v[1];
  v[0] = c2add(a, b);
  v[1] = c2sub(a, b);
}
template <>
__device__ __forceinline__ void dft<4>(float2* v) {
  const float2 t0 = c2add(v[0], v[2]), t1 = c2sub(v[0], v[2]);
  const float2 t2 = c2add(v[1], v[3]), t3 = c2negi(c2sub(v[1], v[3]));
  v[0] = c2add(t0, t2);
  v[2] = c2sub(t0, t2);
  v[1] = c2add(t1, t3);
  v[3] = c2sub(t1, t3);
}
// radix 2 x 4: X_k = E_k + W8^k O_k, X_{k+4} = E_k - W8^k O_k
template <>
__device__ __forceinline__ void dft<8>(float2* v) {
  float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
  dft<4>(e);
  dft<4>(o);
  const float h = 0.70710678118654752f;  // cos(pi / 4)
  o[1] = make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));   // (1 - i) h
  o[2] = c2negi(o[2]);                                                 // -i
  o[3] = make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));  // -(1 + i) h
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = c2add(e[k], o[k]);
    v[k + 4] = c2sub(e[k], o[k]);
  }
}
// radix 2 x 8: X_k = E_k + W16^k O_k, X_{k+8} = E_k - W16^k O_k
template <>
__device__ __forceinline__ void dft<16>(float2* v) {
  float2 e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  dft<8>(e);
  dft<8>(o);
  const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  o[1] = c2mul(o[1], make_float2(c1, -s1));
  o[2] = make_float2(h * (o[2].x + o[2].y), h * (o[2].y - o[2].x));
  o[3] = c2mul(o[3], make_float2(s1, -c1));
  o[4] = c2negi(o[4]);
  o[5] = c2mul(o[5], make_float2(-s1, -c1));
  o[6] = make_float2(h * (o[6].y - o[6].x), -h * (o[6].x + o[6].y));
  o[7] = c2mul(o[7], make_float2(-c1, -s1));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = c2add(e[k], o[k]);
    v[k + 8] = c2sub(e[k], o[k]);
  }
}

template <int LOGN, int P>
__device__ __forceinline__ void fft_pass(float2 (&v)[kFP], const float2* tws, int t) {
  using SP = SPlan<LOGN>;
  constexpr int R = SP::radix(P), NS = SP::ns(P), S = kFP / R, T = SP::T;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    float2 w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = v[s + S * r];
    if constexpr (NS > 1) {
      const int j = (t + s * T) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) w[r] = c2mul(w[r], tws[SP::tw_off(P) + r * NS + j]);
    }
    dft<R>(w);
#pragma unroll
    for (int r = 0; r < R; ++r) v[s + S * r] = w[r];
  }
}

// outputs of pass P to their Stockham positions
template <int LOGN, int P>
__device__ __forceinline__ void fft_store(float2* buf, const float2 (&v)[kFP], int t) {
  using SP = SPlan<LOGN>;
  constexpr int R = SP::radix(P), NS = SP::ns(P), S = kFP / R, T = SP::T;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int q = t + s * T;
    const int base = (q / NS) * NS * R + (q & (NS - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) buf[fpad(base + r * NS)] = v[s + S * r];
  }
}

template <int LOGN>
__device__ __forceinline__ void fft_load(float2 (&v)[kFP], const float2* buf, int t) {
#pragma unroll
  for (int m = 0; m < kFP; ++m) v[m] = buf[fpad(t + m * SPlan<LOGN>::T)];
}

// the final registers (natural order X[t + s T + r NSL]) to the buffer
template <int LOGN>
__device__ __forceinline__ void fft_store_natural(float2* buf, const float2 (&v)[kFP], int t) {
  using SP = SPlan<LOGN>;
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) buf[fpad(t + s * SP::T + r * SP::NSL)] = v[s + SP::SL * r];
}

// synchronisation of the T threads of one transform: a named barrier per
// transform when it spans whole warps of its own (T >= 64), else the warp
struct TransformSync {
  int id, n;
  __device__ __forceinline__ void operator()() const {
    if (n >= 64)
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    else
      __syncwarp();
  }
};

// passes P .. NP-1, each after an exchange of the previous pass's outputs
template <int LOGN, int P>
__device__ __forceinline__ void fft_passes_from(float2 (&v)[kFP], float2* buf, const float2* tws, int t,
                                                TransformSync sync) {
  if constexpr (P < SPlan<LOGN>::NP) {
    fft_store<LOGN, P - 1>(buf, v, t);
    sync();
    fft_load<LOGN>(v, buf, t);
    sync();
    fft_pass<LOGN, P>(v, tws, t);
    fft_passes_from<LOGN, P + 1>(v, buf, tws, t, sync);
  }
}

// forward transform of the points t + m T in v; on return v[s + SL r] = X[t + s T + r NSL].
// buf is the transform's shared buffer (free on entry and on return)
template <int LOGN>
__device__ __forceinline__ void fft_forward(float2 (&v)[kFP], float2* buf, const float2* tws, int t, TransformSync sync) {
  fft_pass<LOGN, 0>(v, tws, t);
  fft_passes_from<LOGN, 1>(v, buf, tws, t, sync);
}

// unnormalised inverse: conj(forward(conj(x)))
template <int LOGN>
__device__ __forceinline__ void fft_inverse(float2 (&v)[kFP], float2* buf, const float2* tws, int t, TransformSync sync) {
#pragma unroll
  for (int m = 0; m < kFP; ++m) v[m] = c2conj(v[m]);
  fft_forward<LOGN>(v, buf, tws, t, sync);
#pragma unroll
  for (int m = 0; m < kFP; ++m) v[m] = c2conj(v[m]);
}

// transforms per CTA of the row and column kernels: four (one row group of the
// spectrum layout; 512 threads at N = 2048), so that small grids still spread
// over many CTAs; at least one whole warp (the transform syncs are warp-wide
// below 64 threads per transform)
template <int LOGN>
struct RowCfg {
  static constexpr int N = 1 << LOGN, T = N / kFP;
  static constexpr int F = T >= 8 ? 4 : 32 / T;  // row transforms (2 real rows each); whole warps
  static constexpr int NT = F * T;
  static constexpr int RG = 2 * F;  // rows per CTA
  static constexpr size_t SMEM = ((size_t)F * SPlan<LOGN>::BUF + SPlan<LOGN>::TW) * sizeof(float2);
  static_assert(RG % kLRB == 0 || kLRB % RG == 0, "row groups split evenly over CTAs");
};
template <int LOGN>
struct ColCfg {
  static constexpr int N = 1 << LOGN, T = N / kFP;
  static constexpr int C = T >= 8 ? 4 : 32 / T;  // spectrum columns per CTA; whole warps
  static constexpr int NT = C * T;
  static constexpr size_t SMEM = ((size_t)C * SPlan<LOGN>::BUF + SPlan<LOGN>::TW) * sizeof(float2);
};

// ---------------------------------------------------------------------------
// stage kernel: tile of TX x kLTY cells, (TX / 4) x kLTY threads; each thread
// owns a strip of 4 consecutive cells of one row and holds the 5 x 8 window
// of u and v around it in registers, so every face value of the strip is
// formed once from registers (16-byte shared loads, float4 global traffic)
// ---------------------------------------------------------------------------
template <int DORD, int TX>
__global__ void __launch_bounds__(TX / 4 * kLTY, 4) large_stage_kernel(const LargeArgs a, int logn) {
  constexpr int NT = TX / 4 * kLTY;
  constexpr int WX = TX + 4, WY = kLTY + 4, PX = TX + 5, PY = kLTY + 5;
  __shared__ __align__(16) float U[WY][WX];
  __shared__ __align__(16) float V[WY][WX];
  __shared__ float P[PY][PX];
  const int N = 1 << logn, MSK = N - 1;
  const size_t NN = (size_t)N * N;
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * kLTY;
  const int tid = threadIdx.x;
  const float* xu = a.x + (size_t)b * 2 * NN;
  const float* xv = xu + NN;
  pdl_trigger();
  pdl_wait();
  // every global load of the tile is issued before the first use (registers),
  // so the DRAM latency is paid once per CTA, not once per loop trip
  constexpr int NW = (WX * WY + NT - 1) / NT, NPW = (PX * PY + NT - 1) / NT;
  float ru[NW], rv[NW], rp[NPW];
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const int k = tid + q * NT;
    if (k < WX * WY) {
      const int wy = k / WX, wx = k - wy * WX;
      const size_t g = (size_t)((y0 - 2 + wy) & MSK) * N + ((x0 - 2 + wx) & MSK);
      ru[q] = xu[g];
      rv[q] = xv[g];
    }
  }
  if (a.p) {
    const float* pp = a.p + (size_t)b * NN;
#pragma unroll
    for (int q = 0; q < NPW; ++q) {
      const int k = tid + q * NT;
      if (k < PX * PY) {
        const int py = k / PX, px = k - py * PX;
        rp[q] = pp[(size_t)((y0 - 3 + py) & MSK) * N + ((x0 - 3 + px) & MSK)];
      }
    }
#pragma unroll
    for (int q = 0; q < NPW; ++q) {
      const int k = tid + q * NT;
      if (k < PX * PY) P[k / PX][k % PX] = rp[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const int k = tid + q * NT;
    if (k < WX * WY) {
      const int wy = k / WX, wx = k - wy * WX;
      float u = ru[q], v = rv[q];
      if (a.p) {
        // w = x - G2 p: u-face gradient p(i) - p(i - 1), v-face p(j) - p(j - 1)
        u -= (P[wy + 1][wx + 1] - P[wy + 1][wx]) * a.idx;
        v -= (P[wy + 1][wx + 1] - P[wy][wx + 1]) * a.idy;
      }
      U[wy][wx] = u;
      V[wy][wx] = v;
    }
  }
  __syncthreads();

  // window: u[r][c] = U[ly - 2 + r][lx - 2 + c] around the strip's first cell
  // (tile coordinates ly = ty + 2, lx = 4 sx + 2); the strip's cells are c = 2 .. 5
  const int sx = tid % (TX / 4), ty = tid / (TX / 4);
  float u[5][8], v[5][8];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const float4 a0 = *reinterpret_cast<const float4*>(&U[ty + r][4 * sx]);
    const float4 a1 = *reinterpret_cast<const float4*>(&U[ty + r][4 * sx + 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&V[ty + r][4 * sx]);
    const float4 b1 = *reinterpret_cast<const float4*>(&V[ty + r][4 * sx + 4]);
    u[r][0] = a0.x; u[r][1] = a0.y; u[r][2] = a0.z; u[r][3] = a0.w;
    u[r][4] = a1.x; u[r][5] = a1.y; u[r][6] = a1.z; u[r][7] = a1.w;
    v[r][0] = b0.x; v[r][1] = b0.y; v[r][2] = b0.z; v[r][3] = b0.w;
    v[r][4] = b1.x; v[r][5] = b1.y; v[r][6] = b1.z; v[r][7] = b1.w;
  }

  const int j = y0 + ty, i0 = x0 + 4 * sx;
  const size_t g = (size_t)b * 2 * NN + (size_t)j * N + i0;
  const float fx = a.forcing == 1 ? a.frc[j] : 0.0f;
  float tu[4], tv[4];
  strip_tendency<float, DORD>(u, v, a.idx, a.idy, a.nu, a.flow == 0, a.forcing == 1, fx, a.drag, tu, tv);
  const float ca = a.stage == 2 ? a.dt : 0.5f * a.dt;
  const float c6 = a.dt / 6.0f;
  const float4 unu = *reinterpret_cast<const float4*>(a.un + g);
  const float4 unv = *reinterpret_cast<const float4*>(a.un + g + NN);
  float4* wsu = reinterpret_cast<float4*>(a.ws + g);
  float4* wsv = reinterpret_cast<float4*>(a.ws + g + NN);
  float4* acu = reinterpret_cast<float4*>(a.acc + g);
  float4* acv = reinterpret_cast<float4*>(a.acc + g + NN);
  if (a.stage < 3) {
    float4 au = make_float4(tu[0], tu[1], tu[2], tu[3]), av = make_float4(tv[0], tv[1], tv[2], tv[3]);
    if (a.stage > 0) {
      const float4 pu = *acu, pv = *acv;
      au = make_float4(pu.x + 2.0f * tu[0], pu.y + 2.0f * tu[1], pu.z + 2.0f * tu[2], pu.w + 2.0f * tu[3]);
      av = make_float4(pv.x + 2.0f * tv[0], pv.y + 2.0f * tv[1], pv.z + 2.0f * tv[2], pv.w + 2.0f * tv[3]);
    }
    *acu = au;
    *acv = av;
    *wsu = make_float4(unu.x + ca * tu[0], unu.y + ca * tu[1], unu.z + ca * tu[2], unu.w + ca * tu[3]);
    *wsv = make_float4(unv.x + ca * tv[0], unv.y + ca * tv[1], unv.z + ca * tv[2], unv.w + ca * tv[3]);
  } else {
    const float4 pu = *acu, pv = *acv;
    *wsu = make_float4(unu.x + c6 * (pu.x + tu[0]), unu.y + c6 * (pu.y + tu[1]), unu.z + c6 * (pu.z + tu[2]),
                       unu.w + c6 * (pu.w + tu[3]));
    *wsv = make_float4(unv.x + c6 * (pv.x + tv[0]), unv.y + c6 * (pv.y + tv[1]), unv.z + c6 * (pv.z + tv[2]),
                       unv.w + c6 * (pv.w + tv[3]));
  }
}

// ---------------------------------------------------------------------------
// rows_fwd: RG rows per CTA -> RG / 2 complex row transforms
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::NT, kFMB) large_rows_fwd_kernel(const LargeArgs a) {
  using Cfg = RowCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = Cfg::N, T = Cfg::T, H = N / 2, MSK = N - 1;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + Cfg::F * SP::BUF;
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = sm + f * SP::BUF;
  const int b = blockIdx.y, y0 = blockIdx.x * Cfg::RG;
  const size_t NN = (size_t)N * N;
  const float* u = a.ws + (size_t)b * 2 * NN;
  const float* v = u + NN;
  pdl_trigger();
  build_pass_twiddles<LOGN>(tws, a.tw);
  pdl_wait();
  // divergence D2 w* of rows ra and rb as the real and imaginary parts
  const int ra = y0 + 2 * f, rb = ra + 1, rc = (rb + 1) & MSK;
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const int x = t + m * T, xe = (x + 1) & MSK;
    const float da = (u[(size_t)ra * N + xe] - u[(size_t)ra * N + x]) * a.idx +
                     (v[(size_t)rb * N + x] - v[(size_t)ra * N + x]) * a.idy;
    const float db = (u[(size_t)rb * N + xe] - u[(size_t)rb * N + x]) * a.idx +
                     (v[(size_t)rc * N + x] - v[(size_t)rb * N + x]) * a.idy;
    z[m] = make_float2(da, db);
  }
  __syncthreads();  // twiddles
  fft_forward<LOGN>(z, buf, tws, t, TransformSync{1 + f, T});
  fft_store_natural<LOGN>(buf, z, t);
  __syncthreads();
  // unpack the two real rows of each transform: A_k = (Z_k + conj Z_{N-k}) / 2,
  // B_k = (Z_k - conj Z_{N-k}) / (2i); one float4 (A_k, B_k) per (k, transform)
  // at float4 index 4 k + (row % 8) / 2 of the row group's block
  for (int e = threadIdx.x; e < (H + 1) * Cfg::F; e += Cfg::NT) {
    const int k = e / Cfg::F, ff = e - k * Cfg::F;
    const int row = y0 + 2 * ff;
    const float2* bf = sm + ff * SP::BUF;
    const float2 zk = bf[fpad(k & MSK)], zm = bf[fpad((N - k) & MSK)];
    float4* blk = reinterpret_cast<float4*>(a.spec + ((size_t)b * (N / kLRB) + row / kLRB) * (H + 1) * kLRB);
    blk[4 * k + ((row % kLRB) >> 1)] =
        make_float4(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y), 0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
}

// ---------------------------------------------------------------------------
// cols: C spectrum columns per CTA: forward FFT along y, 1 / symbol, inverse
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(ColCfg<LOGN>::NT, kFMB) large_cols_kernel(const LargeArgs a) {
  using Cfg = ColCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = Cfg::N, T = Cfg::T, H = N / 2, G = N / kLRB;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + Cfg::C * SP::BUF;
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = sm + f * SP::BUF;
  const int b = blockIdx.y, kx = blockIdx.x * Cfg::C + f;
  const bool valid = kx <= H;  // idle transforms still take part in the warp-level syncs
  float2* spec = a.spec + (size_t)b * G * (H + 1) * kLRB;
  pdl_trigger();
  build_pass_twiddles<LOGN>(tws, a.tw);
  pdl_wait();
  // column kx, row y = 8 g + yy sits at spec[(g (H + 1) + kx) 8 + yy]
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const int y = t + m * T;
    z[m] = valid ? spec[((size_t)(y >> 3) * (H + 1) + kx) * kLRB + (y & 7)] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();  // twiddles
  const TransformSync sync{1 + f, T};
  fft_forward<LOGN>(z, buf, tws, t, sync);
  // multiply by 1 / (N^2 symbol(kx, ky)); the zero mode is removed
  const float sx = valid ? a.symx[kx] : 1.0f;
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) {
      const int ky = t + s * T + r * SP::NSL;
      const float mlt = (kx == 0 && ky == 0) ? 0.0f : __fdividef(a.inv_nn, sx + __ldg(a.symy + ky));
      float2& zz = z[s + SP::SL * r];
      zz = make_float2(zz.x * mlt, zz.y * mlt);
    }
  fft_store_natural<LOGN>(buf, z, t);
  sync();
  fft_load<LOGN>(z, buf, t);
  sync();
  fft_inverse<LOGN>(z, buf, tws, t, sync);
  if (valid) {
#pragma unroll
    for (int s = 0; s < SP::SL; ++s)
#pragma unroll
      for (int r = 0; r < SP::RL; ++r) {
        const int y = t + s * T + r * SP::NSL;
        spec[((size_t)(y >> 3) * (H + 1) + kx) * kLRB + (y & 7)] = z[s + SP::SL * r];
      }
  }
}

// ---------------------------------------------------------------------------
// rows_inv: RG rows per CTA from the half spectra -> pressure rows
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::NT, kFMB) large_rows_inv_kernel(const LargeArgs a) {
  using Cfg = RowCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = Cfg::N, T = Cfg::T, H = N / 2;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + Cfg::F * SP::BUF;
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  float2* buf = sm + f * SP::BUF;
  const int b = blockIdx.y, y0 = blockIdx.x * Cfg::RG;
  const int ra = y0 + 2 * f;
  pdl_trigger();
  build_pass_twiddles<LOGN>(tws, a.tw);
  pdl_wait();
  // packed transform Z_k = A_k + i B_k of rows ra, ra + 1; the half spectra
  // hold k <= N/2, and Z_k = conj(A_{N-k}) + i conj(B_{N-k}) above
  const float4* blk = reinterpret_cast<const float4*>(a.spec + ((size_t)b * (N / kLRB) + ra / kLRB) * (H + 1) * kLRB) +
                      ((ra % kLRB) >> 1);
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const int k = t + m * T;
    const bool lo = k <= H;
    const float4 q = blk[(size_t)(lo ? k : N - k) * 4];
    z[m] = lo ? make_float2(q.x - q.w, q.y + q.z) : make_float2(q.x + q.w, q.z - q.y);
  }
  __syncthreads();  // twiddles
  fft_inverse<LOGN>(z, buf, tws, t, TransformSync{1 + f, T});
  float* p = a.pout + (size_t)b * N * N;
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) {
      const int x = t + s * T + r * SP::NSL;
      const float2 zz = z[s + SP::SL * r];
      p[(size_t)ra * N + x] = zz.x;
      p[(size_t)(ra + 1) * N + x] = zz.y;
    }
}

// u_{n+1} = w* - G2 p (or w* itself without a projection); four consecutive
// cells of a row per thread (float4 traffic)
__global__ void __launch_bounds__(256) large_final_kernel(const LargeArgs a, int logn, int batch) {
  const int N = 1 << logn, MSK = N - 1;
  const size_t NN = (size_t)N * N, Q = NN / 4;
  const size_t total = (size_t)batch * Q;
  pdl_trigger();
  pdl_wait();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / Q, c = (e - b * Q) * 4;
    const size_t g = b * 2 * NN + c;
    const float4 wu = *reinterpret_cast<const float4*>(a.ws + g);
    const float4 wv = *reinterpret_cast<const float4*>(a.ws + g + NN);
    float4* ou = reinterpret_cast<float4*>(a.uout + g);
    float4* ov = reinterpret_cast<float4*>(a.uout + g + NN);
    if (!a.pout) {  // no projection (Burgers)
      *ou = wu;
      *ov = wv;
      continue;
    }
    const int j = (int)(c >> logn), i = (int)(c & MSK);
    const float* p = a.pout + b * NN;
    const float4 pc = *reinterpret_cast<const float4*>(p + c);
    const float pw = p[(size_t)j * N + ((i - 1) & MSK)];
    const float4 ps = *reinterpret_cast<const float4*>(p + (size_t)((j - 1) & MSK) * N + i);
    const float ix = a.idx, iy = a.idy;
    *ou = make_float4(wu.x - (pc.x - pw) * ix, wu.y - (pc.y - pc.x) * ix, wu.z - (pc.z - pc.y) * ix,
                      wu.w - (pc.w - pc.z) * ix);
    *ov = make_float4(wv.x - (pc.x - ps.x) * iy, wv.y - (pc.y - ps.y) * iy, wv.z - (pc.z - ps.z) * iy,
                      wv.w - (pc.w - ps.w) * iy);
  }
}

}  // namespace ldfv
