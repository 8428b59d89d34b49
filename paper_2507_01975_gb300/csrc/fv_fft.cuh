// fv_fft.cuh -- register-resident Stockham FFTs for the kernels that stream
// through HBM (the projection of the streaming path, the energy spectrum):
// transforms of N = 2^LOGN points by N / kFP threads, the row and column
// kernel shapes, complex helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fv_common.cuh"

namespace ldfv {

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
  // NSL = SL T, so register m = s + SL r holds X[t + m T]: a forward transform
  // leaves every point where an inverse transform of the same thread takes it
  static_assert(NSL == SL * T, "natural output order equals the input order");
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

}  // namespace ldfv
