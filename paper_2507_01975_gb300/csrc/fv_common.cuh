// fv_common.cuh -- complex helpers and in-shared-memory radix-2^K FFT passes.
//
// The spectral Poisson solve of the pressure projection (App. B.4 of the
// paper: p_hat = psi_hat / -(eta_x^2 + eta_y^2)) is done with a forward
// decimation-in-frequency FFT, which leaves the spectrum in bit-reversed
// order, a pointwise multiply that indexes the symbol through the bit
// reversal, and an inverse decimation-in-time FFT that consumes bit-reversed
// input and returns natural order. No reordering pass is ever needed.
//
// A "pass" fuses K consecutive radix-2 stages: each thread loads 2^K
// elements into registers, applies the K butterfly stages, and stores them
// back, so a length-2^L transform costs ceil(L / K) shared-memory round trips
// and block barriers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ldfv {

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
  using t = float2;
};
template <>
struct Cplx<double> {
  using t = double2;
};

template <typename CT>
__device__ __forceinline__ CT cadd(CT a, CT b) {
  return CT{a.x + b.x, a.y + b.y};
}
template <typename CT>
__device__ __forceinline__ CT csub(CT a, CT b) {
  return CT{a.x - b.x, a.y - b.y};
}
template <typename CT>
__device__ __forceinline__ CT cmul(CT a, CT b) {
  return CT{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename CT>
__device__ __forceinline__ CT cmulc(CT a, CT b) {
  return CT{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

template <int LOGN>
__device__ __forceinline__ int brev(int k) {
  return (int)(__brev((unsigned)k) >> (32 - LOGN));
}

// Element (seq, e) of a batch of sequences lives at buf[seq * SS + e * ES].
// SEQ_FAST selects the thread mapping: consecutive threads take consecutive
// sequences (for column transforms with unit sequence stride) or consecutive
// butterfly groups of one sequence (for row transforms).
//
// Forward DIF pass over stages S0 .. S0+K-1 (stage s has half-size N >> (s+1)).
// tw[m] = exp(-2 pi i m / N), m < N/2.
template <typename CT, int LOGN, int K, int S0, bool SEQ_FAST>
__device__ __forceinline__ void dif_pass(CT* buf, int nseq, int SS, int ES, const CT* tw, int tid,
                                         int nthreads) {
  constexpr int N = 1 << LOGN;
  constexpr int M = 1 << K;
  constexpr int HLOW = N >> (S0 + K);
  constexpr int BLK = N >> S0;
  constexpr int GPS = N >> K;
  const int total = nseq * GPS;
  for (int g = tid; g < total; g += nthreads) {
    int seq, gi;
    if (SEQ_FAST) {
      seq = g % nseq;
      gi = g / nseq;
    } else {
      seq = g / GPS;
      gi = g % GPS;
    }
    const int blk = gi / HLOW, t = gi % HLOW;
    const int e0 = blk * BLK + t;
    CT* base = buf + (size_t)seq * SS;
    CT x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = base[(e0 + m * HLOW) * ES];
#pragma unroll
    for (int d = M / 2; d >= 1; d >>= 1) {
      const int hs = HLOW * d;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if (m & d) continue;
        const int pos = e0 + m * HLOW;
        const int tp = pos & (2 * hs - 1);
        const CT w = tw[tp * (N / (2 * hs))];
        const CT a = x[m], b = x[m + d];
        x[m] = cadd(a, b);
        x[m + d] = cmul(csub(a, b), w);
      }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) base[(e0 + m * HLOW) * ES] = x[m];
  }
}

// Inverse DIT pass over half-sizes 2^S0 .. 2^(S0+K-1), conjugate twiddles,
// bit-reversed input, unnormalised (a full transform multiplies by N).
template <typename CT, int LOGN, int K, int S0, bool SEQ_FAST>
__device__ __forceinline__ void dit_pass(CT* buf, int nseq, int SS, int ES, const CT* tw, int tid,
                                         int nthreads) {
  constexpr int N = 1 << LOGN;
  constexpr int M = 1 << K;
  constexpr int HLOW = 1 << S0;
  constexpr int BLK = HLOW << K;
  constexpr int GPS = N >> K;
  const int total = nseq * GPS;
  for (int g = tid; g < total; g += nthreads) {
    int seq, gi;
    if (SEQ_FAST) {
      seq = g % nseq;
      gi = g / nseq;
    } else {
      seq = g / GPS;
      gi = g % GPS;
    }
    const int blk = gi / HLOW, t = gi % HLOW;
    const int e0 = blk * BLK + t;
    CT* base = buf + (size_t)seq * SS;
    CT x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = base[(e0 + m * HLOW) * ES];
#pragma unroll
    for (int d = 1; d < M; d <<= 1) {
      const int hs = HLOW * d;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        if (m & d) continue;
        const int pos = e0 + m * HLOW;
        const int tp = pos & (2 * hs - 1);
        const CT w = tw[tp * (N / (2 * hs))];
        const CT a = x[m];
        const CT b = cmulc(x[m + d], w);
        x[m] = cadd(a, b);
        x[m + d] = csub(a, b);
      }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) base[(e0 + m * HLOW) * ES] = x[m];
  }
}

// Full forward DIF transform of `nseq` sequences: passes of up to KMAX stages,
// each followed by a block barrier.
template <typename CT, int LOGN, int KMAX, int S0, bool SEQ_FAST>
__device__ __forceinline__ void fft_dif(CT* buf, int nseq, int SS, int ES, const CT* tw, int tid,
                                        int nthreads) {
  if constexpr (S0 < LOGN) {
    constexpr int K = (LOGN - S0) < KMAX ? (LOGN - S0) : KMAX;
    dif_pass<CT, LOGN, K, S0, SEQ_FAST>(buf, nseq, SS, ES, tw, tid, nthreads);
    __syncthreads();
    fft_dif<CT, LOGN, KMAX, S0 + K, SEQ_FAST>(buf, nseq, SS, ES, tw, tid, nthreads);
  }
}

template <typename CT, int LOGN, int KMAX, int S0, bool SEQ_FAST>
__device__ __forceinline__ void fft_dit(CT* buf, int nseq, int SS, int ES, const CT* tw, int tid,
                                        int nthreads) {
  if constexpr (S0 < LOGN) {
    constexpr int K = (LOGN - S0) < KMAX ? (LOGN - S0) : KMAX;
    dit_pass<CT, LOGN, K, S0, SEQ_FAST>(buf, nseq, SS, ES, tw, tid, nthreads);
    __syncthreads();
    fft_dit<CT, LOGN, KMAX, S0 + K, SEQ_FAST>(buf, nseq, SS, ES, tw, tid, nthreads);
  }
}

}  // namespace ldfv
