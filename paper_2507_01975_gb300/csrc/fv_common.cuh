// fv_common.cuh -- complex helpers and warp-level FFTs.
//
// The spectral Poisson solve of the pressure projection (App. B.4 of the
// paper: p_hat = psi_hat / -(eta_x^2 + eta_y^2)) is done with a forward
// decimation-in-frequency FFT, which leaves the spectrum in bit-reversed
// order, a pointwise multiply that indexes the symbol through the bit
// reversal, and an inverse decimation-in-time FFT that consumes bit-reversed
// input and returns natural order: no reordering pass is ever needed.
//
// One transform of length N = 2^L lives in one warp (N >= 32: lane q holds
// the E = N/32 elements at positions q + 32 m) or in an aligned group of N
// lanes (N < 32: one element per lane). Butterfly stages whose partners sit in
// the same lane run in registers; the last log2(min(N, 32)) stages exchange
// values with __shfl_xor_sync. No shared memory and no block barrier is used.
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

template <int L>
__device__ __forceinline__ int brev(int k) {
  if constexpr (L == 0) {
    return 0;
  } else {
    return (int)(__brev((unsigned)k) >> (32 - L));
  }
}

template <int L>
__host__ __device__ constexpr int brev_c(int k) {
  int r = 0;
  for (int b = 0; b < L; ++b) r |= ((k >> b) & 1) << (L - 1 - b);
  return r;
}

template <typename CT>
__device__ __forceinline__ CT shfl_xor(CT v, int m) {
  return CT{__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}
template <typename CT>
__device__ __forceinline__ CT shfl_idx(CT v, int src) {
  return CT{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
template <typename CT>
__device__ __forceinline__ CT shfl_up1(CT v) {
  return CT{__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1)};
}

// Warp FFT of length N = 2^LOGN. tw[m] = exp(-2 pi i m / N), m < N/2, in
// shared memory. q = lane index within the transform's lane group.
template <typename T, int LOGN>
struct WarpFFT {
  using CT = typename Cplx<T>::t;
  static constexpr int N = 1 << LOGN;
  static constexpr int LOGW = LOGN < 5 ? LOGN : 5;  // lanes per transform = 2^LOGW
  static constexpr int W = 1 << LOGW;
  static constexpr int LOGE = LOGN - LOGW;
  static constexpr int E = 1 << LOGE;  // elements per lane

  // position p = q + W m holds element p on input (natural order)
  static __device__ __forceinline__ void dif(CT (&x)[E], int q, const CT* tw) {
#pragma unroll
    for (int dm = E / 2; dm >= 1; dm >>= 1) {
      const int h = W * dm;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & dm) continue;
        const int t = (q + W * m) & (2 * h - 1);
        const CT w = tw[t * (N / (2 * h))];
        const CT a = x[m], b = x[m + dm];
        x[m] = cadd(a, b);
        x[m + dm] = cmul(csub(a, b), w);
      }
    }
#pragma unroll
    for (int h = W / 2; h >= 1; h >>= 1) {
      const bool upper = (q & h) != 0;
      const CT w = tw[(q & (h - 1)) * (N / (2 * h))];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const CT p = shfl_xor(x[m], h);
        x[m] = upper ? cmul(csub(p, x[m]), w) : cadd(x[m], p);
      }
    }
  }

  // bit-reversed input at positions q + W m, natural-order output, x N
  static __device__ __forceinline__ void dit_inv(CT (&x)[E], int q, const CT* tw) {
#pragma unroll
    for (int h = 1; h < W; h <<= 1) {
      const bool upper = (q & h) != 0;
      const CT w = tw[(q & (h - 1)) * (N / (2 * h))];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const CT v = upper ? cmulc(x[m], w) : x[m];
        const CT p = shfl_xor(v, h);
        x[m] = upper ? csub(p, v) : cadd(v, p);
      }
    }
#pragma unroll
    for (int dm = 1; dm < E; dm <<= 1) {
      const int h = W * dm;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if (m & dm) continue;
        const int t = (q + W * m) & (2 * h - 1);
        const CT w = tw[t * (N / (2 * h))];
        const CT a = x[m];
        const CT b = cmulc(x[m + dm], w);
        x[m] = cadd(a, b);
        x[m + dm] = csub(a, b);
      }
    }
  }

  // After dif(), position p holds X[brev(p)]. For the element at register m
  // of lane q (k = brev(q + W m)) the element X[(N - k) mod N] sits at register
  // partner_reg(m) of lane partner_lane(q, m); the register index does not
  // depend on the lane.
  static __host__ __device__ constexpr int partner_reg(int m) {
    // k mod E = brev_{LOGE}(m); (N - k) mod E = (E - k mod E) mod E
    return brev_c<LOGE>((E - brev_c<LOGE>(m)) & (E - 1));
  }
  static __device__ __forceinline__ int partner_lane(int q, int m) {
    const int k = brev<LOGN>(q + W * m);
    const int kp = (N - k) & (N - 1);
    return brev<LOGN>(kp) & (W - 1);
  }
};

}  // namespace ldfv
