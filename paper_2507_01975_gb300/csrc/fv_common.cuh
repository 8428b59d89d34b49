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

// Programmatic dependent launch. pdl_trigger lets the next kernel of the
// stream (launched with programmatic stream serialisation) start launching:
// its CTAs take the SMs this kernel's last wave frees and run their prologue.
// pdl_wait blocks until the previous kernel has completed and its writes are
// visible. Both are no-ops for kernels launched without that attribute.
// A kernel whose prologue reads data written two or more launches back calls
// pdl_wait before pdl_trigger, so that its successor's prologue runs only
// after every earlier kernel has completed.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

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


// Tendency H(w) of the flux block (App. B.2: advection, dissipation, forcing,
// and the Burgers correction) for a strip of 4 consecutive cells of one row,
// from the 5 x 8 window u[r][c] = w_u(row - 2 + r, col - 2 + c) (same for v)
// around the strip's first cell (row, col); the strip's cells are c = 2 .. 5.
// Every face value of the strip is formed once: linear interpolation
// [0, 1/2, 1/2, 0] and the derivative [1, -27, 27, -1] / 24h (DORD = 4) or
// [0, -1, 1, 0] / h (DORD = 2).
template <typename T, int DORD>
__device__ __forceinline__ void strip_tendency(const T (&u)[5][8], const T (&v)[5][8], T idx, T idy, T nu,
                                               bool burgers, bool forced, T fx, T drag, T (&tu)[4], T (&tv)[4]) {
  constexpr T d0 = DORD == 4 ? (T)(1.0 / 24.0) : (T)0;
  constexpr T d1 = DORD == 4 ? (T)(-27.0 / 24.0) : (T)-1;
  constexpr T d2 = DORD == 4 ? (T)(27.0 / 24.0) : (T)1;
  constexpr T d3 = DORD == 4 ? (T)(-1.0 / 24.0) : (T)0;
  auto der = [&](T f0, T f1, T f2, T f3, T ih) { return (d0 * f0 + d1 * f1 + d2 * f2 + d3 * f3) * ih; };
  const T h = (T)0.5;
  // cell centres (row, c) carry u along x and v along y; corners (row, c) sit
  // between rows row - 1 and row at u-face column c
  T Uc2[6], Gxc[6], Vc0[6], Vc1[6], Gyc0[6], Gyc1[6];  // centres c = 1 .. 5 (rows j, j - 1 for v)
  T UV0[7], Gxv[7];                                    // corners of row j, c = 2 .. 6
  T UV1[6], Gyu0[6], Gyu1[6], Gxcs[4];                 // corners of rows j + 1, j; centres of row j - 1
#pragma unroll
  for (int c = 1; c <= 5; ++c) {
    const T uc = h * (u[2][c] + u[2][c + 1]);
    Uc2[c] = uc * uc;
    Gxc[c] = der(u[2][c - 1], u[2][c], u[2][c + 1], u[2][c + 2], idx);
    const T vc0 = h * (v[2][c] + v[3][c]), vc1 = h * (v[1][c] + v[2][c]);
    Vc0[c] = vc0 * vc0;
    Vc1[c] = vc1 * vc1;
    Gyc0[c] = der(v[1][c], v[2][c], v[3][c], v[4][c], idy);
    Gyc1[c] = der(v[0][c], v[1][c], v[2][c], v[3][c], idy);
  }
#pragma unroll
  for (int c = 2; c <= 6; ++c) {
    UV0[c] = h * (u[1][c] + u[2][c]) * (h * (v[2][c - 1] + v[2][c]));
    Gxv[c] = der(v[2][c - 2], v[2][c - 1], v[2][c], v[2][c + 1], idx);
  }
#pragma unroll
  for (int c = 2; c <= 5; ++c) {
    UV1[c] = h * (u[2][c] + u[3][c]) * (h * (v[3][c - 1] + v[3][c]));
    Gyu0[c] = der(u[0][c], u[1][c], u[2][c], u[3][c], idy);
    Gyu1[c] = der(u[1][c], u[2][c], u[3][c], u[4][c], idy);
    Gxcs[c - 2] = der(u[1][c - 1], u[1][c], u[1][c + 1], u[1][c + 2], idx);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = q + 2;
    T du = -(Uc2[c] - Uc2[c - 1]) * idx - (UV1[c] - UV0[c]) * idy +
           nu * ((Gxc[c] - Gxc[c - 1]) * idx + (Gyu1[c] - Gyu0[c]) * idy);
    T dv = -(UV0[c + 1] - UV0[c]) * idx - (Vc0[c] - Vc1[c]) * idy +
           nu * ((Gxv[c + 1] - Gxv[c]) * idx + (Gyc0[c] - Gyc1[c]) * idy);
    const T uc = u[2][c], vc = v[2][c];
    if (burgers) {
      const T dc = Gxc[c] + Gyc0[c];
      du += uc * h * ((Gxc[c - 1] + Gyc0[c - 1]) + dc);
      dv += vc * h * ((Gxcs[q] + Gyc1[c]) + dc);
    }
    if (forced) {
      du += fx - drag * uc;
      dv -= drag * vc;
    }
    tu[q] = du;
    tv[q] = dv;
  }
}

// 256-point transforms, one per warp, 8 points per lane: Stockham autosort
// with radices 8, 8, 4. On entry lane t holds the points t + 32 m (m < 8); on
// return register i holds X[t + 32 (i & 1) + 64 (i >> 1)] (natural order).
// The two exchanges between passes go through the warp's buffer xb (288
// entries: one pad entry per 8 keeps the strided writes conflict-free); tw
// holds exp(-2 pi i m / 256) for m < 128. Compared with WarpFFT<T, 8> (three
// register stages, five shuffle stages) it issues about half the instructions.
template <typename T>
struct WarpFFT256 {
  using CT = typename Cplx<T>::t;
  static constexpr int XB = 288;
  static __device__ __forceinline__ int pad(int p) { return p + (p >> 3); }
  static __device__ __forceinline__ int out_index(int t, int i) { return t + 32 * (i & 1) + 64 * (i >> 1); }
  static __device__ __forceinline__ CT twid(const CT* tw, int m) {
    return m < 128 ? tw[m] : CT{-tw[m - 128].x, -tw[m - 128].y};
  }
  static __device__ __forceinline__ CT negi(CT a) { return CT{a.y, -a.x}; }  // -i a
  static __device__ __forceinline__ void dft4(CT* v) {
    const CT t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const CT t2 = cadd(v[1], v[3]), t3 = negi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
  // radix 2 x 4: X_k = E_k + W8^k O_k, X_{k+4} = E_k - W8^k O_k
  static __device__ __forceinline__ void dft8(CT* v) {
    CT e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e);
    dft4(o);
    const T h = (T)0.70710678118654752440;  // cos(pi / 4)
    o[1] = CT{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};   // (1 - i) h
    o[2] = negi(o[2]);                                         // -i
    o[3] = CT{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};  // -(1 + i) h
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
  static __device__ __forceinline__ void forward(CT (&v)[8], CT* xb, const CT* tw, int t) {
    dft8(v);  // pass 0: butterfly t, no twiddles
#pragma unroll
    for (int r = 0; r < 8; ++r) xb[pad(8 * t + r)] = v[r];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = xb[pad(t + 32 * m)];
    __syncwarp();
    const int j = t & 7;  // pass 1: stride 8, twiddles exp(-2 pi i j r / 64)
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], twid(tw, 4 * j * r));
    dft8(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) xb[pad((t >> 3) * 64 + j + 8 * r)] = v[r];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = xb[pad(t + 32 * m)];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2; ++s) {  // pass 2: butterflies t and t + 32, stride 64
      const int q = t + 32 * s;
      CT w[4] = {v[s], v[s + 2], v[s + 4], v[s + 6]};
#pragma unroll
      for (int r = 1; r < 4; ++r) w[r] = cmul(w[r], twid(tw, q * r));
      dft4(w);
      v[s] = w[0];
      v[s + 2] = w[1];
      v[s + 4] = w[2];
      v[s + 6] = w[3];
    }
  }
  // unnormalised inverse: conj(forward(conj(x)))
  static __device__ __forceinline__ void inverse(CT (&v)[8], CT* xb, const CT* tw, int t) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m].y = -v[m].y;
    forward(v, xb, tw, t);
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m].y = -v[m].y;
  }
};

}  // namespace ldfv

namespace ldfv {

// ---------------------------------------------------------------------------
// Tensor memory (TMEM) as per-thread on-chip storage.
//
// Each SM has 128 lanes x 512 columns of 32-bit tensor memory. A warp may only
// touch the 32 lanes of its quarter (warp % 4); with the 32x32b shape every
// thread of the warp reads or writes its own lane. The rollout kernel keeps
// u_n and the RK4 accumulator of the cells a thread owns in its lane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// whole warp; writes the allocated base address to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// four consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3])
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// The four per-cell values (u_n.u, u_n.v, acc.u, acc.v) of one row in
// consecutive columns: 4 columns in FP32, 8 in FP64.
template <typename T>
struct CellSlot;
template <>
struct CellSlot<float> {
  static constexpr int COLS = 4;
  static __device__ __forceinline__ void load(uint32_t ta, float& a, float& b, float& c, float& d) {
    uint32_t r[4];
    tmem_ld4(ta, r);
    tmem_wait_ld();
    a = __uint_as_float(r[0]);
    b = __uint_as_float(r[1]);
    c = __uint_as_float(r[2]);
    d = __uint_as_float(r[3]);
  }
  static __device__ __forceinline__ void store(uint32_t ta, float a, float b, float c, float d) {
    const uint32_t r[4] = {__float_as_uint(a), __float_as_uint(b), __float_as_uint(c), __float_as_uint(d)};
    tmem_st4(ta, r);
  }
};
template <>
struct CellSlot<double> {
  static constexpr int COLS = 8;
  static __device__ __forceinline__ double join(uint32_t lo, uint32_t hi) {
    return __hiloint2double((int)hi, (int)lo);
  }
  static __device__ __forceinline__ void load(uint32_t ta, double& a, double& b, double& c, double& d) {
    uint32_t r[8];
    tmem_ld8(ta, r);
    tmem_wait_ld();
    a = join(r[0], r[1]);
    b = join(r[2], r[3]);
    c = join(r[4], r[5]);
    d = join(r[6], r[7]);
  }
  static __device__ __forceinline__ void store(uint32_t ta, double a, double b, double c, double d) {
    const uint32_t r[8] = {(uint32_t)__double2loint(a), (uint32_t)__double2hiint(a),
                           (uint32_t)__double2loint(b), (uint32_t)__double2hiint(b),
                           (uint32_t)__double2loint(c), (uint32_t)__double2hiint(c),
                           (uint32_t)__double2loint(d), (uint32_t)__double2hiint(d)};
    tmem_st8(ta, r);
  }
};

}  // namespace ldfv
