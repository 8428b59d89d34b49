// fd_fno.cu -- the frequency-domain operator O_F of the learnable module
// (Sec. 3.4, "Frequency Domain Operator"; the FNO appendix; Table S3).
//
// O_F(u) = Q(v_L), v_0 = P(u), v_l = sigma(W_l v_{l-1} + b_l + irfft2(R_l .
// rfft2(v_{l-1}))) with sigma = GELU except after the last layer; P, W_l and Q
// are pointwise channel maps, R_l a complex channel matrix per kept Fourier mode
// (kx < M, ky in [0, M) or [N - M, N)). Its eight output channels are added to
// the eight face-operator instances' face values by the learned flux kernel.
// The same operator with the last k_c states as 2 k_c input channels and two
// output channels is the temporal correction (Sec. 3.5; Table S3).
// Per evaluation: lift, per layer {real 2D FFT of every (trajectory, channel)
// field keeping the M-mode blocks, per-mode channel mixing, inverse real 2D
// FFT with numpy's irfft2 semantics, pointwise map + bias + GELU}, projection:
// 2 + 4 L launches, all FP32 on the CUDA cores (the transforms are the
// register-resident Stockham FFTs of fv_fft.cuh, 16 points per thread).
#include <cuda_runtime.h>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fv_fft.cuh"

using namespace ldfv;

namespace {

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// v[b][o][p] = sum_i P_w[o][i] x[b][i][p] + P_b[o], x = the state (single, two
// channels) or the ns states of hist stacked (channel 2 s + c = component c of
// hist[s])
constexpr int kFnoMaxIn = 16;

template <int C>
__global__ void __launch_bounds__(256) fno_lift_kernel(const float* __restrict__ single,
                                                      const float* const* __restrict__ hist, int ns,
                                                      const float* __restrict__ pw, float* __restrict__ v,
                                                      int batch, int nn) {
  __shared__ float sw[C * kFnoMaxIn + C];
  const int cin = 2 * ns;
  for (int k = threadIdx.x; k < C * cin + C; k += blockDim.x) sw[k] = pw[k];  // P_w[C][cin], then P_b[C]
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)batch * nn) return;
  const size_t b = e / nn, p = e - b * nn;
  float acc[C];
#pragma unroll
  for (int o = 0; o < C; ++o) acc[o] = sw[C * cin + o];
  for (int st = 0; st < ns; ++st) {
    const float* src = single ? single : hist[st];
    const float u0 = src[b * 2 * nn + p], u1 = src[b * 2 * nn + nn + p];
#pragma unroll
    for (int o = 0; o < C; ++o) acc[o] += sw[o * cin + 2 * st] * u0 + sw[o * cin + 2 * st + 1] * u1;
  }
#pragma unroll
  for (int o = 0; o < C; ++o) v[(b * C + o) * nn + p] = acc[o];
}

// out[b][o][p] = act(add[b][o][p] + sum_i W[o][i] v[b][i][p] + bias[o]), one pixel
// per thread (add may be null; act = GELU when gelu != 0)
template <int CI, int CO>
__global__ void __launch_bounds__(256) fno_pointwise_kernel(const float* __restrict__ add,
                                                           const float* __restrict__ v,
                                                           const float* __restrict__ W,
                                                           const float* __restrict__ bias,
                                                           float* __restrict__ out, int batch, int nn, int gelu,
                                                           float* __restrict__ pre_out) {
  __shared__ float sw[CO * CI + CO];
  for (int k = threadIdx.x; k < CO * CI; k += blockDim.x) sw[k] = W[k];
  for (int k = threadIdx.x; k < CO; k += blockDim.x) sw[CO * CI + k] = bias[k];
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)batch * nn) return;
  const size_t b = e / nn, p = e - b * nn;
  float vi[CI], ad[CO];
#pragma unroll
  for (int i = 0; i < CI; ++i) vi[i] = v[(b * CI + i) * nn + p];
#pragma unroll
  for (int o = 0; o < CO; ++o) ad[o] = add ? add[(b * CO + o) * nn + p] : 0.0f;
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    float s = sw[CO * CI + o] + ad[o];
#pragma unroll
    for (int i = 0; i < CI; ++i) s += sw[o * CI + i] * vi[i];
    if (pre_out) pre_out[(b * CO + o) * nn + p] = s;
    out[(b * CO + o) * nn + p] = gelu ? gelu_exact(s) : s;
  }
}

// S2[b][o][m] = sum_i R[m][i][o] S[b][i][m] (complex). The channel matrices come
// in the mode-blocked layout Rp[m / 32][i][o][m % 32] (float2, built once per
// parameter upload by fno_pack_r_kernel), so a warp loads a matrix entry of 32
// consecutive modes in one coalesced access straight into registers. A CTA
// takes 32 modes x 16 trajectories; the spectra follow in slices of 4
// trajectories ([b][i][mode]), double-buffered with cp.async so the next slice
// is in flight while the current one is mixed; lane = mode, so loads and stores
// run along the contiguous mode index.
constexpr int kMixModes = 32, kMixBatch = 16, kMixSlice = 4;

template <int C>
struct MixCfg {
  static constexpr int SLICE = kMixSlice * C * kMixModes;  // float2 per slice buffer
  static constexpr size_t SMEM = 2 * (size_t)SLICE * sizeof(float2);
};

// R[m][i][o][re, im] (m < nm) -> Rp[m / 32][i][o][m % 32], zero for the modes past nm
__global__ void fno_pack_r_kernel(const float* __restrict__ R, float2* __restrict__ Rp, int nm, int C) {
  const int nb = (nm + kMixModes - 1) / kMixModes;
  const size_t total = (size_t)nb * C * C * kMixModes;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int mm = (int)(q % kMixModes);
    const size_t r = q / kMixModes;
    const int io = (int)(r % ((size_t)C * C));
    const int m = (int)(r / ((size_t)C * C)) * kMixModes + mm;
    Rp[q] = m < nm ? make_float2(R[((size_t)m * C * C + io) * 2], R[((size_t)m * C * C + io) * 2 + 1])
                   : make_float2(0.0f, 0.0f);
  }
}

// 8-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int C>
__global__ void __launch_bounds__(256) fno_mix_kernel(const float2* __restrict__ S, const float2* __restrict__ Rp,
                                                     float2* __restrict__ S2, int nm, int batch) {
  extern __shared__ __align__(16) float2 smx[];  // two slices [kMixSlice][C][kMixModes]
  const int m0 = blockIdx.x * kMixModes, b0 = blockIdx.y * kMixBatch;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  // this thread's outputs o = grp + 8 j: their matrix columns in registers
  constexpr int NO = C / 8;
  float2 r[NO][C];
  const float2* rb = Rp + (size_t)blockIdx.x * C * C * kMixModes;
#pragma unroll
  for (int j = 0; j < NO; ++j)
#pragma unroll
    for (int i = 0; i < C; ++i) r[j][i] = rb[(i * C + grp + 8 * j) * kMixModes + lane];
  pdl_wait();
  pdl_trigger();
  auto issue = [&](int sl) {
    float2* dst = smx + (sl & 1) * MixCfg<C>::SLICE;
    for (int e = threadIdx.x; e < MixCfg<C>::SLICE; e += blockDim.x) {
      const int mm = e % kMixModes, bi = e / kMixModes, bb = bi / C, i = bi % C;
      const int b = b0 + sl * kMixSlice + bb;
      const bool ok = b < batch && m0 + mm < nm;
      cp_async8(dst + e, ok ? (const void*)(S + ((size_t)b * C + i) * nm + m0 + mm) : (const void*)S, ok ? 8 : 0);
    }
    cp_async_commit();
  };
  constexpr int NSL = kMixBatch / kMixSlice;
  issue(0);
  const int m = m0 + lane;
  for (int sl = 0; sl < NSL; ++sl) {
    if (b0 + sl * kMixSlice >= batch) break;  // uniform over the CTA; nothing left in flight
    if (sl + 1 < NSL && b0 + (sl + 1) * kMixSlice < batch) {
      issue(sl + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // slice sl visible to every thread
    const float2* cur = smx + (sl & 1) * MixCfg<C>::SLICE;
#pragma unroll
    for (int bb = 0; bb < kMixSlice; ++bb) {
      float2 sv[C];
#pragma unroll
      for (int i = 0; i < C; ++i) sv[i] = cur[(bb * C + i) * kMixModes + lane];
      const int b = b0 + sl * kMixSlice + bb;
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int i = 0; i < C; ++i) {
          re = fmaf(sv[i].x, r[j][i].x, re);
          re = fmaf(-sv[i].y, r[j][i].y, re);
          im = fmaf(sv[i].x, r[j][i].y, im);
          im = fmaf(sv[i].y, r[j][i].x, im);
        }
        if (b < batch && m < nm) S2[((size_t)b * C + grp + 8 * j) * nm + m] = make_float2(re, im);
      }
    }
    __syncthreads();  // slice sl consumed before its buffer is refilled
  }
}

template <int LOGN>
struct FnoFftCfg {
  static constexpr int N = 1 << LOGN, T = N / kFP;
  static constexpr int NTR = N / 2;  // row transforms (pairs of real rows); also >= the kept columns
  static constexpr int NT = NTR * T;
  static_assert(T < 64, "transform syncs are warp-level here");
  // per-transform buffer stride (float2): >= fpad(N - 1) + 1 and = T mod 16, so the
  // 16 / T transforms of a half-warp start on different banks
  static constexpr int FBUF = ((N + N / 16 + 15 - T) / 16) * 16 + T;
  static_assert(FBUF >= N + N / 16 && FBUF % 16 == T, "transform buffer stride");
  // row stride of the [N][M] mode staging: >= M and = 2 mod 8 (the rows written
  // by a half-warp's transforms fall on different banks)
  static __host__ __device__ int rs(int M) { return ((M + 5) & ~7) + 2; }
  static size_t smem(int M) { return ((size_t)NTR * FBUF + SPlan<LOGN>::TW + (size_t)N * rs(M)) * sizeof(float2); }
  // the real field passes through the transform buffers as [N][FS] floats: rows
  // 2f, 2f + 1 of the 16 / T transforms of a half-warp fall on different banks
  static constexpr int FS = N + 2;
  static_assert((size_t)N * FS <= (size_t)NTR * FBUF * 2, "field staging fits the transform buffers");
};

// row index of ky among the kept rows (-1 when not kept)
__device__ __forceinline__ int kept_row(int ky, int N, int M) {
  return ky < M ? ky : (ky >= N - M ? ky - (N - 2 * M) : -1);
}

// real 2D DFT of the field (b, c) = (blockIdx.y, blockIdx.x), keeping kx < M and
// the kept rows: S[b][c][2M][M]
template <int LOGN>
__global__ void __launch_bounds__(FnoFftCfg<LOGN>::NT) fno_rfft_kernel(const float* __restrict__ v, float2* __restrict__ S,
                                                                      const float2* __restrict__ tw,
                                                                      int M) {
  using Cfg = FnoFftCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = Cfg::N, T = Cfg::T, MSK = N - 1;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + Cfg::NTR * Cfg::FBUF;
  float2* Rs = tws + SP::TW;  // [N][rs] row spectra
  const int RS = Cfg::rs(M);
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int C = gridDim.x, b = blockIdx.y, c = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const float* field = v + ((size_t)b * C + c) * NN;
  float2* buf = sm + f * Cfg::FBUF;
  const TransformSync sync{1 + f, T};
  build_pass_twiddles<LOGN>(tws, tw);
  pdl_wait();
  pdl_trigger();
  // the field through shared memory ([N][FS] floats over the transform buffers):
  // coalesced 16-byte global loads, then rows 2f and 2f + 1 as one complex transform
  float* fs = reinterpret_cast<float*>(sm);
  constexpr int NQ = N * N / 4 / Cfg::NT;  // 16-byte loads per thread, all in flight before the first store
  static_assert(NQ * Cfg::NT * 4 == N * N, "the field splits evenly over the threads");
  float4 w[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) w[k] = reinterpret_cast<const float4*>(field)[threadIdx.x + k * Cfg::NT];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const int q = threadIdx.x + k * Cfg::NT, row = q / (N / 4), col = 4 * (q % (N / 4));
    *reinterpret_cast<float2*>(fs + row * Cfg::FS + col) = make_float2(w[k].x, w[k].y);
    *reinterpret_cast<float2*>(fs + row * Cfg::FS + col + 2) = make_float2(w[k].z, w[k].w);
  }
  __syncthreads();
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m)
    z[m] = make_float2(fs[(2 * f) * Cfg::FS + t + m * T], fs[(2 * f + 1) * Cfg::FS + t + m * T]);
  __syncthreads();
  fft_forward<LOGN>(z, buf, tws, t, sync);
  fft_store_natural<LOGN>(buf, z, t);
  sync();
  for (int k = t; k < M; k += T) {
    const float2 zk = buf[fpad(k)], zm = buf[fpad((N - k) & MSK)];
    Rs[(2 * f) * RS + k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    Rs[(2 * f + 1) * RS + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
  __syncthreads();
  // column kx = f (kept when f < M; the others run on column 0 and discard)
  const int kx = f < M ? f : 0;
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = Rs[(t + m * T) * RS + kx];
  fft_forward<LOGN>(z, buf, tws, t, sync);
  if (f < M) {
    float2* out = S + ((size_t)b * C + c) * 2 * M * M;
#pragma unroll
    for (int s = 0; s < SP::SL; ++s)
#pragma unroll
      for (int r = 0; r < SP::RL; ++r) {
        const int row = kept_row(t + s * T + r * SP::NSL, N, M);
        if (row >= 0) out[row * M + kx] = z[s + SP::SL * r];
      }
  }
}

// inverse of the above with numpy's irfft2 semantics (an inverse complex DFT along
// y, then a real inverse along x that ignores the imaginary part of the kx = 0
// term), times scale
template <int LOGN>
__global__ void __launch_bounds__(FnoFftCfg<LOGN>::NT) fno_irfft_kernel(const float2* __restrict__ S2, float* __restrict__ y,
                                                                       const float2* __restrict__ tw, int M, float scale) {
  using Cfg = FnoFftCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = Cfg::N, T = Cfg::T, H = N / 2;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + Cfg::NTR * Cfg::FBUF;
  float2* Rs = tws + SP::TW;  // [N][rs] rows after the inverse column transforms
  const int RS = Cfg::rs(M);
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int C = gridDim.x, b = blockIdx.y, c = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const float2* in = S2 + ((size_t)b * C + c) * 2 * M * M;
  float2* buf = sm + f * Cfg::FBUF;
  const TransformSync sync{1 + f, T};
  build_pass_twiddles<LOGN>(tws, tw);
  pdl_wait();
  pdl_trigger();
  const int kx = f < M ? f : 0;
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const int row = kept_row(t + m * T, N, M);
    z[m] = row >= 0 ? in[row * M + kx] : make_float2(0.0f, 0.0f);
  }
  __syncthreads();
  fft_inverse<LOGN>(z, buf, tws, t, sync);
  if (f < M) {
#pragma unroll
    for (int s = 0; s < SP::SL; ++s)
#pragma unroll
      for (int r = 0; r < SP::RL; ++r) Rs[(t + s * T + r * SP::NSL) * RS + kx] = z[s + SP::SL * r];
  }
  __syncthreads();
  // rows 2f, 2f + 1: Z_k = A_k + i B_k on the Hermitian extension of each row
  const float2* A = Rs + (2 * f) * RS;
  const float2* Bv = Rs + (2 * f + 1) * RS;
#pragma unroll
  for (int m = 0; m < kFP; ++m) {
    const int k = t + m * T;
    float2 zz = make_float2(0.0f, 0.0f);
    if (k == 0) {
      zz = make_float2(A[0].x, Bv[0].x);
    } else if (k < H) {
      if (k < M) zz = make_float2(A[k].x - Bv[k].y, A[k].y + Bv[k].x);
    } else if (k > H) {
      const int kp = N - k;
      if (kp < M) zz = make_float2(A[kp].x + Bv[kp].y, Bv[kp].x - A[kp].y);
    }
    z[m] = zz;
  }
  fft_inverse<LOGN>(z, buf, tws, t, sync);
  // rows 2f, 2f + 1 through shared memory ([N][FS] floats over the transform
  // buffers, free once every transform is done), then coalesced 16-byte stores
  float* fs = reinterpret_cast<float*>(sm);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) {
      const int x = t + s * T + r * SP::NSL;
      fs[(2 * f) * Cfg::FS + x] = z[s + SP::SL * r].x * scale;
      fs[(2 * f + 1) * Cfg::FS + x] = z[s + SP::SL * r].y * scale;
    }
  __syncthreads();
  float* out = y + ((size_t)b * C + c) * NN;
  for (int q = threadIdx.x; q < N * N / 4; q += Cfg::NT) {
    const int row = q / (N / 4), col = 4 * (q % (N / 4));
    const float2 lo = *reinterpret_cast<const float2*>(fs + row * Cfg::FS + col);
    const float2 hi = *reinterpret_cast<const float2*>(fs + row * Cfg::FS + col + 2);
    reinterpret_cast<float4*>(out)[q] = make_float4(lo.x, lo.y, hi.x, hi.y);
  }
}

// ---------------------------------------------------------------------------
// reverse mode (the adjoint of every forward line; oracle.fno.fno_vjp)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu_grad_exact(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// out[b][o][p] = add[b][o][p] + sum_i W[i][o] x[b][i][p] (the transposed channel
// map, W stored [CI][CO] as the forward's [out][in]), times GELU'(pre[b][o][p])
// when pre is set. With ost > 0 channel o goes to out + (o / 2) ost + (b * 2 +
// o % 2) nn + p (the cotangents of the k_c stacked history states), otherwise
// out + (b CO + o) nn + p. add may alias out.
template <int CI, int CO>
__global__ void __launch_bounds__(256) fno_pointwise_t_kernel(const float* add, const float* __restrict__ x,
                                                             const float* __restrict__ W,
                                                             const float* __restrict__ pre, float* out, int batch,
                                                             int nn, size_t ost) {
  __shared__ float sw[CI * CO];
  for (int k = threadIdx.x; k < CI * CO; k += blockDim.x) sw[k] = W[k];
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)batch * nn) return;
  const size_t b = e / nn, p = e - b * nn;
  float xi[CI];
#pragma unroll
  for (int i = 0; i < CI; ++i) xi[i] = x[(b * CI + i) * nn + p];
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const size_t oi = ost ? (size_t)(o >> 1) * ost + (b * 2 + (o & 1)) * nn + p : (b * CO + o) * nn + p;
    float s = add ? add[oi] : 0.0f;
#pragma unroll
    for (int i = 0; i < CI; ++i) s += sw[i * CO + o] * xi[i];
    if (pre) s *= gelu_grad_exact(pre[(b * CO + o) * nn + p]);
    out[oi] = s;
  }
}

// Pixel sums of outer products: dW[a][c] += sum_{b,p} X[b][a][p] Y[b][c][p] and
// db[a] += sum X[b][a][p] (the weight and bias gradients of a channel map).
// Y is a plain [batch][BC][nn] array, or the state / k_c history states (BC =
// 2 ns; channel 2 s + c = component c of state s) like the lift's input.
// Per-CTA partials over a fixed pixel split, summed in a fixed order by
// fno_outer_reduce_kernel: deterministic.
constexpr int kOuterTile = 256;
constexpr int kOuterBlocks = 304;

template <int A, int BC>
__global__ void __launch_bounds__(256) fno_outer_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                                       const float* __restrict__ single,
                                                       const float* const* __restrict__ hist, int batch, int nn,
                                                       float* __restrict__ partial) {
  __shared__ float xs[A][kOuterTile + 1];
  __shared__ float ys[BC][kOuterTile + 1];
  const int t = threadIdx.x;
  const int a = t / BC, c = t % BC;
  const bool pair = t < A * BC;
  float acc = 0.0f, accb = 0.0f;
  pdl_wait();
  pdl_trigger();
  const size_t total = (size_t)batch * nn;
  const size_t ntiles = (total + kOuterTile - 1) / kOuterTile;
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t e = tile * kOuterTile + t;
    const bool ok = e < total;
    const size_t b = ok ? e / nn : 0, p = ok ? e - b * nn : 0;
#pragma unroll
    for (int k = 0; k < A; ++k) xs[k][t] = ok ? X[(b * A + k) * nn + p] : 0.0f;
#pragma unroll
    for (int k = 0; k < BC; ++k) {
      float y = 0.0f;
      if (ok) {
        if (Y)
          y = Y[(b * BC + k) * nn + p];
        else
          y = (single ? single : hist[k >> 1])[(b * 2 + (k & 1)) * nn + p];
      }
      ys[k][t] = y;
    }
    __syncthreads();
    if (pair) {
#pragma unroll 8
      for (int q = 0; q < kOuterTile; ++q) acc = fmaf(xs[a][q], ys[c][q], acc);
    }
    if (t < A) {
#pragma unroll 8
      for (int q = 0; q < kOuterTile; ++q) accb += xs[t][q];
    }
    __syncthreads();
  }
  float* pp = partial + (size_t)blockIdx.x * (A * BC + A);
  if (pair) pp[t] = acc;
  if (t < A) pp[A * BC + t] = accb;
}

__global__ void fno_outer_reduce_kernel(const float* __restrict__ partial, int nblk, int nw, int na,
                                        float* __restrict__ dW, float* __restrict__ db) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nw + na) return;
  float s = 0.0f;
  for (int x = 0; x < nblk; ++x) s += partial[(size_t)x * (nw + na) + k];
  if (k < nw)
    dW[k] += s;
  else
    db[k - nw] += s;
}

// Rbar[m][i][o] += (c_kx / N^2) sum_b Abar[b][o][m] conj(S[b][i][m]), c = 1 for
// kx = 0 and 2 otherwise (irfft2 counts a kept mode with its mirror): the
// gradient of the complex weights written d/dRe + i d/dIm, stored [m][i][o][re,
// im] like the parameters. Abar = the kept modes of rfft2 of the layer's output
// cotangent, S = those of its input. lane = mode; warp w owns the outputs
// o = w + 8 j; each (m, i, o) has one writer.
template <int C>
__global__ void __launch_bounds__(256) fno_rgrad_kernel(const float2* __restrict__ Abar, const float2* __restrict__ S,
                                                       float* __restrict__ Rbar, int nm, int M, int batch,
                                                       float inv_nn) {
  constexpr int NO = C / 8;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = blockIdx.x * 32 + lane;
  pdl_wait();
  pdl_trigger();
  if (m >= nm) return;
  float2 acc[NO][C];
#pragma unroll
  for (int j = 0; j < NO; ++j)
#pragma unroll
    for (int i = 0; i < C; ++i) acc[j][i] = make_float2(0.0f, 0.0f);
  for (int b = 0; b < batch; ++b) {
    float2 sv[C];
#pragma unroll
    for (int i = 0; i < C; ++i) sv[i] = S[((size_t)b * C + i) * nm + m];
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const float2 ab = Abar[((size_t)b * C + w + 8 * j) * nm + m];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        // ab * conj(s)
        acc[j][i].x = fmaf(ab.x, sv[i].x, fmaf(ab.y, sv[i].y, acc[j][i].x));
        acc[j][i].y = fmaf(ab.y, sv[i].x, fmaf(-ab.x, sv[i].y, acc[j][i].y));
      }
    }
  }
  const float f = ((m % M) == 0 ? 1.0f : 2.0f) * inv_nn;
#pragma unroll
  for (int j = 0; j < NO; ++j)
#pragma unroll
    for (int i = 0; i < C; ++i) {
      float* r = Rbar + (((size_t)m * C + i) * C + w + 8 * j) * 2;
      r[0] += f * acc[j][i].x;
      r[1] += f * acc[j][i].y;
    }
}

// R[m][i][o][re, im] -> Rh[m / 32][o][i][m % 32] = conj(R[m][i][o]): the channel
// matrices of the spectral convolution's adjoint in v (conjugate transposes), in
// the mixing kernel's layout
__global__ void fno_pack_rh_kernel(const float* __restrict__ R, float2* __restrict__ Rh, int nm, int C) {
  const int nb = (nm + kMixModes - 1) / kMixModes;
  const size_t total = (size_t)nb * C * C * kMixModes;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int mm = (int)(q % kMixModes);
    const size_t r = q / kMixModes;
    const int oi = (int)(r % ((size_t)C * C));
    const int o = oi / C, i = oi % C;
    const int m = (int)(r / ((size_t)C * C)) * kMixModes + mm;
    Rh[q] = m < nm ? make_float2(R[(((size_t)m * C + i) * C + o) * 2], -R[(((size_t)m * C + i) * C + o) * 2 + 1])
                   : make_float2(0.0f, 0.0f);
  }
}

// one Fourier neural operator: width C, `layers` layers of `modes` kept modes,
// parameters at raw_off (P_w[C][cin], P_b[C], layers, Q_w[cout][C], Q_b[cout]),
// output [batch][cout][N][N]
struct FnoNet {
  int layers, modes, cout;
  size_t raw_off;
  float* out;
  const float2* rp;   // mode-blocked channel matrices of every layer
  const float2* rph;  // their conjugate transposes (reverse mode), or null
};

template <int LOGN, int C, int CO>
cudaError_t fno_run(LearnedState& L, const FnoNet& net, const float* single, const float* const* hist, int ns,
                    const float2* tw, int batch, cudaStream_t st) {
  using Cfg = FnoFftCfg<LOGN>;
  constexpr int N = Cfg::N;
  const int M = net.modes, nl = net.layers, cin = 2 * ns;
  const int nn = N * N, nm = 2 * M * M;
  // fsm <= 35 KB (M <= N/2 <= 32): within the default dynamic shared-memory limit
  const size_t fsm = Cfg::smem(M);
  const float* P = L.d_raw + net.raw_off;
  const size_t layer_size = (size_t)nm * C * C * 2 + (size_t)C * C + C;
  const float* R0 = P + (size_t)C * cin + C;
  const float* Q = R0 + (size_t)nl * layer_size;
  const dim3 pix((unsigned)(((size_t)batch * nn + 255) / 256));
  const int nb = (nm + kMixModes - 1) / kMixModes;
  const dim3 mix(nb, (batch + kMixBatch - 1) / kMixBatch);
  cudaError_t e = launch_pdl(fno_lift_kernel<C>, pix, dim3(256), 0, st, single, hist, ns, P, L.fno_v[0], batch, nn);
  int cur = 0;
  for (int l = 0; l < nl && e == cudaSuccess; ++l) {
    const float* R = R0 + (size_t)l * layer_size;
    const float* W = R + (size_t)nm * C * C * 2;
    const float* Wb = W + (size_t)C * C;
    e = launch_pdl(fno_rfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float*)L.fno_v[cur], L.fno_s,
                   tw, M);
    if (e == cudaSuccess)
      e = launch_pdl(fno_mix_kernel<C>, mix, dim3(256), MixCfg<C>::SMEM, st, (const float2*)L.fno_s,
                     (const float2*)(net.rp + (size_t)l * nb * C * C * kMixModes), L.fno_s2, nm, batch);
    if (e == cudaSuccess)
      e = launch_pdl(fno_irfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float2*)L.fno_s2, L.fno_y,
                     tw, M, 1.0f / (float)nn);
    if (e == cudaSuccess)
      e = launch_pdl(fno_pointwise_kernel<C, C>, pix, dim3(256), 0, st, (const float*)L.fno_y,
                     (const float*)L.fno_v[cur], W, Wb, L.fno_v[cur ^ 1], batch, nn, l < nl - 1 ? 1 : 0,
                     (float*)nullptr);
    cur ^= 1;
  }
  if (e == cudaSuccess)
    e = launch_pdl(fno_pointwise_kernel<C, CO>, pix, dim3(256), 0, st, (const float*)nullptr,
                   (const float*)L.fno_v[cur], Q, Q + (size_t)CO * C, net.out, batch, nn, 0, (float*)nullptr);
  return e;
}

template <int CO>
cudaError_t fno_dispatch(fd_ctx* c, const FnoNet& net, int width, const float* single, const float* const* hist,
                         int ns, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const float2* tw = reinterpret_cast<const float2*>(c->base.tw);
  const int B = c->grid.batch;
  if (c->logn == 6)
    return width == 16 ? fno_run<6, 16, CO>(L, net, single, hist, ns, tw, B, st)
                       : fno_run<6, 8, CO>(L, net, single, hist, ns, tw, B, st);
  return width == 16 ? fno_run<5, 16, CO>(L, net, single, hist, ns, tw, B, st)
                     : fno_run<5, 8, CO>(L, net, single, hist, ns, tw, B, st);
}

// forward of one operator keeping what its reverse mode needs: v_0 .. v_L
// (sb.v, L + 1 fields [batch][C][N][N]), the pre-activations of layers 0 ..
// L - 2 (sb.a), the kept input spectra of every layer (sb.S, [batch][C][2M][M]),
// and the output (sb.out)
template <int LOGN, int C, int CO>
cudaError_t fno_run_saved(LearnedState& L, const FnoNet& net, const float* single, const float* const* hist, int ns,
                          const FnoSavedBufs& sb, const float2* tw, int batch, cudaStream_t st) {
  using Cfg = FnoFftCfg<LOGN>;
  constexpr int N = Cfg::N;
  const int M = net.modes, nl = net.layers, cin = 2 * ns;
  const int nn = N * N, nm = 2 * M * M;
  const size_t fsm = Cfg::smem(M);
  const size_t fld = (size_t)batch * C * nn, spec = (size_t)batch * C * nm;
  const float* P = L.d_raw + net.raw_off;
  const size_t layer_size = (size_t)nm * C * C * 2 + (size_t)C * C + C;
  const float* R0 = P + (size_t)C * cin + C;
  const float* Q = R0 + (size_t)nl * layer_size;
  const dim3 pix((unsigned)(((size_t)batch * nn + 255) / 256));
  const int nb = (nm + kMixModes - 1) / kMixModes;
  const dim3 mix(nb, (batch + kMixBatch - 1) / kMixBatch);
  cudaError_t e = launch_pdl(fno_lift_kernel<C>, pix, dim3(256), 0, st, single, hist, ns, P, sb.v, batch, nn);
  for (int l = 0; l < nl && e == cudaSuccess; ++l) {
    const float* R = R0 + (size_t)l * layer_size;
    const float* W = R + (size_t)nm * C * C * 2;
    const float* Wb = W + (size_t)C * C;
    e = launch_pdl(fno_rfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float*)(sb.v + l * fld),
                   sb.S + l * spec, tw, M);
    if (e == cudaSuccess)
      e = launch_pdl(fno_mix_kernel<C>, mix, dim3(256), MixCfg<C>::SMEM, st, (const float2*)(sb.S + l * spec),
                     (const float2*)(net.rp + (size_t)l * nb * C * C * kMixModes), L.fno_s2, nm, batch);
    if (e == cudaSuccess)
      e = launch_pdl(fno_irfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float2*)L.fno_s2, L.fno_y,
                     tw, M, 1.0f / (float)nn);
    if (e == cudaSuccess)
      e = launch_pdl(fno_pointwise_kernel<C, C>, pix, dim3(256), 0, st, (const float*)L.fno_y,
                     (const float*)(sb.v + l * fld), W, Wb, sb.v + (l + 1) * fld, batch, nn, l < nl - 1 ? 1 : 0,
                     l < nl - 1 ? sb.a + l * fld : (float*)nullptr);
  }
  if (e == cudaSuccess)
    e = launch_pdl(fno_pointwise_kernel<C, CO>, pix, dim3(256), 0, st, (const float*)nullptr,
                   (const float*)(sb.v + nl * fld), Q, Q + (size_t)CO * C, sb.out, batch, nn, 0, (float*)nullptr);
  return e;
}

// dW[A][BC] += sum X (x) Y, db[A] += sum X over every pixel of the batch
template <int A, int BC>
cudaError_t outer_grad(const float* X, const float* Y, const float* single, const float* const* hist, int batch,
                       int nn, float* partial, float* dW, float* db, cudaStream_t st) {
  cudaError_t e = launch_pdl(fno_outer_kernel<A, BC>, dim3(kOuterBlocks), dim3(256), 0, st, X, Y, single, hist, batch,
                             nn, partial);
  if (e == cudaSuccess)
    e = launch_pdl(fno_outer_reduce_kernel, dim3((A * BC + A + 255) / 256), dim3(256), 0, st, (const float*)partial,
                   kOuterBlocks, A * BC, A, dW, db);
  return e;
}

// The operator's reverse mode for the output cotangent gbar [batch][CO][N][N]:
// parameter gradients added to dparams (same layout as the parameters), input
// cotangent added to ubar (accumulate) or written (overwrite); ubar in the
// state layout, or the history layout (ost > 0: input channel 2 s + c ->
// ubar + s ost, component c).
template <int LOGN, int C, int CO, int CIN>
cudaError_t fno_back(LearnedState& L, const FnoNet& net, const FnoSavedBufs& sb, const float* single,
                     const float* const* hist, const float* gbar, float* ubar, size_t ost, bool accumulate,
                     float* dparams, float* partial, const float2* tw, int batch, cudaStream_t st) {
  using Cfg = FnoFftCfg<LOGN>;
  constexpr int N = Cfg::N;
  const int M = net.modes, nl = net.layers;
  const int nn = N * N, nm = 2 * M * M;
  const size_t fsm = Cfg::smem(M);
  const size_t fld = (size_t)batch * C * nn, spec = (size_t)batch * C * nm;
  const size_t layer_size = (size_t)nm * C * C * 2 + (size_t)C * C + C;
  const float* P = L.d_raw + net.raw_off;
  const float* R0 = P + (size_t)C * CIN + C;
  const float* Q = R0 + (size_t)nl * layer_size;
  float* dP = dparams + net.raw_off;
  float* dR0 = dP + (size_t)C * CIN + C;
  float* dQ = dR0 + (size_t)nl * layer_size;
  const dim3 pix((unsigned)(((size_t)batch * nn + 255) / 256));
  const int nb = (nm + kMixModes - 1) / kMixModes;
  const dim3 mix(nb, (batch + kMixBatch - 1) / kMixBatch);
  float* abar[2] = {L.fno_v[0], L.fno_v[1]};
  // Q: gradients, then v_bar_L = Q^T gbar (= a_bar of the last layer: no GELU after it)
  cudaError_t e = dparams ? outer_grad<CO, C>(gbar, sb.v + nl * fld, nullptr, nullptr, batch, nn, partial, dQ,
                                              dQ + (size_t)CO * C, st)
                          : cudaSuccess;
  if (e == cudaSuccess)
    e = launch_pdl(fno_pointwise_t_kernel<CO, C>, pix, dim3(256), 0, st, (const float*)nullptr, gbar, Q,
                   (const float*)nullptr, abar[0], batch, nn, (size_t)0);
  int cur = 0;
  for (int l = nl - 1; l >= 0 && e == cudaSuccess; --l) {
    const float* W = R0 + (size_t)l * layer_size + (size_t)nm * C * C * 2;
    float* dR = dR0 + (size_t)l * layer_size;
    float* dW = dR + (size_t)nm * C * C * 2;
    const float* vl = sb.v + l * fld;
    if (dparams) e = outer_grad<C, C>(abar[cur], vl, nullptr, nullptr, batch, nn, partial, dW, dW + (size_t)C * C, st);
    // spectral part: Abar = rfft2(a_bar) on the kept modes
    if (e == cudaSuccess)
      e = launch_pdl(fno_rfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float*)abar[cur], L.fno_s,
                     tw, M);
    if (e == cudaSuccess && dparams)
      e = launch_pdl(fno_rgrad_kernel<C>, dim3(nb), dim3(256), 0, st, (const float2*)L.fno_s,
                     (const float2*)(sb.S + l * spec), dR, nm, M, batch, 1.0f / (float)nn);
    // v_bar through the spectral convolution: the same convolution with R^H
    if (e == cudaSuccess)
      e = launch_pdl(fno_mix_kernel<C>, mix, dim3(256), MixCfg<C>::SMEM, st, (const float2*)L.fno_s,
                     (const float2*)(net.rph + (size_t)l * nb * C * C * kMixModes), L.fno_s2, nm, batch);
    if (e == cudaSuccess)
      e = launch_pdl(fno_irfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float2*)L.fno_s2, L.fno_y,
                     tw, M, 1.0f / (float)nn);
    // v_bar_l = W^T a_bar + spectral part; a_bar of layer l - 1 = v_bar_l GELU'(a_{l-1})
    if (e == cudaSuccess)
      e = launch_pdl(fno_pointwise_t_kernel<C, C>, pix, dim3(256), 0, st, (const float*)L.fno_y,
                     (const float*)abar[cur], W, l > 0 ? (const float*)(sb.a + (l - 1) * fld) : (const float*)nullptr,
                     abar[cur ^ 1], batch, nn, (size_t)0);
    cur ^= 1;
  }
  // lift: gradients of P, input cotangent P^T v_bar_0
  if (e == cudaSuccess && dparams)
    e = outer_grad<C, CIN>(abar[cur], nullptr, single, hist, batch, nn, partial, dP, dP + (size_t)C * CIN, st);
  if (e == cudaSuccess)
    e = launch_pdl(fno_pointwise_t_kernel<C, CIN>, pix, dim3(256), 0, st, accumulate ? (const float*)ubar : nullptr,
                   (const float*)abar[cur], P, (const float*)nullptr, ubar, batch, nn, ost);
  return e;
}

}  // namespace

int fd_fno_launches(int layers) { return layers > 0 ? 2 + 4 * layers : 0; }

// O_F (which = 0) or the FNO temporal correction (which = 1) of the context
static FnoNet fno_net(const LearnedState& L, int which) {
  return which == 0 ? FnoNet{L.fno_layers, L.fno_modes, 8, L.raw_off_fno, L.fno_out, L.fno_rp, L.fno_rph}
                    : FnoNet{L.tcf_layers, L.tcf_modes, 2, L.raw_off_tcf, L.corr, L.tcf_rp, L.tcf_rph};
}

// floats of the saved activations of one evaluation (v, a) and float2 of its spectra
void fd_fno_saved_sizes(const LearnedState& L, int which, int batch, int nn, size_t* v_floats, size_t* a_floats,
                        size_t* s_float2, size_t* out_floats) {
  const int layers = which == 0 ? L.fno_layers : L.tcf_layers;
  const int modes = which == 0 ? L.fno_modes : L.tcf_modes;
  const int width = which == 0 ? L.fno_width : L.tcf_width;
  const size_t fld = (size_t)batch * width * nn;
  *v_floats = (size_t)(layers + 1) * fld;
  *a_floats = (size_t)(layers > 1 ? layers - 1 : 1) * fld;
  *s_float2 = (size_t)layers * batch * width * 2 * modes * modes;
  *out_floats = (size_t)batch * (which == 0 ? 8 : 2) * nn;
}

// forward of O_F (single = the stage state) or of the FNO correction (hist = the
// k_c history states), keeping the activations in sb
cudaError_t fd_fno_forward_saved(fd_ctx* c, int which, const float* single, const float* const* hist,
                                 const FnoSavedBufs& sb, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  FnoNet net = fno_net(L, which);
  const float2* tw = reinterpret_cast<const float2*>(c->base.tw);
  const int B = c->grid.batch, ns = which == 0 ? 1 : L.kc;
  const int width = which == 0 ? L.fno_width : L.tcf_width;
  if (which == 0) {
    if (c->logn == 6)
      return width == 16 ? fno_run_saved<6, 16, 8>(L, net, single, hist, ns, sb, tw, B, st)
                         : fno_run_saved<6, 8, 8>(L, net, single, hist, ns, sb, tw, B, st);
    return width == 16 ? fno_run_saved<5, 16, 8>(L, net, single, hist, ns, sb, tw, B, st)
                       : fno_run_saved<5, 8, 8>(L, net, single, hist, ns, sb, tw, B, st);
  }
  if (c->logn == 6)
    return width == 16 ? fno_run_saved<6, 16, 2>(L, net, single, hist, ns, sb, tw, B, st)
                       : fno_run_saved<6, 8, 2>(L, net, single, hist, ns, sb, tw, B, st);
  return width == 16 ? fno_run_saved<5, 16, 2>(L, net, single, hist, ns, sb, tw, B, st)
                     : fno_run_saved<5, 8, 2>(L, net, single, hist, ns, sb, tw, B, st);
}

template <int LOGN, int C>
static cudaError_t fno_back_tc(LearnedState& L, const FnoNet& net, const FnoSavedBufs& sb, const float* const* hist,
                               const float* gbar, float* ubar, size_t ost, float* dparams, float* partial,
                               const float2* tw, int B, cudaStream_t st) {
  switch (L.kc) {
    case 1: return fno_back<LOGN, C, 2, 2>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    case 2: return fno_back<LOGN, C, 2, 4>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    case 3: return fno_back<LOGN, C, 2, 6>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    case 4: return fno_back<LOGN, C, 2, 8>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    case 5: return fno_back<LOGN, C, 2, 10>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    case 6: return fno_back<LOGN, C, 2, 12>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    case 7: return fno_back<LOGN, C, 2, 14>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
    default: return fno_back<LOGN, C, 2, 16>(L, net, sb, nullptr, hist, gbar, ubar, ost, false, dparams, partial, tw, B, st);
  }
}

// reverse mode of O_F (which = 0: gbar [batch][8][N][N], the input cotangent
// added to / written into ubar [batch][2][N][N]) or of the FNO correction
// (which = 1: gbar [batch][2][N][N], history cotangents written to ubar with
// state stride ost); dparams (may be null) accumulates the parameter gradients
cudaError_t fd_fno_backward(fd_ctx* c, int which, const FnoSavedBufs& sb, const float* single,
                            const float* const* hist, const float* gbar, float* ubar, size_t ost, bool accumulate,
                            float* dparams, float* partial, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  FnoNet net = fno_net(L, which);
  const float2* tw = reinterpret_cast<const float2*>(c->base.tw);
  const int B = c->grid.batch;
  const int width = which == 0 ? L.fno_width : L.tcf_width;
  if (which == 0) {
    if (c->logn == 6)
      return width == 16 ? fno_back<6, 16, 8, 2>(L, net, sb, single, nullptr, gbar, ubar, 0, accumulate, dparams,
                                                 partial, tw, B, st)
                         : fno_back<6, 8, 8, 2>(L, net, sb, single, nullptr, gbar, ubar, 0, accumulate, dparams,
                                                partial, tw, B, st);
    return width == 16 ? fno_back<5, 16, 8, 2>(L, net, sb, single, nullptr, gbar, ubar, 0, accumulate, dparams, partial,
                                               tw, B, st)
                       : fno_back<5, 8, 8, 2>(L, net, sb, single, nullptr, gbar, ubar, 0, accumulate, dparams, partial,
                                              tw, B, st);
  }
  if (c->logn == 6)
    return width == 16 ? fno_back_tc<6, 16>(L, net, sb, hist, gbar, ubar, ost, dparams, partial, tw, B, st)
                       : fno_back_tc<6, 8>(L, net, sb, hist, gbar, ubar, ost, dparams, partial, tw, B, st);
  return width == 16 ? fno_back_tc<5, 16>(L, net, sb, hist, gbar, ubar, ost, dparams, partial, tw, B, st)
                     : fno_back_tc<5, 8>(L, net, sb, hist, gbar, ubar, ost, dparams, partial, tw, B, st);
}

// partial-sum floats the reverse mode of either operator needs
size_t fd_fno_partial_floats() { return (size_t)kOuterBlocks * (16 * 16 + 16); }

// O_F of the stage state u [batch][2][N][N] into c->lrn->fno_out [batch][8][N][N]
cudaError_t fd_fno_forward(fd_ctx* c, const float* u, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const FnoNet net{L.fno_layers, L.fno_modes, 8, L.raw_off_fno, L.fno_out, L.fno_rp, L.fno_rph};
  return fno_dispatch<8>(c, net, L.fno_width, u, nullptr, 1, st);
}

// FNO temporal correction of the k_c states hist[0 .. k_c-1] (device pointer
// array, oldest first) into c->lrn->corr [batch][2][N][N]
cudaError_t fd_fno_tc(fd_ctx* c, const float* const* hist, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const FnoNet net{L.tcf_layers, L.tcf_modes, 2, L.raw_off_tcf, L.corr, L.tcf_rp, L.tcf_rph};
  return fno_dispatch<2>(c, net, L.tcf_width, nullptr, hist, L.kc, st);
}

// elements of the mode-blocked channel matrices of one operator (all layers)
size_t fd_fno_rp_count(int layers, int modes, int width) {
  const size_t nb = ((size_t)2 * modes * modes + kMixModes - 1) / kMixModes;
  return (size_t)layers * nb * width * width * kMixModes;
}

// after a parameter upload: the channel matrices of O_F and of the FNO temporal
// correction in the mode-blocked layout of the mixing kernel
cudaError_t fd_fno_pack(LearnedState& L, cudaStream_t st) {
  struct Op {
    int layers, modes, width, cin;
    size_t raw_off;
    float2* rp;
    float2* rph;
  };
  const Op ops[2] = {{L.fno_layers, L.fno_modes, L.fno_width, 2, L.raw_off_fno, L.fno_rp, L.fno_rph},
                     {L.tcf_layers, L.tcf_modes, L.tcf_width, 2 * L.kc, L.raw_off_tcf, L.tcf_rp, L.tcf_rph}};
  for (const Op& op : ops) {
    if (op.layers <= 0) continue;
    const int C = op.width, nm = 2 * op.modes * op.modes;
    const size_t layer_size = (size_t)nm * C * C * 2 + (size_t)C * C + C;
    const size_t per = fd_fno_rp_count(1, op.modes, C);
    for (int l = 0; l < op.layers; ++l) {
      const float* R = L.d_raw + op.raw_off + (size_t)C * op.cin + C + l * layer_size;
      fno_pack_r_kernel<<<2 * L.sms, 256, 0, st>>>(R, op.rp + l * per, nm, C);
      fno_pack_rh_kernel<<<2 * L.sms, 256, 0, st>>>(R, op.rph + l * per, nm, C);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// kernel attributes (outside any stream capture): the mixing kernels' shared memory
cudaError_t fd_fno_prepare() {
  cudaError_t e = cudaFuncSetAttribute(fno_mix_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)MixCfg<16>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fno_mix_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MixCfg<8>::SMEM);
  return e;
}
