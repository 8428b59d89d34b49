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
                                                           float* __restrict__ out, int batch, int nn, int gelu) {
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
    out[(b * CO + o) * nn + p] = gelu ? gelu_exact(s) : s;
  }
}

// S2[b][o][m] = sum_i R[m][i][o] S[b][i][m] (complex); R: [nm][C][C][2] floats.
// A CTA takes 32 modes x 32 trajectories: the modes' channel matrices go to
// shared memory once ([i][o][mode], padded), the spectra in slices of 8
// trajectories ([b][i][mode]); lane = mode, so loads and stores run along the
// contiguous mode index.
constexpr int kMixModes = 32, kMixBatch = 32, kMixSlice = 8, kMixPad = 33;

template <int C>
struct MixCfg {
  static constexpr size_t SMEM = ((size_t)C * C * kMixPad + (size_t)kMixSlice * C * kMixModes) * sizeof(float2);
};

template <int C>
__global__ void __launch_bounds__(256) fno_mix_kernel(const float2* __restrict__ S, const float* __restrict__ R,
                                                     float2* __restrict__ S2, int nm, int batch) {
  extern __shared__ __align__(16) float2 smx[];
  float2* Rs = smx;                          // [C * C][kMixPad]
  float2* Ss = smx + C * C * kMixPad;        // [kMixSlice][C][kMixModes]
  const int m0 = blockIdx.x * kMixModes, b0 = blockIdx.y * kMixBatch;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  // R[m0 + mm][i][o] -> Rs[(i C + o) kMixPad + mm]; consecutive threads read consecutive (i, o)
  for (int e = threadIdx.x; e < C * C * kMixModes; e += blockDim.x) {
    const int io = e % (C * C), mm = e / (C * C), m = m0 + mm;
    const float* r = R + ((size_t)m * C * C + io) * 2;
    Rs[io * kMixPad + mm] = m < nm ? make_float2(r[0], r[1]) : make_float2(0.0f, 0.0f);
  }
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  // this thread's outputs o = grp + 8 j: their matrix columns in registers
  constexpr int NO = C / 8;
  float2 r[NO][C];
#pragma unroll
  for (int j = 0; j < NO; ++j)
#pragma unroll
    for (int i = 0; i < C; ++i) r[j][i] = Rs[(i * C + grp + 8 * j) * kMixPad + lane];
  const int m = m0 + lane;
  for (int bt = 0; bt < kMixBatch; bt += kMixSlice) {
    if (bt > 0) __syncthreads();  // the previous slice is consumed
    for (int e = threadIdx.x; e < kMixSlice * C * kMixModes; e += blockDim.x) {
      const int mm = e % kMixModes, bi = e / kMixModes, bb = bi / C, i = bi % C;
      const int b = b0 + bt + bb;
      Ss[e] = (b < batch && m0 + mm < nm) ? S[((size_t)b * C + i) * nm + m0 + mm] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll 2
    for (int bb = 0; bb < kMixSlice; ++bb) {
      float2 sv[C];
#pragma unroll
      for (int i = 0; i < C; ++i) sv[i] = Ss[(bb * C + i) * kMixModes + lane];
      const int b = b0 + bt + bb;
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 0; i < C; ++i) acc = c2add(acc, c2mul(sv[i], r[j][i]));
        if (b < batch && m < nm) S2[((size_t)b * C + grp + 8 * j) * nm + m] = acc;
      }
    }
  }
}

template <int LOGN>
struct FnoFftCfg {
  static constexpr int N = 1 << LOGN, T = N / kFP;
  static constexpr int NTR = N / 2;  // row transforms (pairs of real rows); also >= the kept columns
  static constexpr int NT = NTR * T;
  static_assert(T < 64, "transform syncs are warp-level here");
  static size_t smem(int M) {
    return ((size_t)NTR * SPlan<LOGN>::BUF + SPlan<LOGN>::TW + (size_t)N * M) * sizeof(float2);
  }
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
  float2* tws = sm + Cfg::NTR * SP::BUF;
  float2* Rs = tws + SP::TW;  // [N][M] row spectra
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int C = gridDim.x, b = blockIdx.y, c = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const float* field = v + ((size_t)b * C + c) * NN;
  float2* buf = sm + f * SP::BUF;
  const TransformSync sync{1 + f, T};
  build_pass_twiddles<LOGN>(tws, tw);
  pdl_wait();
  pdl_trigger();
  // rows 2f and 2f + 1 as one complex transform
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = make_float2(field[(2 * f) * N + t + m * T], field[(2 * f + 1) * N + t + m * T]);
  __syncthreads();
  fft_forward<LOGN>(z, buf, tws, t, sync);
  fft_store_natural<LOGN>(buf, z, t);
  sync();
  for (int k = t; k < M; k += T) {
    const float2 zk = buf[fpad(k)], zm = buf[fpad((N - k) & MSK)];
    Rs[(2 * f) * M + k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    Rs[(2 * f + 1) * M + k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  }
  __syncthreads();
  // column kx = f (kept when f < M; the others run on column 0 and discard)
  const int kx = f < M ? f : 0;
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = Rs[(t + m * T) * M + kx];
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
  float2* tws = sm + Cfg::NTR * SP::BUF;
  float2* Rs = tws + SP::TW;  // [N][M] rows after the inverse column transforms
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int C = gridDim.x, b = blockIdx.y, c = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const float2* in = S2 + ((size_t)b * C + c) * 2 * M * M;
  float2* buf = sm + f * SP::BUF;
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
      for (int r = 0; r < SP::RL; ++r) Rs[(t + s * T + r * SP::NSL) * M + kx] = z[s + SP::SL * r];
  }
  __syncthreads();
  // rows 2f, 2f + 1: Z_k = A_k + i B_k on the Hermitian extension of each row
  const float2* A = Rs + (2 * f) * M;
  const float2* Bv = Rs + (2 * f + 1) * M;
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
  float* out = y + ((size_t)b * C + c) * NN;
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) {
      const int x = t + s * T + r * SP::NSL;
      out[(2 * f) * N + x] = z[s + SP::SL * r].x * scale;
      out[(2 * f + 1) * N + x] = z[s + SP::SL * r].y * scale;
    }
}

// one Fourier neural operator: width C, `layers` layers of `modes` kept modes,
// parameters at raw_off (P_w[C][cin], P_b[C], layers, Q_w[cout][C], Q_b[cout]),
// output [batch][cout][N][N]
struct FnoNet {
  int layers, modes, cout;
  size_t raw_off;
  float* out;
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
  const dim3 mix((nm + kMixModes - 1) / kMixModes, (batch + kMixBatch - 1) / kMixBatch);
  cudaError_t e = launch_pdl(fno_lift_kernel<C>, pix, dim3(256), 0, st, single, hist, ns, P, L.fno_v[0], batch, nn);
  int cur = 0;
  for (int l = 0; l < nl && e == cudaSuccess; ++l) {
    const float* R = R0 + (size_t)l * layer_size;
    const float* W = R + (size_t)nm * C * C * 2;
    const float* Wb = W + (size_t)C * C;
    e = launch_pdl(fno_rfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float*)L.fno_v[cur], L.fno_s,
                   tw, M);
    if (e == cudaSuccess)
      e = launch_pdl(fno_mix_kernel<C>, mix, dim3(256), MixCfg<C>::SMEM, st, (const float2*)L.fno_s, R, L.fno_s2, nm,
                     batch);
    if (e == cudaSuccess)
      e = launch_pdl(fno_irfft_kernel<LOGN>, dim3(C, batch), dim3(Cfg::NT), fsm, st, (const float2*)L.fno_s2, L.fno_y,
                     tw, M, 1.0f / (float)nn);
    if (e == cudaSuccess)
      e = launch_pdl(fno_pointwise_kernel<C, C>, pix, dim3(256), 0, st, (const float*)L.fno_y,
                     (const float*)L.fno_v[cur], W, Wb, L.fno_v[cur ^ 1], batch, nn, l < nl - 1 ? 1 : 0);
    cur ^= 1;
  }
  if (e == cudaSuccess)
    e = launch_pdl(fno_pointwise_kernel<C, CO>, pix, dim3(256), 0, st, (const float*)nullptr,
                   (const float*)L.fno_v[cur], Q, Q + (size_t)CO * C, net.out, batch, nn, 0);
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

}  // namespace

int fd_fno_launches(int layers) { return layers > 0 ? 2 + 4 * layers : 0; }

// O_F of the stage state u [batch][2][N][N] into c->lrn->fno_out [batch][8][N][N]
cudaError_t fd_fno_forward(fd_ctx* c, const float* u, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const FnoNet net{L.fno_layers, L.fno_modes, 8, L.raw_off_fno, L.fno_out};
  return fno_dispatch<8>(c, net, L.fno_width, u, nullptr, 1, st);
}

// FNO temporal correction of the k_c states hist[0 .. k_c-1] (device pointer
// array, oldest first) into c->lrn->corr [batch][2][N][N]
cudaError_t fd_fno_tc(fd_ctx* c, const float* const* hist, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const FnoNet net{L.tcf_layers, L.tcf_modes, 2, L.raw_off_tcf, L.corr};
  return fno_dispatch<2>(c, net, L.tcf_width, nullptr, hist, L.kc, st);
}

// kernel attributes (outside any stream capture): the mixing kernels' shared memory
cudaError_t fd_fno_prepare() {
  cudaError_t e = cudaFuncSetAttribute(fno_mix_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)MixCfg<16>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fno_mix_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MixCfg<8>::SMEM);
  return e;
}
