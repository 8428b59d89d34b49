// fv_large.cuh -- the plain FV step for large grids (N = 512 .. 2048) that do
// not fit on chip: the state streams through HBM once per kernel.
//
// One RK4 stage (App. B.5) is four kernels:
//   stage     tiles of 32 x 16 cells with a 2-cell halo in shared memory:
//             w = x - G2 p (the projection of the previous stage, applied on
//             the fly), the eight physics face operators (Sec. 3.4, App. B.2),
//             the flux assembly and source terms, the RK combination with u_n
//             and the accumulator -> w* and acc;
//   rows_fwd  divergence D2 w* (two-point, Sec. 3.6) of 8 rows, real-to-complex
//             row FFTs (two real rows per complex transform), half spectra
//             written column-major (kx-major, y contiguous);
//   cols      column FFTs, multiplication by 1 / symbol(D2 G2) (zero mode 0,
//             App. B.3-B.4), inverse column FFTs;
//   rows_inv  complex-to-real inverse row FFTs -> pressure p.
// A final kernel forms u_{n+1} = w*_4 - G2 p_4. The FFTs are radix-2
// transforms in shared memory (decimation in frequency forward, natural in /
// bit-reversed out; decimation in time inverse, bit-reversed in / natural out),
// so no reordering pass is needed between them.
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
  float2* spec;       // [batch][N/2 + 1][N] complex (column-major half spectra)
  float* pout;        // rows_inv output; final input
  float* uout;        // final output
  int stage, flow, forcing;
  float dt, nu, idx, idy, drag, inv_nn;
  const float2* tw;   // [N/2]: exp(-2 pi i m / N)
  const float* symx;  // [N/2 + 2]
  const float* symy;  // [N]
  const float* frc;   // [N]
};

constexpr int kLTX = 32, kLTY = 16;  // stage tile (cells)
constexpr int kLRB = 8;              // rows per CTA of the row transforms
constexpr int kLCB = 2;              // columns per CTA of the column transforms
constexpr int kLKC = 128;            // spectrum columns staged at a time by rows_inv

__device__ __forceinline__ float2 c2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c2mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c2mulc(float2 a, float2 w) {  // a * conj(w)
  return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
__device__ __forceinline__ int brev_n(int k, int logn) { return (int)(__brev((unsigned)k) >> (32 - logn)); }

// F forward transforms of length N = 2^logn stored at x + f * stride:
// natural-order input, bit-reversed output (radix-2 decimation in frequency)
__device__ void block_fft_dif(float2* x, int F, int stride, int logn, const float2* tw) {
  const int N = 1 << logn, H = N >> 1;
  for (int len = N; len >= 2; len >>= 1) {
    const int half = len >> 1, tstep = N / len;
    for (int t = threadIdx.x; t < F * H; t += blockDim.x) {
      const int f = t / H, r = t - f * H;
      const int blk = r / half, j = r - blk * half;
      float2* b = x + f * stride + blk * len;
      const float2 a = b[j], c = b[j + half];
      b[j] = c2add(a, c);
      b[j + half] = c2mul(c2sub(a, c), tw[j * tstep]);
    }
    __syncthreads();
  }
}

// F inverse (unnormalised) transforms: bit-reversed input, natural output
// (radix-2 decimation in time with conjugate twiddles)
__device__ void block_ifft_dit(float2* x, int F, int stride, int logn, const float2* tw) {
  const int N = 1 << logn, H = N >> 1;
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1, tstep = N / len;
    for (int t = threadIdx.x; t < F * H; t += blockDim.x) {
      const int f = t / H, r = t - f * H;
      const int blk = r / half, j = r - blk * half;
      float2* b = x + f * stride + blk * len;
      const float2 a = b[j];
      const float2 c = c2mulc(b[j + half], tw[j * tstep]);
      b[j] = c2add(a, c);
      b[j + half] = c2sub(a, c);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// stage kernel: tile of kLTX x kLTY cells, 256 threads (two cells each)
// ---------------------------------------------------------------------------
template <int DORD>
__global__ void __launch_bounds__(256) large_stage_kernel(const LargeArgs a, int logn) {
  constexpr int WX = kLTX + 4, WY = kLTY + 4, PX = kLTX + 5, PY = kLTY + 5;
  __shared__ float U[WY][WX];
  __shared__ float V[WY][WX];
  __shared__ float P[PY][PX];
  const int N = 1 << logn, MSK = N - 1;
  const size_t NN = (size_t)N * N;
  const int b = blockIdx.z;
  const int x0 = blockIdx.x * kLTX, y0 = blockIdx.y * kLTY;
  const int tid = threadIdx.x;
  const float* xu = a.x + (size_t)b * 2 * NN;
  const float* xv = xu + NN;
  if (a.p) {
    const float* pp = a.p + (size_t)b * NN;
    for (int k = tid; k < PX * PY; k += 256) {
      const int py = k / PX, px = k - py * PX;
      P[py][px] = pp[(size_t)((y0 - 3 + py) & MSK) * N + ((x0 - 3 + px) & MSK)];
    }
    __syncthreads();
  }
  for (int k = tid; k < WX * WY; k += 256) {
    const int wy = k / WX, wx = k - wy * WX;
    const size_t g = (size_t)((y0 - 2 + wy) & MSK) * N + ((x0 - 2 + wx) & MSK);
    float u = xu[g], v = xv[g];
    if (a.p) {
      // w = x - G2 p: u-face gradient p(i) - p(i - 1), v-face p(j) - p(j - 1)
      u -= (P[wy + 1][wx + 1] - P[wy + 1][wx]) * a.idx;
      v -= (P[wy + 1][wx + 1] - P[wy][wx + 1]) * a.idy;
    }
    U[wy][wx] = u;
    V[wy][wx] = v;
  }
  __syncthreads();

  constexpr float d0 = DORD == 4 ? 1.0f / 24.0f : 0.0f;
  constexpr float d1 = DORD == 4 ? -27.0f / 24.0f : -1.0f;
  constexpr float d2 = DORD == 4 ? 27.0f / 24.0f : 1.0f;
  constexpr float d3 = DORD == 4 ? -1.0f / 24.0f : 0.0f;
  const float idx = a.idx, idy = a.idy;
  // face values at tile-local coordinates (ly, lx) = (j - y0 + 2, i - x0 + 2)
  auto Uc = [&](int ly, int lx) { return 0.5f * (U[ly][lx] + U[ly][lx + 1]); };
  auto Gxc = [&](int ly, int lx) {
    return (d0 * U[ly][lx - 1] + d1 * U[ly][lx] + d2 * U[ly][lx + 1] + d3 * U[ly][lx + 2]) * idx;
  };
  auto Uk = [&](int ly, int lx) { return 0.5f * (U[ly - 1][lx] + U[ly][lx]); };
  auto Gyu = [&](int ly, int lx) {
    return (d0 * U[ly - 2][lx] + d1 * U[ly - 1][lx] + d2 * U[ly][lx] + d3 * U[ly + 1][lx]) * idy;
  };
  auto Vk = [&](int ly, int lx) { return 0.5f * (V[ly][lx - 1] + V[ly][lx]); };
  auto Gxv = [&](int ly, int lx) {
    return (d0 * V[ly][lx - 2] + d1 * V[ly][lx - 1] + d2 * V[ly][lx] + d3 * V[ly][lx + 1]) * idx;
  };
  auto Vc = [&](int ly, int lx) { return 0.5f * (V[ly][lx] + V[ly + 1][lx]); };
  auto Gyc = [&](int ly, int lx) {
    return (d0 * V[ly - 1][lx] + d1 * V[ly][lx] + d2 * V[ly + 1][lx] + d3 * V[ly + 2][lx]) * idy;
  };

  const float ca = a.stage == 2 ? a.dt : 0.5f * a.dt;
  const float c6 = a.dt / 6.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int tx = tid & 31, ty = (tid >> 5) + 8 * h;
    const int lx = tx + 2, ly = ty + 2;
    const int i = x0 + tx, j = y0 + ty;
    const float ukc = Uk(ly, lx) * Vk(ly, lx);
    float tu = -(Uc(ly, lx) * Uc(ly, lx) - Uc(ly, lx - 1) * Uc(ly, lx - 1)) * idx -
               (Uk(ly + 1, lx) * Vk(ly + 1, lx) - ukc) * idy +
               a.nu * ((Gxc(ly, lx) - Gxc(ly, lx - 1)) * idx + (Gyu(ly + 1, lx) - Gyu(ly, lx)) * idy);
    float tv = -(Uk(ly, lx + 1) * Vk(ly, lx + 1) - ukc) * idx -
               (Vc(ly, lx) * Vc(ly, lx) - Vc(ly - 1, lx) * Vc(ly - 1, lx)) * idy +
               a.nu * ((Gxv(ly, lx + 1) - Gxv(ly, lx)) * idx + (Gyc(ly, lx) - Gyc(ly - 1, lx)) * idy);
    const float uc = U[ly][lx], vc = V[ly][lx];
    if (a.flow == 0) {
      const float dc = Gxc(ly, lx) + Gyc(ly, lx);
      tu += uc * 0.5f * ((Gxc(ly, lx - 1) + Gyc(ly, lx - 1)) + dc);
      tv += vc * 0.5f * ((Gxc(ly - 1, lx) + Gyc(ly - 1, lx)) + dc);
    }
    if (a.forcing == 1) {
      tu += a.frc[j] - a.drag * uc;
      tv -= a.drag * vc;
    }
    const size_t g = (size_t)b * 2 * NN + (size_t)j * N + i;
    const float un_u = a.un[g], un_v = a.un[g + NN];
    if (a.stage < 3) {
      float au = tu, av = tv;
      if (a.stage > 0) {
        au = a.acc[g] + 2.0f * tu;
        av = a.acc[g + NN] + 2.0f * tv;
      }
      a.acc[g] = au;
      a.acc[g + NN] = av;
      a.ws[g] = un_u + ca * tu;
      a.ws[g + NN] = un_v + ca * tv;
    } else {
      a.ws[g] = un_u + c6 * (a.acc[g] + tu);
      a.ws[g + NN] = un_v + c6 * (a.acc[g + NN] + tv);
    }
  }
}

// ---------------------------------------------------------------------------
// rows_fwd: kLRB rows per CTA -> kLRB / 2 complex row transforms
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) large_rows_fwd_kernel(const LargeArgs a, int logn) {
  extern __shared__ __align__(16) float2 sm[];
  const int N = 1 << logn, MSK = N - 1, H = N / 2;
  constexpr int F = kLRB / 2;
  float2* buf = sm;           // [F][N]
  float2* tw = sm + F * N;    // [N/2]
  const int b = blockIdx.y, y0 = blockIdx.x * kLRB;
  const size_t NN = (size_t)N * N;
  const float* u = a.ws + (size_t)b * 2 * NN;
  const float* v = u + NN;
  for (int k = threadIdx.x; k < H; k += blockDim.x) tw[k] = a.tw[k];
  for (int t = threadIdx.x; t < F * N; t += blockDim.x) {
    const int f = t / N, x = t - f * N;
    const int ra = y0 + 2 * f, rb = ra + 1;
    const int xe = (x + 1) & MSK;
    const float da = (u[(size_t)ra * N + xe] - u[(size_t)ra * N + x]) * a.idx +
                     (v[(size_t)rb * N + x] - v[(size_t)ra * N + x]) * a.idy;
    const float db = (u[(size_t)rb * N + xe] - u[(size_t)rb * N + x]) * a.idx +
                     (v[(size_t)((rb + 1) & MSK) * N + x] - v[(size_t)rb * N + x]) * a.idy;
    buf[f * N + x] = make_float2(da, db);
  }
  __syncthreads();
  block_fft_dif(buf, F, N, logn, tw);
  // unpack the two real rows of each transform: A_k = (Z_k + conj Z_{N-k}) / 2,
  // B_k = (Z_k - conj Z_{N-k}) / (2i); Z_k sits at bit-reversed position
  float2* spec = a.spec + (size_t)b * (H + 1) * N;
  for (int t = threadIdx.x; t < (H + 1) * kLRB; t += blockDim.x) {
    const int k = t / kLRB, yy = t - k * kLRB;
    const int f = yy >> 1;
    const float2 zk = buf[f * N + brev_n(k & MSK, logn)];
    const float2 zm = buf[f * N + brev_n((N - k) & MSK, logn)];
    float2 val;
    if ((yy & 1) == 0)
      val = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    else
      val = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    spec[(size_t)k * N + y0 + yy] = val;
  }
}

// ---------------------------------------------------------------------------
// cols: kLCB spectrum columns per CTA: forward FFT along y, 1 / symbol, inverse
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) large_cols_kernel(const LargeArgs a, int logn) {
  extern __shared__ __align__(16) float2 sm[];
  const int N = 1 << logn, H = N / 2;
  float2* buf = sm;                 // [kLCB][N]
  float2* tw = sm + kLCB * N;       // [N/2]
  float* sy = reinterpret_cast<float*>(tw + H);  // [N]
  const int b = blockIdx.y, kx0 = blockIdx.x * kLCB;
  const int F = (H + 1 - kx0) < kLCB ? (H + 1 - kx0) : kLCB;
  float2* spec = a.spec + (size_t)b * (H + 1) * N;
  for (int k = threadIdx.x; k < H; k += blockDim.x) tw[k] = a.tw[k];
  for (int k = threadIdx.x; k < N; k += blockDim.x) sy[k] = a.symy[k];
  for (int t = threadIdx.x; t < F * N; t += blockDim.x) buf[t] = spec[(size_t)kx0 * N + t];
  __syncthreads();
  block_fft_dif(buf, F, N, logn, tw);
  for (int t = threadIdx.x; t < F * N; t += blockDim.x) {
    const int f = t / N, pos = t - f * N;
    const int kx = kx0 + f, ky = brev_n(pos, logn);
    const float m = (kx == 0 && ky == 0) ? 0.0f : __fdividef(a.inv_nn, a.symx[kx] + sy[ky]);
    buf[t] = make_float2(buf[t].x * m, buf[t].y * m);
  }
  __syncthreads();
  block_ifft_dit(buf, F, N, logn, tw);
  for (int t = threadIdx.x; t < F * N; t += blockDim.x) spec[(size_t)kx0 * N + t] = buf[t];
}

// ---------------------------------------------------------------------------
// rows_inv: kLRB rows per CTA from the column-major spectrum -> pressure rows
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) large_rows_inv_kernel(const LargeArgs a, int logn) {
  extern __shared__ __align__(16) float2 sm[];
  const int N = 1 << logn, H = N / 2, MSK = N - 1;
  constexpr int F = kLRB / 2;
  float2* buf = sm;                   // [F][N]
  float2* tw = sm + F * N;            // [N/2]
  float2* stg = tw + H;               // [kLKC][kLRB]
  const int b = blockIdx.y, y0 = blockIdx.x * kLRB;
  const float2* spec = a.spec + (size_t)b * (H + 1) * N;
  for (int k = threadIdx.x; k < H; k += blockDim.x) tw[k] = a.tw[k];
  // rebuild the packed transforms Z_k = P_a[k] + i P_b[k] (Hermitian halves for k > N/2)
  for (int k0 = 0; k0 <= H; k0 += kLKC) {
    const int kn = (H + 1 - k0) < kLKC ? (H + 1 - k0) : kLKC;
    __syncthreads();
    for (int t = threadIdx.x; t < kn * kLRB; t += blockDim.x) {
      const int kk = t / kLRB, yy = t - kk * kLRB;
      stg[t] = spec[(size_t)(k0 + kk) * N + y0 + yy];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < F * kn; t += blockDim.x) {
      const int f = t / kn, kk = t - f * kn;
      const int k = k0 + kk;
      const float2 pa = stg[kk * kLRB + 2 * f], pb = stg[kk * kLRB + 2 * f + 1];
      buf[f * N + brev_n(k & MSK, logn)] = make_float2(pa.x - pb.y, pa.y + pb.x);
      if (k > 0 && k < H) buf[f * N + brev_n(N - k, logn)] = make_float2(pa.x + pb.y, pb.x - pa.y);
    }
  }
  __syncthreads();
  block_ifft_dit(buf, F, N, logn, tw);
  float* p = a.pout + (size_t)b * N * N;
  for (int t = threadIdx.x; t < F * N; t += blockDim.x) {
    const int f = t / N, x = t - f * N;
    const float2 z = buf[t];
    p[(size_t)(y0 + 2 * f) * N + x] = z.x;
    p[(size_t)(y0 + 2 * f + 1) * N + x] = z.y;
  }
}

// u_{n+1} = w* - G2 p (or w* itself without a projection)
__global__ void __launch_bounds__(256) large_final_kernel(const LargeArgs a, int logn, int batch) {
  const int N = 1 << logn, MSK = N - 1;
  const size_t NN = (size_t)N * N;
  const size_t total = (size_t)batch * NN;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t b = e / NN, c = e - b * NN;
    const size_t g = b * 2 * NN + c;
    if (!a.pout) {  // no projection (Burgers)
      a.uout[g] = a.ws[g];
      a.uout[g + NN] = a.ws[g + NN];
      continue;
    }
    const int j = (int)(c >> logn), i = (int)(c & MSK);
    const float* p = a.pout + b * NN;
    const float pc = p[c];
    const float pw = p[(size_t)j * N + ((i - 1) & MSK)];
    const float ps = p[(size_t)((j - 1) & MSK) * N + i];
    a.uout[g] = a.ws[g] - (pc - pw) * a.idx;
    a.uout[g + NN] = a.ws[g + NN] - (pc - ps) * a.idy;
  }
}

}  // namespace ldfv
