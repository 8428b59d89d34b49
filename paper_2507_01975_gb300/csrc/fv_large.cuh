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
#include "fv_fft.cuh"

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
  // multiply by 1 / (N^2 symbol(kx, ky)); the zero mode is removed. The
  // registers already hold the points in the inverse transform's input order
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
