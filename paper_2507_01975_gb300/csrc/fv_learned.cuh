// fv_learned.cuh -- one RK stage of the learned FV step (banded flux kernel +
// per-trajectory projection), and the corrected projection of the
// temporal-correction step (N <= 64).
//
// Flux block with learned per-face kernels (Sec. 3.4, integrated operator):
// for each of the eight operator instances q (u/v x x/y x interp/deriv) the
// kernel at output location f is
//   K_q,f = W_P,q + proj(W_L[kind, axis] + C_theta(w)_q,f) / h^(kind==deriv),
// where C_theta(w) is the stencil network's 160-channel output (channel
// 20 q + 5 x 4 tap index, BF16 chunk planes) and proj removes the sum, the
// first axial moment and the first transverse moment of the learned part
// (consistency: W_P + proj(L) still interpolates / differentiates linear data
// exactly). The instance value is sum_rc K[r][c] f[tap(r, c)] on the 5 x 4 tap
// grid (transverse offset r - 2, axial offset c - 3/2 cells).
//
// Then the flux assembly (App. B.2), the RK4 stage combination with u_n and
// the accumulator in global memory, and (Navier-Stokes) the spectral pressure
// projection (Sec. 3.6, App. B.3-B.4) with warp FFTs, in shared memory.
#pragma once

#include <cuda_bf16.h>

#include "fv_common.cuh"

namespace ldfv {

struct LStageArgs {
  const float* w;    // stage state [batch][2][N][N]
  const float* un;   // state at the start of the step
  float* acc;        // RK4 accumulator [batch][2][N][N]
  float* wout;       // projected next stage state (or the step result)
  const __nv_bfloat16* coef;  // [batch][20][N][N][8] network output, or null (C = 0)
  const float* wl;   // W_L [kind 2][axis 2][5][4]
  const float* corr; // correct_project only: correction [batch][2][N][N]
  const float* fno;  // O_F(u) [batch][8][N][N] added to the face values, or null
  int ablation;      // 0 full operator; 1 K = (W_L + C) / h^deriv (no W_P, no projection); 2 face values = O_F only
  int stage;
  int flow;          // 0 Burgers, 1 Navier-Stokes
  int forcing;
  int dord;          // physics derivative order 2 or 4
  float dt, nu, idx, idy, drag, inv_nn;
  const float2* tw;  // [N/2]
  const float* symx; // [N/2 + 1]
  const float* symy; // [N]
  const float* frc;  // [N]
};

// instance table: field, axis (0 x, 1 y), kind (0 interp, 1 deriv), shift
__device__ __constant__ int kInstField[8] = {0, 0, 0, 0, 1, 1, 1, 1};
__device__ __constant__ int kInstAxis[8] = {0, 0, 1, 1, 0, 0, 1, 1};
__device__ __constant__ int kInstKind[8] = {0, 1, 0, 1, 0, 1, 0, 1};
__device__ __constant__ int kInstShift[8] = {-1, -1, -2, -2, -2, -2, -1, -1};

template <int LOGN>
struct LearnedCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int NT = N >= 64 ? 512 : (N >= 32 ? 256 : 128);
  static constexpr int HSTR = N / 2 + 1;
  static constexpr int COLLEN = N + 1;
  static constexpr size_t W_BYTES = (size_t)2 * N * N * 4;
  static constexpr size_t SCR_BYTES = align16(cmax((size_t)N * HSTR * 8, (size_t)(N / 2) * COLLEN * 8));
  static constexpr size_t OFF_SCR = W_BYTES;
  static constexpr size_t OFF_TW = OFF_SCR + SCR_BYTES;
  static constexpr size_t OFF_SX = OFF_TW + (N / 2) * 8;
  static constexpr size_t OFF_SY = OFF_SX + align16((N / 2 + 2) * 4);
  static constexpr size_t OFF_FRC = OFF_SY + N * 4;
  static constexpr size_t SMEM = OFF_FRC + N * 4;
  static_assert(SMEM <= 232448, "one trajectory's state and spectrum scratch in shared memory");
};

// Spectral projection of a trajectory tile wt[2][N][N] in shared memory
// (CS = 1): w -= G2 L^{-1} D2 w with the symbol of D2 G2, zero mode removed.
template <int LOGN, int NT>
__device__ void project_tile(float* wt, unsigned char* scr, const float2* tw, const float* sx, const float* sy,
                             float idx, float idy, float inv_nn) {
  using CT = float2;
  using FFT = WarpFFT<float, LOGN>;
  constexpr int N = 1 << LOGN, HALF = N / 2, HSTR = HALF + 1, COLLEN = N + 1, MSK = N - 1;
  constexpr int W = FFT::W, E = FFT::E, TPW = 32 / W, NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = lane & (W - 1), gbase = lane & ~(W - 1);
  CT* const hs = reinterpret_cast<CT*>(scr);
  CT* const col = reinterpret_cast<CT*>(scr);
  float* const pr = reinterpret_cast<float*>(scr);
  const float* fu = wt;
  const float* fv = wt + N * N;
  // divergence -> forward row FFTs -> half spectra
  for (int t0 = warp * TPW; t0 < N / 2; t0 += NW * TPW) {
    const int jp = t0 + lane / W;
    const bool act = jp < N / 2;
    const int ja = act ? 2 * jp : 0;
    CT z[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int x = q + W * m;
      const int jb = ja + 1, jc = (ja + 2) & MSK;
      const float da = (fu[ja * N + ((x + 1) & MSK)] - fu[ja * N + x]) * idx + (fv[jb * N + x] - fv[ja * N + x]) * idy;
      const float db = (fu[jb * N + ((x + 1) & MSK)] - fu[jb * N + x]) * idx + (fv[jc * N + x] - fv[jb * N + x]) * idy;
      z[m] = CT{da, db};
    }
    FFT::dif(z, q, tw);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = brev<LOGN>(q + W * m);
      const int pl = (k == 0) ? 1 : FFT::partner_lane(q, m);
      const CT zm = shfl_idx(z[FFT::partner_reg(m)], gbase + pl);
      const CT zk = z[m];
      CT A, B;
      if (k == 0) {
        A = CT{zk.x, zm.x};
        B = CT{zk.y, zm.y};
      } else {
        A = CT{0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y)};
        B = CT{0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x)};
      }
      const CT Bo = shfl_up1(B);
      const int s = (q + W * m) >> 1;
      if (act) {
        if ((q & 1) == 0)
          hs[ja * HSTR + s] = A;
        else
          hs[(ja + 1) * HSTR + s] = Bo;
      }
    }
  }
  __syncthreads();
  // transpose rows -> columns in place (through registers)
  {
    constexpr int NR = (HALF * N + NT - 1) / NT;
    CT reg[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int e = tid + k * NT;
      if (e < HALF * N) reg[k] = hs[(e / HALF) * HSTR + (e % HALF)];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int e = tid + k * NT;
      if (e < HALF * N) col[(e % HALF) * COLLEN + e / HALF] = reg[k];
    }
  }
  __syncthreads();
  // column FFTs, spectral multiply, inverse column FFTs
  for (int t0 = warp * TPW; t0 < HALF; t0 += NW * TPW) {
    const int sl = t0 + lane / W;
    const bool act = sl < HALF;
    const int sg = act ? sl : 0;
    const int kx = brev<LOGN - 1>(sg);
    CT z[E];
#pragma unroll
    for (int m = 0; m < E; ++m) z[m] = col[sg * COLLEN + q + W * m];
    FFT::dif(z, q, tw);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int mp = FFT::partner_reg(m);
      if (mp < m) continue;
      const int ky = brev<LOGN>(q + W * m);
      const int kyp = brev<LOGN>(q + W * mp);
      const CT za = z[m], zb = z[mp];
      const CT pa = shfl_idx(zb, gbase + FFT::partner_lane(q, m));
      const CT pb = shfl_idx(za, gbase + FFT::partner_lane(q, mp));
      if (sg != 0) {
        const float ma = __fdividef(inv_nn, sx[kx] + sy[ky]);
        const float mb = __fdividef(inv_nn, sx[kx] + sy[kyp]);
        z[m] = CT{za.x * ma, za.y * ma};
        if (mp != m) z[mp] = CT{zb.x * mb, zb.y * mb};
      } else {
        {
          const float m0 = ky == 0 ? 0.f : __fdividef(inv_nn, sx[0] + sy[ky]);
          const float mn = __fdividef(inv_nn, sx[HALF] + sy[ky]);
          const float hp = 0.5f * (m0 + mn), hm = 0.5f * (m0 - mn);
          z[m] = CT{hp * za.x + hm * pa.x, hp * za.y - hm * pa.y};
        }
        if (mp != m) {
          const float m0 = kyp == 0 ? 0.f : __fdividef(inv_nn, sx[0] + sy[kyp]);
          const float mn = __fdividef(inv_nn, sx[HALF] + sy[kyp]);
          const float hp = 0.5f * (m0 + mn), hm = 0.5f * (m0 - mn);
          z[mp] = CT{hp * zb.x + hm * pb.x, hp * zb.y - hm * pb.y};
        }
      }
    }
    FFT::dit_inv(z, q, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) col[sg * COLLEN + q + W * m] = z[m];
    }
  }
  __syncthreads();
  // transpose back
  {
    constexpr int NR = (HALF * N + NT - 1) / NT;
    CT reg[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int e = tid + k * NT;
      if (e < HALF * N) reg[k] = col[(e / N) * COLLEN + (e % N)];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int e = tid + k * NT;
      if (e < HALF * N) hs[(e % N) * HSTR + e / N] = reg[k];
    }
  }
  __syncthreads();
  // inverse row FFTs -> pressure rows (same bytes as the half-spectrum rows)
  for (int t0 = warp * TPW; t0 < N / 2; t0 += NW * TPW) {
    const int jp = t0 + lane / W;
    const bool act = jp < N / 2;
    const int ra = act ? 2 * jp : 0;
    CT z[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int p = q + W * m;
      const int k = brev<LOGN>(p);
      if (k < HALF) {
        const CT A = hs[ra * HSTR + (p >> 1)];
        const CT B = hs[(ra + 1) * HSTR + (p >> 1)];
        z[m] = (k == 0) ? CT{A.x, B.x} : CT{A.x - B.y, A.y + B.x};
      } else {
        const int kp = N - k;
        const int sp = brev<LOGN>(kp & MSK) >> 1;
        const CT A = hs[ra * HSTR + sp];
        const CT B = hs[(ra + 1) * HSTR + sp];
        z[m] = (kp == HALF) ? CT{A.y, B.y} : CT{A.x + B.y, B.x - A.y};
      }
    }
    FFT::dit_inv(z, q, tw);
    __syncwarp();
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int x = q + W * m;
        pr[ra * (2 * HSTR) + x] = z[m].x;
        pr[(ra + 1) * (2 * HSTR) + x] = z[m].y;
      }
    }
  }
  __syncthreads();
  // w -= G2 p
  for (int c = tid; c < N * N; c += NT) {
    const int j = c / N, i = c % N;
    const float pc = pr[j * (2 * HSTR) + i];
    const float pw = pr[j * (2 * HSTR) + ((i - 1) & MSK)];
    const float ps = pr[((j - 1) & MSK) * (2 * HSTR) + i];
    wt[c] -= (pc - pw) * idx;
    wt[N * N + c] -= (pc - ps) * idy;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Banded variant of one learned stage: the flux block, flux assembly and RK
// combination of RB rows of one trajectory per CTA (grid N/RB x batch, 256
// threads), writing the unprojected stage result w*; fv_project_kernel then
// projects each trajectory. Splitting the trajectory over N/RB CTAs hides the
// latency of the network-output loads that bound the one-CTA-per-trajectory
// kernel at small batch.
// ---------------------------------------------------------------------------
template <int LOGN, int RB>
struct BandCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int NT = 256;
  static constexpr int TR = RB + 6;  // tile rows j0 - 3 .. j0 + RB + 2
  static constexpr int FR = RB + 2;  // face rows j0 - 1 .. j0 + RB
  static constexpr size_t SMEM = (size_t)2 * TR * N * 4 + (size_t)8 * FR * N * 4;
};

template <int LOGN, int RB>
__global__ void __launch_bounds__(256, 4) fv_learned_flux_kernel(const LStageArgs a) {
  using Cfg = BandCfg<LOGN, RB>;
  constexpr int N = Cfg::N, NT = Cfg::NT, MSK = N - 1, TR = Cfg::TR, FR = Cfg::FR;
  extern __shared__ __align__(16) float bsm[];
  float* const wt = bsm;                 // [2][TR][N]
  float* const inst = bsm + 2 * TR * N;  // [8][FR][N]
  __shared__ float swl[80];
  const int tid = threadIdx.x;
  const int b = blockIdx.y, j0 = blockIdx.x * RB;
  const size_t NN = (size_t)N * N;
  const float* w = a.w + (size_t)b * 2 * NN;
  pdl_wait();
  pdl_trigger();
  for (int k = tid; k < 2 * TR * N; k += NT) {
    const int f = k / (TR * N), rem = k - f * TR * N;
    const int tr = rem >> LOGN, i = rem & MSK;
    wt[k] = w[(size_t)f * NN + (size_t)((j0 - 3 + tr) & MSK) * N + i];
  }
  if (tid < 80) swl[tid] = a.wl[tid];
  __syncthreads();
  const float cval[4] = {-1.5f, -0.5f, 0.5f, 1.5f};
  const uint4* cbase = a.coef ? reinterpret_cast<const uint4*>(a.coef) + (size_t)b * 20 * NN : nullptr;
  // face values of rows j0 - 1 .. j0 + RB
  for (int fc = tid; fc < FR * N; fc += NT) {
    const int fr = fc >> LOGN, i = fc & MSK;
    const int j = (j0 - 1 + fr) & MSK;
    const int c = j * N + i;
#pragma unroll 1
    for (int pr_ = 0; pr_ < 4; ++pr_) {
      const int fld = pr_ >> 1, axis = pr_ & 1;
      const int sh = (pr_ == 0 || pr_ == 3) ? -1 : -2;
      const float* f = wt + fld * TR * N;
      float tap[20];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          int tr, ii;
          if (axis == 0) {
            tr = fr + r;  // tile row of j + r - 2
            ii = (i + cc + sh) & MSK;
          } else {
            tr = fr + 2 + cc + sh;
            ii = (i + r - 2) & MSK;
          }
          tap[r * 4 + cc] = f[tr * N + ii];
        }
      const float h = axis == 0 ? 1.0f / a.idx : 1.0f / a.idy;
#pragma unroll
      for (int kind = 0; kind < 2; ++kind) {
        const int qi = 2 * pr_ + kind;
        if (a.ablation == 2) {  // frequency-domain operator only
          inst[(qi * FR + fr) * N + i] = a.fno[((size_t)b * 8 + qi) * NN + c];
          continue;
        }
        float L[20];
#pragma unroll
        for (int t = 0; t < 20; ++t) L[t] = swl[(kind * 2 + axis) * 20 + t];
        if (cbase) {
          const int k0 = (20 * qi) >> 3;
          float fch[24];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const uint4 v = cbase[(size_t)(k0 + k) * NN + c];
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[e]));
              fch[k * 8 + 2 * e] = f2.x;
              fch[k * 8 + 2 * e + 1] = f2.y;
            }
          }
          if (kind == 0) {
#pragma unroll
            for (int t = 0; t < 20; ++t) L[t] += fch[t];
          } else {
#pragma unroll
            for (int t = 0; t < 20; ++t) L[t] += fch[4 + t];
          }
        }
        float s1 = 0.f, sc = 0.f, sr = 0.f;
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const float v = L[r * 4 + cc];
            s1 += v;
            sc += v * cval[cc];
            sr += v * (float)(r - 2);
          }
        // the projection keeps W_P's consistency: without W_P (ablation 1) neither is applied
        const float pk = a.ablation == 0 ? 1.0f : 0.0f;
        s1 *= pk * (1.0f / 20.0f);
        sc *= pk * (1.0f / 25.0f);
        sr *= pk * (1.0f / 40.0f);
        const float scale = kind == 1 ? 1.0f / h : 1.0f;
        float val = 0.f;
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            float k = (L[r * 4 + cc] - s1 - sc * cval[cc] - sr * (float)(r - 2)) * scale;
            if (r == 2 && a.ablation == 0) {
              if (kind == 0) {
                k += (cc == 1 || cc == 2) ? 0.5f : 0.f;
              } else if (a.dord == 4) {
                const float d4[4] = {1.f / 24.f, -27.f / 24.f, 27.f / 24.f, -1.f / 24.f};
                k += d4[cc] / h;
              } else {
                const float d2[4] = {0.f, -1.f, 1.f, 0.f};
                k += d2[cc] / h;
              }
            }
            val += k * tap[r * 4 + cc];
          }
        if (a.fno) val += a.fno[((size_t)b * 8 + qi) * NN + c];
        inst[(qi * FR + fr) * N + i] = val;
      }
    }
  }
  __syncthreads();
  // flux assembly and RK combination of rows j0 .. j0 + RB - 1 (face row = row - j0 + 1)
  const float ca = a.stage == 2 ? a.dt : 0.5f * a.dt;
  const float c6 = a.dt / 6.0f;
  auto I_ = [&](int q, int fr, int i) { return inst[(q * FR + fr) * N + (i & MSK)]; };
  for (int k = tid; k < RB * N; k += NT) {
    const int rr = k >> LOGN, i = k & MSK;
    const int fr = rr + 1, j = j0 + rr;
    const float Uc = I_(0, fr, i), Ucw = I_(0, fr, i - 1);
    const float Gxc = I_(1, fr, i), Gxcw = I_(1, fr, i - 1);
    const float Uk = I_(2, fr, i), Ukn = I_(2, fr + 1, i), Uke = I_(2, fr, i + 1);
    const float Gyu = I_(3, fr, i), Gyun = I_(3, fr + 1, i);
    const float Vk = I_(4, fr, i), Vkn = I_(4, fr + 1, i), Vke = I_(4, fr, i + 1);
    const float Gxv = I_(5, fr, i), Gxve = I_(5, fr, i + 1);
    const float Vc = I_(6, fr, i), Vcs = I_(6, fr - 1, i);
    const float Gyc = I_(7, fr, i), Gycs = I_(7, fr - 1, i);
    float tu = -(Uc * Uc - Ucw * Ucw) * a.idx - (Ukn * Vkn - Uk * Vk) * a.idy +
               a.nu * ((Gxc - Gxcw) * a.idx + (Gyun - Gyu) * a.idy);
    float tv = -(Uke * Vke - Uk * Vk) * a.idx - (Vc * Vc - Vcs * Vcs) * a.idy +
               a.nu * ((Gxve - Gxv) * a.idx + (Gyc - Gycs) * a.idy);
    const float uc = wt[(rr + 3) * N + i], vc = wt[TR * N + (rr + 3) * N + i];
    if (a.flow == 0) {
      const float d0 = Gxc + Gyc;
      tu += uc * 0.5f * ((Gxcw + I_(7, fr, i - 1)) + d0);
      tv += vc * 0.5f * ((I_(1, fr - 1, i) + Gycs) + d0);
    }
    if (a.forcing == 1) {
      tu += a.frc[j] - a.drag * uc;
      tv += -a.drag * vc;
    }
    const size_t g = (size_t)b * 2 * NN + (size_t)j * N + i;
    float* acc = a.acc;
    float au, av;
    if (a.stage == 0) {
      au = tu;
      av = tv;
    } else {
      au = acc[g] + (a.stage < 3 ? 2.0f : 1.0f) * tu;
      av = acc[g + NN] + (a.stage < 3 ? 2.0f : 1.0f) * tv;
    }
    if (a.stage < 3) {
      acc[g] = au;
      acc[g + NN] = av;
      a.wout[g] = a.un[g] + ca * tu;
      a.wout[g + NN] = a.un[g + NN] + ca * tv;
    } else {
      a.wout[g] = a.un[g] + c6 * au;
      a.wout[g + NN] = a.un[g + NN] + c6 * av;
    }
  }
}

// w <- P(w*) for each trajectory (one CTA per trajectory, projection in shared memory;
// a plain copy for Burgers)
template <int LOGN>
__global__ void __launch_bounds__(LearnedCfg<LOGN>::NT, 1) fv_project_kernel(const LStageArgs a) {
  using Cfg = LearnedCfg<LOGN>;
  constexpr int N = Cfg::N, NT = Cfg::NT;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* const wt = reinterpret_cast<float*>(smem);
  unsigned char* const scr = smem + Cfg::OFF_SCR;
  float2* const tw = reinterpret_cast<float2*>(smem + Cfg::OFF_TW);
  float* const sx = reinterpret_cast<float*>(smem + Cfg::OFF_SX);
  float* const sy = reinterpret_cast<float*>(smem + Cfg::OFF_SY);
  const int tid = threadIdx.x;
  const size_t NN = (size_t)N * N;
  const float* src = a.w + (size_t)blockIdx.x * 2 * NN;
  float* dst = a.wout + (size_t)blockIdx.x * 2 * NN;
  for (int k = tid; k < N / 2; k += NT) tw[k] = a.tw[k];
  for (int k = tid; k <= N / 2; k += NT) sx[k] = a.symx[k];
  for (int k = tid; k < N; k += NT) sy[k] = a.symy[k];
  pdl_wait();
  pdl_trigger();
  for (int c = tid; c < 2 * N * N; c += NT) wt[c] = src[c];
  __syncthreads();
  if (a.flow == 1) project_tile<LOGN, NT>(wt, scr, tw, sx, sy, a.idx, a.idy, a.inv_nn);  // Burgers: a copy
  for (int c = tid; c < 2 * N * N; c += NT) dst[c] = wt[c];
}

// Temporal correction (Sec. 3.2, Sec. 3.5): u <- P(u + c - mean(c)) for each
// trajectory, with the correction c from the temporal-correction network.
template <int LOGN>
__global__ void __launch_bounds__(LearnedCfg<LOGN>::NT, 1) fv_correct_project_kernel(const LStageArgs a) {
  using Cfg = LearnedCfg<LOGN>;
  constexpr int N = Cfg::N, NT = Cfg::NT;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* const wt = reinterpret_cast<float*>(smem);
  unsigned char* const scr = smem + Cfg::OFF_SCR;  // the instance-array region is not used
  float2* const tw = reinterpret_cast<float2*>(smem + Cfg::OFF_TW);
  float* const sx = reinterpret_cast<float*>(smem + Cfg::OFF_SX);
  float* const sy = reinterpret_cast<float*>(smem + Cfg::OFF_SY);
  __shared__ float red[2][32];
  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  const size_t NN = (size_t)N * N;
  const float* corr = a.corr + (size_t)b * 2 * NN;
  float* u = a.wout + (size_t)b * 2 * NN;
  for (int k = tid; k < N / 2; k += NT) tw[k] = a.tw[k];
  for (int k = tid; k <= N / 2; k += NT) sx[k] = a.symx[k];
  for (int k = tid; k < N; k += NT) sy[k] = a.symy[k];
  pdl_wait();
  pdl_trigger();
  // per-component mean of the correction
  float s0 = 0.f, s1 = 0.f;
  for (int c = tid; c < N * N; c += NT) {
    s0 += corr[c];
    s1 += corr[NN + c];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = s0;
    red[1][tid >> 5] = s1;
  }
  __syncthreads();
  float m0 = 0.f, m1 = 0.f;
  for (int k = 0; k < NT / 32; ++k) {
    m0 += red[0][k];
    m1 += red[1][k];
  }
  m0 /= (float)NN;
  m1 /= (float)NN;
  for (int c = tid; c < N * N; c += NT) {
    wt[c] = u[c] + (corr[c] - m0);
    wt[NN + c] = u[NN + c] + (corr[NN + c] - m1);
  }
  __syncthreads();
  if (a.flow == 1) project_tile<LOGN, NT>(wt, scr, tw, sx, sy, a.idx, a.idy, a.inv_nn);
  for (int c = tid; c < 2 * N * N; c += NT) u[c] = wt[c];
}

}  // namespace ldfv
