// fv_adjoint.cuh -- reverse mode of one FV stage (flux block, flux assembly,
// direct terms) and of the projection / RK4 combination, one CTA per
// trajectory (N <= 64), FP32.
//
// The forward tendency H(w) (Sec. 3.4 face operators with per-face kernels
// K = W_P + proj(W_L + C_theta(w)) / h^(deriv), App. B.2 flux assembly, Eq. 1
// source terms) is differentiated line by line:
//   * a periodic shift transposes to the opposite shift;
//   * a face value v = sum_rc K[r][c] f[tap(r, c)] gives f_bar[tap] += K v_bar
//     (scattered with shared-memory atomics) and K_bar[r][c] = v_bar f[tap];
//   * the consistency projection is an orthogonal projector (self-adjoint),
//     so the network-output cotangent is C_bar = proj(K_bar) / h^(deriv), and
//     W_L_bar sums the same quantity over the faces;
//   * the products of the flux assembly give the usual product rule.
// The network part of the state cotangent (through C_theta(w)) is added by the
// network's reverse pass; this kernel gives the part with the kernels fixed.
#pragma once

#include <cuda_bf16.h>

#include "fv_common.cuh"
#include "fv_learned.cuh"

namespace ldfv {

struct AdjStageArgs {
  const float* w;              // stage state [batch][2][N][N]
  const float* tbar;           // tendency cotangent [batch][2][N][N]
  const __nv_bfloat16* coef;   // network output at w, [batch][20][N][N][8], or null (plain kernels)
  const float* wl;             // W_L [kind 2][axis 2][5][4] (learned) or null
  float* wbar;                 // out: [batch][2][N][N] (overwritten)
  __nv_bfloat16* cbar;         // out: C_bar as chunk planes [batch][20][N][N][8], or null
  float* cbar_f32;             // out: C_bar as [batch][160][N][N] FP32, or null
  float* wl_bar;               // out: W_L_bar [80], accumulated with atomics, or null
  int flow, forcing, dord;
  float nu, idx, idy, drag;
};

template <int LOGN>
struct AdjCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int NT = N >= 64 ? 512 : 256;
  static constexpr size_t F_BYTES = (size_t)2 * N * N * 4;
  static constexpr size_t OFF_TB = F_BYTES;
  static constexpr size_t OFF_I = 2 * F_BYTES;             // six face-value arrays
  static constexpr size_t OFF_WB = OFF_I + (size_t)6 * N * N * 4;
  static constexpr size_t SMEM = OFF_WB + F_BYTES;
  static_assert(SMEM <= 232448 - 1024, "shared memory");
};

// Per-face kernel of instance qi (axis, kind) at cell c: K[20] (5 x 4, row-major).
__device__ __forceinline__ void adj_kernel_at(int qi, int axis, int kind, const float* swl, const uint4* cbase,
                                              size_t NN, int c, int dord, float h, float (&K)[20]) {
  const float cval[4] = {-1.5f, -0.5f, 0.5f, 1.5f};
  float L[20];
#pragma unroll
  for (int t = 0; t < 20; ++t) L[t] = swl ? swl[(kind * 2 + axis) * 20 + t] : 0.f;
  if (cbase) {
    // channels 20 qi .. 20 qi + 19: three 8-channel chunks from (20 qi) / 8, offset 0 or 4
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
    if (qi & 1) {
#pragma unroll
      for (int t = 0; t < 20; ++t) L[t] += fch[4 + t];
    } else {
#pragma unroll
      for (int t = 0; t < 20; ++t) L[t] += fch[t];
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
  s1 *= (1.0f / 20.0f);
  sc *= (1.0f / 25.0f);
  sr *= (1.0f / 40.0f);
  const float scale = kind == 1 ? 1.0f / h : 1.0f;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      float k = (L[r * 4 + cc] - s1 - sc * cval[cc] - sr * (float)(r - 2)) * scale;
      if (r == 2) {
        if (kind == 0) {
          k += (cc == 1 || cc == 2) ? 0.5f : 0.f;
        } else if (dord == 4) {
          const float d4[4] = {1.f / 24.f, -27.f / 24.f, 27.f / 24.f, -1.f / 24.f};
          k += d4[cc] / h;
        } else {
          const float d2[4] = {0.f, -1.f, 1.f, 0.f};
          k += d2[cc] / h;
        }
      }
      K[r * 4 + cc] = k;
    }
}

// flat index of tap (r, c) of an instance along `axis` with axial shift `sh` at cell (j, i)
template <int N>
__device__ __forceinline__ int adj_tap(int axis, int sh, int j, int i, int r, int cc) {
  constexpr int MSK = N - 1;
  return axis == 0 ? ((j + r - 2) & MSK) * N + ((i + cc + sh) & MSK) : ((j + cc + sh) & MSK) * N + ((i + r - 2) & MSK);
}

template <int LOGN>
__global__ void __launch_bounds__(AdjCfg<LOGN>::NT, 1) fv_adjoint_stage_kernel(const AdjStageArgs a) {
  using Cfg = AdjCfg<LOGN>;
  constexpr int N = Cfg::N, NT = Cfg::NT, MSK = N - 1;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* const wt = reinterpret_cast<float*>(smem);
  float* const tb = reinterpret_cast<float*>(smem + Cfg::OFF_TB);
  float* const inst = reinterpret_cast<float*>(smem + Cfg::OFF_I);
  float* const wb = reinterpret_cast<float*>(smem + Cfg::OFF_WB);
  __shared__ float swl[80];
  __shared__ float swlb[80];
  const int tid = threadIdx.x, lane = tid & 31;
  const int b = blockIdx.x;
  for (size_t c = tid; c < 2 * NN; c += NT) {
    wt[c] = a.w[(size_t)b * 2 * NN + c];
    tb[c] = a.tbar[(size_t)b * 2 * NN + c];
  }
  if (tid < 80) {
    swl[tid] = a.wl ? a.wl[tid] : 0.f;
    swlb[tid] = 0.f;
  }
  __syncthreads();
  const float* swlp = a.wl ? swl : nullptr;
  const uint4* cbase = a.coef ? reinterpret_cast<const uint4*>(a.coef) + (size_t)b * 20 * NN : nullptr;
  const float hx = 1.0f / a.idx, hy = 1.0f / a.idy;
  const bool burgers = a.flow == 0;

  // ---- forward face values needed by the reverse pass --------------------------------
  // slots: 0 Uc (q0), 1 Uk (q2), 2 Vk (q4), 3 Vc (q6), 4 Gxc (q1), 5 Gyc (q7)
  const int nslot = burgers ? 6 : 4;
  for (int c = tid; c < (int)NN; c += NT) {
    const int j = c / N, i = c % N;
#pragma unroll 1
    for (int sl = 0; sl < nslot; ++sl) {
      const int qi = sl < 4 ? 2 * sl : (sl == 4 ? 1 : 7);
      const int pr_ = qi >> 1, fld = pr_ >> 1, axis = pr_ & 1, kind = qi & 1;
      const int sh = (pr_ == 0 || pr_ == 3) ? -1 : -2;
      float K[20];
      adj_kernel_at(qi, axis, kind, swlp, cbase, NN, c, a.dord, axis == 0 ? hx : hy, K);
      float v = 0.f;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) v += K[r * 4 + cc] * wt[fld * NN + adj_tap<N>(axis, sh, j, i, r, cc)];
      inst[sl * NN + c] = v;
    }
  }
  __syncthreads();
  const float* Uc = inst + 0 * NN;
  const float* Uk = inst + 1 * NN;
  const float* Vk = inst + 2 * NN;
  const float* Vc = inst + 3 * NN;
  const float* Gxc = inst + 4 * NN;
  const float* Gyc = inst + 5 * NN;
  const float* Tu = tb;
  const float* Tv = tb + NN;

  // ---- direct terms (Burgers advective correction, linear drag) -------------------
  for (int c = tid; c < (int)NN; c += NT) {
    const int j = c / N, i = c % N;
    float du = 0.f, dv = 0.f;
    if (burgers) {
      const int cw = j * N + ((i - 1) & MSK), cs = ((j - 1) & MSK) * N + i;
      const float d0 = Gxc[c] + Gyc[c];
      du += Tu[c] * 0.5f * ((Gxc[cw] + Gyc[cw]) + d0);
      dv += Tv[c] * 0.5f * ((Gxc[cs] + Gyc[cs]) + d0);
    }
    if (a.forcing == 1) {
      du -= a.drag * Tu[c];
      dv -= a.drag * Tv[c];
    }
    wb[c] = du;
    wb[NN + c] = dv;
  }
  __syncthreads();

  // ---- reverse through the eight face operators ------------------------------------
  const float cval[4] = {-1.5f, -0.5f, 0.5f, 1.5f};
#pragma unroll 1
  for (int qi = 0; qi < 8; ++qi) {
    const int pr_ = qi >> 1, fld = pr_ >> 1, axis = pr_ & 1, kind = qi & 1;
    const int sh = (pr_ == 0 || pr_ == 3) ? -1 : -2;
    const float h = axis == 0 ? hx : hy;
    const float scale = kind == 1 ? 1.0f / h : 1.0f;
    float lsum[20];
#pragma unroll
    for (int t = 0; t < 20; ++t) lsum[t] = 0.f;
    for (int c = tid; c < (int)NN; c += NT) {
      const int j = c / N, i = c % N;
      const int ce = j * N + ((i + 1) & MSK), cw = j * N + ((i - 1) & MSK);
      const int cn = ((j + 1) & MSK) * N + i, cs = ((j - 1) & MSK) * N + i;
      // cotangent of this face value (product rule of the flux assembly)
      float vb;
      switch (qi) {
        case 0: vb = 2.0f * Uc[c] * (Tu[ce] - Tu[c]) * a.idx; break;
        case 1: vb = a.nu * (Tu[c] - Tu[ce]) * a.idx; break;
        case 2: vb = ((Tu[c] - Tu[cs]) * a.idy + (Tv[c] - Tv[cw]) * a.idx) * Vk[c]; break;
        case 3: vb = a.nu * (Tu[cs] - Tu[c]) * a.idy; break;
        case 4: vb = ((Tu[c] - Tu[cs]) * a.idy + (Tv[c] - Tv[cw]) * a.idx) * Uk[c]; break;
        case 5: vb = a.nu * (Tv[cw] - Tv[c]) * a.idx; break;
        case 6: vb = 2.0f * Vc[c] * (Tv[cn] - Tv[c]) * a.idy; break;
        default: vb = a.nu * (Tv[c] - Tv[cn]) * a.idy; break;
      }
      if (burgers && (qi == 1 || qi == 7))
        vb += 0.5f * (Tu[c] * wt[c] + Tu[ce] * wt[ce]) + 0.5f * (Tv[c] * wt[NN + c] + Tv[cn] * wt[NN + cn]);
      float K[20];
      adj_kernel_at(qi, axis, kind, swlp, cbase, NN, c, a.dord, h, K);
      float Kb[20];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int t = adj_tap<N>(axis, sh, j, i, r, cc);
          atomicAdd(&wb[fld * NN + t], K[r * 4 + cc] * vb);
          Kb[r * 4 + cc] = vb * wt[fld * NN + t];
        }
      // C_bar = proj(K_bar) * scale (the projector is symmetric)
      float s1 = 0.f, sc = 0.f, sr = 0.f;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float v = Kb[r * 4 + cc];
          s1 += v;
          sc += v * cval[cc];
          sr += v * (float)(r - 2);
        }
      s1 *= (1.0f / 20.0f);
      sc *= (1.0f / 25.0f);
      sr *= (1.0f / 40.0f);
      float lb[20];
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          lb[r * 4 + cc] = (Kb[r * 4 + cc] - s1 - sc * cval[cc] - sr * (float)(r - 2)) * scale;
          lsum[r * 4 + cc] += lb[r * 4 + cc];
        }
      if (a.cbar_f32) {
#pragma unroll
        for (int t = 0; t < 20; ++t) a.cbar_f32[((size_t)b * 160 + qi * 20 + t) * NN + c] = lb[t];
      }
      if (a.cbar) {
        // channels 20 qi + t: even qi -> chunks k0, k0+1 and the low half of k0+2;
        // odd qi -> the high half of k0, then k0+1 and k0+2 (8-byte halves do not overlap)
        uint32_t pk[10];
#pragma unroll
        for (int e = 0; e < 10; ++e) {
          __nv_bfloat162 h2 = __floats2bfloat162_rn(lb[2 * e], lb[2 * e + 1]);
          pk[e] = *reinterpret_cast<uint32_t*>(&h2);
        }
        const int k0 = (20 * qi) >> 3;
        __nv_bfloat16* base = a.cbar + ((size_t)b * 20 * NN + c) * 8;
        if ((qi & 1) == 0) {
          *reinterpret_cast<uint4*>(base + (size_t)k0 * NN * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(base + (size_t)(k0 + 1) * NN * 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          *reinterpret_cast<uint2*>(base + (size_t)(k0 + 2) * NN * 8) = make_uint2(pk[8], pk[9]);
        } else {
          *reinterpret_cast<uint2*>(base + (size_t)k0 * NN * 8 + 4) = make_uint2(pk[0], pk[1]);
          *reinterpret_cast<uint4*>(base + (size_t)(k0 + 1) * NN * 8) = make_uint4(pk[2], pk[3], pk[4], pk[5]);
          *reinterpret_cast<uint4*>(base + (size_t)(k0 + 2) * NN * 8) = make_uint4(pk[6], pk[7], pk[8], pk[9]);
        }
      }
    }
    if (a.wl_bar) {
      // W_L_bar[kind][axis] gathers the learned-part cotangent of both fields
#pragma unroll
      for (int t = 0; t < 20; ++t) {
        float v = lsum[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&swlb[(kind * 2 + axis) * 20 + t], v);
      }
    }
  }
  __syncthreads();
  for (size_t c = tid; c < 2 * NN; c += NT) a.wbar[(size_t)b * 2 * NN + c] = wb[c];
  if (a.wl_bar && tid < 80) atomicAdd(&a.wl_bar[tid], swlb[tid]);
}

// Reverse-mode combination of the RK4 stages (one CTA per trajectory):
//   y = P(in0 + in1)           (P = identity for Burgers or when project == 0)
//   init:  g = y, lam = y      otherwise: lam += y
//   rb = alpha g + beta y      (when rb is non-null)
// The projection is symmetric, so it is its own adjoint.
struct AdjCombineArgs {
  const float* in0;   // [batch][2][N][N]
  const float* in1;   // optional second addend (network part), or null
  float* g;           // P(lam_out), written when init
  float* lam;         // accumulated state cotangent
  float* rb;          // next stage's tendency cotangent, or null
  float alpha, beta;
  int init, project;
  float idx, idy, inv_nn;
  const float2* tw;
  const float* symx;
  const float* symy;
};

template <int LOGN>
__global__ void __launch_bounds__(LearnedCfg<LOGN>::NT, 1) fv_adjoint_combine_kernel(const AdjCombineArgs a) {
  using Cfg = LearnedCfg<LOGN>;
  constexpr int N = Cfg::N, NT = Cfg::NT;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* const wt = reinterpret_cast<float*>(smem);
  unsigned char* const scr = smem + Cfg::OFF_SCR;
  float2* const tw = reinterpret_cast<float2*>(smem + Cfg::OFF_TW);
  float* const sx = reinterpret_cast<float*>(smem + Cfg::OFF_SX);
  float* const sy = reinterpret_cast<float*>(smem + Cfg::OFF_SY);
  const int tid = threadIdx.x;
  const size_t off = (size_t)blockIdx.x * 2 * NN;
  for (int k = tid; k < N / 2; k += NT) tw[k] = a.tw[k];
  for (int k = tid; k <= N / 2; k += NT) sx[k] = a.symx[k];
  for (int k = tid; k < N; k += NT) sy[k] = a.symy[k];
  for (size_t c = tid; c < 2 * NN; c += NT) wt[c] = a.in0[off + c] + (a.in1 ? a.in1[off + c] : 0.f);
  __syncthreads();
  if (a.project) project_tile<LOGN, NT>(wt, scr, tw, sx, sy, a.idx, a.idy, a.inv_nn);
  for (size_t c = tid; c < 2 * NN; c += NT) {
    const float y = wt[c];
    float gv;
    if (a.init) {
      a.g[off + c] = y;
      a.lam[off + c] = y;
      gv = y;
    } else {
      a.lam[off + c] += y;
      gv = a.g[off + c];
    }
    if (a.rb) a.rb[off + c] = a.alpha * gv + a.beta * y;
  }
}

}  // namespace ldfv
