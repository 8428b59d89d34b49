// fd_gadjoint.cu -- reverse mode on the generic-grid path (FP32): the
// vector-Jacobian product of one RK4 step of the plain or learned solver on any
// grid that path takes, and of the temporal correction. The paper trains its
// models through unrolled rollouts of the differentiable solver (Sec. 3.2,
// Sec. 4 "Model Training"); this is the transpose of every forward operation:
//
//   * RK4 (App. B.5): u' = P(u + dt/6 (r_0 + 2 r_1 + 2 r_2 + r_3)), r_s = H(w_s),
//     w_0 = u, w_1 = P(u + dt/2 r_0), w_2 = P(u + dt/2 r_1), w_3 = P(u + dt r_2):
//     the stage states are recomputed, then the stages run backwards, the
//     projection being its own transpose (Sec. 3.6, P symmetric);
//   * the flux assembly (App. B.2): the face-value cotangents follow from the
//     tendency cotangent by the transposed flux differences and products, plus
//     the Burgers correction's and the drag's direct terms;
//   * the face operators (Sec. 3.4): the state cotangent gathers K_f^T vbar_f
//     over the faces whose taps reach a cell; the per-face kernel cotangent is
//     vbar_f times the taps, which passes through the consistency projection
//     (an orthogonal projector, so its own transpose) and the 1/h of the
//     derivative instances to the network output and W_L;
//   * the network (six periodic 3x3 convolutions, GELU between them): the data
//     gradient is the transposed convolution (weights transposed and flipped)
//     times GELU' of the saved pre-activation, the weight gradient a
//     correlation of the output cotangent with the layer input reduced over
//     pixels in fixed order (deterministic), the bias gradient a channel sum.
//
// The temporal correction u_k = P(V + c - mean(c)), c = TC(history) (Sec. 3.2,
// 3.5) transposes to vbar = P(lam), cbar = P(lam) - mean, then the correction
// network's reverse mode into the history states.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fv_glearned.cuh"

namespace ldfv {
namespace {

// ---------------------------------------------------------------------------
// face-value cotangents from the tendency cotangent (transpose of gstage_kernel)
// ---------------------------------------------------------------------------
struct GVbarArgs {
  const float* T;     // tendency cotangent [batch][2][ny][nx]
  const float* inst;  // face values [batch][8][ny][nx]
  const float* w;     // stage state
  float* vbar;        // [batch][8][ny][nx]
  float* ubar;        // [batch][2][ny][nx], written: the direct terms
  int nx, ny, burgers, forced;
  float nu, idx, idy, drag;
};

__global__ void __launch_bounds__(256) gvbar_kernel(const GVbarArgs a) {
  const int hw = a.nx * a.ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / a.nx, i = p - j * a.nx;
  const int pn = ((j + 1) % a.ny) * a.nx + i, ps = ((j - 1 + a.ny) % a.ny) * a.nx + i;
  const int pe = j * a.nx + (i + 1) % a.nx, pw = j * a.nx + (i - 1 + a.nx) % a.nx;
  const float* Tu = a.T + (size_t)b * 2 * hw;
  const float* Tv = Tu + hw;
  const float* I = a.inst + (size_t)b * 8 * hw;
  const float tu = Tu[p], tue = Tu[pe], tus = Tu[ps];
  const float tv = Tv[p], tvw = Tv[pw], tvn = Tv[pn];
  const float Uc = I[p], Uk = I[2 * hw + p], Vk = I[4 * hw + p], Vc = I[6 * hw + p];
  float vb[8];
  // advection: -(Uc^2 - Uc(i-1)^2) idx in tu, the corner products Uk Vk in both
  // components, -(Vc^2 - Vc(j-1)^2) idy in tv
  vb[0] = 2.0f * Uc * (tue - tu) * a.idx;
  const float pbar = (tu - tus) * a.idy + (tv - tvw) * a.idx;
  vb[2] = pbar * Vk;
  vb[4] = pbar * Uk;
  vb[6] = 2.0f * Vc * (tvn - tv) * a.idy;
  // diffusion
  vb[1] = a.nu * (tu - tue) * a.idx;
  vb[3] = a.nu * (tus - tu) * a.idy;
  vb[5] = a.nu * (tvw - tv) * a.idx;
  vb[7] = a.nu * (tv - tvn) * a.idy;
  float ub = 0.f, vbv = 0.f;
  if (a.burgers) {
    // tu += u 0.5 (divc(i-1) + divc), tv += v 0.5 (divc(j-1) + divc), divc = Gxc + Gyc
    const float* u = a.w + (size_t)b * 2 * hw;
    const float* v = u + hw;
    const float dc = I[hw + p] + I[7 * hw + p];
    const float dcw = I[hw + pw] + I[7 * hw + pw];
    const float dcs = I[hw + ps] + I[7 * hw + ps];
    ub += tu * 0.5f * (dcw + dc);
    vbv += tv * 0.5f * (dcs + dc);
    const float db = 0.5f * (tue * u[pe] + tu * u[p] + tvn * v[pn] + tv * v[p]);
    vb[1] += db;
    vb[7] += db;
  }
  if (a.forced) {
    ub -= a.drag * tu;
    vbv -= a.drag * tv;
  }
  float* V = a.vbar + (size_t)b * 8 * hw + p;
#pragma unroll
  for (int q = 0; q < 8; ++q) V[(size_t)q * hw] = vb[q];
  a.ubar[(size_t)b * 2 * hw + p] = ub;
  a.ubar[(size_t)b * 2 * hw + hw + p] = vbv;
}

// instance q = 2 pr + kind, pr = 2 field + axis; the tap (r, c) of the face at
// (j, i) reads the field at (j + dj, i + di)
__device__ __forceinline__ void tap_offset(int pr, int r, int cc, int& dj, int& di) {
  const int axis = pr & 1;
  const int sh = (pr == 0 || pr == 3) ? -1 : -2;
  dj = axis == 0 ? r - 2 : cc + sh;
  di = axis == 0 ? cc + sh : r - 2;
}

// ubar[field](j, i) += sum over the field's instances q and taps t of
// K_q,t(f) vbar_q(f) at the face f = (j - dj_t, i - di_t) whose tap t reads (j, i)
__global__ void __launch_bounds__(256) gscatter_kernel(const float* K, const float* vbar, float* ubar, int nx, int ny,
                                                       int ncoef) {
  const int hw = nx * ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / nx, i = p - j * nx;
  const float* Kb = K + (size_t)b * ncoef * hw;
  const float* Vb = vbar + (size_t)b * 8 * hw;
#pragma unroll 1
  for (int fld = 0; fld < 2; ++fld) {
    float acc = 0.f;
#pragma unroll 1
    for (int ax = 0; ax < 2; ++ax) {
      const int pr = 2 * fld + ax;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          int dj, di;
          tap_offset(pr, r, cc, dj, di);
          const int f = ((j - dj + 2 * ny) % ny) * nx + (i - di + 2 * nx) % nx;
#pragma unroll
          for (int kind = 0; kind < 2; ++kind) {
            const int q = 2 * pr + kind;
            acc = fmaf(Kb[(size_t)(q * 20 + r * 4 + cc) * hw + f], Vb[(size_t)q * hw + f], acc);
          }
        }
    }
    ubar[((size_t)b * 2 + fld) * hw + p] += acc;
  }
}

// network-output cotangent: Cbar_q,t(f) = scale proj(vbar_q(f) taps(f))_t
// (ablation 1: without the projection)
__global__ void __launch_bounds__(256) gkbar_kernel(const float* w, const float* vbar, float* cbar, int nx, int ny,
                                                    int ablation, float idx, float idy, int ncoef) {
  const int hw = nx * ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / nx, i = p - j * nx;
  const float cval[4] = {-1.5f, -0.5f, 0.5f, 1.5f};
#pragma unroll 1
  for (int pr = 0; pr < 4; ++pr) {
    const float* f = w + ((size_t)b * 2 + (pr >> 1)) * hw;
    float tap[20];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        int dj, di;
        tap_offset(pr, r, cc, dj, di);
        tap[r * 4 + cc] = f[((j + dj + 2 * ny) % ny) * nx + (i + di + 2 * nx) % nx];
      }
    const int axis = pr & 1;
    const float ih = axis == 0 ? idx : idy;
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const int q = 2 * pr + kind;
      const float vb = vbar[((size_t)b * 8 + q) * hw + p];
      float s1 = 0.f, sc = 0.f, sr = 0.f;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float v = vb * tap[r * 4 + cc];
          s1 += v;
          sc += v * cval[cc];
          sr += v * (float)(r - 2);
        }
      const float pk = ablation == 0 ? 1.0f : 0.0f;
      s1 *= pk * (1.0f / 20.0f);
      sc *= pk * (1.0f / 25.0f);
      sr *= pk * (1.0f / 40.0f);
      const float scale = kind == 1 ? ih : 1.0f;
      float* out = cbar + ((size_t)b * ncoef + q * 20) * hw + p;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          out[(size_t)(r * 4 + cc) * hw] = (vb * tap[r * 4 + cc] - s1 - sc * cval[cc] - sr * (float)(r - 2)) * scale;
    }
  }
}

// ---------------------------------------------------------------------------
// weight gradient of one 3x3 layer: part[chunk][o][c][tap] = sum over the
// chunk's pixels of zbar[o](p) in[c](p + (dy, dx)); the layer input is a
// tensor (optionally through GELU: the saved pre-activation of the layer
// before) or cin / 2 states by pointer (the correction network's history)
// ---------------------------------------------------------------------------
constexpr int kWgO = 64, kWgC = 16, kWgK = 32, kWgKP = 33;

struct GWgradArgs {
  const float* zbar;          // [batch][cout][ny][nx]
  const float* in;            // [batch][cin][ny][nx]
  const float* const* hist;   // or cin / 2 states [batch][2][ny][nx]
  const float* const* sptr;   // with hist: the last channel, a scalar [batch][ny][nx]
  float* part;                // [nchunk][cout][cin][9]
  int cin, cout, nx, ny, in_gelu;
  long long total;            // batch * nx * ny
  long long chunk;            // pixels per CTA (a multiple of kWgK)
};

__global__ void __launch_bounds__(256) gwgrad_kernel(const GWgradArgs a) {
  __shared__ float zs[kWgO][kWgK];
  __shared__ float xs[kWgC * 9 * kWgKP];
  const int hw = a.nx * a.ny;
  const int o0 = blockIdx.x * kWgO, c0 = blockIdx.y * kWgC;
  const long long pb = (long long)blockIdx.z * a.chunk;
  const long long pe = min(pb + a.chunk, a.total);
  const int tid = threadIdx.x;
  const int og = tid / kWgC, cl = tid % kWgC;
  float acc[4][9];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[i][t] = 0.f;
  for (long long k0 = pb; k0 < pe; k0 += kWgK) {
    for (int e = tid; e < kWgO * kWgK; e += 256) {
      const int o = e / kWgK, k = e % kWgK;
      const long long P = k0 + k;
      float v = 0.f;
      if (o0 + o < a.cout && P < pe) {
        const int b = (int)(P / hw), p = (int)(P - (long long)b * hw);
        v = a.zbar[((size_t)b * a.cout + o0 + o) * hw + p];
      }
      zs[o][k] = v;
    }
    for (int e = tid; e < kWgC * 9 * kWgK; e += 256) {
      const int c = e / (9 * kWgK), rem = e % (9 * kWgK), tap = rem / kWgK, k = rem % kWgK;
      const long long P = k0 + k;
      float v = 0.f;
      if (c0 + c < a.cin && P < pe) {
        const int b = (int)(P / hw), p = (int)(P - (long long)b * hw);
        const int y = p / a.nx, x = p - y * a.nx;
        const int yy = (y + tap / 3 - 1 + a.ny) % a.ny, xx = (x + tap % 3 - 1 + a.nx) % a.nx;
        const int ch = c0 + c;
        const float* src = !a.hist                        ? a.in + ((size_t)b * a.cin + ch) * hw
                           : (a.sptr && ch == a.cin - 1) ? a.sptr[0] + (size_t)b * hw
                                                         : a.hist[ch >> 1] + ((size_t)b * 2 + (ch & 1)) * hw;
        v = src[yy * a.nx + xx];
        if (a.in_gelu) v = gelu_exact(v);
      }
      xs[(c * 9 + tap) * kWgKP + k] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kWgK; ++k) {
      float z[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) z[i] = zs[4 * og + i][k];
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const float xv = xs[(cl * 9 + t) * kWgKP + k];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][t] = fmaf(z[i], xv, acc[i][t]);
      }
    }
    __syncthreads();
  }
  const int c = c0 + cl;
  if (c >= a.cin) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int o = o0 + 4 * og + i;
    if (o >= a.cout) continue;
    float* dst = a.part + (((size_t)blockIdx.z * a.cout + o) * a.cin + c) * 9;
#pragma unroll
    for (int t = 0; t < 9; ++t) dst[t] = acc[i][t];
  }
}

// dst[i] += sum_k part[k][i], in chunk order
__global__ void reduce_partials_kernel(const float* part, int nchunk, size_t n, float* dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < nchunk; ++k) s += part[(size_t)k * n + i];
    dst[i] += s;
  }
}

// sums[o] = sum over batch and pixels of t[b][o] (FP64, fixed order), one CTA per channel
__global__ void __launch_bounds__(256) chansum_kernel(const float* t, int C, int hw, int batch, double* sums) {
  const int o = blockIdx.x;
  double s = 0.0;
  for (int b = 0; b < batch; ++b) {
    const float* src = t + ((size_t)b * C + o) * hw;
    for (int k = threadIdx.x; k < hw; k += blockDim.x) s += src[k];
  }
  __shared__ double red[8];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += red[k];
    sums[o] = tot;
  }
}

// bias gradient: dst[o] += sums[o]; with wl: also W_L[kind][axis][t] += the
// sums of the two instances (u and v) that share it; with wls: W_Ls[kind][axis][t]
// += the sum of the scalar instance m = 2 axis + kind
__global__ void add_sums_kernel(const double* sums, int C, float* dst, float* wl, float* wls) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < C) dst[k] += (float)sums[k];
  if (k < 80) {
    const int kind = k / 40, axis = (k / 20) % 2, t = k % 20;
    if (wl) {
      const int q1 = 2 * axis + kind, q2 = 2 * (2 + axis) + kind;
      wl[k] += (float)(sums[q1 * 20 + t] + sums[q2 * 20 + t]);
    }
    if (wls) wls[k] += (float)sums[kNCoef + (2 * axis + kind) * 20 + t];
  }
}

// ---------------------------------------------------------------------------
// the passive scalar's reverse mode: tendency -div(u s_f - D grad_f s) with
// F_x = u s_x - D g_x on the west faces and F_y = v s_y - D g_y on the south faces
// ---------------------------------------------------------------------------
// face cotangents of the four scalar instances from the scalar tendency
// cotangent qb, and the velocity's direct terms (F_x, F_y are products with u, v)
__global__ void __launch_bounds__(256) gsvbar_kernel(const float* qb, const float* sinst, const float* w, float* svbar,
                                                     float* ubar, int nx, int ny, float idx, float idy, float diff) {
  const int hw = nx * ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / nx, i = p - j * nx;
  const float* q = qb + (size_t)b * hw;
  const float fxb = (q[p] - q[j * nx + (i - 1 + nx) % nx]) * idx;
  const float fyb = (q[p] - q[((j - 1 + ny) % ny) * nx + i]) * idy;
  const float* SI = sinst + (size_t)b * 4 * hw;
  const size_t e = (size_t)b * 2 * hw + p;
  ubar[e] += fxb * SI[p];
  ubar[e + hw] += fyb * SI[2 * hw + p];
  float* V = svbar + (size_t)b * 4 * hw + p;
  V[0] = fxb * w[e];
  V[hw] = -diff * fxb;
  V[2 * (size_t)hw] = fyb * w[e + hw];
  V[3 * (size_t)hw] = -diff * fyb;
}

// the scalar instance m = 2 axis + kind reads s at (j + dj, i + di) for tap (r, c)
__device__ __forceinline__ void scalar_tap_offset(int axis, int r, int cc, int& dj, int& di) {
  dj = axis == 0 ? r - 2 : cc - 2;
  di = axis == 0 ? cc - 2 : r - 2;
}

// zbar(j, i) = sum over the scalar instances m and taps t of K_m,t(f) svbar_m(f)
// at the face f whose tap t reads (j, i); K at channel 160 + 20 m + t
__global__ void __launch_bounds__(256) gsscatter_kernel(const float* K, const float* svbar, float* zbar, int nx, int ny,
                                                        int ncoef) {
  const int hw = nx * ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / nx, i = p - j * nx;
  const float* Kb = K + ((size_t)b * ncoef + kNCoef) * hw;
  const float* Vb = svbar + (size_t)b * 4 * hw;
  float acc = 0.f;
#pragma unroll 1
  for (int axis = 0; axis < 2; ++axis)
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        int dj, di;
        scalar_tap_offset(axis, r, cc, dj, di);
        const int f = ((j - dj + 2 * ny) % ny) * nx + (i - di + 2 * nx) % nx;
#pragma unroll
        for (int kind = 0; kind < 2; ++kind) {
          const int m = 2 * axis + kind;
          acc = fmaf(Kb[(size_t)(m * 20 + r * 4 + cc) * hw + f], Vb[(size_t)m * hw + f], acc);
        }
      }
  zbar[(size_t)b * hw + p] = acc;
}

// the scalar instances' network-output cotangent: scale proj(svbar_m(f) taps(f))
// into channels 160 + 20 m + t
__global__ void __launch_bounds__(256) gskbar_kernel(const float* z, const float* svbar, float* cbar, int nx, int ny,
                                                     float idx, float idy, int ncoef) {
  const int hw = nx * ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / nx, i = p - j * nx;
  const float cval[4] = {-1.5f, -0.5f, 0.5f, 1.5f};
  const float* f = z + (size_t)b * hw;
#pragma unroll 1
  for (int axis = 0; axis < 2; ++axis) {
    float tap[20];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        int dj, di;
        scalar_tap_offset(axis, r, cc, dj, di);
        tap[r * 4 + cc] = f[((j + dj + 2 * ny) % ny) * nx + (i + di + 2 * nx) % nx];
      }
    const float ih = axis == 0 ? idx : idy;
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const int m = 2 * axis + kind;
      const float vb = svbar[((size_t)b * 4 + m) * hw + p];
      float s1 = 0.f, sc = 0.f, sr = 0.f;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float v = vb * tap[r * 4 + cc];
          s1 += v;
          sc += v * cval[cc];
          sr += v * (float)(r - 2);
        }
      s1 *= 1.0f / 20.0f;
      sc *= 1.0f / 25.0f;
      sr *= 1.0f / 40.0f;
      const float scale = kind == 1 ? ih : 1.0f;
      float* out = cbar + ((size_t)b * ncoef + kNCoef + m * 20) * hw + p;
#pragma unroll
      for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          out[(size_t)(r * 4 + cc) * hw] = (vb * tap[r * 4 + cc] - s1 - sc * cval[cc] - sr * (float)(r - 2)) * scale;
    }
  }
}

// the network input's cotangent (u, v, s) split into the state cotangents
__global__ void split_add_kernel(const float* x3, float* ubar, float* zbar, int hw, int batch) {
  const size_t n = (size_t)batch * hw;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const size_t b = k / hw, p = k - b * hw;
    ubar[b * 2 * hw + p] += x3[b * 3 * hw + p];
    ubar[b * 2 * hw + hw + p] += x3[b * 3 * hw + hw + p];
    zbar[k] += x3[b * 3 * hw + 2 * hw + p];
  }
}

// wt[c][o][8 - tap] = w[o][c][tap]: the transposed convolution's weights
__global__ void transpose_weights_kernel(const float* w, float* wt, int cout, int cin) {
  const int n = cout * cin * 9;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int tap = e % 9, c = (e / 9) % cin, o = e / (9 * cin);
    wt[((size_t)c * cout + o) * 9 + 8 - tap] = w[e];
  }
}

// y = a x + b y over n elements (b = 0: y is not read)
__global__ void axpby_kernel(float* y, const float* x, float a, float b, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    y[k] = b == 0.0f ? a * x[k] : a * x[k] + b * y[k];
}

// out = g - mean(g) per trajectory and component (one CTA each, FP64 mean)
__global__ void __launch_bounds__(256) mean_free_kernel(const float* g, float* out, int hw) {
  const size_t base = (size_t)blockIdx.x * hw;
  __shared__ double red[8];
  double s = 0.0;
  for (int k = threadIdx.x; k < hw; k += blockDim.x) s += g[base + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double m = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m += red[k];
  const float mean = (float)(m / hw);
  for (int k = threadIdx.x; k < hw; k += blockDim.x) out[base + k] = g[base + k] - mean;
}

unsigned grid1(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16); }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Ctx {
  fd_ctx* c;
  GenAdjoint& A;
  cudaStream_t st;
  int launches = 0;
  int B, nx, ny, hw;
  size_t slot;  // floats of one state [batch][2][ny][nx]
};

cudaError_t last(Ctx& x) {
  ++x.launches;
  return cudaGetLastError();
}

cudaError_t project(Ctx& x, float* w) {
  if (x.c->grid.flow != FD_NAVIER_STOKES) return cudaSuccess;
  x.launches += 5;
  return fd_generic_project(x.c, w, x.st);
}

// the transposed weights of both networks, refreshed after a parameter upload
cudaError_t refresh_wt(Ctx& x) {
  GenericLearned& G = *x.c->glrn;
  if (x.A.wt_version == G.version) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 6 && e == cudaSuccess; ++l) {
    const int ci = stencil_cin(l, G.scalar), co = stencil_cout(l, G.scalar);
    transpose_weights_kernel<<<grid1((size_t)co * ci * 9), 256, 0, x.st>>>(G.d_params + G.off_sw[l],
                                                                          x.A.wt + x.A.off_wt_s[l], co, ci);
    e = last(x);
    if (e == cudaSuccess && G.kc > 0) {
      const int cit = l == 0 ? 2 * G.kc : kHid, cot = l == 5 ? 2 : kHid;
      transpose_weights_kernel<<<grid1((size_t)cot * cit * 9), 256, 0, x.st>>>(G.d_params + G.off_tw[l],
                                                                            x.A.wt + x.A.off_wt_t[l], cot, cit);
      e = last(x);
    }
  }
  if (e == cudaSuccess) x.A.wt_version = G.version;
  return e;
}

// dparams[off_w ..] += the weight gradient of a layer, dparams[off_b ..] += its bias gradient
cudaError_t layer_param_grads(Ctx& x, const float* zbar, const float* in, const float* const* hist,
                              const float* const* sptr, int in_gelu, int cin, int cout, float* dw, float* db,
                              float* dwl, float* dwls) {
  const long long total = (long long)x.B * x.hw;
  const int ob = (cout + kWgO - 1) / kWgO, cb = (cin + kWgC - 1) / kWgC;
  // about four CTAs per SM in all, within the partial-sum buffer
  long long nchunk = std::max<long long>(1, 608 / (ob * cb));
  nchunk = std::min<long long>(nchunk, (total + kWgK - 1) / kWgK);
  nchunk = std::min<long long>(nchunk, (long long)(x.A.npart / ((size_t)cout * cin * 9)));
  long long chunk = (total + nchunk - 1) / nchunk;
  chunk = (chunk + kWgK - 1) / kWgK * kWgK;
  nchunk = (total + chunk - 1) / chunk;
  GWgradArgs a;
  a.zbar = zbar;
  a.in = in;
  a.hist = hist;
  a.sptr = sptr;
  a.part = x.A.part;
  a.cin = cin;
  a.cout = cout;
  a.nx = x.nx;
  a.ny = x.ny;
  a.in_gelu = in_gelu;
  a.total = total;
  a.chunk = chunk;
  gwgrad_kernel<<<dim3((unsigned)ob, (unsigned)cb, (unsigned)nchunk), 256, 0, x.st>>>(a);
  cudaError_t e = last(x);
  const size_t n = (size_t)cout * cin * 9;
  if (e == cudaSuccess) {
    reduce_partials_kernel<<<grid1(n), 256, 0, x.st>>>(x.A.part, (int)nchunk, n, dw);
    e = last(x);
  }
  if (e == cudaSuccess) {
    chansum_kernel<<<(unsigned)cout, 256, 0, x.st>>>(zbar, cout, x.hw, x.B, x.A.sums);
    e = last(x);
  }
  if (e == cudaSuccess) {
    add_sums_kernel<<<1, 256, 0, x.st>>>(x.A.sums, cout, db, dwl, dwls);
    e = last(x);
  }
  return e;
}

// transposed convolution of a layer: out = convT(zbar) (* GELU'(gz)), cin and
// cout of the forward layer
cudaError_t layer_data_grad(Ctx& x, const float* zbar, const float* wt, int cin, int cout, float* out,
                            const float* gz, int accum, size_t ostride) {
  GConvArgs a = {};
  a.in = zbar;
  a.w = wt;
  a.out = out;
  a.gz = gz;
  a.accum = accum;
  a.ostride = ostride;
  a.cin = cout;
  a.cout = cin;
  a.nx = x.nx;
  a.ny = x.ny;
  ++x.launches;
  return launch_gconv_auto(a, x.B, x.st);
}

// reverse mode of a six-layer network whose forward pre-activations are in
// A.zsave, from the output cotangent zbar5 (cout5 channels, overwritten);
// the input cotangent goes to xout (accumulated into a [batch][2][ny][nx]
// state, or written per history state with ostride)
cudaError_t net_backward(Ctx& x, float* zbar5, int cout5, int cin0, const float* in0, const float* const* hist,
                         const float* const* sptr, const size_t* off_w, const size_t* off_b, const size_t* off_wt,
                         float* dparams, float* dwl, float* dwls, float* xout, int xaccum, size_t xstride) {
  cudaError_t e = cudaSuccess;
  const float* zbar = zbar5;
  for (int l = 5; l >= 0 && e == cudaSuccess; --l) {
    const int cin = l == 0 ? cin0 : kHid, cout = l == 5 ? cout5 : kHid;
    if (dparams)
      e = layer_param_grads(x, zbar, l == 0 ? in0 : x.A.zsave[l - 1], l == 0 ? hist : nullptr,
                            l == 0 ? sptr : nullptr, l > 0, cin, cout, dparams + off_w[l], dparams + off_b[l],
                            l == 5 ? dwl : nullptr, l == 5 ? dwls : nullptr);
    if (e != cudaSuccess) break;
    if (l > 0) {
      float* out = x.A.zb[l & 1];
      e = layer_data_grad(x, zbar, x.A.wt + off_wt[l], cin, cout, out, x.A.zsave[l - 1], 0, 0);
      zbar = out;
    } else {
      e = layer_data_grad(x, zbar, x.A.wt + off_wt[0], cin, cout, xout, nullptr, xaccum, xstride);
    }
  }
  return e;
}

// face values (and per-face kernels into A.kbuf) of the stage state w: the
// network output sits in A.kbuf for learned contexts
cudaError_t faces(Ctx& x, const float* w, bool learned, bool want_k) {
  GFaceArgs fa = {};
  fa.w = w;
  fa.coef = learned ? x.A.kbuf : nullptr;
  fa.wl = learned ? x.c->glrn->d_params + x.c->glrn->off_wl : nullptr;
  fa.inst = x.A.inst;
  fa.kout = want_k ? x.A.kbuf : nullptr;
  fa.nx = x.nx;
  fa.ny = x.ny;
  fa.dord = x.c->opts.deriv_order;
  fa.ablation = learned ? x.c->glrn->ablation : 0;
  fa.ncoef = kNCoef;
  fa.idx = (float)(x.nx / x.c->grid.lx);
  fa.idy = (float)(x.ny / x.c->grid.ly);
  gface_kernel<<<dim3((unsigned)((x.hw + 255) / 256), (unsigned)x.B), 256, 0, x.st>>>(fa);
  return last(x);
}

// w_out = P(u + a_s dt H(w)) for the forward stages s = 0, 1, 2
cudaError_t stage_forward(Ctx& x, int s, const float* w, const float* u, float* w_out, bool learned) {
  GenericState& S = *x.c->gen;
  cudaError_t e = cudaSuccess;
  if (learned) {
    GenericLearned& G = *x.c->glrn;
    e = run_net(x.c, nullptr, nullptr, w, 2, G.off_sw, G.off_sb, kNCoef, x.A.kbuf, x.st);
    x.launches += 6;
  }
  if (e == cudaSuccess) e = faces(x, w, learned, false);
  if (e != cudaSuccess) return e;
  GStageArgs sa = {};
  sa.inst = x.A.inst;
  sa.w = w;
  sa.un = u;
  sa.acc = x.A.acc;
  sa.wout = w_out;
  sa.frc = static_cast<const float*>(S.frc);
  sa.nx = x.nx;
  sa.ny = x.ny;
  sa.stage = s;
  sa.forced = x.c->forcing.kind;
  sa.burgers = x.c->grid.flow == FD_BURGERS;
  sa.dt = (float)x.c->dt;
  sa.nu = (float)x.c->nu;
  sa.idx = (float)(x.nx / x.c->grid.lx);
  sa.idy = (float)(x.ny / x.c->grid.ly);
  sa.drag = (float)(x.c->forcing.kind == 1 ? x.c->forcing.drag : 0.0);
  gstage_kernel<<<dim3((unsigned)((x.hw + 255) / 256), (unsigned)x.B), 256, 0, x.st>>>(sa);
  e = last(x);
  if (e == cudaSuccess) e = project(x, w_out);
  return e;
}

// A.ubar = (dH/dw)^T T at the stage state w (H the tendency); dparams accumulates
cudaError_t tendency_vjp(Ctx& x, const float* w, const float* T, bool learned, float* dparams) {
  GenericLearned* G = x.c->glrn;
  const dim3 cells((unsigned)((x.hw + 255) / 256), (unsigned)x.B);
  cudaError_t e = cudaSuccess;
  if (learned) {
    e = run_net(x.c, nullptr, nullptr, w, 2, G->off_sw, G->off_sb, kNCoef, x.A.kbuf, x.st, x.A.zsave);
    x.launches += 6;
  }
  if (e == cudaSuccess) e = faces(x, w, learned, true);
  if (e != cudaSuccess) return e;
  GVbarArgs va;
  va.T = T;
  va.inst = x.A.inst;
  va.w = w;
  va.vbar = x.A.vbar;
  va.ubar = x.A.ubar;
  va.nx = x.nx;
  va.ny = x.ny;
  va.burgers = x.c->grid.flow == FD_BURGERS;
  va.forced = x.c->forcing.kind == 1;
  va.nu = (float)x.c->nu;
  va.idx = (float)(x.nx / x.c->grid.lx);
  va.idy = (float)(x.ny / x.c->grid.ly);
  va.drag = (float)(x.c->forcing.kind == 1 ? x.c->forcing.drag : 0.0);
  gvbar_kernel<<<cells, 256, 0, x.st>>>(va);
  e = last(x);
  if (e == cudaSuccess) {
    gscatter_kernel<<<cells, 256, 0, x.st>>>(x.A.kbuf, x.A.vbar, x.A.ubar, x.nx, x.ny, kNCoef);
    e = last(x);
  }
  if (e != cudaSuccess || !learned) return e;
  // the network-output cotangent replaces the per-face kernels in A.kbuf
  gkbar_kernel<<<cells, 256, 0, x.st>>>(w, x.A.vbar, x.A.kbuf, x.nx, x.ny, G->ablation, va.idx, va.idy, kNCoef);
  e = last(x);
  if (e == cudaSuccess)
    e = net_backward(x, x.A.kbuf, kNCoef, 2, w, nullptr, nullptr, G->off_sw, G->off_sb, x.A.off_wt_s, dparams,
                     dparams ? dparams + G->off_wl : nullptr, nullptr, x.A.ubar, 1, 0);
  return e;
}

fd_status gadjoint_alloc(fd_ctx* c) {
  GenAdjoint* A = new (std::nothrow) GenAdjoint();
  if (!A) return fd_set_error(c, FD_ENOMEM, "generic-grid reverse mode: out of host memory");
  c->gadj = A;
  const size_t hw = (size_t)c->grid.nx * c->grid.ny, B = c->grid.batch;
  const size_t st = B * 2 * hw * sizeof(float);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  for (int s = 1; s < 4; ++s) alloc((void**)&A->w[s], st);
  for (float** p : {&A->acc, &A->ubar, &A->g, &A->y, &A->rb, &A->lam}) alloc((void**)p, st);
  alloc((void**)&A->kbuf, B * kNCoef * hw * sizeof(float));
  A->kbuf_ch = kNCoef;
  alloc((void**)&A->inst, B * 8 * hw * sizeof(float));
  alloc((void**)&A->vbar, B * 8 * hw * sizeof(float));
  if (c->glrn) {
    GenericLearned& G = *c->glrn;
    for (int l = 0; l < 5; ++l) alloc((void**)&A->zsave[l], B * kHid * hw * sizeof(float));
    for (int k = 0; k < 2; ++k) alloc((void**)&A->zb[k], B * kHid * hw * sizeof(float));
    size_t off = 0;
    for (int l = 0; l < 6; ++l) {
      A->off_wt_s[l] = off;
      off += (size_t)stencil_cin(l, G.scalar) * stencil_cout(l, G.scalar) * 9;
    }
    for (int l = 0; l < 6 && G.kc > 0; ++l) {
      A->off_wt_t[l] = off;
      off += (size_t)(l == 0 ? 2 * G.kc : kHid) * (l == 5 ? 2 : kHid) * 9;
    }
    alloc((void**)&A->wt, off * sizeof(float));
    // partial sums: about four CTAs per SM of any layer's gradient (608 chunks
    // of 16 x 64 x 9, 152 of 64 x 64 x 9, 50 of 160 x 64 x 9); the chunk count
    // is clamped to this size
    A->npart = (size_t)608 * kHid * kHid * 9 / 4;
    alloc((void**)&A->part, A->npart * sizeof(float));
    alloc((void**)&A->sums, 256 * sizeof(double));
    alloc((void**)&A->d_hist, 8 * sizeof(const float*));
  }
  if (e != cudaSuccess) {
    fd_gadjoint_free(c);
    return fd_set_error(c, FD_ENOMEM, "generic-grid reverse mode workspace: %s", cudaGetErrorString(e));
  }
  return FD_OK;
}

// ---------------------------------------------------------------------------
// joint velocity-scalar reverse mode
// ---------------------------------------------------------------------------
fd_status gadjoint_alloc_joint(fd_ctx* c) {
  GenAdjoint& A = *c->gadj;
  const size_t hw = (size_t)c->grid.nx * c->grid.ny, B = c->grid.batch;
  const size_t sb = B * hw * sizeof(float);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  // the per-face kernels of the scalar's instances sit in channels 160 .. 239
  if (A.kbuf_ch < kNCoefScalar) {
    cudaFree(A.kbuf);
    A.kbuf = nullptr;
    alloc((void**)&A.kbuf, B * kNCoefScalar * hw * sizeof(float));
    A.kbuf_ch = e == cudaSuccess ? kNCoefScalar : 0;
  }
  for (int s = 1; s < 4; ++s) alloc((void**)&A.z[s], sb);
  for (float** p : {&A.sacc, &A.zbar, &A.qb, &A.ys, &A.lams, &A.ls0}) alloc((void**)p, sb);
  alloc((void**)&A.sinst, 4 * sb);
  alloc((void**)&A.svbar, 4 * sb);
  alloc((void**)&A.x3, 3 * sb);
  alloc((void**)&A.d_wptr, 4 * sizeof(const float*));
  alloc((void**)&A.d_zptr, 4 * sizeof(const float*));
  if (e != cudaSuccess) {
    // drop the whole workspace (its kernel buffer may be gone): the next call allocates afresh
    fd_gadjoint_free(c);
    return fd_set_error(c, FD_ENOMEM, "joint reverse mode workspace: %s", cudaGetErrorString(e));
  }
  A.joint = true;
  return FD_OK;
}

// face values of velocity and scalar at the stage state (w, z) (and, with want_k,
// the per-face kernels over the network output in A.kbuf)
cudaError_t faces_joint(Ctx& x, const float* w, const float* z, bool learned, bool want_k) {
  GenericLearned* G = x.c->glrn;
  GFaceArgs fa = {};
  fa.w = w;
  fa.coef = learned ? x.A.kbuf : nullptr;
  fa.wl = learned ? G->d_params + G->off_wl : nullptr;
  fa.wls = learned ? G->d_params + G->off_wls : nullptr;
  fa.inst = x.A.inst;
  fa.kout = want_k ? x.A.kbuf : nullptr;
  fa.skout = want_k ? x.A.kbuf : nullptr;
  fa.s = z;
  fa.sinst = x.A.sinst;
  fa.nx = x.nx;
  fa.ny = x.ny;
  fa.dord = x.c->opts.deriv_order;
  fa.ablation = 0;
  fa.ncoef = kNCoefScalar;
  fa.idx = (float)(x.nx / x.c->grid.lx);
  fa.idy = (float)(x.ny / x.c->grid.ly);
  gface_kernel<<<dim3((unsigned)((x.hw + 255) / 256), (unsigned)x.B), 256, 0, x.st>>>(fa);
  return last(x);
}

// the stencil network on (w_s, z_s) through the stage pointer tables into A.kbuf
cudaError_t net_joint(Ctx& x, int s, float* const* zsave) {
  GenericLearned& G = *x.c->glrn;
  x.launches += 6;
  return run_net(x.c, x.A.d_wptr + s, x.A.d_zptr + s, nullptr, 3, G.off_sw, G.off_sb, kNCoefScalar, x.A.kbuf, x.st,
                 zsave);
}

// (w_{s+1}, z_{s+1}) from (w_s, z_s) for the forward stages s = 0, 1, 2
cudaError_t stage_forward_joint(Ctx& x, int s, const float* w, const float* z, const float* u, const float* sn,
                                float* w_out, float* z_out, bool learned, float diff) {
  GenericState& S = *x.c->gen;
  cudaError_t e = learned ? net_joint(x, s, nullptr) : cudaSuccess;
  if (e == cudaSuccess) e = faces_joint(x, w, z, learned, false);
  if (e != cudaSuccess) return e;
  GStageArgs sa = {};
  sa.inst = x.A.inst;
  sa.w = w;
  sa.un = u;
  sa.acc = x.A.acc;
  sa.wout = w_out;
  sa.frc = static_cast<const float*>(S.frc);
  sa.sinst = x.A.sinst;
  sa.sn = sn;
  sa.sacc = x.A.sacc;
  sa.sout = z_out;
  sa.diff = diff;
  sa.nx = x.nx;
  sa.ny = x.ny;
  sa.stage = s;
  sa.forced = x.c->forcing.kind;
  sa.burgers = x.c->grid.flow == FD_BURGERS;
  sa.dt = (float)x.c->dt;
  sa.nu = (float)x.c->nu;
  sa.idx = (float)(x.nx / x.c->grid.lx);
  sa.idy = (float)(x.ny / x.c->grid.ly);
  sa.drag = (float)(x.c->forcing.kind == 1 ? x.c->forcing.drag : 0.0);
  gstage_kernel<<<dim3((unsigned)((x.hw + 255) / 256), (unsigned)x.B), 256, 0, x.st>>>(sa);
  e = last(x);
  if (e == cudaSuccess) e = project(x, w_out);
  return e;
}

// (A.ubar, A.zbar) = the transposed joint tendency at stage s applied to (rb, qb)
cudaError_t joint_tendency_vjp(Ctx& x, int s, const float* w, const float* z, const float* rb, const float* qb,
                               bool learned, float diff, float* dparams) {
  GenericLearned* G = x.c->glrn;
  const dim3 cells((unsigned)((x.hw + 255) / 256), (unsigned)x.B);
  const float idx = (float)(x.nx / x.c->grid.lx), idy = (float)(x.ny / x.c->grid.ly);
  cudaError_t e = learned ? net_joint(x, s, x.A.zsave) : cudaSuccess;
  if (e == cudaSuccess) e = faces_joint(x, w, z, learned, true);
  if (e != cudaSuccess) return e;
  GVbarArgs va;
  va.T = rb;
  va.inst = x.A.inst;
  va.w = w;
  va.vbar = x.A.vbar;
  va.ubar = x.A.ubar;
  va.nx = x.nx;
  va.ny = x.ny;
  va.burgers = x.c->grid.flow == FD_BURGERS;
  va.forced = x.c->forcing.kind == 1;
  va.nu = (float)x.c->nu;
  va.idx = idx;
  va.idy = idy;
  va.drag = (float)(x.c->forcing.kind == 1 ? x.c->forcing.drag : 0.0);
  gvbar_kernel<<<cells, 256, 0, x.st>>>(va);
  e = last(x);
  if (e == cudaSuccess) {
    gsvbar_kernel<<<cells, 256, 0, x.st>>>(qb, x.A.sinst, w, x.A.svbar, x.A.ubar, x.nx, x.ny, idx, idy, diff);
    e = last(x);
  }
  if (e == cudaSuccess) {
    gscatter_kernel<<<cells, 256, 0, x.st>>>(x.A.kbuf, x.A.vbar, x.A.ubar, x.nx, x.ny, kNCoefScalar);
    e = last(x);
  }
  if (e == cudaSuccess) {
    gsscatter_kernel<<<cells, 256, 0, x.st>>>(x.A.kbuf, x.A.svbar, x.A.zbar, x.nx, x.ny, kNCoefScalar);
    e = last(x);
  }
  if (e != cudaSuccess || !learned) return e;
  // the network-output cotangent of all twelve instances replaces the kernels
  gkbar_kernel<<<cells, 256, 0, x.st>>>(w, x.A.vbar, x.A.kbuf, x.nx, x.ny, 0, idx, idy, kNCoefScalar);
  e = last(x);
  if (e == cudaSuccess) {
    gskbar_kernel<<<cells, 256, 0, x.st>>>(z, x.A.svbar, x.A.kbuf, x.nx, x.ny, idx, idy, kNCoefScalar);
    e = last(x);
  }
  if (e == cudaSuccess)
    e = net_backward(x, x.A.kbuf, kNCoefScalar, 3, nullptr, x.A.d_wptr + s, x.A.d_zptr + s, G->off_sw, G->off_sb,
                     x.A.off_wt_s, dparams, dparams ? dparams + G->off_wl : nullptr,
                     dparams ? dparams + G->off_wls : nullptr, x.A.x3, 0, 0);
  if (e == cudaSuccess) {
    split_add_kernel<<<grid1((size_t)x.B * x.hw), 256, 0, x.st>>>(x.A.x3, x.A.ubar, x.A.zbar, x.hw, x.B);
    e = last(x);
  }
  return e;
}

}  // namespace
}  // namespace ldfv

using namespace ldfv;

void fd_gadjoint_free(fd_ctx* c) {
  GenAdjoint* A = c->gadj;
  if (!A) return;
  std::vector<void*> ps = {A->acc, A->kbuf, A->inst, A->vbar, A->ubar, A->g, A->y, A->rb, A->lam, A->wt, A->part,
                           A->sums, (void*)A->d_hist, A->sacc, A->sinst, A->svbar, A->zbar, A->qb, A->ys, A->lams,
                           A->ls0, A->x3, (void*)A->d_wptr, (void*)A->d_zptr};
  for (int s = 1; s < 4; ++s) ps.push_back(A->w[s]);
  for (int s = 1; s < 4; ++s) ps.push_back(A->z[s]);
  for (float* z : A->zsave) ps.push_back(z);
  for (float* z : A->zb) ps.push_back(z);
  for (void* p : ps)
    if (p) cudaFree(p);
  delete A;
  c->gadj = nullptr;
}

fd_status fd_gadjoint_step(fd_ctx* c, const float* u_in, const float* lam_out, float* lam_in, float* dparams,
                           cudaStream_t st) {
  if (c->grid.dtype != FD_F32)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_step_adjoint: the generic-grid reverse mode is built for FP32");
  GenericLearned* G = c->glrn;
  if (G && G->scalar)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_step_adjoint: not built for a model that learns the scalar");
  if (G && !G->ready) return fd_set_error(c, FD_EINVAL, "fd_step_adjoint: learned parameters not set (fd_set_params)");
  if (dparams && !G) return fd_set_error(c, FD_EINVAL, "fd_step_adjoint: dparams needs a learned context");
  if (!c->gadj) {
    const fd_status s = gadjoint_alloc(c);
    if (s != FD_OK) return s;
  }
  Ctx x{c, *c->gadj, st};
  x.B = c->grid.batch;
  x.nx = c->grid.nx;
  x.ny = c->grid.ny;
  x.hw = x.nx * x.ny;
  x.slot = (size_t)x.B * 2 * x.hw;
  GenAdjoint& A = x.A;
  const bool learned = G != nullptr;
  const float dt = (float)c->dt;
  cudaError_t e = learned ? refresh_wt(x) : cudaSuccess;
  // forward: the stage states w_1, w_2, w_3
  const float* w[4] = {u_in, A.w[1], A.w[2], A.w[3]};
  for (int s = 0; s < 3 && e == cudaSuccess; ++s) e = stage_forward(x, s, w[s], u_in, A.w[s + 1], learned);
  // reverse: g = P(lam_out); lam = g + sum of the stages' P(wbar) (the first stage's unprojected)
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.g, lam_out, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = project(x, A.g);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.lam, A.g, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  // tendency cotangent of stage s: cg g + cy P(wbar_{s+1})
  const float cg[4] = {dt / 6.0f, dt / 3.0f, dt / 3.0f, dt / 6.0f};
  const float cy[4] = {0.5f * dt, 0.5f * dt, dt, 0.0f};
  for (int s = 3; s >= 0 && e == cudaSuccess; --s) {
    if (s == 3) {
      axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.rb, A.g, cg[3], 0.0f, x.slot);
      e = last(x);
    } else {
      // rb = cg g + cy y
      e = cudaMemcpyAsync(A.rb, A.y, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) {
        axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.rb, A.g, cg[s], cy[s], x.slot);
        e = last(x);
      }
    }
    if (e == cudaSuccess) e = tendency_vjp(x, w[s], A.rb, learned, dparams);
    if (e != cudaSuccess) break;
    if (s > 0) {
      e = cudaMemcpyAsync(A.y, A.ubar, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = project(x, A.y);
      if (e == cudaSuccess) {
        axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.lam, A.y, 1.0f, 1.0f, x.slot);
        e = last(x);
      }
    } else {
      axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.lam, A.ubar, 1.0f, 1.0f, x.slot);
      e = last(x);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(lam_in, A.lam, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  c->launches = x.launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_step_adjoint (generic grid): %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_gadjoint_tc(fd_ctx* c, const float* const* hist_host, const float* lam, float* vbar, float* hist_bar,
                         size_t state_stride, float* dparams, cudaStream_t st, int* launches) {
  GenericLearned* G = c->glrn;
  if (!G || G->kc == 0)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_tc_adjoint: needs a learned context with a temporal correction");
  if (!G->ready) return fd_set_error(c, FD_EINVAL, "fd_tc_adjoint: learned parameters not set (fd_set_params)");
  if (!c->gadj) {
    const fd_status s = gadjoint_alloc(c);
    if (s != FD_OK) return s;
  }
  Ctx x{c, *c->gadj, st};
  x.B = c->grid.batch;
  x.nx = c->grid.nx;
  x.ny = c->grid.ny;
  x.hw = x.nx * x.ny;
  x.slot = (size_t)x.B * 2 * x.hw;
  GenAdjoint& A = x.A;
  cudaError_t e = refresh_wt(x);
  // vbar = P(lam), cbar = vbar - mean(vbar) (into A.rb)
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.g, lam, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = project(x, A.g);
  if (e == cudaSuccess && vbar) e = cudaMemcpyAsync(vbar, A.g, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    mean_free_kernel<<<(unsigned)(x.B * 2), 256, 0, st>>>(A.g, A.rb, x.hw);
    e = last(x);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(A.d_hist, hist_host, sizeof(const float*) * G->kc, cudaMemcpyHostToDevice, st);
  // forward of the correction network on the history, keeping its pre-activations
  if (e == cudaSuccess) {
    e = run_net(c, A.d_hist, nullptr, nullptr, 2 * G->kc, G->off_tw, G->off_tb, 2, A.y, st, A.zsave);
    x.launches += 6;
  }
  if (e == cudaSuccess)
    e = net_backward(x, A.rb, 2, 2 * G->kc, nullptr, A.d_hist, nullptr, G->off_tw, G->off_tb, A.off_wt_t, dparams,
                     nullptr, nullptr, hist_bar, 0, state_stride);
  *launches += x.launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_tc_adjoint (generic grid): %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_gadjoint_step_scalar(fd_ctx* c, double diff, const float* u_in, const float* s_in, const float* lam_u_out,
                                  const float* lam_s_out, float* lam_u_in, float* lam_s_in, float* dparams,
                                  cudaStream_t st) {
  const char* who = "fd_step_adjoint_scalar";
  if (!c->gen)
    return fd_set_error(c, FD_EUNSUPPORTED, "%s: the passive scalar runs on the generic-grid path (path 3)", who);
  if (c->grid.dtype != FD_F32) return fd_set_error(c, FD_EUNSUPPORTED, "%s: built for FP32", who);
  GenericLearned* G = c->glrn;
  if (G && !G->scalar)
    return fd_set_error(c, FD_EUNSUPPORTED, "%s: the learned model does not read the scalar (scalar_learned = 0)", who);
  if (G && !G->ready) return fd_set_error(c, FD_EINVAL, "%s: learned parameters not set (fd_set_params)", who);
  if (dparams && !G) return fd_set_error(c, FD_EINVAL, "%s: dparams needs a learned context", who);
  if (!(diff >= 0) || !std::isfinite(diff)) return fd_set_error(c, FD_EINVAL, "%s: the diffusivity must be >= 0", who);
  if (!c->gadj) {
    const fd_status r = gadjoint_alloc(c);
    if (r != FD_OK) return r;
  }
  if (!c->gadj->joint) {
    const fd_status r = gadjoint_alloc_joint(c);
    if (r != FD_OK) return r;
  }
  Ctx x{c, *c->gadj, st};
  x.B = c->grid.batch;
  x.nx = c->grid.nx;
  x.ny = c->grid.ny;
  x.hw = x.nx * x.ny;
  x.slot = (size_t)x.B * 2 * x.hw;
  const size_t sslot = (size_t)x.B * x.hw;
  GenAdjoint& A = x.A;
  const bool learned = G != nullptr;
  const float dt = (float)c->dt, fd = (float)diff;
  const float* w[4] = {u_in, A.w[1], A.w[2], A.w[3]};
  const float* z[4] = {s_in, A.z[1], A.z[2], A.z[3]};
  cudaError_t e = learned ? refresh_wt(x) : cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.d_wptr, w, sizeof w, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.d_zptr, z, sizeof z, cudaMemcpyHostToDevice, st);
  // forward: the stage states (w_s, z_s), s = 1, 2, 3
  for (int s = 0; s < 3 && e == cudaSuccess; ++s)
    e = stage_forward_joint(x, s, w[s], z[s], u_in, s_in, A.w[s + 1], A.z[s + 1], learned, fd);
  // reverse: g = P(lam_u_out); the scalar is not projected
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.g, lam_u_out, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = project(x, A.g);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.lam, A.g, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.ls0, lam_s_out, sslot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A.lams, lam_s_out, sslot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  const float cg[4] = {dt / 6.0f, dt / 3.0f, dt / 3.0f, dt / 6.0f};
  const float cy[4] = {0.5f * dt, 0.5f * dt, dt, 0.0f};
  for (int s = 3; s >= 0 && e == cudaSuccess; --s) {
    // tendency cotangents: cg g + cy P(wbar_{s+1}) and cg lam_s + cy zbar_{s+1}
    if (s == 3) {
      axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.rb, A.g, cg[3], 0.0f, x.slot);
      axpby_kernel<<<grid1(sslot), 256, 0, st>>>(A.qb, A.ls0, cg[3], 0.0f, sslot);
    } else {
      axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.y, A.g, cg[s], cy[s], x.slot);  // y <- cg g + cy y
      axpby_kernel<<<grid1(sslot), 256, 0, st>>>(A.ys, A.ls0, cg[s], cy[s], sslot);
    }
    e = last(x);
    if (e == cudaSuccess) e = last(x);
    if (e != cudaSuccess) break;
    const float* rb = s == 3 ? A.rb : A.y;
    const float* qb = s == 3 ? A.qb : A.ys;
    e = joint_tendency_vjp(x, s, w[s], z[s], rb, qb, learned, fd, dparams);
    if (e != cudaSuccess) break;
    // the scalar stage state's cotangent passes unprojected; the velocity's through P
    axpby_kernel<<<grid1(sslot), 256, 0, st>>>(A.lams, A.zbar, 1.0f, 1.0f, sslot);
    e = last(x);
    if (e == cudaSuccess && s > 0) {
      e = cudaMemcpyAsync(A.y, A.ubar, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = project(x, A.y);
      if (e == cudaSuccess) e = cudaMemcpyAsync(A.ys, A.zbar, sslot * sizeof(float), cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) {
        axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.lam, A.y, 1.0f, 1.0f, x.slot);
        e = last(x);
      }
    } else if (e == cudaSuccess) {
      axpby_kernel<<<grid1(x.slot), 256, 0, st>>>(A.lam, A.ubar, 1.0f, 1.0f, x.slot);
      e = last(x);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(lam_u_in, A.lam, x.slot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lam_s_in, A.lams, sslot * sizeof(float), cudaMemcpyDeviceToDevice, st);
  c->launches = x.launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "%s: %s", who, cudaGetErrorString(e));
  return FD_OK;
}
