// fv_glearned.cuh -- kernels of the learnable module on the generic-grid path,
// shared by its forward pass (fd_glearned.cu) and reverse mode (fd_gadjoint.cu):
// the CUDA-core 3x3 periodic convolution, the per-face kernels and face values
// of the operator instances, the flux assembly with the RK4 combination, the
// temporal correction's mean-free update, and the network driver.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fd_ctx.h"

namespace ldfv {
namespace {

constexpr int kHid = 64;
constexpr int kNCoef = 160;        // the velocity's eight instances x 20 taps
constexpr int kNCoefScalar = 240;  // with the scalar's four instances

// out[b][o][p] = act(bias[o] + sum_{c, dy, dx} W[o][c][dy + 1][dx + 1] in[b][c][p + (dy, dx)])
// with periodic wrap; the input is either one tensor [batch][cin][ny][nx] or
// cin / 2 states [batch][2][ny][nx] given by pointers (the network inputs), the
// last channel then optionally a scalar [batch][ny][nx] given by pointer.
// The reverse mode runs the same kernel as a transposed convolution (weights
// transposed and flipped, no bias) with the epilogue multiplying by GELU' of
// the forward pre-activation, and accumulating or strided output.
struct GConvArgs {
  const float* in;
  const float* const* hist;
  const float* const* sptr;
  const float* w;
  const float* b;        // [cout] or null (no bias)
  float* out;            // [batch][cout][ny][nx]; with ostride > 0 channel c of batch b
                         // sits at out + (c / 2) ostride + (2 b + c % 2) nx ny
  float* zout;           // optional: the pre-activation [batch][cout][ny][nx]
  const float* gz;       // optional: out = acc GELU'(gz) [batch][cout][ny][nx]
  size_t ostride;
  int cin, cout, nx, ny, gelu, accum;
};

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
// d GELU / dx = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_deriv(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// kGCO output channels per thread: 16 on large grids (weights reused by more
// FMAs), 4 on small ones (four times the CTAs, a quarter of each thread's chain);
// kPX pixels per thread (p and p + 256, so each load instruction stays coalesced):
// 2 on grids large enough to keep two CTAs per SM busy, where every broadcast
// weight read then feeds 2 kGCO FMAs
template <int kGCO, int kPX>
__global__ void __launch_bounds__(256) gconv3x3_kernel(const GConvArgs a) {
  extern __shared__ float sw[];  // [cin][9][kGCO]: the block's output channels side by side
  const int co0 = blockIdx.y * kGCO;
  const int nco = min(kGCO, a.cout - co0);
  for (int e = threadIdx.x; e < a.cin * 9 * kGCO; e += blockDim.x) {
    const int o = e % kGCO, ck = e / kGCO;
    sw[e] = o < nco ? a.w[(size_t)(co0 + o) * a.cin * 9 + ck] : 0.f;
  }
  __syncthreads();
  const int hw = a.nx * a.ny;
  const int b = blockIdx.z;
  int pix[kPX], off[kPX][9];
  bool live[kPX];
  bool any = false;
#pragma unroll
  for (int q = 0; q < kPX; ++q) {
    const int p = (blockIdx.x * kPX + q) * blockDim.x + threadIdx.x;
    live[q] = p < hw;
    any |= live[q];
    pix[q] = live[q] ? p : 0;  // a dead pixel reads pixel 0 and stores nothing
    const int y = pix[q] / a.nx, x = pix[q] - y * a.nx;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int yy = (y + dy + a.ny) % a.ny, xx = (x + dx + a.nx) % a.nx;
        off[q][(dy + 1) * 3 + dx + 1] = yy * a.nx + xx;
      }
  }
  if (!any) return;
  float acc[kPX][kGCO];
#pragma unroll
  for (int q = 0; q < kPX; ++q)
#pragma unroll
    for (int o = 0; o < kGCO; ++o) acc[q][o] = (o < nco && a.b) ? a.b[co0 + o] : 0.f;
  for (int c = 0; c < a.cin; ++c) {
    const float* src = !a.hist ? a.in + ((size_t)b * a.cin + c) * hw
                       : a.sptr && c == a.cin - 1 ? a.sptr[0] + (size_t)b * hw
                                                  : a.hist[c >> 1] + ((size_t)b * 2 + (c & 1)) * hw;
    const float4* wc = reinterpret_cast<const float4*>(sw + c * 9 * kGCO);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float v[kPX];
#pragma unroll
      for (int q = 0; q < kPX; ++q) v[q] = src[off[q][k]];
#pragma unroll
      for (int o4 = 0; o4 < kGCO / 4; ++o4) {
        const float4 w4 = wc[k * (kGCO / 4) + o4];
#pragma unroll
        for (int q = 0; q < kPX; ++q) {
          acc[q][4 * o4] = fmaf(w4.x, v[q], acc[q][4 * o4]);
          acc[q][4 * o4 + 1] = fmaf(w4.y, v[q], acc[q][4 * o4 + 1]);
          acc[q][4 * o4 + 2] = fmaf(w4.z, v[q], acc[q][4 * o4 + 2]);
          acc[q][4 * o4 + 3] = fmaf(w4.w, v[q], acc[q][4 * o4 + 3]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kPX; ++q) {
    if (!live[q]) continue;
    const int p = pix[q];
#pragma unroll
    for (int o = 0; o < kGCO; ++o) {
      if (o >= nco) continue;
      const int co = co0 + o;
      const size_t e = ((size_t)b * a.cout + co) * hw + p;
      if (a.zout) a.zout[e] = acc[q][o];
      float v = a.gelu ? gelu_exact(acc[q][o]) : acc[q][o];
      if (a.gz) v *= gelu_deriv(a.gz[e]);
      float* dst = a.ostride ? a.out + (size_t)(co >> 1) * a.ostride + ((size_t)b * 2 + (co & 1)) * hw + p : a.out + e;
      *dst = a.accum ? *dst + v : v;
    }
  }
}

// face values of the eight instances at every output location (instance q =
// 2 pr + kind, pr = (field, axis)); 20 taps on the 5 x 4 grid: transverse
// offset r - 2, axial offset c + sh (sh = -1 or -2 by where the output sits).
// Scalar models add the scalar's four instances m = 2 axis + kind (sh = -2).
struct GFaceArgs {
  const float* w;     // stage state [batch][2][ny][nx]
  const float* coef;  // network output [batch][ncoef][ny][nx], or null (physics kernels alone)
  const float* wl;    // W_L[kind 2][axis 2][5][4] (with coef)
  float* inst;        // [batch][8][ny][nx]
  float* kout;        // optional: the velocity's per-face kernels [batch][ncoef][ny][nx]
                      // (channel 20 q + t; may be coef itself: each cell rewrites its own)
  float* skout;       // optional: the scalar's per-face kernels, channel 160 + 20 m + t of
                      // the same layout
  const float* s;     // stage scalar [batch][ny][nx], or null
  const float* wls;   // W_Ls[kind 2][axis 2][5][4]
  float* sinst;       // [batch][4][ny][nx]
  int nx, ny, dord, ablation, ncoef;
  float idx, idy;
};

// one face value: the learned part L (20 taps) through the consistency
// projection onto the kernels that leave W_P's order conditions intact, scaled
// by 1/h for a derivative, plus W_P (Sec. 3.4), applied to the 20 taps;
// ablation 1 takes L alone, without W_P or the projection
__device__ __forceinline__ float face_value(const float (&L)[20], const float (&tap)[20], int kind, float h, int dord,
                                            int ablation, float* kout = nullptr, size_t kstride = 0) {
  const float cval[4] = {-1.5f, -0.5f, 0.5f, 1.5f};
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
  const float pk = ablation == 0 ? 1.0f : 0.0f;
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
      if (r == 2 && ablation == 0) {
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
      if (kout) kout[(size_t)(r * 4 + cc) * kstride] = k;
      val += k * tap[r * 4 + cc];
    }
  return val;
}

__global__ void __launch_bounds__(256) gface_kernel(const GFaceArgs a) {
  const int hw = a.nx * a.ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / a.nx, i = p - j * a.nx;
  const float* fu = a.w + (size_t)b * 2 * hw;
  const float* cf = a.coef ? a.coef + (size_t)b * a.ncoef * hw + p : nullptr;
#pragma unroll 1
  for (int pr = 0; pr < 4; ++pr) {
    const int fld = pr >> 1, axis = pr & 1;
    const int sh = (pr == 0 || pr == 3) ? -1 : -2;
    const float* f = fu + (size_t)fld * hw;
    float tap[20];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int jj = axis == 0 ? j + r - 2 : j + cc + sh;
        const int ii = axis == 0 ? i + cc + sh : i + r - 2;
        tap[r * 4 + cc] = f[((jj + a.ny) % a.ny) * a.nx + (ii + a.nx) % a.nx];
      }
    const float h = axis == 0 ? 1.0f / a.idx : 1.0f / a.idy;
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const int q = 2 * pr + kind;
      float L[20];
#pragma unroll
      for (int t = 0; t < 20; ++t) L[t] = cf ? a.wl[(kind * 2 + axis) * 20 + t] + cf[(size_t)(q * 20 + t) * hw] : 0.f;
      float* ko = a.kout ? a.kout + ((size_t)b * a.ncoef + q * 20) * hw + p : nullptr;
      a.inst[((size_t)b * 8 + q) * hw + p] = face_value(L, tap, kind, h, a.dord, a.ablation, ko, hw);
    }
  }
  if (!a.s) return;
  const float* fs = a.s + (size_t)b * hw;
#pragma unroll 1
  for (int axis = 0; axis < 2; ++axis) {
    float tap[20];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int jj = axis == 0 ? j + r - 2 : j + cc - 2;
        const int ii = axis == 0 ? i + cc - 2 : i + r - 2;
        tap[r * 4 + cc] = fs[((jj + a.ny) % a.ny) * a.nx + (ii + a.nx) % a.nx];
      }
    const float h = axis == 0 ? 1.0f / a.idx : 1.0f / a.idy;
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const int m = 2 * axis + kind;
      float L[20];
#pragma unroll
      for (int t = 0; t < 20; ++t)
        L[t] = cf ? a.wls[(kind * 2 + axis) * 20 + t] + cf[(size_t)(kNCoef + m * 20 + t) * hw] : 0.f;
      float* ko = a.skout ? a.skout + ((size_t)b * a.ncoef + kNCoef + m * 20) * hw + p : nullptr;
      a.sinst[((size_t)b * 4 + m) * hw + p] = face_value(L, tap, kind, h, a.dord, 0, ko, hw);
    }
  }
}

// flux assembly + divergence (App. B.2) from the face values, Burgers
// correction, forcing, and the RK4 combination (App. B.5); scalar models also
// the scalar's flux-form tendency -div(u s_f - D grad_f s) from the stage
// velocity and its RK4 combination
struct GStageArgs {
  const float* inst;  // [batch][8][ny][nx]
  const float* w;     // stage state
  const float* un;    // state at the start of the step
  float* acc;         // RK4 accumulator
  float* wout;        // next stage state (stage 3: the new state)
  const float* frc;   // [ny]
  const float* sinst; // the scalar's face values [batch][4][ny][nx], or null
  const float* sn;    // scalar at the start of the step [batch][ny][nx]
  float* sacc;        // its RK4 accumulator
  float* sout;        // next stage scalar
  int nx, ny, stage, forced, burgers;
  float dt, nu, idx, idy, drag, diff;
};

__device__ __forceinline__ void rk4_combine(int stage, float r, float dt, const float* un, float* acc, float* out,
                                            size_t e) {
  const float h6 = dt / 6.0f, h3 = dt / 3.0f, h2 = dt * 0.5f;
  switch (stage) {
    case 0: {
      const float u0 = un[e];
      acc[e] = u0 + h6 * r;
      out[e] = u0 + h2 * r;
      break;
    }
    case 1:
      acc[e] += h3 * r;
      out[e] = un[e] + h2 * r;
      break;
    case 2:
      acc[e] += h3 * r;
      out[e] = un[e] + dt * r;
      break;
    default:
      out[e] = acc[e] + h6 * r;
  }
}

__global__ void __launch_bounds__(256) gstage_kernel(const GStageArgs a) {
  const int hw = a.nx * a.ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.y;
  const int j = p / a.nx, i = p - j * a.nx;
  const int jn = (j + 1) % a.ny, js = (j - 1 + a.ny) % a.ny;
  const int ie = (i + 1) % a.nx, iw = (i - 1 + a.nx) % a.nx;
  const float* I = a.inst + (size_t)b * 8 * hw;
  auto at = [&](int q, int jj, int ii) { return I[(size_t)q * hw + jj * a.nx + ii]; };
  const float Uc = at(0, j, i), Ucw = at(0, j, iw);
  const float Gxc = at(1, j, i), Gxcw = at(1, j, iw);
  const float Uk = at(2, j, i), Ukn = at(2, jn, i), Uke = at(2, j, ie);
  const float Gyu = at(3, j, i), Gyun = at(3, jn, i);
  const float Vk = at(4, j, i), Vkn = at(4, jn, i), Vke = at(4, j, ie);
  const float Gxv = at(5, j, i), Gxve = at(5, j, ie);
  const float Vc = at(6, j, i), Vcs = at(6, js, i);
  const float Gyc = at(7, j, i), Gycs = at(7, js, i);
  float tu = -(Uc * Uc - Ucw * Ucw) * a.idx - (Ukn * Vkn - Uk * Vk) * a.idy +
             a.nu * ((Gxc - Gxcw) * a.idx + (Gyun - Gyu) * a.idy);
  float tv = -(Uke * Vke - Uk * Vk) * a.idx - (Vc * Vc - Vcs * Vcs) * a.idy +
             a.nu * ((Gxve - Gxv) * a.idx + (Gyc - Gycs) * a.idy);
  const size_t e = (size_t)b * 2 * hw + p;
  const float uc = a.w[e], vc = a.w[e + hw];
  if (a.burgers) {
    const float d0 = Gxc + Gyc;
    tu += uc * 0.5f * ((Gxcw + at(7, j, iw)) + d0);
    tv += vc * 0.5f * ((at(1, js, i) + Gycs) + d0);
  }
  if (a.forced) {
    tu += a.frc[j] - a.drag * uc;
    tv += -a.drag * vc;
  }
  rk4_combine(a.stage, tu, a.dt, a.un, a.acc, a.wout, e);
  rk4_combine(a.stage, tv, a.dt, a.un, a.acc, a.wout, e + hw);
  if (!a.sinst) return;
  // F_x on the west face of a cell (u there), F_y on its south face (v there)
  const float* SI = a.sinst + (size_t)b * 4 * hw;
  const float* wu = a.w + (size_t)b * 2 * hw;
  const float* wv = wu + hw;
  auto fx = [&](int q) { return wu[q] * SI[q] - a.diff * SI[hw + q]; };
  auto fy = [&](int q) { return wv[q] * SI[2 * hw + q] - a.diff * SI[3 * hw + q]; };
  const float ts = -(fx(j * a.nx + ie) - fx(p)) * a.idx - (fy(jn * a.nx + i) - fy(p)) * a.idy;
  rk4_combine(a.stage, ts, a.dt, a.sn, a.sacc, a.sout, (size_t)b * hw + p);
}

// u += c - mean(c), per trajectory and component (one CTA each)
__global__ void __launch_bounds__(256) gtc_apply_kernel(float* u, const float* corr, int hw) {
  const size_t base = (size_t)blockIdx.x * hw;
  __shared__ double red[8];
  double s = 0.0;
  for (int k = threadIdx.x; k < hw; k += blockDim.x) s += corr[base + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double m = 0.0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m += red[k];
  const float mean = (float)(m / hw);
  for (int k = threadIdx.x; k < hw; k += blockDim.x) u[base + k] += corr[base + k] - mean;
}

__global__ void round_bf16_kernel(float* v, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    v[k] = __bfloat162float(__float2bfloat16_rn(v[k]));
}

inline int stencil_cin(int l, bool scalar) { return l == 0 ? (scalar ? 3 : 2) : kHid; }
inline int stencil_cout(int l, bool scalar) { return l == 5 ? (scalar ? kNCoefScalar : kNCoef) : kHid; }

template <int GCO, int PX = 1>
cudaError_t launch_gconv(const GConvArgs& a, int batch, cudaStream_t st) {
  const int hw = a.nx * a.ny;
  const dim3 grid((unsigned)((hw + 256 * PX - 1) / (256 * PX)), (unsigned)((a.cout + GCO - 1) / GCO), (unsigned)batch);
  gconv3x3_kernel<GCO, PX><<<grid, 256, (size_t)a.cin * 9 * GCO * sizeof(float), st>>>(a);
  return cudaGetLastError();
}

// the variant for a layer: 4 channels per thread below two CTAs per SM at 16, or
// with more than 64 input channels (the 16-channel weights would pass 48 KB of
// shared memory); two pixels per thread where that still leaves two CTAs per SM
inline cudaError_t launch_gconv_auto(const GConvArgs& a, int batch, cudaStream_t st) {
  const size_t ctas16 = (size_t)((a.nx * a.ny + 255) / 256) * ((a.cout + 15) / 16) * batch;
  if (ctas16 < 304 || a.cin > 64) return launch_gconv<4>(a, batch, st);
  if (ctas16 >= 4 * 304) return launch_gconv<16, 2>(a, batch, st);
  return launch_gconv<16>(a, batch, st);
}

// one network (six layers) into `out` (cout5 channels) from cin0 channels: the
// state(s) behind `in_ptrs` (and, with `s_ptrs`, a scalar as the last channel),
// or the tensor `in0` [batch][cin0][ny][nx]; hidden activations in act0 / act1.
// With `zsave` (five [batch][64][ny][nx] buffers) the pre-activations of the
// five hidden layers are kept for the reverse mode.
cudaError_t run_net(fd_ctx* c, const float* const* in_ptrs, const float* const* s_ptrs, const float* in0, int cin0,
                    const size_t* off_w, const size_t* off_b, int cout5, float* out, cudaStream_t st,
                    float* const* zsave = nullptr) {
  GenericLearned& G = *c->glrn;
  const int nx = c->grid.nx, ny = c->grid.ny, B = c->grid.batch;
  const float* in = in0;
  for (int l = 0; l < 6; ++l) {
    GConvArgs a = {};
    a.cin = l == 0 ? cin0 : kHid;
    a.cout = l == 5 ? cout5 : kHid;
    a.hist = l == 0 ? in_ptrs : nullptr;
    a.sptr = l == 0 ? s_ptrs : nullptr;
    a.in = in;
    a.w = G.d_params + off_w[l];
    a.b = G.d_params + off_b[l];
    a.out = l == 5 ? out : (l % 2 == 0 ? G.act0 : G.act1);
    a.nx = nx;
    a.ny = ny;
    a.gelu = l < 5;
    a.zout = (zsave && l < 5) ? zsave[l] : nullptr;
    cudaError_t e = launch_gconv_auto(a, B, st);
    if (e != cudaSuccess) return e;
    in = a.out;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace ldfv
