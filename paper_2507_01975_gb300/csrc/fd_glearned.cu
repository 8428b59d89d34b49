// fd_glearned.cu -- the learnable module on the generic-grid path: learned
// contexts on any grid the tensor-core path does not take (non-power-of-two
// and rectangular Burgers grids such as the 25^2 and 100^2 presets of App. C.1,
// rectangular Navier-Stokes grids such as the 128 x 64 shear-flow grid, square
// grids other than 32^2 and 64^2, or any grid with path 3), FP32.
//
// One learned RK stage (Sec. 3.2, 3.4):
//   * the stencil network C_theta (six 3x3 periodic convolutions, 2 -> 64 x 5 ->
//     160, GELU between them) on CUDA cores, FP32 activations, weights rounded
//     to BF16 at upload like the tensor-core path's;
//   * the face values of the eight operator instances with the per-face kernels
//     K_f = W_P + proj(W_L + C_theta(w)_f) / h^deriv (consistency projection;
//     ablation 1 drops W_P and the projection), one thread per cell;
//   * flux assembly, divergence, Burgers correction, forcing and the RK
//     combination (App. B.2, B.5), one thread per cell;
//   * for Navier-Stokes the generic path's spectral projection (Sec. 3.6).
// Every k_c steps the temporal-correction network (2 k_c -> 64 x 5 -> 2) on the
// last k_c states gives c, and u <- P(u + c - mean(c)) (Sec. 3.2, 3.5).
// A rollout captures one group of max(k_c, 1) steps as a CUDA graph and replays it.
//
// A model that learns the passive scalar of the shear flow (App. C.1) extends
// the flux block to the scalar's four operator instances (face value and face
// derivative along x at the u-faces and along y at the v-faces) with per-face
// kernels W_P + proj(W_Ls + C_s) / h^deriv of their own; the network then reads
// (u, v, s) and emits 240 channels, the last 80 being C_s, and each stage also
// advances s by -div(u s_f - D grad_f s) (flux form; the temporal correction
// stays on the velocity).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"

using namespace ldfv;

namespace {

constexpr int kHid = 64;
constexpr int kNCoef = 160;        // the velocity's eight instances x 20 taps
constexpr int kNCoefScalar = 240;  // with the scalar's four instances

// out[b][o][p] = act(bias[o] + sum_{c, dy, dx} W[o][c][dy + 1][dx + 1] in[b][c][p + (dy, dx)])
// with periodic wrap; the input is either one tensor [batch][cin][ny][nx] or
// cin / 2 states [batch][2][ny][nx] given by pointers (the network inputs), the
// last channel then optionally a scalar [batch][ny][nx] given by pointer
struct GConvArgs {
  const float* in;
  const float* const* hist;
  const float* const* sptr;
  const float* w;
  const float* b;
  float* out;
  int cin, cout, nx, ny, gelu;
};

__device__ __forceinline__ float gelu_exact(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// GCO output channels per thread: 16 on large grids (weights reused by more
// FMAs), 4 on small ones (four times the CTAs, a quarter of each thread's chain)
template <int kGCO>
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
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  const int b = blockIdx.z;
  const int y = p / a.nx, x = p - y * a.nx;
  int off[9];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int yy = (y + dy + a.ny) % a.ny, xx = (x + dx + a.nx) % a.nx;
      off[(dy + 1) * 3 + dx + 1] = yy * a.nx + xx;
    }
  float acc[kGCO];
#pragma unroll
  for (int o = 0; o < kGCO; ++o) acc[o] = o < nco ? a.b[co0 + o] : 0.f;
  for (int c = 0; c < a.cin; ++c) {
    const float* src = !a.hist ? a.in + ((size_t)b * a.cin + c) * hw
                       : a.sptr && c == a.cin - 1 ? a.sptr[0] + (size_t)b * hw
                                                  : a.hist[c >> 1] + ((size_t)b * 2 + (c & 1)) * hw;
    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = src[off[k]];
    const float4* wc = reinterpret_cast<const float4*>(sw + c * 9 * kGCO);
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int o4 = 0; o4 < kGCO / 4; ++o4) {
        const float4 w4 = wc[k * (kGCO / 4) + o4];
        acc[4 * o4] = fmaf(w4.x, v[k], acc[4 * o4]);
        acc[4 * o4 + 1] = fmaf(w4.y, v[k], acc[4 * o4 + 1]);
        acc[4 * o4 + 2] = fmaf(w4.z, v[k], acc[4 * o4 + 2]);
        acc[4 * o4 + 3] = fmaf(w4.w, v[k], acc[4 * o4 + 3]);
      }
  }
#pragma unroll
  for (int o = 0; o < kGCO; ++o)
    if (o < nco) a.out[((size_t)b * a.cout + co0 + o) * hw + p] = a.gelu ? gelu_exact(acc[o]) : acc[o];
}

// face values of the eight instances at every output location (instance q =
// 2 pr + kind, pr = (field, axis)); 20 taps on the 5 x 4 grid: transverse
// offset r - 2, axial offset c + sh (sh = -1 or -2 by where the output sits).
// Scalar models add the scalar's four instances m = 2 axis + kind (sh = -2).
struct GFaceArgs {
  const float* w;     // stage state [batch][2][ny][nx]
  const float* coef;  // network output [batch][ncoef][ny][nx]
  const float* wl;    // W_L[kind 2][axis 2][5][4]
  float* inst;        // [batch][8][ny][nx]
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
                                            int ablation) {
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
  const float* cf = a.coef + (size_t)b * a.ncoef * hw + p;
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
      for (int t = 0; t < 20; ++t) L[t] = a.wl[(kind * 2 + axis) * 20 + t] + cf[(size_t)(q * 20 + t) * hw];
      a.inst[((size_t)b * 8 + q) * hw + p] = face_value(L, tap, kind, h, a.dord, a.ablation);
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
        L[t] = a.wls[(kind * 2 + axis) * 20 + t] + cf[(size_t)(kNCoef + m * 20 + t) * hw];
      a.sinst[((size_t)b * 4 + m) * hw + p] = face_value(L, tap, kind, h, a.dord, 0);
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

int stencil_cin(int l, bool scalar) { return l == 0 ? (scalar ? 3 : 2) : kHid; }
int stencil_cout(int l, bool scalar) { return l == 5 ? (scalar ? kNCoefScalar : kNCoef) : kHid; }

template <int GCO>
cudaError_t launch_gconv(const GConvArgs& a, int batch, cudaStream_t st) {
  const int hw = a.nx * a.ny;
  const dim3 grid((unsigned)((hw + 255) / 256), (unsigned)((a.cout + GCO - 1) / GCO), (unsigned)batch);
  gconv3x3_kernel<GCO><<<grid, 256, (size_t)a.cin * 9 * GCO * sizeof(float), st>>>(a);
  return cudaGetLastError();
}

// one network (six layers) into `out` (cout5 channels) from cin0 channels: the
// state(s) behind `in_ptrs` (and, with `s_ptrs`, a scalar as the last channel),
// or the tensor `in0` [batch][cin0][ny][nx]; hidden activations in act0 / act1
cudaError_t run_net(fd_ctx* c, const float* const* in_ptrs, const float* const* s_ptrs, const float* in0, int cin0,
                    const size_t* off_w, const size_t* off_b, int cout5, float* out, cudaStream_t st) {
  GenericLearned& G = *c->glrn;
  const int nx = c->grid.nx, ny = c->grid.ny, B = c->grid.batch;
  const int hw = nx * ny;
  const float* in = in0;
  for (int l = 0; l < 6; ++l) {
    GConvArgs a;
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
    // fewer than two CTAs per SM with 16 channels per thread: 4 per thread
    const size_t ctas16 = (size_t)((hw + 255) / 256) * ((a.cout + 15) / 16) * B;
    cudaError_t e = ctas16 < 304 ? launch_gconv<4>(a, B, st) : launch_gconv<16>(a, B, st);
    if (e != cudaSuccess) return e;
    in = a.out;
  }
  return cudaSuccess;
}

// one learned step of the state in the generic-grid buffers (S.un in place);
// scalar models also advance the scalar (S.sn in place) with diffusivity diff
cudaError_t learned_step(fd_ctx* c, cudaStream_t st, float diff = 0.f) {
  GenericState& S = *c->gen;
  GenericLearned& G = *c->glrn;
  const fd_grid& g = c->grid;
  const int hw = g.nx * g.ny;
  float* const un = static_cast<float*>(S.un);
  float* const stage_out[4] = {static_cast<float*>(S.wa), static_cast<float*>(S.wb), static_cast<float*>(S.wa), un};
  const float* const stage_in[4] = {un, static_cast<float*>(S.wa), static_cast<float*>(S.wb),
                                    static_cast<float*>(S.wa)};
  float* const s_out[4] = {static_cast<float*>(S.sa), static_cast<float*>(S.sb), static_cast<float*>(S.sa),
                           static_cast<float*>(S.sn)};
  const float* const s_in[4] = {static_cast<float*>(S.sn), static_cast<float*>(S.sa), static_cast<float*>(S.sb),
                                static_cast<float*>(S.sa)};
  const dim3 cells((unsigned)((hw + 255) / 256), (unsigned)g.batch);
  const float idx = (float)(g.nx / g.lx), idy = (float)(g.ny / g.ly);
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
    // the network reads its input through one-entry pointer arrays: stage 0
    // reads u_n (and s_n), stages 1 and 3 the first stage buffers, stage 2 the second
    const int slot = s == 0 ? 0 : s == 2 ? 2 : 1;
    e = run_net(c, G.d_single + slot, G.scalar ? G.d_ssingle + slot : nullptr, nullptr, G.scalar ? 3 : 2, G.off_sw,
                G.off_sb, G.ncoef, G.coef, st);
    if (e != cudaSuccess) break;
    GFaceArgs fa;
    fa.w = stage_in[s];
    fa.coef = G.coef;
    fa.wl = G.d_params + G.off_wl;
    fa.inst = G.inst;
    fa.s = G.scalar ? s_in[s] : nullptr;
    fa.wls = G.d_params + G.off_wls;
    fa.sinst = G.sinst;
    fa.nx = g.nx;
    fa.ny = g.ny;
    fa.dord = c->opts.deriv_order;
    fa.ablation = G.ablation;
    fa.ncoef = G.ncoef;
    fa.idx = idx;
    fa.idy = idy;
    gface_kernel<<<cells, 256, 0, st>>>(fa);
    GStageArgs sa;
    sa.inst = G.inst;
    sa.w = stage_in[s];
    sa.un = un;
    sa.acc = static_cast<float*>(S.acc);
    sa.wout = stage_out[s];
    sa.frc = static_cast<const float*>(S.frc);
    sa.sinst = G.scalar ? G.sinst : nullptr;
    sa.sn = static_cast<const float*>(S.sn);
    sa.sacc = static_cast<float*>(S.sacc);
    sa.sout = s_out[s];
    sa.diff = diff;
    sa.nx = g.nx;
    sa.ny = g.ny;
    sa.stage = s;
    sa.forced = c->forcing.kind;
    sa.burgers = g.flow == FD_BURGERS;
    sa.dt = (float)c->dt;
    sa.nu = (float)c->nu;
    sa.idx = idx;
    sa.idy = idy;
    sa.drag = (float)(c->forcing.kind == 1 ? c->forcing.drag : 0.0);
    gstage_kernel<<<cells, 256, 0, st>>>(sa);
    e = cudaGetLastError();
    if (e == cudaSuccess && g.flow == FD_NAVIER_STOKES) e = fd_generic_project(c, stage_out[s], st);
  }
  return e;
}

// u <- P(u + c - mean(c)), c = the correction network on the ring's k_c states
cudaError_t correct(fd_ctx* c, cudaStream_t st) {
  GenericState& S = *c->gen;
  GenericLearned& G = *c->glrn;
  const fd_grid& g = c->grid;
  cudaError_t e = run_net(c, G.d_hist, nullptr, nullptr, 2 * G.kc, G.off_tw, G.off_tb, 2, G.corr, st);
  if (e != cudaSuccess) return e;
  gtc_apply_kernel<<<(unsigned)(g.batch * 2), 256, 0, st>>>(static_cast<float*>(S.un), G.corr, g.nx * g.ny);
  e = cudaGetLastError();
  if (e == cudaSuccess && g.flow == FD_NAVIER_STOKES) e = fd_generic_project(c, static_cast<float*>(S.un), st);
  return e;
}

int launches_per_step(const fd_ctx* c) { return 4 * (6 + 2 + (c->grid.flow == FD_NAVIER_STOKES ? 5 : 0)); }

}  // namespace

fd_status fd_glearned_check(const fd_grid& g, const fd_options& o) {
  if (g.dtype != FD_F32) return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: the learned module is built for FP32");
  if (o.fno_layers != 0 || o.tc_fno_layers != 0)
    return fd_set_error(nullptr, FD_EUNSUPPORTED,
                        "fd_init: the Fourier operators of the learned module are built for the 32^2 and 64^2 "
                        "tensor-core path");
  if (o.ablation != 0 && o.ablation != 1)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: ablation must be 0 or 1 (the O_F-only variant needs the Fourier operator)");
  if (o.k_c < 0 || o.k_c > 8) return fd_set_error(nullptr, FD_EINVAL, "fd_init: k_c must be in [0, 8]");
  if (o.scalar_learned && o.ablation != 0)
    return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: a model that learns the scalar is built for the full operator");
  return FD_OK;
}

fd_status fd_glearned_init(fd_ctx* c) {
  GenericLearned* G = new (std::nothrow) GenericLearned();
  if (!G) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: out of host memory");
  c->glrn = G;
  const fd_grid& g = c->grid;
  G->kc = c->opts.k_c;
  G->ablation = c->opts.ablation;
  G->scalar = c->opts.scalar_learned != 0;
  G->ncoef = G->scalar ? kNCoefScalar : kNCoef;
  G->nparams = fd_learned_param_count(c->opts);
  size_t off = 0;
  G->off_wl = off;
  off += 80;
  if (G->scalar) {
    G->off_wls = off;
    off += 80;
  }
  for (int l = 0; l < 6; ++l) {
    G->off_sw[l] = off;
    off += (size_t)stencil_cout(l, G->scalar) * stencil_cin(l, G->scalar) * 9;
    G->off_sb[l] = off;
    off += stencil_cout(l, G->scalar);
  }
  for (int l = 0; l < 6 && G->kc > 0; ++l) {
    const int ci = l == 0 ? 2 * G->kc : kHid, co = l == 5 ? 2 : kHid;
    G->off_tw[l] = off;
    off += (size_t)co * ci * 9;
    G->off_tb[l] = off;
    off += co;
  }
  if ((int64_t)off != G->nparams)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: learned parameter layout mismatch (%lld vs %lld)",
                        (long long)off, (long long)G->nparams);
  const size_t hw = (size_t)g.nx * g.ny, B = g.batch;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&G->d_params, (size_t)G->nparams * sizeof(float));
  alloc((void**)&G->act0, B * kHid * hw * sizeof(float));
  alloc((void**)&G->act1, B * kHid * hw * sizeof(float));
  alloc((void**)&G->coef, B * G->ncoef * hw * sizeof(float));
  alloc((void**)&G->inst, B * 8 * hw * sizeof(float));
  alloc((void**)&G->d_single, 4 * sizeof(const float*));
  if (e == cudaSuccess) {
    // the stage inputs u_n, first and second stage buffers, and a slot for fd_network_forward
    const float* h[4] = {static_cast<const float*>(c->gen->un), static_cast<const float*>(c->gen->wa),
                         static_cast<const float*>(c->gen->wb), nullptr};
    e = cudaMemcpy(G->d_single, h, sizeof h, cudaMemcpyHostToDevice);
  }
  if (G->scalar) {
    // the scalar's state, stage buffers and accumulator (those fd_rollout_scalar
    // otherwise allocates on its first call), its face values and input pointers
    GenericState& S = *c->gen;
    for (void** q : {&S.sn, &S.sa, &S.sb, &S.sacc}) alloc(q, B * hw * sizeof(float));
    alloc((void**)&G->sinst, B * 4 * hw * sizeof(float));
    alloc((void**)&G->d_ssingle, 4 * sizeof(const float*));
    if (e == cudaSuccess) {
      const float* h[4] = {static_cast<const float*>(S.sn), static_cast<const float*>(S.sa),
                           static_cast<const float*>(S.sb), nullptr};
      e = cudaMemcpy(G->d_ssingle, h, sizeof h, cudaMemcpyHostToDevice);
    }
  }
  if (G->kc > 0) {
    alloc((void**)&G->corr, B * 2 * hw * sizeof(float));
    alloc((void**)&G->ring, (size_t)G->kc * B * 2 * hw * sizeof(float));
    alloc((void**)&G->d_hist, (size_t)G->kc * sizeof(const float*));
    if (e == cudaSuccess) {
      std::vector<const float*> h(G->kc);
      for (int s = 0; s < G->kc; ++s) h[s] = G->ring + (size_t)s * B * 2 * hw;
      e = cudaMemcpy(G->d_hist, h.data(), h.size() * sizeof(const float*), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: learned workspace: %s", cudaGetErrorString(e));
  return FD_OK;
}

void fd_glearned_free(fd_ctx* c) {
  GenericLearned* G = c->glrn;
  if (!G) return;
  if (G->graph) cudaGraphExecDestroy(G->graph);
  void* ps[] = {G->d_params, G->act0, G->act1, G->coef, G->inst, G->sinst, G->corr, G->ring, (void*)G->d_hist,
                (void*)G->d_single, (void*)G->d_ssingle};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete G;
  c->glrn = nullptr;
}

fd_status fd_glearned_set_params(fd_ctx* c, const float* params, int64_t count, bool device, cudaStream_t st) {
  GenericLearned& G = *c->glrn;
  const char* who = device ? "fd_set_params_device" : "fd_set_params";
  if (count != G.nparams)
    return fd_set_error(c, FD_EINVAL, "%s: expected %lld values, got %lld", who, (long long)G.nparams, (long long)count);
  cudaError_t e = cudaMemcpyAsync(G.d_params, params, (size_t)count * sizeof(float),
                                  device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  // the convolution weights (not the biases or W_L) in BF16, as on the tensor cores
  for (int l = 0; l < 6 && e == cudaSuccess; ++l) {
    const size_t n = G.off_sb[l] - G.off_sw[l];
    round_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G.d_params + G.off_sw[l], n);
    e = cudaGetLastError();
    if (e == cudaSuccess && G.kc > 0) {
      const size_t nt = G.off_tb[l] - G.off_tw[l];
      round_bf16_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(G.d_params + G.off_tw[l], nt);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && !device) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "%s: %s", who, cudaGetErrorString(e));
  G.ready = true;
  return FD_OK;
}

fd_status fd_glearned_network(fd_ctx* c, const void* u, float* coef_out, cudaStream_t st) {
  GenericLearned& G = *c->glrn;
  const float* in = static_cast<const float*>(u);
  cudaError_t e = cudaSuccess;
  if (G.scalar) {  // (u, v, s) as one tensor [batch][3][ny][nx]
    e = run_net(c, nullptr, nullptr, in, 3, G.off_sw, G.off_sb, G.ncoef, coef_out ? coef_out : G.coef, st);
  } else {
    e = cudaMemcpyAsync(G.d_single + 3, &in, sizeof(const float*), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = run_net(c, G.d_single + 3, nullptr, nullptr, 2, G.off_sw, G.off_sb, kNCoef, coef_out ? coef_out : G.coef, st);
  }
  c->launches = 6;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_network_forward: %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_glearned_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                              cudaStream_t st, bool allow_graph) {
  GenericState& S = *c->gen;
  GenericLearned& G = *c->glrn;
  if (G.scalar)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_rollout: the model reads the passive scalar (use fd_rollout_scalar)");
  if (!G.ready) return fd_set_error(c, FD_EINVAL, "fd_rollout: learned parameters not set (fd_set_params)");
  const size_t bytes = fd_state_bytes(c->grid);
  const size_t slot = bytes / sizeof(float);
  const int grp = G.kc > 0 ? G.kc : 1;
  // step k (1-based): ring slot (k - 1) mod k_c takes u_{k-1}; at k = M k_c the
  // slots hold u_{k-k_c} .. u_{k-1} in slot order and the correction follows.
  // A group of k_c steps (one step without the correction) is the same work
  // every time, so it is captured once as a graph and replayed.
  auto step = [&](int k, cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (G.kc > 0) e = cudaMemcpyAsync(G.ring + (size_t)((k - 1) % G.kc) * slot, S.un, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = learned_step(c, s);
    if (e == cudaSuccess && G.kc > 0 && k % G.kc == 0) e = correct(c, s);
    return e;
  };
  const int per_step = launches_per_step(c), per_corr = G.kc > 0 ? 7 + (c->grid.flow == FD_NAVIER_STOKES ? 5 : 0) : 0;
  cudaError_t e = cudaMemcpyAsync(S.un, u0, bytes, cudaMemcpyDeviceToDevice, st);
  const bool use_graph = allow_graph && save_every == 0;
  if (e == cudaSuccess && use_graph && n_steps >= grp && !G.graph) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaSuccess;
      for (int k = 1; k <= grp && e1 == cudaSuccess; ++k) e1 = step(k, S.cap_stream);
      const cudaError_t e2 = cudaStreamEndCapture(S.cap_stream, &g);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.graph, g, 0);
    if (g) cudaGraphDestroy(g);
  }
  int done = 0, snap = 0, launches = 0;
  if (e == cudaSuccess && use_graph && G.graph) {
    for (; done + grp <= n_steps && e == cudaSuccess; done += grp) {
      e = cudaGraphLaunch(G.graph, st);
      launches += grp * per_step + per_corr;
    }
  }
  for (int k = done + 1; k <= n_steps && e == cudaSuccess; ++k) {
    e = step(k, st);
    launches += per_step + (G.kc > 0 && k % G.kc == 0 ? per_corr : 0);
    if (e == cudaSuccess && traj && save_every > 0 && k % save_every == 0) {
      e = cudaMemcpyAsync(static_cast<char*>(traj) + (size_t)snap * bytes, S.un, bytes, cudaMemcpyDeviceToDevice, st);
      ++snap;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, S.un, bytes, cudaMemcpyDeviceToDevice, st);
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout (generic-grid learned): %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_glearned_rollout_scalar(fd_ctx* c, double diff, const void* u0, const void* s0, void* u_final,
                                     void* s_final, int n_steps, cudaStream_t st) {
  GenericState& S = *c->gen;
  GenericLearned& G = *c->glrn;
  if (!G.scalar)
    return fd_set_error(c, FD_EUNSUPPORTED,
                        "fd_rollout_scalar: the learned model does not read the scalar (fd_init with scalar_learned = 1)");
  if (!G.ready) return fd_set_error(c, FD_EINVAL, "fd_rollout_scalar: learned parameters not set (fd_set_params)");
  const size_t bytes = fd_state_bytes(c->grid);
  const size_t slot = bytes / sizeof(float);
  const size_t sbytes = (size_t)c->grid.batch * c->grid.nx * c->grid.ny * sizeof(float);
  const int grp = G.kc > 0 ? G.kc : 1;
  // the velocity's history ring and temporal correction as in the velocity-only rollout
  auto step = [&](int k, cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (G.kc > 0) e = cudaMemcpyAsync(G.ring + (size_t)((k - 1) % G.kc) * slot, S.un, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = learned_step(c, s, (float)diff);
    if (e == cudaSuccess && G.kc > 0 && k % G.kc == 0) e = correct(c, s);
    return e;
  };
  const int per_step = launches_per_step(c), per_corr = G.kc > 0 ? 7 + (c->grid.flow == FD_NAVIER_STOKES ? 5 : 0) : 0;
  cudaError_t e = cudaMemcpyAsync(S.un, u0, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.sn, s0, sbytes, cudaMemcpyDeviceToDevice, st);
  // the diffusivity is a kernel argument: a graph captured with another one is replaced
  if (e == cudaSuccess && n_steps >= grp && (!G.graph || G.graph_diff != diff)) {
    if (G.graph) {
      e = cudaStreamSynchronize(st);
      if (e == cudaSuccess) e = cudaGraphExecDestroy(G.graph);
      G.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaSuccess;
      for (int k = 1; k <= grp && e1 == cudaSuccess; ++k) e1 = step(k, S.cap_stream);
      const cudaError_t e2 = cudaStreamEndCapture(S.cap_stream, &g);
      e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    G.graph_diff = e == cudaSuccess ? diff : -1.0;
  }
  int done = 0, launches = 0;
  if (e == cudaSuccess && G.graph && G.graph_diff == diff) {
    for (; done + grp <= n_steps && e == cudaSuccess; done += grp) {
      e = cudaGraphLaunch(G.graph, st);
      launches += grp * per_step + per_corr;
    }
  }
  for (int k = done + 1; k <= n_steps && e == cudaSuccess; ++k) {
    e = step(k, st);
    launches += per_step + (G.kc > 0 && k % G.kc == 0 ? per_corr : 0);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, S.un, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s_final, S.sn, sbytes, cudaMemcpyDeviceToDevice, st);
  c->launches = launches;
  if (e != cudaSuccess)
    return fd_set_error(c, FD_ECUDA, "fd_rollout_scalar (generic-grid learned): %s", cudaGetErrorString(e));
  return FD_OK;
}
