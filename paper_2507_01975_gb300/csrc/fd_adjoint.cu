// fd_adjoint.cu -- reverse mode of one time step behind the C ABI
// (fd_step_adjoint): recompute the RK4 stages keeping the stage states and
// every network activation, then run the stages backwards (RK4 combination and
// projection adjoints, flux-block adjoint, network data and weight gradients on
// the tensor cores).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/fd.h"
#include "conv_tc.cuh"
#include "conv_wgrad.cuh"
#include "fd_ctx.h"
#include "fd_net.cuh"
#include "fv_adjoint.cuh"
#include "fv_learned.cuh"

using namespace ldfv;

fd_status fd_learned_error_flag(fd_ctx* c);
cudaError_t fd_fno_forward_saved(fd_ctx* c, int which, const float* single, const float* const* hist,
                                 const FnoSavedBufs& sb, cudaStream_t st);
cudaError_t fd_fno_backward(fd_ctx* c, int which, const FnoSavedBufs& sb, const float* single,
                            const float* const* hist, const float* gbar, float* ubar, size_t ost, bool accumulate,
                            float* dparams, float* partial, cudaStream_t st);
void fd_fno_saved_sizes(const LearnedState& L, int which, int batch, int nn, size_t* v_floats, size_t* a_floats,
                        size_t* s_float2, size_t* out_floats);
size_t fd_fno_partial_floats();

namespace {

// name of the launch that failed last (for the error message)
thread_local const char* g_where = "";

inline cudaError_t mark(cudaError_t e, const char* where) {
  if (e != cudaSuccess && !*g_where) g_where = where;
  return e;
}

constexpr int kAdjBandRows = 8;  // rows per CTA of the flux-block reverse kernel
constexpr int kWgradMaxCols = 3 * 2 * 80;  // largest per-CTA partial: 3 dx x 2 MMAs x 80 channels

// ---------------------------------------------------------------------------
// reverse mode of the temporal correction u_k = P(V + c - mean(c)), c = TC(hist)
// (Sec. 3.2, Sec. 3.5): with g = P(lam) (P symmetric), V_bar = g and
// c_bar = g - mean(g) per trajectory and component (the mean removal is an
// orthogonal projector, so its own transpose)
// ---------------------------------------------------------------------------
struct TcCbarArgs {
  const float* lam;      // [batch][2][N][N] cotangent of the corrected state
  float* vbar;           // P(lam), or null
  __nv_bfloat16* cbar;   // [batch][2][N][N][8]: channels 0, 1 = c_bar, 2 .. 15 = 0, or null
  float* cbar_f32;       // c_bar as [batch][2][N][N] FP32, or null
  int project;
  float idx, idy, inv_nn;
  const float2* tw;
  const float* symx;
  const float* symy;
};

template <int LOGN>
__global__ void __launch_bounds__(LearnedCfg<LOGN>::NT, 1) tc_cbar_kernel(const TcCbarArgs a) {
  using Cfg = LearnedCfg<LOGN>;
  constexpr int N = Cfg::N, NT = Cfg::NT;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* const wt = reinterpret_cast<float*>(smem);
  unsigned char* const scr = smem + Cfg::OFF_SCR;
  float2* const tw = reinterpret_cast<float2*>(smem + Cfg::OFF_TW);
  float* const sx = reinterpret_cast<float*>(smem + Cfg::OFF_SX);
  float* const sy = reinterpret_cast<float*>(smem + Cfg::OFF_SY);
  __shared__ float red[2][NT / 32];
  const int tid = threadIdx.x;
  const size_t off = (size_t)blockIdx.x * 2 * NN;
  for (int k = tid; k < N / 2; k += NT) tw[k] = a.tw[k];
  for (int k = tid; k <= N / 2; k += NT) sx[k] = a.symx[k];
  for (int k = tid; k < N; k += NT) sy[k] = a.symy[k];
  pdl_wait();
  pdl_trigger();
  for (size_t c = tid; c < 2 * NN; c += NT) wt[c] = a.lam[off + c];
  __syncthreads();
  if (a.project) project_tile<LOGN, NT>(wt, scr, tw, sx, sy, a.idx, a.idy, a.inv_nn);
  float s0 = 0.f, s1 = 0.f;
  for (size_t c = tid; c < NN; c += NT) {
    s0 += wt[c];
    s1 += wt[NN + c];
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
  for (int w = 0; w < NT / 32; ++w) {
    m0 += red[0][w];
    m1 += red[1][w];
  }
  m0 *= a.inv_nn;
  m1 *= a.inv_nn;
  for (size_t c = tid; c < NN; c += NT) {
    if (a.vbar) {
      a.vbar[off + c] = wt[c];
      a.vbar[off + NN + c] = wt[NN + c];
    }
    if (a.cbar_f32) {
      a.cbar_f32[off + c] = wt[c] - m0;
      a.cbar_f32[off + NN + c] = wt[NN + c] - m1;
    }
    if (a.cbar) {
      uint4 pk0, pk1 = make_uint4(0u, 0u, 0u, 0u);
      __nv_bfloat162 h0 = __floats2bfloat162_rn(wt[c] - m0, wt[NN + c] - m1);
      pk0.x = *reinterpret_cast<uint32_t*>(&h0);
      pk0.y = pk0.z = pk0.w = 0u;
      __nv_bfloat16* dst = a.cbar + ((size_t)blockIdx.x * 2 * NN + c) * 8;
      *reinterpret_cast<uint4*>(dst) = pk0;
      *reinterpret_cast<uint4*>(dst + NN * 8) = pk1;
    }
  }
}

// First-layer data gradient of the correction network (64 -> K = 2 k_c) on
// CUDA cores: x_bar[ci][p] = sum_{o, tap} W0t[ci][o][tap] z_bar[o][p + tap],
// with channel ci = 2 s + component written to the history cotangent of state s
// (out + s * state_stride).
struct ConvOutKArgs {
  const __nv_bfloat16* in;  // [batch][8][N][N][8]
  const float* w;           // [K][64][3][3], transposed and flipped
  float* out;               // K/2 states [batch][2][N][N], state_stride apart
  size_t state_stride;      // floats
  int batch, k;
};

template <int LOGN>
__global__ void __launch_bounds__(256) conv_outk_kernel(const ConvOutKArgs a) {
  constexpr int N = 1 << LOGN;
  __shared__ float sw[16 * 64 * 9];
  for (int q = threadIdx.x; q < a.k * 64 * 9; q += blockDim.x) sw[q] = a.w[q];
  __syncthreads();
  pdl_wait();
  pdl_trigger();
  const size_t total = (size_t)a.batch * N * N;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / (N * N));
    const int y = (int)((p / N) % N), x = (int)(p % N);
    float o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) o[j] = 0.f;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int yy = (y + dy) & (N - 1), xx = (x + dx) & (N - 1);
        const int t = (dy + 1) * 3 + dx + 1;
        for (int c8 = 0; c8 < 8; ++c8) {
          const uint4 pk = *reinterpret_cast<const uint4*>(a.in + ((((size_t)b * 8 + c8) * N + yy) * N + xx) * 8);
          const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&pk);
#pragma unroll
          for (int j2 = 0; j2 < 4; ++j2) {
            const float2 f = __bfloat1622float2(h[j2]);
            const int c0 = c8 * 8 + 2 * j2;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (j < a.k) o[j] += sw[(j * 64 + c0) * 9 + t] * f.x + sw[(j * 64 + c0 + 1) * 9 + t] * f.y;
          }
        }
      }
    const size_t pix = (size_t)y * N + x;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < a.k) a.out[(size_t)(j >> 1) * a.state_stride + ((size_t)b * 2 + (j & 1)) * N * N + pix] = o[j];
  }
}

template <int LOGN>
cudaError_t prepare_adjoint(bool learned) {
  cudaError_t e = cudaFuncSetAttribute(fv_adjoint_band_kernel<LOGN, kAdjBandRows>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)AdjBandCfg<LOGN, kAdjBandRows>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fv_adjoint_combine_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)LearnedCfg<LOGN>::SMEM);
  if (e == cudaSuccess) e = prepare_learned_stage<LOGN>();
  if (!learned || e != cudaSuccess) return e;
  // kernel templates are instantiated per translation unit: the forward
  // convolutions launched from here need their attributes set from here too
  e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, 64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ConvCfg<LOGN, 64, 64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, 64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ConvCfg<LOGN, 64, 32>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, 16, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ConvCfg<LOGN, 16, 64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, kCoef, 32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ConvCfg<LOGN, kCoef, 32, 1>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_kernel<LOGN, 64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)WgradCfg<LOGN, 64, 64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_kernel<LOGN, 64, 80>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)WgradCfg<LOGN, 64, 80>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_kernel<LOGN, 16, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)WgradCfg<LOGN, 16, 64>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_kernel<LOGN, 64, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)WgradCfg<LOGN, 64, 16>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_cbar_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)LearnedCfg<LOGN>::SMEM);
  return e;
}

void adjoint_free(AdjointState* A) {
  if (!A) return;
  void* ps[] = {A->wst[0], A->wst[1], A->wst[2], A->acc,     A->g,         A->rb,
                A->wbar,   A->xbar,   A->zeros,  A->cbar,    A->zbar[0],   A->zbar[1],
                A->partial, A->partial_b, A->tc_cbar, (void*)A->d_hist, A->fnobar, A->tc_cbar_f32,
                A->fno_partial};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (FnoSavedBufs* sb : {&A->fsv[0], &A->fsv[1], &A->fsv[2], &A->fsv[3], &A->tcs}) {
    void* fp[] = {sb->v, sb->a, sb->S, sb->out};
    for (void* p : fp)
      if (p) cudaFree(p);
  }
  for (int s = 0; s < 4; ++s) {
    for (int l = 0; l < 6; ++l)
      if (A->h[s][l]) cudaFree(A->h[s][l]);
    for (int l = 0; l < 5; ++l)
      if (A->z[s][l]) cudaFree(A->z[s][l]);
    if (A->coef[s]) cudaFree(A->coef[s]);
  }
  delete A;
}

fd_status adjoint_alloc(fd_ctx* c) {
  AdjointState* A = new (std::nothrow) AdjointState();
  if (!A) return fd_set_error(c, FD_ENOMEM, "fd_step_adjoint: out of host memory");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&A->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    A->sms = 1;
  const size_t NN = (size_t)c->grid.nx * c->grid.ny;
  const size_t B = c->grid.batch;
  const size_t state = fd_state_bytes(c->grid);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  for (int s = 0; s < 3; ++s) alloc((void**)&A->wst[s], state);
  alloc((void**)&A->acc, state);
  alloc((void**)&A->g, state);
  alloc((void**)&A->rb, state);
  alloc((void**)&A->wbar, state);
  alloc((void**)&A->xbar, state);
  alloc((void**)&A->zeros, 80 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(A->zeros, 0, 80 * sizeof(float));
  if (c->lrn) {
    const int sms = c->lrn->sms;
    for (int s = 0; s < 4; ++s) {
      alloc((void**)&A->h[s][0], B * 16 * NN * 2);
      for (int l = 1; l < 6; ++l) alloc((void**)&A->h[s][l], B * kHidden * NN * 2);
      for (int l = 0; l < 5; ++l) alloc((void**)&A->z[s][l], B * kHidden * NN * 2);
      alloc((void**)&A->coef[s], B * kCoef * NN * 2);
    }
    alloc((void**)&A->cbar, B * kCoef * NN * 2);
    alloc((void**)&A->zbar[0], B * kHidden * NN * 2);
    alloc((void**)&A->zbar[1], B * kHidden * NN * 2);
    alloc((void**)&A->partial, (size_t)sms * kWgradMaxCols * 128 * sizeof(float));
    alloc((void**)&A->partial_b, (size_t)sms * 80 * sizeof(float));
    if (c->lrn->kc > 0) {
      alloc((void**)&A->tc_cbar, B * 16 * NN * 2);
      alloc((void**)&A->d_hist, 8 * sizeof(float*));
    }
    auto alloc_saved = [&](FnoSavedBufs& sb, int which) {
      size_t nv, na, ns, no;
      fd_fno_saved_sizes(*c->lrn, which, (int)B, (int)NN, &nv, &na, &ns, &no);
      alloc((void**)&sb.v, nv * sizeof(float));
      alloc((void**)&sb.a, na * sizeof(float));
      alloc((void**)&sb.S, ns * sizeof(float2));
      alloc((void**)&sb.out, no * sizeof(float));
    };
    if (c->lrn->fno_layers > 0) {
      for (int s = 0; s < 4; ++s) alloc_saved(A->fsv[s], 0);
      alloc((void**)&A->fnobar, B * 8 * NN * sizeof(float));
    }
    if (c->lrn->kc > 0 && c->lrn->tcf_layers > 0) {
      alloc_saved(A->tcs, 1);
      alloc((void**)&A->tc_cbar_f32, state);
    }
    if (c->lrn->fno_layers > 0 || c->lrn->tcf_layers > 0)
      alloc((void**)&A->fno_partial, fd_fno_partial_floats() * sizeof(float));
  }
  if (e == cudaSuccess) e = (c->logn == 6) ? prepare_adjoint<6>(c->lrn != nullptr) : prepare_adjoint<5>(c->lrn != nullptr);
  if (e != cudaSuccess) {
    adjoint_free(A);
    return fd_set_error(c, FD_ENOMEM, "fd_step_adjoint: workspace: %s", cudaGetErrorString(e));
  }
  A->ready = true;
  c->adj = A;
  return FD_OK;
}

// weight and bias gradients of one layer: tensor-core partial sums, then a
// deterministic reduction added to dW / db
template <int LOGN, int CIN, int O_TILE>
cudaError_t wgrad(fd_ctx* c, const __nv_bfloat16* h, const __nv_bfloat16* z, int cout_total, int parts, int cin_real,
                  float* dW, float* db, cudaStream_t st, int* launches, int cout_real = 1 << 30) {
  using Cfg = WgradCfg<LOGN, CIN, O_TILE>;
  LearnedState& L = *c->lrn;
  AdjointState& A = *c->adj;
  const int B = c->grid.batch;
  const int nitems = B * (Cfg::N / Cfg::R);
  int gx = L.sms / parts;
  if (gx > nitems) gx = nitems;
  if (gx < 1) gx = 1;
  WgradArgs a;
  std::memset(&a, 0, sizeof a);
  a.h = h;
  a.z = z;
  a.partial = A.partial;
  a.partial_b = A.partial_b;
  a.batch = B;
  a.cout_total = cout_total;
  a.err = L.d_err;
  a.spin_limit = L.spin;
  cudaError_t e = mark(launch_pdl(conv_wgrad_kernel<LOGN, CIN, O_TILE>, dim3(gx, parts), dim3(Cfg::NT), Cfg::SMEM, st, a),
                       "weight-gradient kernel");
  if (e != cudaSuccess) return e;
  WgradReduceArgs r;
  r.partial = A.partial;
  r.partial_b = A.partial_b;
  r.dW = dW;
  r.db = db;
  r.gx = gx;
  r.parts = parts;
  r.cin = cin_real;
  r.co_base = 0;
  r.cout_real = cout_real;
  const int total = parts * O_TILE * cin_real * 9 + parts * O_TILE;
  *launches += 2;
  return mark(launch_pdl(conv_wgrad_reduce_kernel<CIN, O_TILE>, dim3((total + 255) / 256), dim3(256), 0, st, r),
              "weight-gradient reduction");
}

// stencil network at stage state w, keeping every layer input and pre-activation
template <int LOGN>
cudaError_t net_forward_saved(fd_ctx* c, int s, const float* w, cudaStream_t st, int* launches) {
  LearnedState& L = *c->lrn;
  AdjointState& A = *c->adj;
  const int B = c->grid.batch;
  PackArgs pa;
  pa.hist = nullptr;
  pa.single = w;
  pa.out = A.h[s][0];
  pa.batch = B;
  pa.cin = 2;
  const size_t pix = (size_t)B << (2 * LOGN);
  const int blocks = (int)((pix + 255) / 256 < (size_t)(4 * L.sms) ? (pix + 255) / 256 : (size_t)(4 * L.sms));
  cudaError_t e = mark(launch_pdl(pack_input_kernel<LOGN>, dim3(blocks), dim3(256), 0, st, pa), "input packing");
  if (e == cudaSuccess)
    e = launch_conv<LOGN, 64, 16>(L, A.h[s][0], L.d_wpack + L.pk_stencil_first, L.d_raw + L.raw_off_sb[0], A.h[s][1],
                                  B, 1, 0, 64, 1, st, nullptr, A.z[s][0]);
  for (int l = 1; l <= 4 && e == cudaSuccess; ++l)
    e = launch_conv<LOGN, 64>(L, A.h[s][l], L.d_wpack + L.pk_stencil[l - 1], L.d_raw + L.raw_off_sb[l], A.h[s][l + 1],
                              B, 1, 0, 64, 1, st, nullptr, A.z[s][l]);
  if (e == cudaSuccess)
    e = launch_conv<LOGN, 64>(L, A.h[s][5], L.d_wpack + L.pk_stencil[4], L.d_raw + L.raw_off_sb[5], A.coef[s], B, 2, 0,
                              kCoef, 0, st);
  if (e == cudaSuccess)
    e = launch_conv<LOGN, 32>(L, A.h[s][5], L.d_wpack + L.pk_stencil_last32, L.d_raw + L.raw_off_sb[5], A.coef[s], B,
                              1, 128, kCoef, 0, st);
  *launches += 8;
  return mark(e, "network forward");
}

// reverse pass of the stencil network at stage s: A.cbar -> A.xbar (FP32 state
// cotangent of the network input); weight gradients added to dparams when set
template <int LOGN>
cudaError_t net_backward(fd_ctx* c, int s, float* dparams, cudaStream_t st, int* launches) {
  LearnedState& L = *c->lrn;
  AdjointState& A = *c->adj;
  const int B = c->grid.batch;
  cudaError_t e = cudaSuccess;
  // Bias gradients are pixel sums of FP32 cotangents: the last layer's from the
  // flux-block reverse kernel, the others from the data-gradient epilogues, so
  // the weight-gradient kernels skip them (their BF16 operands would lose the
  // cancellations of those sums).
  auto bias_at = [&](int l) { return dparams ? dparams + L.raw_off_sb[l] : nullptr; };
  // last layer 64 -> 160 (no activation after it): z_bar = C_bar
  if (dparams)
    e = wgrad<LOGN, 64, 80>(c, A.h[s][5], A.cbar, kCoef, 2, 64, dparams + L.raw_off_sw[5], nullptr, st, launches);
  if (e == cudaSuccess)
    e = mark(launch_conv<LOGN, 32, kCoef, 1>(L, A.cbar, L.d_wpack + L.pk_t5, nullptr, A.zbar[0], B, 2, 0, 64, 2, st,
                                             A.z[s][4], nullptr, bias_at(4)),
             "last-layer data gradient");
  ++*launches;
  int cur = 0;
  for (int l = 4; l >= 1 && e == cudaSuccess; --l) {
    if (dparams)
      e = wgrad<LOGN, 64, 64>(c, A.h[s][l], A.zbar[cur], 64, 1, 64, dparams + L.raw_off_sw[l], nullptr, st, launches);
    if (e == cudaSuccess)
      e = mark(launch_conv<LOGN, 64>(L, A.zbar[cur], L.d_wpack + L.pk_t[l - 1], nullptr, A.zbar[cur ^ 1], B, 1, 0,
                                     64, 2, st, A.z[s][l - 1], nullptr, bias_at(l - 1)),
               "hidden-layer data gradient");
    ++*launches;
    cur ^= 1;
  }
  // first layer 2 -> 64: weight gradient with the 16-channel packed input,
  // data gradient (64 -> 2) on CUDA cores
  if (e == cudaSuccess && dparams)
    e = wgrad<LOGN, 16, 64>(c, A.h[s][0], A.zbar[cur], 64, 1, 2, dparams + L.raw_off_sw[0], nullptr, st, launches);
  if (e == cudaSuccess) {
    ConvOut2Args oa;
    oa.in = A.zbar[cur];
    oa.w = L.d_raw + L.raw_off_w0t;
    oa.bias = L.d_raw + L.raw_off_zero;
    oa.out = A.xbar;
    oa.batch = B;
    const size_t pix = (size_t)B << (2 * LOGN);
    const int blocks = (int)((pix + 255) / 256 < (size_t)(4 * L.sms) ? (pix + 255) / 256 : (size_t)(4 * L.sms));
    e = mark(launch_pdl(conv_out2_kernel<LOGN>, dim3(blocks), dim3(256), 0, st, oa), "first-layer data gradient");
    ++*launches;
  }
  return e;
}

// Reverse mode of the temporal correction's CNN head at one correction step:
// hist = the k_c states u_{k-k_c} .. u_{k-1} (device pointer array), lam = the
// cotangent of the corrected state u_k. Writes vbar = P(lam) (the cotangent of
// the FV output, when non-null) and the history cotangents hbar (k_c states,
// state_stride floats apart); adds the network's weight and bias gradients
// to dparams when set. The forward activations are recomputed into the stage-0
// buffers of the step reverse mode.
template <int LOGN>
cudaError_t tc_adjoint(fd_ctx* c, const float* const* hist, const float* lam, float* vbar, float* hbar,
                       size_t state_stride, float* dparams, cudaStream_t st, int* launches) {
  LearnedState& L = *c->lrn;
  AdjointState& A = *c->adj;
  const int B = c->grid.batch;
  const int kc = L.kc;
  const FvArgs& fb = c->base;
  TcCbarArgs ca;
  ca.lam = lam;
  ca.vbar = vbar;
  ca.cbar = A.tc_cbar;
  ca.cbar_f32 = nullptr;
  ca.project = c->grid.flow == FD_NAVIER_STOKES ? 1 : 0;
  ca.idx = (float)fb.idx;
  ca.idy = (float)fb.idy;
  ca.inv_nn = (float)fb.inv_nn;
  ca.tw = reinterpret_cast<const float2*>(fb.tw);
  ca.symx = reinterpret_cast<const float*>(fb.symx);
  ca.symy = reinterpret_cast<const float*>(fb.symy);
  if (L.tcf_layers > 0) {
    // the correction as a Fourier neural operator: its saved forward, c_bar in
    // FP32, then the operator's reverse mode into the history cotangents
    cudaError_t e = mark(fd_fno_forward_saved(c, 1, nullptr, hist, A.tcs, st), "correction operator forward");
    *launches += 2 + 4 * L.tcf_layers;
    ca.cbar = nullptr;
    ca.cbar_f32 = A.tc_cbar_f32;
    if (e == cudaSuccess)
      e = mark(launch_pdl(tc_cbar_kernel<LOGN>, dim3(B), dim3(LearnedCfg<LOGN>::NT), LearnedCfg<LOGN>::SMEM, st, ca),
               "correction output cotangent");
    ++*launches;
    if (e == cudaSuccess)
      e = mark(fd_fno_backward(c, 1, A.tcs, nullptr, hist, A.tc_cbar_f32, hbar, state_stride, false, dparams,
                               A.fno_partial, st),
               "correction operator reverse");
    *launches += 4 + 7 * L.tcf_layers;
    return e;
  }
  // forward of the trunk, keeping every layer input and pre-activation
  PackArgs pa;
  pa.hist = hist;
  pa.single = nullptr;
  pa.out = A.h[0][0];
  pa.batch = B;
  pa.cin = 2 * kc;
  const size_t pix = (size_t)B << (2 * LOGN);
  const int blocks = (int)((pix + 255) / 256 < (size_t)(4 * L.sms) ? (pix + 255) / 256 : (size_t)(4 * L.sms));
  cudaError_t e = mark(launch_pdl(pack_input_kernel<LOGN>, dim3(blocks), dim3(256), 0, st, pa), "correction input");
  if (e == cudaSuccess)
    e = launch_conv<LOGN, 64, 16>(L, A.h[0][0], L.d_wpack + L.pk_tc_first, L.d_raw + L.raw_off_tb[0], A.h[0][1], B, 1,
                                  0, 64, 1, st, nullptr, A.z[0][0]);
  for (int l = 1; l <= 4 && e == cudaSuccess; ++l)
    e = launch_conv<LOGN, 64>(L, A.h[0][l], L.d_wpack + L.pk_tc[l - 1], L.d_raw + L.raw_off_tb[l], A.h[0][l + 1], B,
                              1, 0, 64, 1, st, nullptr, A.z[0][l]);
  *launches += 6;
  e = mark(e, "correction network forward");
  // c_bar = P(lam) - mean, packed for the tensor cores
  if (e == cudaSuccess) {
    e = mark(launch_pdl(tc_cbar_kernel<LOGN>, dim3(B), dim3(LearnedCfg<LOGN>::NT), LearnedCfg<LOGN>::SMEM, st, ca),
             "correction output cotangent");
    ++*launches;
  }
  // last layer 64 -> 2 (no activation): weight gradient with the 2 real of 16
  // output channels; its bias gradient, the pixel sum of c_bar, is zero (the
  // mean removal), so nothing is added. Data gradient 2 -> 64 times GELU'(z_4);
  // the other bias gradients are FP32 sums from the data-gradient epilogues.
  auto bias_at = [&](int l) { return dparams ? dparams + L.raw_off_tb[l] : nullptr; };
  if (e == cudaSuccess && dparams)
    e = wgrad<LOGN, 64, 16>(c, A.h[0][5], A.tc_cbar, 16, 1, 64, dparams + L.raw_off_tw[5], nullptr, st, launches, 2);
  if (e == cudaSuccess)
    e = mark(launch_conv<LOGN, 64, 16>(L, A.tc_cbar, L.d_wpack + L.pk_tc_t5, nullptr, A.zbar[0], B, 1, 0, 64, 2, st,
                                       A.z[0][4], nullptr, bias_at(4)),
             "correction last-layer data gradient");
  ++*launches;
  int cur = 0;
  for (int l = 4; l >= 1 && e == cudaSuccess; --l) {
    if (dparams)
      e = wgrad<LOGN, 64, 64>(c, A.h[0][l], A.zbar[cur], 64, 1, 64, dparams + L.raw_off_tw[l], nullptr, st, launches);
    if (e == cudaSuccess)
      e = mark(launch_conv<LOGN, 64>(L, A.zbar[cur], L.d_wpack + L.pk_tc_t[l - 1], nullptr, A.zbar[cur ^ 1], B, 1, 0,
                                     64, 2, st, A.z[0][l - 1], nullptr, bias_at(l - 1)),
               "correction hidden-layer data gradient");
    ++*launches;
    cur ^= 1;
  }
  if (e == cudaSuccess && dparams)
    e = wgrad<LOGN, 16, 64>(c, A.h[0][0], A.zbar[cur], 64, 1, 2 * kc, dparams + L.raw_off_tw[0], nullptr, st,
                            launches);
  if (e == cudaSuccess) {
    ConvOutKArgs oa;
    oa.in = A.zbar[cur];
    oa.w = L.d_raw + L.raw_off_tw0t;
    oa.out = hbar;
    oa.state_stride = state_stride;
    oa.batch = B;
    oa.k = 2 * kc;
    e = mark(launch_pdl(conv_outk_kernel<LOGN>, dim3(blocks), dim3(256), 0, st, oa),
             "correction first-layer data gradient");
    ++*launches;
  }
  return e;
}

template <int LOGN>
cudaError_t combine(fd_ctx* c, const float* in0, const float* in1, float* lam, float* rb, float alpha, float beta,
                    int init, int project, cudaStream_t st) {
  AdjointState& A = *c->adj;
  const FvArgs& b = c->base;
  AdjCombineArgs a;
  a.in0 = in0;
  a.in1 = in1;
  a.g = A.g;
  a.lam = lam;
  a.rb = rb;
  a.alpha = alpha;
  a.beta = beta;
  a.init = init;
  a.project = project;
  a.idx = (float)b.idx;
  a.idy = (float)b.idy;
  a.inv_nn = (float)b.inv_nn;
  a.tw = reinterpret_cast<const float2*>(b.tw);
  a.symx = reinterpret_cast<const float*>(b.symx);
  a.symy = reinterpret_cast<const float*>(b.symy);
  return mark(launch_pdl(fv_adjoint_combine_kernel<LOGN>, dim3(c->grid.batch), dim3(LearnedCfg<LOGN>::NT),
                         LearnedCfg<LOGN>::SMEM, st, a),
              "stage combination");
}

// u' = P(u + dt/6 (r1 + 2 r2 + 2 r3 + r4)), r_s = H(w_s), w_1 = u,
// w_2 = P(u + dt/2 r1), w_3 = P(u + dt/2 r2), w_4 = P(u + dt r3)  (Sec. 3.6, App. B.3)
template <int LOGN>
cudaError_t step_adjoint(fd_ctx* c, const float* u, const float* lam_out, float* lam_in, float* dparams,
                         cudaStream_t st, int* launches) {
  AdjointState& A = *c->adj;
  const bool learned = c->lrn != nullptr;
  const int B = c->grid.batch;
  const int ns = c->grid.flow == FD_NAVIER_STOKES ? 1 : 0;
  const float dt = (float)c->dt;
  const float* ws[4] = {u, A.wst[0], A.wst[1], A.wst[2]};
  cudaError_t e = cudaSuccess;
  // ---- forward: stage states (and network activations) --------------------------
  // the stencil network runs unless the ablation keeps the frequency-domain
  // operator only; O_F runs when the model has one
  const bool net = learned && c->lrn->ablation != 2;
  const bool fno = learned && c->lrn->fno_layers > 0;
  const int fno_launches = fno ? 2 + 4 * c->lrn->fno_layers : 0;
  LStageArgs fa = stage_args(c);
  fa.un = u;
  fa.acc = A.acc;
  if (!learned) fa.wl = A.zeros;
  for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
    if (net) e = net_forward_saved<LOGN>(c, s, ws[s], st, launches);
    if (e == cudaSuccess && fno) {
      e = mark(fd_fno_forward_saved(c, 0, ws[s], nullptr, A.fsv[s], st), "frequency-domain operator");
      *launches += fno_launches;
    }
    if (e != cudaSuccess) break;
    fa.stage = s;
    fa.w = ws[s];
    fa.wout = A.wst[s];
    fa.coef = net ? A.coef[s] : nullptr;
    fa.fno = fno ? A.fsv[s].out : nullptr;
    e = mark(launch_learned_stage<LOGN>(fa, A.xbar, B, A.sms, st), "forward stage");  // xbar is free until the reverse pass
    *launches += 2;
  }
  if (e == cudaSuccess && net) e = net_forward_saved<LOGN>(c, 3, ws[3], st, launches);
  if (e == cudaSuccess && fno) {
    e = mark(fd_fno_forward_saved(c, 0, ws[3], nullptr, A.fsv[3], st), "frequency-domain operator");
    *launches += fno_launches;
  }
  // ---- reverse ------------------------------------------------------------------------
  // g = P(lam_out), lam_in = g, rb_4 = dt/6 g
  if (e == cudaSuccess) e = combine<LOGN>(c, lam_out, nullptr, lam_in, A.rb, 0.f, dt / 6.0f, 1, ns, st);
  ++*launches;
  const float cg[4] = {dt / 6.0f, dt / 3.0f, dt / 3.0f, dt / 6.0f};  // weights of r_1 .. r_4 in u'
  const float aw[4] = {0.f, 0.5f * dt, 0.5f * dt, dt};               // w_s = P(u + aw[s] r_{s-1})
  AdjStageArgs sa;
  std::memset(&sa, 0, sizeof sa);
  sa.tbar = A.rb;
  sa.wl = learned ? c->lrn->d_raw + c->lrn->raw_off_wl : nullptr;
  sa.wbar = A.wbar;
  sa.cbar = net ? A.cbar : nullptr;
  sa.wl_bar = (net && dparams) ? dparams + c->lrn->raw_off_wl : nullptr;
  sa.cbias = (net && dparams) ? dparams + c->lrn->raw_off_sb[5] : nullptr;
  sa.fnobar = fno ? A.fnobar : nullptr;
  sa.ablation = learned ? c->lrn->ablation : 0;
  sa.flow = c->grid.flow;
  sa.forcing = c->forcing.kind;
  sa.dord = c->opts.deriv_order;
  sa.nu = (float)c->base.nu;
  sa.idx = (float)c->base.idx;
  sa.idy = (float)c->base.idy;
  sa.drag = (float)c->base.drag;
  for (int s = 3; s >= 0 && e == cudaSuccess; --s) {
    sa.w = ws[s];
    sa.coef = net ? A.coef[s] : nullptr;
    sa.fno = fno ? A.fsv[s].out : nullptr;
    // banded flux-block reverse: bands add their scatter into the zeroed w_bar
    e = mark(cudaMemsetAsync(A.wbar, 0, fd_state_bytes(c->grid), st), "stage adjoint");
    if (e != cudaSuccess) break;
    e = mark(launch_pdl(fv_adjoint_band_kernel<LOGN, kAdjBandRows>, dim3((1 << LOGN) / kAdjBandRows, B), dim3(256),
                        AdjBandCfg<LOGN, kAdjBandRows>::SMEM, st, sa),
             "stage adjoint");
    ++*launches;
    if (e == cudaSuccess && net) e = net_backward<LOGN>(c, s, dparams, st, launches);
    if (e == cudaSuccess && fno) {
      // O_F's output cotangent is the face-value cotangent; its input cotangent
      // joins the network's (or starts it, without a network)
      e = mark(fd_fno_backward(c, 0, A.fsv[s], ws[s], nullptr, A.fnobar, A.xbar, 0, net, dparams, A.fno_partial, st),
               "frequency-domain operator reverse");
      *launches += 4 + 7 * c->lrn->fno_layers;
    }
    if (e != cudaSuccess) break;
    const float* x = (net || fno) ? A.xbar : nullptr;
    if (s > 0)
      e = combine<LOGN>(c, A.wbar, x, lam_in, A.rb, cg[s - 1], aw[s], 0, ns, st);  // y = P(w_bar)
    else
      e = combine<LOGN>(c, A.wbar, x, lam_in, nullptr, 0.f, 0.f, 0, 0, st);       // w_1 = u: no projection
    ++*launches;
  }
  return e;
}

}  // namespace

void fd_adjoint_free(fd_ctx* c) {
  if (c->adj) adjoint_free(c->adj);
  c->adj = nullptr;
}

extern "C" {

fd_status fd_step_adjoint(fd_ctx* c, const void* u_in, const void* lam_out, void* lam_in, float* dparams,
                          void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_step_adjoint: null context");
  c->launches = 0;
  if (!u_in || !lam_out || !lam_in) return fd_set_error(c, FD_EINVAL, "fd_step_adjoint: null state pointer");
  if (c->gen)
    return fd_gadjoint_step(c, static_cast<const float*>(u_in), static_cast<const float*>(lam_out),
                            static_cast<float*>(lam_in), dparams, static_cast<cudaStream_t>(stream));
  if (c->grid.dtype != FD_F32 || (c->grid.nx != 32 && c->grid.nx != 64))
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_step_adjoint: built for FP32 grids of 32 or 64 cells per side");
  if (c->lrn && !c->lrn->ready)
    return fd_set_error(c, FD_EINVAL, "fd_step_adjoint: learned parameters not set (fd_set_params)");
  if (dparams && !c->lrn) return fd_set_error(c, FD_EINVAL, "fd_step_adjoint: dparams needs a learned context");
  if (!c->adj) {
    fd_status s = adjoint_alloc(c);
    if (s != FD_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int launches = 0;
  g_where = "";
  const float* u = static_cast<const float*>(u_in);
  const float* lo = static_cast<const float*>(lam_out);
  float* li = static_cast<float*>(lam_in);
  cudaError_t e = (c->logn == 6) ? step_adjoint<6>(c, u, lo, li, dparams, st, &launches)
                                 : step_adjoint<5>(c, u, lo, li, dparams, st, &launches);
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_step_adjoint: %s: %s", g_where, cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_step_adjoint_scalar(fd_ctx* c, double diffusivity, const void* u_in, const void* s_in,
                                 const void* lam_u_out, const void* lam_s_out, void* lam_u_in, void* lam_s_in,
                                 float* dparams, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_step_adjoint_scalar: null context");
  c->launches = 0;
  if (!u_in || !s_in || !lam_u_out || !lam_s_out || !lam_u_in || !lam_s_in)
    return fd_set_error(c, FD_EINVAL, "fd_step_adjoint_scalar: null pointer");
  return fd_gadjoint_step_scalar(c, diffusivity, static_cast<const float*>(u_in), static_cast<const float*>(s_in),
                                 static_cast<const float*>(lam_u_out), static_cast<const float*>(lam_s_out),
                                 static_cast<float*>(lam_u_in), static_cast<float*>(lam_s_in), dparams,
                                 static_cast<cudaStream_t>(stream));
}

fd_status fd_tc_adjoint(fd_ctx* c, const void* hist, const void* lam, void* vbar, void* hist_bar, float* dparams,
                        void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_tc_adjoint: null context");
  c->launches = 0;
  if (c->gen) {
    if (!hist || !lam || !hist_bar) return fd_set_error(c, FD_EINVAL, "fd_tc_adjoint: null pointer");
    const size_t slot = fd_state_bytes(c->grid) / sizeof(float);
    const float* h[8] = {};
    const int kc = c->glrn ? c->glrn->kc : 0;
    for (int s = 0; s < kc && s < 8; ++s) h[s] = static_cast<const float*>(hist) + (size_t)s * slot;
    int launches = 0;
    const fd_status r = fd_gadjoint_tc(c, h, static_cast<const float*>(lam), static_cast<float*>(vbar),
                                       static_cast<float*>(hist_bar), slot, dparams, static_cast<cudaStream_t>(stream),
                                       &launches);
    c->launches = launches;
    return r;
  }
  if (!c->lrn || c->lrn->kc == 0)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_tc_adjoint: needs a learned context with a temporal correction");
  if (!hist || !lam || !hist_bar) return fd_set_error(c, FD_EINVAL, "fd_tc_adjoint: null pointer");
  if (!c->lrn->ready) return fd_set_error(c, FD_EINVAL, "fd_tc_adjoint: learned parameters not set (fd_set_params)");
  if (!c->adj) {
    fd_status s = adjoint_alloc(c);
    if (s != FD_OK) return s;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t slot = fd_state_bytes(c->grid) / sizeof(float);
  const float* h[8];
  for (int s = 0; s < c->lrn->kc; ++s) h[s] = static_cast<const float*>(hist) + (size_t)s * slot;
  g_where = "";
  int launches = 0;
  cudaError_t e = mark(cudaMemcpyAsync(c->adj->d_hist, h, sizeof(const float*) * c->lrn->kc, cudaMemcpyHostToDevice,
                                       st),
                       "history pointers");
  if (e == cudaSuccess)
    e = (c->logn == 6) ? tc_adjoint<6>(c, c->adj->d_hist, static_cast<const float*>(lam), static_cast<float*>(vbar),
                                       static_cast<float*>(hist_bar), slot, dparams, st, &launches)
                       : tc_adjoint<5>(c, c->adj->d_hist, static_cast<const float*>(lam), static_cast<float*>(vbar),
                                       static_cast<float*>(hist_bar), slot, dparams, st, &launches);
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_tc_adjoint: %s: %s", g_where, cudaGetErrorString(e));
  return FD_OK;
}

}  // extern "C"

// used by the rollout reverse mode: the history is an array of k_c state pointers
fd_status fd_tc_adjoint_ptrs(fd_ctx* c, const float* const* hist_host, const float* lam, float* hist_bar,
                             size_t state_stride, float* dparams, cudaStream_t st, int* launches) {
  if (c->gen) return fd_gadjoint_tc(c, hist_host, lam, nullptr, hist_bar, state_stride, dparams, st, launches);
  if (!c->adj) {
    fd_status s = adjoint_alloc(c);
    if (s != FD_OK) return s;
  }
  g_where = "";
  cudaError_t e = mark(cudaMemcpyAsync(c->adj->d_hist, hist_host, sizeof(const float*) * c->lrn->kc,
                                       cudaMemcpyHostToDevice, st),
                       "history pointers");
  if (e == cudaSuccess)
    e = (c->logn == 6) ? tc_adjoint<6>(c, c->adj->d_hist, lam, nullptr, hist_bar, state_stride, dparams, st, launches)
                       : tc_adjoint<5>(c, c->adj->d_hist, lam, nullptr, hist_bar, state_stride, dparams, st, launches);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "temporal-correction reverse mode: %s: %s", g_where,
                                            cudaGetErrorString(e));
  return FD_OK;
}
