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

namespace {

// name of the launch that failed last (for the error message)
thread_local const char* g_where = "";

inline cudaError_t mark(cudaError_t e, const char* where) {
  if (e != cudaSuccess && !*g_where) g_where = where;
  return e;
}

constexpr int kAdjBandRows = 8;  // rows per CTA of the flux-block reverse kernel
constexpr int kWgradMaxCols = 3 * 2 * 80;  // largest per-CTA partial: 3 dx x 2 MMAs x 80 channels

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
  return e;
}

void adjoint_free(AdjointState* A) {
  if (!A) return;
  void* ps[] = {A->wst[0], A->wst[1], A->wst[2], A->acc, A->g, A->rb, A->wbar, A->xbar, A->zeros,
                A->cbar, A->zbar[0], A->zbar[1], A->partial, A->partial_b};
  for (void* p : ps)
    if (p) cudaFree(p);
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
                  float* dW, float* db, cudaStream_t st, int* launches) {
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
  a.spin_limit = kSpin;
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
  // last layer 64 -> 160 (no activation after it): z_bar = C_bar
  if (dparams)
    e = wgrad<LOGN, 64, 80>(c, A.h[s][5], A.cbar, kCoef, 2, 64, dparams + L.raw_off_sw[5], dparams + L.raw_off_sb[5],
                            st, launches);
  if (e == cudaSuccess)
    e = mark(launch_conv<LOGN, 32, kCoef, 1>(L, A.cbar, L.d_wpack + L.pk_t5, nullptr, A.zbar[0], B, 2, 0, 64, 2, st,
                                             A.z[s][4]),
             "last-layer data gradient");
  ++*launches;
  int cur = 0;
  for (int l = 4; l >= 1 && e == cudaSuccess; --l) {
    if (dparams)
      e = wgrad<LOGN, 64, 64>(c, A.h[s][l], A.zbar[cur], 64, 1, 64, dparams + L.raw_off_sw[l],
                              dparams + L.raw_off_sb[l], st, launches);
    if (e == cudaSuccess)
      e = mark(launch_conv<LOGN, 64>(L, A.zbar[cur], L.d_wpack + L.pk_t[l - 1], nullptr, A.zbar[cur ^ 1], B, 1, 0,
                                     64, 2, st, A.z[s][l - 1]),
               "hidden-layer data gradient");
    ++*launches;
    cur ^= 1;
  }
  // first layer 2 -> 64: weight gradient with the 16-channel packed input,
  // data gradient (64 -> 2) on CUDA cores
  if (e == cudaSuccess && dparams)
    e = wgrad<LOGN, 16, 64>(c, A.h[s][0], A.zbar[cur], 64, 1, 2, dparams + L.raw_off_sw[0], dparams + L.raw_off_sb[0],
                            st, launches);
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
  LStageArgs fa = stage_args(c);
  fa.un = u;
  fa.acc = A.acc;
  if (!learned) fa.wl = A.zeros;
  for (int s = 0; s < 3 && e == cudaSuccess; ++s) {
    if (learned) e = net_forward_saved<LOGN>(c, s, ws[s], st, launches);
    if (e != cudaSuccess) break;
    fa.stage = s;
    fa.w = ws[s];
    fa.wout = A.wst[s];
    fa.coef = learned ? A.coef[s] : nullptr;
    e = mark(launch_learned_stage<LOGN>(fa, A.xbar, B, A.sms, st), "forward stage");  // xbar is free until the reverse pass
    *launches += 2;
  }
  if (e == cudaSuccess && learned) e = net_forward_saved<LOGN>(c, 3, ws[3], st, launches);
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
  sa.cbar = learned ? A.cbar : nullptr;
  sa.wl_bar = (learned && dparams) ? dparams + c->lrn->raw_off_wl : nullptr;
  sa.flow = c->grid.flow;
  sa.forcing = c->forcing.kind;
  sa.dord = c->opts.deriv_order;
  sa.nu = (float)c->base.nu;
  sa.idx = (float)c->base.idx;
  sa.idy = (float)c->base.idy;
  sa.drag = (float)c->base.drag;
  for (int s = 3; s >= 0 && e == cudaSuccess; --s) {
    sa.w = ws[s];
    sa.coef = learned ? A.coef[s] : nullptr;
    // banded flux-block reverse: bands add their scatter into the zeroed w_bar
    e = mark(cudaMemsetAsync(A.wbar, 0, fd_state_bytes(c->grid), st), "stage adjoint");
    if (e != cudaSuccess) break;
    e = mark(launch_pdl(fv_adjoint_band_kernel<LOGN, kAdjBandRows>, dim3((1 << LOGN) / kAdjBandRows, B), dim3(256),
                        AdjBandCfg<LOGN, kAdjBandRows>::SMEM, st, sa),
             "stage adjoint");
    ++*launches;
    if (e == cudaSuccess && learned) e = net_backward<LOGN>(c, s, dparams, st, launches);
    if (e != cudaSuccess) break;
    const float* x = learned ? A.xbar : nullptr;
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
  if (c->gen) return fd_set_error(c, FD_EUNSUPPORTED, "fd_step_adjoint: not built for the generic-grid path");
  if (c->lrn && (c->lrn->fno_layers > 0 || c->lrn->ablation != 0))
    return fd_set_error(c, FD_EUNSUPPORTED,
                        "fd_step_adjoint: the frequency-domain operator and the ablation variants have no reverse mode "
                        "in this build");
  c->launches = 0;
  if (!u_in || !lam_out || !lam_in) return fd_set_error(c, FD_EINVAL, "fd_step_adjoint: null state pointer");
  if (c->grid.dtype != FD_F32 || (c->grid.nx != 32 && c->grid.nx != 64))
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_step_adjoint: built for FP32 grids of 32 or 64 cells per side");
  if (c->lrn && c->lrn->kc > 0)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_step_adjoint: the temporal correction (k_c > 0) is not differentiated");
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

}  // extern "C"
