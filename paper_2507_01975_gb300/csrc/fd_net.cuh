// fd_net.cuh -- host-side helpers shared by the learned forward path and its
// reverse mode: layer shapes, the launch of one tensor-core convolution and
// the stage-kernel arguments.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "conv_tc.cuh"
#include "fd_ctx.h"
#include "fv_learned.cuh"

namespace ldfv {
// Every helper here that launches or configures kernel templates is static:
// kernel stubs are private to each translation unit, so the helpers must be
// too (an inline function merged across units could set an attribute on one
// unit's kernel and launch the other's).

constexpr int kHidden = 64;
constexpr int kCoef = 160;
// default iteration limit of a bounded mbarrier wait (fd_options.spin_limit <= 0)
constexpr long long kSpin = 1ll << 20;

inline int stencil_cin(int l) { return l == 0 ? 2 : kHidden; }
inline int stencil_cout(int l) { return l == 5 ? kCoef : kHidden; }
inline int tc_cin(int l, int kc) { return l == 0 ? 2 * kc : kHidden; }
inline int tc_cout(int l) { return l == 5 ? 2 : kHidden; }

// One tensor-core convolution over `parts` output-channel parts of COUT_TILE.
// gelu: 0 none, 1 GELU (pre-activation to aux_out when set), 2 multiply by GELU'(aux_in)
// (with dbias set, the output's per-channel FP32 sums are added there: a bias gradient).
template <int LOGN, int COUT_TILE, int CIN = 64, int NBUF = 4>
static cudaError_t launch_conv(const LearnedState& L, const __nv_bfloat16* in, const __nv_bfloat16* wpack,
                        const float* bias, __nv_bfloat16* out, int batch, int parts, int co_base, int cout_total,
                        int gelu, cudaStream_t st, const __nv_bfloat16* aux_in = nullptr,
                        __nv_bfloat16* aux_out = nullptr, float* dbias = nullptr) {
  using Cfg = ConvCfg<LOGN, CIN, COUT_TILE, NBUF>;
  ConvArgs a;
  std::memset(&a, 0, sizeof a);
  a.in = in;
  a.w = wpack;
  a.bias = bias;
  a.out = out;
  a.batch = batch;
  a.parts = parts;
  a.co_base = co_base;
  a.cout_total = cout_total;
  a.gelu = gelu;
  a.aux_in = aux_in;
  a.aux_out = aux_out;
  a.dbias = dbias;
  a.err = L.d_err;
  a.spin_limit = L.spin;
  const int ntiles = batch * (Cfg::N / Cfg::TROWS) * parts;
  const int grid = ntiles < L.sms ? ntiles : L.sms;
  return launch_pdl(conv3x3_tc_kernel<LOGN, CIN, COUT_TILE, NBUF>, dim3(grid), dim3(Cfg::NT), Cfg::SMEM, st, a);
}

// One learned RK stage: the banded flux kernel writes the unprojected stage
// result to `scratch` (a state-sized buffer distinct from a.w and a.wout), then
// the projection kernel writes a.wout. 2 launches. Bands of kBandRows rows;
// when those would leave SMs idle (small batches) bands of kBandRowsSmall
// rows, which recompute more face rows per cell row but spread the stage over
// four times as many CTAs.
constexpr int kBandRows = 8;
constexpr int kBandRowsSmall = 2;

template <int LOGN>
static cudaError_t launch_learned_stage(const LStageArgs& a_in, float* scratch, int batch, int sms, cudaStream_t st) {
  LStageArgs a = a_in;
  a.wout = scratch;
  const bool small = batch * ((1 << LOGN) / kBandRows) < sms;
  cudaError_t e =
      small ? launch_pdl(fv_learned_flux_kernel<LOGN, kBandRowsSmall>, dim3((1 << LOGN) / kBandRowsSmall, batch),
                         dim3(256), BandCfg<LOGN, kBandRowsSmall>::SMEM, st, a)
            : launch_pdl(fv_learned_flux_kernel<LOGN, kBandRows>, dim3((1 << LOGN) / kBandRows, batch), dim3(256),
                         BandCfg<LOGN, kBandRows>::SMEM, st, a);
  LStageArgs p = a_in;
  p.w = scratch;
  if (e == cudaSuccess)
    e = launch_pdl(fv_project_kernel<LOGN>, dim3(batch), dim3(LearnedCfg<LOGN>::NT), LearnedCfg<LOGN>::SMEM, st, p);
  return e;
}

template <int LOGN>
static cudaError_t prepare_learned_stage() {
  cudaError_t e = cudaFuncSetAttribute(fv_learned_flux_kernel<LOGN, kBandRows>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BandCfg<LOGN, kBandRows>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fv_learned_flux_kernel<LOGN, kBandRowsSmall>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BandCfg<LOGN, kBandRowsSmall>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fv_project_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)LearnedCfg<LOGN>::SMEM);
}

inline LStageArgs stage_args(fd_ctx* c) {
  LStageArgs a;
  std::memset(&a, 0, sizeof a);
  const FvArgs& b = c->base;
  a.flow = c->grid.flow;
  a.forcing = c->forcing.kind;
  a.dord = c->opts.deriv_order;
  a.dt = (float)b.dt;
  a.nu = (float)b.nu;
  a.idx = (float)b.idx;
  a.idy = (float)b.idy;
  a.drag = (float)b.drag;
  a.inv_nn = (float)b.inv_nn;
  a.tw = reinterpret_cast<const float2*>(b.tw);
  a.symx = reinterpret_cast<const float*>(b.symx);
  a.symy = reinterpret_cast<const float*>(b.symy);
  a.frc = reinterpret_cast<const float*>(b.frc);
  if (c->lrn) {
    a.wl = c->lrn->d_raw + c->lrn->raw_off_wl;
    a.acc = c->lrn->acc;
    a.ablation = c->lrn->ablation;
  }
  return a;
}

}  // namespace ldfv
