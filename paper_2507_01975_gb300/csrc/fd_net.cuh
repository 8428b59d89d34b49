// fd_net.cuh -- host-side helpers shared by the learned forward path and its
// reverse mode: layer shapes, BF16 rounding, tensor-core weight tiles and the
// launch of one tensor-core convolution.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "conv_tc.cuh"
#include "fd_ctx.h"
#include "fv_learned.cuh"

namespace ldfv {

constexpr int kHidden = 64;
constexpr int kCoef = 160;
constexpr long long kSpin = 1ll << 20;

inline int stencil_cin(int l) { return l == 0 ? 2 : kHidden; }
inline int stencil_cout(int l) { return l == 5 ? kCoef : kHidden; }
inline int tc_cin(int l, int kc) { return l == 0 ? 2 * kc : kHidden; }
inline int tc_cout(int l) { return l == 5 ? 2 : kHidden; }

// round to the nearest BF16 (ties to even), as the weights are rounded on upload
inline uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t r = u + 0x7FFF + ((u >> 16) & 1);
  return (uint16_t)(r >> 16);
}

// tensor-core tile of one conv layer part: [9 taps][cin_pad/8][cout_tile/8][8 co][8 ci]; input
// channels cin .. cin_pad - 1 are zero
inline void pack_part(const float* W, int cin, int cout_total, int co0, int cout_tile, uint16_t* dst, int cin_pad = 0) {
  if (cin_pad == 0) cin_pad = cin;
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e) {
      const int tap = a * 3 + e;
      for (int c8 = 0; c8 < cin_pad / 8; ++c8)
        for (int n8 = 0; n8 < cout_tile / 8; ++n8)
          for (int n = 0; n < 8; ++n)
            for (int k = 0; k < 8; ++k) {
              const int co = co0 + n8 * 8 + n, ci = c8 * 8 + k;
              const float w = ci < cin ? W[(((size_t)co * cin + ci) * 3 + a) * 3 + e] : 0.0f;
              const size_t idx = ((((size_t)tap * (cin_pad / 8) + c8) * (cout_tile / 8) + n8) * 8 + n) * 8 + k;
              dst[idx] = bf16_bits(w);
            }
      (void)cout_total;
    }
}

inline size_t part_elems(int cin, int cout_tile) { return (size_t)9 * cin * cout_tile; }

// Weight tile of the reverse-mode (data-gradient) convolution of a layer
// W[cout][cin][3][3]: the transposed, flipped kernel Wt[ci'][co'][a][e] =
// W[co'][ci'][2 - a][2 - e] seen as a layer with cin' = cout and cout' = cin.
inline void pack_part_transposed(const float* W, int cin, int cout, int co0, int cout_tile, uint16_t* dst) {
  std::vector<float> wt((size_t)cin * cout * 9);
  for (int o = 0; o < cout; ++o)
    for (int ci = 0; ci < cin; ++ci)
      for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 3; ++e)
          wt[(((size_t)ci * cout + o) * 3 + a) * 3 + e] = W[(((size_t)o * cin + ci) * 3 + (2 - a)) * 3 + (2 - e)];
  pack_part(wt.data(), cout, cin, co0, cout_tile, dst);
}

// One tensor-core convolution over `parts` output-channel parts of COUT_TILE.
// gelu: 0 none, 1 GELU (pre-activation to aux_out when set), 2 multiply by GELU'(aux_in).
template <int LOGN, int COUT_TILE, int CIN = 64, int NBUF = 2>
cudaError_t launch_conv(const LearnedState& L, const __nv_bfloat16* in, const __nv_bfloat16* wpack,
                        const float* bias, __nv_bfloat16* out, int batch, int parts, int co_base, int cout_total,
                        int gelu, cudaStream_t st, const __nv_bfloat16* aux_in = nullptr,
                        __nv_bfloat16* aux_out = nullptr) {
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
  a.err = L.d_err;
  a.spin_limit = kSpin;
  const int ntiles = batch * (Cfg::N / Cfg::TROWS) * parts;
  const int grid = ntiles < L.sms ? ntiles : L.sms;
  conv3x3_tc_kernel<LOGN, CIN, COUT_TILE, NBUF><<<grid, Cfg::NT, Cfg::SMEM, st>>>(a);
  return cudaGetLastError();
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
  }
  return a;
}

}  // namespace ldfv
