// fd_learned.cu -- the learnable module behind the C ABI: parameter upload
// and packing, workspace, and the launch sequence of one learned time step
// (stencil network on the tensor cores, learned FV stage, temporal
// correction), replayed as a CUDA graph of k_c steps during rollouts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/fd.h"
#include "conv_tc.cuh"
#include "fd_ctx.h"
#include "fd_net.cuh"
#include "fv_learned.cuh"

using namespace ldfv;

// frequency-domain operator O_F of one stage state (fd_fno.cu): writes L.fno_out
cudaError_t fd_fno_forward(fd_ctx* c, const float* u, cudaStream_t st);
int fd_fno_launches(int layers);
int64_t fd_fno_param_count(int layers, int modes, int width, int cin, int cout);
cudaError_t fd_fno_prepare();
cudaError_t fd_fno_tc(fd_ctx* c, const float* const* hist, cudaStream_t st);
size_t fd_fno_rp_count(int layers, int modes, int width);
cudaError_t fd_fno_pack(LearnedState& L, cudaStream_t st);

namespace {

// kernel launches of one learned step: per stage the stencil network (input
// packing, six layers with the last one in two launches) and the flux and
// projection kernels; the temporal correction adds its network and the
// corrected projection
constexpr int kLaunchesPerStep = 4 * (8 + 2);
constexpr int kLaunchesPerStepFreqOnly = 4 * 2;  // ablation 2: no stencil network
constexpr int kLaunchesTc = 7 + 1;

// launches of the four stages of one step without O_F and the temporal correction
int step_launches(const LearnedState& L) { return L.ablation == 2 ? kLaunchesPerStepFreqOnly : kLaunchesPerStep; }

// launches of one temporal correction (CNN head or FNO, plus the corrected projection)
int tc_launches(const LearnedState& L) { return L.tcf_layers > 0 ? fd_fno_launches(L.tcf_layers) + 1 : kLaunchesTc; }

thread_local const char* g_where = "";  // the launch group that failed last

template <int LOGN>
cudaError_t prepare_kernels() {
  cudaError_t e;
  e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, 64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ConvCfg<LOGN, 64, 64>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, 64, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ConvCfg<LOGN, 64, 32>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(conv3x3_tc_kernel<LOGN, 16, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ConvCfg<LOGN, 16, 64>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fv_correct_project_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)LearnedCfg<LOGN>::SMEM);
  if (e != cudaSuccess) return e;
  e = prepare_learned_stage<LOGN>();
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(conv_in_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((64 * 16 * 9 + 64) * sizeof(float)));
}

// network of six conv3x3 layers from first-layer inputs (pointer array `hist`
// of cin/2 states) to the chunk-plane output of the last hidden layer in act0
template <int LOGN>
cudaError_t run_trunk(fd_ctx* c, const float* const* hist, int cin, size_t pk_first, const float* b0,
                      const size_t* pk_hidden, const size_t* raw_b, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const int B = c->grid.batch;
  // first layer on the tensor cores: inputs packed to 16 BF16 channels
  PackArgs pa;
  pa.hist = hist;
  pa.single = nullptr;
  pa.out = L.act1;
  pa.batch = B;
  pa.cin = cin;
  const size_t pix = (size_t)B << (2 * LOGN);
  const int blocks = (int)((pix + 255) / 256 < (size_t)(4 * L.sms) ? (pix + 255) / 256 : (size_t)(4 * L.sms));
  cudaError_t e = launch_pdl(pack_input_kernel<LOGN>, dim3(blocks), dim3(256), 0, st, pa);
  if (e == cudaSuccess)
    e = launch_conv<LOGN, 64, 16>(L, L.act1, L.d_wpack + pk_first, b0, L.act0, B, 1, 0, 64, 1, st);
  __nv_bfloat16* bufs[2] = {L.act0, L.act1};
  for (int l = 1; l <= 4 && e == cudaSuccess; ++l) {
    e = launch_conv<LOGN, 64>(L, bufs[(l - 1) & 1], L.d_wpack + pk_hidden[l - 1], L.d_raw + raw_b[l], bufs[l & 1], B,
                              1, 0, 64, 1, st);
  }
  return e;  // layer 4 output is in act0
}

template <int LOGN>
cudaError_t run_stencil_net(fd_ctx* c, const float* const* hist, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const int B = c->grid.batch;
  size_t hidden[4] = {L.pk_stencil[0], L.pk_stencil[1], L.pk_stencil[2], L.pk_stencil[3]};
  cudaError_t e = run_trunk<LOGN>(c, hist, 2, L.pk_stencil_first, L.d_raw + L.raw_off_sb[0], hidden,
                                  L.raw_off_sb, st);
  if (e != cudaSuccess) return e;
  // last layer 64 -> 160: two 64-channel parts and one 32-channel part
  e = launch_conv<LOGN, 64>(L, L.act0, L.d_wpack + L.pk_stencil[4], L.d_raw + L.raw_off_sb[5], L.coef, B, 2, 0,
                            kCoef, 0, st);
  if (e != cudaSuccess) return e;
  return launch_conv<LOGN, 32>(L, L.act0, L.d_wpack + L.pk_stencil_last32, L.d_raw + L.raw_off_sb[5], L.coef, B, 1,
                               128, kCoef, 0, st);
}

template <int LOGN>
cudaError_t run_tc_net(fd_ctx* c, const float* const* hist, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const int B = c->grid.batch;
  cudaError_t e = run_trunk<LOGN>(c, hist, 2 * L.kc, L.pk_tc_first, L.d_raw + L.raw_off_tb[0], L.pk_tc,
                                  L.raw_off_tb, st);
  if (e != cudaSuccess) return e;
  ConvOut2Args oa;
  oa.in = L.act0;
  oa.w = L.d_raw + L.raw_off_tw[5];
  oa.bias = L.d_raw + L.raw_off_tb[5];
  oa.out = L.corr;
  oa.batch = B;
  const size_t pix = (size_t)B << (2 * LOGN);
  const int blocks = (int)((pix + 255) / 256 < (size_t)(4 * L.sms) ? (pix + 255) / 256 : (size_t)(4 * L.sms));
  return launch_pdl(conv_out2_kernel<LOGN>, dim3(blocks), dim3(256), 0, st, oa);
}

// One learned time step s_in -> s_out. ptr_in / ptr_w: device pointer arrays
// {s_in} and {wbuf} for the first network layer; tc_hist: k_c states or null.
template <int LOGN>
cudaError_t learned_step(fd_ctx* c, const float* s_in, float* s_out, const float* const* ptr_in,
                         const float* const* ptr_w, const float* const* tc_hist, cudaStream_t st) {
  LearnedState& L = *c->lrn;
  const int B = c->grid.batch;
  cudaError_t e = cudaSuccess;
  LStageArgs a = stage_args(c);
  a.un = s_in;
  a.coef = L.coef;
  if (L.ablation == 2) a.coef = nullptr;  // frequency-domain operator only: no stencil network
  for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
    if (L.ablation != 2) e = run_stencil_net<LOGN>(c, s == 0 ? ptr_in : ptr_w, st);
    if (e != cudaSuccess) {
      g_where = "stencil network";
      break;
    }
    if (L.fno_layers > 0) {
      e = fd_fno_forward(c, s == 0 ? s_in : L.wbuf, st);
      if (e != cudaSuccess) {
        g_where = "frequency-domain operator";
        break;
      }
      a.fno = L.fno_out;
    }
    a.stage = s;
    a.w = s == 0 ? s_in : L.wbuf;
    a.wout = s < 3 ? L.wbuf : s_out;
    e = launch_learned_stage<LOGN>(a, L.ws, B, L.sms, st);
    if (e != cudaSuccess) g_where = "flux / projection kernels";
  }
  if (e == cudaSuccess && tc_hist) {
    e = L.tcf_layers > 0 ? fd_fno_tc(c, tc_hist, st) : run_tc_net<LOGN>(c, tc_hist, st);
    if (e == cudaSuccess) {
      a.corr = L.corr;
      a.wout = s_out;
      e = launch_pdl(fv_correct_project_kernel<LOGN>, dim3(B), dim3(LearnedCfg<LOGN>::NT), LearnedCfg<LOGN>::SMEM,
                     st, a);
    }
  }
  return e;
}

template <int LOGN>
cudaError_t coef_to_f32(fd_ctx* c, float* out, cudaStream_t st);

__global__ void coef_unpack_kernel(const __nv_bfloat16* in, float* out, int batch, int logn) {
  const int N = 1 << logn;
  const size_t total = (size_t)batch * kCoef * N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % N), j = (int)((e / N) % N);
    const int ch = (int)((e / ((size_t)N * N)) % kCoef);
    const int b = (int)(e / ((size_t)N * N * kCoef));
    out[e] = __bfloat162float(in[((((size_t)b * (kCoef / 8) + ch / 8) * N + j) * N + i) * 8 + (ch & 7)]);
  }
}

// ---------------------------------------------------------------------------
// parameter upload on the device: BF16 rounding of the network weights, the
// first layer's transposed kernel in FP32, and every tensor-core weight tile
// (forward tiles and the transposed, flipped tiles of the data gradients)
// ---------------------------------------------------------------------------
struct PackDesc {
  uint32_t src_off;     // layer weights W[cout][cin][3][3] in the raw array
  uint32_t dst_off;     // first element of the tile in the packed array
  uint32_t count;       // 9 x cin_pad x cout_tile
  uint32_t cin_tile;    // input channels of the tile that carry data
  uint32_t cin_pad;     // input channels of the tile (multiple of 16)
  uint32_t cout_tile;   // output channels of the tile
  uint32_t co0;         // first output channel of the tile
  uint32_t layer_cin;   // Cin of the layer
  uint32_t transposed;  // 1: tile of the data gradient (transposed, flipped kernel)
};

__device__ __forceinline__ float round_bf16_dev(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void prep_raw_kernel(const float* params, float* raw, size_t nparams, const uint32_t* ranges, int nranges,
                                size_t off_w0, size_t off_w0t, size_t off_zero, size_t off_tw0, size_t off_tw0t,
                                int tc_cin) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nparams; k += (size_t)gridDim.x * blockDim.x) {
    float v = params[k];
    for (int r = 0; r < nranges; ++r)
      if (k >= ranges[2 * r] && k < (size_t)ranges[2 * r] + ranges[2 * r + 1]) v = round_bf16_dev(v);
    raw[k] = v;
  }
  // first layer, transposed and flipped: w0t[ci][o][t] = W0[o][ci][8 - t]
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < 2 * 64 * 9; k += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(k / 576), o = (int)((k / 9) % 64), t = (int)(k % 9);
    raw[off_w0t + k] = round_bf16_dev(params[off_w0 + (o * 2 + ci) * 9 + 8 - t]);
  }
  // the same for the temporal-correction network's first layer (tc_cin = 2 k_c inputs)
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < (size_t)tc_cin * 64 * 9;
       k += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(k / 576), o = (int)((k / 9) % 64), t = (int)(k % 9);
    raw[off_tw0t + k] = round_bf16_dev(params[off_tw0 + (o * tc_cin + ci) * 9 + 8 - t]);
  }
  if (blockIdx.x == 0 && threadIdx.x < 8) raw[off_zero + threadIdx.x] = 0.f;
}

// tile element (dy, c8, dx, n8, n, k): input channel ci = 8 c8 + k, output
// channel co = co0 + 8 n8 + n, tap = 3 dy + dx. The three dx blocks of one
// (dy, c8) are adjacent, so one MMA with N = 3 x cout_tile covers all three.
__global__ void pack_tiles_kernel(const float* raw, __nv_bfloat16* pk, const PackDesc* descs) {
  const PackDesc d = descs[blockIdx.y];
  const float* W = raw + d.src_off;
  const uint32_t n8s = d.cout_tile / 8, c8s = d.cin_pad / 8;
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < d.count; idx += gridDim.x * blockDim.x) {
    const uint32_t k = idx & 7, n = (idx >> 3) & 7;
    const uint32_t n8 = (idx >> 6) % n8s;
    const uint32_t dx = (idx / (64 * n8s)) % 3;
    const uint32_t c8 = (idx / (64 * n8s * 3)) % c8s;
    const uint32_t dy = idx / (64 * n8s * 3 * c8s);
    const uint32_t tap = dy * 3 + dx;
    const uint32_t ci = c8 * 8 + k, co = d.co0 + n8 * 8 + n;
    float v = 0.f;
    if (ci < d.cin_tile)
      v = d.transposed ? W[((size_t)ci * d.layer_cin + co) * 9 + (8 - tap)] : W[((size_t)co * d.layer_cin + ci) * 9 + tap];
    pk[d.dst_off + idx] = __float2bfloat16_rn(v);
  }
}

// raw offsets, tile offsets and the tile recipe of a context (fixed by k_c)
void plan_layout(LearnedState& L, std::vector<PackDesc>& descs, std::vector<uint32_t>& ranges) {
  size_t off = 0;
  L.raw_off_wl = off;
  off += 80;
  for (int l = 0; l < 6; ++l) {
    L.raw_off_sw[l] = off;
    ranges.push_back((uint32_t)off);
    ranges.push_back((uint32_t)(stencil_cout(l) * stencil_cin(l) * 9));
    off += (size_t)stencil_cout(l) * stencil_cin(l) * 9;
    L.raw_off_sb[l] = off;
    off += stencil_cout(l);
  }
  if (L.kc > 0 && L.tcf_layers > 0) {  // FNO temporal correction: FP32, no rounding range
    L.raw_off_tcf = off;
    off += (size_t)fd_fno_param_count(L.tcf_layers, L.tcf_modes, L.tcf_width, 2 * L.kc, 2);
  } else if (L.kc > 0)
    for (int l = 0; l < 6; ++l) {
      L.raw_off_tw[l] = off;
      ranges.push_back((uint32_t)off);
      ranges.push_back((uint32_t)(tc_cout(l) * tc_cin(l, L.kc) * 9));
      off += (size_t)tc_cout(l) * tc_cin(l, L.kc) * 9;
      L.raw_off_tb[l] = off;
      off += tc_cout(l);
    }
  L.raw_off_fno = off;  // O_F parameters stay FP32 (no rounding range)
  off += (size_t)fd_fno_param_count(L.fno_layers, L.fno_modes, L.fno_width, 2, 8);
  L.raw_off_w0t = off;
  off += 2 * 64 * 9;
  L.raw_off_tw0t = off;
  if (L.kc > 0 && L.tcf_layers == 0) off += (size_t)2 * L.kc * 64 * 9;
  L.raw_off_zero = off;
  off += 8;
  L.raw_total = off;
  size_t pk = 0;
  auto add = [&](size_t src, int cin_tile, int cin_pad, int cout_tile, int co0, int layer_cin, int tr) {
    PackDesc d;
    d.src_off = (uint32_t)src;
    d.dst_off = (uint32_t)pk;
    d.count = (uint32_t)(9 * cin_pad * cout_tile);
    d.cin_tile = (uint32_t)cin_tile;
    d.cin_pad = (uint32_t)cin_pad;
    d.cout_tile = (uint32_t)cout_tile;
    d.co0 = (uint32_t)co0;
    d.layer_cin = (uint32_t)layer_cin;
    d.transposed = (uint32_t)tr;
    descs.push_back(d);
    pk += d.count;
    return (size_t)d.dst_off;
  };
  L.pk_stencil_first = add(L.raw_off_sw[0], 2, 16, 64, 0, 2, 0);
  for (int l = 1; l <= 4; ++l) L.pk_stencil[l - 1] = add(L.raw_off_sw[l], 64, 64, 64, 0, 64, 0);
  L.pk_stencil[4] = add(L.raw_off_sw[5], 64, 64, 64, 0, 64, 0);
  add(L.raw_off_sw[5], 64, 64, 64, 64, 64, 0);
  L.pk_stencil_last32 = add(L.raw_off_sw[5], 64, 64, 32, 128, 64, 0);
  for (int l = 1; l <= 4; ++l) L.pk_t[l - 1] = add(L.raw_off_sw[l], 64, 64, 64, 0, 64, 1);
  L.pk_t5 = add(L.raw_off_sw[5], kCoef, kCoef, 32, 0, 64, 1);
  add(L.raw_off_sw[5], kCoef, kCoef, 32, 32, 64, 1);
  if (L.kc > 0 && L.tcf_layers == 0) {
    L.pk_tc_first = add(L.raw_off_tw[0], 2 * L.kc, 16, 64, 0, 2 * L.kc, 0);
    for (int l = 1; l <= 4; ++l) L.pk_tc[l - 1] = add(L.raw_off_tw[l], 64, 64, 64, 0, 64, 0);
    // reverse mode: transposed, flipped tiles of the hidden layers and of the
    // last layer (2 cotangent channels, padded to 16, -> 64)
    for (int l = 1; l <= 4; ++l) L.pk_tc_t[l - 1] = add(L.raw_off_tw[l], 64, 64, 64, 0, 64, 1);
    L.pk_tc_t5 = add(L.raw_off_tw[5], 2, 16, 64, 0, 64, 1);
  }
  L.pk_total = pk;
}

cudaError_t upload_params(LearnedState& L, const float* params, cudaStream_t st) {
  const int tc_cin = (L.kc > 0 && L.tcf_layers == 0) ? 2 * L.kc : 0;
  prep_raw_kernel<<<2 * L.sms, 256, 0, st>>>(params, L.d_raw, (size_t)L.nparams, L.d_ranges, L.nranges,
                                             L.raw_off_sw[0], L.raw_off_w0t, L.raw_off_zero, L.raw_off_tw[0],
                                             L.raw_off_tw0t, tc_cin);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  pack_tiles_kernel<<<dim3(32, L.ndesc), 256, 0, st>>>(L.d_raw, L.d_wpack, reinterpret_cast<const PackDesc*>(L.d_desc));
  e = cudaGetLastError();
  if (e == cudaSuccess && (L.fno_layers > 0 || L.tcf_layers > 0)) e = fd_fno_pack(L, st);
  return e;
}

}  // namespace

// ---------------------------------------------------------------------------
// entry points used by fd_api.cu
// ---------------------------------------------------------------------------
// parameters of a Fourier neural operator with cin inputs and cout outputs
// (O_F: 2 -> 8; the FNO temporal correction: 2 k_c -> 2; layout in include/fd.h)
int64_t fd_fno_param_count(int layers, int modes, int width, int cin, int cout) {
  if (layers <= 0) return 0;
  const int64_t c = width;
  return c * cin + c + (int64_t)layers * (2 * (int64_t)modes * modes * c * c * 2 + c * c + c) + cout * c + cout;
}

int64_t fd_learned_param_count(const fd_options& o) {
  // a model that learns the scalar: W_Ls, one more input channel, 80 more outputs
  const int sl = o.scalar_learned ? 1 : 0;
  int64_t n = 80 + 80 * sl;
  for (int l = 0; l < 6; ++l) {
    const int64_t ci = stencil_cin(l) + (l == 0 ? sl : 0), co = stencil_cout(l) + (l == 5 ? 80 * sl : 0);
    n += co * ci * 9 + co;
  }
  if (o.k_c > 0 && o.tc_fno_layers > 0)
    n += fd_fno_param_count(o.tc_fno_layers, o.tc_fno_modes, o.tc_fno_width, 2 * o.k_c, 2);
  else if (o.k_c > 0)
    for (int l = 0; l < 6; ++l) n += (int64_t)tc_cout(l) * tc_cin(l, o.k_c) * 9 + tc_cout(l);
  return n + fd_fno_param_count(o.fno_layers, o.fno_modes, o.fno_width, 2, 8);
}

fd_status fd_learned_init(fd_ctx* c) {
  const fd_grid& g = c->grid;
  if (g.dtype != FD_F32) return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: the learned path is built for FP32");
  if (g.nx != 32 && g.nx != 64)
    return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: the learned path is built for N = 32 or 64");
  if (c->opts.k_c < 0 || c->opts.k_c > 8) return fd_set_error(nullptr, FD_EINVAL, "fd_init: k_c must be in [0, 8]");
  LearnedState* L = new (std::nothrow) LearnedState();
  if (!L) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: out of host memory");
  c->lrn = L;
  L->kc = c->opts.k_c;
  L->fno_layers = c->opts.fno_layers;
  L->fno_modes = c->opts.fno_modes;
  L->fno_width = c->opts.fno_width;
  L->tcf_layers = c->opts.tc_fno_layers;
  L->tcf_modes = c->opts.tc_fno_modes;
  L->tcf_width = c->opts.tc_fno_width;
  L->ablation = c->opts.ablation;
  L->spin = c->opts.spin_limit > 0 ? (long long)c->opts.spin_limit : kSpin;
  L->nparams = fd_learned_param_count(c->opts);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&L->sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t NN = (size_t)g.nx * g.ny;
  const size_t B = g.batch;
  const size_t state = B * 2 * NN * sizeof(float);
  L->nring = (L->kc > 0 ? L->kc : 1) + 1;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void**)&L->act0, B * kHidden * NN * 2);
  alloc((void**)&L->act1, B * kHidden * NN * 2);
  alloc((void**)&L->coef, B * kCoef * NN * 2);
  alloc((void**)&L->acc, state);
  alloc((void**)&L->wbuf, state);
  alloc((void**)&L->ws, state);
  alloc((void**)&L->corr, state);
  alloc((void**)&L->ring, state * L->nring);
  alloc((void**)&L->d_err, sizeof(unsigned));
  alloc((void**)&L->d_ptrs, sizeof(float*) * (L->nring + 1 + 8 * L->nring));
  if (L->fno_layers > 0 || L->tcf_layers > 0) {  // scratch shared by O_F and the FNO temporal correction
    const size_t C = L->fno_width > L->tcf_width ? L->fno_width : L->tcf_width;
    const size_t M = L->fno_modes > L->tcf_modes ? L->fno_modes : L->tcf_modes;
    alloc((void**)&L->fno_v[0], B * C * NN * sizeof(float));
    alloc((void**)&L->fno_v[1], B * C * NN * sizeof(float));
    alloc((void**)&L->fno_y, B * C * NN * sizeof(float));
    alloc((void**)&L->fno_s, B * C * 2 * M * M * sizeof(float2));
    alloc((void**)&L->fno_s2, B * C * 2 * M * M * sizeof(float2));
  }
  if (L->fno_layers > 0) {
    alloc((void**)&L->fno_out, B * 8 * NN * sizeof(float));
    alloc((void**)&L->fno_rp, fd_fno_rp_count(L->fno_layers, L->fno_modes, L->fno_width) * sizeof(float2));
    alloc((void**)&L->fno_rph, fd_fno_rp_count(L->fno_layers, L->fno_modes, L->fno_width) * sizeof(float2));
  }
  if (L->tcf_layers > 0) {
    alloc((void**)&L->tcf_rp, fd_fno_rp_count(L->tcf_layers, L->tcf_modes, L->tcf_width) * sizeof(float2));
    alloc((void**)&L->tcf_rph, fd_fno_rp_count(L->tcf_layers, L->tcf_modes, L->tcf_width) * sizeof(float2));
  }
  std::vector<PackDesc> descs;
  std::vector<uint32_t> ranges;
  plan_layout(*L, descs, ranges);
  L->ndesc = (int)descs.size();
  L->nranges = (int)(ranges.size() / 2);
  alloc((void**)&L->d_raw, L->raw_total * sizeof(float));
  alloc((void**)&L->d_wpack, L->pk_total * sizeof(__nv_bfloat16));
  alloc((void**)&L->d_stage, (size_t)L->nparams * sizeof(float));
  alloc(&L->d_desc, descs.size() * sizeof(PackDesc));
  alloc((void**)&L->d_ranges, ranges.size() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(L->d_desc, descs.data(), descs.size() * sizeof(PackDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(L->d_ranges, ranges.data(), ranges.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(L->d_err, 0, sizeof(unsigned));
  if (e == cudaSuccess) {
    // pointer arrays: [0, nring) single ring slots, [nring] wbuf, then k_c-long
    // histories ending at each ring slot
    std::vector<const float*> h(L->nring + 1 + 8 * L->nring, nullptr);
    for (int r = 0; r < L->nring; ++r) h[r] = L->ring + r * B * 2 * NN;
    h[L->nring] = L->wbuf;
    for (int r = 0; r < L->nring; ++r)
      for (int s = 0; s < L->kc; ++s) h[L->nring + 1 + 8 * r + s] = L->ring + (r - L->kc + s + 1) * B * 2 * NN;
    e = cudaMemcpy(L->d_ptrs, h.data(), sizeof(float*) * h.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = (g.nx == 64) ? prepare_kernels<6>() : prepare_kernels<5>();
  if (e == cudaSuccess && (L->fno_layers > 0 || L->tcf_layers > 0)) e = fd_fno_prepare();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: learned workspace: %s", cudaGetErrorString(e));
  return FD_OK;
}

void fd_learned_free(fd_ctx* c) {
  LearnedState* L = c->lrn;
  if (!L) return;
  if (L->graph) cudaGraphExecDestroy(L->graph);
  if (L->cap_stream) cudaStreamDestroy(L->cap_stream);
  void* ps[] = {L->d_raw,  L->d_wpack, L->d_stage, L->d_desc,         (void*)L->d_ranges, L->act0, L->act1,
                L->coef,   L->acc,     L->wbuf,    L->ws,             L->corr,            L->ring,
                (void*)L->d_ptrs,
                L->d_err,  L->fno_v[0], L->fno_v[1], L->fno_y,        L->fno_s,           L->fno_s2,
                L->fno_out, L->fno_rp, L->tcf_rp, L->fno_rph, L->tcf_rph};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete L;
  c->lrn = nullptr;
}

extern "C" {

int64_t fd_param_count(const fd_ctx* c) {
  return (c && c->lrn) ? c->lrn->nparams : (c && c->glrn) ? c->glrn->nparams : 0;
}

fd_status fd_set_params(fd_ctx* c, const float* params, int64_t count, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_set_params: null context");
  if (!c->lrn && !c->glrn)
    return fd_set_error(c, FD_EINVAL, "fd_set_params: context was created without the learned option");
  if (!params) return fd_set_error(c, FD_EINVAL, "fd_set_params: null parameter array");
  if (c->glrn) return fd_glearned_set_params(c, params, count, false, static_cast<cudaStream_t>(stream));
  LearnedState& L = *c->lrn;
  if (count != L.nparams)
    return fd_set_error(c, FD_EINVAL, "fd_set_params: expected %lld values, got %lld", (long long)L.nparams,
                        (long long)count);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(L.d_stage, params, (size_t)count * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = upload_params(L, L.d_stage, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_set_params: %s", cudaGetErrorString(e));
  L.ready = true;
  return FD_OK;
}

fd_status fd_set_params_device(fd_ctx* c, const float* params, int64_t count, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_set_params_device: null context");
  if (!c->lrn && !c->glrn)
    return fd_set_error(c, FD_EINVAL, "fd_set_params_device: context was created without the learned option");
  if (!params) return fd_set_error(c, FD_EINVAL, "fd_set_params_device: null parameter array");
  if (c->glrn) return fd_glearned_set_params(c, params, count, true, static_cast<cudaStream_t>(stream));
  LearnedState& L = *c->lrn;
  if (count != L.nparams)
    return fd_set_error(c, FD_EINVAL, "fd_set_params_device: expected %lld values, got %lld", (long long)L.nparams,
                        (long long)count);
  cudaError_t e = upload_params(L, params, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_set_params_device: %s", cudaGetErrorString(e));
  L.ready = true;
  return FD_OK;
}

fd_status fd_network_forward(fd_ctx* c, const void* u, float* coef_out, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_network_forward: null context");
  if (c->glrn) {
    if (!c->glrn->ready) return fd_set_error(c, FD_EINVAL, "fd_network_forward: parameters not set");
    if (!u) return fd_set_error(c, FD_EINVAL, "fd_network_forward: null state pointer");
    return fd_glearned_network(c, u, coef_out, static_cast<cudaStream_t>(stream));
  }
  if (!c->lrn || !c->lrn->ready) return fd_set_error(c, FD_EINVAL, "fd_network_forward: parameters not set");
  if (!u) return fd_set_error(c, FD_EINVAL, "fd_network_forward: null state pointer");
  LearnedState& L = *c->lrn;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = fd_state_bytes(c->grid);
  // the first layer reads its input through a pointer array: stage through wbuf
  cudaError_t e = cudaMemcpyAsync(L.wbuf, u, bytes, cudaMemcpyDeviceToDevice, st);
  const float* const* pw = L.d_ptrs + L.nring;
  if (e == cudaSuccess) e = (c->grid.nx == 64) ? run_stencil_net<6>(c, pw, st) : run_stencil_net<5>(c, pw, st);
  c->launches = 8;
  if (e == cudaSuccess && coef_out) {
    coef_unpack_kernel<<<4 * L.sms, 256, 0, st>>>(L.coef, coef_out, c->grid.batch, c->logn);
    e = cudaGetLastError();
    ++c->launches;
  }
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_network_forward: %s", cudaGetErrorString(e));
  return FD_OK;
}

}  // extern "C"

// learned rollout: ring slot r holds the state after step (base + r) of the
// current group; a group of G = max(k_c, 1) steps is captured once as a CUDA
// graph (with the temporal correction at its last step) and replayed.
fd_status fd_learned_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                             cudaStream_t st, bool allow_graph) {
  LearnedState& L = *c->lrn;
  if (!L.ready) return fd_set_error(c, FD_EINVAL, "fd_rollout: learned parameters not set (fd_set_params)");
  const size_t bytes = fd_state_bytes(c->grid);
  const size_t slot = bytes / sizeof(float);
  const int G = L.kc > 0 ? L.kc : 1;
  auto step_fn = [&](int r, bool tc, cudaStream_t s) -> cudaError_t {
    const float* const* pin = L.d_ptrs + r;
    const float* const* pw = L.d_ptrs + L.nring;
    const float* const* ph = tc ? L.d_ptrs + L.nring + 1 + 8 * r : nullptr;  // ring[r - k_c + 1 .. r]
    if (c->grid.nx == 64) return learned_step<6>(c, L.ring + r * slot, L.ring + (r + 1) * slot, pin, pw, ph, s);
    return learned_step<5>(c, L.ring + r * slot, L.ring + (r + 1) * slot, pin, pw, ph, s);
  };
  int launches = 0;
  g_where = "state copy";
  cudaError_t e = cudaMemcpyAsync(L.ring, u0, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) g_where = "";
  const bool use_graph = allow_graph && save_every == 0;
  if (e == cudaSuccess && use_graph && n_steps >= G && !L.graph) {
    // capture one group on the side stream; the history for the temporal
    // correction of the group's last step is ring[0 .. k_c - 1]
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(L.cap_stream, cudaStreamCaptureModeThreadLocal);
    for (int r = 0; r < G && e == cudaSuccess; ++r) e = step_fn(r, L.kc > 0 && r == G - 1, L.cap_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.ring, L.ring + G * slot, bytes, cudaMemcpyDeviceToDevice, L.cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(L.cap_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&L.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    L.graph_steps = G;
  }
  int done = 0;
  int snap = 0;
  if (e == cudaSuccess && use_graph && L.graph) {
    for (; done + G <= n_steps && e == cudaSuccess; done += G) {
      e = cudaGraphLaunch(L.graph, st);
      launches += G * (step_launches(L) + 4 * fd_fno_launches(L.fno_layers)) + (L.kc > 0 ? tc_launches(L) : 0);
    }
  }
  // remaining steps (or every step when snapshots are requested): direct launches
  for (; done < n_steps && e == cudaSuccess; ++done) {
    const int r = done % G;
    const bool tc = L.kc > 0 && ((done + 1) % L.kc == 0);
    e = step_fn(r, tc, st);
    launches += step_launches(L) + 4 * fd_fno_launches(L.fno_layers) + (tc ? tc_launches(L) : 0);
    if (e == cudaSuccess && save_every > 0 && traj && ((done + 1) % save_every) == 0) {
      e = cudaMemcpyAsync(static_cast<float*>(traj) + (size_t)snap * slot, L.ring + (r + 1) * slot, bytes,
                          cudaMemcpyDeviceToDevice, st);
      ++snap;
    }
    if (e == cudaSuccess && r == G - 1)
      e = cudaMemcpyAsync(L.ring, L.ring + G * slot, bytes, cudaMemcpyDeviceToDevice, st);
  }
  const int rlast = n_steps == 0 ? 0 : (n_steps % G == 0 ? 0 : n_steps % G);
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, L.ring + rlast * slot, bytes, cudaMemcpyDeviceToDevice, st);
  c->launches = launches;
  if (e != cudaSuccess)
    return fd_set_error(c, FD_ECUDA, "fd_rollout (learned): %s: %s", g_where, cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_learned_error_flag(fd_ctx* c) {
  if (!c->lrn) return FD_OK;
  unsigned h = 0;
  if (cudaMemcpy(&h, c->lrn->d_err, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fd_set_error(c, FD_ECUDA, "error flag read failed");
  if (h) {
    // reported once: the next check sees only waits that give up after this one
    cudaMemset(c->lrn->d_err, 0, sizeof h);
    return fd_set_error(c, FD_ETIMEOUT, "a bounded device wait of the tensor-core convolution gave up (0x%x)", h);
  }
  return FD_OK;
}
