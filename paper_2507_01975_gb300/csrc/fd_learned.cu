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

namespace {

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
  e = cudaFuncSetAttribute(fv_learned_stage_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)LearnedCfg<LOGN>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fv_correct_project_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)LearnedCfg<LOGN>::SMEM);
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
  pack_input_kernel<LOGN><<<blocks, 256, 0, st>>>(pa);
  cudaError_t e = cudaGetLastError();
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
  conv_out2_kernel<LOGN><<<blocks, 256, 0, st>>>(oa);
  return cudaGetLastError();
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
  for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
    e = run_stencil_net<LOGN>(c, s == 0 ? ptr_in : ptr_w, st);
    if (e != cudaSuccess) break;
    a.stage = s;
    a.w = s == 0 ? s_in : L.wbuf;
    a.wout = s < 3 ? L.wbuf : s_out;
    fv_learned_stage_kernel<LOGN><<<B, LearnedCfg<LOGN>::NT, LearnedCfg<LOGN>::SMEM, st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && tc_hist) {
    e = run_tc_net<LOGN>(c, tc_hist, st);
    if (e == cudaSuccess) {
      a.corr = L.corr;
      a.wout = s_out;
      fv_correct_project_kernel<LOGN><<<B, LearnedCfg<LOGN>::NT, LearnedCfg<LOGN>::SMEM, st>>>(a);
      e = cudaGetLastError();
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

}  // namespace

// ---------------------------------------------------------------------------
// entry points used by fd_api.cu
// ---------------------------------------------------------------------------
int64_t fd_learned_param_count(int kc) {
  int64_t n = 80;
  for (int l = 0; l < 6; ++l) n += (int64_t)stencil_cout(l) * stencil_cin(l) * 9 + stencil_cout(l);
  if (kc > 0)
    for (int l = 0; l < 6; ++l) n += (int64_t)tc_cout(l) * tc_cin(l, kc) * 9 + tc_cout(l);
  return n;
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
  L->nparams = fd_learned_param_count(L->kc);
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
  alloc((void**)&L->corr, state);
  alloc((void**)&L->ring, state * L->nring);
  alloc((void**)&L->d_err, sizeof(unsigned));
  alloc((void**)&L->d_ptrs, sizeof(float*) * (L->nring + 1 + 8 * L->nring));
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
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: learned workspace: %s", cudaGetErrorString(e));
  return FD_OK;
}

void fd_learned_free(fd_ctx* c) {
  LearnedState* L = c->lrn;
  if (!L) return;
  if (L->graph) cudaGraphExecDestroy(L->graph);
  if (L->cap_stream) cudaStreamDestroy(L->cap_stream);
  void* ps[] = {L->d_raw, L->d_wpack, L->act0, L->act1, L->coef, L->acc, L->wbuf, L->corr, L->ring,
                (void*)L->d_ptrs, L->d_err};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete L;
  c->lrn = nullptr;
}

extern "C" {

int64_t fd_param_count(const fd_ctx* c) { return (c && c->lrn) ? c->lrn->nparams : 0; }

fd_status fd_set_params(fd_ctx* c, const float* params, int64_t count, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_set_params: null context");
  if (!c->lrn) return fd_set_error(c, FD_EINVAL, "fd_set_params: context was created without the learned option");
  if (!params) return fd_set_error(c, FD_EINVAL, "fd_set_params: null parameter array");
  LearnedState& L = *c->lrn;
  if (count != L.nparams)
    return fd_set_error(c, FD_EINVAL, "fd_set_params: expected %lld values, got %lld", (long long)L.nparams,
                        (long long)count);
  // raw offsets
  size_t off = 0;
  L.raw_off_wl = off;
  off += 80;
  for (int l = 0; l < 6; ++l) {
    L.raw_off_sw[l] = off;
    off += (size_t)stencil_cout(l) * stencil_cin(l) * 9;
    L.raw_off_sb[l] = off;
    off += stencil_cout(l);
  }
  if (L.kc > 0)
    for (int l = 0; l < 6; ++l) {
      L.raw_off_tw[l] = off;
      off += (size_t)tc_cout(l) * tc_cin(l, L.kc) * 9;
      L.raw_off_tb[l] = off;
      off += tc_cout(l);
    }
  // network weights rounded to BF16 everywhere (also for the CUDA-core layers)
  std::vector<float> raw(params, params + count);
  auto round_range = [&](size_t o, size_t n) {
    for (size_t k = 0; k < n; ++k) {
      const uint32_t b = (uint32_t)bf16_bits(raw[o + k]) << 16;
      std::memcpy(&raw[o + k], &b, 4);
    }
  };
  for (int l = 0; l < 6; ++l) round_range(L.raw_off_sw[l], (size_t)stencil_cout(l) * stencil_cin(l) * 9);
  if (L.kc > 0)
    for (int l = 0; l < 6; ++l) round_range(L.raw_off_tw[l], (size_t)tc_cout(l) * tc_cin(l, L.kc) * 9);
  // tensor-core tiles
  std::vector<uint16_t> pk;
  auto add = [&](size_t elems) {
    const size_t o = pk.size();
    pk.resize(o + elems);
    return o;
  };
  {
    const size_t o = add(part_elems(16, 64));
    pack_part(&raw[L.raw_off_sw[0]], 2, 64, 0, 64, &pk[o], 16);
    L.pk_stencil_first = o;
  }
  for (int l = 1; l <= 4; ++l) {
    const size_t o = add(part_elems(64, 64));
    pack_part(&raw[L.raw_off_sw[l]], 64, 64, 0, 64, &pk[o]);
    L.pk_stencil[l - 1] = o;
  }
  {
    const size_t o = add(2 * part_elems(64, 64));
    pack_part(&raw[L.raw_off_sw[5]], 64, kCoef, 0, 64, &pk[o]);
    pack_part(&raw[L.raw_off_sw[5]], 64, kCoef, 64, 64, &pk[o + part_elems(64, 64)]);
    L.pk_stencil[4] = o;
    const size_t o2 = add(part_elems(64, 32));
    pack_part(&raw[L.raw_off_sw[5]], 64, kCoef, 128, 32, &pk[o2]);
    L.pk_stencil_last32 = o2;
  }
  // reverse-mode (data-gradient) tiles: transposed, flipped kernels
  for (int l = 1; l <= 4; ++l) {
    const size_t o = add(part_elems(64, 64));
    pack_part_transposed(&raw[L.raw_off_sw[l]], 64, 64, 0, 64, &pk[o]);
    L.pk_t[l - 1] = o;
  }
  {
    const size_t o = add(2 * part_elems(kCoef, 32));
    pack_part_transposed(&raw[L.raw_off_sw[5]], 64, kCoef, 0, 32, &pk[o]);
    pack_part_transposed(&raw[L.raw_off_sw[5]], 64, kCoef, 32, 32, &pk[o + part_elems(kCoef, 32)]);
    L.pk_t5 = o;
  }
  if (L.kc > 0) {
    const size_t o = add(part_elems(16, 64));
    pack_part(&raw[L.raw_off_tw[0]], 2 * L.kc, 64, 0, 64, &pk[o], 16);
    L.pk_tc_first = o;
    for (int l = 1; l <= 4; ++l) {
      const size_t o2 = add(part_elems(64, 64));
      pack_part(&raw[L.raw_off_tw[l]], 64, 64, 0, 64, &pk[o2]);
      L.pk_tc[l - 1] = o2;
    }
  }
  // after the parameters: the first layer's transposed, flipped kernel in FP32
  // ([2][64][3][3], for its data gradient on CUDA cores) and a few zeros
  L.raw_off_w0t = raw.size();
  raw.resize(raw.size() + 2 * 64 * 9 + 8, 0.0f);
  L.raw_off_zero = L.raw_off_w0t + 2 * 64 * 9;
  for (int ci = 0; ci < 2; ++ci)
    for (int o = 0; o < 64; ++o)
      for (int a = 0; a < 3; ++a)
        for (int e2 = 0; e2 < 3; ++e2)
          raw[L.raw_off_w0t + ((ci * 64 + o) * 3 + a) * 3 + e2] =
              raw[L.raw_off_sw[0] + ((o * 2 + ci) * 3 + (2 - a)) * 3 + (2 - e2)];
  cudaError_t e = cudaSuccess;
  if (!L.d_raw) e = cudaMalloc(&L.d_raw, raw.size() * sizeof(float));
  if (e == cudaSuccess && !L.d_wpack) e = cudaMalloc(&L.d_wpack, pk.size() * sizeof(uint16_t));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.d_raw, raw.data(), raw.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L.d_wpack, pk.data(), pk.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_set_params: %s", cudaGetErrorString(e));
  L.ready = true;
  return FD_OK;
}

fd_status fd_network_forward(fd_ctx* c, const void* u, float* coef_out, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_network_forward: null context");
  if (!c->lrn || !c->lrn->ready) return fd_set_error(c, FD_EINVAL, "fd_network_forward: parameters not set");
  if (!u || !coef_out) return fd_set_error(c, FD_EINVAL, "fd_network_forward: null pointer");
  LearnedState& L = *c->lrn;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = fd_state_bytes(c->grid);
  // the first layer reads its input through a pointer array: stage through wbuf
  cudaError_t e = cudaMemcpyAsync(L.wbuf, u, bytes, cudaMemcpyDeviceToDevice, st);
  const float* const* pw = L.d_ptrs + L.nring;
  if (e == cudaSuccess) e = (c->grid.nx == 64) ? run_stencil_net<6>(c, pw, st) : run_stencil_net<5>(c, pw, st);
  if (e == cudaSuccess) {
    coef_unpack_kernel<<<4 * L.sms, 256, 0, st>>>(L.coef, coef_out, c->grid.batch, c->logn);
    e = cudaGetLastError();
  }
  c->launches = 8;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_network_forward: %s", cudaGetErrorString(e));
  return FD_OK;
}

}  // extern "C"

// learned rollout: ring slot r holds the state after step (base + r) of the
// current group; a group of G = max(k_c, 1) steps is captured once as a CUDA
// graph (with the temporal correction at its last step) and replayed.
fd_status fd_learned_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                             cudaStream_t st) {
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
  cudaError_t e = cudaMemcpyAsync(L.ring, u0, bytes, cudaMemcpyDeviceToDevice, st);
  const bool use_graph = save_every == 0;
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
      launches += G * (4 * 7);
    }
  }
  // remaining steps (or every step when snapshots are requested): direct launches
  for (; done < n_steps && e == cudaSuccess; ++done) {
    const int r = done % G;
    const bool tc = L.kc > 0 && ((done + 1) % L.kc == 0);
    e = step_fn(r, tc, st);
    launches += 4 * 7 + (tc ? 7 : 0);
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
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout (learned): %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_learned_error_flag(fd_ctx* c) {
  if (!c->lrn) return FD_OK;
  unsigned h = 0;
  if (cudaMemcpy(&h, c->lrn->d_err, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fd_set_error(c, FD_ECUDA, "error flag read failed");
  if (h) return fd_set_error(c, FD_ETIMEOUT, "a bounded device wait of the tensor-core convolution gave up (0x%x)", h);
  return FD_OK;
}
