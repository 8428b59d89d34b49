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
#include "fv_glearned.cuh"

using namespace ldfv;

namespace {

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
    GFaceArgs fa = {};
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
    GStageArgs sa = {};
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
  ++G.version;
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
                                     void* s_final, int n_steps, cudaStream_t st, void* traj_u, void* traj_s) {
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
  // the diffusivity is a kernel argument: a graph captured with another one is
  // replaced; a rollout that keeps every step's state runs its launches directly
  const bool use_graph = !traj_u;
  if (e == cudaSuccess && use_graph && n_steps >= grp && (!G.graph || G.graph_diff != diff)) {
    if (G.graph) {
      // an earlier replay may sit on any stream: wait for the device before the
      // graph is destroyed (a rare event: only a new diffusivity recaptures)
      e = cudaDeviceSynchronize();
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
  if (e == cudaSuccess && use_graph && G.graph && G.graph_diff == diff) {
    for (; done + grp <= n_steps && e == cudaSuccess; done += grp) {
      e = cudaGraphLaunch(G.graph, st);
      launches += grp * per_step + per_corr;
    }
  }
  for (int k = done + 1; k <= n_steps && e == cudaSuccess; ++k) {
    e = step(k, st);
    launches += per_step + (G.kc > 0 && k % G.kc == 0 ? per_corr : 0);
    if (e == cudaSuccess && traj_u) {
      e = cudaMemcpyAsync(static_cast<char*>(traj_u) + (size_t)(k - 1) * bytes, S.un, bytes, cudaMemcpyDeviceToDevice,
                          st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char*>(traj_s) + (size_t)(k - 1) * sbytes, S.sn, sbytes,
                            cudaMemcpyDeviceToDevice, st);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u_final, S.un, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s_final, S.sn, sbytes, cudaMemcpyDeviceToDevice, st);
  c->launches = launches;
  if (e != cudaSuccess)
    return fd_set_error(c, FD_ECUDA, "fd_rollout_scalar (generic-grid learned): %s", cudaGetErrorString(e));
  return FD_OK;
}
