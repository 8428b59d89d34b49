// fd_plan.cu -- launch plans of plain contexts and their autotuner.
//
// A plain context on the on-chip path runs a batch as one launch of the
// cluster-resident rollout kernel. Two choices decide how fast that is:
//   * the cluster shape (CTAs per trajectory): more CTAs put more SMs on one
//     trajectory, fewer keep more trajectories resident at once;
//   * what happens to the trajectories that do not fit in one wave of
//     clusters: a second wave on the same kernel, or the streaming kernels
//     (tiled flux kernels + FFT projection through L2/HBM) on the SMs that the
//     resident clusters leave idle, concurrently on a second stream.
// fd_autotune times every candidate plan on a zero state of the context's
// shape and keeps the fastest; fd_set_plan picks one explicitly. Every plan
// computes the same method; plans differ in rounding only (the streaming
// kernels evaluate the same operators in another order).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"

using namespace ldfv;

bool fd_large_supported(int dtype, int n);
fd_status fd_rollout_impl(fd_ctx* c, const void* u0, void* traj, void* u_final, int32_t n_steps, int32_t save_every,
                          void* stream, bool allow_graph);

namespace {

bool stream_ok(const fd_ctx* c) { return fd_large_supported(c->grid.dtype, c->grid.nx); }

// (re)create the streaming context of the split part for nb trajectories
fd_status ensure_side(fd_ctx* c, int nb) {
  if (c->side && (nb == 0 || c->side->grid.batch != nb)) {
    fd_destroy(c->side);
    c->side = nullptr;
  }
  if (nb == 0 || c->side) return FD_OK;
  fd_grid g = c->grid;
  g.batch = nb;
  fd_options o = c->opts;
  o.path = 2;
  o.learned = 0;
  o.k_c = 0;
  fd_ctx* s = nullptr;
  fd_status st = fd_init(&g, c->nu, c->dt, &c->forcing, &o, &s);
  if (st != FD_OK) return fd_set_error(c, st, "launch plan: streaming part: %s", fd_last_error(nullptr));
  c->side = s;
  cudaError_t e = cudaSuccess;
  if (!c->side_stream) e = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !c->ev_fork) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !c->ev_join) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "launch plan: %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status apply_plan(fd_ctx* c, int variant, int n_onchip, int n_stream) {
  fd_status s = ensure_side(c, n_stream);
  if (s != FD_OK) return s;
  c->variant = variant;
  c->n_onchip = n_onchip;
  c->n_stream = n_stream;
  c->plan_us = 0;
  ++c->epoch;
  return FD_OK;
}

int plan_path(const fd_ctx* c) { return c->gen ? 4 : c->lrn ? 3 : c->big ? 2 : 1; }

void describe(const fd_ctx* c, fd_plan* p) {
  p->path = plan_path(c);
  p->cluster = 0;
  p->n_onchip = 0;
  p->n_stream = 0;
  p->resident = 0;
  p->us_per_step = c->plan_us;
  if (c->lrn) {
    p->n_onchip = c->grid.batch;
  } else if (c->big || c->gen) {
    p->n_stream = c->grid.batch;
  } else {
    p->n_onchip = c->n_onchip;
    p->n_stream = c->n_stream;
    if (c->n_onchip > 0) {
      p->cluster = c->variants[c->variant].cs;
      p->resident = c->capacity[c->variant];
    }
  }
}

}  // namespace

// rollout of a plain on-chip context under its launch plan
fd_status fd_plain_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                           cudaStream_t st, bool allow_graph) {
  const int B = c->grid.batch;
  const Launcher& L = c->variants[c->variant];
  FvArgs a = c->base;
  a.u_in = u0;
  a.u_out = u_final;
  a.traj = save_every > 0 ? traj : nullptr;
  a.n_steps = n_steps;
  a.save_every = save_every;
  a.traj_batch = B;
  if (c->n_stream == 0) {
    cudaError_t e = L.launch(a, B, L.smem, st);
    if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout: launch failed: %s", cudaGetErrorString(e));
    c->launches = 1;
    return FD_OK;
  }
  const size_t per = fd_state_bytes(c->grid) / (size_t)B;  // one trajectory
  const size_t off = per * (size_t)c->n_onchip;
  cudaError_t e = cudaEventRecord(c->ev_fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout: fork: %s", cudaGetErrorString(e));
  int launches = 0;
  if (c->n_onchip > 0) {
    e = L.launch(a, c->n_onchip, L.smem, st);
    launches = 1;
  }
  fd_status s = FD_OK;
  if (e == cudaSuccess) {
    c->side->big->snap_stride = (save_every > 0 && traj) ? per * (size_t)B : 0;
    s = fd_rollout_impl(c->side, static_cast<const char*>(u0) + off,
                        (save_every > 0 && traj) ? static_cast<char*>(traj) + off : nullptr,
                        static_cast<char*>(u_final) + off, n_steps, save_every, c->side_stream, allow_graph);
    launches += c->side->launches;
  }
  // join in every case so that a captured stream stays well formed
  cudaError_t ej = cudaEventRecord(c->ev_join, c->side_stream);
  if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, c->ev_join, 0);
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout: launch failed: %s", cudaGetErrorString(e));
  if (s != FD_OK) return fd_set_error(c, s, "fd_rollout (streaming part): %s", fd_last_error(c->side));
  if (ej != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout: join: %s", cudaGetErrorString(ej));
  return FD_OK;
}

extern "C" {

fd_status fd_get_plan(const fd_ctx* c, fd_plan* out) {
  if (!c || !out) return FD_EINVAL;
  describe(c, out);
  return FD_OK;
}

fd_status fd_set_plan(fd_ctx* c, const fd_plan* p) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_set_plan: null context");
  if (!p) return fd_set_error(c, FD_EINVAL, "fd_set_plan: null plan");
  const int B = c->grid.batch;
  if (p->n_onchip < 0 || p->n_stream < 0 || p->n_onchip + p->n_stream != B)
    return fd_set_error(c, FD_EINVAL, "fd_set_plan: n_onchip + n_stream must equal the batch (%d)", B);
  if (c->lrn) return fd_set_error(c, FD_EUNSUPPORTED, "fd_set_plan: a learned context has a fixed launch plan");
  if (c->big || c->gen) {
    if (p->n_stream != B)
      return fd_set_error(c, FD_EUNSUPPORTED, "fd_set_plan: this grid runs through HBM only (streaming or generic-grid path)");
    return FD_OK;
  }
  int variant = c->variant;
  if (p->n_onchip > 0) {
    variant = -1;
    for (size_t v = 0; v < c->variants.size(); ++v)
      if (c->variants[v].cs == p->cluster) variant = (int)v;
    if (variant < 0)
      return fd_set_error(c, FD_EUNSUPPORTED, "fd_set_plan: no on-chip kernel with %d CTAs per trajectory for N=%d",
                          p->cluster, c->grid.nx);
  }
  if (p->n_stream > 0 && !stream_ok(c))
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_set_plan: the streaming path needs FP32 and N in [32, 2048]");
  cudaError_t e = cudaDeviceSynchronize();  // a plan change must not race a running rollout
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_set_plan: %s", cudaGetErrorString(e));
  return apply_plan(c, variant, p->n_onchip, p->n_stream);
}

fd_status fd_autotune(fd_ctx* c, int32_t probe_steps, fd_plan* report, int32_t max_report, int32_t* n_report,
                      void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_autotune: null context");
  if (max_report < 0 || (max_report > 0 && !report))
    return fd_set_error(c, FD_EINVAL, "fd_autotune: report needs max_report entries");
  if (probe_steps <= 0) probe_steps = 32;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = c->grid.batch;

  struct Cand {
    int variant, n_onchip, n_stream;
    double us;
  };
  std::vector<Cand> cands;
  const bool plain_onchip = !c->lrn && !c->big && !c->gen;
  if (plain_onchip) {
    for (size_t v = 0; v < c->variants.size(); ++v) {
      cands.push_back({(int)v, B, 0, 0});
      const int cap = c->capacity[v];
      if (!stream_ok(c) || cap <= 0) continue;
      // on-chip shares: the full waves (remainder streaming), and 3/4, 1/2, 1/4
      // of one wave (the streaming kernels take the SMs the clusters leave free)
      std::vector<int> shares;
      if (B > cap && B % cap != 0) shares.push_back(B - B % cap);
      const int wave = B < cap ? B : cap;
      for (int f = 3; f >= 1; --f) shares.push_back((wave * f + 2) / 4);
      for (int on : shares) {
        if (on <= 0 || on >= B) continue;
        bool dup = false;
        for (const Cand& x : cands) dup |= x.variant == (int)v && x.n_onchip == on;
        if (!dup) cands.push_back({(int)v, on, B - on, 0});
      }
    }
    if (stream_ok(c)) cands.push_back({0, 0, B, 0});
  } else {
    cands.push_back({0, 0, 0, 0});  // the fixed plan of a learned, streaming-only or generic-grid context
  }
  const int old_variant = c->variant, old_on = c->n_onchip, old_st = c->n_stream;

  const size_t bytes = fd_state_bytes(c->grid);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, 2 * bytes);
  if (e != cudaSuccess) return fd_set_error(c, FD_ENOMEM, "fd_autotune: cudaMalloc: %s", cudaGetErrorString(e));
  void* uin = buf;
  void* uout = static_cast<char*>(buf) + bytes;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMemsetAsync(buf, 0, 2 * bytes, st);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  fd_status s = e == cudaSuccess ? FD_OK : fd_set_error(c, FD_ECUDA, "fd_autotune: %s", cudaGetErrorString(e));
  for (Cand& cd : cands) {
    if (s != FD_OK) break;
    if (plain_onchip) {
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        s = fd_set_error(c, FD_ECUDA, "fd_autotune: %s", cudaGetErrorString(e));
        break;
      }
      s = apply_plan(c, cd.variant, cd.n_onchip, cd.n_stream);
      if (s != FD_OK) break;
    }
    float best = 0;
    for (int rep = 0; rep < 4 && s == FD_OK; ++rep) {  // rep 0 warms up (and captures graphs)
      e = cudaEventRecord(t0, st);
      if (e == cudaSuccess) s = fd_rollout_impl(c, uin, nullptr, uout, probe_steps, 0, st, true);
      if (s != FD_OK) break;
      if (e == cudaSuccess) e = cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e != cudaSuccess) s = fd_set_error(c, FD_ECUDA, "fd_autotune: %s", cudaGetErrorString(e));
      if (rep > 0 && (best == 0 || ms < best)) best = ms;
    }
    cd.us = 1e3 * (double)best / probe_steps;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  if (s != FD_OK) {
    if (plain_onchip) apply_plan(c, old_variant, old_on, old_st);
    return s;
  }
  size_t best = 0;
  for (size_t i = 1; i < cands.size(); ++i)
    if (cands[i].us < cands[best].us) best = i;
  if (plain_onchip) {
    s = apply_plan(c, cands[best].variant, cands[best].n_onchip, cands[best].n_stream);
    if (s != FD_OK) return s;
  }
  c->plan_us = cands[best].us;
  // report: every candidate in the order timed
  const int saved_variant = c->variant, saved_on = c->n_onchip, saved_st = c->n_stream;
  const double saved_us = c->plan_us;
  const int nrep = std::min<int>(max_report, (int)cands.size());
  for (int i = 0; i < nrep; ++i) {
    if (plain_onchip) {
      c->variant = cands[i].variant;
      c->n_onchip = cands[i].n_onchip;
      c->n_stream = cands[i].n_stream;
    }
    c->plan_us = cands[i].us;
    describe(c, &report[i]);
  }
  c->variant = saved_variant;
  c->n_onchip = saved_on;
  c->n_stream = saved_st;
  c->plan_us = saved_us;
  if (n_report) *n_report = (int32_t)cands.size();
  return FD_OK;
}

}  // extern "C"
