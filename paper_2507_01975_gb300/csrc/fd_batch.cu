// fd_batch.cu -- many rollouts of different contexts (grid sizes, flow types,
// learned and plain) as one CUDA graph, replayed with a single graph launch.
// The trajectories of the plain single-precision contexts with N <= 64 run in
// one persistent launch (fd_mixed.cu: a work list that the launch's CTAs take
// trajectories from); every other context is a parallel branch of its own,
// forked from and joined back into one capture stream. Branches run
// concurrently wherever the GPU has room.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"

fd_status fd_rollout_impl(fd_ctx* c, const void* u0, void* traj, void* u_final, int32_t n_steps, int32_t save_every,
                          void* stream, bool allow_graph);

struct fd_batch {
  struct Entry {
    fd_ctx* ctx;
    const void* u0;
    void* u_final;
    int n_steps;
    cudaStream_t stream;
    cudaEvent_t done;
    unsigned long long epoch;  // ctx->epoch when the graph was captured
  };
  std::vector<Entry> entries;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int launches = 0;
  std::string err;
  // persistent launch of the eligible trajectories (one per derivative order)
  bool persistent = true;
  cudaStream_t mixed_stream[2] = {nullptr, nullptr};
  cudaEvent_t mixed_done[2] = {nullptr, nullptr};
  ldfv::MixedItem* d_items = nullptr;
  unsigned* d_counter = nullptr;  // [2]
  int n_persistent = 0;           // trajectories in the persistent launches of the graph
};

namespace {

fd_status batch_error(fd_batch* b, fd_status s, const std::string& msg) {
  b->err = msg;
  return s;
}

void drop_graph(fd_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

void free_items(fd_batch* b) {
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counter) cudaFree(b->d_counter);
  b->d_items = nullptr;
  b->d_counter = nullptr;
}

}  // namespace

extern "C" {

fd_status fd_batch_create(fd_batch** out) {
  if (!out) return fd_set_error(nullptr, FD_EINVAL, "fd_batch_create: null out pointer");
  *out = nullptr;
  fd_batch* b = new (std::nothrow) fd_batch();
  if (!b) return fd_set_error(nullptr, FD_ENOMEM, "fd_batch_create: out of host memory");
  if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return fd_set_error(nullptr, FD_ECUDA, "fd_batch_create: stream or event creation failed");
  }
  *out = b;
  return FD_OK;
}

fd_status fd_batch_add(fd_batch* b, fd_ctx* ctx, const void* u0, void* u_final, int32_t n_steps) {
  if (!b) return fd_set_error(nullptr, FD_EINVAL, "fd_batch_add: null batch");
  if (!ctx || !u0 || !u_final) return batch_error(b, FD_EINVAL, "fd_batch_add: null context or state pointer");
  if (n_steps < 1) return batch_error(b, FD_EINVAL, "fd_batch_add: n_steps must be >= 1");
  for (const auto& e : b->entries)
    if (e.ctx == ctx) return batch_error(b, FD_EINVAL, "fd_batch_add: a context may appear once per batch");
  fd_batch::Entry e{ctx, u0, u_final, n_steps, nullptr, nullptr, 0};
  if (cudaStreamCreateWithFlags(&e.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming) != cudaSuccess)
    return batch_error(b, FD_ECUDA, "fd_batch_add: stream or event creation failed");
  b->entries.push_back(e);
  drop_graph(b);
  return FD_OK;
}

fd_status fd_batch_run(fd_batch* b, void* stream) {
  if (!b) return fd_set_error(nullptr, FD_EINVAL, "fd_batch_run: null batch");
  if (b->entries.empty()) return batch_error(b, FD_EINVAL, "fd_batch_run: empty batch");
  // a member whose launch plan changed since the capture (fd_set_plan,
  // fd_autotune) may have replaced the buffers and launch shapes the graph
  // holds: capture again
  for (const auto& en : b->entries)
    if (b->graph && en.ctx->epoch != en.epoch) drop_graph(b);
  if (!b->graph) {
    // the persistent launches' work lists (derivative order 2 and 4), uploaded
    // before the capture; the graph resets their counters
    std::vector<ldfv::MixedItem> items[2];
    std::vector<bool> in_list(b->entries.size(), false);
    for (size_t k = 0; k < b->entries.size() && b->persistent; ++k) {
      const auto& en = b->entries[k];
      if (!fd_mixed_eligible(en.ctx)) continue;
      fd_mixed_items(en.ctx, en.u0, en.u_final, en.n_steps, items[en.ctx->opts.deriv_order == 2 ? 0 : 1]);
      in_list[k] = true;
    }
    free_items(b);
    const size_t n0 = items[0].size(), n1 = items[1].size();
    cudaError_t e = cudaSuccess;
    if (n0 + n1 > 0) {
      fd_mixed_order(items[0]);
      fd_mixed_order(items[1]);
      e = cudaMalloc(&b->d_items, (n0 + n1) * sizeof(ldfv::MixedItem));
      if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 2 * sizeof(unsigned));
      if (e == cudaSuccess && n0)
        e = cudaMemcpy(b->d_items, items[0].data(), n0 * sizeof(ldfv::MixedItem), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && n1)
        e = cudaMemcpy(b->d_items + n0, items[1].data(), n1 * sizeof(ldfv::MixedItem), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && n0) e = fd_mixed_prepare(2);
      if (e == cudaSuccess && n1) e = fd_mixed_prepare(4);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (!b->mixed_stream[k]) e = cudaStreamCreateWithFlags(&b->mixed_stream[k], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b->mixed_done[k])
          e = cudaEventCreateWithFlags(&b->mixed_done[k], cudaEventDisableTiming);
      }
      if (e != cudaSuccess) {
        free_items(b);
        return batch_error(b, FD_ECUDA, std::string("fd_batch_run: work list: ") + cudaGetErrorString(e));
      }
    }
    cudaGraph_t g = nullptr;
    int launches = 0;
    e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_error(b, FD_ECUDA, std::string("fd_batch_run: capture: ") + cudaGetErrorString(e));
    fd_status st = FD_OK;
    std::string why;
    e = cudaEventRecord(b->fork, b->origin);
    const size_t ncount[2] = {n0, n1};
    const ldfv::MixedItem* list[2] = {b->d_items, b->d_items ? b->d_items + n0 : nullptr};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      if (ncount[k] == 0) continue;
      e = cudaStreamWaitEvent(b->mixed_stream[k], b->fork, 0);
      if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter + k, 0, sizeof(unsigned), b->mixed_stream[k]);
      if (e == cudaSuccess)
        e = fd_mixed_launch(list[k], (int)ncount[k], b->d_counter + k, k == 0 ? 2 : 4, b->mixed_stream[k]);
      if (e == cudaSuccess) e = cudaEventRecord(b->mixed_done[k], b->mixed_stream[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->mixed_done[k], 0);
      ++launches;
    }
    for (size_t k = 0; k < b->entries.size(); ++k) {
      auto& en = b->entries[k];
      en.epoch = en.ctx->epoch;
      if (in_list[k]) continue;
      if (e != cudaSuccess || st != FD_OK) break;
      e = cudaStreamWaitEvent(en.stream, b->fork, 0);
      if (e != cudaSuccess) break;
      st = fd_rollout_impl(en.ctx, en.u0, nullptr, en.u_final, en.n_steps, 0, en.stream, false);
      if (st != FD_OK) {
        why = fd_last_error(en.ctx);
        break;
      }
      launches += fd_last_launch_count(en.ctx);
      e = cudaEventRecord(en.done, en.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, en.done, 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
    if (st != FD_OK) {
      if (g) cudaGraphDestroy(g);
      return batch_error(b, st, "fd_batch_run: " + why);
    }
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_error(b, FD_ECUDA, std::string("fd_batch_run: ") + cudaGetErrorString(e));
    b->launches = launches;
    b->n_persistent = (int)(n0 + n1);
  }
  cudaError_t e = cudaGraphLaunch(b->graph, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return batch_error(b, FD_ECUDA, std::string("fd_batch_run: ") + cudaGetErrorString(e));
  return FD_OK;
}

int32_t fd_batch_launch_count(const fd_batch* b) { return b ? b->launches : 0; }

fd_status fd_batch_set_persistent(fd_batch* b, int32_t enable) {
  if (!b) return fd_set_error(nullptr, FD_EINVAL, "fd_batch_set_persistent: null batch");
  if (b->persistent != (enable != 0)) drop_graph(b);
  b->persistent = enable != 0;
  return FD_OK;
}

int32_t fd_batch_persistent_count(const fd_batch* b) { return b ? b->n_persistent : 0; }

const char* fd_batch_last_error(const fd_batch* b) { return b ? b->err.c_str() : ""; }

fd_status fd_batch_destroy(fd_batch* b) {
  if (!b) return FD_OK;
  cudaDeviceSynchronize();
  drop_graph(b);
  for (auto& e : b->entries) {
    if (e.stream) cudaStreamDestroy(e.stream);
    if (e.done) cudaEventDestroy(e.done);
  }
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int k = 0; k < 2; ++k) {
    if (b->mixed_stream[k]) cudaStreamDestroy(b->mixed_stream[k]);
    if (b->mixed_done[k]) cudaEventDestroy(b->mixed_done[k]);
  }
  free_items(b);
  delete b;
  return FD_OK;
}

}  // extern "C"
