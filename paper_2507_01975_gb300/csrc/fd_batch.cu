// fd_batch.cu -- many rollouts of different contexts (grid sizes, flow types,
// learned and plain) as one CUDA graph: one parallel branch per context,
// forked from and joined back into one capture stream, replayed with a single
// graph launch. Branches run concurrently wherever the GPU has room.
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
    cudaGraph_t g = nullptr;
    int launches = 0;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_error(b, FD_ECUDA, std::string("fd_batch_run: capture: ") + cudaGetErrorString(e));
    fd_status st = FD_OK;
    std::string why;
    e = cudaEventRecord(b->fork, b->origin);
    for (auto& en : b->entries) {
      if (e != cudaSuccess || st != FD_OK) break;
      e = cudaStreamWaitEvent(en.stream, b->fork, 0);
      if (e != cudaSuccess) break;
      st = fd_rollout_impl(en.ctx, en.u0, nullptr, en.u_final, en.n_steps, 0, en.stream, false);
      if (st != FD_OK) {
        why = fd_last_error(en.ctx);
        break;
      }
      launches += fd_last_launch_count(en.ctx);
      en.epoch = en.ctx->epoch;
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
  }
  cudaError_t e = cudaGraphLaunch(b->graph, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return batch_error(b, FD_ECUDA, std::string("fd_batch_run: ") + cudaGetErrorString(e));
  return FD_OK;
}

int32_t fd_batch_launch_count(const fd_batch* b) { return b ? b->launches : 0; }

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
  delete b;
  return FD_OK;
}

}  // extern "C"
