// fd_ctx.h -- the library-private context shared by the C ABI translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/fd.h"
#include "fv_fused.cuh"

namespace ldfv {

struct Launcher {
  int cs = 0, nt = 0;
  size_t smem = 0;
  cudaError_t (*launch)(const FvArgs&, int batch, size_t smem, cudaStream_t) = nullptr;
  cudaError_t (*prepare)(size_t smem) = nullptr;
};

// Device buffers and launch state of the learnable module.
struct LearnedState {
  bool ready = false;          // parameters uploaded
  int kc = 0;
  int64_t nparams = 0;
  float* d_raw = nullptr;      // the float32 parameter array as uploaded
  __nv_bfloat16* d_wpack = nullptr;  // tensor-core weight tiles
  size_t raw_off_wl = 0;
  size_t raw_off_sw[6] = {}, raw_off_sb[6] = {};  // stencil layer weights / biases
  size_t raw_off_tw[6] = {}, raw_off_tb[6] = {};  // temporal-correction layers
  size_t pk_stencil[5] = {};   // packed tiles: hidden layers 1..4, last layer (64-wide parts)
  size_t pk_stencil_last32 = 0;
  size_t pk_stencil_first = 0; // first layer, input channels padded to 16
  size_t pk_tc[4] = {};
  size_t pk_tc_first = 0;
  __nv_bfloat16* act0 = nullptr;
  __nv_bfloat16* act1 = nullptr;
  __nv_bfloat16* coef = nullptr;
  float* acc = nullptr;
  float* wbuf = nullptr;
  float* corr = nullptr;
  float* ring = nullptr;       // kc + 1 (or 2) states
  int nring = 0;
  const float** d_ptrs = nullptr;  // device pointer arrays for the first-layer inputs
  unsigned* d_err = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  int sms = 0;
};

}  // namespace ldfv

struct fd_ctx {
  fd_grid grid;
  fd_forcing forcing;
  fd_options opts;
  double nu = 0, dt = 0;
  int logn = 0;
  ldfv::Launcher L;
  bool prepared = false;
  void* d_tables = nullptr;  // tw | symx | symy | frc
  size_t off_symx = 0, off_symy = 0, off_frc = 0;
  void* d_state = nullptr;   // device state for fd_rollout_host
  unsigned* d_flag = nullptr;
  int launches = 0;
  std::string err;
  ldfv::FvArgs base;
  ldfv::LearnedState* lrn = nullptr;
};

// shared helpers of the ABI translation units
fd_status fd_set_error(fd_ctx* c, fd_status s, const char* fmt, ...);
size_t fd_state_bytes(const fd_grid& g);
