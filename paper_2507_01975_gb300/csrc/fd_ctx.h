// fd_ctx.h -- the library-private context shared by the C ABI translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fd.h"
#include "fv_fused.cuh"

namespace ldfv {

struct Launcher {
  int cs = 0, nt = 0;
  size_t smem = 0;
  cudaError_t (*launch)(const FvArgs&, int batch, size_t smem, cudaStream_t) = nullptr;
  cudaError_t (*prepare)(size_t smem) = nullptr;
  // trajectories resident at once (after prepare)
  cudaError_t (*occupancy)(size_t smem, int* trajectories) = nullptr;
};

// Device buffers and launch state of the learnable module.
// activations of one Fourier-operator evaluation kept for its reverse mode
struct FnoSavedBufs {
  float* v = nullptr;    // v_0 .. v_L: [L + 1][batch][width][N][N]
  float* a = nullptr;    // pre-activations of layers 0 .. L - 2
  float2* S = nullptr;   // kept input spectra of every layer [L][batch][width][2M][M]
  float* out = nullptr;  // the operator's output [batch][cout][N][N]
};

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
  size_t pk_tc_t[4] = {};      // data-gradient tiles of the correction network's hidden layers 1..4
  size_t pk_tc_t5 = 0;         // data-gradient tile of its last layer: 2 (padded to 16) -> 64
  size_t raw_off_tw0t = 0;     // FP32 [2 k_c][64][3][3] transposed, flipped first layer of the correction
  size_t pk_t[4] = {};         // data-gradient tiles of hidden layers 1..4 (transposed, flipped)
  size_t pk_t5 = 0;            // data-gradient tiles of the last layer: 160 -> 64 in two parts of 32
  size_t raw_off_w0t = 0;      // FP32 [2][64][3][3] transposed, flipped first layer
  size_t raw_off_zero = 0;     // eight zeros
  size_t raw_total = 0;        // raw array length (parameters, w0t, zeros)
  size_t pk_total = 0;         // packed tile elements
  float* d_stage = nullptr;    // host-uploaded parameters before rounding / packing
  void* d_desc = nullptr;      // tile recipe (one descriptor per tile)
  uint32_t* d_ranges = nullptr;  // (offset, length) of every network weight array in the raw layout
  int ndesc = 0, nranges = 0;
  __nv_bfloat16* act0 = nullptr;
  __nv_bfloat16* act1 = nullptr;
  __nv_bfloat16* coef = nullptr;
  float* acc = nullptr;
  float* wbuf = nullptr;
  float* ws = nullptr;         // unprojected stage result of the banded flux kernel
  float* corr = nullptr;
  float* ring = nullptr;       // kc + 1 (or 2) states
  int nring = 0;
  const float** d_ptrs = nullptr;  // device pointer arrays for the first-layer inputs
  unsigned* d_err = nullptr;
  long long spin = 0;          // iteration limit of the tensor-core kernels' bounded waits
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  int sms = 0;
  // frequency-domain operator O_F (fno_layers > 0)
  int fno_layers = 0, fno_modes = 0, fno_width = 0;
  size_t raw_off_fno = 0;      // P_w, P_b, layers (R, W, b), Q_w, Q_b in the raw array
  float* fno_v[2] = {};        // channel fields [batch][width][N][N] (ping-pong)
  float* fno_y = nullptr;      // inverse spectral convolution [batch][width][N][N]
  float2* fno_s = nullptr;     // kept modes [batch][width][2M][M]
  float2* fno_s2 = nullptr;    // mixed modes
  float* fno_out = nullptr;    // O_F(u) [batch][8][N][N]
  // temporal correction as a Fourier neural operator (tcf_layers > 0, k_c > 0):
  // 2 k_c -> 2 channels into corr; shares the O_F scratch above
  int tcf_layers = 0, tcf_modes = 0, tcf_width = 0;
  int ablation = 0;  // 0 full flux block, 1 without the physics conv, 2 frequency operator only
  size_t raw_off_tcf = 0;
  // channel matrices of both operators in the mixing kernel's mode-blocked layout
  // (rebuilt from the raw parameters on every upload)
  float2* fno_rp = nullptr;
  float2* tcf_rp = nullptr;
  float2* fno_rph = nullptr;   // conjugate-transposed channel matrices (the reverse mode's mixing)
  float2* tcf_rph = nullptr;
};

// Workspace of the reverse mode of one step (allocated by the first
// fd_step_adjoint call): stage states, cotangents, and for the learned path
// every network activation of the four stages plus weight-gradient partials.
struct AdjointState {
  float* wst[3] = {};          // stage states w2, w3, w4
  float* acc = nullptr;        // RK accumulator of the recomputed forward stages
  float* g = nullptr;          // P(lam_out)
  float* rb = nullptr;         // tendency cotangent of the current stage
  float* wbar = nullptr;       // state cotangent through the FV part
  float* xbar = nullptr;       // state cotangent through the network input
  float* zeros = nullptr;      // 80 zeros (W_L of a plain context)
  __nv_bfloat16* h[4][6] = {}; // layer inputs per stage (h[s][0]: packed state, 16 channels)
  __nv_bfloat16* z[4][5] = {}; // pre-activations of layers 0..4 per stage
  __nv_bfloat16* coef[4] = {}; // network outputs per stage
  __nv_bfloat16* cbar = nullptr;   // network-output cotangent (160 channels)
  __nv_bfloat16* zbar[2] = {};     // hidden-layer cotangents (64 channels, ping-pong)
  float* partial = nullptr;        // weight-gradient partial sums
  float* partial_b = nullptr;
  // temporal correction (CNN head): packed 2-channel cotangent of its output and
  // a device array of k_c history-state pointers
  __nv_bfloat16* tc_cbar = nullptr;
  const float** d_hist = nullptr;
  // Fourier operators: O_F's activations per stage, the FNO correction's, the
  // face-value cotangents (O_F's output cotangent), the correction's output
  // cotangent in FP32, and the partial sums of their weight gradients
  FnoSavedBufs fsv[4];
  FnoSavedBufs tcs;
  float* fnobar = nullptr;
  float* tc_cbar_f32 = nullptr;
  float* fno_partial = nullptr;
  int sms = 0;                     // SM count of the device (plain contexts have no learned state)
  bool ready = false;
};

// Buffers of the streaming (HBM) path for large grids.
struct LargeState {
  float* un = nullptr;         // state
  float* acc = nullptr;        // RK accumulator
  float* wsA = nullptr;        // stage results w* (ping-pong: a stage reads the previous one with halos)
  float* wsB = nullptr;
  float* p = nullptr;          // pressure of the latest projection
  void* spec = nullptr;        // [batch][N/8][N/2 + 1][8] complex half spectra (8-row groups)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;  // one step
  size_t snap_stride = 0;      // bytes between snapshots in traj (0: one state)
};

// Workspace of the rollout reverse mode and the training step: checkpoints
// every k steps, the recomputed states of one segment, the running state
// cotangent and the partial sums of the loss reduction.
struct TrainState {
  float* ckpt = nullptr;
  float* seg = nullptr;
  float* lam = nullptr;
  double* partial = nullptr;
  double* corr = nullptr;      // partial sums of fd_vorticity_pcc
  float* pend = nullptr;       // k_c history cotangents of the temporal correction
  size_t ncorr = 0;
  int nckpt = 0, nseg = 0;
  // the passive scalar's checkpoints, segment and cotangent (joint training)
  float* ckpt_s = nullptr;
  float* seg_s = nullptr;
  float* lam_s = nullptr;
  int nckpt_s = 0, nseg_s = 0;
};

}  // namespace ldfv

namespace ldfv {
// generic-grid path (fd_generic.cu): state, two stage buffers, accumulator,
// the forcing table of the ny u-face rows, the projection workspace, and the
// captured step
struct GenericState {
  void* un = nullptr;
  void* wa = nullptr;
  void* wb = nullptr;
  void* acc = nullptr;
  void* frc = nullptr;
  // Navier-Stokes only: complex spectrum [batch][ny][nx], pressure, twiddles and
  // Poisson symbols of both axes
  void* z = nullptr;
  void* p = nullptr;
  void* twx = nullptr;
  void* twy = nullptr;
  void* symx = nullptr;
  void* symy = nullptr;
  // passive scalar (fd_rollout_scalar, allocated by its first call): state,
  // two stage buffers, accumulator [batch][ny][nx]
  void* sn = nullptr;
  void* sa = nullptr;
  void* sb = nullptr;
  void* sacc = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  // one step with the scalar, captured by fd_rollout_scalar for the diffusivity sgraph_diff
  cudaGraphExec_t sgraph = nullptr;
  double sgraph_diff = -1.0;
};

// learned module on the generic-grid path (fd_glearned.cu): FP32 parameters
// (network weights rounded to BF16 at upload), FP32 network activations, the
// per-face coefficients and face values of a stage, the temporal-correction
// history ring
struct GenericLearned {
  int64_t nparams = 0;
  int kc = 0;
  int ablation = 0;
  bool scalar = false;              // the model learns the passive scalar (network on (u, v, s))
  int ncoef = 160;                  // network output channels: 160, 240 with the scalar
  bool ready = false;
  float* d_params = nullptr;        // the parameter array (fd_set_params layout)
  size_t off_wl = 0;                // W_L[2][2][5][4]
  size_t off_wls = 0;               // W_Ls[2][2][5][4] (scalar models)
  size_t off_sw[6] = {}, off_sb[6] = {};  // stencil network layers
  size_t off_tw[6] = {}, off_tb[6] = {};  // temporal-correction network layers
  float* act0 = nullptr;            // [batch][64][ny][nx]
  float* act1 = nullptr;
  float* coef = nullptr;            // [batch][ncoef][ny][nx]
  float* inst = nullptr;            // [batch][8][ny][nx] face values
  float* sinst = nullptr;           // [batch][4][ny][nx] the scalar's face values (scalar models)
  float* corr = nullptr;            // [batch][2][ny][nx] temporal correction
  float* ring = nullptr;            // [kc][batch][2][ny][nx] the last kc states
  const float** d_hist = nullptr;   // [kc] pointers to the ring slots, oldest first
  const float** d_single = nullptr; // [4] the network's input states: u_n, the two stage buffers, a free slot
  const float** d_ssingle = nullptr; // [4] the same for the scalar (scalar models): s_n, its two stage buffers
  cudaGraphExec_t graph = nullptr;  // one group of max(k_c, 1) steps, captured by the first rollout
  double graph_diff = -1.0;         // scalar models: the diffusivity the graph was captured with
  uint64_t version = 0;             // bumped by every parameter upload
};

// reverse mode on the generic-grid path (fd_gadjoint.cu), allocated by its
// first call: the recomputed stage states, the per-face kernels (then the
// network-output cotangent), face values and their cotangents, the RK4
// cotangent bookkeeping, and for learned contexts the saved pre-activations,
// the reverse activations, the transposed weights and the weight-gradient
// partial sums
struct GenAdjoint {
  float* w[4] = {};                 // w[1..3]: stage states [batch][2][ny][nx]
  float* acc = nullptr;             // scratch RK accumulator
  float* kbuf = nullptr;            // [batch][160][ny][nx]
  float* inst = nullptr;            // [batch][8][ny][nx] face values
  float* vbar = nullptr;            // [batch][8][ny][nx] their cotangents
  float* ubar = nullptr;            // [batch][2][ny][nx] stage-state cotangent
  float* g = nullptr;               // P(lam)
  float* y = nullptr;               // P(stage-state cotangent)
  float* rb = nullptr;              // tendency cotangent
  float* lam = nullptr;             // accumulated input cotangent
  float* zsave[5] = {};             // [batch][64][ny][nx] hidden pre-activations
  float* zb[2] = {};                // [batch][64][ny][nx] reverse activations
  float* wt = nullptr;              // transposed, flipped weights of both networks
  size_t off_wt_s[6] = {}, off_wt_t[6] = {};
  uint64_t wt_version = ~0ull;      // parameter version the transposed weights belong to
  float* part = nullptr;            // weight-gradient partial sums
  size_t npart = 0;                 // floats in part
  double* sums = nullptr;           // [240] channel sums
  const float** d_hist = nullptr;   // [8] history pointers of the correction network
  int kbuf_ch = 0;                  // channels of kbuf (160; 240 once the joint reverse mode ran)
  // joint velocity-scalar reverse mode (allocated by its first call): the scalar
  // stage states, face values and their cotangents, the scalar cotangents, the
  // network input's three-channel cotangent, and the stage-state pointer tables
  bool joint = false;
  float* z[4] = {};                 // z[1..3]: scalar stage states [batch][ny][nx]
  float* sacc = nullptr;
  float* sinst = nullptr;           // [batch][4][ny][nx]
  float* svbar = nullptr;           // [batch][4][ny][nx]
  float* zbar = nullptr;            // scalar stage-state cotangent
  float* qb = nullptr;              // scalar tendency cotangent
  float* ys = nullptr;              // the previous stage's scalar cotangent
  float* lams = nullptr;            // accumulated scalar input cotangent
  float* ls0 = nullptr;             // copy of the scalar output cotangent
  float* x3 = nullptr;              // [batch][3][ny][nx] network-input cotangent
  const float** d_wptr = nullptr;   // [4] velocity stage states
  const float** d_zptr = nullptr;   // [4] scalar stage states
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
  void* d_spec = nullptr;    // complex scratch of fd_energy_spectrum
  size_t spec_bytes = 0;
  unsigned* d_flag = nullptr;
  int launches = 0;
  std::string err;
  ldfv::FvArgs base;
  ldfv::LearnedState* lrn = nullptr;
  ldfv::AdjointState* adj = nullptr;
  ldfv::TrainState* trn = nullptr;
  ldfv::LargeState* big = nullptr;   // set when the streaming path runs this context
  ldfv::GenericState* gen = nullptr; // set for the generic-grid path (non-power-of-two / rectangular grids)
  ldfv::GenericLearned* glrn = nullptr;  // learned module of a generic-grid context
  ldfv::GenAdjoint* gadj = nullptr;      // reverse mode of a generic-grid context
  // launch plan of a plain on-chip context: on-chip configurations valid for
  // this grid ([0] = default), the one in use, and how the batch is split
  // between it and a streaming context that runs the trajectories
  // [n_onchip, batch) concurrently on side_stream
  std::vector<ldfv::Launcher> variants;
  std::vector<int> capacity;          // trajectories resident at once, per variant
  int variant = 0;
  int n_onchip = 0, n_stream = 0;
  double plan_us = 0;                 // per-step time measured by fd_autotune
  fd_ctx* side = nullptr;
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // bumped whenever a change would make a captured rollout stale (a new launch
  // plan, which can also replace the streaming sub-context and its buffers);
  // fd_batch recaptures its graph when a member's epoch moved since capture
  unsigned long long epoch = 0;
  // plain-FV fallback of a learned context (fd_rollout_guarded): a plain
  // context of the same grid and three state buffers, both made by the first call
  fd_ctx* fallback = nullptr;
  void* d_guard = nullptr;
};

// Launch with programmatic stream serialisation: the kernel may start while
// the previous kernel of the stream finishes (see pdl_wait / pdl_trigger).
// Translation-unit local, like the kernel stubs it takes.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// shared helpers of the ABI translation units
fd_status fd_set_error(fd_ctx* c, fd_status s, const char* fmt, ...);
size_t fd_state_bytes(const fd_grid& g);

// generic-grid path (fd_generic.cu) and its learned module (fd_glearned.cu)
cudaError_t fd_generic_project(fd_ctx* c, float* w, cudaStream_t st);
int64_t fd_learned_param_count(const fd_options& o);
fd_status fd_glearned_check(const fd_grid& g, const fd_options& o);
fd_status fd_glearned_init(fd_ctx* c);
void fd_glearned_free(fd_ctx* c);
fd_status fd_glearned_set_params(fd_ctx* c, const float* params, int64_t count, bool device, cudaStream_t st);
fd_status fd_glearned_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                              cudaStream_t st, bool allow_graph);
fd_status fd_glearned_network(fd_ctx* c, const void* u, float* coef_out, cudaStream_t st);
// reverse mode on the generic-grid path (fd_gadjoint.cu)
fd_status fd_gadjoint_step(fd_ctx* c, const float* u_in, const float* lam_out, float* lam_in, float* dparams,
                           cudaStream_t st);
fd_status fd_gadjoint_tc(fd_ctx* c, const float* const* hist_host, const float* lam, float* vbar, float* hist_bar,
                         size_t state_stride, float* dparams, cudaStream_t st, int* launches);
// reverse mode of one joint velocity-scalar step (fd_rollout_scalar's step)
fd_status fd_gadjoint_step_scalar(fd_ctx* c, double diff, const float* u_in, const float* s_in, const float* lam_u_out,
                                  const float* lam_s_out, float* lam_u_in, float* lam_s_in, float* dparams,
                                  cudaStream_t st);
void fd_gadjoint_free(fd_ctx* c);
// traj_u / traj_s (optional, both or neither): the states after every step, [n_steps][...]
fd_status fd_glearned_rollout_scalar(fd_ctx* c, double diff, const void* u0, const void* s0, void* u_final,
                                     void* s_final, int n_steps, cudaStream_t st, void* traj_u = nullptr,
                                     void* traj_s = nullptr);
// the joint rollout behind fd_rollout_scalar, optionally keeping every step's states
fd_status fd_rollout_scalar_impl(fd_ctx* c, double diffusivity, const void* u0, const void* s0, void* u_final,
                                 void* s_final, int n_steps, cudaStream_t st, void* traj_u, void* traj_s);

// persistent mixed-batch rollout (fd_mixed.cu)
bool fd_mixed_eligible(const fd_ctx* c);
void fd_mixed_items(const fd_ctx* c, const void* u0, void* u_final, int n_steps, std::vector<ldfv::MixedItem>& out);
void fd_mixed_order(std::vector<ldfv::MixedItem>& items);
cudaError_t fd_mixed_prepare(int dord);
cudaError_t fd_mixed_launch(const ldfv::MixedItem* d_items, int n, unsigned* d_counter, int dord, cudaStream_t st);
