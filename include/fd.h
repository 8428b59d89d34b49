/*
 * fd.h -- C ABI of the GB300-native LDSolver coarse-grid finite-volume step.
 *
 * The library advances velocity fields on a periodic 2D box with the
 * learnable-differentiable finite-volume method of "Learnable-Differentiable
 * Finite Volume Solver for Accelerated Simulation of Flows" (KDD'25):
 *
 *   du/dt + div F(u, mu) = S(u)                      (Sec. 3.1, Eq. 1)
 *
 * discretised on a staggered (MAC) grid (App. B.1), with face interpolation
 * and derivative operators (Sec. 3.4, App. B.2), an advection/diffusion flux
 * assembly (App. B.2), a spectral pressure projection for the incompressible
 * flows (Sec. 3.6, App. B.3-B.4) and classical RK4 stages (App. B.5).
 *
 * Conventions shared by every call:
 *   - Field pointers passed to fd_step / fd_rollout are DEVICE pointers owned
 *     by the caller. The library owns only the context and its small constant
 *     tables, allocated in fd_init and released in fd_destroy.
 *   - A state is laid out [batch][2][ny][nx], row-major, element type given by
 *     fd_grid.dtype. Channel 0 is u, stored on the west face of cell (i, j) at
 *     (i dx, (j + 1/2) dy); channel 1 is v, on the south face at
 *     ((i + 1/2) dx, j dy). Pressure and divergence live at cell centres.
 *   - Work is ordered on the CUDA stream passed as `stream` (a cudaStream_t;
 *     NULL = the legacy default stream). No call synchronises the device
 *     except fd_rollout_host, fd_check_finite and fd_destroy.
 *   - Errors are returned as fd_status codes; nothing is thrown across the
 *     ABI. fd_last_error(ctx) returns a message for the last failing call on
 *     that context (or for fd_init failures, fd_last_error(NULL)).
 *   - A context may be used from one host thread at a time.
 */
#ifndef LDFV_FD_H
#define LDFV_FD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FD_OK = 0,
  FD_EINVAL = 1,        /* invalid argument (sizes, null pointers, dt <= 0, nu < 0) */
  FD_ENOMEM = 2,        /* device or host allocation failed */
  FD_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  FD_ENONFINITE = 4,    /* fd_check_finite found a NaN or Inf */
  FD_ETIMEOUT = 5,      /* a bounded device wait gave up (reported by fd_check_finite) */
  FD_EUNSUPPORTED = 6   /* valid request that this build does not implement */
} fd_status;

typedef enum { FD_F32 = 0, FD_F64 = 1 } fd_dtype;

/* Flow families of App. C.1. FD_BURGERS: S = 0, F = u^2/2 - nu grad u,
 * advective form, no pressure. FD_NAVIER_STOKES: incompressible momentum
 * equation with a pressure projection after every RK sub-step. */
typedef enum { FD_BURGERS = 0, FD_NAVIER_STOKES = 1 } fd_flow;

/* Grid: nx = ny = N with N a power of two in [8, 2048], box [0, lx] x [0, ly],
 * `batch` independent trajectories. Two plain paths: the on-chip rollout
 * kernel (one thread-block cluster per trajectory holds the state in shared
 * and tensor memory for the whole rollout; FP32 N <= 256, FP64 N <= 128) and
 * the streaming path for larger grids (FP32, N up to 2048: tiled flux kernels
 * and a three-pass FFT projection through HBM, one CUDA graph per step).
 * The generic-grid path (path 3) takes the other grids, state layout
 * [batch][2][ny][nx]: Burgers (no projection, hence no FFT) on any grid,
 * including non-power-of-two and rectangular ones (nx, ny in [4, 8192], FP32
 * or FP64; the paper's Burgers case is [0, 1]^2 at 100^2 and 25^2, App. C.1),
 * and Navier-Stokes on rectangular power-of-two grids (nx, ny in [32, 2048],
 * FP32; the shear-flow grids 128 x 64 ... 2048 x 1024), four stage kernels per
 * step through HBM, each followed for Navier-Stokes by an FFT projection. */
typedef struct {
  int32_t nx, ny;
  double lx, ly;
  int32_t batch;
  int32_t dtype; /* fd_dtype */
  int32_t flow;  /* fd_flow */
} fd_grid;

/* Source term S (App. C.1, forced flow): kind 0 = none, kind 1 = Kolmogorov
 * forcing f = [amp sin(k y) - drag u, -drag v] evaluated at the faces. */
typedef struct {
  int32_t kind;
  double amp;   /* 1.0 in the paper */
  int32_t k;    /* 4 in the paper */
  double drag;  /* 0.1 in the paper */
} fd_forcing;

/* Options (NULL = defaults shown). */
typedef struct {
  int32_t deriv_order;    /* 4 (paper's physics kernel, default) or 2 */
  int32_t interp_order;   /* 2 (linear interpolation); the only value accepted */
  int32_t learned;        /* 0 = physics kernels only (default), 1 = learnable module */
  int32_t k_c;            /* temporal-correction interval, 0 = off (default) */
  int32_t poisson_symbol; /* 0 = discrete D2 G2 symbol (default, exact projection) */
  int32_t ckpt_every;     /* reserved for the adjoint: checkpoint interval */
  int64_t spin_limit;     /* iteration limit of each bounded mbarrier wait in the
                             tensor-core kernels of the learned path (<= 0: the
                             default, 2^20 tries); a wait that runs out sets the
                             context's error word (fd_check_finite then returns
                             FD_ETIMEOUT), and the kernel drains its own copies and
                             MMAs in flight with a fixed limit, frees its tensor
                             memory and returns. The outputs of that call are then
                             undefined; the context stays usable */
  int32_t path;           /* 0 = automatic (default): on chip where built (FP32 N <= 256,
                             FP64 N <= 128), streaming through HBM otherwise, and the
                             generic-grid kernels for Burgers on a non-power-of-two or
                             rectangular grid and Navier-Stokes on a rectangular power-of-two
                             grid; 1 = on chip only; 2 = streaming (FP32, N in [32, 2048]);
                             3 = generic grid (Burgers on any nx x ny in [4, 8192]^2, FP32 or
                             FP64; Navier-Stokes on power-of-two nx, ny in [32, 2048], FP32;
                             learned contexts FP32, without the Fourier operators) */
  int32_t fno_layers;     /* frequency-domain operator O_F of the learnable module (Sec. 3.4):
                             Fourier layers, 0 = off (default); needs learned = 1; built on the
                             32^2 / 64^2 tensor-core path, forward and reverse mode */
  int32_t fno_modes;      /* kept Fourier modes M per axis, 1 <= M <= N/2 (Table S3: 16 or 32) */
  int32_t fno_width;      /* channels of the Fourier layers: 8 or 16 (the widths of Table S3) */
  int32_t tc_fno_layers;  /* temporal correction as a Fourier neural operator (Sec. 3.5; Table S3:
                             4 layers, 32 modes, width 8) instead of the CNN head: Fourier layers,
                             0 = CNN head (default); needs k_c > 0 */
  int32_t tc_fno_modes;   /* its kept modes per axis, 1 <= M <= N/2 */
  int32_t tc_fno_width;   /* its channels: 8 or 16 */
  int32_t ablation;       /* flux-block variant of the ablation study (Sec. 4, Table 4): 0 = the full
                             operator (default); 1 = without the physics-based convolution: per-face
                             kernels W_L + C_theta (derivative parts / h), no W_P and no consistency
                             projection; 2 = the frequency-domain operator only: face values O_F(u)
                             (needs fno_layers > 0; the stencil network does not run). Needs
                             learned = 1; forward and reverse mode on the tensor-core path,
                             variant 1 forward on the generic-grid path */
  int32_t scalar_learned; /* 1 = the learnable module also learns the passive scalar's transport
                             (shear flow, App. C.1): the scalar's four operator instances take
                             per-face kernels W_P + proj(W_Ls + C_s) / h^deriv like the
                             velocity's eight, the stencil network reads (u, v, s) and emits 240
                             channels (the last 80 are C_s); the temporal correction stays on
                             the velocity. Needs learned = 1 and ablation = 0; runs on the
                             generic-grid path (FP32) and only through fd_rollout_scalar
                             (fd_rollout / fd_step refuse such a context). 0 = off (default) */
} fd_options;

typedef struct fd_ctx fd_ctx; /* opaque, library-owned */

/* Create a solver context for `grid`, viscosity nu (1/Re for Navier-Stokes),
 * time step dt, forcing (NULL = none) and options (NULL = defaults).
 * Allocates the context and its device tables; *out is set on FD_OK only.
 * Errors: FD_EINVAL for bad sizes / dt <= 0 / nu < 0 / null out,
 * FD_EUNSUPPORTED for a valid grid this build has no kernel for,
 * FD_ENOMEM / FD_ECUDA when device set-up fails. */
fd_status fd_init(const fd_grid* grid, double nu, double dt, const fd_forcing* forcing,
                  const fd_options* opts, fd_ctx** out);

/* One time step u_{k+1} = FV(u_k) (Sec. 3.2, Eq. for u_k; App. B.5):
 * four RK4 stages, each evaluating the flux block on the stage state and,
 * for Navier-Stokes, projecting the stage result. u_in and u_out are device
 * pointers to [batch][2][ny][nx] states; they may alias. */
fd_status fd_step(fd_ctx* ctx, const void* u_in, void* u_out, void* stream);

/* n_steps time steps from u0 (device), result in u_final (device; may alias
 * u0). When save_every > 0 and traj != NULL, the state after steps
 * save_every, 2 save_every, ... is written to traj[s][batch][2][ny][nx]
 * (n_steps / save_every snapshots). On the on-chip path the whole rollout is
 * one kernel launch with the state resident on chip; on the streaming path a
 * step is 17 launches replayed as a CUDA graph (direct launches when
 * snapshots are taken). A context built with scalar_learned = 1 advances
 * only through fd_rollout_scalar: fd_rollout and fd_step return
 * FD_EUNSUPPORTED for it (its network reads the scalar). */
fd_status fd_rollout(fd_ctx* ctx, const void* u0, void* traj, void* u_final, int32_t n_steps,
                     int32_t save_every, void* stream);

/* Same as fd_rollout with HOST buffers: copies u0_host to a context-owned
 * device buffer, runs the rollout on `stream`, copies the result back to
 * u_final_host and synchronises the stream. Pinned host memory gives the
 * fastest copies. */
fd_status fd_rollout_host(fd_ctx* ctx, const void* u0_host, void* u_final_host, int32_t n_steps,
                          void* stream);

/* Learned rollout with the plain FV step as its fallback. The paper's learned
 * module only adds learnable parts to the FV module; without them the step is
 * the traditional solver (Sec. 3.4, O = O_P; the DNS solver of the Sec. 4
 * ablation). The paper itself has no fallback mechanism; this call is the
 * serving safeguard built on that relation. The batch advances in chunks of
 * `chunk` time steps (<= 0: k_c, or 8 without a temporal correction; with
 * k_c > 0 it must be a multiple of k_c, so the corrections fall on the same
 * steps as in fd_rollout): each chunk runs the learned rollout and the plain
 * rollout from the same chunk-start state, and a trajectory whose learned
 * chunk produced a NaN or Inf takes the plain result and stays on the plain
 * solver for the rest of the call. Trajectories that never fell back are
 * bit-identical to fd_rollout's. A trajectory whose chunk-start state is
 * already non-finite cannot be rescued: it falls back and stays non-finite.
 * ctx: a learned context (FD_EUNSUPPORTED otherwise). u0 / u_final: device
 * states [batch][2][n][n] FP32 (may alias). fell_back: device int32[batch],
 * written: -1 for a trajectory that stayed learned, else the time step
 * (0-based, a multiple of chunk) at which its fallback chunk started. The
 * first call makes a plain context of the same grid and three state buffers
 * (library-owned, freed by fd_destroy). No host synchronisation.
 * FD_EINVAL for null pointers, n_steps < 0 or a chunk that is not a multiple
 * of k_c. */
fd_status fd_rollout_guarded(fd_ctx* ctx, const void* u0, void* u_final, int32_t n_steps, int32_t chunk,
                             int32_t* fell_back, void* stream);

/* Rollout of the velocity together with a passive scalar s (shear flow,
 * App. C.1: s_t - D lap s = -u . grad s), on a context of the generic-grid
 * path (path 3; e.g. the shear flow's 128 x 64 grid on [0, 8] x [0, 4]).
 * s lives at the cell centres, layout [batch][ny][nx] in the grid's dtype,
 * and is advanced in flux form, -div(u s_f - D grad_f s), with its face values
 * and face derivatives from the physics kernels (four more operator
 * instances) and RK4 stages taken from the same (projected) stage velocities;
 * it is not projected and does not act on the velocity. u0 / s0 are read,
 * u_final / s_final written (they may alias u0 / s0). The first call
 * allocates the scalar's device buffers. On a learned context built with
 * scalar_learned = 1 every RK stage runs the stencil network on (u, v, s):
 * the velocity's eight instances and the scalar's four take their learned
 * per-face kernels, and every k_c steps the temporal correction acts on the
 * velocity (after the first call with a given diffusivity the k_c-step group
 * is replayed as a CUDA graph). FD_EUNSUPPORTED on other paths and on a
 * learned context without scalar_learned; FD_EINVAL for null pointers,
 * n_steps < 0, a negative or non-finite diffusivity, or parameters not set. */
fd_status fd_rollout_scalar(fd_ctx* ctx, double diffusivity, const void* u0, const void* s0, void* u_final,
                            void* s_final, int32_t n_steps, void* stream);

/* Scan a device state [batch][2][ny][nx] for NaN/Inf. Synchronises `stream`.
 * Returns FD_OK, FD_ENONFINITE, or (learned contexts, state finite) FD_ETIMEOUT
 * when a bounded wait of a tensor-core kernel gave up since the last check
 * (see fd_options.spin_limit); the timeout is reported once and then cleared. */
fd_status fd_check_finite(fd_ctx* ctx, const void* u, void* stream);

/* Number of kernel launches issued by the last fd_step / fd_rollout call. */
int32_t fd_last_launch_count(const fd_ctx* ctx);

/* ---- learnable module (options.learned = 1) ------------------------------
 *
 * The flux block's per-face kernels become W_P + proj(W_L + C_theta(u)_f)
 * (Sec. 3.4, integrated operator), where C_theta is a 6-layer conv3x3 network
 * (2 -> 64 x5 -> 160 channels, GELU between layers, periodic padding) run on
 * the tensor cores with BF16 weights and activations and FP32 accumulation,
 * and proj removes the sum and the first axial and transverse moments of the
 * learned part. With k_c > 0 the temporal correction (Sec. 3.2, Eq. for u_k;
 * Sec. 3.5) u_k <- P(u_k + TC(u_{k-k_c} .. u_{k-1}) - mean) is applied after
 * every k_c-th step of a rollout, with TC a network of the same shape
 * (2 k_c -> 64 x5 -> 2). The learned module is built for FP32 and runs on two
 * paths. Square 32^2 and 64^2 grids run it on the tensor cores (BF16
 * activations), with everything below: the frequency-domain operator, the FNO
 * temporal correction, the ablation variants, the reverse mode and training.
 * Every other grid runs it on the generic-grid path (path 3, also selectable for
 * 32^2 and 64^2): Burgers on any nx x ny in [4, 8192]^2 (the 25^2 and 100^2
 * presets of App. C.1), Navier-Stokes on power-of-two nx x ny in [32, 2048]^2
 * (rectangular, e.g. the 128 x 64 shear grid, or square beyond 64^2). There the
 * network runs on the CUDA cores with FP32 activations; the stencil network, W_L,
 * the CNN temporal correction and ablation 1 are built, forward and reverse mode
 * (training included), the Fourier operators are not (FD_EUNSUPPORTED at
 * fd_init).
 *
 * Parameter layout (float32, fd_param_count values):
 *   W_L[kind 2][axis 2][5][4]                      (kind 0 interp, 1 deriv;
 *                                                   axis 0 x, 1 y; derivative
 *                                                   parts are in units of 1/h)
 *   W_Ls[kind 2][axis 2][5][4] (only with scalar_learned): the scalar's W_L
 *   stencil layer l = 0..5: W[Cout][Cin][3][3], b[Cout]
 *                   with (Cin, Cout) = (2,64) (64,64) x4 (64,160);
 *                   output channel 20 q + 4 r + c is tap (r, c) of instance q
 *                   (q: 0 u-x-interp, 1 u-x-deriv, 2 u-y-interp, 3 u-y-deriv,
 *                    4 v-x-interp, 5 v-x-deriv, 6 v-y-interp, 7 v-y-deriv).
 *                   With scalar_learned: (3,64) ... (64,240), input channel 2
 *                   is s, and channels 160 + 20 m + 4 r + c are the scalar's
 *                   instances m (0 s-x-interp, 1 s-x-deriv, 2 s-y-interp,
 *                   3 s-y-deriv; their 5 x 4 taps sit at transverse offset
 *                   r - 2 and axial offset c - 2 from the face's cell)
 *   temporal correction (only when k_c > 0): layers as above with
 *                   (Cin, Cout) = (2 k_c, 64) (64,64) x4 (64, 2); input channel
 *                   2 s + c is component c of u_{k-k_c+s}. With tc_fno_layers > 0
 *                   instead a Fourier neural operator in the layout of O_F below
 *                   with P_w[C][2 k_c] (same input channels) and Q_w[2][C],
 *                   Q_b[2] (width, modes and layers from the tc_fno_* options).
 *   frequency-domain operator O_F (only when fno_layers = L > 0; width C,
 *                   modes M): P_w[C][2], P_b[C]; per layer R[2M][M][C][C][2]
 *                   (complex channel matrices [in][out] of the kept modes, real
 *                   and imaginary parts; rows 0 .. M-1 are ky = 0 .. M-1, rows
 *                   M .. 2M-1 are ky = N-M .. N-1; kx = 0 .. M-1), W[C][C]
 *                   ([out][in]), b[C]; then Q_w[8][C], Q_b[8]. O_F(u) = Q(v_L),
 *                   v_0 = P(u), v_l = sigma(W_l v_{l-1} + b_l + irfft2(R_l .
 *                   rfft2(v_{l-1}))) with sigma = GELU except after the last
 *                   layer; channel q of O_F(u) is added to instance q's face
 *                   values. All in FP32 on the CUDA cores.
 * Network weights are rounded to BF16 (round to nearest even) on upload;
 * biases, W_L and the O_F parameters stay FP32. */

/* Number of float32 parameters fd_set_params expects (0 when not learned). */
int64_t fd_param_count(const fd_ctx* ctx);

/* Upload the learnable parameters from a HOST float32 array of `count`
 * values (layout above). Synchronises `stream`. FD_EINVAL on a wrong count or
 * a context without the learned option. */
fd_status fd_set_params(fd_ctx* ctx, const float* params, int64_t count, void* stream);

/* Same as fd_set_params from a DEVICE float32 array (for optimisers that keep
 * the parameters on the GPU): stream-ordered, no synchronisation; the array
 * may be overwritten once the work queued on `stream` has run. */
fd_status fd_set_params_device(fd_ctx* ctx, const float* params, int64_t count, void* stream);

/* Stencil-network forward pass alone: coef_out[batch][160][ny][nx] (device,
 * float32) = C_theta(u) for the device state u. For tests and diagnostics;
 * coef_out = NULL runs the network only (its BF16 output stays internal).
 * On a scalar_learned context u is [batch][3][ny][nx] (u, v, s) and coef_out
 * [batch][240][ny][nx]. */
fd_status fd_network_forward(fd_ctx* ctx, const void* u, float* coef_out, void* stream);

/* ---- reverse mode ----------------------------------------------------------
 *
 * Vector-Jacobian product of one time step u' = FV(u) (the solver's
 * differentiability, which the paper's training through unrolled rollouts
 * relies on: Sec. 4.1 loss, Sec. 3.2 integrated solver). Given the state u_in
 * and the cotangent lam_out = dL/du', computes lam_in = (du'/du)^T lam_out and,
 * for a learned context, adds (du'/dtheta)^T lam_out to dparams.
 *
 * The step is recomputed from u_in (stage states and every network activation
 * of the four RK stages are kept in a context-owned workspace, allocated by the
 * first call), then the stages are run backwards: the projection is symmetric
 * (its own adjoint), the face operators transpose to scatters, the per-face
 * kernel cotangent passes through the consistency projection to the network
 * output, and the network's data and weight gradients run on the tensor cores
 * (BF16 operands, FP32 accumulation; the weight gradients are reduced
 * deterministically).
 *
 * u_in, lam_out, lam_in: device float32 [batch][2][ny][nx]; lam_in may alias
 * lam_out. dparams: device float32 array of fd_param_count values in the
 * fd_set_params layout, ACCUMULATED into (+=); NULL skips the parameter
 * gradients. Stream-ordered; the first call allocates and synchronises.
 * With a temporal correction (k_c > 0) this is the VJP of the FV step alone,
 * the step fd_rollout takes before it applies a correction; the correction's
 * own reverse mode is fd_tc_adjoint, and fd_rollout_adjoint / fd_train_step
 * combine the two. Scope: FP32 contexts with N = 32 or 64 off the generic-grid
 * path, plain or learned (with or without the frequency-domain operator, any
 * ablation variant), and FP32 contexts of the generic-grid path, plain or
 * learned (ablation 0 or 1): there the stage states are recomputed, each
 * stage's network forward is run again keeping its pre-activations, and every
 * reverse product runs on the CUDA cores in FP32 (the weight gradients reduced
 * over pixels in a fixed order); the workspace (about 200 floats per cell, 650
 * for learned contexts) is allocated by the first call.
 * FD_EUNSUPPORTED otherwise (FP64 generic-grid contexts, a model that learns the
 * scalar). FD_EINVAL for null pointers, dparams on a plain context or
 * parameters not yet set. */
fd_status fd_step_adjoint(fd_ctx* ctx, const void* u_in, const void* lam_out, void* lam_in, float* dparams,
                          void* stream);

/* Reverse mode of one temporal correction (Sec. 3.2, Sec. 3.5):
 * u_k = P(V + c - mean(c)), c = TC(u_{k-k_c}, .., u_{k-1}), V = FV(u_{k-1}),
 * the CNN head of the correction (2 k_c -> 64 x4 -> 2, GELU) or its Fourier
 * neural operator (tc_fno_layers > 0). Given the
 * cotangent lam of u_k: vbar = P(lam), the cotangent of V (P is symmetric and
 * so is the mean removal, c_bar = P(lam) - mean), and hist_bar = the cotangents
 * of the k_c history states through the network; dparams (may be NULL)
 * accumulates the network's weight and bias gradients. The network's forward
 * activations are recomputed; its data and weight gradients run on the tensor
 * cores (BF16 operands, FP32 accumulation) except the first layer's data
 * gradient (CUDA cores, FP32).
 * hist: device [k_c][batch][2][n][n] float32 (u_{k-k_c} first); lam, vbar:
 * [batch][2][n][n] (vbar may be NULL); hist_bar: [k_c][batch][2][n][n],
 * written. A learned context with k_c > 0 (on the generic-grid path: the CNN
 * head on the CUDA cores, FP32); FD_EUNSUPPORTED otherwise, FD_EINVAL for null
 * pointers or parameters not yet set. */
fd_status fd_tc_adjoint(fd_ctx* ctx, const void* hist, const void* lam, void* vbar, void* hist_bar, float* dparams,
                        void* stream);

/* Reverse mode of an n-step rollout u_0 -> (u_1 .. u_n) with checkpoints:
 * lam_traj[n][batch][2][ny][nx] holds the cotangents dL/du_k of the states
 * after steps 1 .. n (device); lam0 receives dL/du_0; dparams (learned
 * context, may be NULL) accumulates dL/dtheta. The forward pass keeps only the
 * states u_0, u_k, u_2k, ... (k = ckpt_every) and each segment is recomputed
 * before its steps are run backwards with fd_step_adjoint, so the memory
 * is (n/k + k + 1) states plus one step's workspace. With a temporal
 * correction (k_c > 0) the corrected states' cotangents also flow back to
 * their history windows (fd_tc_adjoint), k must be a multiple of k_c (so a
 * window never crosses a checkpoint) and k_c more states are kept. Same scope
 * as fd_step_adjoint; the workspace grows on demand (allocating calls).
 * FD_EINVAL for null pointers, n_steps or ckpt_every < 1, or ckpt_every not a
 * multiple of k_c. */
fd_status fd_rollout_adjoint(fd_ctx* ctx, const void* u0, int32_t n_steps, int32_t ckpt_every,
                             const void* lam_traj, void* lam0, float* dparams, void* stream);

/* One training step of the paper's objective (Sec. 4, Model Training): the
 * rollout of n_steps from u0 is compared with targets[n][batch][2][ny][nx]
 * (device, the coarse-grained labels of u_1 .. u_n) by the mean squared error
 * over every step, trajectory and element; *loss (device double) receives the
 * loss, dparams (device, fd_param_count values) accumulates its gradient.
 * Checkpointing as in fd_rollout_adjoint. */
fd_status fd_train_step(fd_ctx* ctx, const void* u0, const void* targets, int32_t n_steps, int32_t ckpt_every,
                        float* dparams, double* loss, void* stream);

/* Reverse mode of one joint step of the velocity and the passive scalar (the
 * step fd_rollout_scalar takes; shear flow, App. C.1). Given (u_in, s_in) and the
 * cotangents (lam_u_out, lam_s_out) of (u', s'), computes (lam_u_in, lam_s_in) =
 * the transposed Jacobian applied to them and, for a context built with
 * scalar_learned = 1, accumulates the parameter gradient (W_L, W_Ls, the
 * stencil network on (u, v, s)) into dparams (+=, may be NULL). The stage states
 * are recomputed; the scalar's stages read the projected stage velocities, so
 * every stage's velocity cotangent also collects the scalar flux's term; the
 * scalar is not projected. u_in, lam_u_*: device float32 [batch][2][ny][nx];
 * s_in, lam_s_*: [batch][ny][nx]; the outputs may alias the cotangents.
 * Scope: FP32 contexts of the generic-grid path, plain or with scalar_learned
 * (FD_EUNSUPPORTED otherwise); FD_EINVAL for null pointers, a negative or
 * non-finite diffusivity, dparams on a plain context or parameters not set.
 * The first call allocates its workspace. */
fd_status fd_step_adjoint_scalar(fd_ctx* ctx, double diffusivity, const void* u_in, const void* s_in,
                                 const void* lam_u_out, const void* lam_s_out, void* lam_u_in, void* lam_s_in,
                                 float* dparams, void* stream);

/* One training step of a model that learns the scalar: the joint rollout of
 * n_steps from (u0, s0) (with the velocity's temporal correction every k_c
 * steps) against targets_u[n][batch][2][ny][nx] and targets_s[n][batch][ny][nx]
 * by the mean squared error over every step, trajectory and element of the
 * velocity and the scalar together; *loss (device double) receives it, dparams
 * accumulates its gradient. Checkpointing as in fd_rollout_adjoint (ckpt_every
 * a multiple of k_c). Needs scalar_learned = 1 (FD_EUNSUPPORTED otherwise). */
fd_status fd_train_step_scalar(fd_ctx* ctx, double diffusivity, const void* u0, const void* s0, const void* targets_u,
                               const void* targets_s, int32_t n_steps, int32_t ckpt_every, float* dparams,
                               double* loss, void* stream);

/* *loss = mean((pred - target)^2) over `count` float32 device elements (FP64
 * accumulation, fixed reduction order: deterministic); when grad is non-NULL,
 * grad = 2 (pred - target) / count. Uses the context's workspace. */
fd_status fd_mse_loss(fd_ctx* ctx, const float* pred, const float* target, int64_t count, double* loss,
                      float* grad, void* stream);

/* Kinetic-energy spectrum (the energy spectra of the forced-flow comparison,
 * Sec. 4 / Fig. 5): for each trajectory b of the device state u (FP32
 * [batch][2][N][N], N >= 32), spectrum[b][k] = 1/2 sum over the integer
 * wavevectors whose length rounds to k of |u^|^2 + |v^|^2, where u^ is the DFT
 * normalised by 1/N^2 (so that sum_k spectrum[b][k] over k <= N/sqrt(2) is
 * 1/2 mean(u^2 + v^2)), for k = 0 .. kmax (kmax <= N). spectrum: device
 * double[batch][kmax + 1], overwritten. A complex scratch of the state's size
 * is allocated on the first call and kept by the context. Errors: FD_EINVAL,
 * FD_EUNSUPPORTED (FP64 or N < 32), FD_ENOMEM, FD_ECUDA. */
fd_status fd_energy_spectrum(fd_ctx* ctx, const void* u, double* spectrum, int32_t kmax, void* stream);

/* Vorticity correlation (App. D.1, PCC; the accuracy measure of the paper's
 * correlation curves): for each trajectory b, the Pearson correlation of the
 * corner vorticities w = (v - v[i-1]) / dx - (u - u[j-1]) / dy of the device
 * states a[b] and b[b] (context grid and dtype), accumulated in FP64 in a fixed
 * order. pcc: device double[batch]. Uses the context's workspace. */
fd_status fd_vorticity_pcc(fd_ctx* ctx, const void* a, const void* b, double* pcc, void* stream);

/* One Adam update (the optimiser of the paper's training; Kingma & Ba 2015)
 * of `count` float32 device parameters: m, v are the caller-owned first and
 * second moment buffers (zero before step t = 1), t >= 1 the step number.
 * When zero_grads != 0 the gradient buffer is cleared after use.
 * Context-free; errors are reported through fd_last_error(NULL). */
fd_status fd_adam_step(float* params, float* grads, float* m, float* v, int64_t count, int32_t t, float lr,
                       float beta1, float beta2, float eps, int32_t zero_grads, void* stream);

/* Coarse-graining of fine-grid states into training labels (Sec. 4,
 * Simulation Datasets; App. C.1): fine[batch][2][n_fine][n_fine] ->
 * coarse[batch][2][n_fine/ratio][n_fine/ratio] by face averages: a coarse
 * face value is the mean of the `ratio` fine face values that tile the coarse
 * face, which keeps a divergence-free field divergence-free. dtype: fd_dtype.
 * Context-free; errors are reported through fd_last_error(NULL). */
fd_status fd_downsample(const void* fine, void* coarse, int32_t batch, int32_t n_fine, int32_t ratio,
                        int32_t dtype, void* stream);

/* ---- launch plans and the autotuner ------------------------------------------
 *
 * How a plain context's batch is laid out on the GPU. The paper has no
 * counterpart (it runs one trajectory at a time on its own hardware); every
 * plan computes the same step, and plans differ only in rounding order.
 *   path 1 (plain, on chip): trajectories [0, n_onchip) run on the on-chip
 *     rollout kernel with `cluster` CTAs per trajectory (each CTA owns
 *     N / cluster rows); `resident` of them fit on the device at once, the
 *     rest run in further waves. Trajectories [n_onchip, batch) run on the
 *     streaming kernels (FP32, N >= 32) on a second, library-owned stream,
 *     concurrently, on the SMs the resident clusters leave free; the call's
 *     stream waits for both parts (graph capture of the call's stream
 *     captures both).
 *   path 2 (plain, streaming only) and path 3 (learned) have one plan each.
 * A new context starts on its default plan: the first cluster shape of its
 * grid, the whole batch on chip. */
typedef struct {
  int32_t path;       /* 1 plain on chip (+ streaming part), 2 streaming only, 3 learned,
                         4 generic grid (output) */
  int32_t cluster;    /* CTAs per on-chip trajectory; 0 when n_onchip == 0 */
  int32_t n_onchip;   /* trajectories [0, n_onchip) on the on-chip kernel */
  int32_t n_stream;   /* trajectories [n_onchip, batch) on the streaming kernels */
  int32_t resident;   /* on-chip trajectories resident at once on this device (output) */
  double us_per_step; /* per-step time measured by fd_autotune (output; 0 = not measured) */
} fd_plan;

/* The context's current plan. Errors: FD_EINVAL for null pointers. */
fd_status fd_get_plan(const fd_ctx* ctx, fd_plan* plan);

/* Select a plan: cluster, n_onchip and n_stream are read (n_onchip +
 * n_stream = batch). Synchronises the device. Errors: FD_EINVAL for a split
 * that does not add up to the batch; FD_EUNSUPPORTED for a cluster size this
 * build has no kernel for at this N, a streaming part the grid cannot take
 * (FP64, N < 32), or any change to a learned or streaming-only context. */
fd_status fd_set_plan(fd_ctx* ctx, const fd_plan* plan);

/* Time every candidate plan of the context for `probe_steps` time steps
 * (<= 0: 32) on a zero state of the context's shape (a library-owned scratch
 * buffer of two states, freed before return), keep the fastest, and
 * describe the candidates in report[0 .. min(max_report, *n_report) - 1]
 * with their measured us_per_step. Candidates: every cluster shape with the
 * whole batch on chip; for each shape, splits that keep on chip the full
 * waves (when the resident count does not divide the batch) or 3/4, 1/2 or
 * 1/4 of one wave, with the rest on the streaming kernels; the whole batch on
 * the streaming kernels. Learned and
 * streaming-only contexts have one candidate, which is timed. Runs on
 * `stream` and synchronises it; report may be NULL when max_report is 0.
 * Errors: FD_EINVAL, FD_ENOMEM, FD_ECUDA (the previous plan is kept). */
fd_status fd_autotune(fd_ctx* ctx, int32_t probe_steps, fd_plan* report, int32_t max_report, int32_t* n_report,
                      void* stream);

/* ---- batches of rollouts ----------------------------------------------------
 *
 * Many concurrent trajectories of uneven grid sizes and flow types, learned
 * and plain: one context per (grid, flow, dtype, learned) group, each with its
 * own device states; a batch runs every member's rollout as one CUDA graph
 * (captured by the first fd_batch_run after the last fd_batch_add, replayed by
 * a single graph launch afterwards). The trajectories of every plain FP32
 * member with N = 16, 32 or 64 whose plan keeps the whole batch on chip run
 * in ONE persistent launch: a work list of (context, trajectory) items, larger
 * grids first, that the launch's CTAs take items from until it is exhausted
 * (per derivative order one launch); each item's result is bit-identical to
 * its context's own on-chip rollout. Every other member is a parallel branch
 * of the graph running its own rollout. The
 * paper has no counterpart (it advances one trajectory at a time); this is the
 * serving form of fd_rollout. A context may appear once per batch and must not
 * be used by other calls while its batch runs; the state pointers are fixed at
 * fd_batch_add (u_final may alias u0). A member whose launch plan changes
 * between runs (fd_set_plan, fd_autotune) makes the next fd_batch_run capture
 * the graph again, since a plan change can replace buffers the old graph used.
 * Destroy the batch before any of its member contexts. */
typedef struct fd_batch fd_batch; /* opaque, library-owned */

fd_status fd_batch_create(fd_batch** out);
fd_status fd_batch_add(fd_batch* batch, fd_ctx* ctx, const void* u0, void* u_final, int32_t n_steps);
fd_status fd_batch_run(fd_batch* batch, void* stream);
/* kernel launches inside one fd_batch_run (the graph's kernel nodes) */
int32_t fd_batch_launch_count(const fd_batch* batch);
/* Turn the persistent launch on (default) or off (every member its own
 * branch); takes effect at the next fd_batch_run (which captures again).
 * Errors: FD_EINVAL for a null batch. */
fd_status fd_batch_set_persistent(fd_batch* batch, int32_t enable);
/* trajectories that the graph of the last fd_batch_run runs in the persistent
 * launch */
int32_t fd_batch_persistent_count(const fd_batch* batch);
const char* fd_batch_last_error(const fd_batch* batch);
fd_status fd_batch_destroy(fd_batch* batch);

/* Release the context and its device tables (synchronises the device). */
fd_status fd_destroy(fd_ctx* ctx);

/* Message of the last error on ctx (ctx may be NULL for fd_init errors).
 * The string is owned by the library and valid until the next call. */
const char* fd_last_error(const fd_ctx* ctx);

/* Largest element count fd_check_finite_noalloc accepts (2^24 elements: a
 * batch of 128 256^2 states, or of two 2048^2 states). */
#define FD_NOALLOC_MAX_ELEMS (1 << 24)

/* Allocation-free NaN/Inf scan for callers that must not allocate device
 * memory (a framework pool that forbids raw cudaMalloc, a latency-critical
 * path that must not enter the allocator). The paper has no counterpart: this
 * is a service of the library, not a step of the method.
 * u: device pointer to `count` elements of type `dtype` (fd_dtype), any layout.
 * nonfinite: host pointer, receives the number of NaN/Inf elements.
 * Work runs on `stream`, which the call synchronises. The only scratch is a
 * 32 KB array in the library's static device memory (held on every GPU that
 * loads the library until exit); the call allocates nothing. The first call
 * on a device looks up that array's address: make it before any stream
 * capture. Calls that overlap on the GPU share the array and race.
 * Returns FD_OK (no NaN/Inf), FD_ENONFINITE, FD_EINVAL (null pointer, unknown
 * dtype, count < 0 or count > FD_NOALLOC_MAX_ELEMS), FD_EUNSUPPORTED (the
 * current device's index is 64 or more) or FD_ECUDA. */
fd_status fd_check_finite_noalloc(const void* u, int64_t count, int32_t dtype, int64_t* nonfinite,
                                  void* stream);

/* Library version string. */
const char* fd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LDFV_FD_H */
