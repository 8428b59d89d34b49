// fd_api.cu -- C ABI of the FV step library (declared in include/fd.h).
//
// Host-side validation, the per-context constant tables (FFT twiddles,
// Laplacian symbols, forcing profile, stencil taps) and the dispatch to the
// cluster-resident rollout kernel instantiated for each grid size and type.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fd_launch.cuh"
#include "fv_fused.cuh"

using namespace ldfv;

// learned path (fd_learned.cu)
fd_status fd_learned_init(fd_ctx* c);
void fd_learned_free(fd_ctx* c);
void fd_adjoint_free(fd_ctx* c);
void fd_train_free(fd_ctx* c);
fd_status fd_learned_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                             cudaStream_t st, bool allow_graph);
fd_status fd_learned_error_flag(fd_ctx* c);
// generic-grid path (fd_generic.cu): Burgers on any grid, Navier-Stokes on
// rectangular power-of-two grids
bool fd_generic_wanted(const fd_grid& g, int path);
fd_status fd_generic_init(fd_ctx* c);
void fd_generic_free(fd_ctx* c);
fd_status fd_generic_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                             cudaStream_t st, bool allow_graph);

// streaming path (fd_large.cu)
bool fd_large_supported(int dtype, int n);
fd_status fd_large_init(fd_ctx* c);
void fd_large_free(fd_ctx* c);
fd_status fd_large_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                           cudaStream_t st, bool allow_graph);
// launch plans (fd_variants.cu, fd_plan.cu)
void fd_extra_launchers(int dtype, int logn, int dord, std::vector<Launcher>& out);
fd_status fd_plain_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int n_steps, int save_every,
                           cudaStream_t st, bool allow_graph);

namespace {

thread_local std::string g_init_error;



// Cluster size and block size per (type, N): CTAs own R = N / CS rows, each
// thread one column of R * N / NT of those rows. Every configuration with
// N >= 64 fits two CTAs per SM, so all clusters of a batch are co-resident.
bool pick_launcher(int dtype, int logn, int dord, Launcher* out) {
  if (dtype == FD_F32) {
    switch (logn) {
      case 3: *out = make_launcher<float, 3, 1, 64>(dord); return true;
      case 4: *out = make_launcher<float, 4, 1, 128>(dord); return true;
      case 5: *out = make_launcher<float, 5, 1, 256>(dord); return true;
      case 6: *out = make_launcher<float, 6, 1, 512>(dord); return true;
      case 7: *out = make_launcher<float, 7, 2, 512>(dord); return true;
      case 8: *out = make_launcher<float, 8, 8, 512>(dord); return true;
      default: return false;
    }
  } else {
    switch (logn) {
      case 3: *out = make_launcher<double, 3, 1, 64>(dord); return true;
      case 4: *out = make_launcher<double, 4, 1, 128>(dord); return true;
      case 5: *out = make_launcher<double, 5, 1, 256>(dord); return true;
      case 6: *out = make_launcher<double, 6, 1, 512>(dord); return true;
      case 7: *out = make_launcher<double, 7, 4, 512>(dord); return true;
      default: return false;
    }
  }
}

}  // namespace



fd_status fd_set_error(fd_ctx* c, fd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_init_error = buf;
  return s;
}

static size_t elem_size(const fd_grid& g) { return g.dtype == FD_F64 ? 8 : 4; }
size_t fd_state_bytes(const fd_grid& g) {
  return (size_t)g.batch * 2 * (size_t)g.nx * (size_t)g.ny * elem_size(g);
}

template <typename T>
static void fill_tables(fd_ctx* c, std::vector<unsigned char>& host) {
  const int n = c->grid.nx;
  const double dx = c->grid.lx / n, dy = c->grid.ly / n;
  const size_t nt = (size_t)(n / 2) * 2, ns = n / 2 + 2, ny = n, nf = n;
  c->off_symx = nt * sizeof(T);
  c->off_symy = c->off_symx + ns * sizeof(T);
  c->off_frc = c->off_symy + ny * sizeof(T);
  host.assign(c->off_frc + nf * sizeof(T), 0);
  T* tw = reinterpret_cast<T*>(host.data());
  T* sx = reinterpret_cast<T*>(host.data() + c->off_symx);
  T* sy = reinterpret_cast<T*>(host.data() + c->off_symy);
  T* fr = reinterpret_cast<T*>(host.data() + c->off_frc);
  const double pi = 3.14159265358979323846;
  for (int m = 0; m < n / 2; ++m) {
    tw[2 * m] = (T)std::cos(2 * pi * m / n);
    tw[2 * m + 1] = (T)-std::sin(2 * pi * m / n);
  }
  for (int k = 0; k <= n / 2; ++k) {
    if (c->opts.poisson_symbol == 0) {
      const double s = std::sin(pi * k / n);
      sx[k] = (T)(-4.0 / (dx * dx) * s * s);
    } else {
      const double e = 2 * pi * k / c->grid.lx;
      sx[k] = (T)(-e * e);
    }
  }
  for (int k = 0; k < n; ++k) {
    if (c->opts.poisson_symbol == 0) {
      const double s = std::sin(pi * k / n);
      sy[k] = (T)(-4.0 / (dy * dy) * s * s);
    } else {
      const int ks = k < n / 2 ? k : k - n;
      const double e = 2 * pi * ks / c->grid.ly;
      sy[k] = (T)(-e * e);
    }
  }
  for (int j = 0; j < n; ++j) {
    const double y = (j + 0.5) * dy;
    fr[j] = c->forcing.kind == 1 ? (T)(c->forcing.amp * std::sin(c->forcing.k * y)) : (T)0;
  }
}

extern "C" {

const char* fd_version(void) { return "ldfv 0.1 (sm_103a)"; }

const char* fd_last_error(const fd_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

int32_t fd_last_launch_count(const fd_ctx* ctx) { return ctx ? ctx->launches : 0; }

fd_status fd_init(const fd_grid* grid, double nu, double dt, const fd_forcing* forcing,
                  const fd_options* opts, fd_ctx** out) {
  if (!grid || !out) return fd_set_error(nullptr, FD_EINVAL, "fd_init: null grid or out pointer");
  *out = nullptr;
  const fd_grid g = *grid;
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  // Burgers on a non-power-of-two or rectangular grid, Navier-Stokes on a
  // rectangular power-of-two grid (or either with path 3) run on the
  // generic-grid kernels; every other grid must be a square power of two
  // learned contexts run on the tensor-core path on square 32^2 and 64^2 grids
  // (unless path 3 asks for the generic-grid path or the model learns the
  // passive scalar) and on the generic-grid path everywhere else
  const bool learned_req = opts && opts->learned == 1;
  const bool tc_grid = g.nx == g.ny && (g.nx == 32 || g.nx == 64);
  const bool scalar_req = learned_req && opts->scalar_learned != 0;
  const bool generic = fd_generic_wanted(g, opts ? opts->path : 0) ||
                       (learned_req && (!tc_grid || opts->path == 3 || scalar_req) && g.nx > 0 && g.ny > 0);
  if (generic && (g.nx < 4 || g.ny < 4 || g.nx > 8192 || g.ny > 8192))
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: nx, ny must be in [4, 8192] (got %d x %d)", g.nx, g.ny);
  if (generic && g.flow == FD_NAVIER_STOKES &&
      (g.dtype != FD_F32 || g.nx < 32 || g.ny < 32 || g.nx > 2048 || g.ny > 2048))
    return fd_set_error(nullptr, FD_EUNSUPPORTED,
                        "fd_init: Navier-Stokes on the generic-grid path is built for FP32, nx, ny in [32, 2048]");
  if (!generic && (!pow2(g.nx) || !pow2(g.ny) || g.nx < 8 || g.ny < 8 || g.nx > 2048 || g.ny > 2048))
    return fd_set_error(nullptr, FD_EINVAL,
                        "fd_init: nx, ny must be powers of two in [8, 2048] (got %d x %d; other grids are built for "
                        "Burgers only)", g.nx, g.ny);
  if (g.batch < 1 || g.batch > 65535) return fd_set_error(nullptr, FD_EINVAL, "fd_init: batch must be in [1, 65535]");
  if (!(g.lx > 0) || !(g.ly > 0)) return fd_set_error(nullptr, FD_EINVAL, "fd_init: box lengths must be positive");
  if (g.dtype != FD_F32 && g.dtype != FD_F64) return fd_set_error(nullptr, FD_EINVAL, "fd_init: unknown dtype");
  if (g.flow != FD_BURGERS && g.flow != FD_NAVIER_STOKES)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: unknown flow");
  if (!(dt > 0) || !std::isfinite(dt)) return fd_set_error(nullptr, FD_EINVAL, "fd_init: dt must be positive");
  if (!(nu >= 0) || !std::isfinite(nu)) return fd_set_error(nullptr, FD_EINVAL, "fd_init: nu must be >= 0");
  fd_options o = {4, 2, 0, 0, 0, 8, 1 << 26, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  static_assert(sizeof(fd_options) == 72, "fd_options layout");
  if (opts) o = *opts;
  if (o.deriv_order != 2 && o.deriv_order != 4)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: deriv_order must be 2 or 4");
  if (o.interp_order != 2) return fd_set_error(nullptr, FD_EINVAL, "fd_init: interp_order must be 2");
  if (o.poisson_symbol != 0 && o.poisson_symbol != 1)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: poisson_symbol must be 0 or 1");
  fd_forcing f = {0, 1.0, 4, 0.1};
  if (forcing) f = *forcing;
  if (f.kind != 0 && f.kind != 1) return fd_set_error(nullptr, FD_EINVAL, "fd_init: unknown forcing kind");
  if (!generic && g.nx != g.ny)
    return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: rectangular grids are built for Burgers only");
  if (o.learned != 0 && o.learned != 1) return fd_set_error(nullptr, FD_EINVAL, "fd_init: learned must be 0 or 1");
  if (!o.learned && o.k_c) return fd_set_error(nullptr, FD_EINVAL, "fd_init: k_c needs the learned option");
  if (o.scalar_learned != 0 && o.scalar_learned != 1)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: scalar_learned must be 0 or 1");
  if (o.scalar_learned && !o.learned)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: scalar_learned needs the learned option");
  if (o.path < 0 || o.path > 3) return fd_set_error(nullptr, FD_EINVAL, "fd_init: path must be 0, 1, 2 or 3");
  if (o.path == 3 && !generic)
    return fd_set_error(nullptr, FD_EUNSUPPORTED,
                        "fd_init: the generic-grid path (3) takes Burgers on any grid and Navier-Stokes on "
                        "power-of-two grids");
  if (generic && o.learned) {
    const fd_status ls = fd_glearned_check(g, o);
    if (ls != FD_OK) return ls;
  }
  if (generic && o.path != 0 && o.path != 3)
    return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: this grid runs on the generic-grid path (path 3) only");
  if (generic) {
    fd_ctx* c = new (std::nothrow) fd_ctx();
    if (!c) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: out of host memory");
    c->grid = g;
    c->forcing = f;
    c->opts = o;
    c->opts.path = 3;
    c->nu = nu;
    c->dt = dt;
    std::memset(&c->base, 0, sizeof c->base);
    fd_status gs = fd_generic_init(c);
    if (gs == FD_OK && o.learned) gs = fd_glearned_init(c);
    if (gs != FD_OK) {
      fd_glearned_free(c);
      fd_generic_free(c);
      delete c;
      return gs;
    }
    *out = c;
    return FD_OK;
  }
  if (o.fno_layers < 0 || o.fno_layers > 8)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: fno_layers must be in [0, 8]");
  if (o.fno_layers > 0) {
    if (!o.learned) return fd_set_error(nullptr, FD_EINVAL, "fd_init: the frequency-domain operator needs learned = 1");
    if (o.fno_width != 8 && o.fno_width != 16)
      return fd_set_error(nullptr, FD_EINVAL, "fd_init: fno_width must be 8 or 16 (the widths of Table S3)");
    if (o.fno_modes < 1 || 2 * o.fno_modes > g.nx)
      return fd_set_error(nullptr, FD_EINVAL, "fd_init: fno_modes must be in [1, N/2]");
  } else {
    o.fno_modes = o.fno_width = 0;
  }
  if (o.ablation < 0 || o.ablation > 2) return fd_set_error(nullptr, FD_EINVAL, "fd_init: ablation must be 0, 1 or 2");
  if (o.ablation && !o.learned) return fd_set_error(nullptr, FD_EINVAL, "fd_init: ablation variants need learned = 1");
  if (o.ablation == 2 && o.fno_layers <= 0)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: the frequency-operator-only variant needs fno_layers > 0");
  if (o.tc_fno_layers < 0 || o.tc_fno_layers > 8)
    return fd_set_error(nullptr, FD_EINVAL, "fd_init: tc_fno_layers must be in [0, 8]");
  if (o.tc_fno_layers > 0) {
    if (o.k_c <= 0) return fd_set_error(nullptr, FD_EINVAL, "fd_init: the FNO temporal correction needs k_c > 0");
    if (o.tc_fno_width != 8 && o.tc_fno_width != 16)
      return fd_set_error(nullptr, FD_EINVAL, "fd_init: tc_fno_width must be 8 or 16");
    if (o.tc_fno_modes < 1 || 2 * o.tc_fno_modes > g.nx)
      return fd_set_error(nullptr, FD_EINVAL, "fd_init: tc_fno_modes must be in [1, N/2]");
  } else {
    o.tc_fno_modes = o.tc_fno_width = 0;
  }
  int logn = 0;
  while ((1 << logn) < g.nx) ++logn;
  Launcher L;
  const bool onchip = o.path != 2 && pick_launcher(g.dtype, logn, o.deriv_order, &L);
  if (!onchip) {
    if (o.path == 1)
      return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: no on-chip kernel for N=%d dtype=%d", g.nx, g.dtype);
    if (!fd_large_supported(g.dtype, g.nx))
      return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: no kernel for N=%d dtype=%d (the streaming path is FP32, "
                          "N in [32, 2048])", g.nx, g.dtype);
    if (o.learned)
      return fd_set_error(nullptr, FD_EUNSUPPORTED, "fd_init: the learned path runs on chip (N = 32 or 64)");
  }

  fd_ctx* c = new (std::nothrow) fd_ctx();
  if (!c) return fd_set_error(nullptr, FD_ENOMEM, "fd_init: out of host memory");
  c->grid = g;
  c->forcing = f;
  c->opts = o;
  c->nu = nu;
  c->dt = dt;
  c->logn = logn;
  c->L = L;

  std::vector<unsigned char> host;
  if (g.dtype == FD_F64)
    fill_tables<double>(c, host);
  else
    fill_tables<float>(c, host);
  cudaError_t e = cudaMalloc(&c->d_tables, host.size());
  if (e != cudaSuccess) {
    delete c;
    return fd_set_error(nullptr, FD_ENOMEM, "fd_init: cudaMalloc: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpy(c->d_tables, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && onchip) e = L.prepare(L.smem);
  if (e == cudaSuccess && onchip) {
    // launch plan: the default configuration first, then the other cluster
    // shapes this build has for the grid (a shape that cannot be prepared on
    // this device is left out)
    std::vector<Launcher> extra;
    if (!o.learned) fd_extra_launchers(g.dtype, logn, o.deriv_order, extra);
    c->variants.push_back(L);
    for (const Launcher& x : extra)
      if (x.prepare(x.smem) == cudaSuccess) c->variants.push_back(x);
    cudaGetLastError();
    for (const Launcher& x : c->variants) {
      int cap = 0;
      if (x.occupancy(x.smem, &cap) != cudaSuccess) cap = 0;
      c->capacity.push_back(cap);
    }
    cudaGetLastError();
    c->n_onchip = g.batch;
  }
  if (e != cudaSuccess) {
    cudaFree(c->d_tables);
    delete c;
    return fd_set_error(nullptr, FD_ECUDA, "fd_init: device set-up: %s", cudaGetErrorString(e));
  }

  const int n = g.nx;
  const double dx = g.lx / n, dy = g.ly / n;
  FvArgs& a = c->base;
  std::memset(&a, 0, sizeof a);
  a.flow = g.flow;
  a.forcing = f.kind;
  a.dt = dt;
  a.nu = nu;
  a.idx = 1.0 / dx;
  a.idy = 1.0 / dy;
  a.drag = f.kind == 1 ? f.drag : 0.0;
  a.inv_nn = 1.0 / ((double)n * n);
  const char* base = static_cast<const char*>(c->d_tables);
  a.tw = base;
  a.symx = base + c->off_symx;
  a.symy = base + c->off_symy;
  a.frc = base + c->off_frc;
  if (!onchip) {
    fd_status ls = fd_large_init(c);
    if (ls != FD_OK) {
      fd_large_free(c);
      cudaFree(c->d_tables);
      delete c;
      return ls;
    }
  }
  if (o.learned) {
    fd_status ls = fd_learned_init(c);
    if (ls != FD_OK) {
      fd_learned_free(c);
      cudaFree(c->d_tables);
      delete c;
      return ls;
    }
  }
  *out = c;
  return FD_OK;
}

}  // extern "C"

// rollout behind fd_rollout; allow_graph = false issues every launch directly
// (for callers that capture the work into a graph of their own)
fd_status fd_rollout_impl(fd_ctx* c, const void* u0, void* traj, void* u_final, int32_t n_steps, int32_t save_every,
                          void* stream, bool allow_graph) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_rollout: null context");
  c->launches = 0;
  if (!u0 || !u_final) return fd_set_error(c, FD_EINVAL, "fd_rollout: null state pointer");
  if (n_steps < 0) return fd_set_error(c, FD_EINVAL, "fd_rollout: n_steps must be >= 0");
  if (save_every < 0) return fd_set_error(c, FD_EINVAL, "fd_rollout: save_every must be >= 0");
  if (save_every > 0 && !traj) return fd_set_error(c, FD_EINVAL, "fd_rollout: save_every > 0 needs traj");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->gen) return fd_generic_rollout(c, u0, traj, u_final, n_steps, save_every, st, allow_graph);
  if (c->lrn) return fd_learned_rollout(c, u0, traj, u_final, n_steps, save_every, st, allow_graph);
  if (c->big) return fd_large_rollout(c, u0, traj, u_final, n_steps, save_every, st, allow_graph);
  return fd_plain_rollout(c, u0, traj, u_final, n_steps, save_every, st, allow_graph);
}

extern "C" {

fd_status fd_rollout(fd_ctx* c, const void* u0, void* traj, void* u_final, int32_t n_steps,
                     int32_t save_every, void* stream) {
  return fd_rollout_impl(c, u0, traj, u_final, n_steps, save_every, stream, true);
}

fd_status fd_step(fd_ctx* c, const void* u_in, void* u_out, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_step: null context");
  return fd_rollout(c, u_in, nullptr, u_out, 1, 0, stream);
}

fd_status fd_rollout_host(fd_ctx* c, const void* u0_host, void* u_final_host, int32_t n_steps,
                          void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_rollout_host: null context");
  if (!u0_host || !u_final_host) return fd_set_error(c, FD_EINVAL, "fd_rollout_host: null host pointer");
  const size_t bytes = fd_state_bytes(c->grid);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!c->d_state) {
    cudaError_t e = cudaMalloc(&c->d_state, bytes);
    if (e != cudaSuccess) {
      c->d_state = nullptr;
      return fd_set_error(c, FD_ENOMEM, "fd_rollout_host: cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaMemcpyAsync(c->d_state, u0_host, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout_host: H2D copy: %s", cudaGetErrorString(e));
  fd_status s = fd_rollout(c, c->d_state, nullptr, c->d_state, n_steps, 0, stream);
  if (s != FD_OK) return s;
  e = cudaMemcpyAsync(u_final_host, c->d_state, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_rollout_host: D2H copy: %s", cudaGetErrorString(e));
  return fd_learned_error_flag(c);
}

}  // extern "C"

namespace {
template <typename T>
__global__ void finite_scan_kernel(const T* u, size_t n, unsigned* flag) {
  unsigned bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= isfinite((double)u[i]) ? 0u : 1u;
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}
}  // namespace

extern "C" {

fd_status fd_check_finite(fd_ctx* c, const void* u, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_check_finite: null context");
  if (!u) return fd_set_error(c, FD_EINVAL, "fd_check_finite: null state pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!c->d_flag) {
    e = cudaMalloc(&c->d_flag, sizeof(unsigned));
    if (e != cudaSuccess) {
      c->d_flag = nullptr;
      return fd_set_error(c, FD_ENOMEM, "fd_check_finite: cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  e = cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned), st);
  const size_t n = fd_state_bytes(c->grid) / elem_size(c->grid);
  if (e == cudaSuccess) {
    if (c->grid.dtype == FD_F64)
      finite_scan_kernel<double><<<152, 256, 0, st>>>(static_cast<const double*>(u), n, c->d_flag);
    else
      finite_scan_kernel<float><<<152, 256, 0, st>>>(static_cast<const float*>(u), n, c->d_flag);
    e = cudaGetLastError();
  }
  unsigned h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->d_flag, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_check_finite: %s", cudaGetErrorString(e));
  if (h) return fd_set_error(c, FD_ENONFINITE, "fd_check_finite: state holds NaN or Inf");
  return fd_learned_error_flag(c);
}

fd_status fd_destroy(fd_ctx* c) {
  if (!c) return FD_OK;
  cudaDeviceSynchronize();
  if (c->d_tables) cudaFree(c->d_tables);
  if (c->d_state) cudaFree(c->d_state);
  if (c->d_flag) cudaFree(c->d_flag);
  if (c->d_spec) cudaFree(c->d_spec);
  if (c->side) fd_destroy(c->side);
  if (c->fallback) fd_destroy(c->fallback);
  if (c->d_guard) cudaFree(c->d_guard);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  fd_train_free(c);
  fd_adjoint_free(c);
  fd_learned_free(c);
  fd_large_free(c);
  fd_gadjoint_free(c);
  fd_glearned_free(c);
  fd_generic_free(c);
  delete c;
  return FD_OK;
}

}  // extern "C"
