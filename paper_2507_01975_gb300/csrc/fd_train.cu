// fd_train.cu -- the training runtime behind the C ABI: coarse-graining of
// fine-grid fields into training labels, the MSE objective of the paper's
// training (Sec. 4, Model Training), the checkpointed reverse mode of an
// n-step rollout, one fused training step (forward, loss, backward) and Adam.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "../../include/fd.h"
#include "fd_ctx.h"

using namespace ldfv;

fd_status fd_tc_adjoint_ptrs(fd_ctx* c, const float* const* hist_host, const float* lam, float* hist_bar,
                             size_t state_stride, float* dparams, cudaStream_t st, int* launches);

namespace {

constexpr int kRedBlocks = 512;  // fixed grid of the deterministic reductions

// Coarse value on a coarse face = mean of the r fine face values that tile it
// (u: the fine west faces i = r I, j = r J .. r J + r - 1; v: the fine south
// faces j = r J, i = r I .. r I + r - 1). Summing the fine divergences of a
// block telescopes to r times the coarse divergence, so a divergence-free fine
// field stays divergence-free.
template <typename T>
__global__ void face_average_kernel(const T* fine, T* coarse, int batch, int nf, int r) {
  const int nc = nf / r;
  const size_t total = (size_t)batch * 2 * nc * nc;
  const T inv = (T)1 / (T)r;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(idx % nc), J = (int)((idx / nc) % nc);
    const size_t bc = idx / ((size_t)nc * nc);  // b * 2 + component
    const T* f = fine + bc * (size_t)nf * nf;
    T s = 0;
    if ((bc & 1) == 0) {
      for (int k = 0; k < r; ++k) s += f[(size_t)(r * J + k) * nf + (size_t)r * I];
    } else {
      const T* row = f + (size_t)r * J * nf + (size_t)r * I;
      for (int k = 0; k < r; ++k) s += row[k];
    }
    coarse[idx] = s * inv;
  }
}

// sum of (pred - target)^2 per block (FP64); optional gradient scale (pred - target)
// written (mode 1) or added (mode 2) to grad
__global__ void mse_partial_kernel(const float* pred, const float* target, size_t n, float scale, float* grad,
                                   int grad_mode, double* partial) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = pred[i] - target[i];
    s += (double)d * (double)d;
    if (grad_mode == 1)
      grad[i] = scale * d;
    else if (grad_mode == 2)
      grad[i] += scale * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// out (+)= factor * sum(partial[0 .. n)), one block, fixed order
__global__ void sum_partials_kernel(const double* partial, int n, double factor, double* out, int accumulate) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = (accumulate ? *out : 0.0) + factor * s;
  }
}

__global__ void axpy_kernel(float* y, const float* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) y[i] += x[i];
}

// Adam (Kingma & Ba, 2015, Algorithm 1) with the bias corrections folded into
// the step: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
// p <- p - lr (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t
__global__ void adam_kernel(float* p, float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2, int zero_grads) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    if (zero_grads) g[i] = 0.0f;
  }
}

// Per-trajectory partial sums for the Pearson correlation of corner vorticities
// w = (v - v[i-1]) / dx - (u - u[j-1]) / dy of two states a, b: (sum wa, sum wb,
// sum wa^2, sum wb^2, sum wa wb) in FP64, one row of 5 per block.
template <typename T>
__global__ void vort_partial_kernel(const T* a, const T* b, int nx, int ny, double idx, double idy, double* partial) {
  __shared__ double red[5][32];
  const size_t NN = (size_t)nx * ny;
  const int tr = blockIdx.y;
  const T* ua = a + (size_t)tr * 2 * NN;
  const T* ub = b + (size_t)tr * 2 * NN;
  double s[5] = {0, 0, 0, 0, 0};
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < NN; c += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(c / nx), i = (int)(c - (size_t)j * nx);
    const size_t cw = (size_t)j * nx + (i - 1 + nx) % nx, cs = (size_t)((j - 1 + ny) % ny) * nx + i;
    const double wa = ((double)ua[NN + c] - (double)ua[NN + cw]) * idx - ((double)ua[c] - (double)ua[cs]) * idy;
    const double wb = ((double)ub[NN + c] - (double)ub[NN + cw]) * idx - ((double)ub[c] - (double)ub[cs]) * idy;
    s[0] += wa;
    s[1] += wb;
    s[2] += wa * wa;
    s[3] += wb * wb;
    s[4] += wa * wb;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
    if (lane == 0) red[k][w] = s[k];
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
    partial[((size_t)tr * gridDim.x + blockIdx.x) * 5 + threadIdx.x] = t;
  }
}

__global__ void vort_pcc_kernel(const double* partial, int nblk, double n, double* out) {
  const int tr = blockIdx.x;
  if (threadIdx.x != 0) return;
  double s[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k < nblk; ++k)
    for (int m = 0; m < 5; ++m) s[m] += partial[((size_t)tr * nblk + k) * 5 + m];
  const double cov = s[4] - s[0] * s[1] / n;
  const double va = s[2] - s[0] * s[0] / n, vb = s[3] - s[1] * s[1] / n;
  out[tr] = cov / sqrt(va * vb);
}

int grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t mse(fd_ctx* c, const float* pred, const float* target, size_t n, float scale, float* grad, int grad_mode,
                double factor, double* loss, int accumulate, cudaStream_t st) {
  mse_partial_kernel<<<kRedBlocks, 256, 0, st>>>(pred, target, n, scale, grad, grad_mode, c->trn->partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (loss) {
    sum_partials_kernel<<<1, 256, 0, st>>>(c->trn->partial, kRedBlocks, factor, loss, accumulate);
    e = cudaGetLastError();
  }
  return e;
}

// workspace of the rollout reverse mode: nseg + 1 checkpoints, one segment, one
// cotangent (and, with a temporal correction, the k_c history cotangents)
fd_status train_reserve(fd_ctx* c, int nseg, int seglen) {
  TrainState*& T = c->trn;
  if (!T) {
    T = new (std::nothrow) TrainState();
    if (!T) return fd_set_error(c, FD_ENOMEM, "out of host memory");
    if (cudaMalloc(&T->partial, kRedBlocks * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&T->lam, fd_state_bytes(c->grid)) != cudaSuccess)
      return fd_set_error(c, FD_ENOMEM, "training workspace: out of device memory");
  }
  const int kc = c->lrn ? c->lrn->kc : c->glrn ? c->glrn->kc : 0;
  if (kc > 0 && !T->pend) {
    if (cudaMalloc(&T->pend, fd_state_bytes(c->grid) * kc) != cudaSuccess) {
      T->pend = nullptr;
      return fd_set_error(c, FD_ENOMEM, "training workspace: history cotangents do not fit");
    }
  }
  const size_t bytes = fd_state_bytes(c->grid);
  if (nseg + 1 > T->nckpt) {
    if (T->ckpt) cudaFree(T->ckpt);
    T->ckpt = nullptr;
    T->nckpt = 0;
    if (cudaMalloc(&T->ckpt, bytes * (nseg + 1)) != cudaSuccess)
      return fd_set_error(c, FD_ENOMEM, "training workspace: %d checkpoints do not fit", nseg + 1);
    T->nckpt = nseg + 1;
  }
  if (seglen > T->nseg) {
    if (T->seg) cudaFree(T->seg);
    T->seg = nullptr;
    T->nseg = 0;
    if (cudaMalloc(&T->seg, bytes * seglen) != cudaSuccess)
      return fd_set_error(c, FD_ENOMEM, "training workspace: a segment of %d states does not fit", seglen);
    T->nseg = seglen;
  }
  return FD_OK;
}

// The reverse mode of u_0 -> (u_1 .. u_n) with checkpoints every k steps.
// Either lam_traj (cotangents of u_1 .. u_n) is given, or targets: then the
// cotangents are those of L = mean((u_k - t_k)^2) over every step and element,
// and L is written to *loss.
//
// With a temporal correction every k_c-th state u_m (m = M k_c) was formed
// from the k_c states u_{m-k_c} .. u_{m-1} as well (Sec. 3.2); its cotangent
// also reaches them (fd_tc_adjoint) through T.pend, slot s holding the
// cotangent of u_{m-k_c+s}, which is added once the sweep arrives there. The
// checkpoint interval is a multiple of k_c, so a window never crosses a
// segment. The FV step before a correction is differentiated by
// fd_step_adjoint with the corrected state's cotangent: its output is already
// projected and P is idempotent, so P(lam) and lam give the same result.
fd_status rollout_reverse(fd_ctx* c, const float* u0, int n, int k, const float* lam_traj, const float* targets,
                          float* lam0, float* dparams, double* loss, cudaStream_t st, const char* who) {
  const int kc = c->lrn ? c->lrn->kc : c->glrn ? c->glrn->kc : 0;
  if (kc > 0 && k % kc != 0)
    return fd_set_error(c, FD_EINVAL, "%s: ckpt_every must be a multiple of k_c (%d)", who, kc);
  const int nseg = (n + k - 1) / k;
  fd_status s = train_reserve(c, nseg, k);
  if (s != FD_OK) return s;
  TrainState& T = *c->trn;
  const size_t bytes = fd_state_bytes(c->grid);
  const size_t slot = bytes / sizeof(float);
  int launches = 0;
  // forward: checkpoints u_0, u_k, u_2k, ..., u_n
  cudaError_t e = cudaMemcpyAsync(T.ckpt, u0, bytes, cudaMemcpyDeviceToDevice, st);
  for (int g = 0; g < nseg && e == cudaSuccess; ++g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    s = fd_rollout(c, T.ckpt + g * slot, nullptr, T.ckpt + (g + 1) * slot, len, 0, st);
    if (s != FD_OK) return s;
    launches += c->launches;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(T.lam, 0, bytes, st);
  const double total = (double)n * (double)slot;
  const float gscale = (float)(2.0 / total);
  bool first_loss = true;
  // backward over the segments
  for (int g = nseg - 1; g >= 0 && e == cudaSuccess; --g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    if (len > 1) {
      // recompute u_{gk+1} .. u_{gk+len-1}
      s = fd_rollout(c, T.ckpt + g * slot, T.seg, T.seg + (size_t)(len - 1) * slot, len - 1, 1, st);
      if (s != FD_OK) return s;
      launches += c->launches;
    }
    auto state = [&](int m) -> const float* {  // u_m, m in [g k, g k + len]
      const int jj = m - g * k;
      return jj == 0 ? T.ckpt + g * slot : (jj == len ? T.ckpt + (g + 1) * slot : T.seg + (size_t)(jj - 1) * slot);
    };
    for (int j = len - 1; j >= 0 && e == cudaSuccess; --j) {
      const int step = g * k + j;  // u_step -> u_{step + 1}
      const float* out = j == len - 1 ? T.ckpt + (g + 1) * slot : T.seg + (size_t)j * slot;
      const float* in = j == 0 ? T.ckpt + g * slot : T.seg + (size_t)(j - 1) * slot;
      if (kc > 0 && step + 1 < n && (step + 1) / kc * kc + kc <= n) {
        // u_{step+1} lies in the history window of the correction at the end of
        // its k_c block: add what that correction sent back to it
        axpy_kernel<<<grid_for(slot), 256, 0, st>>>(T.lam, T.pend + (size_t)((step + 1) % kc) * slot, slot);
        e = cudaGetLastError();
        ++launches;
        if (e != cudaSuccess) break;
      }
      if (targets) {
        e = mse(c, out, targets + (size_t)step * slot, slot, gscale, T.lam, 2, 1.0 / total, loss, first_loss ? 0 : 1,
                st);
        first_loss = false;
        launches += 2;
      } else {
        axpy_kernel<<<grid_for(slot), 256, 0, st>>>(T.lam, lam_traj + (size_t)step * slot, slot);
        e = cudaGetLastError();
        ++launches;
      }
      if (e != cudaSuccess) break;
      if (kc > 0 && (step + 1) % kc == 0) {
        // u_{step+1} is a corrected state: its history u_{step+1-k_c} .. u_step
        const float* hist[8];
        for (int q = 0; q < kc; ++q) hist[q] = state(step + 1 - kc + q);
        s = fd_tc_adjoint_ptrs(c, hist, T.lam, T.pend, slot, dparams, st, &launches);
        if (s != FD_OK) return s;
      }
      s = fd_step_adjoint(c, in, T.lam, T.lam, dparams, st);
      if (s != FD_OK) return s;
      launches += c->launches;
    }
    if (kc > 0 && g == 0 && e == cudaSuccess) {
      // u_0 is never a step's output above (a later segment's first state is
      // the previous segment's last): add its history cotangent here
      if (kc <= n) {
        axpy_kernel<<<grid_for(slot), 256, 0, st>>>(T.lam, T.pend, slot);
        e = cudaGetLastError();
        ++launches;
      }
    }
  }
  if (e == cudaSuccess && lam0) e = cudaMemcpyAsync(lam0, T.lam, bytes, cudaMemcpyDeviceToDevice, st);
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "%s: %s", who, cudaGetErrorString(e));
  return FD_OK;
}

// the scalar's part of the joint training workspace
fd_status train_reserve_scalar(fd_ctx* c, int nseg, int seglen) {
  TrainState& T = *c->trn;
  const size_t sb = (size_t)c->grid.batch * c->grid.nx * c->grid.ny * sizeof(float);
  if (!T.lam_s && cudaMalloc(&T.lam_s, sb) != cudaSuccess) {
    T.lam_s = nullptr;
    return fd_set_error(c, FD_ENOMEM, "training workspace: out of device memory");
  }
  if (nseg + 1 > T.nckpt_s) {
    if (T.ckpt_s) cudaFree(T.ckpt_s);
    T.ckpt_s = nullptr;
    T.nckpt_s = 0;
    if (cudaMalloc(&T.ckpt_s, sb * (nseg + 1)) != cudaSuccess)
      return fd_set_error(c, FD_ENOMEM, "training workspace: %d scalar checkpoints do not fit", nseg + 1);
    T.nckpt_s = nseg + 1;
  }
  if (seglen > T.nseg_s) {
    if (T.seg_s) cudaFree(T.seg_s);
    T.seg_s = nullptr;
    T.nseg_s = 0;
    if (cudaMalloc(&T.seg_s, sb * seglen) != cudaSuccess)
      return fd_set_error(c, FD_ENOMEM, "training workspace: a scalar segment of %d states does not fit", seglen);
    T.nseg_s = seglen;
  }
  return FD_OK;
}

// The reverse mode of the joint rollout (u_0, s_0) -> (u_1, s_1) .. (u_n, s_n)
// with checkpoints every k steps and the loss L = mean over every step,
// trajectory and element of (u_k - tu_k)^2 and (s_k - ts_k)^2 together (the
// velocity's two components and the scalar weigh alike). The temporal
// correction acts on the velocity only, so its history cotangents are the
// velocity's, as in rollout_reverse.
fd_status rollout_reverse_scalar(fd_ctx* c, double diff, const float* u0, const float* s0, int n, int k,
                                 const float* tu, const float* ts, float* dparams, double* loss, cudaStream_t st) {
  const char* who = "fd_train_step_scalar";
  const int kc = c->glrn ? c->glrn->kc : 0;
  if (kc > 0 && k % kc != 0) return fd_set_error(c, FD_EINVAL, "%s: ckpt_every must be a multiple of k_c (%d)", who, kc);
  const int nseg = (n + k - 1) / k;
  fd_status s = train_reserve(c, nseg, k);
  if (s == FD_OK) s = train_reserve_scalar(c, nseg, k);
  if (s != FD_OK) return s;
  TrainState& T = *c->trn;
  const size_t bytes = fd_state_bytes(c->grid), slot = bytes / sizeof(float);
  const size_t sslot = (size_t)c->grid.batch * c->grid.nx * c->grid.ny, sbytes = sslot * sizeof(float);
  int launches = 0;
  cudaError_t e = cudaMemcpyAsync(T.ckpt, u0, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(T.ckpt_s, s0, sbytes, cudaMemcpyDeviceToDevice, st);
  for (int g = 0; g < nseg && e == cudaSuccess; ++g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    s = fd_rollout_scalar_impl(c, diff, T.ckpt + g * slot, T.ckpt_s + g * sslot, T.ckpt + (g + 1) * slot,
                               T.ckpt_s + (g + 1) * sslot, len, st, nullptr, nullptr);
    if (s != FD_OK) return s;
    launches += c->launches;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(T.lam, 0, bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(T.lam_s, 0, sbytes, st);
  const double total = (double)n * (double)(slot + sslot);
  const float gscale = (float)(2.0 / total);
  bool first_loss = true;
  for (int g = nseg - 1; g >= 0 && e == cudaSuccess; --g) {
    const int len = (g + 1) * k <= n ? k : n - g * k;
    if (len > 1) {
      // recompute (u, s) at steps g k + 1 .. g k + len - 1
      s = fd_rollout_scalar_impl(c, diff, T.ckpt + g * slot, T.ckpt_s + g * sslot, T.seg + (size_t)(len - 1) * slot,
                                 T.seg_s + (size_t)(len - 1) * sslot, len - 1, st, T.seg, T.seg_s);
      if (s != FD_OK) return s;
      launches += c->launches;
    }
    auto state = [&](int m) -> const float* {  // u_m, m in [g k, g k + len]
      const int jj = m - g * k;
      return jj == 0 ? T.ckpt + g * slot : (jj == len ? T.ckpt + (g + 1) * slot : T.seg + (size_t)(jj - 1) * slot);
    };
    for (int j = len - 1; j >= 0 && e == cudaSuccess; --j) {
      const int step = g * k + j;
      const float* out_u = j == len - 1 ? T.ckpt + (g + 1) * slot : T.seg + (size_t)j * slot;
      const float* out_s = j == len - 1 ? T.ckpt_s + (g + 1) * sslot : T.seg_s + (size_t)j * sslot;
      const float* in_u = j == 0 ? T.ckpt + g * slot : T.seg + (size_t)(j - 1) * slot;
      const float* in_s = j == 0 ? T.ckpt_s + g * sslot : T.seg_s + (size_t)(j - 1) * sslot;
      if (kc > 0 && step + 1 < n && (step + 1) / kc * kc + kc <= n) {
        axpy_kernel<<<grid_for(slot), 256, 0, st>>>(T.lam, T.pend + (size_t)((step + 1) % kc) * slot, slot);
        e = cudaGetLastError();
        ++launches;
        if (e != cudaSuccess) break;
      }
      e = mse(c, out_u, tu + (size_t)step * slot, slot, gscale, T.lam, 2, 1.0 / total, loss, first_loss ? 0 : 1, st);
      if (e == cudaSuccess)
        e = mse(c, out_s, ts + (size_t)step * sslot, sslot, gscale, T.lam_s, 2, 1.0 / total, loss, 1, st);
      first_loss = false;
      launches += 4;
      if (e != cudaSuccess) break;
      if (kc > 0 && (step + 1) % kc == 0) {
        const float* hist[8];
        for (int q = 0; q < kc; ++q) hist[q] = state(step + 1 - kc + q);
        s = fd_tc_adjoint_ptrs(c, hist, T.lam, T.pend, slot, dparams, st, &launches);
        if (s != FD_OK) return s;
      }
      s = fd_gadjoint_step_scalar(c, diff, in_u, in_s, T.lam, T.lam_s, T.lam, T.lam_s, dparams, st);
      if (s != FD_OK) return s;
      launches += c->launches;
    }
    if (kc > 0 && g == 0 && e == cudaSuccess && kc <= n) {
      axpy_kernel<<<grid_for(slot), 256, 0, st>>>(T.lam, T.pend, slot);
      e = cudaGetLastError();
      ++launches;
    }
  }
  c->launches = launches;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "%s: %s", who, cudaGetErrorString(e));
  return FD_OK;
}

}  // namespace

void fd_train_free(fd_ctx* c) {
  TrainState* T = c->trn;
  if (!T) return;
  void* ps[] = {T->ckpt, T->seg, T->lam, T->partial, T->corr, T->pend, T->ckpt_s, T->seg_s, T->lam_s};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete T;
  c->trn = nullptr;
}

extern "C" {

fd_status fd_downsample(const void* fine, void* coarse, int32_t batch, int32_t n_fine, int32_t ratio, int32_t dtype,
                        void* stream) {
  if (!fine || !coarse) return fd_set_error(nullptr, FD_EINVAL, "fd_downsample: null pointer");
  if (batch < 1 || n_fine < 1 || ratio < 1 || n_fine % ratio != 0)
    return fd_set_error(nullptr, FD_EINVAL, "fd_downsample: need batch >= 1 and ratio dividing n_fine");
  if (dtype != FD_F32 && dtype != FD_F64) return fd_set_error(nullptr, FD_EINVAL, "fd_downsample: unknown dtype");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nc = (size_t)(n_fine / ratio);
  const int blocks = grid_for((size_t)batch * 2 * nc * nc);
  if (dtype == FD_F32)
    face_average_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(fine), static_cast<float*>(coarse),
                                                       batch, n_fine, ratio);
  else
    face_average_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(fine),
                                                        static_cast<double*>(coarse), batch, n_fine, ratio);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ECUDA, "fd_downsample: %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_mse_loss(fd_ctx* c, const float* pred, const float* target, int64_t count, double* loss,
                      float* grad, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_mse_loss: null context");
  if (!pred || !target || !loss) return fd_set_error(c, FD_EINVAL, "fd_mse_loss: null pointer");
  if (count < 1) return fd_set_error(c, FD_EINVAL, "fd_mse_loss: count must be >= 1");
  fd_status s = train_reserve(c, 0, 0);
  if (s != FD_OK) return s;
  cudaError_t e = mse(c, pred, target, (size_t)count, (float)(2.0 / (double)count), grad, grad ? 1 : 0,
                      1.0 / (double)count, loss, 0, static_cast<cudaStream_t>(stream));
  c->launches = 2;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_mse_loss: %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_rollout_adjoint(fd_ctx* c, const void* u0, int32_t n_steps, int32_t ckpt_every, const void* lam_traj,
                             void* lam0, float* dparams, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_rollout_adjoint: null context");
  if (!u0 || !lam_traj || !lam0) return fd_set_error(c, FD_EINVAL, "fd_rollout_adjoint: null pointer");
  if (n_steps < 1 || ckpt_every < 1) return fd_set_error(c, FD_EINVAL, "fd_rollout_adjoint: n_steps, ckpt_every >= 1");
  return rollout_reverse(c, static_cast<const float*>(u0), n_steps, ckpt_every, static_cast<const float*>(lam_traj),
                         nullptr, static_cast<float*>(lam0), dparams, nullptr, static_cast<cudaStream_t>(stream),
                         "fd_rollout_adjoint");
}

fd_status fd_train_step(fd_ctx* c, const void* u0, const void* targets, int32_t n_steps, int32_t ckpt_every,
                        float* dparams, double* loss, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_train_step: null context");
  if (!u0 || !targets || !loss) return fd_set_error(c, FD_EINVAL, "fd_train_step: null pointer");
  if (n_steps < 1 || ckpt_every < 1) return fd_set_error(c, FD_EINVAL, "fd_train_step: n_steps, ckpt_every >= 1");
  return rollout_reverse(c, static_cast<const float*>(u0), n_steps, ckpt_every, nullptr,
                         static_cast<const float*>(targets), nullptr, dparams, loss,
                         static_cast<cudaStream_t>(stream), "fd_train_step");
}

fd_status fd_train_step_scalar(fd_ctx* c, double diffusivity, const void* u0, const void* s0, const void* targets_u,
                               const void* targets_s, int32_t n_steps, int32_t ckpt_every, float* dparams,
                               double* loss, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_train_step_scalar: null context");
  c->launches = 0;
  if (!u0 || !s0 || !targets_u || !targets_s || !loss)
    return fd_set_error(c, FD_EINVAL, "fd_train_step_scalar: null pointer");
  if (n_steps < 1 || ckpt_every < 1)
    return fd_set_error(c, FD_EINVAL, "fd_train_step_scalar: n_steps, ckpt_every >= 1");
  if (!c->gen || !c->glrn || !c->glrn->scalar)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_train_step_scalar: needs a learned context with scalar_learned = 1");
  if (!(diffusivity >= 0) || !std::isfinite(diffusivity))
    return fd_set_error(c, FD_EINVAL, "fd_train_step_scalar: the diffusivity must be >= 0");
  return rollout_reverse_scalar(c, diffusivity, static_cast<const float*>(u0), static_cast<const float*>(s0), n_steps,
                                ckpt_every, static_cast<const float*>(targets_u), static_cast<const float*>(targets_s),
                                dparams, loss, static_cast<cudaStream_t>(stream));
}

fd_status fd_vorticity_pcc(fd_ctx* c, const void* a, const void* b, double* pcc, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_vorticity_pcc: null context");
  if (!a || !b || !pcc) return fd_set_error(c, FD_EINVAL, "fd_vorticity_pcc: null pointer");
  fd_status s = train_reserve(c, 0, 0);
  if (s != FD_OK) return s;
  TrainState& T = *c->trn;
  constexpr int kBlk = 64;
  const int B = c->grid.batch;
  if (T.ncorr < (size_t)B * kBlk * 5) {
    if (T.corr) cudaFree(T.corr);
    T.corr = nullptr;
    T.ncorr = 0;
    if (cudaMalloc(&T.corr, (size_t)B * kBlk * 5 * sizeof(double)) != cudaSuccess)
      return fd_set_error(c, FD_ENOMEM, "fd_vorticity_pcc: out of device memory");
    T.ncorr = (size_t)B * kBlk * 5;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const dim3 grid(kBlk, B);
  const fd_grid& g = c->grid;
  const double idx = g.nx / g.lx, idy = g.ny / g.ly;
  if (g.dtype == FD_F64)
    vort_partial_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(a), static_cast<const double*>(b),
                                                     g.nx, g.ny, idx, idy, T.corr);
  else
    vort_partial_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(a), static_cast<const float*>(b),
                                                    g.nx, g.ny, idx, idy, T.corr);
  vort_pcc_kernel<<<B, 32, 0, st>>>(T.corr, kBlk, (double)c->grid.nx * c->grid.ny, pcc);
  cudaError_t e = cudaGetLastError();
  c->launches = 2;
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_vorticity_pcc: %s", cudaGetErrorString(e));
  return FD_OK;
}

fd_status fd_adam_step(float* params, float* grads, float* m, float* v, int64_t count, int32_t t, float lr,
                       float beta1, float beta2, float eps, int32_t zero_grads, void* stream) {
  if (!params || !grads || !m || !v) return fd_set_error(nullptr, FD_EINVAL, "fd_adam_step: null pointer");
  if (count < 1 || t < 1) return fd_set_error(nullptr, FD_EINVAL, "fd_adam_step: count >= 1 and t >= 1 required");
  const float c1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  const float c2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  adam_kernel<<<grid_for((size_t)count), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grads, m, v, (size_t)count, lr, beta1, beta2, eps, c1, c2, zero_grads);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fd_set_error(nullptr, FD_ECUDA, "fd_adam_step: %s", cudaGetErrorString(e));
  return FD_OK;
}

}  // extern "C"
