// fd_spectrum.cu -- kinetic-energy spectrum E(k) of a state (the energy spectra
// the paper compares for the forced flow, Sec. 4 / Fig. 5).
//
// E(k) = 1/2 sum over the wavevectors whose length rounds to k of
// (|u^|^2 + |v^|^2), u^ = N^-2 DFT(u). With z = u + i v, Z = DFT(z) gives
// u^(k) = (Z(k) + conj Z(-k)) / 2N^2 and v^(k) = (Z(k) - conj Z(-k)) / 2iN^2, so
// |u^(k)|^2 + |v^(k)|^2 + |u^(-k)|^2 + |v^(-k)|^2 = (|Z(k)|^2 + |Z(-k)|^2) / N^4: a
// shell, being symmetric under k -> -k, sums to sum |Z|^2 / N^4 over its
// wavevectors. One complex 2D FFT per trajectory: register-resident Stockham
// row transforms into a scratch spectrum, then column transforms whose squared
// magnitudes go into a shared-memory shell histogram (FP64) and from there into
// the caller's array.
#include <cuda_runtime.h>

#include "../../include/fd.h"
#include "fd_ctx.h"
#include "fv_fft.cuh"

using namespace ldfv;

namespace {

// nearest integer to sqrt(q), exact: the k with k^2 - k < q <= k^2 + k
__device__ __forceinline__ int shell_of(int q) {
  int k = (int)sqrtf((float)q);
  while (k * k > q) --k;
  while ((k + 1) * (k + 1) <= q) ++k;
  return q > k * k + k ? k + 1 : k;
}

// rows: z(y, .) = u(y, .) + i v(y, .) -> Z_rows(y, kx), natural order
template <int LOGN>
__global__ void __launch_bounds__(RowCfg<LOGN>::NT) spectrum_rows_kernel(const float* u, float2* zs,
                                                                        const float2* tw) {
  using C = RowCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = C::N, T = C::T;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + C::F * SP::BUF;
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int b = blockIdx.y, y = blockIdx.x * C::F + f;
  const size_t NN = (size_t)N * N;
  const float* ur = u + (size_t)b * 2 * NN + (size_t)y * N;
  const float* vr = ur + NN;
  build_pass_twiddles<LOGN>(tws, tw);
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = make_float2(ur[t + m * T], vr[t + m * T]);
  __syncthreads();
  fft_forward<LOGN>(z, sm + f * SP::BUF, tws, t, TransformSync{1 + f, T});
  float2* zr = zs + (size_t)b * NN + (size_t)y * N;
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) zr[t + s * T + r * SP::NSL] = z[s + SP::SL * r];
}

// columns: Z(ky, kx) = DFT_y(Z_rows(., kx)); |Z|^2 into the shells 0 .. kmax
template <int LOGN>
__global__ void __launch_bounds__(ColCfg<LOGN>::NT) spectrum_cols_kernel(const float2* zs, const float2* tw,
                                                                        double* spec, int kmax, double scale) {
  using C = ColCfg<LOGN>;
  using SP = SPlan<LOGN>;
  constexpr int N = C::N, T = C::T;
  extern __shared__ __align__(16) float2 sm[];
  float2* tws = sm + C::C * SP::BUF;
  double* hist = reinterpret_cast<double*>(tws + SP::TW);  // [kmax + 1]
  const int f = threadIdx.x / T, t = threadIdx.x % T;
  const int b = blockIdx.y, kx = blockIdx.x * C::C + f;
  const size_t NN = (size_t)N * N;
  build_pass_twiddles<LOGN>(tws, tw);
  for (int k = threadIdx.x; k <= kmax; k += blockDim.x) hist[k] = 0.0;
  const float2* zc = zs + (size_t)b * NN + kx;
  float2 z[kFP];
#pragma unroll
  for (int m = 0; m < kFP; ++m) z[m] = zc[(size_t)(t + m * T) * N];
  __syncthreads();
  fft_forward<LOGN>(z, sm + f * SP::BUF, tws, t, TransformSync{1 + f, T});
  const int kxs = kx < N / 2 ? kx : kx - N;
#pragma unroll
  for (int s = 0; s < SP::SL; ++s)
#pragma unroll
    for (int r = 0; r < SP::RL; ++r) {
      const int ky = t + s * T + r * SP::NSL;
      const int kys = ky < N / 2 ? ky : ky - N;
      const int k = shell_of(kxs * kxs + kys * kys);
      const float2 v = z[s + SP::SL * r];
      if (k <= kmax) atomicAdd(&hist[k], (double)v.x * v.x + (double)v.y * v.y);
    }
  __syncthreads();
  double* sb = spec + (size_t)b * (kmax + 1);
  for (int k = threadIdx.x; k <= kmax; k += blockDim.x)
    if (hist[k] != 0.0) atomicAdd(&sb[k], hist[k] * scale);
}

template <int LOGN>
cudaError_t run_spectrum(const float* u, float2* zs, const float2* tw, double* spec, int kmax, int batch,
                         cudaStream_t st) {
  using R = RowCfg<LOGN>;
  using C = ColCfg<LOGN>;
  const size_t rsm = R::SMEM;
  const size_t csm = C::SMEM + (size_t)(kmax + 1) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(spectrum_rows_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spectrum_cols_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
  if (e != cudaSuccess) return e;
  spectrum_rows_kernel<LOGN><<<dim3(R::N / R::F, batch), R::NT, rsm, st>>>(u, zs, tw);
  const double n2 = (double)R::N * R::N;
  spectrum_cols_kernel<LOGN><<<dim3(R::N / C::C, batch), C::NT, csm, st>>>(zs, tw, spec, kmax, 0.5 / (n2 * n2));
  return cudaGetLastError();
}

}  // namespace

extern "C" {

fd_status fd_energy_spectrum(fd_ctx* c, const void* u, double* spectrum, int32_t kmax, void* stream) {
  if (!c) return fd_set_error(nullptr, FD_EINVAL, "fd_energy_spectrum: null context");
  if (c->gen) return fd_set_error(c, FD_EUNSUPPORTED, "fd_energy_spectrum: not built for the generic-grid path");
  if (!u || !spectrum) return fd_set_error(c, FD_EINVAL, "fd_energy_spectrum: null pointer");
  const int n = c->grid.nx;
  if (kmax < 0 || kmax > n) return fd_set_error(c, FD_EINVAL, "fd_energy_spectrum: kmax must be in [0, N]");
  if (c->grid.dtype != FD_F32 || n < 32)
    return fd_set_error(c, FD_EUNSUPPORTED, "fd_energy_spectrum: FP32 states with N >= 32");
  const int B = c->grid.batch;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t zbytes = (size_t)B * n * n * sizeof(float2);
  if (c->spec_bytes < zbytes) {
    if (c->d_spec) cudaFree(c->d_spec);
    c->d_spec = nullptr;
    c->spec_bytes = 0;
    cudaError_t e = cudaMalloc(&c->d_spec, zbytes);
    if (e != cudaSuccess) return fd_set_error(c, FD_ENOMEM, "fd_energy_spectrum: cudaMalloc: %s", cudaGetErrorString(e));
    c->spec_bytes = zbytes;
  }
  cudaError_t e = cudaMemsetAsync(spectrum, 0, (size_t)B * (kmax + 1) * sizeof(double), st);
  const float* uf = static_cast<const float*>(u);
  float2* zs = static_cast<float2*>(c->d_spec);
  const float2* tw = reinterpret_cast<const float2*>(c->base.tw);
  if (e == cudaSuccess) {
    switch (c->logn) {
      case 5: e = run_spectrum<5>(uf, zs, tw, spectrum, kmax, B, st); break;
      case 6: e = run_spectrum<6>(uf, zs, tw, spectrum, kmax, B, st); break;
      case 7: e = run_spectrum<7>(uf, zs, tw, spectrum, kmax, B, st); break;
      case 8: e = run_spectrum<8>(uf, zs, tw, spectrum, kmax, B, st); break;
      case 9: e = run_spectrum<9>(uf, zs, tw, spectrum, kmax, B, st); break;
      case 10: e = run_spectrum<10>(uf, zs, tw, spectrum, kmax, B, st); break;
      case 11: e = run_spectrum<11>(uf, zs, tw, spectrum, kmax, B, st); break;
      default: return fd_set_error(c, FD_EUNSUPPORTED, "fd_energy_spectrum: N = %d", n);
    }
  }
  if (e != cudaSuccess) return fd_set_error(c, FD_ECUDA, "fd_energy_spectrum: %s", cudaGetErrorString(e));
  c->launches = 2;
  return FD_OK;
}

}  // extern "C"
