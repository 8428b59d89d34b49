// fd_noalloc.cu -- allocation-free NaN/Inf scan (fd_check_finite_noalloc).
//
// fd_check_finite keeps its result flag in device memory that it allocates on
// first use. Some callers must not allocate device memory at the point where
// they check a state: code that runs under a framework's caching allocator or
// memory pool that owns the whole device budget and forbids raw cudaMalloc,
// and code on a latency-critical path that must not enter the driver's
// allocator (cudaMalloc can synchronise the device). This entry point serves
// them. Its only scratch is the file-scope array below, which the loader
// places in device memory of every GPU that loads the library and which stays
// there until the process exits (32 KB per GPU).
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (the host-side name of a __device__ array is not a
// device address); make that first call before any stream capture. All calls
// share the one array, so calls that overlap on the GPU (two streams, two
// threads) race on it and must be serialised by the caller. The array keeps
// the last call's contents; nothing in it has to start at zero, because every
// slot a call reads is first written by a plain store of the same call.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fd.h"

namespace {

constexpr int kThreads = 256;
constexpr int kElemsPerThread = 16;
constexpr long long kElemsPerBlock = (long long)kThreads * kElemsPerThread;
constexpr int kMaxBlocks = FD_NOALLOC_MAX_ELEMS / (kThreads * kElemsPerThread);
static_assert((long long)kMaxBlocks * kElemsPerBlock == FD_NOALLOC_MAX_ELEMS, "exact block split");

// Per-block counts of non-finite elements in [0, kMaxBlocks), the total in
// slot kMaxBlocks. 4097 x 8 bytes; every call overwrites the slots it uses.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

template <typename T>
__global__ void __launch_bounds__(kThreads) count_nonfinite_blocks(const T* __restrict__ u, long long n,
                                                                   unsigned long long* scratch) {
  const long long base = (long long)blockIdx.x * kElemsPerBlock;
  unsigned long long bad = 0;
#pragma unroll
  for (int k = 0; k < kElemsPerThread; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i < n) bad += isfinite((double)u[i]) ? 0ull : 1ull;
  }
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffffu, bad, o);
  __shared__ unsigned long long warp_sum[kThreads / 32];
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += warp_sum[w];
    scratch[blockIdx.x] = s;  // plain store: no slot needs clearing beforehand
  }
}

__global__ void __launch_bounds__(kThreads) sum_block_counts(unsigned long long* scratch, int nblocks) {
  unsigned long long s = 0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) s += scratch[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ unsigned long long warp_sum[kThreads / 32];
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += warp_sum[w];
    scratch[kMaxBlocks] = t;
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not a device address).
fd_status scratch_on_current_device(unsigned long long** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return FD_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) {
    return FD_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      return FD_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned long long*>(g_scratch_ptr[dev]);
  return FD_OK;
}

}  // namespace

extern "C" {

fd_status fd_check_finite_noalloc(const void* u, int64_t count, int32_t dtype, int64_t* nonfinite,
                                  void* stream) {
  if (!u || !nonfinite) {
    return FD_EINVAL;
  }
  if (dtype != FD_F32 && dtype != FD_F64) {
    return FD_EINVAL;
  }
  if (count < 0 || count > (int64_t)FD_NOALLOC_MAX_ELEMS) {
    return FD_EINVAL;
  }
  *nonfinite = 0;
  if (count == 0) return FD_OK;
  unsigned long long* scratch = nullptr;
  fd_status s = scratch_on_current_device(&scratch);
  if (s != FD_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nblocks = (int)((count + kElemsPerBlock - 1) / kElemsPerBlock);
  if (dtype == FD_F64)
    count_nonfinite_blocks<double><<<nblocks, kThreads, 0, st>>>(static_cast<const double*>(u), count, scratch);
  else
    count_nonfinite_blocks<float><<<nblocks, kThreads, 0, st>>>(static_cast<const float*>(u), count, scratch);
  sum_block_counts<<<1, kThreads, 0, st>>>(scratch, nblocks);
  cudaError_t e = cudaGetLastError();
  unsigned long long total = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, scratch + kMaxBlocks, sizeof total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    return FD_ECUDA;
  }
  *nonfinite = (int64_t)total;
  if (total) {
    return FD_ENONFINITE;
  }
  return FD_OK;
}

}  // extern "C"
