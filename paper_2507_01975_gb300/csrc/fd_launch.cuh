// fd_launch.cuh -- launch, attribute and occupancy helpers of the on-chip
// rollout kernel. Each translation unit that instantiates configurations of
// fv_rollout_kernel includes this header; the helpers are translation-unit
// local because the kernel stubs they take the address of are.
#pragma once

#include <cuda_runtime.h>

#include "fd_ctx.h"
#include "fv_fused.cuh"

namespace ldfv {

template <typename T, int LOGN, int CS, int NT, int DORD>
static cudaError_t launch_fused(const FvArgs& a, int batch, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS, batch, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CS > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fv_rollout_kernel<T, LOGN, CS, NT, DORD>, a);
}

template <typename T, int LOGN, int CS, int NT, int DORD>
static cudaError_t prepare_fused(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(fv_rollout_kernel<T, LOGN, CS, NT, DORD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CS > 8) {
    e = cudaFuncSetAttribute(fv_rollout_kernel<T, LOGN, CS, NT, DORD>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  return e;
}

// Trajectories that run at once on this device (co-resident clusters); the
// kernel attributes must have been set by prepare_fused first.
template <typename T, int LOGN, int CS, int NT, int DORD>
static cudaError_t occupancy_fused(size_t smem, int* trajectories) {
  *trajectories = 0;
  if constexpr (CS == 1) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fv_rollout_kernel<T, LOGN, CS, NT, DORD>, NT, smem);
    if (e == cudaSuccess) *trajectories = per_sm * sms;
    return e;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(trajectories, fv_rollout_kernel<T, LOGN, CS, NT, DORD>, &cfg);
  }
}

template <typename T, int LOGN, int CS, int NT>
static Launcher make_launcher(int dord) {
  Launcher l;
  l.cs = CS;
  l.nt = NT;
  l.smem = FusedCfg<T, LOGN, CS, NT>::SMEM;
  if (dord == 4) {
    l.launch = &launch_fused<T, LOGN, CS, NT, 4>;
    l.prepare = &prepare_fused<T, LOGN, CS, NT, 4>;
    l.occupancy = &occupancy_fused<T, LOGN, CS, NT, 4>;
  } else {
    l.launch = &launch_fused<T, LOGN, CS, NT, 2>;
    l.prepare = &prepare_fused<T, LOGN, CS, NT, 2>;
    l.occupancy = &occupancy_fused<T, LOGN, CS, NT, 2>;
  }
  return l;
}

}  // namespace ldfv
