// Kernels of the 1536-bit size class (k = 54 channels per base).
#include "kernels.cuh"
#include "kernels_api.h"

namespace mr {

using C1536 = Cfg<54, 48, 50, 8, 128, 4>;

static cudaError_t launch_modexp_1536(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C1536>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C1536><<<grid, C1536::THREADS, C1536::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1536(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C1536>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C1536><<<grid, C1536::THREADS, C1536::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass1536 = {
    1536, C1536::K, C1536::W, C1536::WX, C1536::TPI, C1536::THREADS, C1536::IPB, C1536::NPT, C1536::SMEM_BYTES,
    launch_modexp_1536, launch_crt_1536};

}  // namespace mr
