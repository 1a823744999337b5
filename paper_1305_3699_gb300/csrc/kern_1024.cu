// Kernels of the 1024-bit size class (k = 36 channels per base).
#include "kernels.cuh"
#include "kernels_api.h"

namespace mr {

using C1024 = Cfg<36, 32, 34, 4, 128, 4>;

static cudaError_t launch_modexp_1024(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C1024><<<grid, C1024::THREADS, C1024::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1024(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1024::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C1024><<<grid, C1024::THREADS, C1024::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass1024 = {
    1024, C1024::K, C1024::W, C1024::WX, C1024::TPI, C1024::THREADS, C1024::IPB, C1024::NPT, C1024::SMEM_BYTES,
    launch_modexp_1024, launch_crt_1024};

}  // namespace mr
