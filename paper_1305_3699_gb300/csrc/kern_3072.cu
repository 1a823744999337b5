// Kernels of the 3072-bit size class (k = 108 channels per base).
#include "kernels.cuh"
#include "kernels_api.h"

namespace mr {

using C3072 = Cfg<108, 96, 97, 16, 256, 4>;

static cudaError_t launch_modexp_3072(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C3072>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C3072><<<grid, C3072::THREADS, C3072::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_3072(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C3072>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C3072><<<grid, C3072::THREADS, C3072::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass3072 = {
    3072, C3072::K, C3072::W, C3072::WX, C3072::TPI, C3072::THREADS, C3072::IPB, C3072::NPT, C3072::SMEM_BYTES,
    launch_modexp_3072, launch_crt_3072};

}  // namespace mr
