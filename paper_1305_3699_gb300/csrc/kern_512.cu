// Kernels of the 512-bit size class (k = 18 channels per base).
#include "kernels.cuh"
#include "kernels_api.h"

namespace mr {

using C512 = Cfg<18, 16, 17, 2, 128, 4>;

static cudaError_t launch_modexp_512(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C512>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C512><<<grid, C512::THREADS, C512::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_512(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C512>, cudaFuncAttributeMaxDynamicSharedMemorySize, C512::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C512><<<grid, C512::THREADS, C512::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass512 = {
    512, C512::K, C512::W, C512::WX, C512::TPI, C512::THREADS, C512::IPB, C512::NPT, C512::SMEM_BYTES,
    launch_modexp_512, launch_crt_512};

}  // namespace mr
