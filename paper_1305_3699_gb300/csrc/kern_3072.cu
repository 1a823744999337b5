// Kernels of the 3072-bit size class (k = 108 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C3072v0 = Cfg<108, 96, 97, 16, 256, 4>;
static cudaError_t launch_modexp_3072_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(modexp_kernel<C3072v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072v0::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  modexp_kernel<C3072v0><<<grid, C3072v0::THREADS, C3072v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_3072_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(crt_kernel<C3072v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072v0::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  crt_kernel<C3072v0><<<grid, C3072v0::THREADS, C3072v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_3072_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(mr_kernel<C3072v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072v0::SMEM_BYTES);
  if (attr != cudaSuccess) return attr;
  mr_kernel<C3072v0><<<grid, C3072v0::THREADS, C3072v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

extern const ClassKernels kClass3072 = {
    3072, 108, 96, 97, 1,
    {
     {C3072v0::TPI, C3072v0::THREADS, C3072v0::IPB, C3072v0::NPT, C3072v0::SMEM_BYTES, launch_modexp_3072_0, launch_crt_3072_0, launch_mr_3072_0}}};

}  // namespace mr
