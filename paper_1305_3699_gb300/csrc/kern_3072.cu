// Kernels of the 3072-bit size class (k = 108 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C3072v0 = Cfg<108, 96, 97, 16, 256, 4, 0, 0>;
static cudaError_t launch_modexp_3072_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C3072v0><<<grid, C3072v0::THREADS, C3072v0::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_3072_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C3072v0><<<grid, C3072v0::THREADS, C3072v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_3072_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C3072v0><<<grid, C3072v0::THREADS, C3072v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_3072_0() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C3072v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072v0::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C3072v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072v0::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C3072v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C3072v0::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_3072_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C3072v0>, C3072v0::THREADS, C3072v0::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

extern const ClassKernels kClass3072 = {
    3072, 108, 96, 97, 1,
    {
     {C3072v0::TPI, C3072v0::THREADS, C3072v0::IPB, C3072v0::NPT, C3072v0::SMEM_MODEXP_BYTES, C3072v0::TC, launch_modexp_3072_0, launch_crt_3072_0, launch_mr_3072_0, prepare_3072_0, occupancy_3072_0}},
    nullptr, 0};

}  // namespace mr
