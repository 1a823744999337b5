// Kernels of the 1536-bit size class (k = 54 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C1536v0 = Cfg<54, 48, 50, 8, 256, 4, 2, 1>;
static cudaError_t launch_modexp_1536_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C1536v0><<<grid, C1536v0::THREADS, C1536v0::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1536_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C1536v0><<<grid, C1536v0::THREADS, C1536v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_1536_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C1536v0><<<grid, C1536v0::THREADS, C1536v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_1536_0() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C1536v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v0::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C1536v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v0::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C1536v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v0::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_1536_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C1536v0>, C1536v0::THREADS, C1536v0::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C1536v1 = Cfg<54, 48, 50, 8, 128, 4, 0, 0>;
static cudaError_t launch_modexp_1536_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C1536v1><<<grid, C1536v1::THREADS, C1536v1::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_1536_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C1536v1><<<grid, C1536v1::THREADS, C1536v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_1536_1(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C1536v1><<<grid, C1536v1::THREADS, C1536v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_1536_1() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C1536v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v1::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C1536v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v1::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C1536v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C1536v1::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_1536_1() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C1536v1>, C1536v1::THREADS, C1536v1::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

extern const ClassKernels kClass1536 = {
    1536, 54, 48, 50, 2,
    {
     {C1536v0::TPI, C1536v0::THREADS, C1536v0::IPB, C1536v0::NPT, C1536v0::SMEM_MODEXP_BYTES, C1536v0::TC, launch_modexp_1536_0, launch_crt_1536_0, launch_mr_1536_0, prepare_1536_0, occupancy_1536_0},
     {C1536v1::TPI, C1536v1::THREADS, C1536v1::IPB, C1536v1::NPT, C1536v1::SMEM_MODEXP_BYTES, C1536v1::TC, launch_modexp_1536_1, launch_crt_1536_1, launch_mr_1536_1, prepare_1536_1, occupancy_1536_1}},
    nullptr, 0};

}  // namespace mr
