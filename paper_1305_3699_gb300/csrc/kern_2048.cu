// Kernels of the 2048-bit size class (k = 72 channels per base). Generated by gen_kernels.py.
#include "kernels.cuh"
#include "kernels_api.h"
#include "mr_kernel.cuh"

namespace mr {

using C2048v0 = Cfg<72, 64, 66, 8, 256, 4, 1, 1>;
static cudaError_t launch_modexp_2048_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C2048v0><<<grid, C2048v0::THREADS, C2048v0::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_2048_0(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C2048v0><<<grid, C2048v0::THREADS, C2048v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_2048_0(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C2048v0><<<grid, C2048v0::THREADS, C2048v0::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_2048_0() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C2048v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v0::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C2048v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v0::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C2048v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v0::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_2048_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C2048v0>, C2048v0::THREADS, C2048v0::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C2048v1 = Cfg<72, 64, 66, 8, 128, 4, 0, 0>;
static cudaError_t launch_modexp_2048_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C2048v1><<<grid, C2048v1::THREADS, C2048v1::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_2048_1(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C2048v1><<<grid, C2048v1::THREADS, C2048v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_2048_1(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C2048v1><<<grid, C2048v1::THREADS, C2048v1::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_2048_1() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C2048v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v1::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C2048v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v1::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C2048v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v1::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_2048_1() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C2048v1>, C2048v1::THREADS, C2048v1::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

using C2048v2 = Cfg<72, 64, 66, 16, 128, 4, 1, 0>;
static cudaError_t launch_modexp_2048_2(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  modexp_kernel<C2048v2><<<grid, C2048v2::THREADS, C2048v2::SMEM_MODEXP_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_crt_2048_2(const LaunchArgs& a, unsigned grid, cudaStream_t s) {
  crt_kernel<C2048v2><<<grid, C2048v2::THREADS, C2048v2::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t launch_mr_2048_2(const MRArgs& a, unsigned grid, cudaStream_t s) {
  mr_kernel<C2048v2><<<grid, C2048v2::THREADS, C2048v2::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

static cudaError_t prepare_2048_2() {
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncSetAttribute(modexp_kernel<C2048v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v2::SMEM_MODEXP_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(crt_kernel<C2048v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v2::SMEM_BYTES)) != cudaSuccess) e = r;
  if ((r = cudaFuncSetAttribute(mr_kernel<C2048v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C2048v2::SMEM_BYTES)) != cudaSuccess) e = r;
  return e;
}

static int occupancy_2048_2() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, modexp_kernel<C2048v2>, C2048v2::THREADS, C2048v2::SMEM_MODEXP_BYTES) != cudaSuccess) n = 1;
  return n > 0 ? n : 1;
}

extern const ClassKernels kClass2048 = {
    2048, 72, 64, 66, 3,
    {
     {C2048v0::TPI, C2048v0::THREADS, C2048v0::IPB, C2048v0::NPT, C2048v0::SMEM_MODEXP_BYTES, C2048v0::TC, launch_modexp_2048_0, launch_crt_2048_0, launch_mr_2048_0, prepare_2048_0, occupancy_2048_0},
     {C2048v1::TPI, C2048v1::THREADS, C2048v1::IPB, C2048v1::NPT, C2048v1::SMEM_MODEXP_BYTES, C2048v1::TC, launch_modexp_2048_1, launch_crt_2048_1, launch_mr_2048_1, prepare_2048_1, occupancy_2048_1},
     {C2048v2::TPI, C2048v2::THREADS, C2048v2::IPB, C2048v2::NPT, C2048v2::SMEM_MODEXP_BYTES, C2048v2::TC, launch_modexp_2048_2, launch_crt_2048_2, launch_mr_2048_2, prepare_2048_2, occupancy_2048_2}},
    nullptr, 0};

}  // namespace mr
