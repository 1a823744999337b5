// Kernel of the 8192-bit size class (k = 295 channels per base). Generated by gen_kernels.py.
#include "big_kernel.cuh"
#include "kernels_api.h"

namespace mr {

using CB8192v0 = BigCfg<295, 256, 258, 4, 8>;
static size_t slot_words_8192_0(uint32_t wbits) { return CB8192v0::slot_words(wbits); }

static cudaError_t launch_big_8192_0(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB8192v0>, dim3(a.slots * CB8192v0::SLICES),
                                     dim3(CB8192v0::THREADS), args, CB8192v0::SMEM_BYTES, s);
}

static cudaError_t prepare_big_8192_0() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB8192v0>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB8192v0::SMEM_BYTES);
}

static int occupancy_big_8192_0() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB8192v0>, CB8192v0::THREADS, CB8192v0::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

using CB8192v1 = BigCfg<295, 256, 258, 4, 12>;
static size_t slot_words_8192_1(uint32_t wbits) { return CB8192v1::slot_words(wbits); }

static cudaError_t launch_big_8192_1(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB8192v1>, dim3(a.slots * CB8192v1::SLICES),
                                     dim3(CB8192v1::THREADS), args, CB8192v1::SMEM_BYTES, s);
}

static cudaError_t prepare_big_8192_1() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB8192v1>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB8192v1::SMEM_BYTES);
}

static int occupancy_big_8192_1() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB8192v1>, CB8192v1::THREADS, CB8192v1::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

using CB8192v2 = BigTcCfg<295, 256, 258>;
static size_t slot_words_8192_2(uint32_t wbits) { return CB8192v2::slot_words(wbits); }

static cudaError_t launch_big_8192_2(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB8192v2>, dim3(a.slots * CB8192v2::SLICES),
                                     dim3(CB8192v2::THREADS), args, CB8192v2::SMEM_BYTES, s);
}

static cudaError_t prepare_big_8192_2() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB8192v2>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB8192v2::SMEM_BYTES);
}

static int occupancy_big_8192_2() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB8192v2>, CB8192v2::THREADS, CB8192v2::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

static const BigKernel kBig8192[3] = {
    {CB8192v0::SC, CB8192v0::SLICES, CB8192v0::THREADS, CB8192v0::SMEM_BYTES, 0, 1.000f, slot_words_8192_0, launch_big_8192_0, prepare_big_8192_0, occupancy_big_8192_0},
    {CB8192v1::SC, CB8192v1::SLICES, CB8192v1::THREADS, CB8192v1::SMEM_BYTES, 0, 1.330f, slot_words_8192_1, launch_big_8192_1, prepare_big_8192_1, occupancy_big_8192_1},
    {CB8192v2::SC, CB8192v2::SLICES, CB8192v2::THREADS, CB8192v2::SMEM_BYTES, 1, 0.495f, slot_words_8192_2, launch_big_8192_2, prepare_big_8192_2, occupancy_big_8192_2}};
extern const ClassKernels kClass8192 = {8192, 295, 256, 258, 0, {}, kBig8192, 3};

}  // namespace mr
