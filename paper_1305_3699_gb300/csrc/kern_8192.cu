// Kernel of the 8192-bit size class (k = 295 channels per base). Generated by gen_kernels.py.
#include "big_kernel.cuh"
#include "kernels_api.h"

namespace mr {

using CB8192 = BigCfg<295, 256, 258, 4, 8>;
static size_t slot_words_8192(uint32_t wbits) { return CB8192::slot_words(wbits); }

static cudaError_t launch_big_8192(const BigArgs& a, cudaStream_t s) {
  void* args[] = {const_cast<BigArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)big_modexp_kernel<CB8192>, dim3(a.slots * CB8192::SLICES),
                                     dim3(CB8192::THREADS), args, CB8192::SMEM_BYTES, s);
}

static cudaError_t prepare_big_8192() {
  return cudaFuncSetAttribute(big_modexp_kernel<CB8192>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB8192::SMEM_BYTES);
}

static int occupancy_big_8192() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big_modexp_kernel<CB8192>, CB8192::THREADS, CB8192::SMEM_BYTES) != cudaSuccess) n = 0;
  return n;
}

static const BigKernel kBig8192 = {CB8192::SC, CB8192::SLICES, CB8192::THREADS, CB8192::SMEM_BYTES, slot_words_8192,
                                 launch_big_8192, prepare_big_8192, occupancy_big_8192};
extern const ClassKernels kClass8192 = {8192, 295, 256, 258, 0, {}, &kBig8192};

}  // namespace mr
