// Host interface of the allocation-free exponentiation (noalloc.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

namespace mr {

// Size of the static device scratch array that holds the window tables.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;

struct NoallocCall {
  int device;                 // ordinal of the current device
  uint32_t class_bits;        // size class of the modulus (512..2048)
  const uint32_t* cls;        // class table block (device)
  const uint32_t* key;        // modulus block (device)
  const uint32_t* x;          // device, n rows of x_stride limbs
  const uint32_t* e;          // device, n rows of e_stride limbs
  uint32_t* out;              // device, n rows of out_stride limbs
  uint8_t* status;            // device, n bytes, or nullptr
  uint32_t n, x_stride, e_stride, out_stride, wbits;
  cudaStream_t stream;
};

// Launch; returns an mr_status code (0 = ok) and a message in err on failure.
// The first call on a device looks up the device address of the static scratch.
int noalloc_modexp(const NoallocCall& c, std::string& err);

}  // namespace mr
