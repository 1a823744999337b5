// Registry of the compiled size classes. Generated by gen_kernels.py.
#include "kernels_api.h"

namespace mr {

extern const ClassKernels kClass512;
extern const ClassKernels kClass1024;
extern const ClassKernels kClass1536;
extern const ClassKernels kClass2048;
extern const ClassKernels kClass3072;
extern const ClassKernels kClass4096;
extern const ClassKernels kClass8192;
extern const ClassKernels kClass16384;

const ClassKernels* class_kernels(uint32_t L) {
  switch (L) {
    case 512:
      return &kClass512;
    case 1024:
      return &kClass1024;
    case 1536:
      return &kClass1536;
    case 2048:
      return &kClass2048;
    case 3072:
      return &kClass3072;
    case 4096:
      return &kClass4096;
    case 8192:
      return &kClass8192;
    case 16384:
      return &kClass16384;
    default:
      return nullptr;
  }
}

}  // namespace mr
