// Host interface of the integer-multiply throughput probe (peak.cu) behind mr_imad_peak.
#pragma once
#include <cuda_runtime.h>

namespace mr {
// Multiply-adds per second of a dependent-free stream on `device`: wide = mad.wide.u32
// (32x32 -> 64-bit product added to a 64-bit accumulator), else mad.lo.u32.
cudaError_t imad_stream_rate(int device, cudaStream_t stream, bool wide, double* per_second);
}  // namespace mr
