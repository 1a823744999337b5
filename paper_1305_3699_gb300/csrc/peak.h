// Host interface of the integer-multiply throughput probe (peak.cu) behind mr_imad_peak.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mr {
// Multiply-adds per second of a dependent-free stream on `device`: kind 0 mad.wide.u32
// (32x32 -> 64-bit product added to a 64-bit accumulator), 1 mad.lo.u32, 2 the same 64-bit
// accumulation as a carry pair (mad.lo.cc.u32 + madc.hi.u32; products per second), 3 mad.hi.u32.
cudaError_t imad_stream_rate(int device, cudaStream_t stream, int kind, double* per_second);
// Tensor-core operations (2 per multiply-add) per second: kind 0 tcgen05 kind::f16, 1 mma.sync s8,
// 2 mma.sync f16 (tc_peak.cu).  cudaErrorLaunchTimeout when a probe's bounded wait ran out.
cudaError_t tensor_rate(int device, cudaStream_t stream, int kind, double* per_second);
// One 128 x n x kdim fp16 product through tcgen05 with the operand layout of tc_device.cuh.
cudaError_t tensor_debug_mma(const uint16_t* a_host, const uint16_t* b_host, uint32_t n, uint32_t kdim,
                             uint32_t swap_strides, float* d_host, cudaStream_t stream);
}  // namespace mr
