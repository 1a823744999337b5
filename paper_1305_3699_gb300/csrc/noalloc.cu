// Allocation-free exponentiation (mr_modexp_batch_noalloc in include/mr.h).
//
// Some callers cannot allocate device memory at the moment they need an
// exponentiation: an engine that reserved all of the GPU's memory for its own
// pool up front, a latency-bound serving loop that must not hit the CUDA
// allocator (cudaMalloc may synchronise the device, and a pool may have to grow),
// or code that is forbidden from taking allocator locks.  This variant takes
// everything it needs from the caller (inputs, outputs, status bytes) and keeps
// its only scratch -- the per-warp window tables of the fixed-window
// exponentiation -- in one statically sized device array defined below.  It
// builds no work-item array: every item's pointers are derived in the kernel
// from the caller's base pointers and strides, for one modulus per call.
//
// Limits: moduli of at most 2048 bits (the 512..2048-bit size classes), and a
// batch whose window tables fit NOALLOC_SCRATCH_BYTES; larger batches are
// refused with MR_ERR_SIZE and must be split by the caller.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "kernels.cuh"
#include "noalloc.h"

namespace mr {

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / 4];

struct PackedArgs {
  const uint32_t* cls;
  const uint32_t* key;
  const uint32_t* x;
  const uint32_t* e;
  uint32_t* out;
  uint8_t* status;
  uint32_t* scratch;  // device address of g_noalloc_scratch
  uint32_t n, x_stride, e_stride, out_stride, wbits;
};

template <class C>
__global__ void __launch_bounds__(C::THREADS) modexp_packed_kernel(PackedArgs a) {
  extern __shared__ __align__(16) uint32_t smem_raw[];
  Smem<C> sm{smem_raw};
  load_class_smem<C>(sm, a.cls);
  __syncthreads();

  constexpr int NPT = C::NPT, TPI = C::TPI;
  const int lane = threadIdx.x & 31;
  const int t = threadIdx.x % TPI;
  const int item_in_block = threadIdx.x / TPI;
  const uint32_t g_raw = blockIdx.x * C::IPB + item_in_block;
  const bool live = g_raw < a.n;
  const uint32_t g = live ? g_raw : a.n - 1;
  const KeyOff ko = key_offsets(C::K, C::W);
  const uint32_t* key = a.key;
  const uint32_t* x = a.x + (size_t)g * a.x_stride;
  const uint32_t* e = a.e + (size_t)g * a.e_stride;
  uint32_t* out = a.out + (size_t)g * a.out_stride;
  uint32_t* xib = sm.xi(item_in_block);
  uint32_t* xpb = xib + C::KP;
  const int warp_global = (blockIdx.x * C::THREADS + threadIdx.x) >> 5;
  uint32_t* wt = a.scratch + (size_t)warp_global * ((size_t)1 << a.wbits) * (2 * NPT) * 32;

  uint32_t bad = 0;
  if (t == 0) bad = less_than(x, a.x_stride, key + ko.N, C::W) ? 0u : 1u;
  bad = __shfl_sync(0xffffffffu, bad, lane - t);

  uint32_t kxp[NPT], kxs[NPT], cmul[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    kxp[s] = o < C::K ? __ldg(key + ko.kxp + o) : 0u;
    kxs[s] = o < C::K ? __ldg(key + ko.kxs + o) : 0u;
    cmul[s] = o < C::K ? __ldg(key + ko.cmul + o) : 0u;
  }

  // x < N, so one chunk of W limbs holds it: x~ = MM(x, M^2 mod N)
  uint32_t xb[NPT], xp[NPT], yb[NPT], yp[NPT];
  const int nl0 = bad ? 0 : (int)(a.x_stride < (uint32_t)C::W ? a.x_stride : C::W);
  to_rns<C>(xb, xp, x, nl0, a.cls, sm, t);
  load_vec<C>(yb, yp, key + ko.r2, t);
  mont_mul<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t);

  const int wb = (int)a.wbits, E = 1 << wb;
  load_vec<C>(yb, yp, key + ko.one, t);
  tab_store<C>(wt, 0, yb, yp, lane);
  tab_store<C>(wt, 1, xb, xp, lane);
  {
    uint32_t cb[NPT], cp[NPT];
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      cb[s] = xb[s];
      cp[s] = xp[s];
    }
    for (int j = 2; j < E; j++) {
      mont_mul<C>(cb, cp, xb, xp, kxp, kxs, cmul, sm, xib, xpb, t);
      tab_store<C>(wt, j, cb, cp, lane);
    }
  }

  uint32_t ebits = 0;
  if (t == 0) ebits = bad ? 0u : exp_bits(e, a.e_stride);
  ebits = __shfl_sync(0xffffffffu, ebits, lane - t);
  const uint32_t nwin = __reduce_max_sync(0xffffffffu, (ebits + wb - 1) / wb);
  uint32_t d = (nwin && !bad) ? exp_digit(e, a.e_stride, (nwin - 1) * wb, wb) : 0u;
  __syncwarp();
  tab_load<C>(wt, d, xb, xp, lane);
  for (int widx = (int)nwin - 2; widx >= 0; widx--) {
    for (int q = 0; q < wb; q++) mont_mul<C>(xb, xp, xb, xp, kxp, kxs, cmul, sm, xib, xpb, t);
    d = bad ? 0u : exp_digit(e, a.e_stride, (uint32_t)widx * wb, wb);
    if (__any_sync(0xffffffffu, d != 0)) {
      tab_load<C>(wt, d, yb, yp, lane);
      mont_mul<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t);
    }
  }

#pragma unroll
  for (int s = 0; s < NPT; s++) {
    yb[s] = sm.cb4(t, s).z;
    yp[s] = sm.cp4(t, s).z;
  }
  mont_mul<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t);
  from_rns_reduce<C>(xb, a.cls, key, sm, xib, t, out, (int)a.out_stride, live && !bad);
  if (live && t == 0) {
    if (bad)
      for (uint32_t w = 0; w < a.out_stride; w++) out[w] = 0u;
    if (a.status) a.status[g] = bad ? 5u : 0u;
  }
}

namespace {

std::mutex g_mu;
std::map<int, uint32_t*> g_scratch_addr;  // device ordinal -> device address of g_noalloc_scratch
std::map<std::pair<int, int>, bool> g_smem_set;  // (device, channels per base) -> shared-memory limit raised

// Device address of the static scratch array on the current device (looked up once per device).
cudaError_t scratch_address(int device, uint32_t** out) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_scratch_addr.find(device);
  if (it != g_scratch_addr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[device] = static_cast<uint32_t*>(p);
  *out = static_cast<uint32_t*>(p);
  return cudaSuccess;
}

// Raise the kernel's dynamic shared-memory limit on the current device (a per-device setting: done
// once per device and class; a failure is not remembered, the next call tries again).
template <class C>
cudaError_t prepare_packed(int device) {
  std::lock_guard<std::mutex> g(g_mu);
  const auto key = std::make_pair(device, C::K);
  if (g_smem_set.count(key)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(modexp_packed_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       C::SMEM_BYTES);
  if (e == cudaSuccess) g_smem_set[key] = true;
  return e;
}

template <class C>
int launch_packed(const NoallocCall& c, std::string& err) {
  // window tables: one per warp of the grid, 2^w entries of 2 NPT words per lane
  const size_t per_block = (size_t)(C::THREADS / 32) * ((size_t)1 << c.wbits) * 2 * C::NPT * 32 * 4;
  const size_t grid = (c.n + C::IPB - 1) / C::IPB;
  if (grid * per_block > NOALLOC_SCRATCH_BYTES) {
    const size_t max_items = NOALLOC_SCRATCH_BYTES / per_block * C::IPB;
    err = "batch needs " + std::to_string(grid * per_block) +
          " bytes of window tables; the allocation-free entry point has " + std::to_string(NOALLOC_SCRATCH_BYTES) +
          " (at most " + std::to_string(max_items) + " items of this modulus size and exponent stride): split the batch";
    return 4;  // MR_ERR_SIZE
  }
  uint32_t* scratch = nullptr;
  cudaError_t e = scratch_address(c.device, &scratch);
  if (e != cudaSuccess) {
    err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return 7;  // MR_ERR_CUDA
  }
  if ((e = prepare_packed<C>(c.device)) != cudaSuccess) {
    err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
    return 7;
  }
  PackedArgs a{c.cls, c.key, c.x, c.e, c.out, c.status, scratch, c.n, c.x_stride, c.e_stride, c.out_stride, c.wbits};
  modexp_packed_kernel<C><<<(unsigned)grid, C::THREADS, C::SMEM_BYTES, c.stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return 7;
  }
  return 0;
}

}  // namespace

int noalloc_modexp(const NoallocCall& c, std::string& err) {
  switch (c.class_bits) {
    case 512:
      return launch_packed<Cfg<18, 16, 17, 2, 128, 4>>(c, err);
    case 1024:
      return launch_packed<Cfg<36, 32, 34, 4, 128, 4>>(c, err);
    case 1536:
      return launch_packed<Cfg<54, 48, 50, 8, 128, 4>>(c, err);
    case 2048:
      return launch_packed<Cfg<72, 64, 66, 8, 128, 4>>(c, err);
    default:
      err = "the allocation-free entry point handles moduli of at most 2048 bits";
      return 4;  // MR_ERR_SIZE
  }
}

}  // namespace mr
