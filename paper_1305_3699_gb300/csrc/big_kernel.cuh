// Exponentiation kernel of the large size classes (8192 and 16384 bits, k = 295
// and 599 channels per base): the same RNS Montgomery multiplication and
// fixed-window loop as the lane-group kernel (Sec. 3.1), spread over several
// CTAs because one number's channels no longer fit one warp.
//
// Mapping.  Numbers are taken 32 at a time ("item group"; lane = number).  The
// 2k channels of a group are split into SLICES channel slices of SC = NW * NPT
// channels of each base; CTA (slot, slice) owns one slice, warp w of it the NPT
// channels [slice*SC + w*NPT, +NPT) of B and of B' for the 32 numbers.  Residues
// stay in registers; the CTA's columns of both extension matrices stay in
// shared memory for the whole launch.  The two base extensions exchange the
// CRT coefficients xi / xi' of all channels through a per-slot buffer in global
// memory (L2-resident): every CTA writes its slice, the CTAs of the slot meet at
// a barrier, and each CTA brings the k rows into shared memory in thirds with
// bulk copies (cp.async.bulk, completion on an mbarrier) into two buffers, the
// copy of the next third overlapping the dot products of the current one.  The
// fixed-point correction factor is summed from one partial per slice.  Two
// barriers per multiplication.
//
// The CTAs of a slot wait on one another, so the kernel is started as one
// cooperative launch (every CTA resident).  Each barrier wait is bounded: on
// timeout the kernel raises an abort flag that every waiting CTA sees, marks
// the unfinished items MR_ERR_TIMEOUT and returns.
#pragma once
#include <cstdint>

#include "kernels.cuh"
#include "kernels_api.h"
#include "rns_device.cuh"
#include "tc_device.cuh"

namespace mr {

template <int K_, int W_, int WX_, int NPT_, int NW_>
struct BigCfg {
  static constexpr bool TC = false;                   // base extensions on the integer pipe
  static constexpr int K = K_, W = W_, WX = WX_, NPT = NPT_, NW = NW_;
  static constexpr int SC = NPT * NW;                 // channels per slice and base
  static constexpr int SLICES = (K + SC - 1) / SC;
  static constexpr int THREADS = NW * 32;
  static constexpr int R = (K + 2) / 3;              // rows per staged third of xi
  // shared memory (words)
  static constexpr int SM_T1 = 0;                     // [K][SC] this slice's columns of T1
  static constexpr int SM_T2 = SM_T1 + K * SC;        // [K][SC] of T2
  static constexpr int SM_X = SM_T2 + K * SC;         // 2 x [R][32] staged xi rows (double buffer)
  static constexpr int SM_C4A = SM_X + 2 * R * 32;    // per slot uint4 {m, mi, r32, E}   B  (E = -M' 2^64 mod m)
  static constexpr int SM_C4B = SM_C4A + 4 * SC;      // per slot uint4 {m, mi, r32, ahat} B'
  static constexpr int SM_C2A = SM_C4B + 4 * SC;      // per slot uint2 {mmiinv, ub}       B
  static constexpr int SM_C2B = SM_C2A + 2 * SC;      // per slot uint2 {ad, ubp}          B'
  static constexpr int SM_KAW = SM_C2B + 2 * SC;      // [NW][32] correction-factor partials
  static constexpr int SM_MISC = SM_KAW + NW * 32;    // [32]
  static constexpr int SM_MBAR = SM_MISC + 32;        // two mbarriers (8 bytes each) of the staging copies
  static constexpr int SM_WORDS = SM_MBAR + 4;
  static constexpr int SMEM_BYTES = SM_WORDS * 4;
  // per-slot global scratch (words): xi, xi', slice partials, then the window table
  static constexpr size_t XG = 0, XPG = (size_t)K * 32, KAWG = (size_t)2 * K * 32;
  static constexpr size_t KAWX = KAWG;  // slice partials of the exit conversion (barriers separate the uses)
  static constexpr size_t TAB = KAWG + (size_t)SLICES * 32;
  MR_HD static constexpr size_t slot_words(uint32_t wbits) { return TAB + ((size_t)1 << wbits) * 2 * K * 32; }
  static_assert(NPT == 4, "four channels per thread and base (one 16-byte matrix load per row)");
  static_assert((SM_X % 4) == 0 && (SM_C4A % 4) == 0 && (SC % 4) == 0 && (SM_MBAR % 4) == 0, "alignment");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
  static_assert(K * 32 <= 2 * K * SC, "RNS -> binary stages all k rows in the matrix area");
};

// Tensor-core form of the same kernel.  The two base extensions of a slice's CTA are the product
// D (32 numbers x 32 channels) = X (32 x k) T (k x 32) of the CRT coefficients with its columns of
// the class's extension matrix, every entry below 2^28 and the exact sum below 2^64.  Both factors
// are split into four 7-bit slices, X = sum_a 2^(7a) X_a and T = sum_b 2^(7b) T_b, and multiplied on
// the tensor cores in fp16 with fp32 accumulation: every entry of a slice product is a sum of k
// products below 127^2, exact in fp32 for k <= 1040, and the recombination
// sum_{a,b} 2^(7(a+b)) X_a T_b is exact in 64 bits.  The data slices form a 128 x k operand, row
// 32a + n, written by the slot's CTAs (each its 32 channels, in the shared-memory operand layout of
// tc_device.cuh) into a per-slot buffer in global memory; the matrix slices form a k x 128 operand,
// row 32b + j, of a class table in the same layout.  The first extension's matrix slices stay in
// tensor memory for the whole launch (the A operand, columns TM_T1 ..; the product is
// D^T = T1^T X^T, accumulator row 32b + j, column 32a + n), so that extension streams only the
// data; the second streams data and T2 chunks (D = X T2, accumulator row 32a + n, column 32b + j).
// A block publishes its slices of a data operand with a release increment of that chunk's counter
// (two blocks write each chunk of 64 columns); the copy of a data chunk waits (acquire) for its
// counter to reach the multiplication's target, so the chunks of early blocks stream while the last
// ones are still being written, and no slot barrier separates the multiplications' exchanges.  Every
// extension reads every chunk, so a block that has passed an extension knows that all blocks have
// finished the previous one (the buffers' reuse is ordered without a barrier).
// Everything streamed passes through a ring of STAGES 16 KB shared-memory stages (64 columns of k
// of one operand each) filled by bulk copies completing on mbarriers, one copy thread per stage:
// the stream is bound by the round trip of a stage (copy latency from L2 plus the products), so
// the ring is as deep as shared memory allows.  Thread 0 waits for each chunk and issues its tcgen05
// products (128 x 128 x 16 each) into a 128-column accumulator; the tensor core's completion frees
// the stages.  The epilogue reads the accumulator back, combines the slices through shared memory
// (aliasing the idle ring) and hands every thread the same 64-bit dot products the integer form
// computes.
// Everything else is the integer kernel's.
template <int K_, int W_, int WX_>
struct BigTcCfg {
  static constexpr bool TC = true;
  static constexpr int K = K_, W = W_, WX = WX_, NPT = 4, NW = 8;
  static constexpr int SC = NPT * NW;                 // 32 channels per slice and base
  static constexpr int SLICES = (K + SC - 1) / SC;
  static constexpr int THREADS = NW * 32;
  static constexpr int KC = 64;                       // columns of k per staged chunk
  static constexpr int NCH = (K + KC - 1) / KC;       // chunks per operand
  static constexpr int KP = NCH * KC;                 // padded k
  static constexpr int STAGES = 14;                   // ring stages of one operand chunk each
  static constexpr uint32_t CHUNK_BYTES = 128u * KC * 2u;  // one operand chunk: 128 rows x 64 fp16
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr uint32_t TM_T1 = 128;              // first tensor-memory column of the resident T1 slices
  static constexpr int EX_LS = 17;                    // second-extension exchange: 64-bit words per lane
  static constexpr int EX1_LS = 33;                   // first-extension exchange: 32-bit words per row
  // shared memory (words)
  static constexpr int SM_RING = 0;                   // STAGES operand chunks
  static constexpr int SM_T1 = SM_RING;               // staging of the RNS -> binary conversion
  static constexpr int SM_EX = SM_RING;               // exchange buffers of the epilogues (ring, idle then)
  static constexpr int SM_C4A = SM_RING + STAGES * (int)CHUNK_BYTES / 4;
  static constexpr int SM_C4B = SM_C4A + 4 * SC;
  static constexpr int SM_C2A = SM_C4B + 4 * SC;
  static constexpr int SM_C2B = SM_C2A + 2 * SC;
  static constexpr int SM_KAW = SM_C2B + 2 * SC;
  static constexpr int SM_MISC = SM_KAW + NW * 32;
  static constexpr int SM_MBAR = SM_MISC + 32;        // full[S], empty[S], done (8 bytes each)
  static constexpr int SM_TMEM = SM_MBAR + 2 * (2 * STAGES + 1);
  static constexpr int SM_PH = SM_TMEM + 4;           // phase counters: BIG_PHASES sums, last time stamp (u64)
  static constexpr int SM_WORDS = SM_PH + 2 * (BIG_PHASES + 1);
  static constexpr int SMEM_BYTES = SM_WORDS * 4;
  // per-slot global scratch (words): the data operands of the two extensions, the plain CRT
  // coefficients of the exit conversion, slice partials, then the window table
  static constexpr size_t AOP_WORDS = (size_t)NCH * CHUNK_BYTES / 4;
  static constexpr size_t AG1 = 0, AG2 = AOP_WORDS, XG = 2 * AOP_WORDS, KAWG = XG + (size_t)K * 32;
  // the exit conversion's slice partials: a buffer of their own, since no barrier separates them from the
  // last multiplication's partials, which slower blocks may still be reading
  static constexpr size_t KAWX = KAWG + (size_t)SLICES * 32;
  static constexpr size_t TAB = KAWX + (size_t)SLICES * 32;
  MR_HD static constexpr size_t slot_words(uint32_t wbits) { return TAB + ((size_t)1 << wbits) * 2 * K * 32; }
  // class table: [slice][extension][chunk] operand chunks of the matrix slices
  static constexpr size_t BTAB_BYTES = (size_t)2 * SLICES * NCH * CHUNK_BYTES;
  static_assert(K * 32 <= SM_C4A, "RNS -> binary staging fits the ring");
  static_assert(4 * 2 * 32 * EX_LS * 2 <= SM_C4A, "second exchange fits the ring");
  static_assert(2 * 4 * 32 * EX1_LS <= SM_C4A, "first exchange fits the ring");
  static_assert(TM_T1 + KP / 2 <= TMEM_COLS, "accumulator and resident T1 fit tensor memory");
  static_assert(SLICES * SC <= KP, "every slice's columns lie inside the padded operand");
  static_assert((SM_MBAR % 2) == 0 && (SM_C4A % 4) == 0 && (SM_PH % 2) == 0, "alignment");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
  static_assert(K <= 1040, "7-bit slices: k * 127^2 < 2^24 keeps every fp32 partial sum exact");
  static_assert(STAGES <= 32, "copy threads are lanes of warp 1");
  static_assert(2 * NCH <= (int)BIG_FLAG_WORDS, "chunk-ready counters");
  // blocks (channel slices) writing chunk c of a data operand: slices 2c and 2c + 1
  __device__ static constexpr uint32_t producers(int c) { return SLICES - 2 * c >= 2 ? 2u : 1u; }
};

template <class C>
struct BigGroup {
  uint32_t* s;         // shared memory
  uint32_t* slot;      // this slot's global scratch
  uint32_t* ctr;       // this slot's barrier counter
  uint32_t* abort;     // launch-wide abort flag
  uint32_t* flags;     // tensor-core form: this slot's chunk-ready counters [extension][chunk]
  uint32_t nmul;       // tensor-core form: multiplications started by this block
  uint32_t nbar;       // barriers passed so far (target = nbar * SLICES)
  uint32_t spin_limit; // polls before a wait gives up
  uint32_t ph;         // parity bits of the two staging mbarriers
  uint32_t chunk;      // tensor-core form: operand chunks staged so far (ring position and parities)
  uint32_t done_ph;    // tensor-core form: parity of the accumulator-complete mbarrier
  const uint8_t* btab; // tensor-core form: this slice's B operand chunks [extension][chunk]
  uint32_t stag;       // tensor-core form: first chunk of k this block streams (the order is rotated per
                       // block so that blocks sharing an operand do not read the same chunk at once)
  unsigned long long* phases;  // tensor-core form: phase counters of the launch, or nullptr
  int c, w, lane;
  // Phase counters: thread 0 closes the interval since the previous mark into phase i.
  __device__ __forceinline__ void mark(int i) {
    if constexpr (C::TC) {
      if (phases && threadIdx.x == 0) {
        unsigned long long* ph = reinterpret_cast<unsigned long long*>(s + C::SM_PH);
        const unsigned long long t = clock64();
        ph[i] += t - ph[BIG_PHASES];
        ph[BIG_PHASES] = t;
      }
    }
  }
  __device__ uint4 a4(int q) const { return reinterpret_cast<const uint4*>(s + C::SM_C4A)[q]; }
  __device__ uint4 b4(int q) const { return reinterpret_cast<const uint4*>(s + C::SM_C4B)[q]; }
  __device__ uint2 a2(int q) const { return reinterpret_cast<const uint2*>(s + C::SM_C2A)[q]; }
  __device__ uint2 b2(int q) const { return reinterpret_cast<const uint2*>(s + C::SM_C2B)[q]; }

  // All CTAs of the slot meet; false when the wait ran out or another CTA aborted.
  __device__ bool barrier();

};

// acc[s] += sum_{i in [r0, r1)} X[i - r0][lane] * T[i][w*NPT + s]   (X rows relative to r0)
template <class C>
__device__ __forceinline__ void big_dot(uint64_t (&acc)[C::NPT], const uint32_t* X, const uint32_t* T, int r0, int r1,
                                        int w, int lane) {
  const uint32_t* xr = X + lane;
  const uint32_t* tr = T + w * C::NPT;
#pragma unroll 8
  for (int i = r0; i < r1; i++) {
    const uint32_t x = xr[(i - r0) * 32];
    const uint4 t = *reinterpret_cast<const uint4*>(tr + i * C::SC);
    acc[0] = madw(x, t.x, acc[0]);
    acc[1] = madw(x, t.y, acc[1]);
    acc[2] = madw(x, t.z, acc[2]);
    acc[3] = madw(x, t.w, acc[3]);
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One elected thread: copy `bytes` (a multiple of 16) of global memory to shared memory with the
// tensor-memory-access unit; completion is counted on `mbar`.  The fences order this thread's view
// of earlier generic accesses (the other blocks' stores seen through the slot barrier, this block's
// reads of the buffer) before the asynchronous copy.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

// Wait for phase `parity` of `mbar` to complete; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; it++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One extension's dot products over all k rows of a global xi buffer: the rows arrive in three
// bulk copies into two shared-memory buffers, the copy of the next third overlapping the dot
// products of the current one.  False (abort raised) when a copy does not complete in time.
template <class C>
__device__ bool big_ext(uint64_t (&acc)[C::NPT], BigGroup<C>& g, const uint32_t* src, const uint32_t* T) {
  constexpr int R = C::R;
  uint32_t* const buf0 = g.s + C::SM_X;
  uint32_t* const buf1 = buf0 + R * 32;
  uint64_t* const mb = reinterpret_cast<uint64_t*>(g.s + C::SM_MBAR);
  if (threadIdx.x == 0) bulk_copy_g2s(buf0, src, (uint32_t)min(R, C::K) * 128u, &mb[0]);
  for (int t = 0; t < 3; t++) {
    const int r0 = t * R, r1 = min(C::K, r0 + R);
    if (t < 2 && threadIdx.x == 0) {
      const int n0 = r1, n1 = min(C::K, n0 + R);
      if (n1 > n0) bulk_copy_g2s((t & 1) ? buf0 : buf1, src + (size_t)n0 * 32, (uint32_t)(n1 - n0) * 128u, &mb[(t + 1) & 1]);
    }
    const int b = t & 1;
    bool ok = r1 <= r0 || mbar_wait(&mb[b], (g.ph >> b) & 1u, g.spin_limit);
    if (r1 > r0) g.ph ^= 1u << b;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(g.abort, 1u);
        // the copy of the next third may still be in flight: give it a bounded chance to land
        if (t < 2) mbar_wait(&mb[(t + 1) & 1], (g.ph >> ((t + 1) & 1)) & 1u, g.spin_limit);
      }
      __syncthreads();
      return false;
    }
    if (r1 > r0) big_dot<C>(acc, b ? buf1 : buf0, T, r0, r1, g.w, g.lane);
    __syncthreads();  // the buffer is refilled by the copy issued in the next iteration
  }
  return true;
}

// Tensor-core form: this thread's four CRT coefficients (channels o0 .. o0+3 of number `lane`) as four
// 7-bit fp16 slices into the A operand `aop` of an extension: row 32a + lane, columns o0 .. o0+3 of
// slice a (one 8-byte store per slice; o0 is a multiple of 4).
template <class C>
__device__ __forceinline__ void tc_put_slices(uint8_t* aop, const uint32_t (&v)[4], int o0, int lane) {
  uint8_t* chunk = aop + (size_t)(o0 / C::KC) * C::CHUNK_BYTES;
  const uint32_t col = (uint32_t)(o0 % C::KC);
#pragma unroll
  for (int a = 0; a < 4; a++) {
    uint32_t h[4];
#pragma unroll
    for (int s = 0; s < 4; s++) h[s] = __half_as_ushort(__uint2half_rn((v[s] >> (7 * a)) & 127u));
    const uint2 pk = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    *reinterpret_cast<uint2*>(chunk + tc::tile_off(128, 32u * a + lane, col)) = pk;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) completing on `mbar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

// Copy threads: lanes 0 .. STAGES - 1 of warp 1; lane st copies every operand chunk that lands in
// stage st, completing on that stage's mbarrier.  A stage's copy thread alone refills it, so it never
// runs more than one mbarrier phase ahead.  Returns the stage, or -1.
template <class C>
__device__ __forceinline__ int tc_copier() {
  return (threadIdx.x >= 32 && threadIdx.x < 32 + C::STAGES) ? (int)threadIdx.x - 32 : -1;
}

// The unit (operand chunk) of the extension starting at ring position g0 that is the first to land in
// stage st.
template <class C>
__device__ __forceinline__ int tc_first_unit(uint32_t g0, int st) {
  return (st - (int)(g0 % C::STAGES) + C::STAGES) % C::STAGES;
}

// Tensor-core form: publish this block's slices of the data operand of extension e (every thread has
// stored its part; the counter of the chunk they lie in is raised with release semantics).  The proxy
// fences make each thread's generic stores visible to the copy engines (async proxy) of the readers,
// and order its generic accesses to the ring before the copies that refill it.
template <class C>
__device__ __forceinline__ void tc_publish(BigGroup<C>& g, int e) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  // and this thread's generic accesses to the ring (epilogue exchanges) before the next copies into it
  tc::fence_smem_async();
  __syncthreads();
  if (threadIdx.x == 0)  // release, cumulative over the block's stores ordered by the barrier
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(g.flags + e * (BIG_FLAG_WORDS / 2) + g.c / 2)
                 : "memory");
}

// Wait (acquire) until chunk c of extension e's data operand holds every producer's slices for this
// block's current multiplication; false when the wait ran out (abort raised) or another block aborted.
template <class C>
__device__ __forceinline__ bool tc_wait_chunk(const BigGroup<C>& g, int e, int c) {
  const uint32_t target = g.nmul * C::producers(c);
  const uint32_t* f = g.flags + e * (BIG_FLAG_WORDS / 2) + c;
  for (uint32_t it = 0;; it++) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if ((int32_t)(v - target) >= 0) return true;
    if (*(volatile uint32_t*)g.abort) return false;
    if (it >= g.spin_limit) {
      atomicExch(g.abort, 1u);
      return false;
    }
    if (it >= 2048) __nanosleep(128);
  }
}

// One base extension on the tensor cores (see BigTcCfg): acc[s] = sum_i X[lane][i] T[i][4w + s], exact,
// from the slot's data operand `aop` (all slices written, the slot barrier passed).  E = 1: the first
// extension, T1 resident in tensor memory (D^T = T1^T X^T), one streamed unit per chunk of k (data);
// E = 2: the second, two units per chunk (data, then this slice's T2 chunk `bop`).  Chunk positions
// are rotated by the block's offset so that blocks sharing an operand do not read the same chunk at
// once.  Thread 0 waits for each chunk and issues its products; the copy threads refill the stages.
// False (abort raised) when a copy or the tensor core does not complete in time.
template <class C, int E>
__device__ bool tc_ext(uint64_t (&acc)[4], BigGroup<C>& g, const uint8_t* aop, const uint8_t* bop, int ph0,
                       const uint32_t* kawg = nullptr, uint32_t* ksum = nullptr) {
  constexpr int S = C::STAGES, NCH = C::NCH, U = E * NCH;  // units streamed by this extension
  constexpr uint32_t CB = C::CHUNK_BYTES;
  uint8_t* const ring = reinterpret_cast<uint8_t*>(g.s + C::SM_RING);
  uint64_t* const full = reinterpret_cast<uint64_t*>(g.s + C::SM_MBAR);
  uint64_t* const empty = full + S;
  uint64_t* const done = empty + S;
  const uint32_t taddr = g.s[C::SM_TMEM];
  const uint32_t g0 = g.chunk;
  uint32_t ok = 1;
  const int t = tc_copier<C>();
  if (t >= 0) {
    const int st = t;
    uint8_t* const dst = ring + (size_t)st * CB;
    int last = -1;
    for (int u = tc_first_unit<C>(g0, st); u < U; u += S) {
      // the stage's previous unit (u - S, or the previous extension's, complete) must have been
      // consumed by the tensor core before the refill
      if (u >= S && !mbar_wait(&empty[st], ((g0 + u - S) / S) & 1u, g.spin_limit)) {
        ok = 0;
        break;
      }
      const int c = (u / E + g.stag) % NCH;  // position u / E holds chunk u / E + stag
      const bool data = !(E == 2 && (u & 1));
      if (data && !tc_wait_chunk<C>(g, E - 1, c)) {  // the producers' slices of this chunk are published
        ok = 0;
        break;
      }
      const uint8_t* src = data ? aop + (size_t)c * CB : bop + (size_t)c * CB;
      mbar_expect_tx(&full[st], CB);
      bulk_g2s(dst, src, CB, &full[st]);
      last = u;
    }
    if (!ok) {
      atomicExch(g.abort, 1u);
      if (last >= 0) mbar_wait(&full[st], ((g0 + last) / S) & 1u, g.spin_limit);  // no copy left in flight
    }
  } else if (threadIdx.x == 0) {
    constexpr uint32_t idesc = tc::idesc_f16_f32(128, 128);
    for (int c = 0; c < NCH && ok; c++) {
      const uint32_t cc = (c + g.stag) % NCH;  // the chunk of k at position c
      uint32_t sx = 0, sb = 0;                 // stages of the data and (second extension) T2 units
#pragma unroll
      for (int e = 0; e < E; e++) {
        const uint32_t gu = g0 + E * c + e, st = gu % S;
        if (!mbar_wait(&full[st], (gu / S) & 1u, g.spin_limit)) {
          ok = 0;
          break;
        }
        if (e == 0) sx = st;
        else sb = st;
      }
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t x0 = smem_u32(ring + (size_t)sx * CB), b0 = smem_u32(ring + (size_t)sb * CB);
#pragma unroll
      for (int ks = 0; ks < C::KC / 16; ks++) {
        // K step ks: column groups 2ks, 2ks + 1 (leading offset 16 x 128 rows, stride offset 128 bytes)
        const uint64_t xd = tc::sdesc(x0 + ks * 4096u, 2048u, 128u);
        const uint32_t acc_in = (c | ks) ? 1u : 0u;
        if constexpr (E == 1) {
          tc::mma_f16_ts(taddr, taddr + C::TM_T1 + 32u * cc + 8u * ks, xd, idesc, acc_in);
        } else {
          tc::mma_f16(taddr, xd, tc::sdesc(b0 + ks * 4096u, 2048u, 128u), idesc, acc_in);
        }
      }
      tc::mma_commit(&empty[sx]);
      if constexpr (E == 2) tc::mma_commit(&empty[sb]);
    }
    tc::mma_commit(done);
    // on failure, still give the issued products a bounded chance to finish before the tensor memory is
    // reused or the block exits
    if (!mbar_wait(done, g.done_ph, g.spin_limit)) ok = 0;
    if (!ok) atomicExch(g.abort, 1u);
    g.mark(ph0);
  }
  g.chunk += U;
  g.done_ph ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  tc::fence_after_sync();
  // second extension: every chunk has been seen (acquire, then the block barrier above), so every
  // block's correction-factor partial is visible; the loads overlap the epilogue
  uint32_t kp[E == 2 ? C::SLICES : 1];
  if constexpr (E == 2) {
#pragma unroll
    for (int u = 0; u < C::SLICES; u++) kp[u] = __ldcg(kawg + u * 32 + g.lane);
  }
  if constexpr (E == 1) {
    // epilogue of D^T: warp w reads lane quarter b = w % 4 (matrix slice b, channel j = lane) and the
    // columns of data slices 2h, 2h + 1 (h = w / 4) of all 32 numbers; the two data slices combine in
    // 32 bits (below 2^24 + 2^31), then the owner of (number, channel) sums the eight partials
    const int b = g.w & 3, h = g.w >> 2;
    uint32_t* ex = g.s + C::SM_EX;  // [2 h][4 b][32 j][EX1_LS] u32
    uint32_t* row = ex + ((h * 4 + b) * 32 + g.lane) * C::EX1_LS;
#pragma unroll
    for (int nn = 0; nn < 32; nn += 16) {
      uint32_t va[16], vb[16];
      tc::tmem_ld16(taddr + ((uint32_t)(32 * b) << 16) + 64u * h + nn, va);
      tc::tmem_ld16(taddr + ((uint32_t)(32 * b) << 16) + 64u * h + 32u + nn, vb);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; j++)
        row[nn + j] = __float2uint_rn(__uint_as_float(va[j])) + (__float2uint_rn(__uint_as_float(vb[j])) << 7);
    }
    tc::fence_before_sync();
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; s++) {
      const int ch = 4 * g.w + s;
      uint64_t v = 0;
#pragma unroll
      for (int q = 0; q < 8; q++)  // q = 4 hh + bb: shift 7 (2 hh + bb)
        v += (uint64_t)ex[(q * 32 + ch) * C::EX1_LS + g.lane] << (7 * (2 * (q >> 2) + (q & 3)));
      acc[s] = v;
    }
  } else {
    // epilogue of D: warp w reads the lanes of data slice a = w % 4 (its number = lane), columns of the
    // channels 16h .. 16h+15 (h = w / 4) of all four matrix slices; combines the matrix slices, then
    // the four warps of each half combine the data slices through shared memory
    const int qa = g.w & 3, h = g.w >> 2;
    uint64_t part[16];
#pragma unroll
    for (int j = 0; j < 16; j++) part[j] = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      uint32_t v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(32 * qa) << 16) + 32u * b + 16u * h, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; j++) part[j] += (uint64_t)__float2uint_rn(__uint_as_float(v[j])) << (7 * b);
    }
    uint64_t* ex = reinterpret_cast<uint64_t*>(g.s + C::SM_EX);
#pragma unroll
    for (int j = 0; j < 16; j++) ex[((qa * 2 + h) * 32 + g.lane) * C::EX_LS + j] = part[j] << (7 * qa);
    tc::fence_before_sync();
    __syncthreads();
    const int jb = 4 * g.w - 16 * h;  // this thread's channels 4w .. 4w+3 within half h
#pragma unroll
    for (int s = 0; s < 4; s++) {
      uint64_t v = 0;
#pragma unroll
      for (int q = 0; q < 4; q++) v += ex[((q * 2 + h) * 32 + g.lane) * C::EX_LS + jb + s];
      acc[s] = v;
    }
  }
  if constexpr (E == 2) {
    uint32_t v = 0;
#pragma unroll
    for (int u = 0; u < C::SLICES; u++) v += kp[u];
    *ksum = v;
  }
  g.mark(ph0 + 1);
  return true;
}

template <class C>
__device__ bool BigGroup<C>::barrier() {
  nbar++;
  // the ring's generic accesses (epilogue exchanges, the exit conversion's staging) before any copy into it
  if constexpr (C::TC) tc::fence_smem_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t target = nbar * (uint32_t)C::SLICES;
    __threadfence();
    atomicAdd(ctr, 1u);
    uint32_t ok = 1;
    for (uint32_t it = 0;; it++) {
      uint32_t v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if ((int32_t)(v - target) >= 0) break;
      if (*(volatile uint32_t*)abort) {
        ok = 0;
        break;
      }
      if (it >= spin_limit) {
        atomicExch(abort, 1u);
        ok = 0;
        break;
      }
      if (it >= 2048) __nanosleep(128);  // poll at L2 latency first, then back off
    }
    s[C::SM_MISC] = ok;
  }
  __syncthreads();
  return s[C::SM_MISC] != 0;
}

// RNS Montgomery multiplication x <- x*y*M^-1 mod N (outputs below (k+1)N), this thread's channels.
template <class C>
__device__ bool big_mont_mul(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT], const uint32_t (&yb)[C::NPT],
                             const uint32_t (&yp)[C::NPT], const uint32_t (&kxi)[C::NPT],
                             const uint32_t (&cmul)[C::NPT], const uint32_t (&cd)[C::NPT], BigGroup<C>& g) {
  constexpr int NPT = C::NPT, K = C::K;
  uint32_t* KAWg = g.slot + C::KAWG;
  uint32_t sp[NPT];
  uint32_t xv[NPT];
  g.mark(7);  // the previous multiplication's tail and the work between multiplications
  // 1-2. s = x*y in both bases; xi_i = s_i |-N^-1 (M/m_i)^-1| to the exchange buffer (zero on padding slots)
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s;
    const uint4 cb = g.a4(q);
    uint32_t sb = redc_lazy(mulw(xb[s], yb[s]), cb.x, cb.y);  // [0, 2m): only multiplied again
    xv[s] = redc(mulw(sb, kxi[s]), cb.x, cb.y);
    const uint4 cp = g.b4(q);
    sp[s] = redc_lazy(mulw(xp[s], yp[s]), cp.x, cp.y);
  }
  if constexpr (C::TC) {
    g.nmul++;
    tc_put_slices<C>(reinterpret_cast<uint8_t*>(g.slot + C::AG1), xv, g.c * C::SC + g.w * NPT, g.lane);
    g.mark(0);
    tc_publish<C>(g, 0);
  } else {
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int o = g.c * C::SC + g.w * NPT + s;
      if (o < K) g.slot[C::XG + (size_t)o * 32 + g.lane] = xv[s];
    }
    g.mark(0);
    if (!g.barrier()) return false;
  }
  g.mark(1);
  // 3. extension B -> B'
  uint64_t acc[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) acc[s] = 0;
  if constexpr (C::TC) {
    if (!tc_ext<C, 1>(acc, g, reinterpret_cast<const uint8_t*>(g.slot + C::AG1), nullptr, 2)) return false;
  } else {
    if (!big_ext<C>(acc, g, g.slot + C::XG, g.s + C::SM_T1)) return false;
  }
  // 4-5. new B' residues and xi'_j; partial correction-factor sums
  uint32_t kaw = 0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s;
    const uint4 cp = g.b4(q);
    const uint2 c2 = g.b2(q);
    uint32_t qh = redc64_lazy(acc[s], cp.x, cp.y, cp.z);
    xp[s] = redc(madw(sp[s], cp.w, mulw(qh, cmul[s])), cp.x, cp.y);
    xv[s] = redc(madw(sp[s], c2.x, mulw(qh, cd[s])), cp.x, cp.y);  // xi'_j, zero on padding slots
    kaw += hi32(mulw(xv[s], c2.y));  // zero on padding slots (ubp = 0)
  }
  if constexpr (C::TC) {
    tc_put_slices<C>(reinterpret_cast<uint8_t*>(g.slot + C::AG2), xv, g.c * C::SC + g.w * NPT, g.lane);
  } else {
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int o = g.c * C::SC + g.w * NPT + s;
      if (o < K) g.slot[C::XPG + (size_t)o * 32 + g.lane] = xv[s];
    }
  }
  g.s[C::SM_KAW + g.w * 32 + g.lane] = kaw;
  __syncthreads();
  if (g.w == 0) {
    uint32_t v = 0;
#pragma unroll
    for (int u = 0; u < C::NW; u++) v += g.s[C::SM_KAW + u * 32 + g.lane];
    KAWg[g.c * 32 + g.lane] = v;
  }
  g.mark(4);
  // 6. exact extension B' -> B with a' from the slice partials; the correction -a'|M'| enters as a' E
  //    with E = -M' 2^64 mod m_i
#pragma unroll
  for (int s = 0; s < NPT; s++) acc[s] = 0;
  uint32_t ks = 0;
  if constexpr (C::TC) {
    tc_publish<C>(g, 1);  // after the partial: every block's partial is visible once its chunk is
    g.mark(5);
    if (!tc_ext<C, 2>(acc, g, reinterpret_cast<const uint8_t*>(g.slot + C::AG2),
                      g.btab + (size_t)C::NCH * C::CHUNK_BYTES, 6, KAWg, &ks))
      return false;
  } else {
    if (!g.barrier()) return false;
    g.mark(5);
    // loaded before the dot products, summed after them
    uint32_t kp[C::SLICES];
#pragma unroll
    for (int u = 0; u < C::SLICES; u++) kp[u] = __ldcg(KAWg + u * 32 + g.lane);
    if (!big_ext<C>(acc, g, g.slot + C::XPG, g.s + C::SM_T2)) return false;
#pragma unroll
    for (int u = 0; u < C::SLICES; u++) ks += kp[u];
  }
  const uint32_t alpha = (ks + (1u << (KAW_Q - 2))) >> KAW_Q;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const uint4 cb = g.a4(g.w * NPT + s);
    xb[s] = redc64(madw(alpha, cb.w, acc[s]), cb.x, cb.y, cb.z);
  }
  return true;
}

// Binary -> hat residues of this thread's channels (x: nl limbs, zero beyond).
template <class C>
__device__ void big_to_rns(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT], const uint32_t* x, int nl,
                           const uint32_t* cls, const BigGroup<C>& g) {
  constexpr int NPT = C::NPT, K = C::K;
  const ClassOff co = class_offsets(C::K, C::W, C::WX);
  const uint32_t* P = cls + co.P;
  uint64_t ab[NPT], ap[NPT];
  int ob[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    ab[s] = ap[s] = 0;
    const int o = g.c * C::SC + g.w * NPT + s;
    ob[s] = o < K ? o : K - 1;
  }
  for (int wl = 0; wl < C::W; wl++) {
    const uint32_t xw = wl < nl ? x[wl] : 0u;
    const uint32_t* prow = P + (size_t)wl * 2 * K;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      ab[s] = madw(xw, __ldg(prow + ob[s]), ab[s]);
      ap[s] = madw(xw, __ldg(prow + K + ob[s]), ap[s]);
    }
    if (wl & 1) {
#pragma unroll
      for (int s = 0; s < NPT; s++) {
        const int q = g.w * NPT + s;
        ab[s] = madw(hi32(ab[s]), g.a4(q).z, lo32(ab[s]));
        ap[s] = madw(hi32(ap[s]), g.b4(q).z, lo32(ap[s]));
      }
    }
  }
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s;
    const uint4 cb = g.a4(q), cp = g.b4(q);
    xb[s] = redc64(ab[s], cb.x, cb.y, cb.z);
    xp[s] = redc64(ap[s], cp.x, cp.y, cp.z);
  }
}

template <class C>
__device__ __forceinline__ void big_load_vec(uint32_t (&vb)[C::NPT], uint32_t (&vp)[C::NPT], const uint32_t* v,
                                             const BigGroup<C>& g) {
#pragma unroll
  for (int s = 0; s < C::NPT; s++) {
    const int o = g.c * C::SC + g.w * C::NPT + s;
    vb[s] = o < C::K ? __ldg(v + o) : 0u;
    vp[s] = o < C::K ? __ldg(v + C::K + o) : 0u;
  }
}

template <class C>
__device__ __forceinline__ void big_tab(uint32_t* tab, int ent, uint32_t (&b)[C::NPT], uint32_t (&p)[C::NPT],
                                        const BigGroup<C>& g, bool store) {
#pragma unroll
  for (int s = 0; s < C::NPT; s++) {
    const int o = g.c * C::SC + g.w * C::NPT + s;
    if (o >= C::K) continue;
    uint32_t* eb = tab + ((size_t)ent * 2 * C::K + o) * 32 + g.lane;
    uint32_t* ep = eb + (size_t)C::K * 32;
    if (store) {
      *eb = b[s];
      *ep = p[s];
    } else {
      b[s] = *eb;
      p[s] = *ep;
    }
  }
}

// RNS -> binary of this group's 32 results, reduced mod N, by warp 0 of slice 0 (lane = number).
// Every CTA has published its plain CRT coefficients and partial factor sums; the caller has passed
// a barrier.  The slice's matrix area of shared memory serves as the staging buffer (reloaded by the
// caller before further multiplications).
template <class C>
__device__ void big_from_rns(const MxItem& it, const uint32_t* cls, bool write, BigGroup<C>& g) {
  constexpr int K = C::K, WX = C::WX, W = C::W;
  const ClassOff co = class_offsets(C::K, C::W, C::WX);
  const KeyOff ko = key_offsets(C::K, C::W);
  uint32_t* xs = g.s + C::SM_T1;  // K x 32 staged coefficients (fits in the 2 K SC matrix words)
  {
    const uint4* src = reinterpret_cast<const uint4*>(g.slot + C::XG);
    uint4* d = reinterpret_cast<uint4*>(xs);
    for (int i = threadIdx.x; i < K * 8; i += C::THREADS) d[i] = __ldcg(src + i);
  }
  __syncthreads();
  if (g.w != 0) return;
  uint32_t ks = 0;
  for (int u = 0; u < C::SLICES; u++) ks += __ldcg(g.slot + C::KAWX + u * 32 + g.lane);
  const uint32_t alpha = (ks + (1u << (KAW_Q - 2))) >> KAW_Q;
  uint32_t X[WX];
  const uint32_t* MD = cls + co.MD;
  const uint32_t* ML = cls + co.ML;
  uint32_t c0 = 0, c1 = 0;
  for (int wl = 0; wl < WX; wl++) {
    uint32_t s0 = c0, s1 = c1, s2 = 0;
    for (int i = 0; i < K; i++) mac96(s0, s1, s2, xs[i * 32 + g.lane], __ldg(MD + (size_t)i * WX + wl));
    X[wl] = s0;
    c0 = s1;
    c1 = s2;
  }
  uint32_t carry = 0, br = 0;
  for (int wl = 0; wl < WX; wl++) {
    uint64_t pw = mulw(alpha, __ldg(ML + wl)) + carry;
    carry = hi32(pw);
    uint64_t d = (uint64_t)X[wl] - lo32(pw) - br;
    X[wl] = lo32(d);
    br = hi32(d) ? 1u : 0u;
  }
  const uint32_t* key = it.key;
  const uint32_t nbits = __ldg(key + ko.hdr);
  const uint32_t* N = key + ko.N;
  const int sh = nbits > 32 ? (int)nbits - 32 : 0;
  auto bits64 = [&](const uint32_t* a, int na, int pos) -> uint64_t {
    int l = pos >> 5, b = pos & 31;
    uint64_t v0 = l < na ? a[l] : 0u, v1 = l + 1 < na ? a[l + 1] : 0u, v2 = l + 2 < na ? a[l + 2] : 0u;
    uint64_t lo = (v0 >> b) | (v1 << (32 - b));
    if (b == 0) lo = v0 | (v1 << 32);
    else lo |= (v2 << (64 - b));
    return lo;
  };
  const uint64_t xt = bits64(X, WX, sh);
  const uint64_t nt = (uint32_t)bits64(N, W, sh);
  uint64_t qe = xt / (nt + 1);
  if (qe) {
    uint32_t cq = 0, b2 = 0;
    for (int wl = 0; wl < WX; wl++) {
      uint64_t pw = mulw((uint32_t)qe, wl < W ? __ldg(N + wl) : 0u) + cq;
      cq = hi32(pw);
      uint64_t d = (uint64_t)X[wl] - lo32(pw) - b2;
      X[wl] = lo32(d);
      b2 = hi32(d) ? 1u : 0u;
    }
  }
  for (int rep = 0; rep < 4; rep++) {  // at most 2 are ever needed
    bool ge = true;
    for (int wl = WX - 1; wl >= 0; wl--) {
      uint32_t nv = wl < W ? __ldg(N + wl) : 0u;
      if (X[wl] != nv) {
        ge = X[wl] > nv;
        break;
      }
    }
    if (!ge) break;
    uint32_t b3 = 0;
    for (int wl = 0; wl < WX; wl++) {
      uint64_t d = (uint64_t)X[wl] - (wl < W ? __ldg(N + wl) : 0u) - b3;
      X[wl] = lo32(d);
      b3 = hi32(d) ? 1u : 0u;
    }
  }
  if (write)
    for (uint32_t wl = 0; wl < it.out_limbs; wl++) it.out[wl] = wl < (uint32_t)WX ? X[wl] : 0u;
}

// This slice's matrix columns and channel constants into shared memory.
template <class C>
__device__ void big_load_smem(uint32_t* s, const uint32_t* cls, const uint32_t* tslice, int c) {
  const ClassOff o = class_offsets(C::K, C::W, C::WX);
  const uint4* t1 = reinterpret_cast<const uint4*>(tslice + (size_t)c * C::K * C::SC);
  const uint4* t2 = reinterpret_cast<const uint4*>(tslice + (size_t)(C::SLICES + c) * C::K * C::SC);
  uint4* d1 = reinterpret_cast<uint4*>(s + C::SM_T1);
  uint4* d2 = reinterpret_cast<uint4*>(s + C::SM_T2);
  for (int i = threadIdx.x; i < C::K * C::SC / 4; i += C::THREADS) {
    d1[i] = __ldg(t1 + i);
    d2[i] = __ldg(t2 + i);
  }
}

template <class C>
__device__ void big_load_consts(uint32_t* s, const uint32_t* cls, int c) {
  const ClassOff o = class_offsets(C::K, C::W, C::WX);
  for (int q = threadIdx.x; q < C::SC; q += C::THREADS) {
    const int ch = c * C::SC + q;
    const bool ok = ch < C::K;
    const uint32_t m = ok ? cls[o.m + ch] : 0u, mphh = ok ? cls[o.mphh + ch] : 0u;
    uint32_t* a4 = s + C::SM_C4A + 4 * q;
    a4[0] = m;
    a4[1] = ok ? cls[o.mi + ch] : 0u;
    a4[2] = ok ? cls[o.r32 + ch] : 0u;
    a4[3] = mphh ? m - mphh : 0u;
    uint32_t* b4 = s + C::SM_C4B + 4 * q;
    b4[0] = ok ? cls[o.m + C::K + ch] : 0u;
    b4[1] = ok ? cls[o.mi + C::K + ch] : 0u;
    b4[2] = ok ? cls[o.r32 + C::K + ch] : 0u;
    b4[3] = ok ? cls[o.ahat + ch] : 0u;
    uint32_t* a2 = s + C::SM_C2A + 2 * q;
    a2[0] = ok ? cls[o.mmiinv + ch] : 0u;
    a2[1] = ok ? cls[o.ub + ch] : 0u;
    uint32_t* b2 = s + C::SM_C2B + 2 * q;
    b2[0] = ok ? cls[o.ad + ch] : 0u;
    b2[1] = ok ? cls[o.ubp + ch] : 0u;
  }
}

// One item group: x^e mod N for items [grp*32, grp*32+32).  Returns false on abort.
template <class C>
__device__ bool big_modexp_group(const BigArgs& a, BigGroup<C>& g, uint32_t grp) {
  constexpr int NPT = C::NPT;
  const uint32_t g_raw = grp * 32 + g.lane;
  const bool live = g_raw < a.n_items;
  const MxItem it = a.items[live ? g_raw : a.n_items - 1];
  const KeyOff ko = key_offsets(C::K, C::W);
  const uint32_t* key = it.key;
  const bool bad = !less_than(it.x, it.x_limbs, it.xlim, it.xlim_limbs);
  uint32_t* tab = g.slot + C::TAB;
  uint32_t kxi[NPT], cmul[NPT], cd[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = g.c * C::SC + g.w * NPT + s;
    kxi[s] = o < C::K ? __ldg(key + ko.kxi + o) : 0u;
    cmul[s] = o < C::K ? __ldg(key + ko.cmul + o) : 0u;
    cd[s] = o < C::K ? __ldg(key + ko.cd + o) : 0u;
  }
  uint32_t xb[NPT], xp[NPT], yb[NPT], yp[NPT];
  const int nl0 = bad ? 0 : (int)(it.x_limbs < (uint32_t)C::W ? it.x_limbs : C::W);
  big_to_rns<C>(xb, xp, it.x, nl0, a.cls, g);
  big_load_vec<C>(yb, yp, key + ko.r2, g);
  if (!big_mont_mul<C>(xb, xp, yb, yp, kxi, cmul, cd, g)) return false;
  const bool two = !bad && it.x_limbs > (uint32_t)C::W;
  if (__any_sync(0xffffffffu, two)) {
    uint32_t hb[NPT], hp[NPT];
    const int nl1 = two ? min((int)it.x_limbs - C::W, C::W) : 0;
    big_to_rns<C>(hb, hp, it.x + C::W, nl1, a.cls, g);
    big_load_vec<C>(yb, yp, key + ko.r2h, g);
    if (!big_mont_mul<C>(hb, hp, yb, yp, kxi, cmul, cd, g)) return false;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int q = g.w * NPT + s;
      const uint32_t mb = g.a4(q).x, mp = g.b4(q).x;
      uint32_t u = xb[s] + hb[s];
      xb[s] = min(u, u - mb);
      uint32_t v = xp[s] + hp[s];
      xp[s] = min(v, v - mp);
    }
  }
  // window table: entry 0 = Montgomery form of 1, entry j = x~^j
  const int wb = (int)a.wbits, E = 1 << wb;
  big_load_vec<C>(yb, yp, key + ko.one, g);
  big_tab<C>(tab, 0, yb, yp, g, true);
  big_tab<C>(tab, 1, xb, xp, g, true);
  {
    uint32_t cb[NPT], cp[NPT];
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      cb[s] = xb[s];
      cp[s] = xp[s];
    }
    for (int j = 2; j < E; j++) {
      if (!big_mont_mul<C>(cb, cp, xb, xp, kxi, cmul, cd, g)) return false;
      big_tab<C>(tab, j, cb, cp, g, true);
    }
  }
  // fixed windows from the top; every CTA of the slot sees the same 32 exponents, so the
  // warp-wide decisions below agree across the slot
  const uint32_t el = it.e_limbs;
  const uint32_t ebits = bad ? 0u : exp_bits(it.e, el);
  const uint32_t nwin = __reduce_max_sync(0xffffffffu, (ebits + wb - 1) / wb);
  uint32_t d = (nwin && !bad) ? exp_digit(it.e, el, (nwin - 1) * wb, wb) : 0u;
  __syncwarp();
  big_tab<C>(tab, d, xb, xp, g, false);
  for (int widx = (int)nwin - 2; widx >= 0; widx--) {
    for (int q = 0; q < wb; q++)
      if (!big_mont_mul<C>(xb, xp, xb, xp, kxi, cmul, cd, g)) return false;
    d = bad ? 0u : exp_digit(it.e, el, (uint32_t)widx * wb, wb);
    if (__any_sync(0xffffffffu, d != 0)) {
      big_tab<C>(tab, d, yb, yp, g, false);
      if (!big_mont_mul<C>(xb, xp, yb, yp, kxi, cmul, cd, g)) return false;
    }
  }
  // leave the domain: MM(x, 1); plain CRT coefficients and partial factor sums to the slot buffers
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s;
    yb[s] = g.a4(q).z;
    yp[s] = g.b4(q).z;
  }
  if (!big_mont_mul<C>(xb, xp, yb, yp, kxi, cmul, cd, g)) return false;
  uint32_t kaw = 0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s, o = g.c * C::SC + q;
    const uint4 cb = g.a4(q);
    const uint2 c2 = g.a2(q);
    uint32_t xi = redc(mulw(xb[s], c2.x), cb.x, cb.y);
    if (o < C::K) g.slot[C::XG + (size_t)o * 32 + g.lane] = xi;
    kaw += hi32(mulw(xi, c2.y));
  }
  g.s[C::SM_KAW + g.w * 32 + g.lane] = kaw;
  __syncthreads();
  if (g.w == 0) {
    uint32_t v = 0;
    for (int u = 0; u < C::NW; u++) v += g.s[C::SM_KAW + u * 32 + g.lane];
    g.slot[C::KAWX + g.c * 32 + g.lane] = v;
  }
  if (!g.barrier()) return false;
  if (g.c == 0) {
    big_from_rns<C>(it, a.cls, live && !bad, g);
    if (g.w == 0 && live) {
      if (bad)
        for (uint32_t wl = 0; wl < it.out_limbs; wl++) it.out[wl] = 0u;
      if (a.status && it.status != 0xffffffffu) a.status[it.status] = bad ? 5u : 0u;
    }
  }
  // the exchange buffers are reused by the next group only after slice 0 has read them
  return g.barrier();
}

template <class C>
__global__ void __launch_bounds__(C::THREADS, 1) big_modexp_kernel(BigArgs a) {
  extern __shared__ __align__(16) uint32_t smem_raw[];
  const uint32_t slot_id = blockIdx.x / C::SLICES;
  BigGroup<C> g;
  g.s = smem_raw;
  g.c = (int)(blockIdx.x % C::SLICES);
  g.w = (int)(threadIdx.x >> 5);
  g.lane = (int)(threadIdx.x & 31);
  g.slot = a.scratch + (size_t)slot_id * C::slot_words(a.wbits);
  g.ctr = a.sync + slot_id;
  g.abort = a.sync + a.slots;
  g.flags = a.sync + a.slots + 1 + (size_t)slot_id * BIG_FLAG_WORDS;
  g.nmul = 0;
  g.nbar = 0;
  g.spin_limit = a.spin_limit;
  g.ph = 0;
  g.chunk = 0;
  g.done_ph = 0;
  g.btab = nullptr;
  g.phases = a.phases;
  g.stag = 0;
  if constexpr (C::TC) g.stag = (uint32_t)(g.c + slot_id) % C::NCH;
  if (g.c == a.absent_slice) return;  // test hook: this slice never arrives; the others time out
  if (threadIdx.x == 0) {
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem_raw + C::SM_MBAR);
    int nmb = 2;  // staging copies of the integer form
    if constexpr (C::TC) nmb = 2 * C::STAGES + 1;  // full and empty per stage, accumulator complete
    for (int i = 0; i < nmb; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mb[i])));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if constexpr (C::TC) {
    g.btab = reinterpret_cast<const uint8_t*>(a.tslice) + (size_t)g.c * 2 * C::NCH * C::CHUNK_BYTES;
    if (threadIdx.x < 32) {
      tc::tmem_alloc(smem_raw + C::SM_TMEM, C::TMEM_COLS);
      tc::tmem_relinquish();
    }
    // columns of k beyond the last slice are never written: zero them once in both A operands
    if (g.c == 0 && C::KP > C::SLICES * C::SC) {
      constexpr uint32_t tail_col = C::SLICES * C::SC % C::KC;  // first padding column in the last chunk
      constexpr uint32_t tail_off = tail_col / 8 * 16 * 128, tail_bytes = C::CHUNK_BYTES - tail_off;
      for (int e = 0; e < 2; e++) {
        uint4* t = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(g.slot + (e ? C::AG2 : C::AG1)) +
                                            (size_t)(C::NCH - 1) * C::CHUNK_BYTES + tail_off);
        for (uint32_t i = threadIdx.x; i < tail_bytes / 16; i += C::THREADS) t[i] = make_uint4(0, 0, 0, 0);
      }
    }
    if (g.phases && threadIdx.x == 0) {
      unsigned long long* ph = reinterpret_cast<unsigned long long*>(smem_raw + C::SM_PH);
      for (int i = 0; i < BIG_PHASES; i++) ph[i] = 0;
      ph[BIG_PHASES] = clock64();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // this slice's T1 slices into tensor memory for the whole launch: row r = 32b + j in lane r, k in
    // columns TM_T1 + k / 2; warp w writes its lane quarter w % 4, half w / 4 of the columns
    {
      const uint32_t taddr = smem_raw[C::SM_TMEM];
      const int q = g.w & 3, h = g.w >> 2, r = 32 * q + g.lane;
      constexpr int G8 = C::KP / 8;  // groups of 8 values of k: 16 bytes of a row, 4 columns
      for (int kg = h * (G8 / 2); kg < (h + 1) * (G8 / 2); kg++) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(g.btab + (size_t)(kg / 8) * C::CHUNK_BYTES +
                                                             tc::tile_off(128, r, (kg % 8) * 8)));
        tc::tmem_st4(taddr + ((uint32_t)(32 * q) << 16) + C::TM_T1 + 4u * kg, v);
      }
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
    }
  }
  big_load_consts<C>(smem_raw, a.cls, g.c);
  const uint32_t n_groups = (a.n_items + 31) / 32;
  uint32_t grp = slot_id;
  for (; grp < n_groups; grp += a.slots) {
    if constexpr (!C::TC) big_load_smem<C>(smem_raw, a.cls, a.tslice, g.c);
    __syncthreads();
    if (!big_modexp_group<C>(a, g, grp)) break;
  }
  if constexpr (C::TC) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(smem_raw[C::SM_TMEM], C::TMEM_COLS);
    if (g.phases && threadIdx.x == 0) {
      const unsigned long long* ph = reinterpret_cast<const unsigned long long*>(smem_raw + C::SM_PH);
      for (int i = 0; i < BIG_PHASES; i++) atomicAdd(&g.phases[i], ph[i]);
      atomicAdd(&g.phases[BIG_PHASES], 1ull);
    }
  }
  if (grp < n_groups && g.c == (a.absent_slice == 0 ? 1 : 0) && a.status) {
    // aborted: every unfinished item of this slot reports a timeout
    for (uint32_t r = grp; r < n_groups; r += a.slots) {
      const uint32_t i = r * 32 + threadIdx.x;
      if (threadIdx.x < 32 && i < a.n_items && a.items[i].status != 0xffffffffu) a.status[a.items[i].status] = 8u;
    }
  }
}

}  // namespace mr
