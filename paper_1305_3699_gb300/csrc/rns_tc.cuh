// Tensor-core form of the lane-group RNS Montgomery multiplication ("Secrets
// from the GPU", Sec. 3.1): the two base extensions are products of the block's
// CRT coefficients with the class's constant extension matrices, so they are
// formed by tcgen05.mma (kind::f16, fp32 accumulators in tensor memory) instead
// of k-term mad.wide dot products; the channel work around them is the integer
// form's (rns_device.cuh).
//
// Exactness.  Every CRT coefficient xi_i and matrix entry T[i][j] is below 2^30
// (k >= 16 keeps the channel primes there), so each splits into four 8-bit
// slices, xi = sum_a 2^(8a) X_a, T = sum_b 2^(8b) T_b, and each slice is an fp16
// integer.  One product forms every P_ab(j) = sum_i X_a[i] T_b[i][j] for the 32
// numbers of the block: a sum of k products below 255^2, below 2^23 for k <= 129,
// so the fp32 accumulator holds it exactly.  An extra K column of 2048 x 4096
// adds 2^23 to every accumulator; a value in [2^23, 2^24) has the integer
// sum as its 23 mantissa bits.
//
// Layout.  The 4 data slices of number n are accumulator rows 8a + n % 8 of the
// tensor-memory lane quarter n / 8, and the 16 columns of one channel slot hold
// the 4 matrix bytes of the slot's channel for each of the number's 4 lanes, in
// the order the 16x256b load shape delivers them: lane u of the number receives
// all 16 sums P_ab of its own channel (rows n % 8 and n % 8 + 8 of each 16-lane
// half, columns 2u, 2u + 1 of each 8-column group) and forms the 64-bit dot
// product sum_{a,b} 2^(8(a+b)) P_ab alone -- bit for bit the integer form's
// accumulator, with no exchange between lanes.
//
// Block shape.  32 numbers; TPI = 4: 4 lanes per number in one warp (lane 4(n % 8)
// + u of warp n / 8); TPI = 8: the number's two groups of four in warps n / 8
// (h = 0) and n / 8 + 4 (h = 1), which read the same lane quarter, each half its
// own 16 NPT accumulator columns.  All warps take part in every multiplication
// (two block barriers and two tensor-core waits per multiplication), so the
// exponent schedule of a block is uniform (kernels.cuh).
#pragma once
#include <cuda_fp16.h>

#include <cstdint>

#include "rns_device.cuh"
#include "tc_device.cuh"

namespace mr {

// Tensor-core completion wait before the block gives up (far beyond any legitimate completion).
constexpr uint64_t LG_TC_WAIT_NS = 1000000000ull;

struct TcState {
  uint32_t tmem;   // accumulator base address in tensor memory
  uint32_t phase;  // parity of the next completion of the block's mbarrier
  uint32_t skip;   // test hook: thread 0 issues no product (every completion wait runs out)
};

template <class C>
struct TcSmem {
  uint8_t* base;
  __device__ uint8_t* A() const { return base + C::TC_A; }
  __device__ uint8_t* B1() const { return base + C::TC_B1; }
  __device__ uint8_t* B2() const { return base + C::TC_B2; }
  __device__ uint64_t* mbar() const { return reinterpret_cast<uint64_t*>(base + C::TC_MISC); }
  __device__ uint32_t* tslot() const { return reinterpret_cast<uint32_t*>(base + C::TC_MISC + 32); }
  __device__ volatile uint32_t* abort_flag() const { return reinterpret_cast<volatile uint32_t*>(base + C::TC_MISC + 36); }
  __device__ uint32_t* vote() const { return reinterpret_cast<uint32_t*>(base + C::TC_MISC + 64); }  // 8 words
  __device__ uint32_t* part() const { return reinterpret_cast<uint32_t*>(base + C::TC_MISC + 128); }  // [2][32]
};

// K column of lane t's channel slot s is NPTK t + tc_kslot(t, s): with NPTK = 8 the two groups of four
// slots trade places for odd t (an involution), so that the 8-byte stores of one warp instruction
// reach both halves of a core-matrix row (shared-memory banks).
template <class C>
__host__ __device__ constexpr int tc_kslot(int t, int s) {
  return (C::NPTK % 8 == 0 && (t & 1)) ? (s ^ 4) : s;
}

__device__ __forceinline__ uint16_t half_bits_u8(uint32_t v) { return __half_as_ushort(__uint2half_rn(v)); }

// Block prologue of the tensor-core form (after load_class_smem): the two matrix operands as fp16
// slices, the data operand's constant columns, the mbarrier and the block's accumulator columns.
template <class C>
__device__ void tc_prologue(const TcSmem<C>& ts, const uint32_t* cls) {
  constexpr int K = C::K, NPT = C::NPT, NPTK = C::NPTK, KA = C::KA, NB = C::NB;
  const ClassOff o = class_offsets(C::K, C::W, C::WX);
  uint8_t* A = ts.A();
  for (int idx = threadIdx.x; idx < 128 * KA; idx += C::THREADS) {
    const int r = idx / KA, col = idx % KA;
    *reinterpret_cast<uint16_t*>(A + tc::tile_off(128, r, col)) = col == NPT ? (uint16_t)0x6800u : (uint16_t)0u;  // 2048
  }
  uint8_t* B1 = ts.B1();
  uint8_t* B2 = ts.B2();
  for (int idx = threadIdx.x; idx < NB * KA; idx += C::THREADS) {
    const int c = idx / KA, col = idx % KA;
    // column c = 16 NPT h + 16 jj + 8 (b / 2) + 2 u + b % 2 (the 16x256b load order)
    const int h = c / (16 * NPT), jj = (c / 16) % NPT, r16 = c % 16;
    const int u = (r16 % 8) / 2, b = 2 * (r16 / 8) + (r16 % 2);
    const int j = (4 * h + u) * NPT + jj;            // output channel
    const int ti = col / NPTK, si = tc_kslot<C>(ti, col % NPTK);
    const int i = ti * NPT + si;                     // input channel
    uint16_t h1 = 0, h2 = 0;
    if (col == NPT) {
      h1 = h2 = 0x6C00u;  // 4096
    } else if (si < NPT && i < K && j < K) {
      h1 = half_bits_u8((__ldg(cls + o.T1 + i * K + j) >> (8 * b)) & 0xFFu);
      h2 = half_bits_u8((__ldg(cls + o.T2 + i * K + j) >> (8 * b)) & 0xFFu);
    }
    *reinterpret_cast<uint16_t*>(B1 + tc::tile_off(NB, c, col)) = h1;
    *reinterpret_cast<uint16_t*>(B2 + tc::tile_off(NB, c, col)) = h2;
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(ts.mbar(), 1);
    *ts.abort_flag() = 0u;
    for (int q = 0; q < 8; q++) ts.vote()[q] = 0u;
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(ts.tslot(), C::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_smem_async();
  tc::fence_before_sync();
}

// Write byte slices of this lane's coefficients v (its NPT channels; lane t of number n) into rows
// 32 (n / 8) + 8 a + n % 8 of the data operand: four consecutive K columns per 8-byte store.  A byte b becomes the fp16
// value b as the bit pattern of 1024 + b minus 1024.  The rows of one store instruction are the 8
// numbers of the lane quarter (distinct rows of a core matrix), so a warp's stores need the minimum
// two shared-memory wavefronts.
template <class C>
__device__ __forceinline__ void tc_publish(const TcSmem<C>& ts, const uint32_t (&v)[C::NPT], int n, int t) {
  constexpr int NPT = C::NPT, NPTK = C::NPTK, K = C::K;
  uint8_t* A = ts.A();
  const __half2 bias = __halves2half2(__ushort_as_half(0x6400u), __ushort_as_half(0x6400u));
#pragma unroll
  for (int g = 0; g < NPTK / 4; g++) {
    uint32_t x[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int s = 4 * g + q;
      x[q] = (s < NPT && t * NPT + s < K) ? v[s < NPT ? s : 0] : 0u;
    }
    const bool has_off = (t == 0) && (4 * g <= NPT) && (NPT < 4 * g + 4);  // the 2^23 offset column
    const int row0 = 32 * (n / 8) + n % 8;  // row of data slice a: row0 + 8 a
#pragma unroll
    for (int a = 0; a < 4; a++) {
      uint32_t w[2];
#pragma unroll
      for (int p = 0; p < 2; p++) {
        // bytes a of x[2p] and x[2p+1], each followed by 0x64: fp16 (1024 + byte), then minus 1024
        const uint32_t sel = (uint32_t)a | ((uint32_t)(4 + a) << 4);
        const uint32_t two = __byte_perm(x[2 * p], x[2 * p + 1], sel);
        const uint32_t pk = __byte_perm(two, 0x64646464u, 0x4140u);
        __half2 h = *reinterpret_cast<const __half2*>(&pk);
        h = __hsub2(h, bias);
        w[p] = *reinterpret_cast<const uint32_t*>(&h);
      }
      if (has_off) {
        const int q = NPT - 4 * g;  // position of the offset column in this group of four
        const uint32_t off = 0x6800u;
        if (q == 0) w[0] = (w[0] & 0xFFFF0000u) | off;
        if (q == 1) w[0] = (w[0] & 0x0000FFFFu) | (off << 16);
        if (q == 2) w[1] = (w[1] & 0xFFFF0000u) | off;
        if (q == 3) w[1] = (w[1] & 0x0000FFFFu) | (off << 16);
      }
      *reinterpret_cast<uint2*>(A + tc::tile_off(128, row0 + 8 * a, NPTK * t + tc_kslot<C>(t, 4 * g))) =
          make_uint2(w[0], w[1]);
    }
  }
}

// One channel slot's 16 accumulators of this lane's channel, from the two 16x256b loads of the slot
// (lo: the rows of data slices 0, 1; hi: those of slices 2, 3; element [4p + 2e + f] holds data slice
// e (e + 2 for hi) times matrix byte 2p + f), each the bit pattern of 2^23 + P_ab: the exact 64-bit sum
// sum_{a,b} 2^(8(a+b)) P_ab, formed from the digit sums w_s = sum_{a+b=s} P_ab (each below 2^24; a
// pair w_s + 2^8 w_(s+1) stays below 2^32 while the second digit has at most 2 terms, or 4 with k <= 64).
template <int K>
__device__ __forceinline__ uint64_t tc_combine(const uint32_t (&lo)[8], const uint32_t (&hi)[8]) {
  constexpr uint32_t OFF = 0x4B000000u;  // bit pattern of 2^23, carried once per summed accumulator
  const uint32_t w0 = lo[0];
  const uint32_t w1 = lo[1] + lo[2];
  const uint32_t w2 = lo[4] + lo[3] + hi[0];
  const uint32_t w3 = lo[5] + lo[6] + hi[1] + hi[2];
  const uint32_t w4 = lo[7] + hi[4] + hi[3];
  const uint32_t w5 = hi[5] + hi[6];
  const uint32_t w6 = hi[7];
  // digits and pairs of digits with the offsets removed (mod 2^32; each true value is below 2^32)
  const uint32_t x0 = w0 + (w1 << 8) - (uint32_t)(1u * OFF + ((2u * OFF) << 8));
  const uint32_t x2 = w4 + (w5 << 8) - (uint32_t)(3u * OFF + ((2u * OFF) << 8));
  const uint32_t x3 = w6 - OFF;
  if constexpr ((uint64_t)K * 65025u * (4u * 256u + 3u) < (1ull << 32)) {
    const uint32_t x1 = w2 + (w3 << 8) - (uint32_t)(3u * OFF + ((4u * OFF) << 8));
    return (uint64_t)x0 + ((uint64_t)x1 << 16) + ((uint64_t)x2 << 32) + ((uint64_t)x3 << 48);
  } else {
    const uint32_t y2 = w2 - 3u * OFF, y3 = w3 - 4u * OFF;
    return (uint64_t)x0 + ((uint64_t)y2 << 16) + ((uint64_t)y3 << 24) + ((uint64_t)x2 << 32) +
           ((uint64_t)x3 << 48);
  }
}

// One base extension: the block's data operand (already published) times matrix operand B; acc[s]
// receives the k-term dot product of this lane's output channel t NPT + s.  Thread 0 issues the
// product (one tcgen05.mma per K step of 16 and warp half); every thread runs `overlap` and then
// waits for the product's completion on the block's mbarrier.
template <class C, class Overlap>
__device__ __forceinline__ void tc_extension(const TcSmem<C>& ts, TcState& st, const uint8_t* B,
                                             uint64_t (&acc)[C::NPT], int t, Overlap&& overlap) {
  constexpr int NPT = C::NPT, KA = C::KA, NB = C::NB, HALVES = C::TPI / 4;
  tc::fence_smem_async();   // the generic-proxy stores of the data operand, visible to the tensor core
  tc::fence_before_sync();  // the previous extension's accumulator loads complete before the barrier
  __syncthreads();
  if (threadIdx.x == 0 && *ts.abort_flag() == 0u && !st.skip) {
    tc::fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_f16_f32(128, 16 * NPT);
    const uint32_t a0 = tc::saddr(ts.A()), b0 = tc::saddr(B);
#pragma unroll
    for (int h = 0; h < HALVES; h++) {
      const int row0 = 16 * NPT * h;  // first matrix row = first accumulator column of warp half h
#pragma unroll
      for (int ks = 0; ks < KA / 16; ks++) {
        const uint64_t ad = tc::sdesc(a0 + ks * (2 * 16 * 128), 16 * 128, 128);
        const uint64_t bd = tc::sdesc(b0 + ks * (2 * 16 * NB) + (row0 / 8) * 128, 16 * NB, 128);
        tc::mma_f16(st.tmem + row0, ad, bd, idesc, ks > 0 ? 1u : 0u);
      }
    }
    tc::mma_commit(ts.mbar());
  }
  overlap();  // work that does not depend on the product
  if (*ts.abort_flag() == 0u) {
    if (tc::mbar_wait_ns(ts.mbar(), st.phase, LG_TC_WAIT_NS)) st.phase ^= 1u;
    else *ts.abort_flag() = 1u;  // st.phase stays the parity of the product that may still be in flight
  }
  tc::fence_after_sync();
  const int warp = threadIdx.x >> 5;
  // lane quarter warp % 4 (its two 16-lane halves: data slices 0, 1 and 2, 3); warp half h reads its
  // 16 NPT columns
  const uint32_t base = st.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(16 * NPT * tc_half<C>());
#pragma unroll
  for (int j0 = 0; j0 < NPT; j0 += 3) {  // loads and combines in groups of 3 slots
    uint32_t lo[3][8], hi[3][8];
#pragma unroll
    for (int q = 0; q < 3; q++)
      if (j0 + q < NPT) {
        tc::tmem_ld16x256b_x2(base + 16 * (j0 + q), lo[q]);
        tc::tmem_ld16x256b_x2(base + (16u << 16) + 16 * (j0 + q), hi[q]);
      }
    tc::tmem_ld_wait();
#pragma unroll
    for (int q = 0; q < 3; q++)
      if (j0 + q < NPT) acc[j0 + q] = tc_combine<C::K>(lo[q], hi[q]);
  }
}

// RNS Montgomery multiplication with the extensions on the tensor cores: the integer form's steps
// (mont_mul in rns_device.cuh) with ext_dot replaced by tc_extension.  All threads of the block call
// it together.
template <class C>
__device__ __forceinline__ void mont_mul_tc(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT],
                                            const uint32_t (&yb)[C::NPT], const uint32_t (&yp)[C::NPT],
                                            const uint32_t (&kxp)[C::NPT], const uint32_t (&kxs)[C::NPT],
                                            const uint32_t (&cmul)[C::NPT], const Smem<C>& sm, const TcSmem<C>& ts,
                                            TcState& st, int t) {
  constexpr int NPT = C::NPT;
  const int n = tc_number<C>();
  uint32_t sp[NPT], xi[NPT];
  // 1-2. s = x*y in B; xi_i = s_i |-N^-1 (M/m_i)^-1| (plain)
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const uint4 cb = sm.cb4(t, s);
    const uint32_t sb = redc_lazy(mulw(xb[s], yb[s]), cb.x, cb.y);
    const uint32_t u = sb * kxp[s] - __umulhi(sb, kxs[s]) * cb.x;
    xi[s] = min(u, u - cb.x);
  }
  tc_publish<C>(ts, xi, n, t);
  // 3. extension B -> B'; s = x*y in B' is formed while the product runs
  uint64_t acc[NPT];
  tc_extension<C>(ts, st, ts.B1(), acc, t, [&] {
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const uint4 cp = sm.cp4(t, s);
      sp[s] = redc_lazy(mulw(xp[s], yp[s]), cp.x, cp.y);
    }
  });
  // 4-5. new B' residues and xi'_j (as in mont_mul)
  uint32_t kaw = 0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const uint4 cp = sm.cp4(t, s);
    const uint4 cx = sm.cpx(t, s);
    uint32_t qh = redc64_lazy(acc[s], cp.x, cp.y, cp.z);
    xp[s] = redc(madw(sp[s], cp.w, mulw(qh, cmul[s])), cp.x, cp.y);
    const uint32_t u = xp[s] * cx.z - __umulhi(xp[s], cx.w) * cp.x;
    const uint32_t xpj = min(u, u - cp.x);
    xi[s] = xpj;
    kaw += (xpj >> KAW_S) * cx.y;
  }
  tc_publish<C>(ts, xi, n, t);
  // the correction factor's fixed-point sum over the number's 8 lanes: this warp half's part goes to
  // shared memory before the extension's block barrier, the other half's is read after it
  kaw += __shfl_xor_sync(0xffffffffu, kaw, 1);
  kaw += __shfl_xor_sync(0xffffffffu, kaw, 2);
  if constexpr (C::TPI == 8)
    if ((threadIdx.x & 3) == 0) ts.part()[32 * tc_half<C>() + n] = kaw;
  // 6. extension B' -> B, exact, with the correction folded into the accumulator
  tc_extension<C>(ts, st, ts.B2(), acc, t, [] {});
  if constexpr (C::TPI == 8) kaw += ts.part()[32 * (1 - tc_half<C>()) + n];
  const uint32_t alpha = (kaw + (1u << (KAW_Q - 2))) >> KAW_Q;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const uint4 cb = sm.cb4(t, s);
    xb[s] = redc64(madw(alpha, cb.x - cb.w, acc[s]), cb.x, cb.y, cb.z);
  }
}

// Block epilogue: wait (bounded) for a product still in flight after an abort, then free the
// accumulator columns.  (With the skip hook nothing is in flight and this wait also runs out.)
template <class C>
__device__ void tc_release(const TcSmem<C>& ts, const TcState& st) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (*ts.abort_flag() != 0u && threadIdx.x == 0) (void)tc::mbar_wait_ns(ts.mbar(), st.phase, LG_TC_WAIT_NS);
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(st.tmem, C::TMEM_COLS);
}

}  // namespace mr
