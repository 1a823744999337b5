// Device side of the RNS modular exponentiation ("Secrets from the GPU",
// Sec. 3.1): channel arithmetic, RNS Montgomery multiplication with its two
// base extensions, fixed-window exponentiation, binary <-> RNS conversion.
//
// Mapping.  One number is owned by a group of TPI consecutive lanes of a warp
// (32/TPI numbers per warp).  Lane t of the group owns the NPT = ceil(k/TPI)
// consecutive channels [t*NPT, t*NPT+NPT) of base B and the same positions of
// base B'; its residues stay in registers for the whole exponentiation.  The
// two base extensions are the only all-to-all steps: each lane publishes its
// CRT coefficients xi to shared memory, the group reads all k of them
// (broadcast loads) and every lane forms the k-term dot products of its own
// output channels against the extension matrix, which is shared by every
// number of the size class and kept in shared memory.  A group only ever
// synchronises with __syncwarp; no block-wide barrier after the prologue.
//
// Word arithmetic.  Channel primes m < 2^31 with k*m^2 < 2^64 (chosen at
// setup), so a k-term dot product of residues accumulates exactly in one
// 64-bit register with one mad.wide.u32 per term (two issue slots of the
// integer-multiply pipe, the cheapest exact 32x32->64 product; a carry-chain
// accumulation costs more) and is reduced once.  Residues are kept in
// per-channel Montgomery form x*2^32 mod m ("hat"); reductions use mad.wide;
// one product by a per-class constant uses Shoup's precomputed quotient
// (mad.hi and two mad.lo).
#pragma once
#include <cstdint>

#include "layout.h"

namespace mr {

__device__ __forceinline__ uint64_t madw(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t r;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
  return r;
}
__device__ __forceinline__ uint64_t mulw(uint32_t a, uint32_t b) {
  uint64_t r;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t lo32(uint64_t v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t hi32(uint64_t v) { return (uint32_t)(v >> 32); }

// Word Montgomery reduction: v * 2^-32 mod m for v < 2^32 (m + 1), mi = -m^-1 mod 2^32.
// Result in [0, m] (in [0, m) when v < 2^32 m).  Requires m < 2^31.
__device__ __forceinline__ uint32_t redc(uint64_t v, uint32_t m, uint32_t mi) {
  uint32_t q = lo32(v) * mi;
  uint32_t r = hi32(madw(q, m, v));
  return min(r, r - m);
}
// The same without the final conditional subtraction: for v < 2^32 m the result is in [0, 2m).
// Used for temporaries that only feed further products: with m < 2^30 a product of such a value
// with a residue below 2m stays below 2^32 m, so a later reduction still applies.
__device__ __forceinline__ uint32_t redc_lazy(uint64_t v, uint32_t m, uint32_t mi) {
  uint32_t q = lo32(v) * mi;
  return hi32(madw(q, m, v));
}
// Any v < 2^64: fold the high word with r32 = 2^32 mod m, then reduce.  Result v 2^-32 mod m in [0, m].
__device__ __forceinline__ uint32_t redc64(uint64_t v, uint32_t m, uint32_t mi, uint32_t r32) {
  return redc(madw(hi32(v), r32, lo32(v)), m, mi);
}
// The same with a result in [0, 2m) (see redc_lazy).
__device__ __forceinline__ uint32_t redc64_lazy(uint64_t v, uint32_t m, uint32_t mi, uint32_t r32) {
  return redc_lazy(madw(hi32(v), r32, lo32(v)), m, mi);
}

// 96-bit accumulate (s2:s1:s0) += a*b (one-time conversions only)
__device__ __forceinline__ void mac96(uint32_t& s0, uint32_t& s1, uint32_t& s2, uint32_t a, uint32_t b) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
      : "+r"(s0), "+r"(s1), "+r"(s2)
      : "r"(a), "r"(b));
}

template <int K_, int W_, int WX_, int TPI_, int THREADS_, int VEC_, int MINB_ = 0, int TC_ = 0>
struct Cfg {
  static constexpr int MINB = MINB_;             // exponentiation kernel's minimum resident blocks per SM
                                                  // (register budget; 0 leaves the choice to the compiler)
  static constexpr int TC = TC_;                  // 1: the exponentiation kernel forms the two base
                                                  // extensions on the tensor cores (rns_tc.cuh)
  static constexpr int K = K_;                    // channels per base
  static constexpr int W = W_;                    // limbs of the class bound
  static constexpr int WX = WX_;                  // limbs of k*M (RNS -> binary)
  static constexpr int TPI = TPI_;                // lanes per number
  static constexpr int NPT = (K + TPI - 1) / TPI; // channels per lane and base
  static constexpr int VEC = VEC_;                // words per shared-memory load of a matrix row (2 or 4)
  static constexpr int NPTP = (NPT + VEC - 1) / VEC * VEC;  // padded to whole vector loads
  // per-lane stride of a matrix row: an odd number of vectors, so that the distinct lanes of one
  // shared-memory wavefront (8 for 16-byte loads, 16 for 8-byte loads) hit distinct banks
  static constexpr int LS = ((NPTP / VEC) % 2 == 0) ? NPTP + VEC : NPTP;
  static constexpr int ROW = TPI * LS;            // words per extension-matrix row in smem
  static constexpr int NPTC = NPT | 1;            // per-lane stride of the channel-constant arrays (odd)
  static constexpr int SL = TPI * NPTC;           // slots of the constant arrays
  static constexpr int KP = (K + 3) & ~3;         // xi / xi' buffer length
  static constexpr int XS = 2 * KP + 4;           // per-number stride of the two buffers: XS/4 odd
                                                  // keeps broadcast loads and stores bank-conflict free
  static constexpr int THREADS = THREADS_;
  static constexpr int IPB = THREADS / TPI;       // numbers per block
  static constexpr int IPW = 32 / TPI;            // numbers per warp
  // shared memory, in 16-byte units where vectors live
  static constexpr int SM_T1 = 0;
  static constexpr int SM_T2 = SM_T1 + K * ROW;
  static constexpr int SM_CB4 = SM_T2 + K * ROW;  // uint4 {m, mi, r32, mphh}        B
  static constexpr int SM_CP4 = SM_CB4 + 4 * SL;  // uint4 {m, mi, r32, ahat}        B'
  static constexpr int SM_CPX = SM_CP4 + 4 * SL;  // uint4 {ad, ubs, xpc, xpcs}      B'
  static constexpr int SM_CB2 = SM_CPX + 4 * SL;  // uint2 {mmiinv, ub}              B
  static constexpr int SM_XI = SM_CB2 + 2 * SL;   // IPB x XS
  static constexpr int SM_WORDS = SM_XI + IPB * XS;
  static constexpr int SMEM_BYTES = SM_WORDS * 4;
  static_assert(TPI == 1 || TPI == 2 || TPI == 4 || TPI == 8 || TPI == 16 || TPI == 32, "TPI must divide 32");
  static_assert(K >= 16, "k >= 16 keeps every channel prime below isqrt(2^64/16) = 2^30 (lazy reductions)");
  static_assert(VEC == 2 || VEC == 4, "vector width");
  static_assert((SM_T2 % 4) == 0 && (SM_CB4 % 4) == 0 && (SM_CPX % 4) == 0 && (SM_CB2 % 2) == 0 && (SM_XI % 4) == 0,
                "alignment");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

  // Tensor-core form (TC = 1, rns_tc.cuh).  The block's 32 numbers x 4 byte slices are the 128 rows of
  // the data operand (row 32 (n / 8) + 8 a + n % 8: byte a of number n's CRT coefficients).  Lane t of
  // number n has its NPT input channels in K columns [NPTK t, NPTK t + NPT); the rest is zero except
  // one offset column (K index NPT) whose product 2048 * 4096 = 2^23 is added to every accumulator.
  // With TPI = 4 the number's lanes are 4n .. 4n + 3 of the block; with TPI = 8 they are split over
  // two warps of the same tensor-memory lane quarter (lane t = 4 h + u in warp half h).  The matrix
  // operand has NB = 16 NPT TPI / 4 rows, row 16 NPT h + 16 s + 8 (b / 2) + 2 u + b % 2 holding byte b
  // of the matrix column of output channel (4 h + u) NPT + s (the 16x256b load order), so that warp
  // half h reads its channels' accumulators from its own 16 NPT columns.
  static constexpr int NPTK = (NPT / 4 + 1) * 4;  // K columns per lane's channel set (>= NPT + 1)
  static constexpr int KA = TPI * NPTK;            // K extent, a multiple of 16
  static constexpr int NB = 4 * NPT * TPI;         // accumulator columns (N of the product)
  static constexpr int TC_A = (SMEM_BYTES + 127) / 128 * 128;  // byte offsets of the operand tiles
  static constexpr int TC_B1 = TC_A + 128 * KA * 2;
  static constexpr int TC_B2 = TC_B1 + NB * KA * 2;
  static constexpr int TC_MISC = TC_B2 + NB * KA * 2;  // mbarrier, tensor-memory address, abort flag, votes,
                                                       // then [2 warp halves][32 numbers] partial sums
  static constexpr int TC_END = TC_MISC + 128 + 256;
  // accumulator columns allocated per block (a power of two), and the blocks that fit the SM's 512
  static constexpr int TMEM_COLS = NB <= 32 ? 32 : NB <= 64 ? 64 : NB <= 128 ? 128 : NB <= 256 ? 256 : 512;
  static constexpr int TC_BLOCKS = 512 / TMEM_COLS;
  // the tensor-core kernel asks for enough shared memory that no more than TC_BLOCKS blocks share an SM
  // (228 KB per SM, 1 KB reserved per block)
  static constexpr int TC_SMEM_MIN = TC_BLOCKS >= 4 ? 0 : 233472 / (TC_BLOCKS + 1) - 1024 + 128;
  static constexpr int SMEM_MODEXP_BYTES = TC ? (TC_END > TC_SMEM_MIN ? TC_END : TC_SMEM_MIN) : SMEM_BYTES;
  static_assert(!TC || (TPI == 4 && THREADS == 128) || (TPI == 8 && THREADS == 256),
                "tensor-core form: 32 numbers x 4 or 8 lanes");
  static_assert(!TC || (16 * NPT <= 256 && NB <= 512), "tensor-core form: N <= 256 per warp half");
  static_assert(!TC || K * 255 * 255 < (1 << 23), "tensor-core form: every fp32 sum stays below 2^23");
  static_assert(SMEM_MODEXP_BYTES <= 227 * 1024, "shared memory");
};

template <class C>
struct Smem {
  uint32_t* base;
  __device__ const uint32_t* T1() const { return base + C::SM_T1; }
  __device__ const uint32_t* T2() const { return base + C::SM_T2; }
  // constants of channel t*NPT + s (lane t of a group, its s-th channel)
  __device__ uint4 cb4(int t, int s) const { return reinterpret_cast<const uint4*>(base + C::SM_CB4)[t * C::NPTC + s]; }
  __device__ uint4 cp4(int t, int s) const { return reinterpret_cast<const uint4*>(base + C::SM_CP4)[t * C::NPTC + s]; }
  __device__ uint2 cb2(int t, int s) const { return reinterpret_cast<const uint2*>(base + C::SM_CB2)[t * C::NPTC + s]; }
  __device__ uint4 cpx(int t, int s) const { return reinterpret_cast<const uint4*>(base + C::SM_CPX)[t * C::NPTC + s]; }
  __device__ uint32_t* xi(int item_in_block) const { return base + C::SM_XI + item_in_block * C::XS; }
};

// Block prologue: copy the class tables into shared memory in the lane-slot layout.
template <class C>
__device__ void load_class_smem(const Smem<C>& sm, const uint32_t* cls) {
  const ClassOff o = class_offsets(C::K, C::W, C::WX);
  uint32_t* s = sm.base;
  for (int idx = threadIdx.x; idx < C::K * C::ROW; idx += blockDim.x) {
    int row = idx / C::ROW, col = idx % C::ROW;
    int t = col / C::LS, sl = col % C::LS;
    int ch = t * C::NPT + sl;
    bool ok = sl < C::NPT && ch < C::K;
    s[C::SM_T1 + idx] = ok ? cls[o.T1 + row * C::K + ch] : 0u;
    s[C::SM_T2 + idx] = ok ? cls[o.T2 + row * C::K + ch] : 0u;
  }
  for (int q = threadIdx.x; q < C::SL; q += blockDim.x) {
    const int ch = (q / C::NPTC) * C::NPT + q % C::NPTC;
    bool ok = q % C::NPTC < C::NPT && ch < C::K;
    uint32_t* cb4 = s + C::SM_CB4 + 4 * q;
    uint32_t* cp4 = s + C::SM_CP4 + 4 * q;
    uint32_t* cb2 = s + C::SM_CB2 + 2 * q;
    uint32_t* cpx = s + C::SM_CPX + 4 * q;
    cb4[0] = ok ? cls[o.m + ch] : 0u;
    cb4[1] = ok ? cls[o.mi + ch] : 0u;
    cb4[2] = ok ? cls[o.r32 + ch] : 0u;
    cb4[3] = ok ? cls[o.mphh + ch] : 0u;
    cp4[0] = ok ? cls[o.m + C::K + ch] : 0u;
    cp4[1] = ok ? cls[o.mi + C::K + ch] : 0u;
    cp4[2] = ok ? cls[o.r32 + C::K + ch] : 0u;
    cp4[3] = ok ? cls[o.ahat + ch] : 0u;
    cb2[0] = ok ? cls[o.mmiinv + ch] : 0u;
    cb2[1] = ok ? cls[o.ub + ch] : 0u;
    cpx[0] = ok ? cls[o.ad + ch] : 0u;
    cpx[1] = ok ? cls[o.ubs + ch] : 0u;
    cpx[2] = ok ? cls[o.xpc + ch] : 0u;
    cpx[3] = ok ? cls[o.xpcs + ch] : 0u;
  }
  for (int idx = threadIdx.x; idx < C::IPB * C::XS; idx += blockDim.x) s[C::SM_XI + idx] = 0u;
}

// Thread roles of a tensor-core block (rns_tc.cuh): number n (0..31) and the number's lane t = 4 h + u,
// u the position in a group of four lanes.  TPI = 4: one warp per 8 numbers (h = 0).  TPI = 8: the two
// groups of four of number n sit in warps n / 8 (h = 0) and n / 8 + 4 (h = 1).
template <class C>
__device__ __forceinline__ int tc_number() {
  if constexpr (C::TPI == 8) return 8 * ((threadIdx.x >> 5) & 3) + ((threadIdx.x & 31) >> 2);
  else return (int)(threadIdx.x >> 2);
}
template <class C>
__device__ __forceinline__ int tc_half() {
  if constexpr (C::TPI == 8) return (int)(threadIdx.x >> 7);
  else return 0;
}
template <class C>
__device__ __forceinline__ int tc_lane_t() { return 4 * tc_half<C>() + (int)(threadIdx.x & 3); }

// Sum of v over a tensor-core block number's lanes; with two warp halves through `part` ([2][32]
// words of shared memory, two block barriers).  Every thread of the block calls it; shared-memory
// stores of the number's lanes before the call are visible to all of them after it.
template <class C>
__device__ __forceinline__ uint32_t tc_number_sum(uint32_t v, uint32_t* part) {
  if constexpr (C::TPI != 8) __syncwarp();
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  if constexpr (C::TPI == 8) {
    const int n = tc_number<C>(), h = tc_half<C>();
    __syncthreads();
    if ((threadIdx.x & 3) == 0) part[32 * h + n] = v;
    __syncthreads();
    v += part[32 * (1 - h) + n];
  }
  return v;
}

// Sum a value over the TPI lanes of this lane's group.
template <int TPI>
__device__ __forceinline__ uint32_t group_sum(uint32_t v) {
#pragma unroll
  for (int off = 1; off < TPI; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// acc[s] = sum_{i<k} xs[i] * T[i][slot s of lane t]  (64-bit, exact: k m^2 < 2^64)
template <class C>
__device__ __forceinline__ void ext_dot(uint64_t (&acc)[C::NPT], const uint32_t* xs, const uint32_t* T, int t) {
  constexpr int NPT = C::NPT, K = C::K;
#pragma unroll
  for (int s = 0; s < NPT; s++) acc[s] = 0;
#pragma unroll
  for (int i0 = 0; i0 < K; i0 += 4) {
    const uint4 x4 = *reinterpret_cast<const uint4*>(xs + i0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (i0 + q < K) {
        const uint32_t xv = q == 0 ? x4.x : q == 1 ? x4.y : q == 2 ? x4.z : x4.w;
        const uint32_t* row = T + (i0 + q) * C::ROW + t * C::LS;
        if constexpr (C::VEC == 4) {
#pragma unroll
          for (int s4 = 0; s4 < C::NPTP; s4 += 4) {
            const uint4 tv = *reinterpret_cast<const uint4*>(row + s4);
            if (s4 + 0 < NPT) acc[s4 + 0] = madw(xv, tv.x, acc[s4 + 0]);
            if (s4 + 1 < NPT) acc[s4 + 1] = madw(xv, tv.y, acc[s4 + 1]);
            if (s4 + 2 < NPT) acc[s4 + 2] = madw(xv, tv.z, acc[s4 + 2]);
            if (s4 + 3 < NPT) acc[s4 + 3] = madw(xv, tv.w, acc[s4 + 3]);
          }
        } else {
#pragma unroll
          for (int s2 = 0; s2 < C::NPTP; s2 += 2) {
            const uint2 tv = *reinterpret_cast<const uint2*>(row + s2);
            if (s2 + 0 < NPT) acc[s2 + 0] = madw(xv, tv.x, acc[s2 + 0]);
            if (s2 + 1 < NPT) acc[s2 + 1] = madw(xv, tv.y, acc[s2 + 1]);
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------------
// RNS Montgomery multiplication (Sec. 3.1, R = M): x <- x*y*M^-1 mod N, with
// outputs below (k+1)N for operands whose product is below 4(k+1)^2 2^L N.
//   xb, xp: hat residues of x in this lane's B and B' channels (in/out)
//   yb, yp: hat residues of y (may alias xb, xp for a squaring)
//   kxp:    |-N^-1 (M/m_i)^-1|_{m_i} 2^-32, kxs = floor(kxp 2^32 / m_i) (Shoup pair),
//   cmul:   |N M^-1|_{m'_j} hat                                          (per modulus)
//   xib, xpb: this number's xi / xi' exchange buffers in shared memory
// ------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ void mont_mul(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT], const uint32_t (&yb)[C::NPT],
                                         const uint32_t (&yp)[C::NPT], const uint32_t (&kxp)[C::NPT],
                                         const uint32_t (&kxs)[C::NPT], const uint32_t (&cmul)[C::NPT],
                                         const Smem<C>& sm, uint32_t* xib, uint32_t* xpb, int t) {
  constexpr int NPT = C::NPT, K = C::K;
  uint32_t sp[NPT];
  // 1-2. s = x*y in both bases; xi_i = s_i |-N^-1 (M/m_i)^-1| (plain CRT coefficients of q)
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    const uint4 cb = sm.cb4(t, s);
    const uint32_t sb = redc_lazy(mulw(xb[s], yb[s]), cb.x, cb.y);  // hat(s_i) in [0, 2m)
    // xi_i = hat(s_i) kxp mod m_i by Shoup's product: [0, 2m), one subtraction
    const uint32_t u = sb * kxp[s] - __umulhi(sb, kxs[s]) * cb.x;
    const uint32_t xi = min(u, u - cb.x);
    if (o < K) xib[o] = xi;
    const uint4 cp = sm.cp4(t, s);
    sp[s] = redc_lazy(mulw(xp[s], yp[s]), cp.x, cp.y);  // [0, 2m'): only multiplied again
  }
  __syncwarp();
  // 3. extension B -> B': qhat_j = sum_i xi_i |M/m_i|_{m'_j}   (k-term 64-bit dot products)
  uint64_t acc[NPT];
  ext_dot<C>(acc, xib, sm.T1(), t);
  // 4-5. r_j = s_j |M^-1| + qhat_j |N M^-1| (hat, the new B' residues), then xi'_j = r_j |(M'/m'_j)^-1|
  //      (plain) from hat(r_j) by Shoup's product with the constant xpc = |(M'/m'_j)^-1| 2^-32 and its
  //      quotient factor xpcs = floor(xpc 2^32 / m'_j): hat(r_j) xpc - floor(hat(r_j) xpcs / 2^32) m'_j
  //      lies in [0, 2m'_j) (one mad.hi and two mad.lo instead of two products and a reduction)
  uint32_t kaw = 0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    const uint4 cp = sm.cp4(t, s);
    const uint4 cx = sm.cpx(t, s);  // {ad, ubp, xpc, xpcs}
    uint32_t qh = redc64_lazy(acc[s], cp.x, cp.y, cp.z);  // [0, 2m'): only multiplied again
    xp[s] = redc(madw(sp[s], cp.w, mulw(qh, cmul[s])), cp.x, cp.y);
    const uint32_t u = xp[s] * cx.z - __umulhi(xp[s], cx.w) * cp.x;
    const uint32_t xpj = min(u, u - cp.x);
    if (o < K) xpb[o] = xpj;
    // xi'_j 2^Q / m'_j from the top bits: (xi' >> S) floor(2^(Q+S) / m'_j) is below it by less than
    // 2^(Q+S) / m'_j + xi' / 2^S units; over the k channels of a lane-group class (k <= 145, primes
    // above 2^27.4) that stays below 2^(Q-2), the margin of the 1/4 offset
    kaw += (xpj >> KAW_S) * cx.y;
  }
  __syncwarp();
  // 6. extension B' -> B, exact: a' = floor(sum xi'_j / m'_j) from the fixed-point sum with a 1/4 offset
  const uint32_t alpha = (group_sum<C::TPI>(kaw) + (1u << (KAW_Q - 2))) >> KAW_Q;
  ext_dot<C>(acc, xpb, sm.T2(), t);
  // r_i = t_i - a' |M'|_{m_i}  (hat, the new B residues): the correction enters the accumulator as
  // a' (m_i - mphh) before its one reduction (mphh = |M'| 2^64 mod m_i; the sum stays below
  // k m (m + 1) <= 2^64 - 1 for the class's primes)
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const uint4 cb = sm.cb4(t, s);
    xb[s] = redc64(madw(alpha, cb.x - cb.w, acc[s]), cb.x, cb.y, cb.z);
  }
}

// Binary -> hat residues of this lane's channels: x = sum_w X_w 2^(32w), read
// from `x` (nl limbs, limbs past nl are zero), with the class table P.
template <class C>
__device__ __forceinline__ void to_rns(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT], const uint32_t* x, int nl,
                                       const uint32_t* cls, const Smem<C>& sm, int t) {
  constexpr int NPT = C::NPT, K = C::K;
  const ClassOff co = class_offsets(C::K, C::W, C::WX);
  const uint32_t* P = cls + co.P;
  uint64_t ab[NPT], ap[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) ab[s] = ap[s] = 0;
  for (int w = 0; w < C::W; w++) {
    const uint32_t xw = w < nl ? x[w] : 0u;
    const uint32_t* prow = P + w * 2 * K;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int o = t * NPT + s;
      if (o < K) {
        ab[s] = madw(xw, __ldg(prow + o), ab[s]);
        ap[s] = madw(xw, __ldg(prow + K + o), ap[s]);
      }
    }
    if (w & 1) {  // keep the sums below 2^64: fold every two limbs
#pragma unroll
      for (int s = 0; s < NPT; s++) {
        const uint32_t rb = sm.cb4(t, s).z, rp = sm.cp4(t, s).z;
        ab[s] = madw(hi32(ab[s]), rb, lo32(ab[s]));
        ap[s] = madw(hi32(ap[s]), rp, lo32(ap[s]));
      }
    }
  }
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const uint4 cb = sm.cb4(t, s), cp = sm.cp4(t, s);
    xb[s] = redc64(ab[s], cb.x, cb.y, cb.z);
    xp[s] = redc64(ap[s], cp.x, cp.y, cp.z);
  }
}

// Load this lane's hat residues of an RNS vector laid out [B: k][B': k].
template <class C>
__device__ __forceinline__ void load_vec(uint32_t (&vb)[C::NPT], uint32_t (&vp)[C::NPT], const uint32_t* v, int t) {
#pragma unroll
  for (int s = 0; s < C::NPT; s++) {
    const int o = t * C::NPT + s;
    vb[s] = o < C::K ? __ldg(v + o) : 0u;
    vp[s] = o < C::K ? __ldg(v + C::K + o) : 0u;
  }
}

// (a + b) mod m channel-wise on hat residues in [0, m]
template <class C>
__device__ __forceinline__ void add_vec(uint32_t (&ab)[C::NPT], uint32_t (&ap)[C::NPT], const uint32_t (&bb)[C::NPT],
                                        const uint32_t (&bp)[C::NPT], const Smem<C>& sm, int t) {
#pragma unroll
  for (int s = 0; s < C::NPT; s++) {
    const uint32_t mb = sm.cb4(t, s).x, mp = sm.cp4(t, s).x;
    uint32_t u = ab[s] + bb[s];
    ab[s] = min(u, u - mb);
    uint32_t v = ap[s] + bp[s];
    ap[s] = min(v, v - mp);
  }
}

// a < b for little-endian numbers of na and nb limbs
__device__ __forceinline__ bool less_than(const uint32_t* a, int na, const uint32_t* b, int nb) {
  int n = na > nb ? na : nb;
  for (int i = n - 1; i >= 0; i--) {
    uint32_t av = i < na ? a[i] : 0u, bv = i < nb ? b[i] : 0u;
    if (av != bv) return av < bv;
  }
  return false;
}

// RNS (hat residues of a value X < (k+1) N, X < M/4) -> binary X mod N, written
// to dst[0..dst_limbs) (zero-padded).  CRT: X = sum_i xi_i (M/m_i) - a M with
// xi_i = |x_i (M/m_i)^-1|_{m_i}; a = floor(sum xi_i/m_i) from the fixed-point
// sum; then X mod N by a quotient estimate from the top bits and at most a few
// corrective subtractions.  All lanes of the group must call it; lane 0 of the
// group does the serial carry work.
// BLOCK = false: a lane group within one warp.  BLOCK = true: a tensor-core block (a number's lanes in
// two warps; every thread of the block calls it) with its [2][32]-word partial-sum area tc_part.
template <class C, bool BLOCK = false>
__device__ void from_rns_reduce(const uint32_t (&xb)[C::NPT], const uint32_t* cls, const uint32_t* key,
                                const Smem<C>& sm, uint32_t* xib, int t, uint32_t* dst, int dst_limbs, bool write,
                                uint32_t* tc_part = nullptr) {
  constexpr int NPT = C::NPT, K = C::K, WX = C::WX, W = C::W;
  const ClassOff co = class_offsets(C::K, C::W, C::WX);
  const KeyOff ko = key_offsets(C::K, C::W);
  uint32_t kaw = 0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    const uint4 cb = sm.cb4(t, s);
    const uint2 c2 = sm.cb2(t, s);
    uint32_t xi = redc(mulw(xb[s], c2.x), cb.x, cb.y);  // plain, [0, m)
    if (o < K) xib[o] = xi;
    kaw += hi32(mulw(xi, c2.y));
  }
  uint32_t kaw_sum;
  if constexpr (BLOCK) {
    kaw_sum = tc_number_sum<C>(kaw, tc_part);  // also publishes xib to the number's lanes
  } else {
    __syncwarp();
    kaw_sum = group_sum<C::TPI>(kaw);
  }
  const uint32_t alpha = (kaw_sum + (1u << (KAW_Q - 2))) >> KAW_Q;
  if (t == 0) {
    uint32_t X[WX];
    const uint32_t* MD = cls + co.MD;
    const uint32_t* ML = cls + co.ML;
    uint32_t c0 = 0, c1 = 0;
    for (int w = 0; w < WX; w++) {
      uint32_t s0 = c0, s1 = c1, s2 = 0;
      for (int i = 0; i < K; i++) mac96(s0, s1, s2, xib[i], __ldg(MD + i * WX + w));
      X[w] = s0;
      c0 = s1;
      c1 = s2;
    }
    // X -= alpha * M
    uint32_t carry = 0, br = 0;
    for (int w = 0; w < WX; w++) {
      uint64_t pw = mulw(alpha, __ldg(ML + w)) + carry;
      carry = hi32(pw);
      uint64_t d = (uint64_t)X[w] - lo32(pw) - br;
      X[w] = lo32(d);
      br = hi32(d) ? 1u : 0u;
    }
    // X mod N: X < (k+1) N
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
      for (int w = 0; w < WX; w++) {
        uint64_t pw = mulw((uint32_t)qe, w < W ? __ldg(N + w) : 0u) + cq;
        cq = hi32(pw);
        uint64_t d = (uint64_t)X[w] - lo32(pw) - b2;
        X[w] = lo32(d);
        b2 = hi32(d) ? 1u : 0u;
      }
    }
    for (int it = 0; it < 4; it++) {  // at most 2 are ever needed
      bool ge = true;
      for (int w = WX - 1; w >= 0; w--) {
        uint32_t nv = w < W ? __ldg(N + w) : 0u;
        if (X[w] != nv) {
          ge = X[w] > nv;
          break;
        }
      }
      if (!ge) break;
      uint32_t b3 = 0;
      for (int w = 0; w < WX; w++) {
        uint64_t d = (uint64_t)X[w] - (w < W ? __ldg(N + w) : 0u) - b3;
        X[w] = lo32(d);
        b3 = hi32(d) ? 1u : 0u;
      }
    }
    if (write)
      for (int w = 0; w < dst_limbs; w++) dst[w] = w < WX ? X[w] : 0u;
  }
  if constexpr (BLOCK) __syncthreads();
  else __syncwarp();
}

}  // namespace mr
