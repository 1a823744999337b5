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

namespace mr {

template <int K_, int W_, int WX_, int NPT_, int NW_>
struct BigCfg {
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
  static constexpr size_t TAB = KAWG + (size_t)SLICES * 32;
  MR_HD static constexpr size_t slot_words(uint32_t wbits) { return TAB + ((size_t)1 << wbits) * 2 * K * 32; }
  static_assert(NPT == 4, "four channels per thread and base (one 16-byte matrix load per row)");
  static_assert((SM_X % 4) == 0 && (SM_C4A % 4) == 0 && (SC % 4) == 0 && (SM_MBAR % 4) == 0, "alignment");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
  static_assert(K * 32 <= 2 * K * SC, "RNS -> binary stages all k rows in the matrix area");
};

template <class C>
struct BigGroup {
  uint32_t* s;         // shared memory
  uint32_t* slot;      // this slot's global scratch
  uint32_t* ctr;       // this slot's barrier counter
  uint32_t* abort;     // launch-wide abort flag
  uint32_t nbar;       // barriers passed so far (target = nbar * SLICES)
  uint32_t spin_limit; // polls before a wait gives up
  uint32_t ph;         // parity bits of the two staging mbarriers
  int c, w, lane;
  __device__ uint4 a4(int q) const { return reinterpret_cast<const uint4*>(s + C::SM_C4A)[q]; }
  __device__ uint4 b4(int q) const { return reinterpret_cast<const uint4*>(s + C::SM_C4B)[q]; }
  __device__ uint2 a2(int q) const { return reinterpret_cast<const uint2*>(s + C::SM_C2A)[q]; }
  __device__ uint2 b2(int q) const { return reinterpret_cast<const uint2*>(s + C::SM_C2B)[q]; }

  // All CTAs of the slot meet; false when the wait ran out or another CTA aborted.
  __device__ bool barrier() {
    nbar++;
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
        __nanosleep(it < 64 ? 32 : 256);
      }
      s[C::SM_MISC] = ok;
    }
    __syncthreads();
    return s[C::SM_MISC] != 0;
  }

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

// RNS Montgomery multiplication x <- x*y*M^-1 mod N (outputs below (k+1)N), this thread's channels.
template <class C>
__device__ bool big_mont_mul(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT], const uint32_t (&yb)[C::NPT],
                             const uint32_t (&yp)[C::NPT], const uint32_t (&kxi)[C::NPT],
                             const uint32_t (&cmul)[C::NPT], const uint32_t (&cd)[C::NPT], BigGroup<C>& g) {
  constexpr int NPT = C::NPT, K = C::K;
  uint32_t* Xg = g.slot + C::XG;
  uint32_t* XPg = g.slot + C::XPG;
  uint32_t* KAWg = g.slot + C::KAWG;
  uint32_t sp[NPT];
  // 1-2. s = x*y in both bases; xi_i = s_i |-N^-1 (M/m_i)^-1| to the exchange buffer
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s, o = g.c * C::SC + q;
    const uint4 cb = g.a4(q);
    uint32_t sb = redc_lazy(mulw(xb[s], yb[s]), cb.x, cb.y);  // [0, 2m): only multiplied again
    uint32_t xi = redc(mulw(sb, kxi[s]), cb.x, cb.y);
    if (o < K) Xg[(size_t)o * 32 + g.lane] = xi;
    const uint4 cp = g.b4(q);
    sp[s] = redc_lazy(mulw(xp[s], yp[s]), cp.x, cp.y);
  }
  if (!g.barrier()) return false;
  // 3. extension B -> B'
  uint64_t acc[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) acc[s] = 0;
  if (!big_ext<C>(acc, g, Xg, g.s + C::SM_T1)) return false;
  // 4-5. new B' residues and xi'_j; partial correction-factor sums
  uint32_t kaw = 0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int q = g.w * NPT + s, o = g.c * C::SC + q;
    const uint4 cp = g.b4(q);
    const uint2 c2 = g.b2(q);
    uint32_t qh = redc64_lazy(acc[s], cp.x, cp.y, cp.z);
    xp[s] = redc(madw(sp[s], cp.w, mulw(qh, cmul[s])), cp.x, cp.y);
    uint32_t xpj = redc(madw(sp[s], c2.x, mulw(qh, cd[s])), cp.x, cp.y);
    if (o < K) XPg[(size_t)o * 32 + g.lane] = xpj;
    kaw += hi32(mulw(xpj, c2.y));  // zero on padding slots (ubp = 0)
  }
  g.s[C::SM_KAW + g.w * 32 + g.lane] = kaw;
  __syncthreads();
  if (g.w == 0) {
    uint32_t v = 0;
#pragma unroll
    for (int u = 0; u < C::NW; u++) v += g.s[C::SM_KAW + u * 32 + g.lane];
    KAWg[g.c * 32 + g.lane] = v;
  }
  if (!g.barrier()) return false;
  // 6. exact extension B' -> B with a' from the slice partials (loaded before the dot products,
  //    summed after them); the correction -a'|M'| enters as a' E with E = -M' 2^64 mod m_i
  uint32_t kp[C::SLICES];
#pragma unroll
  for (int u = 0; u < C::SLICES; u++) kp[u] = __ldcg(KAWg + u * 32 + g.lane);
#pragma unroll
  for (int s = 0; s < NPT; s++) acc[s] = 0;
  if (!big_ext<C>(acc, g, XPg, g.s + C::SM_T2)) return false;
  uint32_t ks = 0;
#pragma unroll
  for (int u = 0; u < C::SLICES; u++) ks += kp[u];
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
  for (int u = 0; u < C::SLICES; u++) ks += __ldcg(g.slot + C::KAWG + u * 32 + g.lane);
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
    g.slot[C::KAWG + g.c * 32 + g.lane] = v;
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
  g.nbar = 0;
  g.spin_limit = a.spin_limit;
  g.ph = 0;
  if (g.c == a.absent_slice) return;  // test hook: this slice never arrives; the others time out
  if (threadIdx.x == 0) {
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem_raw + C::SM_MBAR);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mb[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mb[1])));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  big_load_consts<C>(smem_raw, a.cls, g.c);
  const uint32_t n_groups = (a.n_items + 31) / 32;
  uint32_t grp = slot_id;
  for (; grp < n_groups; grp += a.slots) {
    big_load_smem<C>(smem_raw, a.cls, a.tslice, g.c);
    __syncthreads();
    if (!big_modexp_group<C>(a, g, grp)) break;
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
