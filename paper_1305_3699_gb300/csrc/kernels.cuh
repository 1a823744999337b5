// Kernels of the RNS exponentiation path, templated on the size class.
//   modexp_kernel  x^e mod N per work item (Sec. 3.1: square-and-multiply chaining
//                  RNS Montgomery products inside the Montgomery domain, the
//                  window table precomputed outside the main loop)
//   crt_kernel     Garner recombination of RSA CRT halves (Sec. 3.3 defines d;
//                  the CRT split is the decryption form of the workload)
#pragma once
#include <cstdint>

#include "kernels_api.h"
#include "rns_device.cuh"
#include "rns_tc.cuh"

namespace mr {

__device__ __forceinline__ uint32_t exp_bits(const uint32_t* e, uint32_t el) {
  for (int w = (int)el - 1; w >= 0; w--) {
    uint32_t v = e[w];
    if (v) return 32u * w + 32u - __clz(v);
  }
  return 0;
}

__device__ __forceinline__ uint32_t exp_digit(const uint32_t* e, uint32_t el, uint32_t pos, uint32_t wb) {
  uint32_t l = pos >> 5, b = pos & 31;
  uint64_t v = (l < el ? e[l] : 0u) | ((uint64_t)(l + 1 < el ? e[l + 1] : 0u) << 32);
  return (uint32_t)(v >> b) & ((1u << wb) - 1u);
}

// Bits [i-31, i] of e (bit i in bit 31); positions below 0 read as zero.
__device__ __forceinline__ uint32_t exp_top32(const uint32_t* e, uint32_t el, int i) {
  const int lo = i - 31;
  const uint32_t p = (uint32_t)(lo > 0 ? lo : 0);
  const uint32_t l = p >> 5, b = p & 31;
  const uint64_t v = (l < el ? e[l] : 0u) | ((uint64_t)(l + 1 < el ? e[l + 1] : 0u) << 32);
  const uint32_t f = (uint32_t)(v >> b);  // bits [p, p + 32)
  return lo >= 0 ? f : f << (31 - i);
}

// Sliding window whose top bit is the set bit `top`: the up to ws bits [lo, top] trimmed to end
// on a set bit.  Returns the table index (value - 1) / 2 of the odd window value; *lo_out = lo.
__device__ __forceinline__ uint32_t slide_window(const uint32_t* e, uint32_t el, int top, int ws, int* lo_out) {
  int lo = max(top - ws + 1, 0);
  uint32_t v = exp_digit(e, el, (uint32_t)lo, (uint32_t)(top - lo + 1));
  const int tz = __ffs(v) - 1;  // v != 0: bit top is set
  v >>= tz;
  *lo_out = lo + tz;
  return (v - 1u) >> 1;
}

template <class C>
__device__ __forceinline__ void tab_store(uint32_t* wt, int ent, const uint32_t (&b)[C::NPT], const uint32_t (&p)[C::NPT],
                                          int lane) {
  uint32_t* base = wt + (size_t)ent * (2 * C::NPT) * 32 + lane;
#pragma unroll
  for (int s = 0; s < C::NPT; s++) {
    base[s * 32] = b[s];
    base[(C::NPT + s) * 32] = p[s];
  }
}

template <class C>
__device__ __forceinline__ void tab_load(const uint32_t* wt, int ent, uint32_t (&b)[C::NPT], uint32_t (&p)[C::NPT],
                                         int lane) {
  const uint32_t* base = wt + (size_t)ent * (2 * C::NPT) * 32 + lane;
#pragma unroll
  for (int s = 0; s < C::NPT; s++) {
    b[s] = base[s * 32];
    p[s] = base[(C::NPT + s) * 32];
  }
}

// Constant-time form: reads all E entries and keeps entry `ent` by masking, so that neither the
// addresses nor the branches depend on the (secret) index.
template <class C>
__device__ __forceinline__ void tab_load_ct(const uint32_t* wt, uint32_t ent, int E, uint32_t (&b)[C::NPT],
                                            uint32_t (&p)[C::NPT], int lane) {
#pragma unroll
  for (int s = 0; s < C::NPT; s++) b[s] = p[s] = 0u;
  for (int j = 0; j < E; j++) {
    const uint32_t mask = 0u - (uint32_t)((uint32_t)j == ent);  // all ones for the wanted entry
    const uint32_t* base = wt + (size_t)j * (2 * C::NPT) * 32 + lane;
#pragma unroll
    for (int s = 0; s < C::NPT; s++) {
      b[s] |= base[s * 32] & mask;
      p[s] |= base[(C::NPT + s) * 32] & mask;
    }
  }
}

// Table lookup of the exponentiation loop: masked over every entry when `ct`, else direct.
template <class C>
__device__ __forceinline__ void tab_get(const uint32_t* wt, uint32_t ent, int E, bool ct, uint32_t (&b)[C::NPT],
                                        uint32_t (&p)[C::NPT], int lane) {
  if (ct) tab_load_ct<C>(wt, ent, E, b, p, lane);
  else tab_load<C>(wt, (int)ent, b, p, lane);
}

// Schedule votes.  The integer form runs the numbers of a warp in lockstep; the tensor-core form
// (C::TC) runs the whole block in lockstep (every multiplication is a block-wide product), so its
// votes are block-wide.  All threads of the warp (block) must call them.
template <class C>
__device__ __forceinline__ bool vote_any(bool p) {
  if constexpr (C::TC) return __syncthreads_or(p) != 0;
  else return __any_sync(0xffffffffu, p);
}
template <class C>
__device__ __forceinline__ uint32_t vote_max(uint32_t v, const TcSmem<C>& ts) {
  v = __reduce_max_sync(0xffffffffu, v);
  if constexpr (C::TC) {
    uint32_t* word = ts.vote() + 4;
    __syncthreads();
    if (threadIdx.x == 0) *word = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(word, v);
    __syncthreads();
    v = *word;
  }
  return v;
}

// One RNS Montgomery multiplication in the kernel's form.
template <class C>
__device__ __forceinline__ void mm(uint32_t (&xb)[C::NPT], uint32_t (&xp)[C::NPT], const uint32_t (&yb)[C::NPT],
                                   const uint32_t (&yp)[C::NPT], const uint32_t (&kxp)[C::NPT],
                                   const uint32_t (&kxs)[C::NPT], const uint32_t (&cmul)[C::NPT], const Smem<C>& sm,
                                   uint32_t* xib, uint32_t* xpb, int t, const TcSmem<C>& ts, TcState& st) {
  if constexpr (C::TC) mont_mul_tc<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, ts, st, t);
  else mont_mul<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t);
}

// One exponentiation per lane group (x^e mod N of work item g_raw); all lanes of the warp (of the
// block, tensor-core form) call it together.  wt: this warp's window-table scratch.
template <class C>
__device__ __forceinline__ void modexp_item(const LaunchArgs& a, const Smem<C>& sm, uint32_t g_raw, uint32_t* wt,
                                            const TcSmem<C>& ts, TcState& st) {
  constexpr int NPT = C::NPT, TPI = C::TPI;
  const int lane = threadIdx.x & 31;
  // lane t of the number, the number's slot in the block, and the first lane of this thread's group
  // within its warp (the tensor-core block splits a number's 8 lanes over two warps, 4 in each)
  const int t = C::TC ? tc_lane_t<C>() : (int)(threadIdx.x % TPI);
  const int item_in_block = C::TC ? tc_number<C>() : (int)(threadIdx.x / TPI);
  const int glead = C::TC ? (lane & ~3) : lane - t;
  const bool leader = lane == glead;
  const bool live = g_raw < a.n_items;
  const uint32_t g = live ? g_raw : a.n_items - 1;  // idle groups shadow the last item, write nothing
  const MxItem it = reinterpret_cast<const MxItem*>(a.items)[g];
  const KeyOff ko = key_offsets(C::K, C::W);
  const uint32_t* key = it.key;
  uint32_t* xib = sm.xi(item_in_block);
  uint32_t* xpb = xib + C::KP;
  // input range check: x < xlim
  uint32_t bad = 0;
  if (leader) bad = less_than(it.x, it.x_limbs, it.xlim, it.xlim_limbs) ? 0u : 1u;
  bad = __shfl_sync(0xffffffffu, bad, glead);

  uint32_t kxp[NPT], kxs[NPT], cmul[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    kxp[s] = o < C::K ? __ldg(key + ko.kxp + o) : 0u;
    kxs[s] = o < C::K ? __ldg(key + ko.kxs + o) : 0u;
    cmul[s] = o < C::K ? __ldg(key + ko.cmul + o) : 0u;
  }

  // entry into the Montgomery domain: x~ = MM(x_lo, M^2 mod N) [+ MM(x_hi, 2^L M^2 mod N)]
  uint32_t xb[NPT], xp[NPT], yb[NPT], yp[NPT];
  const int nl0 = bad ? 0 : (int)(it.x_limbs < (uint32_t)C::W ? it.x_limbs : C::W);
  to_rns<C>(xb, xp, it.x, nl0, a.cls, sm, t);
  load_vec<C>(yb, yp, key + ko.r2, t);
  mm<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t, ts, st);
  const bool two = !bad && it.x_limbs > (uint32_t)C::W;
  if (vote_any<C>(two)) {
    uint32_t hb[NPT], hp[NPT];
    const int nl1 = two ? min((int)it.x_limbs - C::W, C::W) : 0;
    to_rns<C>(hb, hp, it.x + C::W, nl1, a.cls, sm, t);
    load_vec<C>(yb, yp, key + ko.r2h, t);
    mm<C>(hb, hp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t, ts, st);
    add_vec<C>(xb, xp, hb, hp, sm, t);
  }

  // Exponent schedule.  Groups of a warp run in lockstep, so the schedule must be the same for
  // all of them.  When every number of the warp has the same exponent (the halves of one RSA key,
  // sorted together by the host) and windows are long (wb >= 4), sliding windows of up to wb + 1
  // bits are used (left to right: a run of zero bits costs squarings only, a window starts and
  // ends on a set bit, so only odd powers are tabulated; about 4% fewer multiplications than fixed
  // windows for 1024-bit exponents, same table size).  Otherwise fixed wb-bit windows.
  // Constant-time calls (a.ct): a regular schedule that depends on no exponent bit -- fixed windows
  // over every limb of the exponent row, each window multiplied (entry 0 is the Montgomery form of
  // 1), table entries read by masking -- instead of the data-dependent shortcuts below.
  const bool ct = a.ct != 0;
  const int wb = (int)a.wbits, E = 1 << wb;
  const uint32_t el = it.e_limbs;
  uint32_t ebits = 0;
  if (leader) ebits = bad ? 0u : (ct ? 32u * el : exp_bits(it.e, el));
  ebits = __shfl_sync(0xffffffffu, ebits, glead);
  bool uni = false;
  if (wb >= 4 && !ct) {
    // the exponent of the first number of the warp (of the block, tensor-core form)
    const uint32_t* e0;
    uint32_t eb0;
    if constexpr (C::TC) {
      unsigned long long* vp = reinterpret_cast<unsigned long long*>(ts.vote());
      __syncthreads();
      if (threadIdx.x == 0) {
        vp[0] = reinterpret_cast<unsigned long long>(it.e);
        ts.vote()[2] = ebits;
      }
      __syncthreads();
      e0 = reinterpret_cast<const uint32_t*>(vp[0]);
      eb0 = ts.vote()[2];
    } else {
      e0 = reinterpret_cast<const uint32_t*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(it.e), 0));
      eb0 = __shfl_sync(0xffffffffu, ebits, 0);
    }
    int eq = ebits == eb0 && eb0 != 0u;
    if (eq && leader)
      for (uint32_t w = 0; w < (ebits + 31) / 32; w++)
        if (it.e[w] != e0[w]) {
          eq = 0;
          break;
        }
    eq = __shfl_sync(0xffffffffu, eq, glead);
    if constexpr (C::TC) uni = __syncthreads_and(eq) != 0;
    else uni = __all_sync(0xffffffffu, eq);
  }

  // The schedule flag is passed through an empty asm at each place it steers (the table, the
  // first window, the loop), so that the compiler cannot duplicate the code between them per
  // value of the flag (each copy would hold another inlined multiplication).
  int uni_t = uni ? 1 : 0, uni_f = uni ? 1 : 0;
  asm volatile("" : "+r"(uni_t), "+r"(uni_f));

  // window table.  Fixed windows: entry j = x~^j, entry 0 = 1 (Montgomery form M mod N).
  // Sliding windows: entry i = x~^(2i+1).  One multiplication site: the multiplier (y) is x~, or
  // x~^2 once the first product has formed it.
  if (!uni_t) {
    load_vec<C>(yb, yp, key + ko.one, t);
    tab_store<C>(wt, 0, yb, yp, lane);
  }
  tab_store<C>(wt, uni_t ? 0 : 1, xb, xp, lane);
  {
    uint32_t cb[NPT], cp[NPT];
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      cb[s] = xb[s];
      cp[s] = xp[s];
      yb[s] = xb[s];
      yp[s] = xp[s];
    }
    const int iters = uni_t ? E : E - 2;
    for (int j = 0; j < iters; j++) {
      mm<C>(cb, cp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t, ts, st);
      // opaque to the compiler: keeps one copy of the loop (no peeled first iteration)
      int first = (uni_t && j == 0) ? 1 : 0;
      asm volatile("" : "+r"(first));
      if (first) {
#pragma unroll
        for (int s = 0; s < NPT; s++) {  // y = x~^2; restart the products from x~
          yb[s] = cb[s];
          yp[s] = cp[s];
          cb[s] = xb[s];
          cp[s] = xp[s];
        }
      } else {
        tab_store<C>(wt, uni_t ? j : j + 2, cb, cp, lane);
      }
    }
  }

  // first window.  cur: sliding: bits below the current window still to process; fixed: index of
  // the next window.  Both schedules' values are formed and one is selected (no branch here, so
  // that the compiler keeps a single copy of the loop below).
  const int ws = wb + 1;  // sliding window width
  const uint32_t nwin = vote_max<C>((ebits + wb - 1) / wb, ts);
  const uint32_t d_fixed = (nwin && !bad) ? exp_digit(it.e, el, (nwin - 1) * wb, wb) : 0u;
  int lo_first = 0;
  const uint32_t d_slide = uni_f ? slide_window(it.e, el, (int)ebits - 1, ws, &lo_first) : 0u;
  uint32_t d = uni_f ? d_slide : d_fixed;
  int cur = uni_f ? lo_first : (int)nwin - 2;
  asm volatile("" : "+r"(cur), "+r"(d));  // opaque start values: the loop is not peeled
  __syncwarp();
  tab_get<C>(wt, d, E, ct, xb, xp, lane);
  // each step: nsq squarings (a squaring passes x as both operands), then, when the step has a
  // window (fixed: any number of the warp has a non-zero digit), one multiplication by its entry
  for (;;) {
    int nsq;
    bool mul;
    // opaque to the compiler: one copy of the loop body (no unswitched copy per schedule)
    int slide = uni ? 1 : 0;
    asm volatile("" : "+r"(slide));
    if (slide) {
      if (cur <= 0) break;
      const int i = cur - 1;
      int z = 0;  // zero bits from i down, 32 at a time
      for (;;) {
        if (i - z < 0) break;
        const uint32_t u = exp_top32(it.e, el, i - z);
        if (u) {
          z += __clz(u);
          break;
        }
        z += 32;
      }
      if (i - z < 0) {  // only zeros left: squarings
        nsq = cur;
        mul = false;
        cur = 0;
      } else {
        const int top = i - z;
        int lo;
        d = slide_window(it.e, el, top, ws, &lo);
        nsq = z + (top - lo + 1);
        mul = true;
        cur = lo;
      }
    } else {
      if (cur < 0) break;
      nsq = wb;
      d = bad ? 0u : exp_digit(it.e, el, (uint32_t)cur * wb, wb);
      mul = ct || vote_any<C>(d != 0);  // (ct is uniform: every lane takes the same path)
      cur--;
    }
    // one multiplication site for the squarings and the window product (the second operand is a
    // copy of x, or the table entry), so the loop holds a single copy of the multiplication code
    const int nmm = nsq + (mul ? 1 : 0);
    for (int q = 0; q < nmm; q++) {
      if (q < nsq) {
#pragma unroll
        for (int s = 0; s < NPT; s++) {
          yb[s] = xb[s];
          yp[s] = xp[s];
        }
      } else {
        tab_get<C>(wt, d, E, ct, yb, yp, lane);
      }
      mm<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t, ts, st);
    }
  }

  // leave the domain: MM(x, 1), then RNS -> binary, reduced into [0, N)
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    yb[s] = sm.cb4(t, s).z;  // hat form of 1 = 2^32 mod m
    yp[s] = sm.cp4(t, s).z;
  }
  mm<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t, ts, st);
  from_rns_reduce<C, C::TC != 0>(xb, a.cls, key, sm, xib, t, it.out, (int)it.out_limbs, live && !bad, ts.part());
  // tensor-core form: a completion wait that ran out leaves the block's results undefined (status 8)
  bool failed = false;
  if constexpr (C::TC) failed = *ts.abort_flag() != 0u;
  if (live && t == 0) {
    if (bad)
      for (uint32_t w = 0; w < it.out_limbs; w++) it.out[w] = 0u;
    if (a.status && it.status != 0xffffffffu) a.status[it.status] = bad ? 5u : (failed ? 8u : 0u);
  }
}

template <class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB) modexp_kernel(LaunchArgs a) {
  extern __shared__ __align__(128) uint32_t smem_raw[];
  Smem<C> sm{smem_raw};
  load_class_smem<C>(sm, a.cls);
  const TcSmem<C> ts{reinterpret_cast<uint8_t*>(smem_raw)};
  TcState st{0u, 0u, a.tc_skip};
  if constexpr (C::TC) tc_prologue<C>(ts, a.cls);
  __syncthreads();
  const int warp_global = (blockIdx.x * C::THREADS + threadIdx.x) >> 5;
  uint32_t* wt = a.scratch + (size_t)warp_global * ((size_t)1 << a.wbits) * (2 * C::NPT) * 32;
  if constexpr (C::TC) {
    // tensor-core form: the block runs its 32 numbers in lockstep.  Plain launch: block b runs item group
    // b; persistent launch: the block takes the next group of 32 items from the queue until it is empty
    tc::fence_after_sync();
    st.tmem = *ts.tslot();
    const uint32_t n_groups = (a.n_items + C::IPB - 1) / C::IPB;
    uint32_t bg = blockIdx.x;
    for (;;) {
      if (a.queue) {
        __syncthreads();
        if (threadIdx.x == 0) ts.vote()[6] = atomicAdd(a.queue, 1u);
        __syncthreads();
        bg = ts.vote()[6];
        if (bg >= n_groups) break;
      }
      modexp_item<C>(a, sm, bg * C::IPB + tc_number<C>(), wt, ts, st);
      if (!a.queue) break;
    }
    tc_release<C>(ts, st);
  } else {
    // plain launch: warp w of the grid runs group w once.  Persistent launch: each warp takes the
    // next group of 32/TPI items from the queue (items are ordered by cost, largest first) until it
    // is empty.  One call site for both keeps a single copy of the exponentiation code.
    const uint32_t n_groups = (a.n_items + C::IPW - 1) / C::IPW;
    const int lane = threadIdx.x & 31;
    for (;;) {
      uint32_t wg = (uint32_t)warp_global;
      if (a.queue) {
        if (lane == 0) wg = atomicAdd(a.queue, 1u);
        wg = __shfl_sync(0xffffffffu, wg, 0);
        if (wg >= n_groups) break;
      }
      modexp_item<C>(a, sm, wg * C::IPW + (lane / C::TPI), wt, ts, st);
      if (!a.queue) break;
    }
  }
}

template <class C>
__global__ void __launch_bounds__(C::THREADS) crt_kernel(LaunchArgs a) {
  extern __shared__ __align__(16) uint32_t smem_raw[];
  Smem<C> sm{smem_raw};
  load_class_smem<C>(sm, a.cls);
  __syncthreads();

  constexpr int NPT = C::NPT, TPI = C::TPI, W = C::W;
  const int t = threadIdx.x % TPI;
  const int item_in_block = threadIdx.x / TPI;
  const uint32_t g_raw = blockIdx.x * C::IPB + item_in_block;
  const bool live = g_raw < a.n_items;
  const uint32_t g = live ? g_raw : a.n_items - 1;
  const CrtItem it = reinterpret_cast<const CrtItem*>(a.items)[g];
  const KeyOff ko = key_offsets(C::K, C::W);
  const CrtOff cro = crt_offsets(C::K, C::W);
  const uint32_t* key = it.keyp;
  uint32_t* xib = sm.xi(item_in_block);
  uint32_t* xpb = xib + C::KP;

  uint32_t kxp[NPT], kxs[NPT], cmul[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    kxp[s] = o < C::K ? __ldg(key + ko.kxp + o) : 0u;
    kxs[s] = o < C::K ? __ldg(key + ko.kxs + o) : 0u;
    cmul[s] = o < C::K ? __ldg(key + ko.cmul + o) : 0u;
  }
  // d = m_p + P2 - m_q  (a positive integer below 3 * 2^L, congruent to m_p - m_q mod p)
  uint32_t db[NPT], dp[NPT], qb[NPT], qp[NPT], yb[NPT], yp[NPT];
  to_rns<C>(db, dp, it.mp, W, a.cls, sm, t);
  to_rns<C>(qb, qp, it.mq, W, a.cls, sm, t);
  load_vec<C>(yb, yp, it.crt + cro.p2, t);
  add_vec<C>(db, dp, yb, yp, sm, t);
#pragma unroll
  for (int s = 0; s < NPT; s++) {  // subtract m_q: d + m - q lies in [0, 2m]
    const uint32_t mb = sm.cb4(t, s).x, mp = sm.cp4(t, s).x;
    uint32_t u = db[s] + mb - qb[s];
    db[s] = min(u, u - mb);
    uint32_t v = dp[s] + mp - qp[s];
    dp[s] = min(v, v - mp);
  }
  // h = MM(d, qinv M mod p) = d qinv mod p, then to binary in [0, p)
  load_vec<C>(yb, yp, it.crt + cro.qm, t);
  mont_mul<C>(db, dp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t);
  uint32_t h[W];
  from_rns_reduce<C>(db, a.cls, key, sm, xib, t, h, W, true);
  // m = m_q + h q  (2W limbs)
  if (live && t == 0) {
    const uint32_t* q = it.crt + cro.q;
    const int ol = (int)it.out_limbs;
    // column-wise schoolbook with a 96-bit column accumulator
    uint32_t c0 = 0, c1 = 0;
    for (int w = 0; w < 2 * W; w++) {
      uint32_t s0 = c0, s1 = c1, s2 = 0;
      int ilo = w - (W - 1) > 0 ? w - (W - 1) : 0;
      int ihi = w < W - 1 ? w : W - 1;
      for (int i = ilo; i <= ihi; i++) mac96(s0, s1, s2, h[i], __ldg(q + (w - i)));
      if (w < W) {  // + m_q
        uint32_t mqw = it.mq[w];
        asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, %2, 0;"
            : "+r"(s0), "+r"(s1), "+r"(s2)
            : "r"(mqw));
      }
      if (w < ol) it.out[w] = s0;
      c0 = s1;
      c1 = s2;
    }
    for (int w = 2 * W; w < ol; w++) it.out[w] = 0u;
  }
}

}  // namespace mr
