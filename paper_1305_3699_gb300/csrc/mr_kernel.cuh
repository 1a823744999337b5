// Miller-Rabin rounds on the GPU (Sec. 3.2: primality testing in the Montgomery
// domain, with a caller-chosen number of iterations; the candidates never leave
// the device).
//
// Per candidate N (one group of TPI lanes):
//   1. lane 0 derives M mod N and M^2 mod N by long division (Knuth's
//      Algorithm D on 32-bit limbs) and writes them, with N - (M mod N), to the
//      candidate's scratch row;
//   2. every lane turns N into residues and derives its channels' constants:
//      N^-1 mod m_i (Fermat, in Montgomery form), -N^-1 (M/m_i)^-1 and N M^-1;
//   3. per round: y~ = (a M)^d with n - 1 = 2^s d by the same fixed-window loop
//      as the exponentiation kernel (the digits of d are read straight from N's
//      limbs shifted by s), then the tests y = +-1 and the s - 1 squarings.
// The tests stay in RNS: for v < (k+2) N, v = 0 (mod N) exactly when
// v N^-1 mod m_c is the same integer j <= k+1 in every channel (then v = jN), so
// "y == 1" is a zero test of y~ + (N - M mod N) and "y == -1" of y~ + (M mod N).
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace mr {

// r = a mod n (lane-local; a: na limbs, n: nn limbs with n[nn-1] != 0, nn <= NMAX,
// na <= AMAX).  Knuth's Algorithm D with 32-bit digits.
template <int AMAX, int NMAX>
__device__ __noinline__ void bn_mod(const uint32_t* a, int na, const uint32_t* n, int nn, uint32_t* r) {
  if (nn == 1) {
    uint64_t rem = 0;
    for (int i = na - 1; i >= 0; i--) rem = ((rem << 32) | a[i]) % n[0];
    r[0] = (uint32_t)rem;
    return;
  }
  if (na < nn) {
    for (int i = 0; i < nn; i++) r[i] = i < na ? a[i] : 0u;
    return;
  }
  uint32_t u[AMAX + 1], v[NMAX];
  const int sh = __clz(n[nn - 1]);
  for (int i = nn - 1; i >= 0; i--) v[i] = (n[i] << sh) | (sh && i > 0 ? n[i - 1] >> (32 - sh) : 0u);
  u[na] = sh ? a[na - 1] >> (32 - sh) : 0u;
  for (int i = na - 1; i >= 0; i--) u[i] = (a[i] << sh) | (sh && i > 0 ? a[i - 1] >> (32 - sh) : 0u);
  const uint64_t vtop = v[nn - 1], vnext = v[nn - 2];
  for (int j = na - nn; j >= 0; j--) {
    const uint64_t num = ((uint64_t)u[j + nn] << 32) | u[j + nn - 1];
    uint64_t qhat = num / vtop, rhat = num % vtop;
    while (qhat > 0xffffffffull || qhat * vnext > ((rhat << 32) | u[j + nn - 2])) {
      qhat--;
      rhat += vtop;
      if (rhat > 0xffffffffull) break;
    }
    // u[j..j+nn] -= qhat * v
    uint64_t carry = 0;
    int64_t borrow = 0;
    for (int i = 0; i < nn; i++) {
      uint64_t p = qhat * v[i] + carry;
      carry = p >> 32;
      int64_t t = (int64_t)u[i + j] - (int64_t)(uint32_t)p - borrow;
      u[i + j] = (uint32_t)t;
      borrow = t < 0 ? 1 : 0;
    }
    int64_t t = (int64_t)u[j + nn] - (int64_t)carry - borrow;
    u[j + nn] = (uint32_t)t;
    if (t < 0) {  // qhat was one too large: add v back
      uint64_t c = 0;
      for (int i = 0; i < nn; i++) {
        uint64_t s = (uint64_t)u[i + j] + v[i] + c;
        u[i + j] = (uint32_t)s;
        c = s >> 32;
      }
      u[j + nn] += (uint32_t)c;
    }
  }
  for (int i = 0; i < nn; i++) r[i] = (u[i] >> sh) | (sh ? u[i + 1] << (32 - sh) : 0u);
}

// All lanes of the group: is v (hat residues, value < (k+2) N) a multiple of N?
template <class C>
__device__ __forceinline__ bool rns_is_zero_mod_n(const uint32_t (&vb)[C::NPT], const uint32_t (&vp)[C::NPT],
                                                  const uint32_t (&invb)[C::NPT], const uint32_t (&invp)[C::NPT],
                                                  const Smem<C>& sm, int t, int lane) {
  constexpr int NPT = C::NPT, K = C::K;
  uint32_t j = 0xffffffffu;
  bool ok = true;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    if (o < K) {
      const uint4 cb = sm.cb4(t, s), cp = sm.cp4(t, s);
      uint32_t ub = redc(mulw(vb[s], invb[s]), cb.x, cb.y);
      uint32_t up = redc(mulw(vp[s], invp[s]), cp.x, cp.y);
      if (j == 0xffffffffu) j = ub;
      ok = ok && ub == j && up == j;
    }
  }
  // every lane of the group must see the same j (lane 0 of the group always owns channels;
  // a lane whose slots are all padding has nothing to compare)
  const uint32_t j0 = __shfl_sync(0xffffffffu, j, lane - t);
  ok = ok && (j == 0xffffffffu || j == j0) && j0 <= (uint32_t)K + 1;
  const unsigned grp = C::TPI == 32 ? 0xffffffffu : (((1u << (C::TPI & 31)) - 1u) << (lane - t));
  const unsigned vote = __ballot_sync(0xffffffffu, ok) & grp;
  return vote == grp;
}

template <class C>
__global__ void __launch_bounds__(C::THREADS) mr_kernel(MRArgs a) {
  extern __shared__ __align__(16) uint32_t smem_raw[];
  Smem<C> sm{smem_raw};
  load_class_smem<C>(sm, a.cls);
  __syncthreads();

  constexpr int NPT = C::NPT, TPI = C::TPI, K = C::K, W = C::W, WX = C::WX;
  const ClassOff co = class_offsets(C::K, C::W, C::WX);
  const int lane = threadIdx.x & 31;
  const int t = threadIdx.x % TPI;
  const int item_in_block = threadIdx.x / TPI;
  const uint32_t g_raw = blockIdx.x * C::IPB + item_in_block;
  // with a selection the item count is on the device (candidates that passed trial division)
  const uint32_t n_items = a.sel ? min(a.n, *a.n_sel * a.per) : a.n;
  if (n_items == 0) return;  // uniform: every thread of the launch reads the same count
  const bool live = g_raw < n_items;
  const uint32_t g = live ? g_raw : n_items - 1;
  const uint32_t nl = a.n_limbs;
  // item g: candidate g / per (or sel[g / per]); rounds [r0, r1) (all of them when per = 1, round
  // g % per otherwise)
  const uint32_t cidx = a.sel ? a.sel[g / a.per] : g / a.per;
  const uint32_t r0 = a.per == 1 ? 0u : g % a.per, r1 = a.per == 1 ? a.rounds : r0 + 1;
  const uint32_t* N = a.cand + (size_t)cidx * nl;
  uint32_t* crow = a.crow + (size_t)g * 3 * W;
  uint32_t* xib = sm.xi(item_in_block);
  uint32_t* xpb = xib + C::KP;
  const int warp_global = (blockIdx.x * C::THREADS + threadIdx.x) >> 5;
  uint32_t* wt = a.scratch + (size_t)warp_global * ((size_t)1 << a.wbits) * (2 * NPT) * 32;

  // 1. lane 0: special cases, s, M mod N, M^2 mod N, N - (M mod N)
  // special: 0 = RNS test, 1 = composite by definition (N < 2 or even N > 2), 2 = N is 2,
  // 3 = N > 2^31 shares a channel prime (composite: it has that prime as a factor),
  // 5 = N < 2^31, tested in 64-bit scalar arithmetic by lane 0
  uint32_t special = 0;
  uint32_t sbits = 0, nbits = 0, dbg_one0 = 0;
  if (t == 0 && live) {  // idle groups (shadowing the last candidate) must not write its scratch row
    int nn = (int)nl;
    while (nn > 0 && N[nn - 1] == 0) nn--;
    nbits = nn ? 32u * (nn - 1) + 32u - __clz(N[nn - 1]) : 0u;
    if (nbits <= 1) special = 1u;                             // 0 and 1
    else if ((N[0] & 1u) == 0) special = (nbits == 2 && N[0] == 2u) ? 2u : 1u;
    else if (nbits <= 31) special = 5u;
    if (!special) {
      while (((N[sbits >> 5] >> (sbits & 31)) & 1u) == 0 || sbits == 0) sbits++;  // N - 1 = 2^s d, s >= 1
      // M mod N and M^2 mod N go straight to the candidate's scratch row
      uint32_t* one = crow;
      uint32_t* r2 = crow + W;
      {
        uint32_t Ml[WX];
        for (int i = 0; i < WX; i++) Ml[i] = __ldg(a.cls + co.ML + i);
        int ma = WX;
        while (ma > 0 && Ml[ma - 1] == 0) ma--;
        bn_mod<WX, W>(Ml, ma, N, nn, one);
      }
      for (int i = nn; i < W; i++) one[i] = 0u;
      {
        uint32_t sq[2 * W];
        for (int i = 0; i < 2 * nn; i++) sq[i] = 0u;
        for (int i = 0; i < nn; i++) {
          uint64_t c = 0;
          const uint64_t oi = one[i];
          for (int j = 0; j < nn; j++) {
            uint64_t p = oi * one[j] + sq[i + j] + c;
            sq[i + j] = (uint32_t)p;
            c = p >> 32;
          }
          sq[i + nn] = (uint32_t)c;
        }
        bn_mod<2 * W, W>(sq, 2 * nn, N, nn, r2);
      }
      for (int i = nn; i < W; i++) r2[i] = 0u;
      dbg_one0 = one[0];
      uint32_t br = 0;
      for (int i = 0; i < W; i++) {
        uint32_t nv = i < nn ? N[i] : 0u;
        uint64_t d = (uint64_t)nv - one[i] - br;
        crow[2 * W + i] = (uint32_t)d;
        br = (uint32_t)(d >> 63);
      }
    }
  }
  special = __shfl_sync(0xffffffffu, special, lane - t);
  sbits = __shfl_sync(0xffffffffu, sbits, lane - t);
  nbits = __shfl_sync(0xffffffffu, nbits, lane - t);
  __syncwarp();

  // 2. residues of N and the per-channel constants
  uint32_t nb[NPT], np[NPT], kxi[NPT], kxp[NPT], kxs[NPT], cmul[NPT], cd[NPT], invb[NPT], invp[NPT];
  to_rns<C>(nb, np, N, special ? 0 : (int)min(nl, (uint32_t)W), a.cls, sm, t);
  bool coprime = true;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int o = t * NPT + s;
    const uint4 cb = sm.cb4(t, s), cp = sm.cp4(t, s);
    const uint2 c2 = sm.cb2(t, s);
    // N^-1 mod m by Fermat (x^(m-2)), in Montgomery form; hat(1) = 2^32 mod m
    uint32_t ib = cb.z, ip = cp.z, bb = nb[s], bp = np[s];
    const uint32_t eb = cb.x - 2u, ep = cp.x - 2u;
    for (int bit = 0; bit < 31; bit++) {
      if ((eb >> bit) & 1u) ib = redc(mulw(ib, bb), cb.x, cb.y);
      if ((ep >> bit) & 1u) ip = redc(mulw(ip, bp), cp.x, cp.y);
      bb = redc(mulw(bb, bb), cb.x, cb.y);
      bp = redc(mulw(bp, bp), cp.x, cp.y);
    }
    invb[s] = redc(mulw(ib, 1u), cb.x, cb.y);  // plain
    invp[s] = redc(mulw(ip, 1u), cp.x, cp.y);
    if (o < K && (redc(mulw(nb[s], 1u), cb.x, cb.y) == 0 || redc(mulw(np[s], 1u), cp.x, cp.y) == 0))
      coprime = false;
    // |-N^-1 (M/m_i)^-1|_{m_i} plain = REDC(hat(-N^-1) * |(M/m_i)^-1|)
    const uint32_t nib = ib == 0 ? 0u : cb.x - ib;
    kxi[s] = redc(mulw(nib, c2.x), cb.x, cb.y);
    // Shoup pair of the multiplication: kxp = kxi 2^-32 mod m_i, kxs = floor(kxp 2^32 / m_i)
    kxp[s] = redc(kxi[s], cb.x, cb.y);
    kxs[s] = cb.x ? (uint32_t)(((uint64_t)kxp[s] << 32) / cb.x) : 0u;
    // |N M^-1|_{m'_j} hat = REDC(hat(N) * hat(M^-1)); |N M^-1 (M'/m'_j)^-1| plain = REDC(hat(N) * ad)
    cmul[s] = redc(mulw(np[s], cp.w), cp.x, cp.y);
    cd[s] = redc(mulw(np[s], sm.cpx(t, s).x), cp.x, cp.y);  // published by the test hook only
  }
  {
    const unsigned grp = C::TPI == 32 ? 0xffffffffu : (((1u << (C::TPI & 31)) - 1u) << (lane - t));
    const unsigned nc = __ballot_sync(0xffffffffu, !coprime) & grp;
    if (nc && !special) special = 3u;  // N shares a channel prime
  }

  if (a.dbg) {  // test hook: publish the derived constants of this candidate
    uint32_t* dg = a.dbg + (size_t)g * mr_debug_words(K, W);
    if (live && t == 0) {
      dg[0] = special;
      dg[1] = sbits;
      dg[2] = nbits;
      dg[3] = dbg_one0;
      for (int i = 0; i < 2 * W; i++) dg[4 + i] = special ? 0u : crow[i];
    }
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int o = t * NPT + s;
      if (live && o < K) {
        const uint4 cp = sm.cp4(t, s);
        dg[4 + 2 * W + o] = kxi[s];
        dg[4 + 2 * W + K + o] = redc(mulw(cmul[s], 1u), cp.x, cp.y);
        dg[4 + 2 * W + 2 * K + o] = cd[s];
        dg[4 + 2 * W + 3 * K + o] = invb[s];
        dg[4 + 2 * W + 4 * K + o] = invp[s];
      }
    }
  }

  // hat residues of M mod N (= 1 in the domain), M^2 mod N (entry), N - (M mod N)
  uint32_t oneb[NPT], onep[NPT], nmob[NPT], nmop[NPT], r2b[NPT], r2p[NPT];
  __syncwarp();
  const int cl = special ? 0 : W;
  to_rns<C>(oneb, onep, crow, cl, a.cls, sm, t);
  to_rns<C>(r2b, r2p, crow + W, cl, a.cls, sm, t);
  to_rns<C>(nmob, nmop, crow + 2 * W, cl, a.cls, sm, t);

  const int wb = (int)a.wbits, E = 1 << wb;
  const uint32_t dbits = special ? 0u : nbits - sbits;
  const uint32_t my_s = special ? 0u : sbits;
  const uint32_t nwin = __reduce_max_sync(0xffffffffu, (dbits + wb - 1) / wb);
  uint32_t mask = 0;
  bool all_pass = true;
  for (uint32_t r = r0; r < r1; r++) {
    const uint32_t* wit = a.witness + ((size_t)cidx * a.rounds + r) * nl;
    uint32_t xb[NPT], xp[NPT], yb[NPT], yp[NPT];
    to_rns<C>(xb, xp, wit, special ? 0 : (int)min(nl, (uint32_t)W), a.cls, sm, t);
    mont_mul<C>(xb, xp, r2b, r2p, kxp, kxs, cmul, sm, xib, xpb, t);  // a~ = a M mod N
    tab_store<C>(wt, 0, oneb, onep, lane);
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
    // y~ = a~^d; the digits of d = (N - 1) >> s are the bits of N from position s up
    // (N - 1 and N differ only in bit 0, and s >= 1); bits above N's top are zero
    uint32_t d = (nwin && !special) ? exp_digit(N, nl, sbits + (nwin - 1) * (uint32_t)wb, (uint32_t)wb) : 0u;
    __syncwarp();
    tab_load<C>(wt, d, xb, xp, lane);
    for (int widx = (int)nwin - 2; widx >= 0; widx--) {
      for (int q = 0; q < wb; q++) mont_mul<C>(xb, xp, xb, xp, kxp, kxs, cmul, sm, xib, xpb, t);
      d = special ? 0u : exp_digit(N, nl, sbits + (uint32_t)widx * wb, (uint32_t)wb);
      if (__any_sync(0xffffffffu, d != 0)) {
        tab_load<C>(wt, d, yb, yp, lane);
        mont_mul<C>(xb, xp, yb, yp, kxp, kxs, cmul, sm, xib, xpb, t);
      }
    }
    // y == 1: y~ + (N - M mod N) is a multiple of N
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const uint32_t mb = sm.cb4(t, s).x, mp = sm.cp4(t, s).x;
      uint32_t u = xb[s] + nmob[s];
      yb[s] = min(u, u - mb);
      u = xp[s] + nmop[s];
      yp[s] = min(u, u - mp);
    }
    bool pass = rns_is_zero_mod_n<C>(yb, yp, invb, invp, sm, t, lane);
    // y^(2^i) == -1 for some 0 <= i < s: y~ + (M mod N) is a multiple of N
    for (uint32_t i = 0;; i++) {
#pragma unroll
      for (int s = 0; s < NPT; s++) {
        const uint32_t mb = sm.cb4(t, s).x, mp = sm.cp4(t, s).x;
        uint32_t u = xb[s] + oneb[s];
        yb[s] = min(u, u - mb);
        u = xp[s] + onep[s];
        yp[s] = min(u, u - mp);
      }
      const bool m1 = rns_is_zero_mod_n<C>(yb, yp, invb, invp, sm, t, lane);
      if (i < my_s && m1) pass = true;
      const bool finished = pass || i + 1 >= my_s;
      if (__all_sync(0xffffffffu, finished)) break;
      mont_mul<C>(xb, xp, xb, xp, kxp, kxs, cmul, sm, xib, xpb, t);
    }
    if (pass && r < 32) mask |= 1u << r;
    all_pass = all_pass && pass;
  }
  if (live && t == 0) {
    uint8_t prime = all_pass ? 1 : 0;
    uint32_t m = mask;
    uint32_t all_rounds = 0;  // this item's rounds below 32
    for (uint32_t r = r0; r < r1 && r < 32; r++) all_rounds |= 1u << r;
    if (special == 1u || special == 3u) {
      prime = 0;
      m = 0;
    } else if (special == 2u) {
      prime = 1;
      m = all_rounds;
    } else if (special == 5u) {
      // small odd N: the same test in 64-bit arithmetic
      const uint64_t n64 = N[0];
      uint32_t s5 = 1;
      while (((n64 - 1) >> s5 & 1u) == 0) s5++;
      const uint64_t d5 = (n64 - 1) >> s5;
      prime = 1;
      m = 0;
      for (uint32_t r = r0; r < r1; r++) {
        const uint32_t* wit = a.witness + ((size_t)cidx * a.rounds + r) * nl;
        uint64_t w = 0;
        for (int i = (int)nl - 1; i >= 0; i--) w = ((w << 32) | wit[i]) % n64;
        uint64_t y = 1 % n64, b = w, e = d5;
        while (e) {
          if (e & 1) y = y * b % n64;
          b = b * b % n64;
          e >>= 1;
        }
        bool pass = y == 1 || y == n64 - 1;
        for (uint32_t i = 1; i < s5 && !pass; i++) {
          y = y * y % n64;
          if (y == n64 - 1) pass = true;
        }
        if (pass && r < 32) m |= 1u << r;
        if (!pass) prime = 0;
      }
    }
    a.is_prime[g] = prime;  // per = rounds: this round's verdict, combined per candidate afterwards
    if (a.round_mask && a.per == 1) a.round_mask[g] = m;
  }
}

}  // namespace mr
