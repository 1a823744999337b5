// Host-visible description of the compiled kernels of each size class.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "layout.h"

namespace mr {

struct LaunchArgs {
  const uint32_t* cls;   // class table block (device)
  const void* items;     // MxItem[] or CrtItem[] (device)
  uint32_t n_items;
  uint32_t wbits;        // window width (modexp), 1..6
  uint32_t* scratch;     // window tables (modexp): per warp (1 << wbits) x 2 NPT x 32 words
  uint8_t* status;       // per-item status bytes or nullptr
  uint32_t* queue;       // persistent mode: work-group counter (zeroed before the launch), else nullptr
  uint32_t ct;           // modexp: 1 = constant-time schedule (regular fixed windows over every exponent
                         // limb, every window multiplied, table entries selected by masking)
  uint32_t tc_skip;      // test hook of the tensor-core form's bounded completion wait: 1 = no product is
                         // issued, so every wait runs out (mr_debug_lane_tc_wait); 0 otherwise
};

struct MRArgs {
  const uint32_t* cls;
  const uint32_t* cand;     // candidates, rows of n_limbs
  const uint32_t* witness;  // candidates*rounds rows of n_limbs (candidate-major)
  uint8_t* is_prime;        // per candidate (per = 1) or per item verdict bytes (per = rounds)
  uint32_t* round_mask;     // per candidate or nullptr (only with per = 1)
  uint32_t* scratch;        // window tables, per warp (1 << wbits) x 2 NPT x 32 words
  uint32_t* crow;           // per item 3W words: M mod N, M^2 mod N, N - (M mod N)
  uint32_t n;               // work items: candidates * per
  uint32_t n_limbs, rounds, wbits;
  uint32_t* dbg;            // nullptr, or per candidate mr_debug_words(k, W) words of derived constants
  uint32_t per;             // items per candidate: 1 (an item runs all rounds) or rounds (one round each)
  const uint32_t* sel;      // nullptr, or the candidates to test: item g takes candidate sel[g / per]
  const uint32_t* n_sel;    // with sel: device word, the number of selected candidates (items = it * per)
};

// Barrier polls of the large-class kernel before a wait gives up (x 0.03-0.3 us each: about 1 s).
constexpr uint32_t BIG_SPIN_POLLS = 1u << 22;

// Exponentiation of a large size class (several CTAs per item group, cooperative launch).
struct BigArgs {
  const uint32_t* cls;     // class table block (device)
  const uint32_t* tslice;  // extension matrices by channel slice: [T1 | T2][slice][k][SC] (u32), or for a
                           // tensor-core variant the fp16 slice operands [T1 | T2][slice][chunk] (big_kernel.cuh)
  const MxItem* items;
  uint32_t n_items;
  uint32_t wbits;          // window width, 1..8
  uint32_t* scratch;       // per group slot: slot_words(wbits) words
  uint8_t* status;         // per-item status bytes or nullptr
  uint32_t* sync;          // [slots] barrier counters, the abort flag, then [slots][BIG_FLAG_WORDS] chunk-ready
                           // counters (tensor-core form); zeroed before the launch (big_sync_words)
  uint32_t slots;          // item groups in flight (grid = slots * slices)
  uint32_t spin_limit;     // barrier polls before a wait gives up
  int32_t absent_slice;    // test hook: CTAs of this channel slice leave at once (-1: none)
  unsigned long long* phases;  // nullptr, or BIG_PHASES + 1 counters: SM cycles per phase summed over the
                               // CTAs (thread 0 of each), then the number of CTAs (tensor-core form only)
};

// Phases of one RNS Montgomery multiplication timed by the large-class kernel's phase counters: channel work
// up to the first exchange, first barrier, first extension's copies and products, its epilogue, channel work
// up to the second exchange, second barrier, second extension's copies and products, its epilogue and the
// final channel work.
constexpr int BIG_PHASES = 8;

// Chunk-ready counters per slot of the tensor-core form: [2 extensions][16 chunks of k].
constexpr uint32_t BIG_FLAG_WORDS = 32;
// Words of a launch's sync area (zeroed before the launch).
inline size_t big_sync_words(uint32_t slots) { return (size_t)slots * (1 + BIG_FLAG_WORDS) + 1; }

// [special, s, nbits, 0][M mod N: W][M^2 mod N: W][kxi: k][N M^-1 (plain): k][cd: k][N^-1 mod m_i: k][N^-1 mod m'_j: k]
MR_HD inline uint32_t mr_debug_words(uint32_t k, uint32_t W) { return 4 + 2 * W + 5 * k; }

// One compiled lane mapping of a size class.
struct KernelVariant {
  uint32_t tpi, threads, ipb, npt, smem_bytes;
  uint32_t tc;  // 1: the exponentiation kernel forms the base extensions on the tensor cores (rns_tc.cuh)
  cudaError_t (*modexp)(const LaunchArgs&, unsigned grid, cudaStream_t);
  cudaError_t (*crt)(const LaunchArgs&, unsigned grid, cudaStream_t);
  cudaError_t (*mr)(const MRArgs&, unsigned grid, cudaStream_t);
  cudaError_t (*prepare)();  // set kernel attributes (call before any stream capture)
  int (*occupancy)();        // resident blocks per SM of the exponentiation kernel
};

constexpr int MAX_VARIANTS = 4;

// Kernel of a large size class: one cooperative launch of slots * slices CTAs.
struct BigKernel {
  uint32_t sc, slices, threads, smem_bytes;
  uint32_t tc;       // 1: base extensions on the tensor cores (slice table in fp16, big_kernel.cuh)
  float group_time;  // time of one item group relative to variant 0 when both fit one wave (measured)
  size_t (*slot_words)(uint32_t wbits);
  cudaError_t (*modexp)(const BigArgs&, cudaStream_t);
  cudaError_t (*prepare)();
  int (*occupancy)();  // resident CTAs per SM
};

struct ClassKernels {
  uint32_t L, k, W, WX;
  uint32_t n_variants;  // lane-group variants (0 for a large class)
  KernelVariant var[MAX_VARIANTS];
  const BigKernel* big;  // non-null for a large class: n_big variants (channel-slice widths)
  uint32_t n_big;
};

// Garner recombination of CRT decryptions whose halves are in a large size class
// (binary, one warp per item): items[i].crt is a CrtBinOff block, p's W limbs sit at
// items[i].keyp + n_off.  W <= CRT_BIN_MAX_W.
constexpr uint32_t CRT_BIN_MAX_W = 512;
cudaError_t launch_crt_bin(const CrtItem* items, uint32_t n_items, uint32_t W, uint32_t n_off, cudaStream_t s);

// Trial division by the first primes ahead of Miller-Rabin (trial.cu).  Device table layout
// (words): [limb w][prime j] 2^(32w) mod p_j (TRIAL_MAX_LIMBS rows of TRIAL_STRIDE), then the
// primes (TRIAL_STRIDE), then the Barrett factors floor((2^64-1)/p_j) as uint64 (2 TRIAL_STRIDE).
constexpr uint32_t TRIAL_MAX_PRIMES = 10000, TRIAL_STRIDE = 10016, TRIAL_MAX_LIMBS = 128;
constexpr uint32_t TRIAL_NONE = 0xffffffffu;
constexpr size_t trial_table_words() { return (size_t)(TRIAL_MAX_LIMBS + 3) * TRIAL_STRIDE; }
std::vector<uint32_t> trial_tables_host();
// Candidates passing trial division by the first np primes are appended to sel (count: *count,
// zeroed by the caller), slot[c] = their position; the others get slot[c] = TRIAL_NONE.
cudaError_t launch_trial(const uint32_t* cand, uint32_t nl, uint32_t n, const uint32_t* tab, uint32_t np,
                         uint32_t* sel, uint32_t* slot, uint32_t* count, cudaStream_t s);
// verdict[c] = 0 (slot NONE), else 2 when the per item verdicts of slot[c] all pass, else 1.
cudaError_t launch_prime_combine(const uint8_t* item_pass, const uint32_t* slot, uint32_t n, uint32_t per,
                                 uint8_t* verdict, cudaStream_t s);

// RSA key assembly from candidate pools (keygen.cu): for key k, p = the first candidate of rows
// [2k pool, 2k pool + pool) with verdict 2 and gcd(e, p-1) = 1, q likewise in the next pool rows
// (q != p); out row k (9 half_limbs words): N 2H | d 2H | p | q | dp | dq | qinv.  status[k]:
// 0, 5 (a pool has no usable prime) or 3 (an inverse does not exist).
constexpr uint32_t KEYGEN_MAX_HALF_LIMBS = 128;
cudaError_t launch_keygen(const uint32_t* cand, const uint8_t* verdict, uint32_t n_keys, uint32_t pool,
                          uint32_t half_limbs, uint32_t e, uint32_t* out, uint8_t* status, cudaStream_t s);

// Message blocks (message.cu): rows of W limbs, block i = bytes [i B, i B + B) of the message,
// little-endian; unpack writes the first len bytes back from such rows.
cudaError_t launch_pack_message(const uint8_t* msg, size_t len, uint32_t B, uint32_t W, size_t n_blocks, uint32_t* rows,
                                cudaStream_t s);
cudaError_t launch_unpack_message(const uint32_t* rows, uint32_t B, uint32_t W, size_t len, uint8_t* msg, cudaStream_t s);

// nullptr when no kernel is compiled for class L
const ClassKernels* class_kernels(uint32_t L);

// scratch words one modexp launch of n items needs
inline size_t modexp_scratch_words(const KernelVariant& kc, uint32_t n, uint32_t wbits) {
  size_t grid = (n + kc.ipb - 1) / kc.ipb;
  size_t warps = grid * (kc.threads / 32);
  return warps * ((size_t)1 << wbits) * 2 * kc.npt * 32;
}

// scratch words of a persistent launch of `blocks` blocks
inline size_t persistent_scratch_words(const KernelVariant& kc, uint32_t blocks, uint32_t wbits) {
  return (size_t)blocks * (kc.threads / 32) * ((size_t)1 << wbits) * 2 * kc.npt * 32;
}

}  // namespace mr
