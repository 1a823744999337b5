// C ABI of the RNS modular-exponentiation library (declared in include/mr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mr.h"
#include "kernels_api.h"
#include "noalloc.h"
#include "setup.h"
#include "peak.h"

using namespace mr;

namespace {

struct ClassEntry {
  ClassHost host;
  uint32_t* dev = nullptr;
  uint32_t* tslice[MAX_VARIANTS] = {};  // large classes: extension matrices by channel slice, per variant
  const ClassKernels* kern = nullptr;
  uint32_t variant = 0;  // selected lane mapping (large classes: slice width, used when pinned)
  uint32_t wcap = 0;     // window-width cap chosen by mr_autotune (0 = the default rule)
  bool tuned = false;
  bool pinned = false;   // lane mapping chosen by the caller (mr_set_variant, MR_VARIANT_<L>) or the tuner
  const KernelVariant& kv() const { return kern->var[variant]; }
  bool big() const { return kern && kern->big; }
  uint32_t n_var() const { return big() ? kern->n_big : kern->n_variants; }
  // threads that hold one number's channels: the lane group, or one lane per warp of every slice
  uint32_t lanes(uint32_t v) const { return big() ? kern->big[v].slices * (kern->big[v].threads / 32) : kern->var[v].tpi; }
};

struct KeyEntry {
  ClassEntry* cls = nullptr;
  KeyHost host;
  uint32_t* dev = nullptr;
  uint32_t nlimbs() const { return (host.nbits + 31) / 32; }
};

// host-only class cache (inspection without a device)
std::mutex g_host_mu;
std::map<uint32_t, std::unique_ptr<ClassHost>> g_host_classes;

const ClassHost* host_class(uint32_t L, std::string& err) {
  std::lock_guard<std::mutex> g(g_host_mu);
  auto it = g_host_classes.find(L);
  if (it != g_host_classes.end()) return it->second.get();
  auto c = std::make_unique<ClassHost>();
  if (!build_class(L, *c, err)) return nullptr;
  const ClassHost* p = c.get();
  g_host_classes[L] = std::move(c);
  return p;
}

}  // namespace

struct mr_ctx {
  int device = 0;
  std::string err;
  std::map<uint32_t, std::unique_ptr<ClassEntry>> classes;
  cudaMemPool_t pool = nullptr;
  void* staging = nullptr;  // pinned host buffer for work-item uploads
  size_t staging_cap = 0;
  cudaEvent_t staging_evt = nullptr;
  bool staging_used = false;
  std::set<mr_key*> keys;
  // instrumentation
  bool prof_on = false;
  uint32_t launches[2] = {0, 0};
  struct Span {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Span> spans;
  std::vector<cudaEvent_t> free_events;
  uint32_t* mr_dbg = nullptr;  // test hook of mr_debug_mr_setup
  uint32_t big_spin_limit = 0;  // large-class barrier polls before giving up (0: the kernel default)
  int32_t big_absent_slice = -1;  // test hook of mr_debug_big_wait
  bool lane_tc_skip = false;       // test hook of mr_debug_lane_tc_wait
  unsigned long long* big_phases = nullptr;  // mr_debug_big_phases: device counters, or nullptr (off)
  bool constant_time = false;  // mr_set_constant_time
  std::vector<cudaStream_t> side;     // streams for concurrent groups of one-shot mixed calls
  std::vector<cudaEvent_t> side_join;
  cudaEvent_t side_fork = nullptr;
  uint32_t* trial_tab = nullptr;  // trial-division tables (mr_prime_test_batch), built on first use
};

struct mr_plan;

struct mr_key {
  mr_ctx* ctx = nullptr;
  KeyEntry pub;
  Big e;
  uint32_t* dev_e = nullptr;
  uint32_t e_limbs = 0;
  bool priv = false;
  KeyEntry p, q;
  uint32_t* dev_crt = nullptr;
  uint64_t device_bytes = 0;
};

namespace {

// NVTX range around a public call (shown by Nsight tools; no cost without a tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

mr_status fail(mr_ctx* ctx, mr_status code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

mr_status cuda_fail(mr_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, MR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

Big big_from(const uint32_t* p, uint32_t n) { return Big::from_limbs(p, n); }

mr_status get_class(mr_ctx* ctx, uint32_t L, ClassEntry** out) {
  auto it = ctx->classes.find(L);
  if (it != ctx->classes.end()) {
    *out = it->second.get();
    return MR_OK;
  }
  auto ce = std::make_unique<ClassEntry>();
  std::string err;
  const ClassHost* hc = host_class(L, err);
  if (!hc) return fail(ctx, MR_ERR_SIZE, "class setup failed: " + err);
  ce->host = *hc;
  ce->kern = class_kernels(L);
  if (!ce->kern) return fail(ctx, MR_ERR_SIZE, "no kernel compiled for class " + std::to_string(L));
  if (ce->kern->k != ce->host.k || ce->kern->W != ce->host.W || ce->kern->WX != ce->host.WX)
    return fail(ctx, MR_ERR_SIZE, "compiled kernel does not match the bases of class " + std::to_string(L));
  for (uint32_t v = 0; v < ce->kern->n_variants; v++) {
    cudaError_t pe = ce->kern->var[v].prepare();  // kernel attributes, once, outside any capture
    if (pe != cudaSuccess) return cuda_fail(ctx, pe, "kernel attributes");
  }
  for (uint32_t v = 0; ce->big() && v < ce->kern->n_big && v < (uint32_t)MAX_VARIANTS; v++) {
    const BigKernel& bk = ce->kern->big[v];
    cudaError_t pe = bk.prepare();
    if (pe != cudaSuccess) return cuda_fail(ctx, pe, "kernel attributes");
    const uint32_t k = ce->host.k, sc = bk.sc, sl = bk.slices;
    const ClassOff o = class_offsets(k, ce->host.W, ce->host.WX);
    std::vector<uint32_t> ts;
    if (!bk.tc) {
      // [T1 | T2][slice][row][SC]: the columns of each channel slice contiguous, zero past channel k
      ts.assign((size_t)2 * sl * k * sc, 0);
      for (uint32_t m = 0; m < 2; m++)
        for (uint32_t c = 0; c < sl; c++)
          for (uint32_t i = 0; i < k; i++)
            for (uint32_t q = 0; q < sc && c * sc + q < k; q++)
              ts[(((size_t)m * sl + c) * k + i) * sc + q] = ce->host.block[(m ? o.T2 : o.T1) + (size_t)i * k + c * sc + q];
    } else if (!tc_slice_table(ce->host.block.data() + o.T1, ce->host.block.data() + o.T2, k, sc, sl, ts)) {
      return fail(ctx, MR_ERR_SIZE, "extension matrix entries exceed the 28 bits of four 7-bit slices");
    }
    cudaError_t e = cudaMalloc(&ce->tslice[v], ts.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(ce->tslice[v], ts.data(), ts.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "class slice tables");
  }
  {
    // default lane mapping: variant 0, unless MR_VARIANT_<L> names another compiled one
    std::string ev = "MR_VARIANT_" + std::to_string(L);
    const char* v = getenv(ev.c_str());
    if (v) {
      unsigned idx = (unsigned)atoi(v);
      if (idx < ce->n_var()) {
        ce->variant = idx;
        ce->pinned = true;
      }
    }
  }
  size_t bytes = ce->host.block.size() * 4;
  cudaError_t e = cudaMalloc(&ce->dev, bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(class)");
  e = cudaMemcpy(ce->dev, ce->host.block.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(class)");
  *out = ce.get();
  ctx->classes[L] = std::move(ce);
  return MR_OK;
}

mr_status upload(mr_ctx* ctx, const std::vector<uint32_t>& v, uint32_t** dev) {
  cudaError_t e = cudaMalloc(dev, v.size() * 4);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc(key)");
  e = cudaMemcpy(*dev, v.data(), v.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(key)");
  return MR_OK;
}

mr_status make_key_entry(mr_ctx* ctx, const Big& N, const Big* exp, uint32_t L, KeyEntry& ke) {
  ClassEntry* ce = nullptr;
  mr_status s = get_class(ctx, L, &ce);
  if (s) return s;
  ke.cls = ce;
  std::string err;
  int rc = build_key(ce->host, N, exp, ke.host, err);
  if (rc) return fail(ctx, (mr_status)rc, err);
  return upload(ctx, ke.host.block, &ke.dev);
}

void free_key_entry(KeyEntry& ke) {
  if (ke.dev) cudaFree(ke.dev);
  ke.dev = nullptr;
}

// window width minimising squarings + multiplications + table size for an exponent of `bits`
// Largest window width a call may use: 5 for the lane-group classes (one table per number: at
// w = 6 the tables of a large batch outgrow L2, which costs more than the two multiplications
// w = 6 saves on a 1024-bit exponent), 8 for the large classes (tables per group slot only), or
// the class's cap chosen by mr_autotune; lowered by MR_MAX_WINDOW when set (1..8).
uint32_t window_cap(const ClassEntry* ce) {
  uint32_t cap = ce && ce->big() ? 8u : 5u;
  if (ce && ce->wcap) cap = ce->wcap;
  if (const char* v = getenv("MR_MAX_WINDOW")) {
    int w = atoi(v);
    if (w >= 1 && (uint32_t)w < cap) cap = (uint32_t)w;
  }
  return cap;
}

uint32_t choose_window(uint32_t bits, uint32_t popcount_hint, uint32_t max_w) {
  if (bits <= 1) return 1;
  uint64_t best = ~0ull;
  uint32_t bw = 1;
  for (uint32_t w = 1; w <= max_w; w++) {
    uint64_t nwin = (bits + w - 1) / w;
    uint64_t mults = (w == 1 && popcount_hint) ? popcount_hint : nwin;
    uint64_t cost = (uint64_t)(nwin - 1) * w + mults + ((1ull << w) - 2);
    if (cost < best) {
      best = cost;
      bw = w;
    }
  }
  return bw;
}

uint32_t popcount_big(const Big& b) {
  uint32_t c = 0;
  for (uint32_t w : b.w) c += (uint32_t)__builtin_popcount(w);
  return c;
}

// Per-class batch of exponentiations (+ optional CRT recombinations) of one call.
struct ClassBatch {
  ClassEntry* ce = nullptr;
  std::vector<MxItem> mx;
  std::vector<CrtItem> crt;
  uint32_t wbits = 1;
  // offsets (bytes) into the call's device scratch allocation
  size_t off_mx = 0, off_crt = 0, off_scratch = 0, off_half = 0;
  size_t scratch_words = 0;
  uint32_t slots = 0;  // large class: item groups in flight
  uint32_t bigv = 0;   // large class: kernel variant (slice width)
};

// Large class: the kernel variant (channel-slice width) for a batch of n items, and its item
// groups in flight.  A variant holds fit = resident CTAs / slices groups in one cooperative wave;
// the estimated time is the number of waves times the variant's relative time per group.  A
// pinned class (mr_set_variant, the tuner) keeps its variant.  Returns false when no variant
// fits the device.
// The policy itself, on given resident CTAs per SM of each variant (pinned < 0: any variant).
bool pick_big_variant(const ClassKernels* kern, uint64_t groups, int sms, const int* ctas_per_sm, int pinned,
                      uint32_t* v_out, uint32_t* slots) {
  double best = 1e300;
  bool found = false;
  for (uint32_t v = 0; v < kern->n_big && v < (uint32_t)MAX_VARIANTS; v++) {
    if (pinned >= 0 && v != (uint32_t)pinned) continue;
    const BigKernel& bk = kern->big[v];
    const uint64_t fit = (uint64_t)(ctas_per_sm[v] * sms) / bk.slices;
    if (fit == 0) continue;
    const double cost = (double)((groups + fit - 1) / fit) * bk.group_time;
    if (cost < best) {
      best = cost;
      found = true;
      *v_out = v;
      *slots = (uint32_t)std::min<uint64_t>(fit, groups);
    }
  }
  return found;
}

bool choose_big_variant(mr_ctx* ctx, const ClassEntry* ce, size_t n_items, uint32_t* v_out, uint32_t* slots) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  int occ[MAX_VARIANTS] = {};
  for (uint32_t v = 0; v < ce->kern->n_big && v < (uint32_t)MAX_VARIANTS; v++) occ[v] = ce->kern->big[v].occupancy();
  return pick_big_variant(ce->kern, (n_items + 31) / 32, sms, occ, ce->pinned ? (int)ce->variant : -1, v_out, slots);
}

// Reserve pinned staging space; waits for the previous upload to finish first.
mr_status staging_reserve(mr_ctx* ctx, size_t bytes) {
  if (ctx->staging_used) {
    cudaError_t e = cudaEventSynchronize(ctx->staging_evt);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize(staging)");
    ctx->staging_used = false;
  }
  if (bytes <= ctx->staging_cap) return MR_OK;
  if (ctx->staging) cudaFreeHost(ctx->staging);
  ctx->staging = nullptr;
  ctx->staging_cap = 0;
  size_t cap = std::max<size_t>(bytes, 1 << 20);
  cudaError_t e = cudaHostAlloc(&ctx->staging, cap, cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaHostAlloc(staging)");
  ctx->staging_cap = cap;
  return MR_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

cudaEvent_t take_event(mr_ctx* ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch one kernel, counting it and (when enabled) bracketing it with events on `stream`.
template <class F>
cudaError_t timed_launch(mr_ctx* ctx, int kind, cudaStream_t stream, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (ctx->prof_on) {
    a = take_event(ctx);
    b = take_event(ctx);
    if (a) cudaEventRecord(a, stream);
  }
  cudaError_t e = launch();
  ctx->launches[kind]++;
  if (a && b) {
    cudaEventRecord(b, stream);
    ctx->spans.push_back({kind, a, b});
  }
  return e;
}

// Lay out, upload and launch a set of class batches on `stream`.
mr_status run_batches(mr_ctx* ctx, std::vector<ClassBatch>& batches, uint8_t* status, cudaStream_t stream,
                      size_t half_words_per_crt) {
  // device layout: [items ...][scratch ...][half results ...]
  size_t upload_bytes = 0;
  for (auto& b : batches) {
    b.off_mx = upload_bytes;
    upload_bytes = align256(upload_bytes + b.mx.size() * sizeof(MxItem));
    b.off_crt = upload_bytes;
    upload_bytes = align256(upload_bytes + b.crt.size() * sizeof(CrtItem));
  }
  size_t total = upload_bytes;
  for (auto& b : batches) {
    if (b.mx.empty()) {
      b.scratch_words = 0;
    } else if (b.ce->big()) {
      // as many groups of 32 in flight as one cooperative launch can hold
      if (!choose_big_variant(ctx, b.ce, b.mx.size(), &b.bigv, &b.slots))
        return fail(ctx, MR_ERR_CUDA, "large-class kernel does not fit the device");
      const BigKernel& bk = b.ce->kern->big[b.bigv];
      b.scratch_words = (size_t)b.slots * bk.slot_words(b.wbits) + align256(big_sync_words(b.slots) * 4) / 4;
    } else {
      b.scratch_words = modexp_scratch_words(b.ce->kv(), (uint32_t)b.mx.size(), b.wbits);
    }
    b.off_scratch = total;
    total = align256(total + b.scratch_words * 4);
  }
  for (auto& b : batches) {
    b.off_half = total;
    total = align256(total + b.crt.size() * 2 * half_words_per_crt * 4);
  }
  if (total == 0) return MR_OK;
  void* dev = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&dev, total, ctx->pool, stream);
  if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
  char* base = static_cast<char*>(dev);
  // patch the per-half result pointers of CRT batches now that the scratch base is known
  for (auto& b : batches) {
    if (b.crt.empty()) continue;
    uint32_t W = b.ce->host.W;
    uint32_t* halves = reinterpret_cast<uint32_t*>(base + b.off_half);
    for (size_t i = 0; i < b.crt.size(); i++) {
      uint32_t* mp = halves + (2 * i) * W;
      uint32_t* mq = halves + (2 * i + 1) * W;
      b.crt[i].mp = mp;
      b.crt[i].mq = mq;
      b.mx[2 * i].out = mp;
      b.mx[2 * i + 1].out = mq;
    }
  }
  // items with the same exponent next to each other: warps of the lane-group kernel whose numbers
  // share one exponent run the sliding-window schedule
  for (auto& b : batches)
    if (!b.ce->big())
      std::stable_sort(b.mx.begin(), b.mx.end(), [](const MxItem& x, const MxItem& y) { return x.e < y.e; });
  mr_status s = staging_reserve(ctx, upload_bytes);
  if (s) {
    cudaFreeAsync(dev, stream);
    return s;
  }
  char* st = static_cast<char*>(ctx->staging);
  for (auto& b : batches) {
    if (!b.mx.empty()) memcpy(st + b.off_mx, b.mx.data(), b.mx.size() * sizeof(MxItem));
    if (!b.crt.empty()) memcpy(st + b.off_crt, b.crt.data(), b.crt.size() * sizeof(CrtItem));
  }
  e = cudaMemcpyAsync(base, st, upload_bytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->staging_evt, stream);
  ctx->staging_used = true;
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, stream);
    return cuda_fail(ctx, e, "item upload");
  }
  for (auto& b : batches) {
    if (b.ce->big()) {
      if (b.mx.empty()) continue;
      const BigKernel& bk = b.ce->kern->big[b.bigv];
      uint32_t* scr = reinterpret_cast<uint32_t*>(base + b.off_scratch);
      uint32_t* sync = scr + (size_t)b.slots * bk.slot_words(b.wbits);
      BigArgs a{b.ce->dev, b.ce->tslice[b.bigv], reinterpret_cast<const MxItem*>(base + b.off_mx), (uint32_t)b.mx.size(),
                b.wbits, scr, status, sync, b.slots, ctx->big_spin_limit ? ctx->big_spin_limit : BIG_SPIN_POLLS,
                ctx->big_absent_slice, ctx->big_phases};
      e = cudaMemsetAsync(sync, 0, big_sync_words(b.slots) * 4, stream);
      if (e == cudaSuccess) e = timed_launch(ctx, 0, stream, [&] { return bk.modexp(a, stream); });
      if (e == cudaSuccess && !b.crt.empty()) {
        const uint32_t n_off = key_offsets(b.ce->host.k, b.ce->host.W).N;
        e = timed_launch(ctx, 1, stream, [&] {
          return launch_crt_bin(reinterpret_cast<const CrtItem*>(base + b.off_crt), (uint32_t)b.crt.size(),
                                b.ce->host.W, n_off, stream);
        });
      }
      if (e != cudaSuccess) break;
      continue;
    }
    const KernelVariant& k = b.ce->kv();
    if (!b.mx.empty()) {
      LaunchArgs a{b.ce->dev, base + b.off_mx, (uint32_t)b.mx.size(), b.wbits,
                   reinterpret_cast<uint32_t*>(base + b.off_scratch), status, nullptr, ctx->constant_time ? 1u : 0u,
                   ctx->lane_tc_skip ? 1u : 0u};
      unsigned grid = (unsigned)((b.mx.size() + k.ipb - 1) / k.ipb);
      e = timed_launch(ctx, 0, stream, [&] { return k.modexp(a, grid, stream); });
      if (e != cudaSuccess) break;
    }
    if (!b.crt.empty()) {
      LaunchArgs a{b.ce->dev, base + b.off_crt, (uint32_t)b.crt.size(), 0, nullptr, status};
      unsigned grid = (unsigned)((b.crt.size() + k.ipb - 1) / k.ipb);
      e = timed_launch(ctx, 1, stream, [&] { return k.crt(a, grid, stream); });
      if (e != cudaSuccess) break;
    }
  }
  cudaError_t e2 = cudaFreeAsync(dev, stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
  return MR_OK;
}


// ------------------------------------------------------------ mixed batches
// A mixed batch holds RSA encryptions and CRT decryptions of any sizes.  Its
// exponentiations are grouped by (size class, window width); each group is one
// kernel launch (plus one CRT-recombination launch for decryption halves).
struct GroupLaunch {
  ClassEntry* ce = nullptr;
  uint32_t wbits = 1;
  std::vector<MxItem> mx;
  std::vector<CrtItem> crt;
  std::vector<uint32_t> ebits;  // per mx item, for ordering
  double work = 0;              // estimated 32x32->64 products
  size_t off_mx = 0, off_crt = 0, off_scratch = 0, off_half = 0;
  uint32_t grid = 0, crt_grid = 0;
  bool persistent = false;
  bool ct = false;              // constant-time schedule (the context's setting when the group was built)
};

double mm_products(uint32_t k) { return 2.0 * k * k + 7.0 * k; }

double modexp_work(uint32_t k, uint32_t ebits, uint32_t w) {
  double nwin = ebits ? std::ceil(ebits / (double)w) : 1.0;
  return (ebits + nwin + (double)(1u << w)) * mm_products(k);
}

// A request of a mixed batch whose exponentiations fall in a large size class (an encryption with a key
// above 4096 bits, a CRT decryption with halves above 4096 bits).
bool large_request(const mr_key* k, uint8_t op) {
  return op == MR_OP_DECRYPT && k->priv ? k->p.cls->big() : k->pub.cls->big();
}

// Group the lane-group requests of a mixed batch by (size class, window).  Large requests are left out
// and their indices appended to `large` when it is given (else they are refused).
mr_status build_groups(mr_ctx* ctx, const mr_key* const* keys, const uint8_t* ops, size_t n, const uint32_t* in,
                       uint32_t in_stride, uint32_t* out, uint32_t out_stride, std::vector<GroupLaunch>& groups,
                       std::vector<size_t>* large = nullptr) {
  std::map<std::pair<ClassEntry*, uint32_t>, size_t> idx;
  auto group = [&](ClassEntry* ce, uint32_t w) -> GroupLaunch& {
    auto key = std::make_pair(ce, w);
    auto it = idx.find(key);
    if (it != idx.end()) return groups[it->second];
    idx[key] = groups.size();
    groups.emplace_back();
    groups.back().ce = ce;
    groups.back().wbits = w;
    groups.back().ct = ctx->constant_time;
    return groups.back();
  };
  for (size_t i = 0; i < n; i++) {
    const mr_key* k = keys[i];
    if (!k || k->ctx != ctx) return fail(ctx, MR_ERR_ARG, "invalid key handle at index " + std::to_string(i));
    if (out_stride < k->pub.nlimbs()) return fail(ctx, MR_ERR_ARG, "out_stride smaller than a modulus");
    const KeyEntry& pub = k->pub;
    const uint32_t* nlim = pub.dev + key_offsets(pub.cls->host.k, pub.cls->host.W).N;
    if (large_request(k, ops[i])) {
      if (!large) return fail(ctx, MR_ERR_SIZE, "plans take keys of at most 4096 bits (halves for decryptions)");
      if (ops[i] != MR_OP_ENCRYPT && ops[i] != MR_OP_DECRYPT)
        return fail(ctx, MR_ERR_ARG, "unknown operation at index " + std::to_string(i));
      large->push_back(i);
      continue;
    }
    if (ops[i] == MR_OP_ENCRYPT) {
      if (!k->dev_e) return fail(ctx, MR_ERR_KEY, "key has no public exponent");
      uint32_t eb = (uint32_t)k->e.bits();
      GroupLaunch& g = group(pub.cls, choose_window(eb, popcount_big(k->e), window_cap(pub.cls)));
      MxItem it{};
      it.key = pub.dev;
      it.x = in + i * in_stride;
      it.e = k->dev_e;
      it.out = out + i * out_stride;
      it.xlim = nlim;
      it.x_limbs = in_stride;
      it.e_limbs = k->e_limbs;
      it.out_limbs = out_stride;
      it.xlim_limbs = pub.cls->host.W;
      it.status = (uint32_t)i;
      g.mx.push_back(it);
      g.ebits.push_back(eb);
      g.work += modexp_work(pub.cls->host.k, eb, g.wbits);
    } else if (ops[i] == MR_OP_DECRYPT) {
      if (!k->priv) return fail(ctx, MR_ERR_KEY, "key has no private CRT parts");
      ClassEntry* ce = k->p.cls;
      uint32_t eb = std::max(k->p.host.block[2], k->q.host.block[2]);
      GroupLaunch& g = group(ce, choose_window(eb, 0, window_cap(ce)));
      const KeyOff ko = key_offsets(ce->host.k, ce->host.W);
      for (int h = 0; h < 2; h++) {
        const KeyEntry& ke = h == 0 ? k->p : k->q;
        MxItem it{};
        it.key = ke.dev;
        it.x = in + i * in_stride;
        it.e = ke.dev + ko.exp;
        it.out = nullptr;                                 // result row of this half, set at staging
        it.pad_ = (uint32_t)(2 * g.crt.size() + h) + 1u;  // 1 + half index
        it.xlim = nlim;
        it.x_limbs = in_stride;
        it.e_limbs = ce->host.W;
        it.out_limbs = ce->host.W;
        it.xlim_limbs = pub.cls->host.W;
        it.status = (uint32_t)i;
        g.mx.push_back(it);
        g.ebits.push_back(h == 0 ? k->p.host.block[2] : k->q.host.block[2]);
        g.work += modexp_work(ce->host.k, g.ebits.back(), g.wbits);
      }
      CrtItem ci{};
      ci.keyp = k->p.dev;
      ci.crt = k->dev_crt;
      ci.out = out + i * out_stride;
      ci.out_limbs = out_stride;
      ci.status = (uint32_t)i;
      g.crt.push_back(ci);
    } else {
      return fail(ctx, MR_ERR_ARG, "unknown operation at index " + std::to_string(i));
    }
  }
  return MR_OK;
}

// Grids, orders and device offsets of the groups; returns the total device bytes.
size_t layout_groups(mr_ctx* ctx, std::vector<GroupLaunch>& groups, uint32_t flags, size_t* upload_bytes,
                     size_t* queue_off) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  size_t off = 0;
  for (auto& g : groups) {
    const KernelVariant& kv = g.ce->kv();
    g.persistent = (flags & MR_PLAN_PERSISTENT) != 0;
    // items in decreasing exponent length: long items first, groups of a warp homogeneous; equal
    // lengths ordered by exponent, so that the halves of one key share warps (one schedule)
    std::vector<size_t> ord(g.mx.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
      return g.ebits[a] != g.ebits[b] ? g.ebits[a] > g.ebits[b] : g.mx[a].e < g.mx[b].e;
    });
    std::vector<MxItem> mx(g.mx.size());
    std::vector<uint32_t> eb(g.mx.size());
    for (size_t i = 0; i < ord.size(); i++) {
      mx[i] = g.mx[ord[i]];
      eb[i] = g.ebits[ord[i]];
    }
    g.mx.swap(mx);
    g.ebits.swap(eb);
    const uint32_t full_grid = (uint32_t)((g.mx.size() + kv.ipb - 1) / kv.ipb);
    if (g.persistent) {
      // a full GPU of resident blocks per group: concurrent groups then fill the SMs that the
      // tail of an earlier group frees, instead of idling on a fixed share
      uint32_t blocks = (uint32_t)(kv.occupancy() * sms);
      g.grid = std::max<uint32_t>(1, std::min<uint32_t>(blocks, full_grid));
    } else {
      g.grid = full_grid;
    }
    g.crt_grid = (uint32_t)((g.crt.size() + kv.ipb - 1) / kv.ipb);
    g.off_mx = off;
    off = align256(off + g.mx.size() * sizeof(MxItem));
    g.off_crt = off;
    off = align256(off + g.crt.size() * sizeof(CrtItem));
  }
  *upload_bytes = off;
  *queue_off = off;
  off = align256(off + groups.size() * 4);
  for (auto& g : groups) {
    const KernelVariant& kv = g.ce->kv();
    size_t words = g.persistent ? persistent_scratch_words(kv, g.grid, g.wbits)
                                : modexp_scratch_words(kv, (uint32_t)g.mx.size(), g.wbits);
    g.off_scratch = off;
    off = align256(off + words * 4);
    g.off_half = off;
    off = align256(off + g.crt.size() * 2 * (size_t)g.ce->host.W * 4);
  }
  return off;
}

// Enqueue the kernels of a laid-out batch on `stream` (optionally one stream per group).
mr_status enqueue_groups(mr_ctx* ctx, std::vector<GroupLaunch>& groups, char* base, size_t queue_off, uint8_t* status,
                         uint32_t flags, cudaStream_t stream, const std::vector<cudaStream_t>& side,
                         cudaEvent_t fork, const std::vector<cudaEvent_t>& joins, uint32_t* launches) {
  cudaError_t e = cudaSuccess;
  uint32_t* queues = reinterpret_cast<uint32_t*>(base + queue_off);
  const bool conc = (flags & MR_PLAN_CONCURRENT) && side.size() >= groups.size();
  if (flags & MR_PLAN_PERSISTENT) e = cudaMemsetAsync(queues, 0, groups.size() * 4, stream);
  if (e == cudaSuccess && conc) e = cudaEventRecord(fork, stream);
  // largest groups first, so that a sequential launch order also starts the long work early
  std::vector<size_t> order(groups.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return groups[a].work > groups[b].work; });
  for (size_t oi = 0; oi < order.size() && e == cudaSuccess; oi++) {
    size_t gi = order[oi];
    GroupLaunch& g = groups[gi];
    cudaStream_t s = conc ? side[gi] : stream;
    if (conc) e = cudaStreamWaitEvent(s, fork, 0);
    const KernelVariant& kv = g.ce->kv();
    if (e == cudaSuccess && !g.mx.empty()) {
      LaunchArgs a{g.ce->dev, base + g.off_mx, (uint32_t)g.mx.size(), g.wbits,
                   reinterpret_cast<uint32_t*>(base + g.off_scratch), status, g.persistent ? queues + gi : nullptr,
                   g.ct ? 1u : 0u};
      e = kv.modexp(a, g.grid, s);
      (*launches)++;
    }
    if (e == cudaSuccess && !g.crt.empty()) {
      LaunchArgs a{g.ce->dev, base + g.off_crt, (uint32_t)g.crt.size(), 0, nullptr, status, nullptr};
      e = kv.crt(a, g.crt_grid, s);
      (*launches)++;
    }
    if (e == cudaSuccess && conc) e = cudaEventRecord(joins[gi], s);
  }
  if (conc)
    for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; gi++) e = cudaStreamWaitEvent(stream, joins[gi], 0);
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "mixed-batch launch");
}

// Device copies of the item arrays, with half-result pointers resolved against `base`.
void stage_items(std::vector<GroupLaunch>& groups, char* base, char* host) {
  for (auto& g : groups) {
    uint32_t W = g.ce->host.W;
    uint32_t* halves = reinterpret_cast<uint32_t*>(base + g.off_half);
    std::vector<MxItem> mx = g.mx;
    for (auto& it : mx)
      if (it.pad_) it.out = halves + (size_t)(it.pad_ - 1u) * W;
    std::vector<CrtItem> crt = g.crt;
    for (size_t i = 0; i < crt.size(); i++) {
      crt[i].mp = halves + (2 * i) * W;
      crt[i].mq = halves + (2 * i + 1) * W;
    }
    if (!mx.empty()) memcpy(host + g.off_mx, mx.data(), mx.size() * sizeof(MxItem));
    if (!crt.empty()) memcpy(host + g.off_crt, crt.data(), crt.size() * sizeof(CrtItem));
  }
}

template <class F>
mr_status guarded(mr_ctx* ctx, F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(ctx, MR_ERR_OOM, "host allocation failed");
  } catch (const std::exception& ex) {
    return fail(ctx, MR_ERR_ARG, ex.what());
  } catch (...) {
    return fail(ctx, MR_ERR_ARG, "unexpected error");
  }
}

// Per-candidate verdicts from per-round items: probable prime when every round passed; bit r of
// the mask set when round r (< 32) passed.
// Size class of Miller-Rabin candidates of n_limbs limbs (lane-group classes only).
mr_status mr_class(mr_ctx* ctx, uint32_t n_limbs, ClassEntry** out) {
  uint32_t L = class_for_bits(32 * n_limbs);
  if (!L) return fail(ctx, MR_ERR_SIZE, "candidates longer than the largest size class");
  mr_status s = get_class(ctx, L, out);
  if (s) return s;
  if ((*out)->big()) return fail(ctx, MR_ERR_SIZE, "Miller-Rabin takes candidates of at most 4096 bits");
  return MR_OK;
}

// Lane mapping of a Miller-Rabin launch of `items` work items: the caller's choice when pinned,
// else the narrowest mapping that gives at least 8 warps per SM (the widest when none does).
uint32_t mr_variant(mr_ctx* ctx, const ClassEntry* ce, size_t items) {
  if (ce->pinned) return ce->variant;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  uint32_t vsel = 0;
  for (uint32_t v = 0; v < ce->kern->n_variants; v++)
    if (ce->kern->var[v].tpi > ce->kern->var[vsel].tpi) vsel = v;
  for (uint32_t v = 0; v < ce->kern->n_variants; v++) {
    const double warps = (double)items * ce->kern->var[v].tpi / 32.0;
    if (warps >= 8.0 * sms && ce->kern->var[v].tpi < ce->kern->var[vsel].tpi) vsel = v;
  }
  return vsel;
}

// Device scratch bytes of mr_launch with lane mapping v: window tables per warp, then per item 3W
// words of constants.
size_t mr_scratch_bytes(const ClassEntry* ce, uint32_t v, uint32_t n_limbs, size_t items) {
  const KernelVariant& k = ce->kern->var[v];
  const uint32_t wbits = choose_window(32 * n_limbs, 0, window_cap(ce));
  return align256(modexp_scratch_words(k, (uint32_t)items, wbits) * 4) + items * 3 * (size_t)ce->host.W * 4;
}

__global__ void mr_combine_kernel(const uint8_t* item_pass, uint32_t n, uint32_t rounds, uint8_t* is_prime,
                                  uint32_t* round_mask) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  uint32_t m = 0;
  uint8_t all = 1;
  for (uint32_t r = 0; r < rounds; r++) {
    const uint8_t p = item_pass[(size_t)c * rounds + r];
    all &= p;
    if (p && r < 32) m |= 1u << r;
  }
  is_prime[c] = all;
  if (round_mask) round_mask[c] = m;
}


// Large-class Miller-Rabin: after y = a^d mod n (step 0) and after each squaring step j, round item i
// passes when y = n - 1, or at step 0 when y = 1; steps j >= s_i (n_i - 1 = 2^s_i d_i) do not count.
__global__ void mr_large_flags_kernel(const uint32_t* y, const uint32_t* nm1, const uint32_t* s_item, uint32_t W,
                                      uint32_t n_items, uint32_t step, uint8_t* pass) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_items || step >= s_item[i]) return;
  const uint32_t* yr = y + (size_t)i * W;
  const uint32_t* nr = nm1 + (size_t)i * W;
  bool is_nm1 = true, is_one = step == 0;
  for (uint32_t w = 0; w < W; w++) {
    const uint32_t v = yr[w];
    is_nm1 = is_nm1 && v == nr[w];
    is_one = is_one && v == (w == 0 ? 1u : 0u);
  }
  if (is_nm1 || is_one) pass[i] = 1;
}

// ------------------------------------------------------------- autotuning

// Seeded host generator for the synthetic tuning batch (SplitMix64).
struct TuneRng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  }
  uint32_t u32() { return (uint32_t)(next() >> 32); }
};

mr_status autotune_class(mr_ctx* ctx, ClassEntry* ce, uint32_t n, uint32_t exp_bits, mr_tune_result* res) {
  const uint32_t L = ce->host.L, W = ce->host.W, EL = (exp_bits + 31) / 32;
  TuneRng r{0x4D52A070ull ^ ((uint64_t)L << 20) ^ exp_bits};
  KeyEntry ke;
  for (int attempt = 0;; attempt++) {  // a seeded L-bit odd modulus, coprime to the channel primes
    std::vector<uint32_t> l(W);
    for (auto& v : l) v = r.u32();
    l[0] |= 1u;
    l[W - 1] |= 0x80000000u;
    mr_status s = make_key_entry(ctx, Big::from_limbs(l.data(), W), nullptr, L, ke);
    if (s == MR_OK) break;
    free_key_entry(ke);
    if (s != MR_ERR_NOT_COPRIME || attempt > 8) return s;
  }
  // bases below 2^(L-32) < N; exponents of exactly exp_bits bits
  std::vector<uint32_t> hx((size_t)n * W, 0u), he((size_t)n * EL, 0u);
  const uint32_t top = exp_bits - 32 * (EL - 1);
  for (uint32_t i = 0; i < n; i++) {
    for (uint32_t w = 0; w + 1 < W; w++) hx[(size_t)i * W + w] = r.u32();
    for (uint32_t w = 0; w < EL; w++) he[(size_t)i * EL + w] = r.u32();
    uint32_t& t = he[(size_t)i * EL + EL - 1];
    t = (top == 32 ? t : (t & ((1u << top) - 1u))) | (1u << (top - 1));
  }
  uint32_t* dx = nullptr;
  const size_t xw = (size_t)n * W, ew = (size_t)n * EL;
  cudaError_t e = cudaMalloc(&dx, (2 * xw + ew) * 4);
  if (e != cudaSuccess) {
    free_key_entry(ke);
    return fail(ctx, MR_ERR_OOM, "tuning buffers");
  }
  uint32_t* de = dx + xw;
  uint32_t* dout = de + ew;
  cudaStream_t st = nullptr;
  cudaEvent_t ea = nullptr, eb = nullptr;
  e = cudaMemcpy(dx, hx.data(), xw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(de, he.data(), ew * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ea);
  if (e == cudaSuccess) e = cudaEventCreate(&eb);
  const bool prof = ctx->prof_on;
  ctx->prof_on = false;  // tuning launches stay out of the profile counters
  const uint32_t saved_launches[2] = {ctx->launches[0], ctx->launches[1]};
  mr_status s = e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "tuning setup");
  const uint32_t nv = ce->n_var();
  const bool was_pinned = ce->pinned;
  ce->pinned = true;  // run_batches takes the variant under test
  auto time_config = [&](uint32_t variant, uint32_t w, double* ms) -> mr_status {
    ce->variant = variant;
    double best = 1e30;
    for (int rep = 0; rep < 3; rep++) {  // warm-up, then best of two
      std::vector<ClassBatch> batches(1);
      ClassBatch& b = batches[0];
      b.ce = ce;
      b.wbits = w;
      b.mx.resize(n);
      for (uint32_t i = 0; i < n; i++) {
        MxItem& it = b.mx[i];
        it = MxItem{};
        it.key = ke.dev;
        it.x = dx + (size_t)i * W;
        it.e = de + (size_t)i * EL;
        it.out = dout + (size_t)i * W;
        it.xlim = ke.dev + key_offsets(ce->host.k, W).N;
        it.x_limbs = W;
        it.e_limbs = EL;
        it.out_limbs = W;
        it.xlim_limbs = W;
        it.status = 0xffffffffu;
      }
      cudaEventRecord(ea, st);
      mr_status rs = run_batches(ctx, batches, nullptr, st, 0);
      cudaEventRecord(eb, st);
      cudaError_t se = cudaEventSynchronize(eb);
      if (rs) return rs;
      if (se != cudaSuccess) return cuda_fail(ctx, se, "tuning run");
      float t = 0;
      cudaEventElapsedTime(&t, ea, eb);
      if (rep > 0) best = std::min(best, (double)t);
    }
    *ms = best;
    return MR_OK;
  };
  const uint32_t wmax = ce->big() ? 8u : 6u;
  const uint32_t wopt = choose_window(exp_bits, 0, wmax);
  const uint32_t wdef = choose_window(exp_bits, 0, ce->big() ? 8u : 5u);
  double best_ms = 1e30, def_ms = 0;
  uint32_t best_v = 0, best_w = wdef, configs = 0;
  if (!s) s = time_config(0, wdef, &def_ms);
  if (!s) {
    configs++;
    best_ms = def_ms;
  }
  for (uint32_t v = 0; v < nv && !s; v++)
    for (uint32_t w = wopt > 2 ? wopt - 2 : 1; w <= wopt && !s; w++) {
      if (v == 0 && w == wdef) continue;
      double ms = 0;
      s = time_config(v, w, &ms);
      configs++;
      if (!s && ms < best_ms) {
        best_ms = ms;
        best_v = v;
        best_w = w;
      }
    }
  ctx->prof_on = prof;
  ctx->launches[0] = saved_launches[0];
  ctx->launches[1] = saved_launches[1];
  if (st) cudaStreamSynchronize(st);
  if (ea) cudaEventDestroy(ea);
  if (eb) cudaEventDestroy(eb);
  if (st) cudaStreamDestroy(st);
  cudaFree(dx);
  free_key_entry(ke);
  if (s) {
    ce->variant = 0;
    ce->pinned = was_pinned;
    return s;
  }
  ce->variant = best_v;
  ce->wcap = best_w;
  ce->tuned = true;
  ce->pinned = true;
  if (res) {
    res->variant = best_v;
    res->lanes_per_number = ce->lanes(best_v);
    res->window = best_w;
    res->configs = configs;
    res->ms = best_ms;
    res->ms_default = def_ms;
  }
  return MR_OK;
}

// MR_PLAN_AUTOTUNE: tune every not yet tuned size class of a mixed batch with the batch's item
// count (at least 256, at most 8192) and longest exponent of that class.
mr_status autotune_mixed(mr_ctx* ctx, const mr_key* const* keys, const uint8_t* ops, size_t n) {
  std::map<ClassEntry*, std::pair<uint32_t, uint32_t>> need;  // class -> (items, longest exponent bits)
  for (size_t i = 0; i < n; i++) {
    const mr_key* k = keys[i];
    if (!k || k->ctx != ctx) return fail(ctx, MR_ERR_ARG, "invalid key handle at index " + std::to_string(i));
    if (ops[i] == MR_OP_ENCRYPT) {
      auto& v = need[k->pub.cls];
      v.first += 1;
      v.second = std::max<uint32_t>(v.second, (uint32_t)k->e.bits());
    } else if (ops[i] == MR_OP_DECRYPT && k->priv) {
      auto& v = need[k->p.cls];
      v.first += 2;
      v.second = std::max<uint32_t>(v.second, std::max(k->p.host.block[2], k->q.host.block[2]));
    }
  }
  for (auto& kv : need) {
    if (kv.first->tuned || kv.first->big()) continue;
    uint32_t items = std::min<uint32_t>(8192, std::max<uint32_t>(256, kv.second.first));
    mr_status s = autotune_class(ctx, kv.first, items, std::max<uint32_t>(2, kv.second.second), nullptr);
    if (s) return s;
  }
  return MR_OK;
}

ClassBatch& batch_for(std::vector<ClassBatch>& v, std::map<ClassEntry*, size_t>& idx, ClassEntry* ce) {
  auto it = idx.find(ce);
  if (it != idx.end()) return v[it->second];
  idx[ce] = v.size();
  v.emplace_back();
  v.back().ce = ce;
  return v.back();
}

// The large requests of a mixed batch: the class batches of mr_rsa_encrypt and mr_rsa_decrypt_crt
// (cooperative large-class launches, then the binary Garner recombination), their items addressed at
// the requests' own rows and status bytes.
mr_status run_large_mixed(mr_ctx* ctx, const mr_key* const* keys, const uint8_t* ops, const std::vector<size_t>& sel,
                          const uint32_t* in, uint32_t in_stride, uint32_t* out, uint32_t out_stride,
                          uint8_t* status, cudaStream_t st) {
  std::vector<ClassBatch> enc, dec;
  std::map<ClassEntry*, size_t> ie, id;
  std::map<ClassEntry*, uint32_t> eb_enc, pop_enc, eb_dec;
  uint32_t maxW = 0;
  for (size_t i : sel) {
    const mr_key* k = keys[i];
    const KeyEntry& pub = k->pub;
    const uint32_t* nlim = pub.dev + key_offsets(pub.cls->host.k, pub.cls->host.W).N;
    if (ops[i] == MR_OP_ENCRYPT) {
      if (!k->dev_e) return fail(ctx, MR_ERR_KEY, "key has no public exponent");
      ClassBatch& b = batch_for(enc, ie, pub.cls);
      MxItem it{};
      it.key = pub.dev;
      it.x = in + i * in_stride;
      it.e = k->dev_e;
      it.out = out + i * out_stride;
      it.xlim = nlim;
      it.x_limbs = in_stride;
      it.e_limbs = k->e_limbs;
      it.out_limbs = out_stride;
      it.xlim_limbs = pub.cls->host.W;
      it.status = (uint32_t)i;
      b.mx.push_back(it);
      eb_enc[pub.cls] = std::max<uint32_t>(eb_enc[pub.cls], (uint32_t)k->e.bits());
      pop_enc[pub.cls] = std::max<uint32_t>(pop_enc[pub.cls], popcount_big(k->e));
    } else {
      if (!k->priv) return fail(ctx, MR_ERR_KEY, "key has no private CRT parts");
      ClassEntry* ce = k->p.cls;
      ClassBatch& b = batch_for(dec, id, ce);
      const KeyOff ko = key_offsets(ce->host.k, ce->host.W);
      for (int h = 0; h < 2; h++) {
        const KeyEntry& ke = h == 0 ? k->p : k->q;
        MxItem it{};
        it.key = ke.dev;
        it.x = in + i * in_stride;
        it.e = ke.dev + ko.exp;
        it.out = nullptr;  // patched to the half-result scratch
        it.xlim = nlim;
        it.x_limbs = in_stride;
        it.e_limbs = ce->host.W;
        it.out_limbs = ce->host.W;
        it.xlim_limbs = pub.cls->host.W;
        it.status = (uint32_t)i;
        b.mx.push_back(it);
      }
      CrtItem ci{};
      ci.keyp = k->p.dev;
      ci.crt = k->dev_crt;
      ci.out = out + i * out_stride;
      ci.out_limbs = out_stride;
      ci.status = (uint32_t)i;
      b.crt.push_back(ci);
      eb_dec[ce] = std::max<uint32_t>(eb_dec[ce], std::max(k->p.host.block[2], k->q.host.block[2]));
      maxW = std::max(maxW, ce->host.W);
    }
  }
  for (auto& b : enc) b.wbits = choose_window(eb_enc[b.ce], pop_enc[b.ce], window_cap(b.ce));
  for (auto& b : dec) b.wbits = choose_window(eb_dec[b.ce], 0, window_cap(b.ce));
  // encryption and decryption batches run separately: a decryption batch holds only CRT halves
  mr_status s = enc.empty() ? MR_OK : run_batches(ctx, enc, status, st, 0);
  if (!s && !dec.empty()) s = run_batches(ctx, dec, status, st, maxW);
  return s;
}

}  // namespace

struct mr_plan {
  mr_ctx* ctx = nullptr;
  uint32_t flags = 0;
  std::vector<GroupLaunch> groups;
  void* dev = nullptr;
  size_t dev_bytes = 0, queue_off = 0;
  uint8_t* status = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t kernels = 0;
  double products = 0;
};

extern "C" {

mr_status mr_init(int device, mr_ctx** out) {
  if (!out) return MR_ERR_ARG;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) return e != cudaSuccess ? MR_ERR_CUDA : MR_ERR_ARG;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return MR_ERR_CUDA;
  auto* ctx = new (std::nothrow) mr_ctx();
  if (!ctx) return MR_ERR_OOM;
  ctx->device = device;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  e = cudaMemPoolCreate(&ctx->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->staging_evt, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete ctx;
    return MR_ERR_CUDA;
  }
  *out = ctx;
  return MR_OK;
}

void mr_shutdown(mr_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (mr_key* k : ctx->keys) {
    free_key_entry(k->pub);
    free_key_entry(k->p);
    free_key_entry(k->q);
    if (k->dev_e) cudaFree(k->dev_e);
    if (k->dev_crt) cudaFree(k->dev_crt);
    delete k;
  }
  for (auto& kv : ctx->classes) {
    if (kv.second->dev) cudaFree(kv.second->dev);
    for (uint32_t* t : kv.second->tslice)
      if (t) cudaFree(t);
  }
  if (ctx->trial_tab) cudaFree(ctx->trial_tab);
  if (ctx->big_phases) cudaFree(ctx->big_phases);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  if (ctx->staging_evt) cudaEventDestroy(ctx->staging_evt);
  for (auto& sp : ctx->spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (cudaEvent_t ev : ctx->free_events) cudaEventDestroy(ev);
  for (auto ss : ctx->side) cudaStreamDestroy(ss);
  for (auto ev : ctx->side_join) cudaEventDestroy(ev);
  if (ctx->side_fork) cudaEventDestroy(ctx->side_fork);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
}

const char* mr_last_error(const mr_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

mr_status mr_class_for_bits(uint32_t bits, uint32_t* class_bits, uint32_t* k) {
  uint32_t L = class_for_bits(bits);
  if (!L || bits == 0) return MR_ERR_SIZE;
  std::string err;
  const ClassHost* c = host_class(L, err);
  if (!c) return MR_ERR_SIZE;
  if (class_bits) *class_bits = L;
  if (k) *k = c->k;
  return MR_OK;
}

mr_status mr_rns_setup(mr_ctx* ctx, const uint32_t* N, uint32_t n_limbs, mr_key** out) {
  NvtxRange nvtx_("mr_rns_setup");
  if (!ctx || !N || !n_limbs || !out) return fail(ctx, MR_ERR_ARG, "null argument");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    Big n = big_from(N, n_limbs);
    uint32_t L = class_for_bits((uint32_t)n.bits());
    if (!L) return fail(ctx, MR_ERR_SIZE, "modulus longer than the largest size class");
    auto key = std::make_unique<mr_key>();
    key->ctx = ctx;
    mr_status s = make_key_entry(ctx, n, nullptr, L, key->pub);
    if (s) {
      free_key_entry(key->pub);
      return s;
    }
    key->device_bytes = key->pub.host.block.size() * 4;
    *out = key.get();
    ctx->keys.insert(key.release());
    return MR_OK;
  });
}

mr_status mr_rsa_key_setup(mr_ctx* ctx, const uint32_t* N, uint32_t n_limbs, const uint32_t* e, uint32_t e_limbs,
                           const uint32_t* p, const uint32_t* q, const uint32_t* dp, const uint32_t* dq,
                           const uint32_t* qinv, uint32_t half_limbs, mr_key** out) {
  NvtxRange nvtx_("mr_rsa_key_setup");
  if (!ctx || !N || !n_limbs || !e || !e_limbs || !out) return fail(ctx, MR_ERR_ARG, "null argument");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    Big n = big_from(N, n_limbs);
    uint32_t L = class_for_bits((uint32_t)n.bits());
    if (!L) return fail(ctx, MR_ERR_SIZE, "modulus longer than the largest size class");
    auto key = std::make_unique<mr_key>();
    key->ctx = ctx;
    auto cleanup = [&]() {
      free_key_entry(key->pub);
      free_key_entry(key->p);
      free_key_entry(key->q);
      if (key->dev_e) cudaFree(key->dev_e);
      if (key->dev_crt) cudaFree(key->dev_crt);
    };
    mr_status s = make_key_entry(ctx, n, nullptr, L, key->pub);
    if (s) {
      cleanup();
      return s;
    }
    key->e = big_from(e, e_limbs);
    key->e_limbs = std::max<uint32_t>(1, (uint32_t)((key->e.bits() + 31) / 32));
    s = upload(ctx, key->e.limbs(key->e_limbs), &key->dev_e);
    if (s) {
      cleanup();
      return s;
    }
    key->device_bytes = key->pub.host.block.size() * 4 + key->e_limbs * 4;
    bool any_priv = p || q || dp || dq || qinv;
    if (any_priv) {
      if (!(p && q && dp && dq && qinv && half_limbs)) {
        cleanup();
        return fail(ctx, MR_ERR_ARG, "private parts must be all given or all NULL");
      }
      Big bp = big_from(p, half_limbs), bq = big_from(q, half_limbs);
      Big bdp = big_from(dp, half_limbs), bdq = big_from(dq, half_limbs), bqi = big_from(qinv, half_limbs);
      if (cmp(mul(bp, bq), n) != 0) {
        cleanup();
        return fail(ctx, MR_ERR_ARG, "N != p*q");
      }
      uint32_t Lh = class_for_bits((uint32_t)std::max(bp.bits(), bq.bits()));
      if (!Lh) {
        cleanup();
        return fail(ctx, MR_ERR_SIZE, "prime longer than the largest size class");
      }
      s = make_key_entry(ctx, bp, &bdp, Lh, key->p);
      if (!s) s = make_key_entry(ctx, bq, &bdq, Lh, key->q);
      if (s) {
        cleanup();
        return s;
      }
      std::vector<uint32_t> crt = key->p.cls->big() ? build_crt_bin(key->p.cls->host.W, bp, bq, bqi)
                                                    : build_crt(key->p.cls->host, bp, bq, bqi);
      s = upload(ctx, crt, &key->dev_crt);
      if (s) {
        cleanup();
        return s;
      }
      key->priv = true;
      key->device_bytes += (key->p.host.block.size() + key->q.host.block.size() + crt.size()) * 4;
    }
    *out = key.get();
    ctx->keys.insert(key.release());
    return MR_OK;
  });
}

mr_status mr_key_info(const mr_key* key, uint32_t* k, uint32_t* k_half, uint64_t* device_bytes) {
  if (!key) return MR_ERR_ARG;
  if (k) *k = key->pub.cls ? key->pub.cls->host.k : 0;
  if (k_half) *k_half = key->priv ? key->p.cls->host.k : 0;
  if (device_bytes) *device_bytes = key->device_bytes;
  return MR_OK;
}

mr_status mr_key_free(mr_ctx* ctx, mr_key* key) {
  if (!key) return MR_OK;
  if (!ctx || key->ctx != ctx || !ctx->keys.count(key)) return fail(ctx, MR_ERR_ARG, "key does not belong to this context");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  free_key_entry(key->pub);
  free_key_entry(key->p);
  free_key_entry(key->q);
  if (key->dev_e) cudaFree(key->dev_e);
  if (key->dev_crt) cudaFree(key->dev_crt);
  ctx->keys.erase(key);
  delete key;
  return MR_OK;
}

static mr_status check_keys(mr_ctx* ctx, const mr_key* const* keys, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!keys[i] || keys[i]->ctx != ctx) return fail(ctx, MR_ERR_ARG, "invalid key handle at index " + std::to_string(i));
  return MR_OK;
}

mr_status mr_modexp_batch(mr_ctx* ctx, const mr_key* const* keys, size_t n, const uint32_t* x, uint32_t x_stride,
                          const uint32_t* e, uint32_t e_stride, uint32_t* out, uint32_t out_stride,
                          uint8_t* dev_status, void* stream) {
  NvtxRange nvtx_("mr_modexp_batch");
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!keys || !x || !e || !out || !x_stride || !e_stride || !out_stride) return fail(ctx, MR_ERR_ARG, "null argument or zero stride");
  if (n > 0xffffffffull) return fail(ctx, MR_ERR_ARG, "batch too large");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    mr_status s = check_keys(ctx, keys, n);
    if (s) return s;
    std::vector<ClassBatch> batches;
    std::map<ClassEntry*, size_t> idx;
    for (size_t i = 0; i < n; i++) {
      const KeyEntry& ke = keys[i]->pub;
      if (out_stride < ke.nlimbs()) return fail(ctx, MR_ERR_ARG, "out_stride smaller than a modulus");
      ClassBatch& b = batch_for(batches, idx, ke.cls);
      MxItem it{};
      it.key = ke.dev;
      it.x = x + i * x_stride;
      it.e = e + i * e_stride;
      it.out = out + i * out_stride;
      it.xlim = ke.dev + key_offsets(ke.cls->host.k, ke.cls->host.W).N;
      it.x_limbs = x_stride;
      it.e_limbs = e_stride;
      it.out_limbs = out_stride;
      it.xlim_limbs = ke.cls->host.W;
      it.status = (uint32_t)i;
      b.mx.push_back(it);
    }
    for (auto& b : batches) {
      std::stable_sort(b.mx.begin(), b.mx.end(), [](const MxItem& a, const MxItem& c) { return a.key < c.key; });
      b.wbits = choose_window(32 * e_stride, 0, window_cap(b.ce));
    }
    return run_batches(ctx, batches, dev_status, (cudaStream_t)stream, 0);
  });
}

mr_status mr_rsa_encrypt(mr_ctx* ctx, const mr_key* const* keys, size_t n, const uint32_t* m, uint32_t m_stride,
                         uint32_t* c, uint32_t c_stride, uint8_t* dev_status, void* stream) {
  NvtxRange nvtx_("mr_rsa_encrypt");
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!keys || !m || !c || !m_stride || !c_stride) return fail(ctx, MR_ERR_ARG, "null argument or zero stride");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    mr_status s = check_keys(ctx, keys, n);
    if (s) return s;
    std::vector<ClassBatch> batches;
    std::map<ClassEntry*, size_t> idx;
    std::map<ClassEntry*, uint32_t> cost_bits, cost_pop;
    for (size_t i = 0; i < n; i++) {
      const mr_key* k = keys[i];
      const KeyEntry& ke = k->pub;
      if (!k->dev_e) return fail(ctx, MR_ERR_KEY, "key has no public exponent (use mr_rsa_key_setup)");
      if (c_stride < ke.nlimbs()) return fail(ctx, MR_ERR_ARG, "c_stride smaller than a modulus");
      ClassBatch& b = batch_for(batches, idx, ke.cls);
      MxItem it{};
      it.key = ke.dev;
      it.x = m + i * m_stride;
      it.e = k->dev_e;
      it.out = c + i * c_stride;
      it.xlim = ke.dev + key_offsets(ke.cls->host.k, ke.cls->host.W).N;
      it.x_limbs = m_stride;
      it.e_limbs = k->e_limbs;
      it.out_limbs = c_stride;
      it.xlim_limbs = ke.cls->host.W;
      it.status = (uint32_t)i;
      b.mx.push_back(it);
      cost_bits[ke.cls] = std::max<uint32_t>(cost_bits[ke.cls], (uint32_t)k->e.bits());
      cost_pop[ke.cls] = std::max<uint32_t>(cost_pop[ke.cls], popcount_big(k->e));
    }
    for (auto& b : batches) {
      std::stable_sort(b.mx.begin(), b.mx.end(), [](const MxItem& a, const MxItem& c2) { return a.key < c2.key; });
      b.wbits = choose_window(cost_bits[b.ce], cost_pop[b.ce], window_cap(b.ce));
    }
    return run_batches(ctx, batches, dev_status, (cudaStream_t)stream, 0);
  });
}

mr_status mr_rsa_decrypt_crt(mr_ctx* ctx, const mr_key* const* keys, size_t n, const uint32_t* c, uint32_t c_stride,
                             uint32_t* m, uint32_t m_stride, uint8_t* dev_status, void* stream) {
  NvtxRange nvtx_("mr_rsa_decrypt_crt");
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!keys || !c || !m || !c_stride || !m_stride) return fail(ctx, MR_ERR_ARG, "null argument or zero stride");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    mr_status s = check_keys(ctx, keys, n);
    if (s) return s;
    std::vector<ClassBatch> batches;
    std::map<ClassEntry*, size_t> idx;
    std::map<ClassEntry*, uint32_t> ebits;
    // sort decryptions by (half class, key) so that the two halves of a key sit together
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return keys[a]->p.dev < keys[b]->p.dev; });
    uint32_t maxW = 0;
    for (size_t i = 0; i < n; i++)
      if (keys[i]->priv) maxW = std::max(maxW, keys[i]->p.cls->host.W);
    for (size_t oi = 0; oi < n; oi++) {
      size_t i = order[oi];
      const mr_key* k = keys[i];
      if (!k->priv) return fail(ctx, MR_ERR_KEY, "key has no private CRT parts");
      if (m_stride < k->pub.nlimbs()) return fail(ctx, MR_ERR_ARG, "m_stride smaller than a modulus");
      ClassEntry* ce = k->p.cls;
      ClassBatch& b = batch_for(batches, idx, ce);
      const KeyOff ko = key_offsets(ce->host.k, ce->host.W);
      const KeyEntry& pub = k->pub;
      const uint32_t* nlim = pub.dev + key_offsets(pub.cls->host.k, pub.cls->host.W).N;
      for (int h = 0; h < 2; h++) {
        const KeyEntry& ke = h == 0 ? k->p : k->q;
        MxItem it{};
        it.key = ke.dev;
        it.x = c + i * c_stride;
        it.e = ke.dev + ko.exp;
        it.out = nullptr;  // patched to the half-result scratch
        it.xlim = nlim;
        it.x_limbs = c_stride;
        it.e_limbs = ce->host.W;
        it.out_limbs = ce->host.W;
        it.xlim_limbs = pub.cls->host.W;
        it.status = (uint32_t)i;
        b.mx.push_back(it);
      }
      CrtItem ci{};
      ci.keyp = k->p.dev;
      ci.crt = k->dev_crt;
      ci.out = m + i * m_stride;
      ci.out_limbs = m_stride;
      ci.status = (uint32_t)i;
      b.crt.push_back(ci);
      uint32_t eb = (uint32_t)std::max(k->p.host.block[2], k->q.host.block[2]);
      ebits[ce] = std::max(ebits[ce], eb);
    }
    for (auto& b : batches) b.wbits = choose_window(ebits[b.ce], 0, window_cap(b.ce));
    return run_batches(ctx, batches, dev_status, (cudaStream_t)stream, maxW);
  });
}

// Miller-Rabin launch shared by mr_miller_rabin_batch and mr_prime_test_batch: n candidates (or the
// *n_sel of them listed in sel), one work item per (candidate, round) when per = rounds.  With
// per > 1 the item verdicts go to `item_pass` (n * per bytes) and the caller combines them.
mr_status mr_launch(mr_ctx* ctx, ClassEntry* ce, uint32_t v, const uint32_t* cand, uint32_t n_limbs, size_t n,
                    const uint32_t* witness, uint32_t rounds, uint32_t per, uint8_t* item_pass,
                    uint32_t* dev_round_mask, const uint32_t* sel, const uint32_t* n_sel, void* scratch,
                    cudaStream_t stream) {
  const size_t items = n * (size_t)per;
  const KernelVariant& k = ce->kern->var[v];
  const uint32_t wbits = choose_window(32 * n_limbs, 0, window_cap(ce));
  const size_t tab_words = modexp_scratch_words(k, (uint32_t)items, wbits);
  const size_t off_crow = align256(tab_words * 4);
  char* base = static_cast<char*>(scratch);
  MRArgs a{ce->dev, cand, witness, item_pass, dev_round_mask, reinterpret_cast<uint32_t*>(base),
           reinterpret_cast<uint32_t*>(base + off_crow), (uint32_t)items, n_limbs, rounds, wbits, ctx->mr_dbg,
           per, sel, n_sel};
  unsigned grid = (unsigned)((items + k.ipb - 1) / k.ipb);
  cudaError_t e = timed_launch(ctx, 0, stream, [&] { return k.mr(a, grid, stream); });
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "kernel launch");
}

}  // extern "C"

// The rounds of the large candidates of mr_miller_rabin_large: sets pass[i * rounds + r] for i in `large`.
template <class WitnessMod>
mr_status mr_large_rounds(mr_ctx* ctx, ClassEntry* ce, const std::vector<size_t>& large, const std::vector<Big>& Ns,
                          WitnessMod&& witness_mod, uint32_t rounds, std::vector<uint8_t>& pass, cudaStream_t st) {
  const uint32_t L = ce->host.L, W = ce->host.W;
  std::vector<KeyEntry> keys(large.size());
  auto release = [&]() {
    for (auto& k : keys) free_key_entry(k);
  };
  std::vector<uint32_t> hx, he, hn, hs;
  std::vector<size_t> slot;  // pass index of each work item
  std::vector<const uint32_t*> item_key;
  uint32_t max_s = 0, max_dbits = 1;
  for (size_t j = 0; j < large.size(); j++) {
    const size_t i = large[j];
    const Big& N = Ns[i];
    const mr_status ks = make_key_entry(ctx, N, nullptr, L, keys[j]);
    if (ks == MR_ERR_NOT_COPRIME) {  // a channel prime divides N (N is far above it): composite
      ctx->err.clear();
      continue;
    }
    if (ks) {
      release();
      return ks;
    }
    const Big nm1 = sub(N, Big(1u));
    uint32_t sv = 0;
    while (!nm1.bit(sv)) sv++;
    // d = (N - 1) / 2^s as W limbs
    const std::vector<uint32_t> nl = nm1.limbs(W + 1), nml = nm1.limbs(W);
    std::vector<uint32_t> d(W, 0);
    const uint32_t ws = sv / 32, bs = sv % 32;
    for (uint32_t w = 0; w < W; w++) {
      const uint32_t lo = w + ws <= W ? nl[w + ws] : 0u, hi = w + ws + 1 <= W ? nl[w + ws + 1] : 0u;
      d[w] = bs ? (lo >> bs) | (hi << (32 - bs)) : lo;
    }
    for (uint32_t r = 0; r < rounds; r++) {
      const Big a = witness_mod(i, r);
      if (a.is_zero()) continue;  // y = 0 at every step: the round fails
      if (cmp(a, Big(1u)) == 0 || cmp(a, nm1) == 0) {  // y = 1 or y = n - 1 (d is odd)
        pass[i * rounds + r] = 1;
        continue;
      }
      const std::vector<uint32_t> al = a.limbs(W);
      hx.insert(hx.end(), al.begin(), al.end());
      he.insert(he.end(), d.begin(), d.end());
      hn.insert(hn.end(), nml.begin(), nml.end());
      hs.push_back(sv);
      slot.push_back(i * rounds + r);
      item_key.push_back(keys[j].dev);
      max_s = std::max(max_s, sv);
      max_dbits = std::max<uint32_t>(max_dbits, (uint32_t)(nm1.bits() - sv));
    }
  }
  mr_status s = MR_OK;
  const size_t items = slot.size();
  const uint32_t two = 2;
  std::vector<uint8_t> hp(items);
  if (items) {
    const size_t rowb = (size_t)W * 4;
    const size_t oE = align256(items * rowb), oN = align256(oE + items * rowb), oY = align256(oN + items * rowb),
                 oS = align256(oY + items * rowb), oP = align256(oS + items * 4), oT = align256(oP + items);
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, oT + 256, ctx->pool, st);
    if (e != cudaSuccess) {
      release();
      return fail(ctx, MR_ERR_OOM, "scratch allocation failed");
    }
    char* base = static_cast<char*>(dev);
    uint32_t* X = reinterpret_cast<uint32_t*>(base);
    uint32_t* E = reinterpret_cast<uint32_t*>(base + oE);
    uint32_t* NM1 = reinterpret_cast<uint32_t*>(base + oN);
    uint32_t* Y = reinterpret_cast<uint32_t*>(base + oY);
    uint32_t* S = reinterpret_cast<uint32_t*>(base + oS);
    uint8_t* P = reinterpret_cast<uint8_t*>(base + oP);
    uint32_t* TWO = reinterpret_cast<uint32_t*>(base + oT);
    e = cudaMemcpyAsync(X, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E, he.data(), he.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(NM1, hn.data(), hn.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S, hs.data(), hs.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(TWO, &two, 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P, 0, items, st);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "round upload");
    const unsigned fgrid = (unsigned)((items + 255) / 256);
    // step j = 0: y = a^d; steps j >= 1: y = y^2 in place (the kernel reads x before it writes out)
    for (uint32_t step = 0; !s && step < std::max<uint32_t>(max_s, 1); step++) {
      std::vector<ClassBatch> bv(1);
      ClassBatch& b = bv[0];
      b.ce = ce;
      b.wbits = step == 0 ? choose_window(max_dbits, 0, window_cap(ce)) : 1u;
      const uint32_t key_n = key_offsets(ce->host.k, W).N;
      for (size_t t = 0; t < items; t++) {
        MxItem it{};
        it.key = item_key[t];
        it.x = step == 0 ? X + t * W : Y + t * W;
        it.e = step == 0 ? E + t * W : TWO;
        it.out = Y + t * W;
        it.xlim = item_key[t] + key_n;
        it.x_limbs = W;
        it.e_limbs = step == 0 ? W : 1u;
        it.out_limbs = W;
        it.xlim_limbs = W;
        it.status = 0xffffffffu;
        b.mx.push_back(it);
      }
      s = run_batches(ctx, bv, nullptr, st, 0);
      if (!s) {
        mr_large_flags_kernel<<<fgrid, 256, 0, st>>>(Y, NM1, S, W, (uint32_t)items, step, P);
        e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "kernel launch");
      }
    }
    if (!s) {
      e = cudaMemcpyAsync(hp.data(), P, items, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "verdict download");
    }
    cudaFreeAsync(dev, st);
  }
  const cudaError_t e = cudaStreamSynchronize(st);  // host sources of the uploads, keys freed after use
  release();
  if (s) return s;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "Miller-Rabin rounds");
  for (size_t t = 0; t < items; t++) pass[slot[t]] = hp[t];
  return MR_OK;
}

// Miller-Rabin on candidates of a large size class (8192, 16384 bits), composed from the large-class
// exponentiation.  The candidates and witnesses come to the host (the call synchronises `st`), which
// settles the definitional cases, hands odd candidates of at most 4096 bits to the lane-group kernel
// (rows repacked), and for the others derives the modulus constants (as mr_rns_setup) and
// n - 1 = 2^s d: y = a^d for every (candidate, round) in one class batch, then up to max(s) - 1 squaring
// batches (exponent 2, in place), mr_large_flags_kernel recording each round's verdict after every
// step.  The rounds combine on the host and the verdicts go back to the device.
mr_status mr_miller_rabin_large(mr_ctx* ctx, ClassEntry* ce, const uint32_t* cand, uint32_t n_limbs, size_t n,
                                const uint32_t* witness, uint32_t rounds, uint8_t* dev_prime, uint32_t* dev_mask,
                                cudaStream_t st) {
  const size_t nr = n * (size_t)rounds;
  std::vector<uint32_t> hc(n * (size_t)n_limbs), hw(nr * n_limbs);
  cudaError_t e = cudaMemcpyAsync(hc.data(), cand, hc.size() * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hw.data(), witness, hw.size() * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "candidate download");
  std::vector<uint8_t> pass(nr, 0);  // per (candidate, round)
  std::vector<Big> Ns(n);
  std::vector<size_t> small, large;
  for (size_t i = 0; i < n; i++) {
    Ns[i] = big_from(hc.data() + i * n_limbs, n_limbs);
    const Big& N = Ns[i];
    if (N.bits() == 2 && !N.bit(0)) {  // 2 is prime
      for (uint32_t r = 0; r < rounds; r++) pass[i * rounds + r] = 1;
      continue;
    }
    if (N.bits() < 2 || !N.bit(0)) continue;  // 0, 1 and even numbers are composite
    (N.bits() <= 4096 ? small : large).push_back(i);
  }
  auto witness_mod = [&](size_t i, uint32_t r) {
    return mod(big_from(hw.data() + (i * rounds + r) * n_limbs, n_limbs), Ns[i]);
  };
  mr_status s = MR_OK;
  if (!small.empty()) {
    ClassEntry* cs = nullptr;
    if ((s = get_class(ctx, 4096, &cs))) return s;
    const uint32_t sw = cs->host.W;
    const size_t ns = small.size(), items = ns * rounds;
    std::vector<uint32_t> rc(ns * sw), rw(items * sw);
    for (size_t j = 0; j < ns; j++) {
      std::vector<uint32_t> l = Ns[small[j]].limbs(sw);
      std::copy(l.begin(), l.end(), rc.begin() + j * sw);
      for (uint32_t r = 0; r < rounds; r++) {
        std::vector<uint32_t> a = witness_mod(small[j], r).limbs(sw);
        std::copy(a.begin(), a.end(), rw.begin() + (j * rounds + r) * sw);
      }
    }
    const uint32_t v = mr_variant(ctx, cs, items);
    const size_t sbytes = align256(mr_scratch_bytes(cs, v, sw, items));
    const size_t off_c = sbytes, off_w = align256(off_c + rc.size() * 4), off_p = align256(off_w + rw.size() * 4);
    void* dev = nullptr;
    e = cudaMallocFromPoolAsync(&dev, off_p + items, ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, "scratch allocation failed");
    char* base = static_cast<char*>(dev);
    std::vector<uint8_t> ip(items);
    e = cudaMemcpyAsync(base + off_c, rc.data(), rc.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + off_w, rw.data(), rw.size() * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "candidate upload");
    if (!s)
      s = mr_launch(ctx, cs, v, reinterpret_cast<uint32_t*>(base + off_c), sw, ns, reinterpret_cast<uint32_t*>(base + off_w),
                    rounds, rounds, reinterpret_cast<uint8_t*>(base + off_p), nullptr, nullptr, nullptr, dev, st);
    if (!s) {
      e = cudaMemcpyAsync(ip.data(), base + off_p, items, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "verdict download");
    }
    cudaFreeAsync(dev, st);
    if (s) return s;
    for (size_t j = 0; j < ns; j++)
      for (uint32_t r = 0; r < rounds; r++) pass[small[j] * rounds + r] = ip[j * rounds + r];
  }
  if (!large.empty()) s = mr_large_rounds(ctx, ce, large, Ns, witness_mod, rounds, pass, st);
  if (s) return s;
  std::vector<uint8_t> prime(n);
  std::vector<uint32_t> mask(n);
  for (size_t i = 0; i < n; i++) {
    uint8_t all = 1;
    uint32_t m = 0;
    for (uint32_t r = 0; r < rounds; r++) {
      all &= pass[i * rounds + r];
      if (pass[i * rounds + r] && r < 32) m |= 1u << r;
    }
    prime[i] = all;
    mask[i] = m;
  }
  e = cudaMemcpyAsync(dev_prime, prime.data(), n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dev_mask) e = cudaMemcpyAsync(dev_mask, mask.data(), n * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors are the copies' sources
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "verdict upload");
}

extern "C" {

mr_status mr_miller_rabin_batch(mr_ctx* ctx, const uint32_t* cand, uint32_t n_limbs, size_t n, const uint32_t* witness,
                                uint32_t rounds, uint8_t* dev_is_probable_prime, uint32_t* dev_round_mask,
                                void* stream) {
  NvtxRange nvtx_("mr_miller_rabin_batch");
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!cand || !n_limbs || !witness || !rounds || !dev_is_probable_prime)
    return fail(ctx, MR_ERR_ARG, "null argument, zero limbs or zero rounds");
  if (dev_round_mask && rounds > 32) return fail(ctx, MR_ERR_ARG, "round mask holds at most 32 rounds");
  if (n > 0xffffffffull) return fail(ctx, MR_ERR_ARG, "batch too large");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    ClassEntry* ce = nullptr;
    const uint32_t Lc = class_for_bits(32 * n_limbs);
    if (Lc > 4096) {  // a large class: composed from the large-class exponentiation (synchronous)
      mr_status sb = get_class(ctx, Lc, &ce);
      if (sb) return sb;
      return mr_miller_rabin_large(ctx, ce, cand, n_limbs, n, witness, rounds, dev_is_probable_prime, dev_round_mask,
                                   st);
    }
    mr_status s = mr_class(ctx, n_limbs, &ce);
    if (s) return s;
    // The rounds of a candidate are independent: each runs as its own work item (the setup of
    // the candidate is repeated per round, a few hundredths of a round's cost) and a second
    // kernel combines the verdicts.  The constant-dump hook keeps one item per candidate.
    const uint32_t per = (rounds > 1 && !ctx->mr_dbg && (uint64_t)n * rounds <= 0xffffffffull) ? rounds : 1u;
    const size_t items = n * (size_t)per;
    const uint32_t v = mr_variant(ctx, ce, items);
    const size_t sbytes = mr_scratch_bytes(ce, v, n_limbs, items);
    const size_t off_pass = align256(sbytes);
    const size_t bytes = per > 1 ? off_pass + items : sbytes;
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, bytes, ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    char* base = static_cast<char*>(dev);
    uint8_t* verdicts = per > 1 ? reinterpret_cast<uint8_t*>(base + off_pass) : dev_is_probable_prime;
    s = mr_launch(ctx, ce, v, cand, n_limbs, n, witness, rounds, per, verdicts, per > 1 ? nullptr : dev_round_mask,
                  nullptr, nullptr, dev, st);
    if (!s && per > 1) {
      mr_combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(verdicts, (uint32_t)n, rounds,
                                                                     dev_is_probable_prime, dev_round_mask);
      e = cudaGetLastError();
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "kernel launch");
    }
    cudaError_t e2 = cudaFreeAsync(dev, st);
    if (s) return s;
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
    return MR_OK;
  });
}

mr_status mr_prime_test_batch(mr_ctx* ctx, const uint32_t* cand, uint32_t n_limbs, size_t n, const uint32_t* witness,
                              uint32_t rounds, uint32_t n_primes, uint8_t* dev_verdict, uint32_t* dev_survivors,
                              void* stream) {
  NvtxRange nvtx_("mr_prime_test_batch");
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) {  // no candidates: no survivors
    if (!dev_survivors) return MR_OK;
    const cudaError_t e = cudaMemsetAsync(dev_survivors, 0, 4, (cudaStream_t)stream);
    return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "cudaMemsetAsync");
  }
  if (!cand || !n_limbs || !witness || !rounds || !dev_verdict)
    return fail(ctx, MR_ERR_ARG, "null argument, zero limbs or zero rounds");
  if (n_primes == 0 || n_primes > TRIAL_MAX_PRIMES) return fail(ctx, MR_ERR_ARG, "n_primes must be 1..10000");
  if ((uint64_t)n * rounds > 0xffffffffull) return fail(ctx, MR_ERR_ARG, "batch too large");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    ClassEntry* ce = nullptr;
    mr_status s = mr_class(ctx, n_limbs, &ce);
    if (s) return s;
    if (n_limbs > TRIAL_MAX_LIMBS) return fail(ctx, MR_ERR_SIZE, "candidates longer than 4096 bits");
    if (!ctx->trial_tab) {
      std::vector<uint32_t> t = trial_tables_host();
      s = upload(ctx, t, &ctx->trial_tab);
      if (s) return s;
    }
    // device scratch: [count][sel n][slot n][Miller-Rabin scratch][item verdicts n * rounds]
    const uint32_t per = rounds;
    const size_t items = n * (size_t)per;
    // the lane mapping is chosen for the expected survivors (about one random odd candidate in ten
    // passes the first 10,000 primes; one in eight is assumed); scratch holds every candidate
    const uint32_t v = mr_variant(ctx, ce, (items + 7) / 8);
    const size_t off_sel = 256, off_slot = align256(off_sel + n * 4), off_mr = align256(off_slot + n * 4);
    const size_t off_pass = align256(off_mr + mr_scratch_bytes(ce, v, n_limbs, items));
    const size_t bytes = off_pass + items;
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, bytes, ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    char* base = static_cast<char*>(dev);
    uint32_t* count = reinterpret_cast<uint32_t*>(base);
    uint32_t* sel = reinterpret_cast<uint32_t*>(base + off_sel);
    uint32_t* slot = reinterpret_cast<uint32_t*>(base + off_slot);
    uint8_t* pass = reinterpret_cast<uint8_t*>(base + off_pass);
    e = cudaMemsetAsync(count, 0, 4, st);
    if (e == cudaSuccess)
      e = timed_launch(ctx, 1, st, [&] { return launch_trial(cand, n_limbs, (uint32_t)n, ctx->trial_tab, n_primes,
                                                             sel, slot, count, st); });
    s = e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "trial division launch");
    if (!s)
      s = mr_launch(ctx, ce, v, cand, n_limbs, n, witness, rounds, per, pass, nullptr, sel, count, base + off_mr, st);
    if (!s) {
      e = launch_prime_combine(pass, slot, (uint32_t)n, per, dev_verdict, st);
      if (e == cudaSuccess && dev_survivors) e = cudaMemcpyAsync(dev_survivors, count, 4, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "kernel launch");
    }
    cudaError_t e2 = cudaFreeAsync(dev, st);
    if (s) return s;
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
    return MR_OK;
  });
}


mr_status mr_rsa_keygen_batch(mr_ctx* ctx, uint32_t half_limbs, size_t n_keys, uint32_t pool, const uint32_t* cand,
                              const uint32_t* witness, uint32_t rounds, uint32_t e, uint32_t* out, uint8_t* dev_status,
                              void* stream) {
  NvtxRange nvtx_("mr_rsa_keygen_batch");
  if (!ctx) return MR_ERR_ARG;
  if (n_keys == 0) return MR_OK;
  if (!cand || !witness || !out || !rounds || !pool) return fail(ctx, MR_ERR_ARG, "null argument, zero pool or rounds");
  if (half_limbs < 2 || half_limbs > KEYGEN_MAX_HALF_LIMBS)
    return fail(ctx, MR_ERR_SIZE, "prime candidates must have 2 to 64 limbs");
  if (e < 3 || !(e & 1u)) return fail(ctx, MR_ERR_ARG, "the public exponent must be odd and at least 3");
  const uint64_t n = (uint64_t)n_keys * 2 * pool;
  if (n * rounds > 0xffffffffull) return fail(ctx, MR_ERR_ARG, "batch too large");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    void* dev = nullptr;
    cudaError_t e1 = cudaMallocFromPoolAsync(&dev, align256((size_t)n), ctx->pool, st);
    if (e1 != cudaSuccess)
      return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e1));
    uint8_t* verdict = static_cast<uint8_t*>(dev);
    // verdicts of every candidate (trial division, then Miller-Rabin on the survivors)
    mr_status s = mr_prime_test_batch(ctx, cand, half_limbs, (size_t)n, witness, rounds, TRIAL_MAX_PRIMES, verdict,
                                      nullptr, stream);
    if (!s) {
      cudaError_t e2 = launch_keygen(cand, verdict, (uint32_t)n_keys, pool, half_limbs, e, out, dev_status, st);
      if (e2 != cudaSuccess) s = cuda_fail(ctx, e2, "key assembly launch");
    }
    cudaError_t e3 = cudaFreeAsync(dev, st);
    if (s) return s;
    if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "cudaFreeAsync");
    return MR_OK;
  });
}

mr_status mr_rsa_message_blocks(const mr_key* key, size_t len, size_t* n_blocks, uint32_t* block_bytes,
                                uint32_t* row_limbs) {
  if (!key) return MR_ERR_ARG;
  const uint32_t B = (key->pub.host.nbits - 1) / 8;
  if (B == 0) return MR_ERR_SIZE;
  if (n_blocks) *n_blocks = (len + B - 1) / B;
  if (block_bytes) *block_bytes = B;
  if (row_limbs) *row_limbs = key->pub.nlimbs();
  return MR_OK;
}

mr_status mr_rsa_encrypt_message(mr_ctx* ctx, const mr_key* key, const uint8_t* msg, size_t len, uint32_t* c,
                                 uint8_t* dev_status, void* stream) {
  NvtxRange nvtx_("mr_rsa_encrypt_message");
  if (!ctx) return MR_ERR_ARG;
  if (!key || key->ctx != ctx) return fail(ctx, MR_ERR_ARG, "invalid key handle");
  if (len == 0) return MR_OK;
  if (!msg || !c) return fail(ctx, MR_ERR_ARG, "null argument");
  size_t nb = 0;
  uint32_t B = 0, W = 0;
  if (mr_rsa_message_blocks(key, len, &nb, &B, &W)) return fail(ctx, MR_ERR_SIZE, "modulus below 2^9");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, nb * W * 4, ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    uint32_t* rows = static_cast<uint32_t*>(dev);
    e = launch_pack_message(msg, len, B, W, nb, rows, st);
    mr_status s = e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "message packing");
    if (!s) {
      std::vector<const mr_key*> keys(nb, key);
      s = mr_rsa_encrypt(ctx, keys.data(), nb, rows, W, c, W, dev_status, stream);
    }
    cudaError_t e2 = cudaFreeAsync(dev, st);
    if (s) return s;
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
    return MR_OK;
  });
}

mr_status mr_rsa_decrypt_message(mr_ctx* ctx, const mr_key* key, const uint32_t* c, size_t n_blocks, uint8_t* msg,
                                 size_t len, uint8_t* dev_status, void* stream) {
  NvtxRange nvtx_("mr_rsa_decrypt_message");
  if (!ctx) return MR_ERR_ARG;
  if (!key || key->ctx != ctx) return fail(ctx, MR_ERR_ARG, "invalid key handle");
  size_t nb = 0;
  uint32_t B = 0, W = 0;
  if (mr_rsa_message_blocks(key, len, &nb, &B, &W)) return fail(ctx, MR_ERR_SIZE, "modulus below 2^9");
  if (nb != n_blocks) return fail(ctx, MR_ERR_ARG, "n_blocks does not match the message length");
  if (len == 0) return MR_OK;
  if (!msg || !c) return fail(ctx, MR_ERR_ARG, "null argument");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, nb * W * 4, ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    uint32_t* rows = static_cast<uint32_t*>(dev);
    std::vector<const mr_key*> keys(nb, key);
    mr_status s = mr_rsa_decrypt_crt(ctx, keys.data(), nb, c, W, rows, W, dev_status, stream);
    if (!s) {
      e = launch_unpack_message(rows, B, W, len, msg, st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "message unpacking");
    }
    cudaError_t e2 = cudaFreeAsync(dev, st);
    if (s) return s;
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
    return MR_OK;
  });
}

mr_status mr_rsa_mixed(mr_ctx* ctx, const mr_key* const* keys, const uint8_t* ops, size_t n, const uint32_t* in,
                       uint32_t in_stride, uint32_t* out, uint32_t out_stride, uint8_t* dev_status, uint32_t flags,
                       void* stream) {
  NvtxRange nvtx_("mr_rsa_mixed");
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!keys || !ops || !in || !out || !in_stride || !out_stride) return fail(ctx, MR_ERR_ARG, "null argument or zero stride");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<GroupLaunch> groups;
    mr_status s = (flags & MR_PLAN_AUTOTUNE) ? autotune_mixed(ctx, keys, ops, n) : MR_OK;
    if (s) return s;
    std::vector<size_t> large;
    s = build_groups(ctx, keys, ops, n, in, in_stride, out, out_stride, groups, &large);
    if (s) return s;
    if (!large.empty()) {
      s = run_large_mixed(ctx, keys, ops, large, in, in_stride, out, out_stride, dev_status, st);
      if (s) return s;
    }
    if (groups.empty()) return MR_OK;
    flags &= (MR_PLAN_CONCURRENT | MR_PLAN_PERSISTENT);
    size_t upload = 0, qoff = 0;
    size_t total = layout_groups(ctx, groups, flags, &upload, &qoff);
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, total, ctx->pool, st);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    char* base = static_cast<char*>(dev);
    s = staging_reserve(ctx, upload);
    if (s) {
      cudaFreeAsync(dev, st);
      return s;
    }
    stage_items(groups, base, static_cast<char*>(ctx->staging));
    e = cudaMemcpyAsync(base, ctx->staging, upload, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->staging_evt, st);
    ctx->staging_used = true;
    if (e != cudaSuccess) {
      cudaFreeAsync(dev, st);
      return cuda_fail(ctx, e, "item upload");
    }
    // side streams of the context for concurrent groups
    while ((flags & MR_PLAN_CONCURRENT) && ctx->side.size() < groups.size()) {
      cudaStream_t ss;
      cudaEvent_t ev;
      if (cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "side streams");
      ctx->side.push_back(ss);
      ctx->side_join.push_back(ev);
    }
    if ((flags & MR_PLAN_CONCURRENT) && !ctx->side_fork &&
        cudaEventCreateWithFlags(&ctx->side_fork, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "fork event");
    uint32_t launches = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (ctx->prof_on) {
      a = take_event(ctx);
      b = take_event(ctx);
      if (a) cudaEventRecord(a, st);
    }
    s = enqueue_groups(ctx, groups, base, qoff, dev_status, flags, st, ctx->side, ctx->side_fork, ctx->side_join,
                       &launches);
    if (a && b) {
      cudaEventRecord(b, st);
      ctx->spans.push_back({0, a, b});
    }
    ctx->launches[0] += launches;
    cudaError_t e2 = cudaFreeAsync(dev, st);
    if (s) return s;
    return e2 == cudaSuccess ? MR_OK : cuda_fail(ctx, e2, "cudaFreeAsync");
  });
}

mr_status mr_plan_create(mr_ctx* ctx, const mr_key* const* keys, const uint8_t* ops, size_t n, const uint32_t* in,
                         uint32_t in_stride, uint32_t* out, uint32_t out_stride, uint8_t* dev_status, uint32_t flags,
                         mr_plan** out_plan) {
  NvtxRange nvtx_("mr_plan_create");
  if (!ctx || !out_plan) return MR_ERR_ARG;
  *out_plan = nullptr;
  if (!n || !keys || !ops || !in || !out || !in_stride || !out_stride)
    return fail(ctx, MR_ERR_ARG, "empty plan, null argument or zero stride");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    auto plan = std::make_unique<mr_plan>();
    plan->ctx = ctx;
    plan->flags = flags;
    plan->status = dev_status;
    mr_status s = (flags & MR_PLAN_AUTOTUNE) ? autotune_mixed(ctx, keys, ops, n) : MR_OK;
    if (s) return s;
    s = build_groups(ctx, keys, ops, n, in, in_stride, out, out_stride, plan->groups);
    if (s) return s;
    size_t upload = 0;
    size_t total = layout_groups(ctx, plan->groups, flags, &upload, &plan->queue_off);
    cudaError_t e = cudaMalloc(&plan->dev, total);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("plan allocation failed: ") + cudaGetErrorString(e));
    plan->dev_bytes = total;
    std::vector<char> host(upload);
    stage_items(plan->groups, static_cast<char*>(plan->dev), host.data());
    e = cudaMemcpy(plan->dev, host.data(), upload, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plan upload");
    for (auto& g : plan->groups) plan->products += g.work;
    if (flags & MR_PLAN_CONCURRENT) {
      for (size_t i = 0; i < plan->groups.size(); i++) {
        cudaStream_t ss;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
          return cuda_fail(ctx, cudaGetLastError(), "plan streams");
        plan->side.push_back(ss);
        plan->joins.push_back(ev);
      }
      if (cudaEventCreateWithFlags(&plan->fork, cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "plan fork event");
    }
    if (flags & MR_PLAN_GRAPH) {
      cudaStream_t cap;
      e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cuda_fail(ctx, e, "begin capture");
      }
      uint32_t launches = 0;
      s = enqueue_groups(ctx, plan->groups, static_cast<char*>(plan->dev), plan->queue_off, plan->status, flags, cap,
                         plan->side, plan->fork, plan->joins, &launches);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cap, &graph);
      cudaStreamDestroy(cap);
      if (s) {
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
      plan->graph = graph;
      e = cudaGraphInstantiate(&plan->exec, graph, 0);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
      plan->kernels = launches;
    } else {
      plan->kernels = 0;
      for (auto& g : plan->groups) plan->kernels += (g.mx.empty() ? 0 : 1) + (g.crt.empty() ? 0 : 1);
    }
    *out_plan = plan.release();
    return MR_OK;
  });
}

mr_status mr_plan_launch(mr_plan* plan, void* stream) {
  NvtxRange nvtx_("mr_plan_launch");
  if (!plan) return MR_ERR_ARG;
  mr_ctx* ctx = plan->ctx;
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    if (ctx->prof_on) {
      a = take_event(ctx);
      b = take_event(ctx);
      if (a) cudaEventRecord(a, st);
    }
    mr_status s = MR_OK;
    if (plan->exec) {
      cudaError_t e = cudaGraphLaunch(plan->exec, st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "graph launch");
    } else {
      uint32_t launches = 0;
      s = enqueue_groups(ctx, plan->groups, static_cast<char*>(plan->dev), plan->queue_off, plan->status, plan->flags, st,
                         plan->side, plan->fork, plan->joins, &launches);
    }
    if (a && b) {
      cudaEventRecord(b, st);
      ctx->spans.push_back({0, a, b});
    }
    ctx->launches[0] += plan->kernels;
    return s;
  });
}

mr_status mr_plan_info(const mr_plan* plan, uint32_t* kernels, uint32_t* groups, uint64_t* device_bytes,
                       double* products) {
  if (!plan) return MR_ERR_ARG;
  if (kernels) *kernels = plan->kernels;
  if (groups) *groups = (uint32_t)plan->groups.size();
  if (device_bytes) *device_bytes = plan->dev_bytes;
  if (products) *products = plan->products;
  return MR_OK;
}

void mr_plan_free(mr_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->ctx->device);
  cudaDeviceSynchronize();
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  for (auto s : plan->side) cudaStreamDestroy(s);
  for (auto ev : plan->joins) cudaEventDestroy(ev);
  if (plan->fork) cudaEventDestroy(plan->fork);
  if (plan->dev) cudaFree(plan->dev);
  delete plan;
}

mr_status mr_modexp_batch_noalloc(mr_ctx* ctx, const mr_key* key, size_t n, const uint32_t* x, uint32_t x_stride,
                                  const uint32_t* e, uint32_t e_stride, uint32_t* out, uint32_t out_stride,
                                  uint8_t* dev_status, void* stream) {
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!key || key->ctx != ctx || !x || !e || !out || !x_stride || !e_stride || !out_stride)
    return fail(ctx, MR_ERR_ARG, "null argument, zero stride or foreign key");
  if (n > 0xffffffffull) return fail(ctx, MR_ERR_ARG, "batch too large");
  if (out_stride < key->pub.nlimbs()) return fail(ctx, MR_ERR_ARG, "out_stride smaller than the modulus");
  cudaSetDevice(ctx->device);
  NoallocCall c{};
  c.device = ctx->device;
  c.class_bits = key->pub.cls->host.L;
  c.cls = key->pub.cls->dev;
  c.key = key->pub.dev;
  c.x = x;
  c.e = e;
  c.out = out;
  c.status = dev_status;
  c.n = (uint32_t)n;
  c.x_stride = x_stride;
  c.e_stride = e_stride;
  c.out_stride = out_stride;
  c.wbits = choose_window(32 * e_stride, 0, window_cap(key->pub.cls));
  c.stream = (cudaStream_t)stream;
  std::string err;
  int rc = noalloc_modexp(c, err);
  return rc ? fail(ctx, (mr_status)rc, err) : MR_OK;
}

mr_status mr_profile_enable(mr_ctx* ctx, int on) {
  if (!ctx) return MR_ERR_ARG;
  ctx->prof_on = on != 0;
  return MR_OK;
}

mr_status mr_profile_read(mr_ctx* ctx, mr_kernel_time* times, uint32_t n_kinds) {
  if (!ctx || (n_kinds && !times) || n_kinds > 2) return fail(ctx, MR_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  double ms[2] = {0, 0};
  cudaError_t err = cudaSuccess;
  for (auto& sp : ctx->spans) {
    cudaError_t e = cudaEventSynchronize(sp.b);
    float t = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, sp.a, sp.b);
    if (e != cudaSuccess) err = e;
    ms[sp.kind] += t;
    ctx->free_events.push_back(sp.a);
    ctx->free_events.push_back(sp.b);
  }
  ctx->spans.clear();
  for (uint32_t k = 0; k < n_kinds; k++) {
    times[k].launches = ctx->launches[k];
    times[k].ms = ms[k];
  }
  ctx->launches[0] = ctx->launches[1] = 0;
  return err == cudaSuccess ? MR_OK : cuda_fail(ctx, err, "profile events");
}

mr_status mr_imad_peak(mr_ctx* ctx, uint32_t kind, void* stream, double* per_second) {
  if (!ctx || !per_second || kind > 3) return fail(ctx, MR_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  cudaError_t e = mr::imad_stream_rate(ctx->device, (cudaStream_t)stream, (int)kind, per_second);
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "integer-multiply probe");
}

mr_status mr_tensor_peak(mr_ctx* ctx, uint32_t kind, void* stream, double* ops_per_second) {
  if (!ctx || !ops_per_second || kind > 2) return fail(ctx, MR_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  cudaError_t e = mr::tensor_rate(ctx->device, (cudaStream_t)stream, (int)kind, ops_per_second);
  if (e == cudaErrorLaunchTimeout) return fail(ctx, MR_ERR_TIMEOUT, "tensor probe: completion wait ran out");
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "tensor probe");
}

mr_status mr_debug_tc_mma(mr_ctx* ctx, const uint16_t* a, const uint16_t* b, uint32_t n, uint32_t kdim,
                          uint32_t swap_strides, float* d, void* stream) {
  // with exchanged offsets the tensor core reads up to 16 x 16 * rows bytes past each operand's start:
  // inside the 32 KB operand regions only for a single K step; A in tensor memory takes columns
  // n .. n + kdim/2 of the 256 allocated, so n <= 128 there; otherwise n <= 256 (32 KB of B at kdim 64)
  const uint32_t n_max = (swap_strides == 0 || swap_strides == 3) ? 256u : 128u;
  if (!ctx || !a || !b || !d || n < 16 || n > n_max || n % 16 || kdim < 16 || kdim > 64 || kdim % 16 ||
      swap_strides > 3 || (swap_strides == 1 && kdim != 16))
    return fail(ctx, MR_ERR_ARG, "bad arguments");
  cudaSetDevice(ctx->device);
  cudaError_t e = mr::tensor_debug_mma(a, b, n, kdim, swap_strides, d, (cudaStream_t)stream);
  if (e == cudaErrorLaunchTimeout) return fail(ctx, MR_ERR_TIMEOUT, "tensor product: completion wait ran out");
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "tensor product");
}

mr_status mr_set_constant_time(mr_ctx* ctx, int on) {
  if (!ctx) return MR_ERR_ARG;
  ctx->constant_time = on != 0;
  return MR_OK;
}

mr_status mr_debug_big_phases(mr_ctx* ctx, int on, uint64_t* out) {
  if (!ctx) return MR_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaSuccess;
  if (out) {
    std::vector<unsigned long long> h(BIG_PHASES + 1, 0);
    if (ctx->big_phases) {
      e = cudaDeviceSynchronize();
      if (e == cudaSuccess) e = cudaMemcpy(h.data(), ctx->big_phases, h.size() * 8, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemset(ctx->big_phases, 0, h.size() * 8);
    }
    for (size_t i = 0; i < h.size(); i++) out[i] = h[i];
  }
  if (e == cudaSuccess && on && !ctx->big_phases) {
    e = cudaMalloc(&ctx->big_phases, (BIG_PHASES + 1) * 8);
    if (e == cudaSuccess) e = cudaMemset(ctx->big_phases, 0, (BIG_PHASES + 1) * 8);
  } else if (e == cudaSuccess && !on && ctx->big_phases) {
    e = cudaDeviceSynchronize();
    cudaFree(ctx->big_phases);
    ctx->big_phases = nullptr;
  }
  return e == cudaSuccess ? MR_OK : cuda_fail(ctx, e, "phase counters");
}

mr_status mr_debug_lane_tc_wait(mr_ctx* ctx, int skip) {
  if (!ctx) return MR_ERR_ARG;
  ctx->lane_tc_skip = skip != 0;
  return MR_OK;
}

mr_status mr_debug_big_wait(mr_ctx* ctx, uint32_t spin_limit, int32_t absent_slice) {
  if (!ctx || absent_slice < -1) return fail(ctx, MR_ERR_ARG, "bad arguments");
  ctx->big_spin_limit = spin_limit;
  ctx->big_absent_slice = absent_slice;
  return MR_OK;
}

mr_status mr_debug_mr_setup(mr_ctx* ctx, const uint32_t* cand, uint32_t n_limbs, size_t n, uint32_t* dev_out,
                            void* stream) {
  if (!ctx || !cand || !dev_out || !n_limbs) return MR_ERR_ARG;
  // one round with witness 2 for every candidate, constants published to dev_out
  uint32_t L = class_for_bits(32 * n_limbs);
  if (!L) return fail(ctx, MR_ERR_SIZE, "candidates longer than the largest size class");
  void* tmp = nullptr;
  size_t wbytes = n * n_limbs * 4;
  cudaError_t e = cudaMallocFromPoolAsync(&tmp, wbytes + n, ctx->pool, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "debug scratch");
  std::vector<uint32_t> w(n * n_limbs, 0);
  for (size_t i = 0; i < n; i++) w[i * n_limbs] = 2;
  cudaMemcpyAsync(tmp, w.data(), wbytes, cudaMemcpyHostToDevice, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  ctx->mr_dbg = dev_out;
  mr_status s = mr_miller_rabin_batch(ctx, cand, n_limbs, n, static_cast<uint32_t*>(tmp), 1,
                                      static_cast<uint8_t*>(tmp) + wbytes, nullptr, stream);
  ctx->mr_dbg = nullptr;
  cudaFreeAsync(tmp, (cudaStream_t)stream);
  return s;
}

mr_status mr_class_variants(uint32_t class_bits, uint32_t* count, uint32_t* lanes_per_number, uint32_t capacity) {
  const ClassKernels* k = class_kernels(class_bits);
  if (!k) return MR_ERR_SIZE;
  const uint32_t nv = k->big ? k->n_big : k->n_variants;
  if (count) *count = nv;
  if (lanes_per_number)
    for (uint32_t i = 0; i < nv && i < capacity; i++)
      lanes_per_number[i] = k->big ? k->big[i].slices * (k->big[i].threads / 32) : k->var[i].tpi;
  return MR_OK;
}

mr_status mr_lane_variant_info(uint32_t class_bits, uint32_t variant, uint32_t* out) {
  const ClassKernels* k = class_kernels(class_bits);
  if (!k || k->big) return MR_ERR_SIZE;
  if (!out || variant >= k->n_variants) return MR_ERR_ARG;
  const KernelVariant& v = k->var[variant];
  out[0] = v.tpi;
  out[1] = v.threads;
  out[2] = v.ipb;
  out[3] = v.tc;
  return MR_OK;
}

mr_status mr_set_variant(mr_ctx* ctx, uint32_t class_bits, uint32_t variant) {
  if (!ctx) return MR_ERR_ARG;
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    ClassEntry* ce = nullptr;
    mr_status s = get_class(ctx, class_bits, &ce);
    if (s) return s;
    if (variant >= ce->n_var()) return fail(ctx, MR_ERR_ARG, "no such variant");
    ce->variant = variant;
    ce->pinned = true;
    return MR_OK;
  });
}

mr_status mr_get_tuning(mr_ctx* ctx, uint32_t class_bits, uint32_t* variant, uint32_t* window_cap, uint32_t* tuned) {
  if (!ctx) return MR_ERR_ARG;
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    ClassEntry* ce = nullptr;
    mr_status s = get_class(ctx, class_bits, &ce);
    if (s) return s;
    if (variant) *variant = ce->variant;
    if (window_cap) *window_cap = ce->wcap;
    if (tuned) *tuned = ce->tuned ? 1u : 0u;
    return MR_OK;
  });
}

mr_status mr_set_tuning(mr_ctx* ctx, uint32_t class_bits, uint32_t variant, uint32_t window_cap) {
  if (!ctx) return MR_ERR_ARG;
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    ClassEntry* ce = nullptr;
    mr_status s = get_class(ctx, class_bits, &ce);
    if (s) return s;
    if (variant >= ce->n_var()) return fail(ctx, MR_ERR_ARG, "no such variant");
    if (window_cap > (ce->big() ? 8u : 6u)) return fail(ctx, MR_ERR_ARG, "window cap out of range");
    ce->variant = variant;
    ce->wcap = window_cap;
    ce->pinned = true;
    ce->tuned = true;
    return MR_OK;
  });
}

mr_status mr_autotune(mr_ctx* ctx, uint32_t class_bits, uint32_t n_items, uint32_t exp_bits, mr_tune_result* res) {
  NvtxRange nvtx_("mr_autotune");
  if (!ctx) return MR_ERR_ARG;
  if (!n_items || !exp_bits || n_items > (1u << 20) || exp_bits > 65536)
    return fail(ctx, MR_ERR_ARG, "n_items and exp_bits must be positive (n_items <= 2^20, exp_bits <= 65536)");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    uint32_t L = class_for_bits(class_bits);
    if (!L) return fail(ctx, MR_ERR_SIZE, "no size class holds " + std::to_string(class_bits) + "-bit moduli");
    ClassEntry* ce = nullptr;
    mr_status s = get_class(ctx, L, &ce);
    if (s) return s;
    return autotune_class(ctx, ce, n_items, exp_bits, res);
  });
}

static mr_status copy_table(const std::vector<uint32_t>& v, uint32_t* out, size_t cap, size_t* count) {
  if (count) *count = v.size();
  if (!out) return MR_OK;
  if (cap < v.size()) return MR_ERR_ARG;
  std::copy(v.begin(), v.end(), out);
  return MR_OK;
}

static std::vector<uint32_t> rns_vec(const ClassHost& c, const Big& X) { return residues(c, X); }

static mr_status debug_class_table(const ClassHost& c, const std::string& nm, uint32_t* out, size_t cap, size_t* count) {
  if (nm == "B") return copy_table(c.B, out, cap, count);
  if (nm == "Bp") return copy_table(c.Bp, out, cap, count);
  if (nm == "M_mi_inv") return copy_table(c.M_mi_inv, out, cap, count);
  if (nm == "M_mi_Bp") return copy_table(c.M_mi_Bp, out, cap, count);
  if (nm == "Minv_Bp") return copy_table(c.Minv_Bp, out, cap, count);
  if (nm == "Mp_mj_inv") return copy_table(c.Mp_mj_inv, out, cap, count);
  if (nm == "Mp_mj_B") return copy_table(c.Mp_mj_B, out, cap, count);
  if (nm == "Mp_B") return copy_table(c.Mp_B, out, cap, count);
  if (nm == "M") return copy_table(c.M.limbs(c.WX), out, cap, count);
  if (nm == "bound") return copy_table({(uint32_t)c.bound, (uint32_t)(c.bound >> 32)}, out, cap, count);
  return MR_ERR_ARG;
}

static mr_status debug_key_table(const ClassHost& c, const KeyHost& k, const std::string& nm, uint32_t* out,
                                 size_t cap, size_t* count) {
  if (nm == "kxi") return copy_table(k.kxi, out, cap, count);
  if (nm == "NMinv_Bp") return copy_table(k.NMinv_Bp, out, cap, count);
  if (nm == "one") return copy_table(rns_vec(c, k.one), out, cap, count);
  if (nm == "r2") return copy_table(rns_vec(c, k.r2), out, cap, count);
  if (nm == "r2h") return copy_table(rns_vec(c, k.r2h), out, cap, count);
  return MR_ERR_ARG;
}

mr_status mr_debug_table(mr_ctx* ctx, uint32_t class_bits, const mr_key* key, const char* name, uint32_t* out,
                         size_t capacity, size_t* count) {
  if (!name) return fail(ctx, MR_ERR_ARG, "null name");
  return guarded(ctx, [&]() -> mr_status {
    std::string nm(name);
    if (key) return debug_key_table(key->pub.cls->host, key->pub.host, nm, out, capacity, count);
    std::string err;
    const ClassHost* c = host_class(class_bits, err);
    if (!c) return fail(ctx, MR_ERR_SIZE, err);
    mr_status s = debug_class_table(*c, nm, out, capacity, count);
    return s ? fail(ctx, s, "unknown table or buffer too small") : MR_OK;
  });
}

mr_status mr_big_variant_info(uint32_t class_bits, uint32_t variant, uint32_t* slice_channels, uint32_t* slices,
                              uint32_t* tensor) {
  const ClassKernels* kern = class_kernels(class_bits);
  if (!kern) return MR_ERR_SIZE;
  if (!kern->big || variant >= kern->n_big) return MR_ERR_ARG;
  const BigKernel& bk = kern->big[variant];
  if (slice_channels) *slice_channels = bk.sc;
  if (slices) *slices = bk.slices;
  if (tensor) *tensor = bk.tc;
  return MR_OK;
}

mr_status mr_debug_tc_slices(uint32_t class_bits, uint32_t* out, size_t capacity, size_t* count) {
  try {
    std::string err;
    const ClassHost* c = host_class(class_bits, err);
    if (!c) return MR_ERR_SIZE;
    const ClassOff o = class_offsets(c->k, c->W, c->WX);
    std::vector<uint32_t> ts;
    if (!tc_slice_table(c->block.data() + o.T1, c->block.data() + o.T2, c->k, 32, (c->k + 31) / 32, ts))
      return MR_ERR_SIZE;
    if (count) *count = ts.size();
    if (!out) return MR_OK;
    if (capacity < ts.size()) return MR_ERR_ARG;
    std::copy(ts.begin(), ts.end(), out);
    return MR_OK;
  } catch (...) {
    return MR_ERR_ARG;
  }
}

mr_status mr_debug_big_variant(uint32_t class_bits, size_t n_items, uint32_t sms, uint32_t ctas_per_sm,
                               uint32_t* variant, uint32_t* slots) {
  const ClassKernels* kern = class_kernels(class_bits);
  if (!kern) return MR_ERR_SIZE;
  if (!kern->big || !sms || !ctas_per_sm || !n_items || !variant || !slots) return MR_ERR_ARG;
  int occ[MAX_VARIANTS];
  for (int v = 0; v < MAX_VARIANTS; v++) occ[v] = (int)ctas_per_sm;
  return pick_big_variant(kern, (n_items + 31) / 32, (int)sms, occ, -1, variant, slots) ? MR_OK : MR_ERR_SIZE;
}

mr_status mr_debug_crt_bin_host(const uint32_t* p, const uint32_t* q, const uint32_t* qinv, uint32_t n_limbs,
                                uint32_t W, uint32_t* out, size_t capacity, size_t* count) {
  if (!p || !q || !qinv || !n_limbs || W < n_limbs || W > CRT_BIN_MAX_W) return MR_ERR_ARG;
  try {
    const Big bp = big_from(p, n_limbs), bq = big_from(q, n_limbs), bqi = big_from(qinv, n_limbs);
    if (!bp.bit(0)) return MR_ERR_EVEN_MODULUS;
    std::vector<uint32_t> blk = build_crt_bin(W, bp, bq, bqi);
    if (count) *count = blk.size();
    if (!out) return MR_OK;
    if (capacity < blk.size()) return MR_ERR_ARG;
    std::copy(blk.begin(), blk.end(), out);
    return MR_OK;
  } catch (...) {
    return MR_ERR_ARG;
  }
}

mr_status mr_debug_trial_table(uint32_t* out, size_t capacity, size_t* count) {
  try {
    if (count) *count = trial_table_words();
    if (!out) return MR_OK;
    if (capacity < trial_table_words()) return MR_ERR_ARG;
    std::vector<uint32_t> t = trial_tables_host();
    std::copy(t.begin(), t.end(), out);
    return MR_OK;
  } catch (...) {
    return MR_ERR_ARG;
  }
}

mr_status mr_debug_key_table_host(const uint32_t* N, uint32_t n_limbs, const char* name, uint32_t* out,
                                  size_t capacity, size_t* count) {
  if (!N || !n_limbs || !name) return MR_ERR_ARG;
  try {
    Big n = big_from(N, n_limbs);
    uint32_t L = class_for_bits((uint32_t)n.bits());
    if (!L) return MR_ERR_SIZE;
    std::string err;
    const ClassHost* c = host_class(L, err);
    if (!c) return MR_ERR_SIZE;
    KeyHost kh;
    int rc = build_key(*c, n, nullptr, kh, err);
    if (rc) return (mr_status)rc;
    return debug_key_table(*c, kh, std::string(name), out, capacity, count);
  } catch (...) {
    return MR_ERR_ARG;
  }
}

}  // extern "C"
