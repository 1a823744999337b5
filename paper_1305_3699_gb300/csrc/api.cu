// C ABI of the RNS modular-exponentiation library (declared in include/mr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "../../include/mr.h"
#include "kernels_api.h"
#include "noalloc.h"
#include "setup.h"

using namespace mr;

namespace {

struct ClassEntry {
  ClassHost host;
  uint32_t* dev = nullptr;
  const ClassKernels* kern = nullptr;
  uint32_t variant = 0;  // selected lane mapping
  const KernelVariant& kv() const { return kern->var[variant]; }
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
};

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
  {
    // default lane mapping: variant 0, unless MR_VARIANT_<L> names another compiled one
    std::string ev = "MR_VARIANT_" + std::to_string(L);
    const char* v = getenv(ev.c_str());
    if (v) {
      unsigned idx = (unsigned)atoi(v);
      if (idx < ce->kern->n_variants) ce->variant = idx;
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
uint32_t choose_window(uint32_t bits, uint32_t popcount_hint) {
  if (bits <= 1) return 1;
  uint64_t best = ~0ull;
  uint32_t bw = 1;
  for (uint32_t w = 1; w <= 6; w++) {
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
};

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
    b.scratch_words = b.mx.empty() ? 0 : modexp_scratch_words(b.ce->kv(), (uint32_t)b.mx.size(), b.wbits);
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
    const KernelVariant& k = b.ce->kv();
    if (!b.mx.empty()) {
      LaunchArgs a{b.ce->dev, base + b.off_mx, (uint32_t)b.mx.size(), b.wbits,
                   reinterpret_cast<uint32_t*>(base + b.off_scratch), status};
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

ClassBatch& batch_for(std::vector<ClassBatch>& v, std::map<ClassEntry*, size_t>& idx, ClassEntry* ce) {
  auto it = idx.find(ce);
  if (it != idx.end()) return v[it->second];
  idx[ce] = v.size();
  v.emplace_back();
  v.back().ce = ce;
  return v.back();
}

}  // namespace

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
  for (auto& kv : ctx->classes)
    if (kv.second->dev) cudaFree(kv.second->dev);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  if (ctx->staging_evt) cudaEventDestroy(ctx->staging_evt);
  for (auto& sp : ctx->spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  for (cudaEvent_t ev : ctx->free_events) cudaEventDestroy(ev);
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
      std::vector<uint32_t> crt = build_crt(key->p.cls->host, bp, bq, bqi);
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
      b.wbits = choose_window(32 * e_stride, 0);
    }
    return run_batches(ctx, batches, dev_status, (cudaStream_t)stream, 0);
  });
}

mr_status mr_rsa_encrypt(mr_ctx* ctx, const mr_key* const* keys, size_t n, const uint32_t* m, uint32_t m_stride,
                         uint32_t* c, uint32_t c_stride, uint8_t* dev_status, void* stream) {
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
      b.wbits = choose_window(cost_bits[b.ce], cost_pop[b.ce]);
    }
    return run_batches(ctx, batches, dev_status, (cudaStream_t)stream, 0);
  });
}

mr_status mr_rsa_decrypt_crt(mr_ctx* ctx, const mr_key* const* keys, size_t n, const uint32_t* c, uint32_t c_stride,
                             uint32_t* m, uint32_t m_stride, uint8_t* dev_status, void* stream) {
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
    for (auto& b : batches) b.wbits = choose_window(ebits[b.ce], 0);
    return run_batches(ctx, batches, dev_status, (cudaStream_t)stream, maxW);
  });
}

mr_status mr_miller_rabin_batch(mr_ctx* ctx, const uint32_t* cand, uint32_t n_limbs, size_t n, const uint32_t* witness,
                                uint32_t rounds, uint8_t* dev_is_probable_prime, uint32_t* dev_round_mask,
                                void* stream) {
  if (!ctx) return MR_ERR_ARG;
  if (n == 0) return MR_OK;
  if (!cand || !n_limbs || !witness || !rounds || !dev_is_probable_prime)
    return fail(ctx, MR_ERR_ARG, "null argument, zero limbs or zero rounds");
  if (dev_round_mask && rounds > 32) return fail(ctx, MR_ERR_ARG, "round mask holds at most 32 rounds");
  if (n > 0xffffffffull) return fail(ctx, MR_ERR_ARG, "batch too large");
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    uint32_t L = class_for_bits(32 * n_limbs);
    if (!L) return fail(ctx, MR_ERR_SIZE, "candidates longer than the largest size class");
    ClassEntry* ce = nullptr;
    mr_status s = get_class(ctx, L, &ce);
    if (s) return s;
    const KernelVariant& k = ce->kv();
    const uint32_t wbits = choose_window(32 * n_limbs, 0);
    const size_t tab_words = modexp_scratch_words(k, (uint32_t)n, wbits);
    const size_t crow_words = n * 3 * (size_t)ce->host.W;
    const size_t off_crow = align256(tab_words * 4);
    void* dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&dev, off_crow + crow_words * 4, ctx->pool, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(ctx, MR_ERR_OOM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    char* base = static_cast<char*>(dev);
    MRArgs a{ce->dev, cand, witness, dev_is_probable_prime, dev_round_mask, reinterpret_cast<uint32_t*>(base),
             reinterpret_cast<uint32_t*>(base + off_crow), (uint32_t)n, n_limbs, rounds, wbits, ctx->mr_dbg};
    unsigned grid = (unsigned)((n + k.ipb - 1) / k.ipb);
    e = timed_launch(ctx, 0, (cudaStream_t)stream, [&] { return k.mr(a, grid, (cudaStream_t)stream); });
    cudaError_t e2 = cudaFreeAsync(dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaFreeAsync");
    return MR_OK;
  });
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
  c.wbits = choose_window(32 * e_stride, 0);
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
  if (count) *count = k->n_variants;
  if (lanes_per_number)
    for (uint32_t i = 0; i < k->n_variants && i < capacity; i++) lanes_per_number[i] = k->var[i].tpi;
  return MR_OK;
}

mr_status mr_set_variant(mr_ctx* ctx, uint32_t class_bits, uint32_t variant) {
  if (!ctx) return MR_ERR_ARG;
  return guarded(ctx, [&]() -> mr_status {
    cudaSetDevice(ctx->device);
    ClassEntry* ce = nullptr;
    mr_status s = get_class(ctx, class_bits, &ce);
    if (s) return s;
    if (variant >= ce->kern->n_variants) return fail(ctx, MR_ERR_ARG, "no such variant");
    ce->variant = variant;
    return MR_OK;
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
