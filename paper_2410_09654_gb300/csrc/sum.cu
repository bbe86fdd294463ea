// Sums: creation, upload/download, memory, status strings, the output-hash tables
// and small validation kernels.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace ps {

// ----------------------------------------------------------------------------- errors
static thread_local std::string g_last_cuda_error;

void set_cuda_error(cudaError_t e, const char* where) {
  g_last_cuda_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e) + " (" + where + ")";
}

// ----------------------------------------------------------------------------- memory
static std::atomic<int64_t> g_fail_after{0};

// Freed blocks are kept in size classes (8 per power of two) per stream and handed back
// to later requests of the same class on the same stream, so steady-state iterations do
// not make the stream-ordered pool map new memory when their sizes drift slightly.
namespace {
struct CachedBlock {
  void* p;
  size_t bytes;
};
std::mutex g_cache_mu;
std::map<std::pair<cudaStream_t, size_t>, std::vector<CachedBlock>> g_cache;  // (stream, class) -> blocks
std::map<void*, size_t> g_live;                                               // pointer -> class bytes
size_t g_cached_bytes = 0;
constexpr size_t kCacheLimit = (size_t)96 << 30;  // keep at most this much in the cache

size_t size_class(size_t bytes) {
  if (bytes <= 4096) return 4096;
  int lg = 63 - __builtin_clzll((unsigned long long)(bytes - 1));  // 2^lg < bytes <= 2^(lg+1)
  size_t step = (size_t)1 << (lg - 3);                             // 8 classes per octave
  return ((bytes + step - 1) / step) * step;
}
}  // namespace

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  int64_t f = g_fail_after.load();
  if (f > 0) {
    if (g_fail_after.fetch_sub(1) == 1) return PS_ERR_NOMEM;
  }
  static std::once_flag once;
  std::call_once(once, [] {
    // Keep freed blocks in the pool instead of returning them to the driver.
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
  const size_t cls = size_class(bytes);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find({s, cls});
    if (it != g_cache.end() && !it->second.empty()) {
      CachedBlock b = it->second.back();
      it->second.pop_back();
      g_cached_bytes -= b.bytes;
      g_live[b.p] = b.bytes;
      *p = b.p;
      return PS_OK;
    }
  }
  cudaError_t e = cudaMallocAsync(p, cls, s);
  if (e == cudaErrorMemoryAllocation) {  // give the cache back to the pool and retry once
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      for (auto& kv : g_cache)
        for (auto& b : kv.second) cudaFreeAsync(b.p, kv.first.first);
      g_cache.clear();
      g_cached_bytes = 0;
    }
    e = cudaMallocAsync(p, cls, s);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      *p = nullptr;
      return PS_ERR_NOMEM;
    }
  }
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaMallocAsync");
    *p = nullptr;
    return PS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_live[*p] = cls;
  return PS_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) {  // not ours: hand straight back to the pool
    cudaFreeAsync(p, s);
    return;
  }
  const size_t cls = it->second;
  g_live.erase(it);
  if (g_cached_bytes + cls > kCacheLimit) {
    cudaFreeAsync(p, s);
    return;
  }
  g_cache[{s, cls}].push_back({p, cls});
  g_cached_bytes += cls;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

uint64_t key_mask(int n_sites) { return n_sites >= 64 ? ~0ull : ((1ull << n_sites) - 1); }

int sum_reserve(pauli_sum* s, int64_t cap, bool keep_contents) {
  if (cap <= s->cap) return PS_OK;
  int64_t nc = std::max<int64_t>(cap, 64);
  Rec* d = nullptr;
  const size_t rb = rec_bytes(s->W);
  PS_TRY(dev_alloc((void**)&d, (size_t)nc * rb, s->stream));
  if (keep_contents && s->n > 0) PS_CUDA(cudaMemcpyAsync(d, s->d, (size_t)s->n * rb, cudaMemcpyDeviceToDevice, s->stream));
  dev_free(s->d, s->stream);
  s->d = d;
  s->cap = nc;
  return PS_OK;
}

int sum_adopt(pauli_sum* s, Rec* d, int64_t cap, int64_t n) {
  dev_free(s->d, s->stream);
  s->d = d;
  s->cap = cap;
  s->n = n;
  return PS_OK;
}

// ----------------------------------------------------------------------------- output hash
static uint64_t splitmix(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct HashRows {
  uint64_t a[kHashRows], b[kHashRows];
  HashRows() {
    uint64_t s = 0x5EED2410096540ull;
    for (int j = 0; j < kHashRows; ++j) {
      a[j] = splitmix(s);
      b[j] = splitmix(s);
    }
  }
};
static const HashRows g_rows;

void host_hash_rows(const uint64_t** a, const uint64_t** b) {
  *a = g_rows.a;
  *b = g_rows.b;
}

uint32_t host_hash(uint64_t v, uint64_t w, int bits) {
  uint32_t f = 0;
  for (int j = 0; j < bits; ++j) {
    uint64_t t = (v & g_rows.a[j]) ^ (w & g_rows.b[j]);
    f |= (uint32_t)(__builtin_popcountll(t) & 1) << j;
  }
  return f;
}

// Solve F(v,w) = target on the low `bits` rows by Gaussian elimination over GF(2).
void host_key_with_hash(uint32_t target, int bits, uint64_t* v, uint64_t* w) {
  struct Row { uint64_t a, b; uint32_t rhs; };
  std::vector<Row> rows(bits);
  for (int j = 0; j < bits; ++j) rows[j] = {g_rows.a[j], g_rows.b[j], (target >> j) & 1u};
  std::vector<int> pivot_col(bits, -1);
  int r = 0;
  for (int col = 0; col < 128 && r < bits; ++col) {
    auto getbit = [&](const Row& x) { return col < 64 ? (x.a >> col) & 1 : (x.b >> (col - 64)) & 1; };
    int p = -1;
    for (int i = r; i < bits; ++i)
      if (getbit(rows[i])) { p = i; break; }
    if (p < 0) continue;
    std::swap(rows[p], rows[r]);
    for (int i = 0; i < bits; ++i)
      if (i != r && getbit(rows[i])) {
        rows[i].a ^= rows[r].a;
        rows[i].b ^= rows[r].b;
        rows[i].rhs ^= rows[r].rhs;
      }
    pivot_col[r] = col;
    ++r;
  }
  uint64_t kv = 0, kw = 0;
  for (int i = 0; i < r; ++i)
    if (rows[i].rhs) {
      int col = pivot_col[i];
      if (col < 64) kv |= 1ull << col; else kw |= 1ull << (col - 64);
    }
  *v = kv;
  *w = kw;
}

// ----------------------------------------------------------------------------- coefficient class
// ----------------------------------------------------------------------------- validation kernels

// Insert every key into an open-addressing table of 2^k 64-bit slots (empty = 0).  A slot
// holds the key's 24-bit fingerprint and its record index + 1 (40 bits), so that the table
// (8 bytes a slot, at most half full) stays small enough for L2; a slot with the same
// fingerprint is resolved by comparing the two records.  A key found already present is a
// duplicate.
__global__ void k_distinct(const Rec* __restrict__ d, int64_t n, unsigned long long* table, uint64_t tmask,
                           int* dup) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    const uint64_t kv = d[i].v, kw = d[i].w;
    const uint64_t h = key_hash64(kv, kw);  // low bits: the slot; top 24 bits: the fingerprint
    const unsigned long long fp = h >> 40;
    const unsigned long long mine = (fp << 40) | (unsigned long long)(i + 1);
    uint64_t slot = h & tmask;
    for (uint64_t probe = 0; probe <= tmask; ++probe) {
      const unsigned long long old = atomicCAS(&table[slot], 0ull, mine);
      if (old == 0ull) break;  // inserted
      if ((old >> 40) == fp) {
        const int64_t j = (int64_t)(old & ((1ull << 40) - 1)) - 1;
        if (d[j].v == kv && d[j].w == kw) {
          atomicOr(dup, 1);
          break;
        }
      }
      slot = (slot + 1) & tmask;
    }
  }
}

// The distinctness check without its synchronisation: *dup is set if two keys are equal
// (the table is sized and filled here and must live until the stream has run the kernel).
int distinct_launch(const Rec* d, int64_t n, cudaStream_t s, Buf<unsigned long long>& table, int* dup) {
  if (n >= (int64_t)(1ull << 40) - 1) return PS_ERR_INVALID;  // record indices must fit the slot
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * n)) slots <<= 1;
  PS_TRY(table.alloc(slots, s));
  PS_CUDA(cudaMemsetAsync(table.p, 0, slots * sizeof(unsigned long long), s));
  int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
  PS_LAUNCH("k_distinct", s, k_distinct<<<blocks, 256, 0, s>>>(d, n, table.p, slots - 1, dup));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

// Device address of caller memory the device can read or write directly: device memory, or
// pinned host memory mapped into the device's address space (its device alias).  Null for
// pageable host memory and for memory of another device.
void* device_alias(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return at.device == dev ? at.devicePointer : nullptr;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer;
  return nullptr;
}

}  // namespace ps

using namespace ps;

// ============================================================================= C ABI
extern "C" {

const char* pauli_status_string(int status) {
  switch (status) {
    case PS_OK: return "ok";
    case PS_ERR_INVALID: return "invalid argument";
    case PS_ERR_CAPACITY: return "capacity too small";
    case PS_ERR_TABLE_FULL: return "merge table full";
    case PS_ERR_CUDA: return "CUDA error";
    case PS_ERR_TIMEOUT: return "device wait timed out";
    case PS_ERR_KRYLOV_EXHAUSTED: return "Krylov space exhausted (b_n = 0)";
    case PS_ERR_NOMEM: return "device out of memory";
    case PS_ERR_UNCERTAIN: return "result rounding uncertain";
    case PS_ERR_NONFINITE: return "non-finite norm (a coefficient overflowed or is NaN)";
    case PS_ERR_IO: return "checkpoint file error";
    default: return "unknown status";
  }
}

const char* pauli_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int pauli_debug_fail_alloc_after(int64_t n) {
  g_fail_after.store(n < 0 ? 0 : n);
  return PS_OK;
}

int pauli_debug_output_hash(const uint64_t* v, const uint64_t* w, int64_t n, uint32_t* out) {
  if (n < 0 || (n > 0 && (!v || !w || !out))) return PS_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i) out[i] = host_hash(v[i], w[i], kHashRows);
  return PS_OK;
}

int pauli_sum_create(int n_sites, int64_t capacity, void* cuda_stream, pauli_sum** out) {
  if (!out || n_sites < 1 || n_sites > 256 || capacity < 0) return PS_ERR_INVALID;
  *out = nullptr;
  PS_TRY(upload_hash_tables());
  pauli_sum* s = new pauli_sum{n_sites, (cudaStream_t)cuda_stream, nullptr, 0, 0, 0, 0, words_for(n_sites)};
  int st = sum_reserve(s, std::max<int64_t>(capacity, 64), false);
  if (st != PS_OK) {
    delete s;
    return st;
  }
  *out = s;
  return PS_OK;
}

int pauli_sum_destroy(pauli_sum* s) {
  if (!s) return PS_ERR_INVALID;
  dev_free(s->d, s->stream);
  delete s;
  return PS_OK;
}

int pauli_sum_n_sites(const pauli_sum* s, int* n_sites) {
  if (!s || !n_sites) return PS_ERR_INVALID;
  *n_sites = s->n_sites;
  return PS_OK;
}

int pauli_sum_size(const pauli_sum* s, int64_t* n) {
  if (!s || !n) return PS_ERR_INVALID;
  PS_CUDA(cudaStreamSynchronize(s->stream));
  *n = s->n;
  return PS_OK;
}

// Pack four arrays into records and validate in the same pass: flags[0] = 1 if a string has
// bits outside the key mask, flags[1] |= the coefficient class (bit 0: a non-zero real part,
// bit 1: a non-zero imaginary part).
// ----------------------------------------------------------------------------- hash order
// The first kOrdBits rows of the merge's output hash F.  Merge outputs come out grouped by
// F's low rows; an operand in that order lets a warp of an emission reserve output slots for
// neighbouring strings in few bins.  pauli_sum_sort_by_hash puts any sum in that order.
constexpr int kOrdBits = 16;
__constant__ uint64_t c_ordA[kOrdBits], c_ordB[kOrdBits];

__global__ void k_ord_key(const Rec* __restrict__ d, int64_t n, uint32_t* __restrict__ key,
                          unsigned* __restrict__ hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Rec r = d[i];
    uint32_t f = 0;
#pragma unroll
    for (int j = 0; j < kOrdBits; ++j) f |= (uint32_t)(__popcll((r.v & c_ordA[j]) ^ (r.w & c_ordB[j])) & 1) << j;
    key[i] = f;
    atomicAdd(&hist[f], 1u);
  }
}

__global__ void k_ord_scatter(const Rec* __restrict__ d, int64_t n, const uint32_t* __restrict__ key,
                              unsigned long long* __restrict__ cur, Rec* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[atomicAdd(&cur[key[i]], 1ull)] = d[i];
}

__global__ void k_pack(Rec* __restrict__ d, const uint64_t* __restrict__ v, const uint64_t* __restrict__ w,
                       const double* __restrict__ re, const double* __restrict__ im, int64_t n, uint64_t inv_mask,
                       int* __restrict__ flags) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0, c = 0;
  for (; i < n; i += stride) {
    const Rec r{v[i], w[i], re[i], im[i]};
    d[i] = r;
    bad |= ((r.v | r.w) & inv_mask) != 0;
    // non-finite coefficients (exponent all ones) are rejected like out-of-range key bits
    bad |= ((__double_as_longlong(r.re) >> 52) & 0x7FF) == 0x7FF || ((__double_as_longlong(r.im) >> 52) & 0x7FF) == 0x7FF;
    c |= (((__double_as_longlong(r.re) << 1) != 0) ? 1 : 0) | (((__double_as_longlong(r.im) << 1) != 0) ? 2 : 0);
  }
  bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
  c = __reduce_or_sync(0xffffffffu, (unsigned)c);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&flags[0], 1);
    if (c) atomicOr(&flags[1], c);
  }
}

int pauli_sum_upload(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re, const double* im,
                     int64_t n) {
  if (!s || n < 0 || (n > 0 && (!v || !w || !re || !im))) return PS_ERR_INVALID;
  if (s->W > 1) return wide_api::upload(s, v, w, re, im, n, true);
  PS_TRY(sum_reserve(s, n, false));
  s->n = 0;
  // The records are packed by one pass that also checks the key bits and the coefficient
  // class: straight from the caller's arrays when they are pinned host memory mapped into the
  // device's address space (the pass reads them over the host link), else from a staging
  // copy.  One pass inserts the keys for the distinctness check; a single synchronisation
  // reads every flag (the caller's host arrays may be released then).
  Buf<uint64_t> stage;
  Buf<int> flags;
  Buf<unsigned long long> table;
  PS_TRY(flags.alloc(4, s->stream));
  PS_CUDA(cudaMemsetAsync(flags.p, 0, 4 * sizeof(int), s->stream));
  if (n > 0) {
    const uint64_t* dv = static_cast<const uint64_t*>(device_alias(v));
    const uint64_t* dw = static_cast<const uint64_t*>(device_alias(w));
    const double* dre = static_cast<const double*>(device_alias(re));
    const double* dim = static_cast<const double*>(device_alias(im));
    if (!dv || !dw || !dre || !dim) {
      PS_TRY(stage.alloc((size_t)n * 4, s->stream));
      uint64_t* sv = stage.p;
      uint64_t* sw = stage.p + n;
      double* sre = reinterpret_cast<double*>(stage.p + 2 * n);
      double* sim = reinterpret_cast<double*>(stage.p + 3 * n);
      const size_t bytes = (size_t)n * sizeof(uint64_t);
      PS_CUDA(cudaMemcpyAsync(sv, v, bytes, cudaMemcpyHostToDevice, s->stream));
      PS_CUDA(cudaMemcpyAsync(sw, w, bytes, cudaMemcpyHostToDevice, s->stream));
      PS_CUDA(cudaMemcpyAsync(sre, re, bytes, cudaMemcpyHostToDevice, s->stream));
      PS_CUDA(cudaMemcpyAsync(sim, im, bytes, cudaMemcpyHostToDevice, s->stream));
      dv = sv;
      dw = sw;
      dre = sre;
      dim = sim;
    }
    int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
    PS_LAUNCH("k_pack", s->stream,
              k_pack<<<blocks, 256, 0, s->stream>>>(s->d, dv, dw, dre, dim, n, ~key_mask(s->n_sites), flags.p));
    PS_CUDA(cudaGetLastError());
  }
  if (n > 1) PS_TRY(distinct_launch(s->d, n, s->stream, table, flags.p + 2));
  int h[4] = {0, 0, 0, 0};
  PS_CUDA(cudaMemcpyAsync(h, flags.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  PS_CUDA(cudaStreamSynchronize(s->stream));
  if (h[0] || h[2]) return PS_ERR_INVALID;
  s->cls = h[1];
  s->n = n;
  return round_f32(s);
}

__global__ void k_unpack(const Rec* __restrict__ d, uint64_t* __restrict__ v, uint64_t* __restrict__ w,
                         double* __restrict__ re, double* __restrict__ im, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    Rec r = d[i];
    v[i] = r.v;
    w[i] = r.w;
    re[i] = r.re;
    im[i] = r.im;
  }
}

int pauli_sum_upload_device(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re,
                            const double* im, int64_t n) {
  if (!s || n < 0 || (n > 0 && (!v || !w || !re || !im))) return PS_ERR_INVALID;
  if (n > 0) {  // device memory, or mapped pinned host memory (read over the host link)
    v = static_cast<const uint64_t*>(device_alias(v));
    w = static_cast<const uint64_t*>(device_alias(w));
    re = static_cast<const double*>(device_alias(re));
    im = static_cast<const double*>(device_alias(im));
    if (!v || !w || !re || !im) return PS_ERR_INVALID;
  }
  if (s->W > 1) return wide_api::upload(s, v, w, re, im, n, false);
  PS_TRY(sum_reserve(s, n, false));
  s->n = 0;
  Buf<int> flags;
  PS_TRY(flags.alloc(2, s->stream));
  PS_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), s->stream));
  if (n > 0) {
    int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
    PS_LAUNCH("k_pack", s->stream,
              k_pack<<<blocks, 256, 0, s->stream>>>(s->d, v, w, re, im, n, ~key_mask(s->n_sites), flags.p));
    PS_CUDA(cudaGetLastError());
  }
  int h[2] = {0, 0};
  PS_CUDA(cudaMemcpyAsync(h, flags.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  PS_CUDA(cudaStreamSynchronize(s->stream));
  if (h[0]) return PS_ERR_INVALID;
  s->cls = h[1];
  s->n = n;
  return round_f32(s);
}

int pauli_sum_download(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im, int64_t cap,
                       int64_t* n) {
  if (!s || !n) return PS_ERR_INVALID;
  PS_CUDA(cudaStreamSynchronize(s->stream));
  *n = s->n;
  if (cap < s->n) return PS_ERR_CAPACITY;
  if (s->n == 0) return PS_OK;
  if (!v || !w || !re || !im) return PS_ERR_INVALID;
  if (s->W > 1) return wide_api::download(s, v, w, re, im);
  std::vector<Rec> h((size_t)s->n);
  PS_CUDA(cudaMemcpyAsync(h.data(), s->d, (size_t)s->n * sizeof(Rec), cudaMemcpyDeviceToHost, s->stream));
  PS_CUDA(cudaStreamSynchronize(s->stream));
  std::sort(h.begin(), h.end(), [](const Rec& a, const Rec& b) { return a.v < b.v || (a.v == b.v && a.w < b.w); });
  for (int64_t i = 0; i < s->n; ++i) {
    v[i] = h[(size_t)i].v;
    w[i] = h[(size_t)i].w;
    re[i] = h[(size_t)i].re;
    im[i] = h[(size_t)i].im;
  }
  return PS_OK;
}

int pauli_sum_download_device(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im, int64_t cap,
                              int64_t* n) {
  if (!s || !n) return PS_ERR_INVALID;
  *n = s->n;
  if (cap < s->n) return PS_ERR_CAPACITY;
  if (s->n == 0) return PS_OK;
  if (!v || !w || !re || !im) return PS_ERR_INVALID;
  // device memory, or pinned host memory mapped into the device's address space (written
  // over the host link by the unpacking pass itself)
  uint64_t* dv = static_cast<uint64_t*>(device_alias(v));
  uint64_t* dw = static_cast<uint64_t*>(device_alias(w));
  double* dre = static_cast<double*>(device_alias(re));
  double* dim = static_cast<double*>(device_alias(im));
  if (!dv || !dw || !dre || !dim) return PS_ERR_INVALID;
  if (s->W > 1) return wide_api::download_device(s, dv, dw, dre, dim);
  int blocks = (int)std::min<int64_t>(ceil_div(s->n, 256), 8 * num_sms());
  PS_LAUNCH("k_unpack", s->stream, k_unpack<<<blocks, 256, 0, s->stream>>>(s->d, dv, dw, dre, dim, s->n));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int pauli_sum_copy(const pauli_sum* src, pauli_sum* dst) {
  if (!src || !dst || src->n_sites != dst->n_sites) return PS_ERR_INVALID;
  if (src == dst) return PS_OK;
  PS_TRY(sum_reserve(dst, src->n, false));
  if (src->n > 0) {
    if (src->stream != dst->stream) PS_CUDA(cudaStreamSynchronize(src->stream));
    PS_CUDA(cudaMemcpyAsync(dst->d, src->d, (size_t)src->n * rec_bytes(src->W), cudaMemcpyDeviceToDevice, dst->stream));
  }
  dst->n = src->n;
  dst->cls = src->cls;
  return round_f32(dst);
}

int pauli_sum_set_precision(pauli_sum* s, int coef_dtype) {
  if (!s || (coef_dtype != PS_COEF_F64 && coef_dtype != PS_COEF_F32 && coef_dtype != PS_COEF_F32C))
    return PS_ERR_INVALID;
  if (s->W > 1 && coef_dtype != PS_COEF_F64) return PS_ERR_INVALID;
  s->f32 = coef_dtype;  // 0 FP64, 1 FP32, 2 FP32 with compensated sums
  return round_f32(s);
}

int pauli_sum_precision(const pauli_sum* s, int* coef_dtype) {
  if (!s || !coef_dtype) return PS_ERR_INVALID;
  *coef_dtype = s->f32;
  return PS_OK;
}

// ----------------------------------------------------------------------------- checkpoint
namespace {

constexpr char kCkpMagic[8] = {'P', 'S', 'U', 'M', 'C', 'K', 'P', '1'};

struct Fnv {
  uint64_t h = 0xCBF29CE484222325ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 0x100000001B3ull;
    }
  }
};

bool put(std::FILE* f, Fnv& fnv, const void* p, size_t n) {
  fnv.add(p, n);
  return std::fwrite(p, 1, n, f) == n;
}

bool get(std::FILE* f, Fnv& fnv, void* p, size_t n) {
  if (std::fread(p, 1, n, f) != n) return false;
  fnv.add(p, n);
  return true;
}

}  // namespace

int pauli_sum_save(const pauli_sum* s, const char* path, const double* meta, int64_t n_meta) {
  if (!s || !path || n_meta < 0 || n_meta > (1 << 20) || (n_meta > 0 && !meta)) return PS_ERR_INVALID;
  PS_NARROW(s);
  const int64_t n = s->n;
  std::vector<uint64_t> v((size_t)n), w((size_t)n);
  std::vector<double> re((size_t)n), im((size_t)n);
  int64_t got = 0;
  PS_TRY(pauli_sum_download(s, v.data(), w.data(), re.data(), im.data(), n, &got));
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return PS_ERR_IO;
  Fnv fnv;
  const uint32_t hdr[4] = {1u, (uint32_t)s->n_sites, (uint32_t)s->f32, (uint32_t)n_meta};
  const uint64_t cnt = (uint64_t)n;
  bool ok = put(f, fnv, kCkpMagic, 8) && put(f, fnv, hdr, sizeof(hdr)) && put(f, fnv, &cnt, 8);
  if (ok && n_meta > 0) ok = put(f, fnv, meta, (size_t)n_meta * sizeof(double));
  for (int64_t i = 0; ok && i < n; ++i) {
    const Rec r{v[(size_t)i], w[(size_t)i], re[(size_t)i], im[(size_t)i]};
    ok = put(f, fnv, &r, sizeof(r));
  }
  const uint64_t sum = fnv.h;
  if (ok) ok = std::fwrite(&sum, 1, 8, f) == 8;
  if (std::fclose(f) != 0) ok = false;
  return ok ? PS_OK : PS_ERR_IO;
}

int pauli_sum_load(pauli_sum* s, const char* path, double* meta, int64_t meta_cap, int64_t* n_meta) {
  if (!s || !path || meta_cap < 0 || (meta_cap > 0 && !meta)) return PS_ERR_INVALID;
  PS_NARROW(s);
  std::FILE* f = std::fopen(path, "rb");
  if (!f) return PS_ERR_IO;
  Fnv fnv;
  char magic[8];
  uint32_t hdr[4];
  uint64_t cnt = 0;
  bool ok = get(f, fnv, magic, 8) && std::memcmp(magic, kCkpMagic, 8) == 0 && get(f, fnv, hdr, sizeof(hdr)) &&
            hdr[0] == 1u && hdr[2] <= (uint32_t)PS_COEF_F32 && hdr[3] <= (1u << 20) && get(f, fnv, &cnt, 8) &&
            cnt < ((uint64_t)1 << 40);
  std::vector<double> m(ok ? hdr[3] : 0);
  if (ok && !m.empty()) ok = get(f, fnv, m.data(), m.size() * sizeof(double));
  std::vector<uint64_t> v, w;
  std::vector<double> re, im;
  if (ok) {
    v.resize((size_t)cnt);
    w.resize((size_t)cnt);
    re.resize((size_t)cnt);
    im.resize((size_t)cnt);
  }
  for (uint64_t i = 0; ok && i < cnt; ++i) {
    Rec r;
    ok = get(f, fnv, &r, sizeof(r));
    v[i] = r.v;
    w[i] = r.w;
    re[i] = r.re;
    im[i] = r.im;
  }
  uint64_t sum = 0;
  if (ok) ok = std::fread(&sum, 1, 8, f) == 8 && sum == fnv.h;
  std::fclose(f);
  if (!ok) return PS_ERR_IO;
  if ((int)hdr[1] != s->n_sites) return PS_ERR_INVALID;
  const int old_f32 = s->f32;
  s->f32 = 0;  // the stored values are loaded as they are; the file's precision is set after
  const int st = pauli_sum_upload(s, v.data(), w.data(), re.data(), im.data(), (int64_t)cnt);
  if (st != PS_OK) {
    s->f32 = old_f32;
    return st;
  }
  s->f32 = hdr[2] <= (uint32_t)PS_COEF_F32C ? (int)hdr[2] : 0;
  if (n_meta) *n_meta = (int64_t)m.size();
  for (int64_t i = 0; i < std::min<int64_t>(meta_cap, (int64_t)m.size()); ++i) meta[i] = m[(size_t)i];
  return PS_OK;
}

int pauli_sum_sort_by_hash(pauli_sum* s) {
  if (!s) return PS_ERR_INVALID;
  PS_NARROW(s);
  const int64_t n = s->n;
  if (n <= 1) return PS_OK;
  cudaStream_t st = s->stream;
  static std::once_flag once;
  static cudaError_t up = cudaSuccess;
  std::call_once(once, [] {
    up = cudaMemcpyToSymbol(c_ordA, g_rows.a, kOrdBits * sizeof(uint64_t));
    if (up == cudaSuccess) up = cudaMemcpyToSymbol(c_ordB, g_rows.b, kOrdBits * sizeof(uint64_t));
  });
  PS_CUDA(up);
  constexpr int64_t nb = (int64_t)1 << kOrdBits;
  Buf<uint32_t> key, hist;
  Buf<uint64_t> off;
  PS_TRY(key.alloc((size_t)n, st));
  PS_TRY(hist.alloc((size_t)nb, st));
  PS_TRY(off.alloc((size_t)nb + 1, st));
  PS_CUDA(cudaMemsetAsync(hist.p, 0, nb * sizeof(uint32_t), st));
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
  PS_LAUNCH("k_ord_key", st, k_ord_key<<<blocks, 256, 0, st>>>(s->d, n, key.p, hist.p));
  PS_CUDA(cudaGetLastError());
  PS_TRY(scan_u32_to_u64(hist.p, off.p, nb, st));
  Rec* out = nullptr;
  PS_TRY(dev_alloc((void**)&out, (size_t)n * sizeof(Rec), st));
  PS_LAUNCH("k_ord_scatter", st,
            k_ord_scatter<<<blocks, 256, 0, st>>>(s->d, n, key.p, reinterpret_cast<unsigned long long*>(off.p), out));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    dev_free(out, st);
    set_cuda_error(e, "pauli_sum_sort_by_hash");
    return PS_ERR_CUDA;
  }
  return sum_adopt(s, out, n, n);
}

}  // extern "C"
