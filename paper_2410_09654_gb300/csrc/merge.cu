// The merge engine: all-pairs H x X string products (Alg. 1 with eq. eps_com),
// duplicate merging with the paper's summation order, and linear combinations.
//
// Data flow for one call (all on one stream):
//   1. bins: every output string c goes to bin F(c) (low b bits of a GF(2)-linear
//      hash).  For a product c = h ^ x, F(c) = F(h) ^ F(x), so the bin is known from
//      the factors.  A per-bin upper bound (histogram of F(x) XOR-convolved with the
//      F(h) of all H terms, plus the extra sources) gives each bin a fixed region.
//   2. emit: one thread per x streams X once, tests it against every H term held in
//      shared memory (XOR, AND, popcount parity) and appends a compact 8-byte entry
//      (x index, h index) to the bin of each anticommuting product.  Extra sources
//      append (index, source id) to bin F(y).
//   3. group: consecutive bins are grouped so that a group holds <= kCap entries.
//   4. merge: one CTA per group (persistent loop) rebuilds each contribution, inserts
//      the product keys in a shared-memory hash table, counts per key, scatters the
//      entries per key and sums each key's contributions in increasing order (H order,
//      then the sources in order).  That is exactly the order in which Alg. 1 with H
//      in the outer loop adds them, so the result is independent of scheduling.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "exact_sum.cuh"

namespace ps {

__constant__ uint64_t c_hashA[kHashRows];
__constant__ uint64_t c_hashB[kHashRows];

int upload_hash_tables() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    const uint64_t *a, *b;
    host_hash_rows(&a, &b);
    err = cudaMemcpyToSymbol(c_hashA, a, kHashRows * sizeof(uint64_t));
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_hashB, b, kHashRows * sizeof(uint64_t));
  });
  if (err != cudaSuccess) {
    set_cuda_error(err, "cudaMemcpyToSymbol(hash rows)");
    return PS_ERR_CUDA;
  }
  return PS_OK;
}

// Rows [lo, lo+bits) of the output hash.
__device__ __forceinline__ uint32_t dev_hash(uint64_t v, uint64_t w, int lo, int bits) {
  uint32_t f = 0;
  for (int j = 0; j < bits; ++j) {
    uint64_t t = (v & c_hashA[lo + j]) ^ (w & c_hashB[lo + j]);
    f |= (uint32_t)(__popcll(t) & 1) << j;
  }
  return f;
}

namespace {

constexpr int kCap = 2048;       // entries per merge pass
constexpr int kTable = 1024;     // shared-memory hash slots (power of two)
constexpr int kMergeThreads = 512;
constexpr int kMaxProbe = 128;
constexpr uint32_t kCodeSrc = 0xF000u;  // entry code of extra source s: kCodeSrc + s
constexpr uint32_t kCodePre = 0xFFFFu;  // entry code of the `pre` operand
constexpr int kMaxH = 0xEFFF;
constexpr int kHChunk = 2048;    // H terms per emission launch (shared memory)
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint16_t kNone16 = 0xFFFFu;
constexpr int kNoPow2 = 0x7FFF;
constexpr uint64_t kFullBudget = (uint64_t)48 << 30;  // bytes of full contribution records per merge
constexpr int kMaxGroupBins = 512;  // bins per group (a group also starts every kMaxGroupBins bins)
constexpr int kGroupQuota = 1536;   // a new group starts when the running entry count crosses a multiple
constexpr int kBatch = 2;           // entries per thread with loads in flight together
constexpr int kBatchFull = 4;       // the same for full records (one load round per pass of 2048)
static_assert(kCap <= 2048, "order key packs the entry index in 11 bits");

__device__ __forceinline__ ulonglong2 cas128_shared(ulonglong2* p, ulonglong2 expect, ulonglong2 desired) {
  ulonglong2 old;
  unsigned addr = (unsigned)__cvta_generic_to_shared(p);
  asm volatile(
      "{\n\t.reg .b128 d, b, c;\n\t"
      "mov.b128 b, {%2, %3};\n\t"
      "mov.b128 c, {%4, %5};\n\t"
      "atom.shared.cas.b128 d, [%6], b, c;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(old.x), "=l"(old.y)
      : "l"(expect.x), "l"(expect.y), "l"(desired.x), "l"(desired.y), "r"(addr)
      : "memory");
  return old;
}

// --------------------------------------------------------------------------- hashing
// With few bins (small sums: every block would hit the same global counters) the counts go
// to a shared-memory histogram first, flushed once per block.
constexpr int kHistSmemBits = 13;

__global__ void k_hash_hist(const Rec* __restrict__ r, int64_t n, int bits, uint32_t* __restrict__ f,
                            uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[1 << kHistSmemBits];
  const bool local = bits <= kHistSmemBits;
  const uint32_t nb = 1u << bits;
  if (local) {
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0;
    __syncthreads();
  }
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    uint32_t h = dev_hash(r[i].v, r[i].w, 0, bits);
    if (f) f[i] = h;
    atomicAdd(local ? &sh[h] : &hist[h], 1u);
  }
  if (local) {
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
      if (sh[b]) atomicAdd(&hist[b], sh[b]);
  }
}

// out[k * n + i] = T_k(G[i]) for k < ring: the translates of G as a list, not merged.
__global__ void k_ts_translates(const Rec* __restrict__ G, int64_t n, int ring, Rec* __restrict__ out) {
  const int64_t total = n * ring;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(j / n);
    const Rec g = G[j - (int64_t)k * n];
    out[j] = Rec{rotl_ring(g.v, k, ring), rotl_ring(g.w, k, ring), g.re, g.im};
  }
}

// Histogram of the bins of a translation-symmetric source: each string's representative
// (kTsCanon) or each of its ring translates (kTsExpand).
__global__ void k_hash_hist_ts(const Rec* __restrict__ r, int64_t n, int bits, int mode, int ring,
                               uint32_t* __restrict__ hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t v = r[i].v, w = r[i].w;
    if (mode == kTsCanon) {
      uint64_t cv, cw;
      int sh;
      ts_canonical(v, w, ring, cv, cw, sh);
      atomicAdd(&hist[dev_hash(cv, cw, 0, bits)], 1u);
    } else {
      for (int k = 0; k < ring; ++k) atomicAdd(&hist[dev_hash(rotl_ring(v, k, ring), rotl_ring(w, k, ring), 0, bits)], 1u);
    }
  }
}

// bound[p] = histY[p] + sum_h histX[p ^ F(h)]: the number of (h, x) pairs routed to bin p,
// plus the source entries of bin p.
__global__ void k_bound(const uint32_t* __restrict__ histX, const uint32_t* __restrict__ histY,
                        const uint32_t* __restrict__ fH, int nH, uint32_t nbins, uint64_t* __restrict__ bound) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x) {
    uint64_t b = histY ? histY[p] : 0;
    if (histX)
      for (int h = 0; h < nH; ++h) b += histX[p ^ __ldg(&fH[h])];
    bound[p] = b;
  }
}

// --------------------------------------------------------------------------- emission
constexpr int kEmitThreads = 256;
constexpr int kQueue = 64;  // per-warp queue of (lane, h) codes

// A finished contribution (single-component mode): output string, signed real value of its
// non-zero component, and order code (H index, kCodeSrc + source, or kCodePre).
struct __align__(16) Contrib {
  uint64_t v, w;
  double val;
  uint32_t code;
  uint32_t pad;
};

// Real factor of an H term in single-component mode and the exponent of |s| when s is a
// power of two (kNoPow2 otherwise).
struct __align__(16) HScal {
  double s;
  int e;
  int pvw;   // popcount(v & w) of the H term (its share of the product phase)
  float sf;  // s rounded to FP32 (the factor of the FP32 arithmetic)
  int per_inst;  // batched instances: 1 when the term's coefficient differs between instances
};

// Scalars of the single-component arithmetic (see build_scalar).
struct EmitScalars {
  int f32c;  // FP32 arithmetic: terms rounded once to FP32 (see prod32)
  int rot, uH, uX;
  double src_s[4];
  float src_sf[4];  // src_s rounded to FP32
  int src_e[4], src_q[4], src_uy[4];
  int pre_u;
};

// Per H term: its output-hash bits and (single-component mode, hscal non-null) its real factor
// with the exponent of |s| when s is a power of two (kNoPow2 otherwise).
__global__ void k_h_prep(const Rec* __restrict__ H, int nh, int bits, int uH, uint32_t* __restrict__ fH,
                         HScal* __restrict__ hscal, const double* __restrict__ huni) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nh) return;
  const Rec h = H[i];
  fH[i] = dev_hash(h.v, h.w, 0, bits);
  if (hscal) {
    // batched instances: a term whose coefficient is the same in every instance (huni[i],
    // NaN when it differs) takes that value here, so the emission treats it as a plain term
    double v = uH ? h.im : h.re;
    int per_inst = 0;
    if (huni) {
      const double u = huni[i];
      if (u != u) per_inst = 1;
      else v = u;
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    const bool p2 = (b & ((1ull << 52) - 1)) == 0 && E >= 1 && E <= 2046;
    hscal[i] = HScal{v, p2 ? E - 1023 : kNoPow2, __popcll(h.v & h.w), __double2float_rn(v), per_inst};
  }
}

// y * 2^e when y is normal and the result stays normal (exact); ok = false otherwise.
__device__ __forceinline__ double scale_pow2(double y, int e, bool& ok) {
  unsigned long long b = (unsigned long long)__double_as_longlong(y);
  int E = (int)((b >> 52) & 0x7FF);
  int E2 = E + e;
  ok = (E != 0 && E != 0x7FF && E2 >= 1 && E2 <= 2046);
  return ok ? __longlong_as_double((long long)(b + ((unsigned long long)(long long)e << 52))) : 0.0;
}

__device__ __forceinline__ double neg_if(double x, bool c) {  // sign flip on the integer pipe
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)c << 63));
}
__device__ __forceinline__ bool sign_bit(double x) { return __double_as_longlong(x) < 0; }

// round(s * y) for a real constant s with pow2 exponent e (kNoPow2: general), times 2^extra.
// For a power of two the product is an exponent shift on the integer pipe; otherwise one
// rounded FP64 product (then an exact doubling when extra == 1).
__device__ __forceinline__ double scaled(double s, int e, double y, int extra) {
  if (e != kNoPow2) {
    bool ok;
    double r = scale_pow2(y, e + extra, ok);
    if (ok) return neg_if(r, sign_bit(s));
  }
  double p = __dmul_rn(s, y);
  return extra ? twice(p) : p;
}

// FP32 arithmetic with compensated sums (output sums of precision PS_COEF_F32C): a term is
// the FP32 product RN32(RN32(s) RN32(y)), doubled exactly for a commutator product; a
// string's terms are added by Sum2 (Ogita, Rump, Oishi: TwoSum of the running sum, errors
// added in FP32, one final rounding) in the same order as the FP64 fold.
// FP32 numbers held in doubles and floats converted into each other on the integer pipe (the
// values are exact FP32 numbers, so no rounding is involved): on this GPU the FP64 unit, which
// would otherwise do the conversions, is the narrowest pipe.
__device__ __forceinline__ float f32_exact(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & ((1ull << 52) - 1);
  uint32_t f;
  if (e == 0) {
    f = sign;  // +-0 (an FP32 number is never an FP64 subnormal)
  } else if (e == 0x7FF) {
    f = sign | 0x7F800000u | (uint32_t)(m >> 29) | (m ? 0x400000u : 0u);  // inf, nan
  } else {
    const int e32 = e - 1023 + 127;
    f = e32 >= 1 ? sign | ((uint32_t)e32 << 23) | (uint32_t)(m >> 29)
                 : sign | (uint32_t)((m | (1ull << 52)) >> (30 - e32));  // FP32 subnormal
  }
  return __uint_as_float(f);
}

__device__ __forceinline__ double f64_of(float x) {
  const uint32_t f = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(f & 0x80000000u) << 32;
  const uint32_t e = (f >> 23) & 0xFFu, m = f & 0x7FFFFFu;
  unsigned long long b;
  if (e == 0xFFu) {
    b = sign | 0x7FF0000000000000ull | ((unsigned long long)m << 29);
  } else if (e != 0) {
    b = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0) {
    b = sign;
  } else {  // subnormal: m 2^-149 with its top bit at position p
    const int p = 31 - __clz(m);
    b = sign | ((unsigned long long)(p - 149 + 1023) << 52) | (((unsigned long long)m << (52 - p)) & ((1ull << 52) - 1));
  }
  return __longlong_as_double((long long)b);
}

// s: the FP32 scalar (H coefficient, alpha or post) already rounded; y: an FP32 number.
__device__ __forceinline__ double prod32(float s, double y, int extra) {
  float p = __fmul_rn(s, f32_exact(y));
  if (extra) p = __fmul_rn(2.0f, p);
  return f64_of(p);
}

__device__ __forceinline__ void two_sum32(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ double add_rn32(double a, double b) {  // FP32 sum, zero terms skipped
  if (is_zero(b)) return a;
  if (is_zero(a)) return b;
  return f64_of(__fadd_rn(f32_exact(a), f32_exact(b)));
}

// Bin cursors: cur[p] starts at the bin's first slot (base[p]) and one 64-bit atomic add
// reserves slots and returns their absolute position.  A warp reserves once per distinct bin
// among its 32 entries (the entries of one h over neighbouring x often share bins).
__device__ __forceinline__ uint64_t reserve_slot(unsigned long long* __restrict__ cur, uint32_t p, bool act, int lane) {
  const unsigned mm = __match_any_sync(0xffffffffu, act ? p : 0xFFFFFFFFu);
  const int leader = __ffs(mm) - 1;
  unsigned long long b = 0;
  if (act && lane == leader) b = atomicAdd(&cur[p], (unsigned long long)__popc(mm));
  b = __shfl_sync(0xffffffffu, b, leader);
  return b + (uint32_t)__popc(mm & ((1u << lane) - 1u));
}

// Reservation for a warp whose active lanes are a prefix and whose equal bins tend to sit in
// adjacent lanes: one atomic per run of equal bins (a bin split over several runs takes one
// per run), no match over the warp.
__device__ __forceinline__ uint64_t reserve_run(unsigned long long* __restrict__ cur, uint32_t p, bool act, int lane) {
  const uint32_t pp = __shfl_up_sync(0xffffffffu, p, 1);
  const unsigned active = __ballot_sync(0xffffffffu, act);
  const unsigned starts = __ballot_sync(0xffffffffu, act && (lane == 0 || pp != p));
  const unsigned le = 0xffffffffu >> (31 - lane);  // lanes 0..lane
  const int leader = 31 - __clz(starts & le);
  const unsigned above = starts & ~le;
  const int next = above ? __ffs(above) - 1 : __popc(active);
  unsigned long long b = 0;
  if (act && lane == leader) b = atomicAdd(&cur[p], (unsigned long long)(next - lane));
  b = __shfl_sync(0xffffffffu, b, leader & 31);
  return b + (uint64_t)(lane - leader);
}

// Emission of the products for |H| > 256 and of operator products (ALL: every pair, not only
// the anticommuting ones) as 8-byte entries, H in chunks [h0, h0 + nh).  A warp
// holds 32 x in registers and walks the H terms; the anticommuting (h, lane) pairs are
// queued as 32-bit codes and, 32 at a time, turned into entries (x index << 16 | H index)
// with every lane active: the lane fetches its x's hash by shuffle and reserves a slot in
// bin F(h) ^ F(x).  The queue is emptied before the warp moves on to its next 32 x.
template <bool ALL>
__global__ void __launch_bounds__(kEmitThreads) k_emit_products(const Rec* __restrict__ X, const uint32_t* __restrict__ fX,
                                                       int64_t nX, const Rec* __restrict__ H,
                                                       const uint32_t* __restrict__ fH, int h0, int nh,
                                                       unsigned long long* __restrict__ cur,
                                                       uint64_t* __restrict__ entries,
                                                       unsigned long long* __restrict__ total) {
  extern __shared__ __align__(16) unsigned char smem[];
  ulonglong2* s_hk = reinterpret_cast<ulonglong2*>(smem);
  uint32_t* s_hf = reinterpret_cast<uint32_t*>(smem + sizeof(ulonglong2) * nh);
  __shared__ uint32_t s_q[kEmitThreads / 32][kQueue];
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    s_hk[i] = make_ulonglong2(H[h0 + i].v, H[h0 + i].w);
    s_hf[i] = fH[h0 + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* q = s_q[warp];
  uint32_t emitted = 0;  // warp-uniform
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t0 = wid * 32; t0 < nX; t0 += nwarps * 32) {
    const int64_t i = t0 + lane;
    const bool valid = i < nX;
    ulonglong2 xk = make_ulonglong2(0, 0);
    uint32_t fx = 0;
    if (valid) {
      xk = *reinterpret_cast<const ulonglong2*>(&X[i]);
      fx = fX[i];
    }
    // entries for queue codes q[0, n): lane l takes q[l]; all lanes take part in the shuffles
    auto flush = [&](int n) {
      const bool act = lane < n;
      const uint32_t c = act ? q[lane] : 0u;
      const int src = (int)(c >> 16);
      const uint32_t h = c & 0xFFFFu;
      const uint32_t p = __shfl_sync(0xffffffffu, fx, src) ^ s_hf[h];
      const uint64_t at = reserve_slot(cur, p, act, lane);
      if (act) entries[at] = ((uint64_t)(t0 + src) << 16) | (uint64_t)(h0 + h);
      emitted += n;
    };
    int qn = 0;  // queued codes of this warp (warp-uniform)
    for (int h = 0; h < nh; ++h) {
      const ulonglong2 hk = s_hk[h];
      const bool anti = valid && (ALL || anticommute(hk.x, hk.y, xk.x, xk.y));
      const unsigned m = __ballot_sync(0xffffffffu, anti);
      if (!m) continue;
      if (anti) q[qn + __popc(m & ((1u << lane) - 1))] = ((uint32_t)lane << 16) | (uint32_t)h;
      qn += __popc(m);
      if (qn >= 32) {  // take the first 32, move the rest (fewer than 32) to the front
        __syncwarp();
        flush(32);
        const int rest = qn - 32;
        const uint32_t rc = lane < rest ? q[32 + lane] : 0u;
        __syncwarp();
        if (lane < rest) q[lane] = rc;
        __syncwarp();
        qn = rest;
      }
    }
    __syncwarp();
    if (qn > 0) flush(qn);
    __syncwarp();
  }
  __shared__ unsigned long long s_tot;
  if (threadIdx.x == 0) s_tot = 0;
  __syncthreads();
  if (lane == 0 && emitted) atomicAdd(&s_tot, (unsigned long long)emitted);
  __syncthreads();
  if (threadIdx.x == 0 && s_tot) atomicAdd(total, s_tot);
}

// ---- table-driven emission (|H| <= 256)
// Whether h and x anticommute is the parity of popcount((h.w & x.v) ^ (h.v & x.w)), a
// GF(2)-linear function of the 128 bits of x.  So the bitmap A(x) (bit h set iff h and x
// anticommute) is the XOR, over the 32 nibbles of x, of a table row indexed by (nibble
// position, nibble value): A(x) = XOR_p T[p][nibble_p(x)].  Positions 0..15 are the nibbles
// of x.v (paired with h.w), 16..31 those of x.w (paired with h.v).  A row holds NW 32-bit
// words and is padded to a stride of kTabStride(NW) words (2 mod 4), so that 16 lanes
// reading 64-bit words of 16 different rows of one position hit 16 distinct bank pairs.
constexpr int kTabPos = 32, kTabVals = 16;

__host__ __device__ constexpr int tab_stride(int nw) { return nw <= 2 ? 2 : (nw <= 6 ? 6 : 10); }

// T[p][val][k]: bit b of word k is the parity of popcount(val & nibble_p(h = 32k + b)).
// The anticommutation table T[p][val][k] (one thread per word) and the preparation of the H
// terms as in k_h_prep, in one launch: threads [0, table words) build the table, the next nh
// threads prepare the terms.
__global__ void k_h_prep_table(const Rec* __restrict__ H, int nh, int bits, int uH, uint32_t* __restrict__ fH,
                               HScal* __restrict__ hscal, const double* __restrict__ huni, int stride,
                               uint32_t* __restrict__ T) {
  const int words = kTabPos * kTabVals * stride;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < words) {
    const int t = u / stride, k = u % stride;
    const int p = t / kTabVals, val = t % kTabVals;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
      const int h = 32 * k + b;
      if (h >= nh) break;
      const uint64_t m = p < 16 ? H[h].w : H[h].v;
      const uint32_t nib = (uint32_t)(m >> (4 * (p & 15))) & 15u;
      word |= (uint32_t)(__popc(nib & (uint32_t)val) & 1) << b;
    }
    T[u] = word;
    return;
  }
  const int i = u - words;
  if (i >= nh) return;
  const Rec h = H[i];
  fH[i] = dev_hash(h.v, h.w, 0, bits);
  if (hscal) {
    double v = uH ? h.im : h.re;
    int per_inst = 0;
    if (huni) {
      const double w = huni[i];
      if (w != w) per_inst = 1;
      else v = w;
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FF);
    const bool p2 = (b & ((1ull << 52) - 1)) == 0 && E >= 1 && E <= 2046;
    hscal[i] = HScal{v, p2 ? E - 1023 : kNoPow2, __popcll(h.v & h.w), __double2float_rn(v), per_inst};
  }
}

// Block-level table emission.  A block takes 256 neighbouring x (hash order), one per
// thread, and forms their anticommutation bitmaps from the nibble table.  Then, for each
// 32-term word of the bitmaps: one ballot per term and warp gives, per (warp, term), the lanes
// that anticommute with it; a scan over the 32 terms and the 8 warps gives every (term, x) pair
// its position in a block-local list ordered by term, then by x; the threads then build the
// list's entries independently (consecutive threads: one term over neighbouring x, so a
// warp's entries fall in few bins and reserve them with one atomic per distinct bin) and write
// them.  No per-term serial chain: every step is a block-parallel pass.
constexpr int kBlkX = kEmitThreads;              // x per block chunk
constexpr int kBlkCodes = kBlkX * 32;            // (x, term) pairs of one bitmap word at most

template <bool FULL, int NW>
__global__ void __launch_bounds__(kEmitThreads, 4) k_emit_blk(const Rec* __restrict__ X, const uint32_t* __restrict__ fX,
                                                  int64_t nX, const Rec* __restrict__ H,
                                                  const uint32_t* __restrict__ fH,
                                                  const HScal* __restrict__ hscal, int nh,
                                                  const uint32_t* __restrict__ T, EmitScalars es,
                                                  unsigned long long* __restrict__ cur,
                                                  uint64_t* __restrict__ entries, Contrib* __restrict__ fout,
                                                  unsigned long long* __restrict__ total,
                                                  const double* __restrict__ hb, int hb_shift) {
  constexpr int S = tab_stride(NW);
  constexpr int kTabWords = kTabPos * kTabVals * S;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  ulonglong2* s_hk = reinterpret_cast<ulonglong2*>(s_tab + kTabWords);
  HScal* s_hs = reinterpret_cast<HScal*>(s_hk + nh);                     // FULL only
  uint32_t* s_hf = reinterpret_cast<uint32_t*>(s_hs + (FULL ? nh : 0));
  __shared__ ulonglong2 s_xk[kBlkX];
  __shared__ double s_xs[FULL ? kBlkX : 1];
  __shared__ uint32_t s_xf[kBlkX];
  __shared__ int s_xp[FULL ? kBlkX : 1];  // popcount(v & w) of x
  __shared__ uint32_t s_bal[kEmitThreads / 32][32];   // lanes of warp w anticommuting with term b
  __shared__ uint32_t s_off[kEmitThreads / 32][32];   // list position of (warp w, term b)'s first pair
  __shared__ uint16_t s_code[kBlkCodes];              // (x << 5 | b) in term-then-x order
  __shared__ uint32_t s_n;
  for (int i = threadIdx.x; i < kTabWords; i += blockDim.x) s_tab[i] = T[i];
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    s_hk[i] = make_ulonglong2(H[i].v, H[i].w);
    if constexpr (FULL) s_hs[i] = hscal[i];
    s_hf[i] = fH[i];
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long emitted = 0;  // thread 0's count
  const int64_t chunks = ceil_div_dev(nX, kBlkX);
  for (int64_t chunk = blockIdx.x; chunk < chunks; chunk += gridDim.x) {
    __syncthreads();  // the previous chunk's x cache and lists are done
    const int64_t i = chunk * kBlkX + tid;
    const bool valid = i < nX;
    ulonglong2 xk = make_ulonglong2(0, 0);
    if (valid) {
      xk = *reinterpret_cast<const ulonglong2*>(&X[i]);
      if constexpr (FULL) {
        s_xs[tid] = es.uX ? X[i].im : X[i].re;
        s_xp[tid] = __popcll(xk.x & xk.y) - es.rot - es.uH - es.uX;  // constant part of the phase
      }
      s_xf[tid] = fX[i];
    }
    s_xk[tid] = xk;
    uint32_t A[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) A[k] = 0u;
    if (valid) {
#pragma unroll
      for (int p = 0; p < kTabPos; ++p) {
        const uint64_t m = p < 16 ? xk.x : xk.y;
        const uint32_t nib = (uint32_t)(m >> (4 * (p & 15))) & 15u;
        const uint32_t* row = s_tab + (p * kTabVals + nib) * S;
#pragma unroll
        for (int k = 0; k < NW; k += 2) {
          const uint2 t = *reinterpret_cast<const uint2*>(row + k);
          A[k] ^= t.x;
          A[k + 1] ^= t.y;
        }
      }
    }
#pragma unroll 1
    for (int k = 0; k < NW; ++k) {
      if (32 * k >= nh) break;  // block-uniform
      uint32_t a = 0;
#pragma unroll
      for (int q = 0; q < NW; ++q)
        if (q == k) a = A[q];
      // ballots: lane b keeps the mask of term 32k + b
      uint32_t mine = 0;
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        const uint32_t m = __ballot_sync(0xffffffffu, (a >> b) & 1u);
        if (lane == b) mine = m;
      }
      s_bal[warp][lane] = mine;
      __syncthreads();
      if (warp == 0) {  // per term b (lane): offsets over the warps, then a scan over the terms
        uint32_t run = 0, c[kEmitThreads / 32];
#pragma unroll
        for (int w = 0; w < kEmitThreads / 32; ++w) {
          c[w] = run;
          run += __popc(s_bal[w][lane]);
        }
        uint32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        const uint32_t base = incl - run;
#pragma unroll
        for (int w = 0; w < kEmitThreads / 32; ++w) s_off[w][lane] = base + c[w];
        if (lane == 31) s_n = incl;
      }
      __syncthreads();
      // every set bit of this thread's word: its pair's list position
      const uint32_t lt = (1u << lane) - 1u;
      for (uint32_t bits = a; bits; bits &= bits - 1u) {
        const int b = __ffs(bits) - 1;
        const uint32_t pos = s_off[warp][b] + __popc(s_bal[warp][b] & lt);
        s_code[pos] = (uint16_t)((tid << 5) | b);
      }
      __syncthreads();
      const uint32_t n = s_n;
      if (tid == 0) emitted += n;
      for (uint32_t e0 = 0; e0 < n; e0 += kEmitThreads) {
        const uint32_t e = e0 + tid;
        const bool act = e < n;
        uint32_t xl = 0, h = 0;
        if (act) {
          const uint32_t c = s_code[e];
          xl = c >> 5;
          h = 32u * (uint32_t)k + (c & 31u);
        }
        Contrib r;
        uint32_t p = 0;
        if (act) {
          const ulonglong2 x = s_xk[xl];
          p = s_xf[xl] ^ s_hf[h];
          if constexpr (FULL) {
            const ulonglong2 hk = s_hk[h];
            const HScal hs = s_hs[h];
            r.v = hk.x ^ x.x;
            r.w = hk.y ^ x.y;
            // product phase k = pop(vc & wc) - pop(vh & wh) - pop(vx & wx) + 2 pop(wh & vx)
            const int ph = (__popcll(r.v & r.w) - hs.pvw - s_xp[xl] + 2 * __popcll(hk.y & x.x)) & 3;
            double hsv = hs.s;
            int hse = hs.e;
            const bool inst = hb && hs.per_inst;
            if (inst) {  // batched instances: the H coefficient of x's instance (tag = v >> hb_shift)
              hsv = hb[(size_t)(x.x >> hb_shift) * (size_t)nh + h];
              hse = kNoPow2;
            }
            r.val = neg_if(es.f32c ? prod32(inst ? __double2float_rn(hsv) : hs.sf, s_xs[xl], 1) : scaled(hsv, hse, s_xs[xl], 1),
                           (ph & 2) != 0);
            r.code = h;
            r.pad = 0;
          }
        }
        const uint64_t at = reserve_run(cur, p, act, lane);
        if (act) {
          if constexpr (FULL) fout[at] = r;
          else entries[at] = ((uint64_t)(chunk * kBlkX + xl) << 16) | (uint64_t)h;
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0 && emitted) atomicAdd(total, emitted);
}

template <bool FULL, int NW>
int launch_emit_tab(const Rec* X, const uint32_t* fX, int64_t nX, const Rec* H, const uint32_t* fH,
                    const HScal* hscal, int nh, const uint32_t* T, const EmitScalars& es,
                    unsigned long long* cur, uint64_t* entries, Contrib* fout, unsigned long long* total, int nsm,
                    cudaStream_t s, const double* hb, int hb_shift) {
  const size_t sm = (size_t)kTabPos * kTabVals * tab_stride(NW) * sizeof(uint32_t) +
                    (size_t)nh * (sizeof(ulonglong2) + (FULL ? sizeof(HScal) : 0) + sizeof(uint32_t));
  PS_CUDA(cudaFuncSetAttribute(k_emit_blk<FULL, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_emit_blk<FULL, NW>, kEmitThreads, sm));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, per_sm) * nsm, ceil_div(nX, kBlkX)));
  PS_LAUNCH("k_emit_products", s, k_emit_blk<FULL, NW><<<grid, kEmitThreads, sm, s>>>(X, fX, nX, H, fH, hscal, nh, T, es, cur, entries, fout, total, hb, hb_shift));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

template <bool FULL>
int emit_tab(const Rec* X, const uint32_t* fX, int64_t nX, const Rec* H, const uint32_t* fH, const HScal* hscal,
             int nh, const uint32_t* T, const EmitScalars& es, unsigned long long* cur,
             uint64_t* entries, Contrib* fout, unsigned long long* total, int nsm, cudaStream_t s,
             const double* hb = nullptr, int hb_shift = 0) {
  const int nw = (nh + 31) / 32;
  if (nw <= 2) return launch_emit_tab<FULL, 2>(X, fX, nX, H, fH, hscal, nh, T, es, cur, entries, fout, total, nsm, s, hb, hb_shift);
  if (nw <= 4) return launch_emit_tab<FULL, 4>(X, fX, nX, H, fH, hscal, nh, T, es, cur, entries, fout, total, nsm, s, hb, hb_shift);
  if (nw <= 6) return launch_emit_tab<FULL, 6>(X, fX, nX, H, fH, hscal, nh, T, es, cur, entries, fout, total, nsm, s, hb, hb_shift);
  return launch_emit_tab<FULL, 8>(X, fX, nX, H, fH, hscal, nh, T, es, cur, entries, fout, total, nsm, s, hb, hb_shift);
}

// Emission of an extra source (code kCodeSrc + i) or of the pre operand (kCodePre): FULL, the
// contribution record; otherwise the 8-byte reference (index << 16 | code).  Warp-strided so
// that all 32 lanes take part in every slot reservation.
// Emission of an extra source (code kCodeSrc + i) or of the pre operand (kCodePre): FULL, the
// contribution record; otherwise the 8-byte reference (index << 16 | code).  Warp-strided so
// that all 32 lanes take part in every slot reservation.  A translation-symmetric source
// (ts, full records only) emits each string at its orbit representative with the shift as
// order code (kTsCanon), or at each of its ring translates with code k (kTsExpand).
template <bool FULL>
__global__ void k_emit_source(const Rec* __restrict__ Y, int64_t n, int bits, uint32_t code, EmitScalars es,
                              unsigned long long* __restrict__ cur, uint64_t* __restrict__ entries,
                              Contrib* __restrict__ out, int ts, int ring) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    const bool act = i < n;
    Rec y = Rec{0, 0, 0.0, 0.0};
    if (act) y = Y[i];
    if constexpr (FULL) {
      double val;
      if (code == kCodePre) {
        val = es.pre_u ? y.im : y.re;
      } else {
        const uint32_t si = code - kCodeSrc;
        const double sy = es.src_uy[si] ? y.im : y.re;
        val = neg_if(es.f32c ? prod32(es.src_sf[si], sy, 0) : scaled(es.src_s[si], es.src_e[si], sy, 0),
                     (es.src_q[si] & 2) != 0);
      }
      if (ts == kTsExpand) {
        for (int k = 0; k < ring; ++k) {
          const uint64_t tv = rotl_ring(y.v, k, ring), tw = rotl_ring(y.w, k, ring);
          const uint64_t at = reserve_slot(cur, dev_hash(tv, tw, 0, bits), act, lane);
          if (act) out[at] = Contrib{tv, tw, val, (uint32_t)k, 0};
        }
        continue;
      }
      Contrib c{y.v, y.w, val, code, 0};
      if (ts == kTsCanon) {
        int sh = 0;
        ts_canonical(y.v, y.w, ring, c.v, c.w, sh);
        c.code = (uint32_t)sh;
      }
      const uint64_t at = reserve_slot(cur, dev_hash(c.v, c.w, 0, bits), act, lane);
      if (act) out[at] = c;
    } else {
      const uint64_t at = reserve_slot(cur, dev_hash(y.v, y.w, 0, bits), act, lane);
      if (act) entries[at] = ((uint64_t)i << 16) | code;
    }
  }
}

// All plain (not translation-symmetric) sources and the pre operand of a merge in one launch:
// the concatenation of up to five operands, each with its order code.
struct SrcSet {
  const Rec* rec[5];
  int64_t off[6];  // operand j covers [off[j], off[j + 1]) of the concatenation
  uint32_t code[5];
  int cnt;
};

__device__ __forceinline__ int src_of_index(const SrcSet& ss, int64_t i) {
  int j = 0;
  while (j + 1 < ss.cnt && i >= ss.off[j + 1]) ++j;
  return j;
}

// The histogram of the operands' bins (as k_hash_hist without the per-string hashes).
__global__ void k_hash_hist_set(SrcSet ss, int bits, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[1 << kHistSmemBits];
  const bool local = bits <= kHistSmemBits;
  const uint32_t nb = 1u << bits;
  if (local) {
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) sh[b] = 0;
    __syncthreads();
  }
  const int64_t n = ss.off[ss.cnt];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = src_of_index(ss, i);
    const Rec& r = ss.rec[j][i - ss.off[j]];
    atomicAdd(local ? &sh[dev_hash(r.v, r.w, 0, bits)] : &hist[dev_hash(r.v, r.w, 0, bits)], 1u);
  }
  if (local) {
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
      if (sh[b]) atomicAdd(&hist[b], sh[b]);
  }
}

// The emission of k_emit_source for every operand of the set (warp-strided over the
// concatenation; a warp may straddle two operands).
template <bool FULL>
__global__ void k_emit_source_set(SrcSet ss, int bits, EmitScalars es, unsigned long long* __restrict__ cur,
                                  uint64_t* __restrict__ entries, Contrib* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t n = ss.off[ss.cnt];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    const bool act = i < n;
    Rec y = Rec{0, 0, 0.0, 0.0};
    uint32_t code = 0;
    int64_t idx = 0;
    if (act) {
      const int j = src_of_index(ss, i);
      idx = i - ss.off[j];
      y = ss.rec[j][idx];
      code = ss.code[j];
    }
    if constexpr (FULL) {
      double val = 0.0;
      if (act) {
        if (code == kCodePre) {
          val = es.pre_u ? y.im : y.re;
        } else {
          const uint32_t si = code - kCodeSrc;
          const double sy = es.src_uy[si] ? y.im : y.re;
          val = neg_if(es.f32c ? prod32(es.src_sf[si], sy, 0) : scaled(es.src_s[si], es.src_e[si], sy, 0),
                       (es.src_q[si] & 2) != 0);
        }
      }
      const uint64_t at = reserve_slot(cur, dev_hash(y.v, y.w, 0, bits), act, lane);
      if (act) out[at] = Contrib{y.v, y.w, val, code, 0};
    } else {
      const uint64_t at = reserve_slot(cur, dev_hash(y.v, y.w, 0, bits), act, lane);
      if (act) entries[at] = ((uint64_t)idx << 16) | code;
    }
  }
}

// Slots used per bin: cnt[p] = cur[p] - base[p].
__global__ void k_bin_counts(const unsigned long long* __restrict__ cur, const uint64_t* __restrict__ base,
                             uint32_t nbins, uint32_t* __restrict__ cnt) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x)
    cnt[p] = (uint32_t)(cur[p] - base[p]);
}

// --------------------------------------------------------------------------- grouping
// Bin p opens a group when the running entry count crosses a multiple of `quota`, and at
// the middle bin (so that no group spans both halves of the bin range).
__global__ void k_group_flags(const uint64_t* __restrict__ cpre, uint32_t nbins, uint64_t quota,
                              uint32_t* __restrict__ flag) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x) {
    bool start = (p == 0) || (p == nbins / 2) || (p % kMaxGroupBins == 0) || (cpre[p] / quota != cpre[p - 1] / quota);
    flag[p] = start ? 1u : 0u;
  }
}

__global__ void k_group_scatter(const uint32_t* __restrict__ flag, const uint64_t* __restrict__ fpre, uint32_t nbins,
                                uint32_t* __restrict__ gstart, uint32_t* __restrict__ ngroups) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x)
    if (flag[p]) gstart[fpre[p]] = p;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t g = (uint32_t)fpre[nbins];
    *ngroups = g;
    gstart[g] = nbins;
  }
}

// Per group: its bin range and entry range, so that a block reads one record per group.
struct __align__(16) GroupHead {
  uint32_t lo, hi;  // bins [lo, hi)
  uint64_t e0;      // entries before the group (prefix of the bin fill counts)
  uint64_t E;       // entries in the group
  uint64_t pad;
};

__global__ void k_group_heads(const uint32_t* __restrict__ gstart, const uint64_t* __restrict__ cpre,
                              const uint32_t* __restrict__ ngroups, GroupHead* __restrict__ heads) {
  const uint32_t n = *ngroups;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
    const uint32_t lo = gstart[g], hi = gstart[g + 1];
    const uint64_t e0 = cpre[lo];
    heads[g] = GroupHead{lo, hi, e0, cpre[hi] - e0, 0};
  }
}

// ---- small merges: the bin bounds and the group plan each in one block of 1024 threads (each
// thread owns up to 16 consecutive bins), in place of the device-wide kernels and scans that
// cost a launch each; the same definitions, so the same groups.
constexpr int kPlanThreads = 1024;
constexpr uint32_t kSmallPlanBins = 16u * kPlanThreads;

// Exclusive scan of one value per thread over the block of kPlanThreads; *total gets the sum.
__device__ __forceinline__ uint64_t plan_scan(uint64_t v, uint64_t* s_w, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t t = s_w[lane];  // kPlanThreads / 32 = 32 warps
    uint64_t ti = t;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t u = __shfl_up_sync(0xffffffffu, ti, d);
      if (lane >= d) ti += u;
    }
    s_w[lane] = ti - t;
    if (lane == 31) s_w[32] = ti;
  }
  __syncthreads();
  const uint64_t r = s_w[warp] + incl - v;
  *total = s_w[32];
  __syncthreads();
  return r;
}

// bound[p] as k_bound, its exclusive prefix base[0..nbins] and the cursors cur = base.
__global__ void __launch_bounds__(kPlanThreads) k_bound_small(const uint32_t* __restrict__ histX,
                                                              const uint32_t* __restrict__ histY,
                                                              const uint32_t* __restrict__ fH, int nH, uint32_t nbins,
                                                              uint64_t* __restrict__ base,
                                                              unsigned long long* __restrict__ cur) {
  __shared__ uint64_t s_w[33];
  const uint32_t per = (nbins + kPlanThreads - 1) / kPlanThreads;
  const uint32_t p0 = threadIdx.x * per;
  uint64_t b[16];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t p = p0 + (uint32_t)k;
    b[k] = 0;
    if ((uint32_t)k < per && p < nbins) {
      uint64_t x = histY ? histY[p] : 0;
      if (histX)
        for (int h = 0; h < nH; ++h) x += histX[p ^ __ldg(&fH[h])];
      b[k] = x;
    }
    sum += b[k];
  }
  uint64_t total;
  uint64_t run = plan_scan(sum, s_w, &total);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t p = p0 + (uint32_t)k;
    if ((uint32_t)k < per && p < nbins) {
      base[p] = run;
      cur[p] = run;
      run += b[k];
    }
  }
  if (threadIdx.x == 0) base[nbins] = total;
}

// The group plan from the filled bins: cpre (as k_bin_counts + the scan), the group starts
// (as k_group_flags + the scan + k_group_scatter) and the group heads (as k_group_heads).
__global__ void __launch_bounds__(kPlanThreads) k_plan_small(const unsigned long long* __restrict__ cur,
                                                             const uint64_t* __restrict__ base, uint32_t nbins,
                                                             uint64_t quota, uint64_t* __restrict__ cpre,
                                                             uint32_t* __restrict__ gstart,
                                                             uint32_t* __restrict__ ngroups,
                                                             GroupHead* __restrict__ heads) {
  __shared__ uint64_t s_w[33];
  const uint32_t per = (nbins + kPlanThreads - 1) / kPlanThreads;
  const uint32_t p0 = threadIdx.x * per;
  uint64_t c[16];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t p = p0 + (uint32_t)k;
    c[k] = ((uint32_t)k < per && p < nbins) ? (uint64_t)(cur[p] - base[p]) : 0;
    sum += c[k];
  }
  uint64_t total;
  uint64_t run = plan_scan(sum, s_w, &total);
  uint64_t pre[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    pre[k] = run;
    const uint32_t p = p0 + (uint32_t)k;
    if ((uint32_t)k < per && p < nbins) cpre[p] = run;
    run += c[k];
  }
  if (threadIdx.x == 0) cpre[nbins] = total;
  // the predecessor of a thread's first bin belongs to the thread before: its prefix is read
  // back from cpre after the barrier
  __syncthreads();
  uint32_t nf = 0;
  bool f[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t p = p0 + (uint32_t)k;
    f[k] = false;
    if ((uint32_t)k < per && p < nbins) {
      const uint64_t prev = p == 0 ? 0 : (k > 0 ? pre[k - 1] : cpre[p - 1]);
      f[k] = (p == 0) || (p == nbins / 2) || (p % kMaxGroupBins == 0) || (pre[k] / quota != prev / quota);
      nf += f[k] ? 1u : 0u;
    }
  }
  uint64_t ng;
  uint64_t g = plan_scan(nf, s_w, &ng);
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (f[k]) gstart[g++] = p0 + (uint32_t)k;
  if (threadIdx.x == 0) {
    gstart[ng] = nbins;
    *ngroups = (uint32_t)ng;
  }
  __syncthreads();
  for (uint32_t q = threadIdx.x; q < (uint32_t)ng; q += kPlanThreads) {
    const uint32_t lo = gstart[q], hi = gstart[q + 1];
    const uint64_t e0 = cpre[lo];
    heads[q] = GroupHead{lo, hi, e0, cpre[hi] - e0, 0};
  }
}

// --------------------------------------------------------------------------- merge
struct MergeArgs {
  const Rec* H;
  int nH;
  const Rec* X;
  int rot;
  int twice;  // 1: commutator contributions 2 i^(k + rot) h x; 0: operator product i^k h x
  const Rec* src[4];
  Cx alpha[4];
  const Rec* pre;
  int has_post;
  Cx post;
  int bits;
  uint32_t nbins;
  const uint64_t* base;   // bin region starts
  const uint64_t* cpre;   // exclusive prefix of cnt
  const uint64_t* entries;
  const Contrib* fent;    // full-record entries (single-component mode), or null
  const uint32_t* gstart;
  const GroupHead* heads;
  const uint32_t* ngroups;
  unsigned* next_group;
  Rec* out;
  unsigned long long* out_n;
  unsigned long long out_cap;
  int* err;               // bit 0: capacity, bit 1: unresolved table overflow
  int round32;            // FP32 output sum: every result rounded once to FP32 before the zero test
  int f32c;               // FP32 arithmetic with compensated sums (single-component ranked merges)
  float src_sf[4];        // src_s and post_s rounded to FP32
  float post_sf;
  unsigned* split_groups;
  ulonglong2 sent_lo, sent_hi;  // empty-slot keys for groups in the lower / upper half
  // structured (single-component) mode: every coefficient is s * i^u with s real
  const HScal* hscal;     // per H term: real factor and its pow2 exponent
  int uH, uX;             // u of the H and X coefficients (0 real, 1 imaginary)
  double src_s[4];        // alpha_s = src_s * i^(src_u)
  int src_e[4];           // pow2 exponent of |src_s| or kNoPow2
  int src_q[4];           // u(alpha_s) + u(Y_s)
  int src_uy[4];          // u(Y_s): the component of Y_s that holds its values
  int pre_u;              // u of the pre operand
  double post_s;          // post = post_s * i^(post_q - u(acc))
  int post_q;             // u(post) + u(acc)
  int out_imag;           // the output's non-zero component: 0 real, 1 imaginary
  uint64_t* okeys;        // optional (single-component mode): per output, the bit pattern of |x|
  int* otop;              // with okeys: max prod_top(x, x) over the outputs (exact norm's bound)
};

// Shared memory of one merge block.  S: single-component mode (no imaginary array).
template <bool S>
struct MergeSmem {
  // hash table over the group's output strings
  ulonglong2 key[kTable];
  uint32_t head[kTable];     // first entry of the slot's contribution list, or kNone
  uint16_t pre[kTable];      // entry holding the pre operand of the slot, or kNone16
  uint16_t ulist[kTable];    // occupied slots (one per distinct output string)
  // the entries of the current pass
  double ere[kCap];
  double eim[S ? 1 : kCap];
  uint16_t eord[kCap];       // order code: H index, or kCodeSrc + s
  uint16_t enext[kCap];      // next entry of the same slot, or kNone16
  // results of the current pass, staged for one contiguous output reservation
  double ore[kTable];
  double oim[S ? 1 : kTable];
  uint16_t oslot[kTable];
  // the group's bins
  unsigned long long gbase[kMaxGroupBins];
  uint32_t gpre[kMaxGroupBins + 1];
  uint16_t longq[kTable];    // slots whose chains are longer than 4
  uint32_t n_e, n_u, n_out, n_long;
  int flags;
  unsigned group;
  unsigned long long out_base;
  ulonglong2 cur_sent;
};

// Insert key c (or find it) in a shared-memory table of kTable slots (any layout with a
// `key` array).  fresh = this thread claimed the empty slot.
template <int TAB = kTable, class SM>
__device__ __forceinline__ int table_insert(SM& s, ulonglong2 c, ulonglong2 sent, bool& fresh) {
  fresh = false;
  // double hashing: an odd step from the hash's high bits (every slot is reachable), so
  // that neighbouring home slots do not build the long clusters of linear probing
  const uint64_t h = key_hash64(c.x, c.y);
  uint32_t slot = (uint32_t)h & (TAB - 1);
  const uint32_t step = (uint32_t)(h >> 32) | 1u;
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    ulonglong2 k = s.key[slot];
    if (k.x == c.x && k.y == c.y) return (int)slot;
    if (k.x == sent.x && k.y == sent.y) {
      ulonglong2 old = cas128_shared(&s.key[slot], sent, c);
      if (old.x == sent.x && old.y == sent.y) {
        fresh = true;
        return (int)slot;
      }
      if (old.x == c.x && old.y == c.y) return (int)slot;
    }
    slot = (slot + step) & (TAB - 1);
  }
  return -1;
}

// Key and contribution of an entry whose operand record y has been loaded: for a product
// (code = H index) the string h^y with 2 i^(k+rot) (h y); for a source, alpha_s y; for
// the pre operand, y itself.
__device__ __forceinline__ void build_contribution(const MergeArgs& a, uint32_t code, const Rec& y, ulonglong2& key,
                                                   Cx& t) {
  if (code < kCodeSrc) {
    const Rec h = a.H[code];
    key = make_ulonglong2(h.v ^ y.v, h.w ^ y.w);
    int k = product_phase(h.v, h.w, y.v, y.w) + a.rot;
    Cx p = cmul(Cx{h.re, h.im}, Cx{y.re, y.im});
    t = a.twice ? rot(Cx{twice(p.re), twice(p.im)}, k) : rot(p, k);
  } else if (code == kCodePre) {
    key = make_ulonglong2(y.v, y.w);
    t = Cx{y.re, y.im};
  } else {
    key = make_ulonglong2(y.v, y.w);
    t = cmul(a.alpha[code - kCodeSrc], Cx{y.re, y.im});
  }
}

// Structured mode: the signed real value of the entry's single non-zero component.
// Product: 2 i^(k+rot) (h y) with h = s_h i^uH, y = s_y i^uX gives 2 round(s_h s_y) i^q,
// q = k + rot + uH + uX; the value is the real factor times i^(q mod 2), the sign from q & 2.
__device__ __forceinline__ void build_scalar(const MergeArgs& a, uint32_t code, const Rec& y, ulonglong2& key,
                                             double& t) {
  if (code < kCodeSrc) {
    const Rec h = a.H[code];
    const HScal hs = a.hscal[code];
    key = make_ulonglong2(h.v ^ y.v, h.w ^ y.w);
    int q = (product_phase(h.v, h.w, y.v, y.w) + a.rot + a.uH + a.uX) & 3;
    double sy = a.uX ? y.im : y.re;
    t = neg_if(a.f32c ? prod32(hs.sf, sy, 1) : scaled(hs.s, hs.e, sy, 1), (q & 2) != 0);
  } else if (code == kCodePre) {
    key = make_ulonglong2(y.v, y.w);
    t = a.pre_u ? y.im : y.re;
  } else {
    const uint32_t si = code - kCodeSrc;
    key = make_ulonglong2(y.v, y.w);
    double sy = a.src_uy[si] ? y.im : y.re;
    t = neg_if(a.f32c ? prod32(a.src_sf[si], sy, 0) : scaled(a.src_s[si], a.src_e[si], sy, 0), (a.src_q[si] & 2) != 0);
  }
}

// FP32 output sums: the result rounded once to FP32 (round to nearest even), before the test
// that drops exact zeros, so that values rounding to zero are dropped too.
__device__ __forceinline__ void round_out(Cx& r, int round32) {
  if (round32) {
    r.re = (double)__double2float_rn(r.re);
    r.im = (double)__double2float_rn(r.im);
  }
}

// Return the table to empty after a pass (only the slots the pass used).
template <bool S>
__device__ __forceinline__ void release_keys(MergeSmem<S>& s, ulonglong2 sent) {
  const uint32_t n_u = s.n_u;
  for (uint32_t u = threadIdx.x; u < n_u; u += kMergeThreads) {
    uint32_t slot = s.ulist[u];
    s.key[slot] = sent;
    s.head[slot] = kNone;
    s.pre[slot] = kNone16;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.n_u = 0;
    s.n_e = 0;
    s.n_out = 0;
    s.n_long = 0;
    s.flags = 0;
  }
  __syncthreads();
}

constexpr int kNet = 16;         // chains up to this length are sorted in registers
constexpr int kLongChain = 64;   // longer chains: local-array insertion sort; beyond it, selection

// Bitonic sorting network on (k, e) pairs, ascending in k, fully unrolled (registers only).
template <int N>
__device__ __forceinline__ void sort_net(int (&k)[N], uint32_t (&e)[N]) {
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int l = i ^ stride;
        if (l > i) {
          const bool up = (i & size) == 0;
          if ((k[i] > k[l]) == up) {
            int t = k[i]; k[i] = k[l]; k[l] = t;
            uint32_t u = e[i]; e[i] = e[l]; e[l] = u;
          }
        }
      }
    }
  }
}

__device__ __forceinline__ uint32_t chain_next(const uint16_t* enext, uint32_t e) {
  return enext[e] == kNone16 ? kNone : (uint32_t)enext[e];
}

template <bool S>
__device__ __forceinline__ void acc_add(MergeSmem<S>& s, Cx& acc, uint32_t e, bool first) {
  if constexpr (S) {
    acc.re = first ? s.ere[e] : add_rn(acc.re, s.ere[e]);
  } else {
    if (first) acc = Cx{s.ere[e], s.eim[e]};
    else {
      acc.re = add_rn(acc.re, s.ere[e]);
      acc.im = add_rn(acc.im, s.eim[e]);
    }
  }
}

// Sum a slot's chain in (order code, entry) order when it holds at most W entries (sorted
// in registers); returns false, summing nothing, when the chain is longer.
template <bool S, int W>
__device__ __forceinline__ bool chain_sum_regs(MergeSmem<S>& s, uint32_t slot, Cx& acc, uint32_t& n) {
  int ko[W];
  uint32_t ke[W];
  uint32_t e = s.head[slot];
  n = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    if (e != kNone) {
      ko[i] = ((int)s.eord[e] << 11) | (int)e;
      ke[i] = e;
      e = chain_next(s.enext, e);
      ++n;
    } else {
      ko[i] = 0x7FFFFFFF;
      ke[i] = 0;
    }
  }
  if (e != kNone) return false;
  sort_net<W>(ko, ke);
#pragma unroll
  for (int i = 0; i < W; ++i)
    if ((uint32_t)i < n) acc_add(s, acc, ke[i], i == 0);
  return true;
}

// Any chain length: a local-array insertion sort up to kLongChain, else repeated selection.
template <bool S>
__device__ __forceinline__ void chain_sum_long(MergeSmem<S>& s, uint32_t slot, Cx& acc, uint32_t& n) {
  int lo_[kLongChain];
  uint32_t le_[kLongChain];
  uint32_t m = 0;
  uint32_t x = s.head[slot];
  for (; x != kNone && m < (uint32_t)kLongChain; x = chain_next(s.enext, x)) {
    int key = ((int)s.eord[x] << 11) | (int)x;
    int j = (int)m - 1;
    while (j >= 0 && lo_[j] > key) {
      lo_[j + 1] = lo_[j];
      le_[j + 1] = le_[j];
      --j;
    }
    lo_[j + 1] = key;
    le_[j + 1] = x;
    ++m;
  }
  if (x == kNone) {
    n = m;
    for (uint32_t i = 0; i < m; ++i) acc_add(s, acc, le_[i], i == 0);
    return;
  }
  n = 0;
  int last = -1;
  for (;;) {
    int best = 0x7FFFFFFF;
    uint32_t bi = kNone;
    for (uint32_t y = s.head[slot]; y != kNone; y = chain_next(s.enext, y)) {
      int key = ((int)s.eord[y] << 11) | (int)y;
      if (key > last && key < best) {
        best = key;
        bi = y;
      }
    }
    if (bi == kNone) break;
    last = best;
    acc_add(s, acc, bi, n == 0);
    ++n;
  }
}

// The output value of a string: acc alone, or pre + post * acc (absent terms are zero).
template <bool S>
__device__ __forceinline__ Cx finish(const MergeArgs& a, MergeSmem<S>& s, Cx acc, uint32_t n, uint32_t pe) {
  Cx r{0.0, 0.0};
  if constexpr (S) {
    if (a.has_post) {
      double sc = (n > 0) ? neg_if(__dmul_rn(a.post_s, acc.re), (a.post_q & 2) != 0) : 0.0;
      if (pe != kNone16) r.re = (n > 0) ? add_rn(s.ere[pe], sc) : s.ere[pe];
      else r.re = sc;
    } else {
      r.re = acc.re;
    }
  } else {
    if (a.has_post) {
      Cx sc = (n > 0) ? cmul(a.post, acc) : Cx{0.0, 0.0};
      if (pe != kNone16) {
        Cx pv{s.ere[pe], s.eim[pe]};
        r = (n > 0) ? Cx{add_rn(pv.re, sc.re), add_rn(pv.im, sc.im)} : pv;
      } else {
        r = sc;
      }
    } else {
      r = acc;
    }
  }
  return r;
}

// Stage a non-zero result of the pass (warp-aggregated slots in shared memory).
template <bool S>
__device__ __forceinline__ void stage_result(MergeSmem<S>& s, bool flag, Cx r, uint32_t slot, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  uint32_t ob = 0;
  if (lane == leader) ob = atomicAdd(&s.n_out, (uint32_t)__popc(m));
  ob = __shfl_sync(0xffffffffu, ob, leader);
  if (flag) {
    const uint32_t o = ob + __popc(m & ((1u << lane) - 1));
    s.ore[o] = r.re;
    if constexpr (!S) s.oim[o] = r.im;
    s.oslot[o] = (uint16_t)slot;
  }
}

template <bool S>
__global__ void __launch_bounds__(kMergeThreads, 2) k_merge(MergeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MergeSmem<S>& s = *reinterpret_cast<MergeSmem<S>*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const uint32_t ngroups = *a.ngroups;
  // full initialisation once; afterwards each pass releases only what it used
  for (int i = tid; i < kTable; i += kMergeThreads) {
    s.key[i] = a.sent_lo;
    s.head[i] = kNone;
    s.pre[i] = kNone16;
  }
  if (tid == 0) {
    s.n_u = 0;
    s.n_e = 0;
    s.n_out = 0;
    s.n_long = 0;
    s.flags = 0;
    s.cur_sent = a.sent_lo;
  }
  __syncthreads();

  for (;;) {
    if (tid == 0) s.group = atomicAdd(a.next_group, 1u);
    __syncthreads();
    const uint32_t g = s.group;
    __syncthreads();
    if (g >= ngroups) break;
    const uint32_t lo = a.gstart[g], hi = a.gstart[g + 1];
    const uint64_t e0 = a.cpre[lo];
    const uint64_t E = a.cpre[hi] - e0;
    if (E == 0) continue;
    const uint32_t nb = hi - lo;  // <= kMaxGroupBins by the grouping rule
    if (nb > (uint32_t)kMaxGroupBins) {
      if (tid == 0) atomicOr(a.err, 2);
      continue;
    }
    const ulonglong2 sent = (lo >= a.nbins / 2) ? a.sent_hi : a.sent_lo;
    if (sent.x != s.cur_sent.x || sent.y != s.cur_sent.y) {  // groups of the other half: new empty key
      __syncthreads();
      for (int i = tid; i < kTable; i += kMergeThreads) s.key[i] = sent;
      __syncthreads();
      if (tid == 0) s.cur_sent = sent;
    }
    for (uint32_t i = tid; i <= nb; i += kMergeThreads) s.gpre[i] = (uint32_t)(a.cpre[lo + i] - e0);
    for (uint32_t i = tid; i < nb; i += kMergeThreads) s.gbase[i] = a.base[lo + i];
    __syncthreads();

    int level0 = 0;  // split level: a pass (level, sub) keeps keys whose next `level` hash bits equal sub
    while (((uint64_t)kCap << level0) < E && level0 < 16) ++level0;
    if (a.bits + level0 > kHashRows) {  // cannot split this far: report, skip the group
      if (tid == 0) atomicOr(a.err, 2);
      continue;
    }
    if (level0 > 0 && tid == 0) atomicAdd(a.split_groups, 1u);

    for (uint32_t sub0 = 0; sub0 < (1u << level0); ++sub0) {
     // a pass that does not fit is replaced by its two halves (next hash bit 0 / 1)
     int stk_level[2 * kHashRows + 2];
     uint32_t stk_sub[2 * kHashRows + 2];
     int sp = 1;
     stk_level[0] = level0;
     stk_sub[0] = sub0;
     while (sp > 0) {
      --sp;
      const int level = stk_level[sp];
      const uint32_t sub = stk_sub[sp];
      // ---- phase 1: rebuild entries, insert keys, chain each key's entries.  Each thread
      // keeps kBatch entry loads and then kBatch operand gathers in flight together.
      for (uint64_t j0 = 0; j0 < E; j0 += (uint64_t)kBatch * kMergeThreads) {
        uint64_t ent[kBatch];
        Rec rec[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          uint64_t j = j0 + (uint64_t)k * kMergeThreads + tid;
          ent[k] = ~0ull;
          if (j < E) {
            uint32_t l = 0, r = nb;  // gpre[l] <= j < gpre[r]
            while (r - l > 1) {
              uint32_t m = (l + r) >> 1;
              if (s.gpre[m] <= j) l = m; else r = m;
            }
            ent[k] = a.entries[s.gbase[l] + (j - s.gpre[l])];
          }
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          if (ent[k] == ~0ull) continue;
          uint32_t code = (uint32_t)(ent[k] & 0xFFFFu);
          uint64_t idx = ent[k] >> 16;
          const Rec* base = code < kCodeSrc ? a.X : (code == kCodePre ? a.pre : a.src[code - kCodeSrc]);
          rec[k] = base[idx];
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          bool keep = ent[k] != ~0ull;
          ulonglong2 key = make_ulonglong2(0, 0);
          Cx t{0.0, 0.0};
          uint32_t code = 0;
          if (keep) {
            code = (uint32_t)(ent[k] & 0xFFFFu);
            if constexpr (S) build_scalar(a, code, rec[k], key, t.re);
            else build_contribution(a, code, rec[k], key, t);
            if (level > 0) keep = dev_hash(key.x, key.y, a.bits, level) == sub;
          }
          // warp-aggregated entry index for the kept entries
          unsigned m = __ballot_sync(0xffffffffu, keep);
          if (!m) continue;
          const int leader = __ffs(m) - 1;
          uint32_t eb = 0;
          if (lane == leader) eb = atomicAdd(&s.n_e, (uint32_t)__popc(m));
          eb = __shfl_sync(0xffffffffu, eb, leader);
          const uint32_t e = eb + __popc(m & ((1u << lane) - 1));
          bool fresh = false;
          int slot = -1;
          if (keep) {
            if (e >= (uint32_t)kCap) {
              atomicOr(&s.flags, 1);
            } else {
              slot = table_insert(s, key, sent, fresh);
              if (slot < 0) atomicOr(&s.flags, 1);
            }
          }
          // warp-aggregated key list positions for the strings this warp inserted first
          const unsigned mf = __ballot_sync(0xffffffffu, fresh);
          if (mf) {
            const int lf = __ffs(mf) - 1;
            uint32_t ub = 0;
            if (lane == lf) ub = atomicAdd(&s.n_u, (uint32_t)__popc(mf));
            ub = __shfl_sync(0xffffffffu, ub, lf);
            if (fresh) s.ulist[ub + __popc(mf & ((1u << lane) - 1))] = (uint16_t)slot;
          }
          if (slot >= 0) {
            s.ere[e] = t.re;
            if constexpr (!S) s.eim[e] = t.im;
            if (code == kCodePre) {
              s.pre[slot] = (uint16_t)e;
            } else {
              s.eord[e] = (uint16_t)code;
              s.enext[e] = (uint16_t)atomicExch(&s.head[slot], e);
            }
          }
        }
      }
      __syncthreads();
      if (s.flags) {  // this pass did not fit: process its two halves instead
        release_keys(s, sent);
        if (level >= 16 || a.bits + level + 1 > kHashRows || sp + 2 > 2 * kHashRows + 2) {
          if (tid == 0) atomicOr(a.err, 2);
          continue;
        }
        if (level == 0 && tid == 0) atomicAdd(a.split_groups, 1u);
        stk_level[sp] = level + 1;
        stk_sub[sp] = sub + (1u << level);
        stk_level[sp + 1] = level + 1;
        stk_sub[sp + 1] = sub;
        sp += 2;
        continue;
      }
      const uint32_t n_u = s.n_u;
      // ---- phase 2: per string, sum its contributions in increasing order code (H order,
      // then the sources), apply the combination, stage the non-zero results.  Chains of at
      // most 4 entries first; longer chains are queued and done densely afterwards.
      for (uint32_t u0 = 0; u0 < n_u; u0 += kMergeThreads) {
        const uint32_t u = u0 + tid;
        Cx r{0.0, 0.0};
        bool flag = false, deferred = false;
        uint32_t slot = 0;
        if (u < n_u) {
          slot = s.ulist[u];
          const uint32_t pe = s.pre[slot];
          Cx acc{0.0, 0.0};
          uint32_t n = 0;
          if (chain_sum_regs<S, 4>(s, slot, acc, n)) {
            r = finish(a, s, acc, n, pe);
            round_out(r, a.round32);
            flag = !(is_zero(r.re) && is_zero(r.im)) && (n > 0 || pe != kNone16);
          } else {
            deferred = true;
          }
        }
        const unsigned md = __ballot_sync(0xffffffffu, deferred);
        if (md) {
          const int leader = __ffs(md) - 1;
          uint32_t qb = 0;
          if (lane == leader) qb = atomicAdd(&s.n_long, (uint32_t)__popc(md));
          qb = __shfl_sync(0xffffffffu, qb, leader);
          if (deferred) s.longq[qb + __popc(md & ((1u << lane) - 1))] = (uint16_t)slot;
        }
        stage_result(s, flag, r, slot, lane);
      }
      __syncthreads();
      const uint32_t n_long = s.n_long;
      for (uint32_t q0 = 0; q0 < n_long; q0 += kMergeThreads) {
        const uint32_t q = q0 + tid;
        Cx r{0.0, 0.0};
        bool flag = false;
        uint32_t slot = 0;
        if (q < n_long) {
          slot = s.longq[q];
          const uint32_t pe = s.pre[slot];
          Cx acc{0.0, 0.0};
          uint32_t n = 0;
          if (!chain_sum_regs<S, kNet>(s, slot, acc, n)) {
            acc = Cx{0.0, 0.0};
            chain_sum_long(s, slot, acc, n);
          }
          r = finish(a, s, acc, n, pe);
          round_out(r, a.round32);
          flag = !(is_zero(r.re) && is_zero(r.im)) && (n > 0 || pe != kNone16);
        }
        stage_result(s, flag, r, slot, lane);
      }
      __syncthreads();
      // ---- phase 3: one output reservation per pass, coalesced writes
      const uint32_t n_out = s.n_out;
      if (tid == 0) s.out_base = n_out ? atomicAdd(a.out_n, (unsigned long long)n_out) : 0ull;
      __syncthreads();
      const unsigned long long ob = s.out_base;
      if (ob + n_out > a.out_cap) {
        if (tid == 0 && n_out) atomicOr(a.err, 1);
      } else {
        for (uint32_t i = tid; i < n_out; i += kMergeThreads) {
          const ulonglong2 k = s.key[s.oslot[i]];
          if constexpr (S) {
            const double x = s.ore[i];
            a.out[ob + i] = a.out_imag ? Rec{k.x, k.y, 0.0, x} : Rec{k.x, k.y, x, 0.0};
          } else {
            a.out[ob + i] = Rec{k.x, k.y, s.ore[i], s.oim[i]};
          }
        }
      }
      __syncthreads();
      release_keys(s, sent);
     }
    }
  }
}

// ----------------------------------------------------------------------------- ranked merge
// The merge used when the order codes fit a kMaskBits-bit mask (|H| + sources <= 256).  Each
// slot records which order codes contributed; once all entries of a pass are in, the rank of
// a contribution among its string's contributions is the popcount of the lower mask bits, so
// it is written straight to its ordered position in a per-string run, and each string is
// summed over its contiguous run in increasing order code.  Valid inputs (distinct strings in
// every operand) give distinct order codes per string.
constexpr int kMaskWords = 8;  // 32-bit words: shared-memory OR on 32 bits is one native atomic
constexpr int kMaskBits = 32 * kMaskWords;

// Geometry of a ranked merge with W mask words: W = 8 (256 order codes) keeps 1024 slots and
// passes of up to kCap entries; W = 16 (512 codes, for larger H) halves both so that two
// blocks still fit an SM.  W = 0 is the chained rank for any number of order codes: no masks;
// each slot chains its entries, and an entry's rank is the number of entries of its chain with
// a smaller order code (a string's order codes are distinct), so the geometry stays at 1024
// slots and kCap entries whatever the number of codes.  kBits is then the number of run-length
// classes of the phase-4 ordering (longer runs share the last class).
template <int W>
struct RankGeom {
  static constexpr int kWords = W;
  static constexpr int kBits = W == 0 ? 64 : 32 * W;
  static constexpr int kTab = W <= 8 ? kTable : kTable / 2;
  static constexpr int kEnt = W <= 8 ? kCap : kCap / 2;
};

// Next-group prefetch (ranked merge with at most six mask words, where shared memory has room):
// while a group is merged, its successor's header and bin table are copied into shared memory
// with cp.async and its entries are prefetched into L2 with bulk prefetches, so the next setup
// and load phase do not wait on DRAM.
template <int W>
struct PfGeom {
  static constexpr int kBins = W <= 6 ? 256 : 1;  // bins of a prefetchable group
  static constexpr bool kOn = W <= 6;
};
constexpr uint32_t kNone32 = 0xFFFFFFFFu;

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2_bulk(const void* gsrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

template <bool S, int W>
struct RankSmem {
  using G = RankGeom<W>;
  GroupHead pfh;                              // header of the prefetched next group
  uint64_t pfbase[PfGeom<W>::kBins];          // its bin starts
  uint64_t pfcpre[PfGeom<W>::kBins + 1];      // its bins' entry prefix
  uint32_t pf_g;                              // the group whose header and bins are in pf*, or kNone
  ulonglong2 key[G::kTab];
  uint32_t mask[W > 0 ? G::kTab : 1][W > 0 ? G::kWords : 1];  // order codes present per slot (W > 0)
  uint32_t head[W == 0 ? G::kTab : 1];            // W = 0: last entry of the slot's chain, or kNone32
  uint16_t enext[W == 0 ? G::kEnt : 1];           // W = 0: previous entry of the same slot, or kNone16
  uint16_t pre[G::kTab];
  uint16_t ulist[G::kTab];
  uint16_t run[G::kTab];        // start of the slot's run in seg[]
  uint16_t rlen[G::kTab];       // length of the slot's run (popcount of its mask)
  double ere[G::kEnt];
  double eim[S ? 1 : G::kEnt];
  uint16_t ebit[G::kEnt];         // order bit (W = 0: order code) of the entry (kNone16: pre operand)
  uint16_t eslot[G::kEnt];
  double seg[G::kEnt];            // contributions ordered by (string, order code)
  double segim[S ? 1 : G::kEnt];
  double ore[G::kTab];
  double oim[S ? 1 : G::kTab];
  uint16_t oslot[G::kTab];
  uint32_t hist[W > 8 ? G::kBits + 1 : 1];  // run-length counters when they outgrow oslot
  unsigned long long gbase[kMaxGroupBins];
  uint32_t gpre[kMaxGroupBins + 1];
  uint32_t n_e, n_u, n_out, n_seg;
  int flags;
  unsigned group;
  unsigned long long out_base;
  ulonglong2 cur_sent;
  uint32_t h_g;  // the block's next group, claimed while the current one is set up
};

template <bool S, int W>
__device__ __forceinline__ void rank_release(RankSmem<S, W>& s, ulonglong2 sent) {
  using G = RankGeom<W>;
  const uint32_t n_u = s.n_u;
  for (uint32_t u = threadIdx.x; u < n_u; u += kMergeThreads) {
    const uint32_t slot = s.ulist[u];
    s.key[slot] = sent;
    if constexpr (W == 0) {
      s.head[slot] = kNone32;
    } else {
#pragma unroll
      for (int w = 0; w < G::kWords; ++w) s.mask[slot][w] = 0u;
    }
    s.pre[slot] = kNone16;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s.n_u = 0;
    s.n_e = 0;
    s.n_out = 0;
    s.n_seg = 0;
    s.flags = 0;
  }
  __syncthreads();
}

__device__ __forceinline__ uint32_t code_bit(uint32_t code, int nH) {
  return code < kCodeSrc ? code : (uint32_t)nH + (code - kCodeSrc);
}

template <bool S, bool FULL, int W>
__global__ void __launch_bounds__(kMergeThreads, 2) k_merge_rank(MergeArgs a) {
  using G = RankGeom<W>;
  constexpr int B = FULL ? kBatchFull : kBatch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RankSmem<S, W>& s = *reinterpret_cast<RankSmem<S, W>*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const uint32_t ngroups = *a.ngroups;
  int top_acc = -100000;  // okeys: this thread's largest exponent bound
  for (int i = tid; i < G::kTab; i += kMergeThreads) {
    s.key[i] = a.sent_lo;
    if constexpr (W == 0) {
      s.head[i] = kNone32;
    } else {
#pragma unroll
      for (int w = 0; w < G::kWords; ++w) s.mask[i][w] = 0u;
    }
    s.pre[i] = kNone16;
  }
  if (tid == 0) {
    s.n_u = s.n_e = s.n_out = s.n_seg = 0;
    s.flags = 0;
    s.cur_sent = a.sent_lo;
    s.pf_g = kNone;
  }
  constexpr bool PF = PfGeom<W>::kOn;
  // Groups are claimed from a shared counter.  The next group is claimed while the current
  // one's setup runs, by the last warp's lane 0 (no bin-table work: a group has fewer bins
  // than the first 480 threads), so the claim's round trip overlaps the header and table
  // reads of the other threads.
  constexpr int kClaimTid = kMergeThreads - 32;
  if (tid == kClaimTid) s.h_g = atomicAdd(a.next_group, 1u);
  for (;;) {
    __syncthreads();
    const uint32_t g = s.h_g;
    __syncthreads();  // g read by all before the next claim overwrites it
    if (g >= ngroups) break;
    if (tid == kClaimTid) s.h_g = atomicAdd(a.next_group, 1u);
    const bool pf_hit = PF && s.pf_g == g;  // header and bins already in shared memory
    const GroupHead gh = pf_hit ? s.pfh : a.heads[g];
    const uint32_t lo = gh.lo, hi = gh.hi;
    const uint64_t e0 = gh.e0;
    const uint64_t E = gh.E;
    if (E == 0 || hi - lo > (uint32_t)kMaxGroupBins) {
      if (E != 0 && tid == 0) atomicOr(a.err, 2);
      continue;
    }
    const uint32_t nb = hi - lo;
    const ulonglong2 sent = (lo >= a.nbins / 2) ? a.sent_hi : a.sent_lo;
    if (sent.x != s.cur_sent.x || sent.y != s.cur_sent.y) {
      __syncthreads();
      for (int i = tid; i < G::kTab; i += kMergeThreads) s.key[i] = sent;
      __syncthreads();
      if (tid == 0) s.cur_sent = sent;
    }
    if (pf_hit) {
      for (uint32_t i = tid; i <= nb; i += kMergeThreads) s.gpre[i] = (uint32_t)(s.pfcpre[i] - e0);
      for (uint32_t i = tid; i < nb; i += kMergeThreads) s.gbase[i] = s.pfbase[i];
    } else {
      for (uint32_t i = tid; i <= nb; i += kMergeThreads) s.gpre[i] = (uint32_t)(a.cpre[lo + i] - e0);
      for (uint32_t i = tid; i < nb; i += kMergeThreads) s.gbase[i] = a.base[lo + i];
    }
    __syncthreads();

    int level0 = 0;
    while (((uint64_t)G::kEnt << level0) < E && level0 < 16) ++level0;
    if (a.bits + level0 > kHashRows) {
      if (tid == 0) atomicOr(a.err, 2);
      continue;
    }
    if (level0 > 0 && tid == 0) atomicAdd(a.split_groups, 1u);
    // the next group (claimed during this setup): its header now, its bins after phase 2, its
    // entries into L2 after phase 3
    const uint32_t gn = s.h_g;
    bool pf_first = PF && gn < ngroups;  // block-uniform; cleared after the group's first pass
    if (pf_first && tid == 0) {
      s.pf_g = kNone;
      cp_async16(&s.pfh, &a.heads[gn]);
      cp_async16(reinterpret_cast<char*>(&s.pfh) + 16, reinterpret_cast<const char*>(&a.heads[gn]) + 16);
      cp_async_commit();
    }

    for (uint32_t sub0 = 0; sub0 < (1u << level0); ++sub0) {
     int stk_level[2 * kHashRows + 2];
     uint32_t stk_sub[2 * kHashRows + 2];
     int sp = 1;
     stk_level[0] = level0;
     stk_sub[0] = sub0;
     while (sp > 0) {
      --sp;
      const int level = stk_level[sp];
      const uint32_t sub = stk_sub[sp];
      // run-length histogram for phase 3b, in oslot (free until phase 4 stages outputs)
      uint32_t* s_hist = W > 8 ? s.hist : reinterpret_cast<uint32_t*>(s.oslot);  // G::kBits + 1 counters
      for (uint32_t i = tid; i <= (uint32_t)G::kBits; i += kMergeThreads) s_hist[i] = 0;
      // ---- phase 1: rebuild entries, insert keys, mark order codes per key
      for (uint64_t j0 = 0; j0 < E; j0 += (uint64_t)B * kMergeThreads) {
        uint64_t ent[B];
        Rec rec[B];
        Contrib cf[B];
        bool has[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
          uint64_t j = j0 + (uint64_t)k * kMergeThreads + tid;
          has[k] = j < E;
          ent[k] = 0;
          if (has[k]) {
            uint32_t l = 0, r = nb;
            while (r - l > 1) {
              uint32_t m = (l + r) >> 1;
              if (s.gpre[m] <= j) l = m; else r = m;
            }
            if constexpr (FULL) cf[k] = a.fent[s.gbase[l] + (j - s.gpre[l])];
            else ent[k] = a.entries[s.gbase[l] + (j - s.gpre[l])];
          }
        }
        if constexpr (!FULL) {
#pragma unroll
          for (int k = 0; k < B; ++k) {
            if (!has[k]) continue;
            uint32_t code = (uint32_t)(ent[k] & 0xFFFFu);
            uint64_t idx = ent[k] >> 16;
            const Rec* base = code < kCodeSrc ? a.X : (code == kCodePre ? a.pre : a.src[code - kCodeSrc]);
            rec[k] = base[idx];
          }
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
          bool keep = has[k];
          ulonglong2 key = make_ulonglong2(0, 0);
          Cx t{0.0, 0.0};
          uint32_t code = 0;
          if (keep) {
            if constexpr (FULL) {
              key = make_ulonglong2(cf[k].v, cf[k].w);
              t.re = cf[k].val;
              code = cf[k].code;
            } else {
              code = (uint32_t)(ent[k] & 0xFFFFu);
              if constexpr (S) build_scalar(a, code, rec[k], key, t.re);
              else build_contribution(a, code, rec[k], key, t);
            }
            if (level > 0) keep = dev_hash(key.x, key.y, a.bits, level) == sub;
          }
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (!m) continue;
          uint32_t e;
          if (level == 0) {
            e = (uint32_t)(j0 + (uint64_t)k * kMergeThreads + tid);  // every entry kept, E <= G::kEnt
          } else {
            const int leader = __ffs(m) - 1;
            uint32_t eb = 0;
            if (lane == leader) eb = atomicAdd(&s.n_e, (uint32_t)__popc(m));
            eb = __shfl_sync(0xffffffffu, eb, leader);
            e = eb + __popc(m & ((1u << lane) - 1));
          }
          bool fresh = false;
          int slot = -1;
          if (keep) {
            if (e >= (uint32_t)G::kEnt) {
              atomicOr(&s.flags, 1);
            } else {
              slot = table_insert<G::kTab>(s, key, sent, fresh);
              if (slot < 0) atomicOr(&s.flags, 1);
            }
          }
          const unsigned mf = __ballot_sync(0xffffffffu, fresh);
          if (mf) {
            const int lf = __ffs(mf) - 1;
            uint32_t ub = 0;
            if (lane == lf) ub = atomicAdd(&s.n_u, (uint32_t)__popc(mf));
            ub = __shfl_sync(0xffffffffu, ub, lf);
            if (fresh) s.ulist[ub + __popc(mf & ((1u << lane) - 1))] = (uint16_t)slot;
          }
          if (slot >= 0) {
            s.ere[e] = t.re;
            if constexpr (!S) s.eim[e] = t.im;
            s.eslot[e] = (uint16_t)slot;
            if (code == kCodePre) {
              s.pre[slot] = (uint16_t)e;
              s.ebit[e] = kNone16;
            } else {
              const uint32_t bit = code_bit(code, a.nH);
              s.ebit[e] = (uint16_t)bit;
              if constexpr (W == 0) {
                const uint32_t prev = atomicExch(&s.head[slot], e);
                s.enext[e] = prev == kNone32 ? kNone16 : (uint16_t)prev;
              } else {
                atomicOr(&s.mask[slot][bit >> 5], 1u << (bit & 31));
              }
            }
          }
        }
      }
      __syncthreads();
      if (pf_first && tid == 0) cp_async_wait_all();  // the next header (visible after the next barrier)
      if (s.flags) {
        pf_first = false;
        rank_release(s, sent);
        if (level >= 16 || a.bits + level + 1 > kHashRows || sp + 2 > 2 * kHashRows + 2) {
          if (tid == 0) atomicOr(a.err, 2);
          continue;
        }
        if (level == 0 && tid == 0) atomicAdd(a.split_groups, 1u);
        stk_level[sp] = level + 1;
        stk_sub[sp] = sub + (1u << level);
        stk_level[sp + 1] = level + 1;
        stk_sub[sp + 1] = sub;
        sp += 2;
        continue;
      }
      const uint32_t n_u = s.n_u, n_e = level == 0 ? (uint32_t)E : s.n_e;
      // ---- phase 2: a run per string (its length is the popcount of its mask)
      for (uint32_t u0 = 0; u0 < n_u; u0 += kMergeThreads) {
        const uint32_t u = u0 + tid;
        uint32_t c = 0, slot = 0;
        if (u < n_u) {
          slot = s.ulist[u];
          if constexpr (W == 0) {
            for (uint32_t y = s.head[slot]; y != kNone32;) {
              ++c;
              const uint16_t nx = s.enext[y];
              y = nx == kNone16 ? kNone32 : (uint32_t)nx;
            }
          } else {
#pragma unroll
            for (int w = 0; w < G::kWords; ++w) c += __popc(s.mask[slot][w]);
          }
        }
        // warp-inclusive scan of c, one shared-memory reservation per warp
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        uint32_t wb = 0;
        if (lane == 31) wb = atomicAdd(&s.n_seg, incl);
        wb = __shfl_sync(0xffffffffu, wb, 31);
        if (u < n_u) {
          s.run[slot] = (uint16_t)(wb + incl - c);
          s.rlen[slot] = (uint16_t)c;
          atomicAdd(&s_hist[G::kBits - min(c, (uint32_t)G::kBits)], 1u);  // longest runs first
        }
      }
      __syncthreads();
      if (pf_first) {  // the next group's bin table into shared memory
        const GroupHead nh = s.pfh;
        const uint32_t nb2 = nh.hi - nh.lo;
        if (nh.E != 0 && nb2 <= (uint32_t)PfGeom<W>::kBins && (uint32_t)tid <= nb2) {
          cp_async8(&s.pfcpre[tid], &a.cpre[nh.lo + tid]);
          if ((uint32_t)tid < nb2) cp_async8(&s.pfbase[tid], &a.base[nh.lo + tid]);
        }
        cp_async_commit();
      }
      if (tid < 32) {  // exclusive scan of the run-length counters, 9 per lane, before phase 3
        constexpr int kPer = (G::kBits + 1 + 31) / 32;
        uint32_t v[kPer], t = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const int i = tid * kPer + k;
          v[k] = i <= G::kBits ? s_hist[i] : 0u;
          t += v[k];
        }
        uint32_t incl = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
          if (tid >= d) incl += y;
        }
        uint32_t run = incl - t;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const int i = tid * kPer + k;
          if (i <= G::kBits) s_hist[i] = run;
          run += v[k];
        }
      }
      // ---- phase 3: every contribution to its ordered position in its string's run
      for (uint32_t e = tid; e < n_e; e += kMergeThreads) {
        const uint32_t bit = s.ebit[e];
        if (bit == kNone16) continue;
        const uint32_t slot = s.eslot[e];
        uint32_t rank = 0;
        if constexpr (W == 0) {  // entries of the chain with a smaller order code
          for (uint32_t y = s.head[slot]; y != kNone32;) {
            rank += s.ebit[y] < bit ? 1u : 0u;
            const uint16_t nx = s.enext[y];
            y = nx == kNone16 ? kNone32 : (uint32_t)nx;
          }
        } else {
          const uint32_t wi = bit >> 5;
          rank = __popc(s.mask[slot][wi] & ((1u << (bit & 31)) - 1u));
#pragma unroll
          for (int w = 0; w < G::kWords; ++w)
            if ((uint32_t)w < wi) rank += __popc(s.mask[slot][w]);
        }
        const uint32_t pos = s.run[slot] + rank;
        s.seg[pos] = s.ere[e];
        if constexpr (!S) s.segim[pos] = s.eim[e];
      }
      if (pf_first) cp_async_wait_all();  // this thread's bin-table copies (visible after the barrier)
      __syncthreads();
      // ---- phase 3b: strings ordered by run length, longest first, so that the lanes of a
      // warp add runs of nearly equal length in phase 4 (the adds of a warp cost as much as
      // its longest run): the scatter of a counting sort whose counts phase 2 took; eslot
      // is free once phase 3 is done.
      uint16_t* s_order = s.eslot;
      for (uint32_t u = tid; u < n_u; u += kMergeThreads) {
        const uint32_t slot = s.ulist[u];
        const uint32_t n = s.rlen[slot];
        s_order[atomicAdd(&s_hist[G::kBits - min(n, (uint32_t)G::kBits)], 1u)] = (uint16_t)slot;
      }
      __syncthreads();
      if (pf_first) {  // the next group's entries into L2; its header and bins are ready
        const GroupHead nh = s.pfh;
        const uint32_t nb2 = nh.hi - nh.lo;
        if (nh.E != 0 && nb2 <= (uint32_t)PfGeom<W>::kBins) {
          if constexpr (FULL) {
            if ((uint32_t)tid < nb2) {
              const uint64_t cnt = s.pfcpre[tid + 1] - s.pfcpre[tid];
              if (cnt) prefetch_l2_bulk(a.fent + s.pfbase[tid], (uint32_t)(cnt * sizeof(Contrib)));
            }
          }
          if (tid == 0) s.pf_g = gn;
        }
        pf_first = false;
      }
      // ---- phase 4: per string, add its run in order, apply the combination, stage.  The
      // fold uses plain IEEE adds: they differ from skipping zero terms only in the sign of
      // a zero sum, and strings whose value is zero are dropped.
      for (uint32_t u0 = 0; u0 < n_u; u0 += kMergeThreads) {
        const uint32_t u = u0 + tid;
        Cx r{0.0, 0.0};
        bool flag = false;
        uint32_t slot = 0;
        if (u < n_u) {
          slot = s_order[u];
          const uint32_t n = s.rlen[slot];
          const uint32_t b0 = s.run[slot];
          Cx acc{0.0, 0.0};
          if (S && a.f32c) {  // Sum2 in FP32
            float sum = n > 0 ? f32_exact(s.seg[b0]) : 0.0f, err = 0.0f;
            for (uint32_t i = 1; i < n; ++i) {
              float e;
              two_sum32(sum, f32_exact(s.seg[b0 + i]), sum, e);
              err = __fadd_rn(err, e);
            }
            acc.re = f64_of(__fadd_rn(sum, err));
          } else {
            if (n > 0) {
              acc.re = s.seg[b0];
              if constexpr (!S) acc.im = s.segim[b0];
            }
            for (uint32_t i = 1; i < n; ++i) {
              acc.re = __dadd_rn(acc.re, s.seg[b0 + i]);
              if constexpr (!S) acc.im = __dadd_rn(acc.im, s.segim[b0 + i]);
            }
          }
          const uint32_t pe = s.pre[slot];
          if constexpr (S) {
            if (a.has_post && a.f32c) {
              const double sc = (n > 0) ? neg_if(prod32(a.post_sf, acc.re, 0), (a.post_q & 2) != 0) : 0.0;
              if (pe != kNone16) r.re = (n > 0) ? add_rn32(s.ere[pe], sc) : s.ere[pe];
              else r.re = sc;
            } else if (a.has_post) {
              double sc = (n > 0) ? neg_if(__dmul_rn(a.post_s, acc.re), (a.post_q & 2) != 0) : 0.0;
              if (pe != kNone16) r.re = (n > 0) ? add_rn(s.ere[pe], sc) : s.ere[pe];
              else r.re = sc;
            } else {
              r.re = acc.re;
            }
          } else {
            if (a.has_post) {
              Cx sc = (n > 0) ? cmul(a.post, acc) : Cx{0.0, 0.0};
              if (pe != kNone16) {
                Cx pv{s.ere[pe], s.eim[pe]};
                r = (n > 0) ? Cx{add_rn(pv.re, sc.re), add_rn(pv.im, sc.im)} : pv;
              } else {
                r = sc;
              }
            } else {
              r = acc;
            }
          }
          round_out(r, a.round32);
          flag = !(is_zero(r.re) && is_zero(r.im)) && (n > 0 || pe != kNone16);
        }
        const unsigned m = __ballot_sync(0xffffffffu, flag);
        if (m) {
          const int leader = __ffs(m) - 1;
          uint32_t ob = 0;
          if (lane == leader) ob = atomicAdd(&s.n_out, (uint32_t)__popc(m));
          ob = __shfl_sync(0xffffffffu, ob, leader);
          if (flag) {
            const uint32_t o = ob + __popc(m & ((1u << lane) - 1));
            s.ore[o] = r.re;
            if constexpr (!S) s.oim[o] = r.im;
            s.oslot[o] = (uint16_t)slot;
          }
        }
      }
      __syncthreads();
      // ---- phase 5: one output reservation per pass, coalesced writes
      const uint32_t n_out = s.n_out;
      if (tid == 0) s.out_base = n_out ? atomicAdd(a.out_n, (unsigned long long)n_out) : 0ull;
      __syncthreads();
      const unsigned long long ob = s.out_base;
      if (ob + n_out > a.out_cap) {
        if (tid == 0 && n_out) atomicOr(a.err, 1);
      } else {
        for (uint32_t i = tid; i < n_out; i += kMergeThreads) {
          const ulonglong2 k = s.key[s.oslot[i]];
          if constexpr (S) {
            const double x = s.ore[i];
            a.out[ob + i] = a.out_imag ? Rec{k.x, k.y, 0.0, x} : Rec{k.x, k.y, x, 0.0};
            if (a.okeys) {  // the norm's first pass, folded in: rank key and exponent bound
              a.okeys[ob + i] = (uint64_t)__double_as_longlong(x) & ~(1ull << 63);
              top_acc = max(top_acc, max(exact::prod_top(x, x), exact::nonfinite_top(x)));
            }
          } else {
            a.out[ob + i] = Rec{k.x, k.y, s.ore[i], s.oim[i]};
          }
        }
      }
      __syncthreads();
      rank_release(s, sent);
     }
    }
  }
  if constexpr (S) {
    if (a.okeys) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) top_acc = max(top_acc, __shfl_down_sync(0xffffffffu, top_acc, o));
      if (lane == 0 && top_acc > -100000) atomicMax(a.otop, top_acc);
    }
  }
}

// Merge geometry: the target entries per hash bin (sets the number of bins) and the group
// quota (entries per group before a new group starts).  Defaults, or the autotuner's choice
// for the size class (log2 of the entry bound) of the merge.
struct MergeGeom {
  int bin_target = 2048;
  int quota = kGroupQuota;
};
std::mutex g_tune_mu;
MergeGeom g_tuned[64];
bool g_has_tuned[64] = {};
thread_local const MergeGeom* t_force = nullptr;  // the autotuner's candidate under test
thread_local int t_last_class = -1;

int size_class(int64_t bound_total) {
  int c = 0;
  while (c < 63 && ((int64_t)1 << (c + 1)) <= bound_total) ++c;
  return c;
}

MergeGeom g_fixed{};        // a geometry set for every class (tests of each geometry)
bool g_has_fixed = false;

MergeGeom geometry_for(int64_t bound_total) {
  const int c = size_class(bound_total);
  t_last_class = c;
  if (t_force) return *t_force;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_has_fixed) return g_fixed;
  return g_has_tuned[c] ? g_tuned[c] : MergeGeom{};
}

int choose_bits(int64_t bound_total, int bin_target) {
  int b = 4;
  while (b < 20 && ((int64_t)1 << b) * bin_target < bound_total) ++b;
  return b;
}

std::mutex g_stats_mu;
pauli_merge_stats g_stats{};

}  // namespace

void record_merge_stats(const pauli_merge_stats& st) {
  std::lock_guard<std::mutex> lk(g_stats_mu);
  g_stats = st;
}

int merge_run(const MergeSpec& sp, cudaStream_t s, pauli_sum* out) {
  if (sp.keys_out) *sp.keys_out = nullptr;
  PS_TRY(upload_hash_tables());
  if (sp.nH > kMaxH || sp.nsrc > 4) return PS_ERR_INVALID;
  const int64_t nX = (sp.X && sp.nH > 0) ? sp.nX : 0;
  int64_t nsrc_total = sp.npre;
  bool has_ts = false;
  for (int i = 0; i < sp.nsrc; ++i) {
    nsrc_total += sp.src[i].n * (sp.src[i].ts == kTsExpand ? sp.ring : 1);
    has_ts |= sp.src[i].ts != 0;
  }
  // translation-symmetric sources: no product operand, their shifts are the first order codes
  if (has_ts && (nX > 0 || sp.ring < 2 || sp.ring > 64)) return PS_ERR_INVALID;
  const int ncode_h = nX > 0 ? sp.nH : (has_ts ? sp.ring : 0);
  const int64_t pairs = (int64_t)sp.nH * nX;
  const int64_t bound_total = pairs + nsrc_total;
  pauli_merge_stats st{};
  st.pair_tests = pairs;
  if (bound_total == 0) {
    out->n = 0;
    out->cls = 0;
    record_merge_stats(st);
    return PS_OK;
  }
  const MergeGeom geom = geometry_for(bound_total);
  // without a product operand the bound is the exact entry count, which fills a bin to the
  // target and leaves no room in a pass for the bin's neighbours: quarter-size bins then
  const int bits = choose_bits(bound_total, nX > 0 ? geom.bin_target : std::max(64, geom.bin_target / 4));
  const uint32_t nbins = 1u << bits;
  const bool small_plan = nbins <= kSmallPlanBins;  // one block each for the bin bounds and the group plan
  const int nsm = num_sms();
  auto grid_for = [&](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 16 * nsm)); };
  // shared-memory histograms: fewer, fuller blocks (one flush of the bins per block)
  auto hist_grid = [&](int64_t n) { return bits <= kHistSmemBits ? std::min(grid_for(n), 2 * nsm) : grid_for(n); };

  // ---- coefficient classes: the merge runs in single-component mode when every term of
  // every output string lies in the same component (real or imaginary)
  auto cls_scalar = [](Cx c) { return cls_of(c.re, c.im); };
  int prod_cls = 0;
  if (nX > 0) {
    if (sp.product) {
      prod_cls = kClsComplex;  // i^k with k of either parity
    } else {
      prod_cls = cls_mul(sp.clsH, sp.clsX);  // then times i^(k + rot) with k odd
      if (!(sp.rot & 1)) prod_cls = cls_swap(prod_cls);
    }
  }
  int acc_cls = prod_cls;
  for (int i = 0; i < sp.nsrc; ++i)
    acc_cls |= sp.src[i].n > 0 ? cls_mul(cls_scalar(sp.src[i].alpha), sp.src[i].cls) : 0;
  int out_cls = acc_cls;
  if (sp.has_post) out_cls = (sp.npre > 0 ? sp.clsPre : 0) | cls_mul(cls_scalar(sp.post), acc_cls);
  const bool structured = acc_cls != kClsComplex && out_cls != kClsComplex;
  // ranked merge when the order codes fit the slot masks, chained merge otherwise; full
  // contribution records (no gather in the merge) when single-component and they fit
  // ranked merge when the order codes fit the slot masks (256 codes; 512 with the wide
  // geometry), chained merge otherwise
  const bool ranked = ncode_h + sp.nsrc <= kMaskBits;
  // beyond 256 codes: single-component merges rank by slot chains (any number of codes),
  // complex ones by 512-bit masks up to 512 codes, else the chained merge
  const bool chained_rank = !ranked && !has_ts && structured;
  const bool ranked_wide = !ranked && !chained_rank && !has_ts && ncode_h + sp.nsrc <= RankGeom<16>::kBits;
  const bool full = structured && ranked && (uint64_t)bound_total * sizeof(Contrib) <= kFullBudget;
  if (has_ts && !full) return PS_ERR_INVALID;  // representatives need full records: one component
  // FP32 arithmetic with compensated sums: single-component ranked merges
  const int f32c = out->f32 == 2 ? 1 : 0;
  if (f32c && !(structured && (ranked || ranked_wide || chained_rank))) return PS_ERR_INVALID;
  // per-instance H coefficients ride on the table emission of full records
  if (sp.hbatch && nX > 0 && !(full && sp.nH <= kMaskBits && !sp.product)) return PS_ERR_INVALID;

  auto pow2_exp = [](double x) -> int {
    uint64_t b;
    memcpy(&b, &x, 8);
    int E = (int)((b >> 52) & 0x7FF);
    return ((b & ((1ull << 52) - 1)) == 0 && E >= 1 && E <= 2046) ? E - 1023 : kNoPow2;
  };
  MergeArgs a{};
  EmitScalars es{};
  Buf<HScal> hscal;
  if (structured) {
    a.uH = sp.clsH == kClsImag;
    a.uX = sp.clsX == kClsImag;
    if (nX > 0) {
      PS_TRY(hscal.alloc(sp.nH, s));
      a.hscal = hscal.p;
    }
    for (int i = 0; i < sp.nsrc; ++i) {
      int ua = cls_scalar(sp.src[i].alpha) == kClsImag;
      int uy = sp.src[i].cls == kClsImag;
      a.src_s[i] = ua ? sp.src[i].alpha.im : sp.src[i].alpha.re;
      a.src_e[i] = pow2_exp(a.src_s[i]);
      a.src_q[i] = ua + uy;
      a.src_uy[i] = uy;
    }
    a.pre_u = sp.clsPre == kClsImag;
    int up = cls_scalar(sp.post) == kClsImag;
    a.post_s = up ? sp.post.im : sp.post.re;
    a.post_sf = (float)a.post_s;
    a.post_q = up + (acc_cls == kClsImag);
    a.out_imag = out_cls == kClsImag;
    es.f32c = out->f32 == 2 ? 1 : 0;
    es.rot = sp.rot;
    es.uH = a.uH;
    es.uX = a.uX;
    for (int i = 0; i < 4; ++i) {
      a.src_sf[i] = (float)a.src_s[i];
      es.src_sf[i] = a.src_sf[i];
      es.src_s[i] = a.src_s[i];
      es.src_e[i] = a.src_e[i];
      es.src_q[i] = a.src_q[i];
      es.src_uy[i] = a.src_uy[i];
    }
    es.pre_u = a.pre_u;
  }

  Buf<uint32_t> fX, fH, histX, histY, cnt, flag, gstart;
  Buf<GroupHead> heads;
  Buf<uint64_t> bound, base, cpre, fpre, entries;
  Buf<Contrib> fent;
  Buf<unsigned long long> counters;  // [0] product entries, [1] out_n
  Buf<unsigned> misc;                // [0] next_group, [1] ngroups, [2] split groups
  Buf<int> err;
  PS_TRY(histY.alloc(nbins, s));
  if (!small_plan) {
    PS_TRY(cnt.alloc(nbins, s));
    PS_TRY(bound.alloc(nbins, s));
  }
  PS_TRY(base.alloc(nbins + 1, s));
  PS_TRY(counters.alloc(2, s));
  PS_TRY(misc.alloc(3, s));
  PS_TRY(err.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(histY.p, 0, nbins * sizeof(uint32_t), s));
  PS_CUDA(cudaMemsetAsync(counters.p, 0, 2 * sizeof(unsigned long long), s));
  PS_CUDA(cudaMemsetAsync(misc.p, 0, 3 * sizeof(unsigned), s));
  PS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));

  // ---- 1. hashes, histograms and bin bounds
  const bool use_tab = nX > 0 && sp.nH <= kMaskBits && !sp.product;  // table emission (|H| <= 256)
  Buf<uint32_t> tab;
  if (nX > 0) {
    PS_TRY(fX.alloc(nX, s));
    PS_TRY(histX.alloc(nbins, s));
    PS_CUDA(cudaMemsetAsync(histX.p, 0, nbins * sizeof(uint32_t), s));
    PS_LAUNCH("k_hash_hist", s, k_hash_hist<<<hist_grid(nX), 256, 0, s>>>(sp.X, nX, bits, fX.p, histX.p));
    PS_CUDA(cudaGetLastError());
    PS_TRY(fH.alloc(sp.nH, s));
    if (use_tab) {  // the H terms and the anticommutation table in one launch
      const int words = kTabPos * kTabVals * tab_stride((sp.nH + 31) / 32);
      PS_TRY(tab.alloc((size_t)words, s));
      PS_LAUNCH("k_h_prep", s, k_h_prep_table<<<(int)ceil_div(words + sp.nH, 256), 256, 0, s>>>(
                                   sp.H, sp.nH, bits, a.uH, fH.p, hscal.p, sp.hbatch ? sp.hbatch_uniform : nullptr,
                                   tab_stride((sp.nH + 31) / 32), tab.p));
    } else {
      PS_LAUNCH("k_h_prep", s, k_h_prep<<<(int)ceil_div(sp.nH, 256), 256, 0, s>>>(sp.H, sp.nH, bits, a.uH, fH.p, hscal.p, sp.hbatch ? sp.hbatch_uniform : nullptr));
    }
    PS_CUDA(cudaGetLastError());
  }
  // the plain sources and the pre operand as one set (one launch each for their histogram and
  // their emission); translation-symmetric sources one by one
  SrcSet sset{};
  for (int i = 0; i < sp.nsrc; ++i)
    if (sp.src[i].n > 0 && !sp.src[i].ts) {
      sset.rec[sset.cnt] = sp.src[i].rec;
      sset.code[sset.cnt] = kCodeSrc + (uint32_t)i;
      sset.off[sset.cnt + 1] = sset.off[sset.cnt] + sp.src[i].n;
      ++sset.cnt;
    }
  if (sp.npre > 0) {
    sset.rec[sset.cnt] = sp.pre;
    sset.code[sset.cnt] = kCodePre;
    sset.off[sset.cnt + 1] = sset.off[sset.cnt] + sp.npre;
    ++sset.cnt;
  }
  const int64_t nset = sset.off[sset.cnt];
  for (int i = 0; i < sp.nsrc; ++i)
    if (sp.src[i].n > 0 && sp.src[i].ts) {
      PS_LAUNCH("k_hash_hist", s, k_hash_hist_ts<<<grid_for(sp.src[i].n), 256, 0, s>>>(sp.src[i].rec, sp.src[i].n, bits, sp.src[i].ts, sp.ring, histY.p));
      PS_CUDA(cudaGetLastError());
    }
  if (nset > 0) {
    PS_LAUNCH("k_hash_hist", s, k_hash_hist_set<<<hist_grid(nset), 256, 0, s>>>(sset, bits, histY.p));
    PS_CUDA(cudaGetLastError());
  }
  // bin regions from the bounds; the emission's bin cursors start at the bins' first slots
  Buf<unsigned long long> cur;
  PS_TRY(cur.alloc(nbins, s));
  {
    int nh = nX > 0 ? sp.nH : 0;
    if (small_plan) {
      PS_LAUNCH("k_bound", s, k_bound_small<<<1, kPlanThreads, 0, s>>>(nX > 0 ? histX.p : nullptr, histY.p, fH.p, nh, nbins,
                                                                         base.p, cur.p));
      PS_CUDA(cudaGetLastError());
    } else {
      int blocks = (int)std::min<int64_t>(ceil_div(nbins, 256), 4 * nsm);
      PS_LAUNCH("k_bound", s, k_bound<<<blocks, 256, 0, s>>>(nX > 0 ? histX.p : nullptr, histY.p, fH.p, nh, nbins, bound.p));
      PS_CUDA(cudaGetLastError());
      PS_TRY(scan_u64(bound.p, base.p, nbins, s));
      PS_CUDA(cudaMemcpyAsync(cur.p, base.p, nbins * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    }
  }
  if (full) PS_TRY(fent.alloc((size_t)bound_total, s));
  else PS_TRY(entries.alloc((size_t)bound_total, s));

  // ---- 2. emission
  if (use_tab) {
    // |H| <= 256: anticommutation bitmaps from the nibble table (built with the H terms)
    if (full) PS_TRY(emit_tab<true>(sp.X, fX.p, nX, sp.H, fH.p, hscal.p, sp.nH, tab.p, es, cur.p, nullptr, fent.p, counters.p, nsm, s, sp.hbatch, sp.hb_shift));
    else PS_TRY(emit_tab<false>(sp.X, fX.p, nX, sp.H, fH.p, nullptr, sp.nH, tab.p, es, cur.p, entries.p, nullptr, counters.p, nsm, s));
  } else if (nX > 0) {
    for (int h0 = 0; h0 < sp.nH; h0 += kHChunk) {
      int nh = std::min(kHChunk, sp.nH - h0);
      size_t sm = (size_t)nh * (sizeof(ulonglong2) + sizeof(uint32_t));
      auto kern = sp.product ? k_emit_products<true> : k_emit_products<false>;
      if (sm > 48 * 1024) PS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      PS_LAUNCH("k_emit_products", s, kern<<<grid_for(nX), kEmitThreads, sm, s>>>(sp.X, fX.p, nX, sp.H, fH.p, h0, nh, cur.p, entries.p, counters.p));
      PS_CUDA(cudaGetLastError());
    }
  }
  auto emit_source = [&](const Rec* y, int64_t n, uint32_t code, int ts) -> int {
    if (full)
      PS_LAUNCH("k_emit_source", s, k_emit_source<true><<<grid_for(n), 256, 0, s>>>(y, n, bits, code, es, cur.p, nullptr, fent.p, ts, sp.ring));
    else
      PS_LAUNCH("k_emit_source", s, k_emit_source<false><<<grid_for(n), 256, 0, s>>>(y, n, bits, code, es, cur.p, entries.p, nullptr, 0, 0));
    PS_CUDA(cudaGetLastError());
    return PS_OK;
  };
  for (int i = 0; i < sp.nsrc; ++i)
    if (sp.src[i].n > 0 && sp.src[i].ts) PS_TRY(emit_source(sp.src[i].rec, sp.src[i].n, kCodeSrc + i, sp.src[i].ts));
  if (nset > 0) {
    if (full)
      PS_LAUNCH("k_emit_source", s, k_emit_source_set<true><<<grid_for(nset), 256, 0, s>>>(sset, bits, es, cur.p, nullptr, fent.p));
    else
      PS_LAUNCH("k_emit_source", s, k_emit_source_set<false><<<grid_for(nset), 256, 0, s>>>(sset, bits, es, cur.p, entries.p, nullptr));
    PS_CUDA(cudaGetLastError());
  }
  if (!small_plan) {
    int blocks = (int)std::min<int64_t>(ceil_div(nbins, 256), 4 * nsm);
    PS_LAUNCH("k_bin_counts", s, k_bin_counts<<<blocks, 256, 0, s>>>(cur.p, base.p, nbins, cnt.p));
    PS_CUDA(cudaGetLastError());
  }
  unsigned long long n_prod = 0;
  PS_CUDA(cudaMemcpyAsync(&n_prod, counters.p, sizeof(n_prod), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  const int64_t total_entries = (int64_t)n_prod + nsrc_total;
  st.contributions = (int64_t)n_prod;

  // ---- 3. groups
  PS_TRY(cpre.alloc(nbins + 1, s));
  PS_TRY(gstart.alloc(nbins + 1, s));
  if (small_plan) {
    PS_TRY(heads.alloc(nbins, s));  // at most one group per bin
    PS_LAUNCH("k_group_heads", s, k_plan_small<<<1, kPlanThreads, 0, s>>>(cur.p, base.p, nbins,
                                                                          (uint64_t)(ranked_wide ? geom.quota / 2 : geom.quota),
                                                                          cpre.p, gstart.p, misc.p + 1, heads.p));
    PS_CUDA(cudaGetLastError());
  } else {
    PS_TRY(scan_u32_to_u64(cnt.p, cpre.p, nbins, s));
    PS_TRY(flag.alloc(nbins, s));
    PS_TRY(fpre.alloc(nbins + 1, s));
    int blocks = (int)std::min<int64_t>(ceil_div(nbins, 256), 4 * nsm);
    PS_LAUNCH("k_group_flags", s, k_group_flags<<<blocks, 256, 0, s>>>(cpre.p, nbins, (uint64_t)(ranked_wide ? geom.quota / 2 : geom.quota), flag.p));
    PS_CUDA(cudaGetLastError());
    PS_TRY(scan_u32_to_u64(flag.p, fpre.p, nbins, s));
    PS_LAUNCH("k_group_scatter", s, k_group_scatter<<<blocks, 256, 0, s>>>(flag.p, fpre.p, nbins, gstart.p, misc.p + 1));
    PS_CUDA(cudaGetLastError());
    PS_TRY(heads.alloc(nbins, s));  // at most one group per bin
    PS_LAUNCH("k_group_heads", s, k_group_heads<<<blocks, 256, 0, s>>>(gstart.p, cpre.p, misc.p + 1, heads.p));
    PS_CUDA(cudaGetLastError());
  }

  // ---- 4. merge into a fresh output buffer
  int64_t out_cap = std::max<int64_t>(total_entries, 1);
  Rec* outbuf = nullptr;
  PS_TRY(dev_alloc((void**)&outbuf, (size_t)out_cap * sizeof(Rec), s));
  a.H = sp.H;
  a.nH = ncode_h;
  a.X = sp.X;
  a.rot = sp.rot;
  a.twice = sp.product ? 0 : 1;
  for (int i = 0; i < sp.nsrc; ++i) {
    a.src[i] = sp.src[i].rec;
    a.alpha[i] = sp.src[i].alpha;
  }
  a.pre = sp.pre;
  a.has_post = sp.has_post ? 1 : 0;
  a.post = sp.post;
  a.bits = bits;
  a.nbins = nbins;
  a.base = base.p;
  a.cpre = cpre.p;
  a.entries = entries.p;
  a.fent = fent.p;
  a.gstart = gstart.p;
  a.heads = heads.p;
  a.ngroups = misc.p + 1;
  a.next_group = misc.p;
  a.out = outbuf;
  a.out_n = counters.p + 1;
  a.out_cap = (unsigned long long)out_cap;
  a.err = err.p;
  a.round32 = out->f32;
  a.f32c = f32c;
  a.split_groups = misc.p + 2;
  uint64_t kv, kw;
  host_key_with_hash(nbins / 2, bits, &kv, &kw);  // hash in the upper half: empty key for lower-half groups
  a.sent_lo = make_ulonglong2(kv, kw);
  a.sent_hi = make_ulonglong2(0ull, 0ull);        // hash 0: empty key for upper-half groups
  size_t sm;
  void (*kern)(MergeArgs);
  const char* kname;
  if (ranked && full && ncode_h + sp.nsrc <= 192) {  // six mask words suffice
    sm = sizeof(RankSmem<true, 6>);
    kern = k_merge_rank<true, true, 6>;
    kname = "k_merge_rank_f";
  } else if (ranked) {
    sm = structured ? sizeof(RankSmem<true, 8>) : sizeof(RankSmem<false, 8>);
    kern = full ? k_merge_rank<true, true, 8> : (structured ? k_merge_rank<true, false, 8> : k_merge_rank<false, false, 8>);
    kname = full ? "k_merge_rank_f" : (structured ? "k_merge_rank_s" : "k_merge_rank");
  } else if (chained_rank) {
    sm = sizeof(RankSmem<true, 0>);
    kern = k_merge_rank<true, false, 0>;
    kname = "k_merge_rank_c";
  } else if (ranked_wide) {
    sm = sizeof(RankSmem<false, 16>);
    kern = k_merge_rank<false, false, 16>;
    kname = "k_merge_rank_w";
  } else {
    sm = structured ? sizeof(MergeSmem<true>) : sizeof(MergeSmem<false>);
    kern = structured ? k_merge<true> : k_merge<false>;
    kname = structured ? "k_merge_s" : "k_merge";
  }
  // rank keys and the norm's exponent bound from the output stage (single-component ranked
  // merges): the caller's norm then reads 8 bytes per string instead of two passes over records
  uint64_t* okeys = nullptr;
  const bool ranked_s = structured && (ranked || chained_rank);  // a k_merge_rank<true, ...> runs
  if (sp.keys_out && sp.keys_top && ranked_s) {
    const int rk = dev_alloc((void**)&okeys, (size_t)out_cap * sizeof(uint64_t), s);
    if (rk != PS_OK) {
      dev_free(outbuf, s);
      return rk;
    }
    a.okeys = okeys;
    a.otop = sp.keys_top;
  }
  auto fail = [&](int rc) {
    if (okeys) dev_free(okeys, s);
    dev_free(outbuf, s);
    return rc;
  };
  cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per_sm = 0;
  if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMergeThreads, sm);
  if (ce != cudaSuccess) {
    set_cuda_error(ce, "merge launch setup");
    return fail(PS_ERR_CUDA);
  }
  int grid = std::max(1, per_sm) * nsm;
  PS_LAUNCH(kname, s, kern<<<grid, kMergeThreads, sm, s>>>(a));
  ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    set_cuda_error(ce, "merge launch");
    return fail(PS_ERR_CUDA);
  }
  unsigned long long hres[2];
  unsigned hmisc[3];
  int herr = 0;
  ce = cudaMemcpyAsync(hres, counters.p, sizeof(hres), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hmisc, misc.p, sizeof(hmisc), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    set_cuda_error(ce, "merge results");
    return fail(PS_ERR_CUDA);
  }
  if (herr) return fail((herr & 2) ? PS_ERR_TABLE_FULL : PS_ERR_CAPACITY);
  {
    const int ra = sum_adopt(out, outbuf, out_cap, (int64_t)hres[1]);
    if (ra != PS_OK) {
      if (okeys) dev_free(okeys, s);
      return ra;
    }
  }
  if (okeys) *sp.keys_out = okeys;
  out->cls = out_cls;
  st.merged = (int64_t)hres[1];
  st.groups = hmisc[1];
  st.split_groups = hmisc[2];
  record_merge_stats(st);
  return PS_OK;
}

}  // namespace ps

extern "C" int pauli_last_merge_stats(pauli_merge_stats* out) {
  if (!out) return PS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(ps::g_stats_mu);
  *out = ps::g_stats;
  return PS_OK;
}

namespace ps {

int ts_translates(const Rec* G, int64_t n, int ring, cudaStream_t s, Rec* out) {
  if (n == 0) return PS_OK;
  const int64_t total = n * ring;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 4 * num_sms()));
  PS_LAUNCH("k_ts_translates", s, k_ts_translates<<<blocks, 256, 0, s>>>(G, n, ring, out));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

// Autotuner: the commutator [H, O] timed (CUDA events on the output's stream, best of reps)
// with each candidate geometry; the fastest is kept for merges of that size class.
int autotune_commutator(const MergeSpec& sp, pauli_sum* out, int reps, int* best_bin, int* best_quota,
                        double* best_ms, double* default_ms) {
  static const int kBinT[] = {1024, 2048, 4096};
  static const int kQuota[] = {1024, 1536};
  cudaStream_t s = out->stream;
  cudaEvent_t e0, e1;
  PS_CUDA(cudaEventCreate(&e0));
  PS_CUDA(cudaEventCreate(&e1));
  double best = 1e300, def = 0.0;
  MergeGeom bestg{};
  int cls = -1;
  int st = PS_OK;
  for (int bt : kBinT)
    for (int q : kQuota) {
      MergeGeom g{bt, q};
      t_force = &g;
      double t = 1e300;
      for (int r = 0; r < std::max(reps, 1) + 1 && st == PS_OK; ++r) {  // the first run warms up
        cudaEventRecord(e0, s);
        st = merge_run(sp, s, out);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) t = std::min(t, (double)ms);
      }
      t_force = nullptr;
      cls = t_last_class;
      if (st != PS_OK) break;
      if (bt == 2048 && q == kGroupQuota) def = t;
      if (t < best) {
        best = t;
        bestg = g;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PS_TRY(st);
  if (cls >= 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[cls] = bestg;
    g_has_tuned[cls] = true;
  }
  if (best_bin) *best_bin = bestg.bin_target;
  if (best_quota) *best_quota = bestg.quota;
  if (best_ms) *best_ms = best;
  if (default_ms) *default_ms = def;
  return PS_OK;
}

void autotune_reset() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int c = 0; c < 64; ++c) g_has_tuned[c] = false;
  g_has_fixed = false;
}

int merge_geometry_fix(int bin_target, int quota) {
  if (bin_target < 64 || bin_target > (1 << 16) || quota < 64 || quota > 4096) return PS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_fixed = MergeGeom{bin_target, quota};
  g_has_fixed = true;
  return PS_OK;
}

}  // namespace ps
