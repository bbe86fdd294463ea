// Masks wider than one word: n_sites 65..256, each mask held in W = 2 (n_sites <= 128) or
// W = 4 (n_sites <= 256) 64-bit words (Methods: a string is a pair of bit masks of any
// length, one bit per site; word k holds sites 64k+1 .. 64k+64).
//
// The same path as the single-word engine, written for W-word keys:
//   * commutator and linear combinations (Alg. 1 with eq. eps_com): products routed to bins by
//     a GF(2)-linear hash of the W-word key (F(h ^ x) = F(h) ^ F(x)), 8-byte entries (operand
//     index, order code), then one block per group of bins merges its entries in shared
//     memory: a table of entry indices (full-key compare), a count and scatter per output
//     string, and a sequential fold of each string's contributions in order-code order (H
//     order, then the sources in formula order) - the summation order of Alg. 1 with H in the
//     outer loop, so results are bit-identical to the oracle's;
//   * truncation (dissipation, weight, cutoff, top-k with key ties, keep set): a filter pass
//     and a most-significant-digit radix select over the (1 + 2W)-word rank key
//     (|c|^2 bits, ~v, ~w);
//   * exact norms and trace products (integer windows, exactly rounded);
//   * RK4 and Lanczos steps composed from these in the single-word steps' order.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "exact_sum.cuh"

namespace ps {
namespace wide {

using namespace exact;

template <int W>
struct __align__(16) RecW {
  uint64_t v[W];
  uint64_t w[W];
  double re, im;
};
static_assert(sizeof(RecW<2>) == 48 && sizeof(RecW<4>) == 80, "wide record layout");

template <int W>
struct KeyW {
  uint64_t v[W];
  uint64_t w[W];
};

constexpr int kMaxW = 4;
constexpr int kRows = 32;  // hash rows

__constant__ uint64_t c_wA[kMaxW][kRows];
__constant__ uint64_t c_wB[kMaxW][kRows];

static uint64_t splitmix(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int upload_rows() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    uint64_t a[kMaxW][kRows], b[kMaxW][kRows];
    uint64_t s = 0x3A1D5EED24109654ull;
    for (int k = 0; k < kMaxW; ++k)
      for (int j = 0; j < kRows; ++j) {
        a[k][j] = splitmix(s);
        b[k][j] = splitmix(s);
      }
    err = cudaMemcpyToSymbol(c_wA, a, sizeof(a));
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(c_wB, b, sizeof(b));
  });
  if (err != cudaSuccess) {
    set_cuda_error(err, "cudaMemcpyToSymbol(wide hash rows)");
    return PS_ERR_CUDA;
  }
  return PS_OK;
}

// ----------------------------------------------------------------------------- key algebra
template <int W>
__device__ __forceinline__ KeyW<W> key_of(const RecW<W>& r) {
  KeyW<W> k;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    k.v[i] = r.v[i];
    k.w[i] = r.w[i];
  }
  return k;
}

template <int W>
__device__ __forceinline__ bool key_eq(const KeyW<W>& a, const KeyW<W>& b) {
  bool e = true;
#pragma unroll
  for (int i = 0; i < W; ++i) e = e && a.v[i] == b.v[i] && a.w[i] == b.w[i];
  return e;
}

template <int W>
__device__ __forceinline__ KeyW<W> key_xor(const KeyW<W>& a, const KeyW<W>& b) {
  KeyW<W> c;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    c.v[i] = a.v[i] ^ b.v[i];
    c.w[i] = a.w[i] ^ b.w[i];
  }
  return c;
}

// Rows [lo, lo + bits) of the output hash: bit j is the parity of the key ANDed with row j.
template <int W>
__device__ __forceinline__ uint32_t whash(const KeyW<W>& k, int lo, int bits) {
  uint32_t f = 0;
  for (int j = 0; j < bits; ++j) {
    uint64_t t = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) t ^= (k.v[i] & c_wA[i][lo + j]) ^ (k.w[i] & c_wB[i][lo + j]);
    f |= (uint32_t)(__popcll(t) & 1) << j;
  }
  return f;
}

// a and b anticommute iff the popcounts of w_a & v_b and v_a & w_b add up to an odd number
// (eq. eps_com), over all words.
template <int W>
__device__ __forceinline__ bool w_anti(const KeyW<W>& a, const KeyW<W>& b) {
  uint64_t t = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) t ^= (a.w[i] & b.v[i]) ^ (a.v[i] & b.w[i]);
  return (__popcll(t) & 1) != 0;
}

// P_a P_b = i^k P_{a^b}, k = pop(vc & wc) - pop(va & wa) - pop(vb & wb) + 2 pop(wa & vb) mod 4.
template <int W>
__device__ __forceinline__ int w_phase(const KeyW<W>& a, const KeyW<W>& b) {
  int k = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const uint64_t vc = a.v[i] ^ b.v[i], wc = a.w[i] ^ b.w[i];
    k += __popcll(vc & wc) - __popcll(a.v[i] & a.w[i]) - __popcll(b.v[i] & b.w[i]) + 2 * __popcll(a.w[i] & b.v[i]);
  }
  return k & 3;
}

template <int W>
__device__ __forceinline__ int w_weight(const KeyW<W>& k) {
  int c = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) c += __popcll(k.v[i] | k.w[i]);
  return c;
}

template <int W>
__device__ __forceinline__ uint32_t thash(const KeyW<W>& k) {
  uint64_t h = 0x2545F4914F6CDD1Dull;  // every word through the full-avalanche finaliser
#pragma unroll
  for (int i = 0; i < W; ++i) h = fmix64(fmix64(h ^ k.v[i]) ^ k.w[i]);
  return (uint32_t)h;
}

// Canonical order of keys: v as a W-word unsigned integer (most significant word last in
// memory), then w the same way.
template <int W>
__host__ __device__ __forceinline__ bool rec_less(const RecW<W>& a, const RecW<W>& b) {
  for (int i = W - 1; i >= 0; --i)
    if (a.v[i] != b.v[i]) return a.v[i] < b.v[i];
  for (int i = W - 1; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return false;
}

template <int W>
RecW<W>* recs(const pauli_sum* s) { return reinterpret_cast<RecW<W>*>(s->d); }

// ----------------------------------------------------------------------------- block helpers
constexpr int kBT = 256;  // threads of the streaming kernels

// One output reservation per block for flagged items (order unspecified): returns the
// position of this thread's item, valid when flag is set.
__device__ __forceinline__ unsigned long long block_reserve(bool flag, unsigned long long* counter) {
  __shared__ unsigned s_wc[kBT / 32];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) s_wc[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int k = 0; k < kBT / 32; ++k) {
      const unsigned c = s_wc[k];
      s_wc[k] = run;
      run += c;
    }
    s_base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
  }
  __syncthreads();
  const unsigned long long pos = s_base + s_wc[warp] + __popc(m & ((1u << lane) - 1u));
  __syncthreads();
  return pos;
}

// ----------------------------------------------------------------------------- upload / download
// Records from row-major word arrays (string i: words v[i*W .. i*W+W)); flags: [0] key bits at
// or above n_sites or a non-finite coefficient, [1] coefficient class.
template <int W>
__global__ void k_wpack(RecW<W>* __restrict__ d, const uint64_t* __restrict__ v, const uint64_t* __restrict__ w,
                        const double* __restrict__ re, const double* __restrict__ im, int64_t n, int n_sites,
                        int* __restrict__ flags) {
  int bad = 0, c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    RecW<W> r;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      r.v[k] = v[i * W + k];
      r.w[k] = w[i * W + k];
      const int lo = 64 * k;
      const uint64_t valid = n_sites >= lo + 64 ? ~0ull : (n_sites <= lo ? 0ull : ((1ull << (n_sites - lo)) - 1ull));
      bad |= ((r.v[k] | r.w[k]) & ~valid) != 0;
    }
    r.re = re[i];
    r.im = im[i];
    d[i] = r;
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

// Insert record i into an index table (-1 empty) keyed by its full key; `dup` set when the key
// is already present.  Probing is bounded by the table size.
template <int W>
__device__ __forceinline__ void index_insert(const RecW<W>* d, int64_t i, long long* tab, uint64_t tmask, int* dup) {
  const KeyW<W> k = key_of(d[i]);
  uint64_t slot = thash(k) & tmask;
  for (uint64_t p = 0; p <= tmask; ++p) {
    const long long old = atomicCAS((unsigned long long*)&tab[slot], ~0ull, (unsigned long long)i);
    if (old == -1) return;
    if (key_eq(key_of(d[old]), k)) {
      atomicOr(dup, 1);
      return;
    }
    slot = (slot + 1) & tmask;
  }
  atomicOr(dup, 2);  // table full (cannot happen at load <= 1/2)
}

template <int W>
__global__ void k_wdistinct(const RecW<W>* __restrict__ d, int64_t n, long long* tab, uint64_t tmask, int* dup) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    index_insert(d, i, tab, tmask, dup);
}

// Index of the record of `tab` (built over T) whose key equals k, or -1.
template <int W>
__device__ __forceinline__ int64_t index_find(const RecW<W>* T, const long long* tab, uint64_t tmask, const KeyW<W>& k) {
  uint64_t slot = thash(k) & tmask;
  for (uint64_t p = 0; p <= tmask; ++p) {
    const long long j = tab[slot];
    if (j < 0) return -1;
    if (key_eq(key_of(T[j]), k)) return j;
    slot = (slot + 1) & tmask;
  }
  return -1;
}

template <int W>
__global__ void k_wunpack(const RecW<W>* __restrict__ d, int64_t n, uint64_t* __restrict__ v, uint64_t* __restrict__ w,
                          double* __restrict__ re, double* __restrict__ im) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const RecW<W> r = d[i];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      v[i * W + k] = r.v[k];
      w[i * W + k] = r.w[k];
    }
    re[i] = r.re;
    im[i] = r.im;
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kBT), 8 * num_sms())); }

template <int W>
int upload_t(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re, const double* im, int64_t n,
             bool host) {
  PS_TRY(sum_reserve(s, n, false));
  s->n = 0;
  Buf<int> flags;
  Buf<uint64_t> stage;
  Buf<long long> tab;
  PS_TRY(flags.alloc(3, s->stream));
  PS_CUDA(cudaMemsetAsync(flags.p, 0, 3 * sizeof(int), s->stream));
  if (n > 0) {
    const uint64_t *dv = v, *dw = w;
    const double *dre = re, *dim = im;
    if (host) {
      PS_TRY(stage.alloc((size_t)n * (2 * W + 2), s->stream));
      uint64_t* sv = stage.p;
      uint64_t* sw = stage.p + (size_t)n * W;
      double* sre = reinterpret_cast<double*>(stage.p + (size_t)2 * n * W);
      double* sim = sre + n;
      PS_CUDA(cudaMemcpyAsync(sv, v, (size_t)n * W * 8, cudaMemcpyHostToDevice, s->stream));
      PS_CUDA(cudaMemcpyAsync(sw, w, (size_t)n * W * 8, cudaMemcpyHostToDevice, s->stream));
      PS_CUDA(cudaMemcpyAsync(sre, re, (size_t)n * 8, cudaMemcpyHostToDevice, s->stream));
      PS_CUDA(cudaMemcpyAsync(sim, im, (size_t)n * 8, cudaMemcpyHostToDevice, s->stream));
      dv = sv;
      dw = sw;
      dre = sre;
      dim = sim;
    }
    PS_LAUNCH("k_wpack", s->stream, k_wpack<W><<<grid_for(n), kBT, 0, s->stream>>>(recs<W>(s), dv, dw, dre, dim, n, s->n_sites, flags.p));
    PS_CUDA(cudaGetLastError());
    if (host && n > 1) {  // distinctness (device uploads leave it to the caller)
      uint64_t slots = 1;
      while (slots < (uint64_t)(2 * n)) slots <<= 1;
      PS_TRY(tab.alloc(slots, s->stream));
      PS_CUDA(cudaMemsetAsync(tab.p, 0xFF, slots * sizeof(long long), s->stream));
      PS_LAUNCH("k_wdistinct", s->stream, k_wdistinct<W><<<grid_for(n), kBT, 0, s->stream>>>(recs<W>(s), n, tab.p, slots - 1, flags.p + 2));
      PS_CUDA(cudaGetLastError());
    }
  }
  int h[3] = {0, 0, 0};
  PS_CUDA(cudaMemcpyAsync(h, flags.p, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  PS_CUDA(cudaStreamSynchronize(s->stream));
  if (h[0] || h[2]) return PS_ERR_INVALID;
  s->cls = h[1];
  s->n = n;
  return PS_OK;
}

template <int W>
int download_t(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im) {
  std::vector<RecW<W>> h((size_t)s->n);
  PS_CUDA(cudaMemcpyAsync(h.data(), s->d, (size_t)s->n * sizeof(RecW<W>), cudaMemcpyDeviceToHost, s->stream));
  PS_CUDA(cudaStreamSynchronize(s->stream));
  std::sort(h.begin(), h.end(), [](const RecW<W>& x, const RecW<W>& y) { return rec_less(x, y); });
  for (int64_t i = 0; i < s->n; ++i) {
    const RecW<W>& r = h[(size_t)i];
    for (int k = 0; k < W; ++k) {
      v[i * W + k] = r.v[k];
      w[i * W + k] = r.w[k];
    }
    re[i] = r.re;
    im[i] = r.im;
  }
  return PS_OK;
}

// ----------------------------------------------------------------------------- exact reductions
template <int W>
__global__ void k_wnorm_top(const RecW<W>* __restrict__ d, int64_t n, int* top) {
  int m = -100000;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double re = d[i].re, im = d[i].im;
    m = max(m, max(prod_top(re, re), prod_top(im, im)));
    m = max(m, max(nonfinite_top(re), nonfinite_top(im)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(top, m);
}

template <int W>
__global__ void __launch_bounds__(kRedThreads) k_wnorm_acc(const RecW<W>* __restrict__ d, int64_t n, const int* top,
                                                           long long* gwin, long long* full, int* wlo_out) {
  const int t = *top;
  if (t <= -100000 || t >= kTopInf) return;
  const int wlo = ((t - 190 + kBias) & ~31) - kBias;
  if (blockIdx.x == 0 && threadIdx.x == 0) *wlo_out = wlo;
  Win acc{{0, 0, 0, 0}};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double re = d[i].re, im = d[i].im;
    add_product(acc, re, re, wlo, full);
    add_product(acc, im, im, wlo, full);
  }
  block_flush(acc, gwin);
}

template <int W>
int norm2_t(const pauli_sum* s, double* out) {
  *out = 0.0;
  if (s->n == 0) return PS_OK;
  cudaStream_t st = s->stream;
  Buf<long long> acc;
  Buf<int> ints;
  PS_TRY(acc.alloc(kWinDigits + kFullDigits, st));
  PS_TRY(ints.alloc(2, st));
  PS_CUDA(cudaMemsetAsync(acc.p, 0, (kWinDigits + kFullDigits) * sizeof(long long), st));
  PS_CUDA(cudaMemsetAsync(ints.p, 0x80, 2 * sizeof(int), st));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(s->n, kRedThreads), 4 * num_sms()));
  PS_LAUNCH("k_wnorm_top", st, k_wnorm_top<W><<<blocks, kRedThreads, 0, st>>>(recs<W>(s), s->n, ints.p));
  PS_LAUNCH("k_wnorm_acc", st, k_wnorm_acc<W><<<blocks, kRedThreads, 0, st>>>(recs<W>(s), s->n, ints.p, acc.p, acc.p + kWinDigits, ints.p + 1));
  PS_CUDA(cudaGetLastError());
  std::vector<long long> h(kWinDigits + kFullDigits);
  int hi[2];
  PS_CUDA(cudaMemcpyAsync(h.data(), acc.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaMemcpyAsync(hi, ints.p, sizeof(hi), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  if (hi[0] <= -100000) return PS_OK;
  if (hi[0] >= kTopInf) {
    *out = hi[0] == kTopNaN ? std::nan("") : HUGE_VAL;
    return PS_OK;
  }
  std::vector<long long> full(h.begin() + kWinDigits, h.end());
  *out = round_exact(full, h.data(), hi[1]);
  return PS_OK;
}

template <int W>
__global__ void k_wtp_build(const RecW<W>* __restrict__ T, int64_t n, long long* tab, uint64_t tmask, int* dup) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    index_insert(T, i, tab, tmask, dup);
}

template <int W>
__global__ void k_wtp_top(const RecW<W>* __restrict__ P, int64_t n, const RecW<W>* __restrict__ T, const long long* tab,
                          uint64_t tmask, int* top) {
  int m = -100000;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const RecW<W> a = P[i];
    const int64_t j = index_find(T, tab, tmask, key_of(a));
    if (j < 0) continue;
    const double br = T[j].re, bi = T[j].im;
    m = max(m, max(max(prod_top(a.re, br), prod_top(a.im, bi)), max(prod_top(a.re, bi), prod_top(a.im, br))));
    if (nonfinite_top(a.re) > 0 || nonfinite_top(a.im) > 0 || nonfinite_top(br) > 0 || nonfinite_top(bi) > 0) m = kTopNaN;
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(top, m);
}

template <int W>
__global__ void __launch_bounds__(kRedThreads) k_wtp_acc(const RecW<W>* __restrict__ P, int64_t n,
                                                         const RecW<W>* __restrict__ T, const long long* tab,
                                                         uint64_t tmask, const int* top, long long* acc, int span,
                                                         int* wlo_out) {
  const int t = *top;
  if (t <= -100000 || t >= kTopInf) return;
  const int wlo = ((t - 190 + kBias) & ~31) - kBias;
  if (blockIdx.x == 0 && threadIdx.x == 0) *wlo_out = wlo;
  Win ar{{0, 0, 0, 0}}, ai{{0, 0, 0, 0}};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const RecW<W> a = P[i];
    const int64_t j = index_find(T, tab, tmask, key_of(a));
    if (j < 0) continue;
    const double br = T[j].re, bi = T[j].im;
    add_product(ar, a.re, br, wlo, acc + kWinDigits);
    add_product(ar, -a.im, bi, wlo, acc + kWinDigits);
    add_product(ai, a.re, bi, wlo, acc + span + kWinDigits);
    add_product(ai, a.im, br, wlo, acc + span + kWinDigits);
  }
  block_flush(ar, acc);
  __syncthreads();
  block_flush(ai, acc + span);
}

template <int W>
int trace_t(const pauli_sum* A, const pauli_sum* B, double* re, double* im) {
  *re = *im = 0.0;
  if (A->n == 0 || B->n == 0) return PS_OK;
  cudaStream_t st = A->stream;
  const bool swap = B->n > A->n;
  const pauli_sum* P = swap ? B : A;  // probed
  const pauli_sum* T = swap ? A : B;  // tabled (smaller)
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * T->n)) slots <<= 1;
  const int span = kWinDigits + kFullDigits;
  Buf<long long> tab, acc;
  Buf<int> ints;
  PS_TRY(tab.alloc(slots, st));
  PS_TRY(acc.alloc(2 * span, st));
  PS_TRY(ints.alloc(3, st));
  PS_CUDA(cudaMemsetAsync(tab.p, 0xFF, slots * sizeof(long long), st));
  PS_CUDA(cudaMemsetAsync(acc.p, 0, 2 * span * sizeof(long long), st));
  PS_CUDA(cudaMemsetAsync(ints.p, 0x80, 2 * sizeof(int), st));
  PS_CUDA(cudaMemsetAsync(ints.p + 2, 0, sizeof(int), st));
  PS_LAUNCH("k_wtp_build", st, k_wtp_build<W><<<grid_for(T->n), kBT, 0, st>>>(recs<W>(T), T->n, tab.p, slots - 1, ints.p + 2));
  const int bp = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(P->n, kRedThreads), 4 * num_sms()));
  PS_LAUNCH("k_wtp_top", st, k_wtp_top<W><<<bp, kRedThreads, 0, st>>>(recs<W>(P), P->n, recs<W>(T), tab.p, slots - 1, ints.p));
  PS_LAUNCH("k_wtp_acc", st, k_wtp_acc<W><<<bp, kRedThreads, 0, st>>>(recs<W>(P), P->n, recs<W>(T), tab.p, slots - 1, ints.p, acc.p, span, ints.p + 1));
  PS_CUDA(cudaGetLastError());
  std::vector<long long> h(2 * span);
  int hi[3];
  PS_CUDA(cudaMemcpyAsync(h.data(), acc.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaMemcpyAsync(hi, ints.p, sizeof(hi), cudaMemcpyDeviceToHost, st));
  PS_CUDA(cudaStreamSynchronize(st));
  if (hi[0] <= -100000) return PS_OK;
  if (hi[0] >= kTopInf) {
    *re = *im = std::nan("");
    return PS_OK;
  }
  std::vector<long long> fre(h.begin() + kWinDigits, h.begin() + span);
  std::vector<long long> fim(h.begin() + span + kWinDigits, h.end());
  *re = round_exact(fre, h.data(), hi[1]);
  *im = round_exact(fim, h.data() + span, hi[1]);
  return PS_OK;
}

// ----------------------------------------------------------------------------- merge engine
// For every output string c: acc(c) = sequential sum, in order, of the products
// 2 i^(k + rot) h x for each H term h (H order) with x in X, h ^ x = c, anticommuting; then
// alpha_s y_s(c) for each extra source s in order.  out(c) = acc(c), or pre(c) + post acc(c)
// with a post factor (absent terms are zero).  Exact zeros are dropped.
constexpr uint32_t kCodeSrc = 0xF000u;
constexpr uint32_t kCodePre = 0xFFFFu;
constexpr int kMaxHW = 0xEFFF;
constexpr int kHChunkW = 256;       // H terms staged per emission block
constexpr int kWE = 1024;           // entries per merge pass
constexpr int kWT = 2048;           // table slots per merge pass
constexpr int kWThreads = 256;
constexpr int kWMaxProbe = 64;
constexpr int kWQuota = 512;        // a new group starts when the running count crosses a multiple
constexpr int kWMaxGroupBins = 256;
constexpr uint16_t kNil = 0xFFFFu;

template <int W>
struct WSpec {
  const RecW<W>* H = nullptr;
  int nH = 0;
  const RecW<W>* X = nullptr;
  int64_t nX = 0;
  int rot = 0;
  const RecW<W>* src[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t nsrc_n[4] = {0, 0, 0, 0};
  Cx alpha[4];
  int nsrc = 0;
  const RecW<W>* pre = nullptr;
  int64_t npre = 0;
  int has_post = 0;
  Cx post{1.0, 0.0};
};

// Bin cursor reservation: lanes with the same bin share one atomic.
__device__ __forceinline__ uint64_t reserve(unsigned long long* cur, uint32_t p, bool act) {
  const int lane = threadIdx.x & 31;
  const unsigned mm = __match_any_sync(0xffffffffu, act ? p : 0xFFFFFFFFu);
  const int leader = __ffs(mm) - 1;
  unsigned long long b = 0;
  if (act && lane == leader) b = atomicAdd(&cur[p], (unsigned long long)__popc(mm));
  b = __shfl_sync(0xffffffffu, b, leader);
  return b + (uint32_t)__popc(mm & ((1u << lane) - 1u));
}

template <int W>
__global__ void k_whash_hist(const RecW<W>* __restrict__ r, int64_t n, int bits, uint32_t* __restrict__ f,
                             uint32_t* __restrict__ hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = whash(key_of(r[i]), 0, bits);
    if (f) f[i] = h;
    atomicAdd(&hist[h], 1u);
  }
}

__global__ void k_wbound(const uint32_t* __restrict__ histX, const uint32_t* __restrict__ histY,
                         const uint32_t* __restrict__ fH, int nH, uint32_t nbins, uint64_t* __restrict__ bound) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x) {
    uint64_t b = histY[p];
    if (histX)
      for (int h = 0; h < nH; ++h) b += histX[p ^ __ldg(&fH[h])];
    bound[p] = b;
  }
}

// Products: a warp holds 32 x and walks the H terms of the block's chunk; every anticommuting
// (h, x) appends the entry (x index << 16 | h) to bin F(h) ^ F(x).
template <int W>
__global__ void __launch_bounds__(kBT) k_wemit(const RecW<W>* __restrict__ X, const uint32_t* __restrict__ fX,
                                               int64_t nX, const RecW<W>* __restrict__ H,
                                               const uint32_t* __restrict__ fH, int h0, int nh,
                                               unsigned long long* __restrict__ cur, uint64_t* __restrict__ entries,
                                               unsigned long long* __restrict__ total) {
  __shared__ KeyW<W> s_h[kHChunkW];
  __shared__ uint32_t s_f[kHChunkW];
  for (int i = threadIdx.x; i < nh; i += blockDim.x) {
    s_h[i] = key_of(H[h0 + i]);
    s_f[i] = fH[h0 + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  unsigned long long emitted = 0;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t0 = wid * 32; t0 < nX; t0 += nw * 32) {
    const int64_t i = t0 + lane;
    const bool valid = i < nX;
    KeyW<W> xk;
    uint32_t fx = 0;
    if (valid) {
      xk = key_of(X[i]);
      fx = fX[i];
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) xk.v[k] = xk.w[k] = 0;
    }
    for (int h = 0; h < nh; ++h) {
      const bool anti = valid && w_anti(s_h[h], xk);
      if (!__ballot_sync(0xffffffffu, anti)) continue;
      const uint32_t p = fx ^ s_f[h];
      const uint64_t at = reserve(cur, p, anti);
      if (anti) {
        entries[at] = ((uint64_t)i << 16) | (uint64_t)(h0 + h);
        ++emitted;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) emitted += __shfl_down_sync(0xffffffffu, emitted, o);
  if (lane == 0 && emitted) atomicAdd(total, emitted);
}

template <int W>
__global__ void k_wemit_src(const RecW<W>* __restrict__ Y, int64_t n, int bits, uint32_t code,
                            unsigned long long* __restrict__ cur, uint64_t* __restrict__ entries) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    const bool act = i < n;
    uint32_t p = 0;
    if (act) p = whash(key_of(Y[i]), 0, bits);
    const uint64_t at = reserve(cur, p, act);
    if (act) entries[at] = ((uint64_t)i << 16) | (uint64_t)code;
  }
}

__global__ void k_wcounts(const unsigned long long* __restrict__ cur, const uint64_t* __restrict__ base, uint32_t nbins,
                          uint32_t* __restrict__ cnt) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x)
    cnt[p] = (uint32_t)(cur[p] - base[p]);
}

// Group starts: bin 0, every kWMaxGroupBins bins, and where the running entry count crosses a
// multiple of the quota.
__global__ void k_wgroup_flags(const uint64_t* __restrict__ cpre, uint32_t nbins, uint32_t* __restrict__ flag) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x)
    flag[p] = (p == 0 || (p % kWMaxGroupBins) == 0 || cpre[p] / kWQuota != cpre[p - 1] / kWQuota) ? 1u : 0u;
}

__global__ void k_wgroup_scatter(const uint32_t* __restrict__ flag, const uint64_t* __restrict__ fpre, uint32_t nbins,
                                 uint32_t* __restrict__ gstart) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nbins; p += gridDim.x * blockDim.x)
    if (flag[p]) gstart[fpre[p]] = p;
  if (blockIdx.x == 0 && threadIdx.x == 0) gstart[fpre[nbins]] = nbins;
}

template <int W>
struct WMergeArgs {
  const RecW<W>* H;
  int nH;
  const RecW<W>* X;
  int rot;
  const RecW<W>* src[4];
  Cx alpha[4];
  const RecW<W>* pre;
  int has_post;
  Cx post;
  int bits;
  const uint64_t* base;
  const uint64_t* cpre;
  const uint64_t* entries;
  const uint32_t* gstart;
  uint32_t ngroups;
  unsigned* next_group;
  RecW<W>* out;
  unsigned long long* out_n;
  unsigned long long out_cap;
  int* err;  // bit 0: output capacity, bit 1: unresolved overflow
};


template <int W>
struct WSmem {
  KeyW<W> key[kWE];
  Cx val[kWE];
  uint16_t code[kWE];     // order: H index, then nH + source; kNil (last) for the pre operand
  uint16_t slot[kWE];
  uint16_t seg[kWE];      // entries grouped by output string
  uint16_t ulist[kWE];    // occupied slots, one per distinct output string
  uint16_t oent[kWE];     // staged outputs: the entry holding the key, and the value
  Cx oval[kWE];
  int32_t tab[kWT];       // entry owning the slot, or -1
  uint32_t cnt[kWT];      // entries per slot
  uint32_t start[kWT];    // segment start per slot (advanced by the scatter)
  uint64_t gbase[kWMaxGroupBins];
  uint32_t gpre[kWMaxGroupBins + 1];
  uint32_t wsum[kWThreads / 32];
  uint32_t n_e, n_u, n_out;
  int flags;
  unsigned group;
  unsigned long long out_base;
};

// Key, contribution and order code of an entry: for a product (code = H index) the string
// h ^ x with 2 i^(k + rot) (h x); for a source, alpha_s y; for the pre operand, y itself.
template <int W>
__device__ __forceinline__ void build_entry(const WMergeArgs<W>& a, uint64_t ent, KeyW<W>& key, Cx& t, uint16_t& ord) {
  const uint32_t code = (uint32_t)(ent & 0xFFFFu);
  const uint64_t idx = ent >> 16;
  if (code < kCodeSrc) {
    const RecW<W> x = a.X[idx];
    const RecW<W> h = a.H[code];
    const KeyW<W> hk = key_of(h), xk = key_of(x);
    key = key_xor(hk, xk);
    const int k = w_phase(hk, xk) + a.rot;
    const Cx p = cmul(Cx{h.re, h.im}, Cx{x.re, x.im});
    t = rot(Cx{twice(p.re), twice(p.im)}, k);
    ord = (uint16_t)code;
  } else if (code == kCodePre) {
    const RecW<W> y = a.pre[idx];
    key = key_of(y);
    t = Cx{y.re, y.im};
    ord = kNil;
  } else {
    const uint32_t si = code - kCodeSrc;
    const RecW<W> y = a.src[si][idx];
    key = key_of(y);
    t = cmul(a.alpha[si], Cx{y.re, y.im});
    ord = (uint16_t)(a.nH + (int)si);
  }
}

// Exclusive scan of cnt[ulist[u]] over u < n_u (n_u <= kWE) into start[ulist[u]].
template <int W>
__device__ __forceinline__ void scan_slots(WSmem<W>& s, uint32_t n_u) {
  constexpr int kPer = kWE / kWThreads;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t c[kPer], tot = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const uint32_t u = tid * kPer + k;
    c[k] = u < n_u ? s.cnt[s.ulist[u]] : 0u;
    tot += c[k];
  }
  uint32_t incl = tot;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s.wsum[warp] = incl;
  __syncthreads();
  uint32_t run = incl - tot;
  for (int k = 0; k < warp; ++k) run += s.wsum[k];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const uint32_t u = tid * kPer + k;
    if (u < n_u) s.start[s.ulist[u]] = run;
    run += c[k];
  }
}

template <int W>
__global__ void __launch_bounds__(kWThreads) k_wmerge(WMergeArgs<W> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WSmem<W>& s = *reinterpret_cast<WSmem<W>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < kWT; i += kWThreads) {
    s.tab[i] = -1;
    s.cnt[i] = 0;
  }
  if (tid == 0) {
    s.n_e = s.n_u = s.n_out = 0;
    s.flags = 0;
  }
  for (;;) {
    __syncthreads();
    if (tid == 0) s.group = atomicAdd(a.next_group, 1u);
    __syncthreads();
    const uint32_t g = s.group;
    if (g >= a.ngroups) break;
    const uint32_t lo = a.gstart[g], hi = a.gstart[g + 1];
    const uint32_t nb = hi - lo;
    const uint64_t e0 = a.cpre[lo];
    const uint64_t E = a.cpre[hi] - e0;
    if (E == 0) continue;
    if (nb > (uint32_t)kWMaxGroupBins) {
      if (tid == 0) atomicOr(a.err, 2);
      continue;
    }
    for (uint32_t i = tid; i <= nb; i += kWThreads) s.gpre[i] = (uint32_t)(a.cpre[lo + i] - e0);
    for (uint32_t i = tid; i < nb; i += kWThreads) s.gbase[i] = a.base[lo + i];
    __syncthreads();
    int level0 = 0;
    while (((uint64_t)kWE << level0) < E && level0 < 16) ++level0;
    if (a.bits + level0 > kRows) {
      if (tid == 0) atomicOr(a.err, 2);
      continue;
    }
    constexpr int kStack = 2 * kRows + 2;
    for (uint32_t sub0 = 0; sub0 < (1u << level0); ++sub0) {
      int stk_level[kStack];
      uint32_t stk_sub[kStack];
      int sp = 1;
      stk_level[0] = level0;
      stk_sub[0] = sub0;
      while (sp > 0) {
        --sp;
        const int level = stk_level[sp];
        const uint32_t sub = stk_sub[sp];
        // ---- phase 1: the pass's entries (those whose next hash bits equal sub)
        for (uint64_t j0 = 0; j0 < E; j0 += kWThreads) {
          const uint64_t j = j0 + tid;
          bool keep = j < E;
          KeyW<W> key;
          Cx t{0.0, 0.0};
          uint16_t ord = 0;
          if (keep) {
            uint32_t l = 0, r = nb;
            while (r - l > 1) {
              const uint32_t m = (l + r) >> 1;
              if (s.gpre[m] <= j) l = m; else r = m;
            }
            build_entry(a, a.entries[s.gbase[l] + (j - s.gpre[l])], key, t, ord);
            if (level > 0) keep = whash(key, a.bits, level) == sub;
          }
          const unsigned m = __ballot_sync(0xffffffffu, keep);
          if (!m) continue;
          const int leader = __ffs(m) - 1;
          uint32_t eb = 0;
          if (lane == leader) eb = atomicAdd(&s.n_e, (uint32_t)__popc(m));
          eb = __shfl_sync(0xffffffffu, eb, leader);
          const uint32_t e = eb + __popc(m & ((1u << lane) - 1u));
          if (keep) {
            if (e < (uint32_t)kWE) {
              s.key[e] = key;
              s.val[e] = t;
              s.code[e] = ord;
            } else {
              atomicOr(&s.flags, 1);
            }
          }
        }
        __syncthreads();
        const uint32_t n_e = min(s.n_e, (uint32_t)kWE);
        // ---- phase 2: one slot per distinct key (full-key compare with the slot's owner)
        if (!s.flags) {
          for (uint32_t e = tid; e < n_e; e += kWThreads) {
            const KeyW<W> k = s.key[e];
            uint32_t slot = thash(k) & (kWT - 1);
            int found = -1;
            for (int p = 0; p < kWMaxProbe; ++p) {
              int cur = s.tab[slot];
              if (cur < 0) {
                cur = atomicCAS(&s.tab[slot], -1, (int)e);
                if (cur < 0) {
                  found = (int)slot;
                  s.ulist[atomicAdd(&s.n_u, 1u)] = (uint16_t)slot;
                  break;
                }
              }
              if (key_eq(s.key[cur], k)) {
                found = (int)slot;
                break;
              }
              slot = (slot + 1) & (kWT - 1);
            }
            if (found < 0) {
              atomicOr(&s.flags, 1);
            } else {
              s.slot[e] = (uint16_t)found;
              atomicAdd(&s.cnt[found], 1u);
            }
          }
        }
        __syncthreads();
        const uint32_t n_u = s.n_u;
        if (s.flags) {  // split the pass by the next hash bit, or give up
          for (uint32_t u = tid; u < n_u; u += kWThreads) {
            s.tab[s.ulist[u]] = -1;
            s.cnt[s.ulist[u]] = 0;
          }
          __syncthreads();
          if (tid == 0) {
            s.n_e = s.n_u = 0;
            s.flags = 0;
          }
          __syncthreads();
          if (level >= 16 || a.bits + level + 1 > kRows || sp + 2 > kStack) {
            if (tid == 0) atomicOr(a.err, 2);
            continue;
          }
          stk_level[sp] = level + 1;
          stk_sub[sp] = sub + (1u << level);
          stk_level[sp + 1] = level + 1;
          stk_sub[sp + 1] = sub;
          sp += 2;
          continue;
        }
        // ---- phase 3: segment starts; phase 4: entries into their string's segment
        scan_slots(s, n_u);
        __syncthreads();
        for (uint32_t e = tid; e < n_e; e += kWThreads) s.seg[atomicAdd(&s.start[s.slot[e]], 1u)] = (uint16_t)e;
        __syncthreads();
        // ---- phase 5: per string, its contributions in order-code order, folded in order
        for (uint32_t u = tid; u < n_u; u += kWThreads) {
          const uint32_t slot = s.ulist[u];
          const uint32_t c = s.cnt[slot];
          const uint32_t b0 = s.start[slot] - c;
          for (uint32_t i = b0 + 1; i < b0 + c; ++i) {  // insertion sort by order code
            const uint16_t x = s.seg[i];
            const uint16_t kx = s.code[x];
            uint32_t j = i;
            while (j > b0 && s.code[s.seg[j - 1]] > kx) {
              s.seg[j] = s.seg[j - 1];
              --j;
            }
            s.seg[j] = x;
          }
          uint32_t n = c;
          int pe = -1;
          if (s.code[s.seg[b0 + c - 1]] == kNil) {  // the pre operand sorts last
            pe = s.seg[b0 + c - 1];
            --n;
          }
          Cx acc{0.0, 0.0};
          if (n > 0) acc = s.val[s.seg[b0]];
          for (uint32_t i = 1; i < n; ++i) {
            const Cx y = s.val[s.seg[b0 + i]];
            acc.re = __dadd_rn(acc.re, y.re);
            acc.im = __dadd_rn(acc.im, y.im);
          }
          Cx r = acc;
          if (a.has_post) {
            const Cx sc = n > 0 ? cmul(a.post, acc) : Cx{0.0, 0.0};
            if (pe >= 0) {
              const Cx pv = s.val[pe];
              r = n > 0 ? Cx{add_rn(pv.re, sc.re), add_rn(pv.im, sc.im)} : pv;
            } else {
              r = sc;
            }
          }
          if (!(is_zero(r.re) && is_zero(r.im))) {
            const uint32_t o = atomicAdd(&s.n_out, 1u);
            s.oent[o] = (uint16_t)s.tab[slot];
            s.oval[o] = r;
          }
        }
        __syncthreads();
        // ---- phase 6: one output reservation per pass, then the table back to empty
        const uint32_t n_out = s.n_out;
        if (tid == 0) s.out_base = n_out ? atomicAdd(a.out_n, (unsigned long long)n_out) : 0ull;
        __syncthreads();
        const unsigned long long ob = s.out_base;
        if (ob + n_out > a.out_cap) {
          if (tid == 0 && n_out) atomicOr(a.err, 1);
        } else {
          for (uint32_t i = tid; i < n_out; i += kWThreads) {
            const KeyW<W> k = s.key[s.oent[i]];
            RecW<W> rec;
#pragma unroll
            for (int q = 0; q < W; ++q) {
              rec.v[q] = k.v[q];
              rec.w[q] = k.w[q];
            }
            rec.re = s.oval[i].re;
            rec.im = s.oval[i].im;
            a.out[ob + i] = rec;
          }
        }
        for (uint32_t u = tid; u < n_u; u += kWThreads) {
          s.tab[s.ulist[u]] = -1;
          s.cnt[s.ulist[u]] = 0;
        }
        __syncthreads();
        if (tid == 0) {
          s.n_e = s.n_u = s.n_out = 0;
          s.flags = 0;
        }
        __syncthreads();
      }
    }
  }
}

int choose_bits(int64_t bound_total) {
  int b = 4;
  while (b < 22 && ((int64_t)1 << b) * kWE < bound_total) ++b;
  return b;
}

template <int W>
int merge_t(const WSpec<W>& sp, cudaStream_t s, pauli_sum* out) {
  PS_TRY(upload_rows());
  if (sp.nH > kMaxHW || sp.nsrc > 4) return PS_ERR_INVALID;
  const int64_t nX = (sp.X && sp.nH > 0) ? sp.nX : 0;
  int64_t nsrc_total = sp.npre;
  for (int i = 0; i < sp.nsrc; ++i) nsrc_total += sp.nsrc_n[i];
  const int64_t bound_total = (int64_t)sp.nH * nX + nsrc_total;
  if (bound_total == 0) {
    out->n = 0;
    out->cls = 0;
    return PS_OK;
  }
  const int bits = choose_bits(bound_total);
  const uint32_t nbins = 1u << bits;
  const int nsm = num_sms();
  Buf<uint32_t> fX, fH, histX, histY, cnt, flag, gstart;
  Buf<uint64_t> bound, base, cpre, fpre, entries;
  Buf<unsigned long long> counters;  // [0] product entries, [1] outputs
  Buf<unsigned> next_group;
  Buf<int> err;
  PS_TRY(histY.alloc(nbins, s));
  PS_TRY(bound.alloc(nbins, s));
  PS_TRY(base.alloc(nbins + 1, s));
  PS_TRY(counters.alloc(2, s));
  PS_TRY(next_group.alloc(1, s));
  PS_TRY(err.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(histY.p, 0, nbins * sizeof(uint32_t), s));
  PS_CUDA(cudaMemsetAsync(counters.p, 0, 2 * sizeof(unsigned long long), s));
  PS_CUDA(cudaMemsetAsync(next_group.p, 0, sizeof(unsigned), s));
  PS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  if (nX > 0) {
    PS_TRY(fX.alloc(nX, s));
    PS_TRY(histX.alloc(nbins, s));
    PS_TRY(fH.alloc(sp.nH, s));
    PS_CUDA(cudaMemsetAsync(histX.p, 0, nbins * sizeof(uint32_t), s));
    PS_LAUNCH("k_whash_hist", s, k_whash_hist<W><<<grid_for(nX), kBT, 0, s>>>(sp.X, nX, bits, fX.p, histX.p));
    Buf<uint32_t> hdummy;
    PS_TRY(hdummy.alloc(nbins, s));
    PS_CUDA(cudaMemsetAsync(hdummy.p, 0, nbins * sizeof(uint32_t), s));
    PS_LAUNCH("k_whash_hist", s, k_whash_hist<W><<<grid_for(sp.nH), kBT, 0, s>>>(sp.H, sp.nH, bits, fH.p, hdummy.p));
    PS_CUDA(cudaGetLastError());
  }
  for (int i = 0; i < sp.nsrc; ++i)
    if (sp.nsrc_n[i] > 0)
      PS_LAUNCH("k_whash_hist", s, k_whash_hist<W><<<grid_for(sp.nsrc_n[i]), kBT, 0, s>>>(sp.src[i], sp.nsrc_n[i], bits, nullptr, histY.p));
  if (sp.npre > 0) PS_LAUNCH("k_whash_hist", s, k_whash_hist<W><<<grid_for(sp.npre), kBT, 0, s>>>(sp.pre, sp.npre, bits, nullptr, histY.p));
  PS_CUDA(cudaGetLastError());
  const int bb = (int)std::min<int64_t>(ceil_div(nbins, 256), 4 * nsm);
  PS_LAUNCH("k_wbound", s, k_wbound<<<bb, 256, 0, s>>>(nX > 0 ? histX.p : nullptr, histY.p, fH.p, nX > 0 ? sp.nH : 0, nbins, bound.p));
  PS_CUDA(cudaGetLastError());
  PS_TRY(scan_u64(bound.p, base.p, nbins, s));
  PS_TRY(entries.alloc((size_t)bound_total, s));
  Buf<unsigned long long> cur;
  PS_TRY(cur.alloc(nbins, s));
  PS_CUDA(cudaMemcpyAsync(cur.p, base.p, nbins * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  if (nX > 0) {
    for (int h0 = 0; h0 < sp.nH; h0 += kHChunkW) {
      const int nh = std::min(kHChunkW, sp.nH - h0);
      PS_LAUNCH("k_wemit", s, k_wemit<W><<<grid_for(nX), kBT, 0, s>>>(sp.X, fX.p, nX, sp.H, fH.p, h0, nh, cur.p, entries.p, counters.p));
      PS_CUDA(cudaGetLastError());
    }
  }
  for (int i = 0; i < sp.nsrc; ++i)
    if (sp.nsrc_n[i] > 0)
      PS_LAUNCH("k_wemit_src", s, k_wemit_src<W><<<grid_for(sp.nsrc_n[i]), kBT, 0, s>>>(sp.src[i], sp.nsrc_n[i], bits, kCodeSrc + i, cur.p, entries.p));
  if (sp.npre > 0) PS_LAUNCH("k_wemit_src", s, k_wemit_src<W><<<grid_for(sp.npre), kBT, 0, s>>>(sp.pre, sp.npre, bits, kCodePre, cur.p, entries.p));
  PS_CUDA(cudaGetLastError());
  PS_TRY(cnt.alloc(nbins, s));
  PS_LAUNCH("k_wcounts", s, k_wcounts<<<bb, 256, 0, s>>>(cur.p, base.p, nbins, cnt.p));
  PS_TRY(cpre.alloc(nbins + 1, s));
  PS_TRY(scan_u32_to_u64(cnt.p, cpre.p, nbins, s));
  PS_TRY(flag.alloc(nbins, s));
  PS_TRY(fpre.alloc(nbins + 1, s));
  PS_LAUNCH("k_wgroup_flags", s, k_wgroup_flags<<<bb, 256, 0, s>>>(cpre.p, nbins, flag.p));
  PS_TRY(scan_u32_to_u64(flag.p, fpre.p, nbins, s));
  PS_TRY(gstart.alloc(nbins + 1, s));
  PS_LAUNCH("k_wgroup_scatter", s, k_wgroup_scatter<<<bb, 256, 0, s>>>(flag.p, fpre.p, nbins, gstart.p));
  PS_CUDA(cudaGetLastError());
  uint64_t hc[2] = {0, 0};
  unsigned long long n_prod = 0;
  PS_CUDA(cudaMemcpyAsync(&hc[0], cpre.p + nbins, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&hc[1], fpre.p + nbins, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&n_prod, counters.p, sizeof(n_prod), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  const int64_t total_entries = (int64_t)hc[0];
  const int64_t out_cap = std::max<int64_t>(total_entries, 1);
  RecW<W>* outbuf = nullptr;
  PS_TRY(dev_alloc((void**)&outbuf, (size_t)out_cap * sizeof(RecW<W>), s));
  WMergeArgs<W> a{};
  a.H = sp.H;
  a.nH = sp.nH;
  a.X = sp.X;
  a.rot = sp.rot;
  for (int i = 0; i < 4; ++i) {
    a.src[i] = sp.src[i];
    a.alpha[i] = sp.alpha[i];
  }
  a.pre = sp.pre;
  a.has_post = sp.has_post;
  a.post = sp.post;
  a.bits = bits;
  a.base = base.p;
  a.cpre = cpre.p;
  a.entries = entries.p;
  a.gstart = gstart.p;
  a.ngroups = (uint32_t)hc[1];
  a.next_group = next_group.p;
  a.out = outbuf;
  a.out_n = counters.p + 1;
  a.out_cap = (unsigned long long)out_cap;
  a.err = err.p;
  const size_t sm = sizeof(WSmem<W>);
  PS_CUDA(cudaFuncSetAttribute(k_wmerge<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wmerge<W>, kWThreads, sm));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, per_sm) * nsm, (int64_t)a.ngroups));
  PS_LAUNCH("k_wmerge", s, k_wmerge<W><<<grid, kWThreads, sm, s>>>(a));
  PS_CUDA(cudaGetLastError());
  unsigned long long n_out = 0;
  int herr = 0;
  PS_CUDA(cudaMemcpyAsync(&n_out, counters.p + 1, sizeof(n_out), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    dev_free(outbuf, s);
    return (herr & 2) ? PS_ERR_TABLE_FULL : PS_ERR_CAPACITY;
  }
  PS_TRY(sum_adopt(out, reinterpret_cast<Rec*>(outbuf), out_cap, (int64_t)n_out));
  out->cls = kClsComplex;
  pauli_merge_stats st{};
  st.pair_tests = (int64_t)sp.nH * nX;
  st.contributions = (int64_t)n_prod;
  st.merged = (int64_t)n_out;
  st.groups = (int64_t)hc[1];
  record_merge_stats(st);
  return PS_OK;
}

// ----------------------------------------------------------------------------- truncation
constexpr int kSelBits = 8;
constexpr int kSelBins = 1 << kSelBits;
constexpr int kMaxWt = 256;

struct WTruncArgs {
  int max_weight;
  double cut2;
  int use_cut;
  int use_gamma;
  int use_div;
  DivConst dc;
  double factor[kMaxWt + 1];  // exp(-(gamma dt) wt), wt = 0..256 (by value: no host copy)
};

// Rank key of a candidate: word 0 the |c|^2 bit pattern, then ~v and ~w from the most
// significant word down; a larger key is kept first (larger |c|, then smaller v, then w).
template <int W>
__device__ __forceinline__ uint64_t rank_word(uint64_t a2, const RecW<W>& r, int q) {
  if (q == 0) return a2;
  if (q <= W) return ~r.v[W - q];
  return ~r.w[2 * W - q];
}

template <int W>
struct WSel {
  static constexpr int kWords = 1 + 2 * W;
  static constexpr int kPasses = 64 * kWords / kSelBits;
  uint64_t prefix[kWords];
  unsigned long long need;
  int done;
};

template <int W>
__global__ void __launch_bounds__(kBT) k_wfilter(const RecW<W>* __restrict__ in, int64_t n, WTruncArgs a,
                                                 RecW<W>* __restrict__ out, uint64_t* __restrict__ ab,
                                                 unsigned* __restrict__ hist0, unsigned long long* __restrict__ n_out) {
  __shared__ unsigned s_hist[kSelBins];
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_round = ceil_div_dev(n, stride) * stride;  // every thread reaches each reservation
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_round; i += stride) {
    bool keep = false;
    RecW<W> r;
    uint64_t a2 = 0;
    if (i < n) {
      r = in[i];
      if (a.use_div) {
        r.re = div_const(r.re, a.dc);
        r.im = div_const(r.im, a.dc);
      }
      const int wt = w_weight(key_of(r));
      if (a.use_gamma) {
        const double f = a.factor[wt];
        r.re = __dmul_rn(r.re, f);
        r.im = __dmul_rn(r.im, f);
      }
      keep = !(a.max_weight >= 0 && wt > a.max_weight) && !(is_zero(r.re) && is_zero(r.im));
      if (keep) {
        const double pr = is_zero(r.re) ? 0.0 : __dmul_rn(r.re, r.re);
        const double pi = is_zero(r.im) ? 0.0 : __dmul_rn(r.im, r.im);
        const double q = add_rn(pr, pi);
        a2 = (uint64_t)__double_as_longlong(q);
        if (a.use_cut) keep = !(q < a.cut2);
      }
    }
    const unsigned long long pos = block_reserve(keep, n_out);
    if (keep) {
      out[pos] = r;
      if (ab) {
        ab[pos] = a2;
        atomicAdd(&s_hist[a2 >> (64 - kSelBits)], 1u);
      }
    }
  }
  __syncthreads();
  if (ab)
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
      if (s_hist[i]) atomicAdd(&hist0[i], s_hist[i]);
}

// Histogram of digit `pass` of the rank keys that match the fixed prefix.
template <int W>
__global__ void k_wsel_hist(const RecW<W>* __restrict__ d, const uint64_t* __restrict__ ab, int64_t n,
                            const WSel<W>* __restrict__ st_p, int pass, unsigned* __restrict__ hist) {
  __shared__ unsigned s_hist[kSelBins];
  const WSel<W> st = *st_p;
  if (st.done) return;
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const int word = pass / (64 / kSelBits);
  const int shift = 64 - kSelBits * (pass % (64 / kSelBits) + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a2 = ab[i];
    // the fixed bits: whole words before `word`, and the high bits of `word` above the digit
    const uint64_t hm = shift + kSelBits >= 64 ? 0ull : (~0ull << (shift + kSelBits));
    bool ok;
    uint64_t kw;
    if (word == 0) {
      ok = (a2 & hm) == (st.prefix[0] & hm);
      kw = a2;
    } else {
      ok = a2 == st.prefix[0];
      if (!ok) continue;
      const RecW<W> r = d[i];
      for (int q = 1; q < word && ok; ++q) ok = rank_word(a2, r, q) == st.prefix[q];
      kw = rank_word(a2, r, word);
      ok = ok && (kw & hm) == (st.prefix[word] & hm);
    }
    if (ok) atomicAdd(&s_hist[(kw >> shift) & (kSelBins - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

// Fix digit `pass` of the threshold: the bin holding the need-th largest key (one block of
// kSelBins threads); clears the histogram for the next pass.
template <int W>
__global__ void __launch_bounds__(kSelBins) k_wsel_pick(WSel<W>* st_p, int pass, unsigned* __restrict__ hist) {
  __shared__ unsigned s_c[kSelBins];
  const WSel<W> st = *st_p;
  const int b = threadIdx.x;  // thread b holds bin b
  const unsigned h = hist[b];
  hist[b] = 0;
  if (st.done) return;
  s_c[b] = h;
  __syncthreads();
  unsigned long long above = 0;  // keys in the bins above b
  for (int k = kSelBins - 1; k > b; --k) above += s_c[k];
  if (above < st.need && st.need <= above + h) {
    const int word = pass / (64 / kSelBits);
    const int shift = 64 - kSelBits * (pass % (64 / kSelBits) + 1);
    st_p->prefix[word] |= (uint64_t)b << shift;
    st_p->need = st.need - above;
    if (h == st.need - above || pass == WSel<W>::kPasses - 1) st_p->done = 1;
  }
}

// keep iff the rank key is >= the threshold, or the string is in the (sorted) keep set
template <int W>
__global__ void __launch_bounds__(kBT) k_wsel_compact(const RecW<W>* __restrict__ in, const uint64_t* __restrict__ ab,
                                                      int64_t n, const WSel<W>* __restrict__ st_p,
                                                      const RecW<W>* __restrict__ keep, int64_t nkeep,
                                                      RecW<W>* __restrict__ out, unsigned long long* __restrict__ n_out) {
  const WSel<W> st = *st_p;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_round = ceil_div_dev(n, stride) * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_round; i += stride) {
    bool kp = false;
    RecW<W> r;
    if (i < n) {
      r = in[i];
      const uint64_t a2 = ab[i];
      int cmp = 0;  // sign of (key - threshold)
      for (int q = 0; q < WSel<W>::kWords && cmp == 0; ++q) {
        const uint64_t kw = rank_word(a2, r, q);
        cmp = kw > st.prefix[q] ? 1 : (kw < st.prefix[q] ? -1 : 0);
      }
      kp = cmp >= 0;
      if (!kp && nkeep > 0) {
        int64_t l = 0, h = nkeep;
        while (l < h) {
          const int64_t m = (l + h) >> 1;
          if (rec_less(keep[m], r)) l = m + 1; else h = m;
        }
        kp = l < nkeep && key_eq(key_of(keep[l]), key_of(r));
      }
    }
    const unsigned long long pos = block_reserve(kp, n_out);
    if (kp) out[pos] = r;
  }
}

template <int W>
__global__ void k_wsel_init(WSel<W>* st, unsigned long long need) {
  WSel<W> z{};
  z.need = need;
  *st = z;
}

template <int W>
int truncate_t(pauli_sum* O, const pauli_trunc_policy* P, const pauli_sum* keep, double dt, const double* divisor) {
  cudaStream_t s = O->stream;
  const bool use_gamma = P && P->gamma != 0.0;
  const bool use_w = P && P->max_weight >= 0;
  const bool use_cut = P && P->cutoff > 0.0;
  const bool use_top = P && P->top_k > 0;
  if (!use_gamma && !use_w && !use_cut && !use_top && !divisor) return PS_OK;
  if (O->n == 0) return PS_OK;
  WTruncArgs a{};
  a.max_weight = use_w ? P->max_weight : -1;
  a.use_cut = use_cut;
  a.cut2 = use_cut ? P->cutoff * P->cutoff : 0.0;
  a.use_gamma = use_gamma;
  a.use_div = divisor != nullptr;
  a.dc = make_divconst(divisor ? *divisor : 1.0);
  if (use_gamma) {
    const double x = P->gamma * dt;
    for (int wt = 0; wt <= kMaxWt; ++wt) a.factor[wt] = std::exp(-(x * (double)wt));
  }
  const bool select = use_top && O->n > P->top_k;
  Buf<unsigned long long> cnt;
  Buf<uint64_t> ab;
  Buf<unsigned> hist;
  PS_TRY(cnt.alloc(2, s));
  PS_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s));
  if (select) {
    PS_TRY(ab.alloc((size_t)O->n, s));
    PS_TRY(hist.alloc(kSelBins, s));
    PS_CUDA(cudaMemsetAsync(hist.p, 0, kSelBins * sizeof(unsigned), s));
  }
  RecW<W>* cand = nullptr;
  PS_TRY(dev_alloc((void**)&cand, (size_t)O->n * sizeof(RecW<W>), s));
  PS_LAUNCH("k_wfilter", s, k_wfilter<W><<<grid_for(O->n), kBT, 0, s>>>(recs<W>(O), O->n, a, cand, ab.p, hist.p, cnt.p));
  cudaError_t e = cudaGetLastError();
  unsigned long long nc = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nc, cnt.p, sizeof(nc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(cand, s);
    set_cuda_error(e, "wide truncate filter");
    return PS_ERR_CUDA;
  }
  if (!use_top || (int64_t)nc <= P->top_k) return sum_adopt(O, reinterpret_cast<Rec*>(cand), O->n, (int64_t)nc);

  Buf<WSel<W>> st;
  Buf<RecW<W>> keepk;
  PS_TRY(st.alloc(1, s));
  PS_LAUNCH("k_wsel_init", s, k_wsel_init<W><<<1, 1, 0, s>>>(st.p, (unsigned long long)P->top_k));
  int64_t nkeep = 0;
  if (keep && keep->n > 0) {
    std::vector<RecW<W>> hk((size_t)keep->n);
    PS_CUDA(cudaMemcpyAsync(hk.data(), keep->d, hk.size() * sizeof(RecW<W>), cudaMemcpyDeviceToHost, keep->stream));
    PS_CUDA(cudaStreamSynchronize(keep->stream));
    std::sort(hk.begin(), hk.end(), [](const RecW<W>& x, const RecW<W>& y) { return rec_less(x, y); });
    nkeep = (int64_t)hk.size();
    PS_TRY(keepk.alloc(hk.size(), s));
    PS_CUDA(cudaMemcpyAsync(keepk.p, hk.data(), hk.size() * sizeof(RecW<W>), cudaMemcpyHostToDevice, s));
  }
  const int hb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)nc, kBT), 4 * num_sms()));
  PS_LAUNCH("k_wsel_pick", s, k_wsel_pick<W><<<1, kSelBins, 0, s>>>(st.p, 0, hist.p));
  for (int pass = 1; pass < WSel<W>::kPasses; ++pass) {
    PS_LAUNCH("k_wsel_hist", s, k_wsel_hist<W><<<hb, kBT, 0, s>>>(cand, ab.p, (int64_t)nc, st.p, pass, hist.p));
    PS_LAUNCH("k_wsel_pick", s, k_wsel_pick<W><<<1, kSelBins, 0, s>>>(st.p, pass, hist.p));
    if (pass % 8 == 7) {  // the |c|^2 word is fixed after pass 7; key words only matter for ties
      WSel<W> hs;
      PS_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
      PS_CUDA(cudaStreamSynchronize(s));
      if (hs.done) break;
    }
  }
  PS_CUDA(cudaGetLastError());
  RecW<W>* outb = nullptr;
  PS_TRY(dev_alloc((void**)&outb, (size_t)std::max<unsigned long long>(nc, 1) * sizeof(RecW<W>), s));
  PS_LAUNCH("k_wsel_compact", s, k_wsel_compact<W><<<grid_for((int64_t)nc), kBT, 0, s>>>(cand, ab.p, (int64_t)nc, st.p, keepk.p, nkeep, outb, cnt.p + 1));
  e = cudaGetLastError();
  unsigned long long nk = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nk, cnt.p + 1, sizeof(nk), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(cand, s);
  if (e != cudaSuccess) {
    dev_free(outb, s);
    set_cuda_error(e, "wide truncate select");
    return PS_ERR_CUDA;
  }
  return sum_adopt(O, reinterpret_cast<Rec*>(outb), (int64_t)std::max<unsigned long long>(nc, 1), (int64_t)nk);
}

// ----------------------------------------------------------------------------- steps
struct WTmp {
  pauli_sum s;
  explicit WTmp(const pauli_sum* like) : s{like->n_sites, like->stream, nullptr, 0, 0, 0, 0, like->W} {}
  ~WTmp() { dev_free(s.d, s.stream); }
  WTmp(const WTmp&) = delete;
  WTmp& operator=(const WTmp&) = delete;
};

void swap_contents(pauli_sum* a, pauli_sum* b) {
  std::swap(a->d, b->d);
  std::swap(a->cap, b->cap);
  std::swap(a->n, b->n);
  std::swap(a->cls, b->cls);
}

template <int W>
void add_source(WSpec<W>& sp, const pauli_sum* y, Cx alpha) {
  sp.src[sp.nsrc] = recs<W>(y);
  sp.nsrc_n[sp.nsrc] = y->n;
  sp.alpha[sp.nsrc] = alpha;
  ++sp.nsrc;
}

template <int W>
int commutator_t(const pauli_sum* H, const pauli_sum* X, int rot, pauli_sum* out) {
  WSpec<W> sp;
  sp.H = recs<W>(H);
  sp.nH = (int)H->n;
  sp.X = recs<W>(X);
  sp.nX = X->n;
  sp.rot = rot;
  return merge_t<W>(sp, out->stream, out);
}

template <int W>
int rk4_t(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* policy, const pauli_sum* keep) {
  const double h2 = dt / 2.0, h6 = dt / 6.0;
  const bool trim = policy && policy->trim_stages && policy->top_k > 0;
  pauli_trunc_policy stage{-1, 0.0, policy ? policy->top_k : 0, 0.0, 0};
  WTmp k1(O), k2(O), k3(O), k4(O), X(O);
  auto L = [&](const pauli_sum* in, pauli_sum* k) -> int {
    PS_TRY(commutator_t<W>(H, in, 1, k));
    if (trim) PS_TRY(truncate_t<W>(k, &stage, nullptr, dt, nullptr));
    return PS_OK;
  };
  auto stage_input = [&](const pauli_sum* k, double c) -> int {  // X = O + c k
    WSpec<W> sp;
    add_source(sp, O, Cx{1.0, 0.0});
    add_source(sp, k, Cx{c, 0.0});
    return merge_t<W>(sp, O->stream, &X.s);
  };
  PS_TRY(L(O, &k1.s));
  PS_TRY(stage_input(&k1.s, h2));
  PS_TRY(L(&X.s, &k2.s));
  PS_TRY(stage_input(&k2.s, h2));
  PS_TRY(L(&X.s, &k3.s));
  PS_TRY(stage_input(&k3.s, dt));
  PS_TRY(L(&X.s, &k4.s));
  WSpec<W> sp;  // S = ((k1 + 2 k2) + 2 k3) + k4;  O' = O + (dt/6) S
  add_source(sp, &k1.s, Cx{1.0, 0.0});
  add_source(sp, &k2.s, Cx{2.0, 0.0});
  add_source(sp, &k3.s, Cx{2.0, 0.0});
  add_source(sp, &k4.s, Cx{1.0, 0.0});
  sp.pre = recs<W>(O);
  sp.npre = O->n;
  sp.has_post = 1;
  sp.post = Cx{h6, 0.0};
  PS_TRY(merge_t<W>(sp, O->stream, &X.s));
  PS_TRY(truncate_t<W>(&X.s, policy, keep, dt, nullptr));
  swap_contents(O, &X.s);
  return PS_OK;
}

template <int W>
int lanczos_t(const pauli_sum* H, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev, const pauli_trunc_policy* policy,
              double* b_out) {
  WTmp A(O_cur);
  WSpec<W> sp;
  sp.H = recs<W>(H);
  sp.nH = (int)H->n;
  sp.X = recs<W>(O_cur);
  sp.nX = O_cur->n;
  if (O_prev->n > 0) add_source(sp, O_prev, Cx{-b_prev, 0.0});
  PS_TRY(merge_t<W>(sp, O_cur->stream, &A.s));
  double n2 = 0.0;
  PS_TRY(norm2_t<W>(&A.s, &n2));
  const double b = std::sqrt(n2);
  *b_out = b;
  if (!std::isfinite(b)) return PS_ERR_NONFINITE;
  if (b == 0.0) return PS_ERR_KRYLOV_EXHAUSTED;
  pauli_trunc_policy p{-1, 0.0, 0, 0.0, 0};
  if (policy) {
    p.max_weight = policy->max_weight;
    p.cutoff = policy->cutoff;
    p.top_k = policy->top_k;
  }
  PS_TRY(truncate_t<W>(&A.s, &p, nullptr, 0.0, &b));
  swap_contents(O_prev, O_cur);
  swap_contents(O_cur, &A.s);
  return PS_OK;
}

#define PS_WIDE_DISPATCH(W_, call2, call4) ((W_) == 2 ? (call2) : (call4))

}  // namespace wide

// ----------------------------------------------------------------------------- entry points used by the C ABI
namespace wide_api {

using namespace wide;

int upload(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re, const double* im, int64_t n,
           bool host) {
  return PS_WIDE_DISPATCH(s->W, (upload_t<2>(s, v, w, re, im, n, host)), (upload_t<4>(s, v, w, re, im, n, host)));
}

int download(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im) {
  return PS_WIDE_DISPATCH(s->W, (download_t<2>(s, v, w, re, im)), (download_t<4>(s, v, w, re, im)));
}

int download_device(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im) {
  if (s->n == 0) return PS_OK;
  if (s->W == 2)
    PS_LAUNCH("k_wunpack", s->stream, k_wunpack<2><<<grid_for(s->n), kBT, 0, s->stream>>>(recs<2>(s), s->n, v, w, re, im));
  else
    PS_LAUNCH("k_wunpack", s->stream, k_wunpack<4><<<grid_for(s->n), kBT, 0, s->stream>>>(recs<4>(s), s->n, v, w, re, im));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int commutator(const pauli_sum* H, const pauli_sum* O, int rot, pauli_sum* out) {
  return PS_WIDE_DISPATCH(O->W, (commutator_t<2>(H, O, rot, out)), (commutator_t<4>(H, O, rot, out)));
}

int add(const pauli_sum* A, Cx alpha, const pauli_sum* B, pauli_sum* out) {
  if (A->W == 2) {
    WSpec<2> sp;
    add_source(sp, A, Cx{1.0, 0.0});
    add_source(sp, B, alpha);
    return merge_t<2>(sp, out->stream, out);
  }
  WSpec<4> sp;
  add_source(sp, A, Cx{1.0, 0.0});
  add_source(sp, B, alpha);
  return merge_t<4>(sp, out->stream, out);
}

int truncate(pauli_sum* O, const pauli_trunc_policy* P, const pauli_sum* keep, double dt, const double* divisor) {
  return PS_WIDE_DISPATCH(O->W, (truncate_t<2>(O, P, keep, dt, divisor)), (truncate_t<4>(O, P, keep, dt, divisor)));
}

int rk4_step(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* P, const pauli_sum* keep) {
  return PS_WIDE_DISPATCH(O->W, (rk4_t<2>(H, O, dt, P, keep)), (rk4_t<4>(H, O, dt, P, keep)));
}

int lanczos_step(const pauli_sum* H, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev, const pauli_trunc_policy* P,
                 double* b_out) {
  return PS_WIDE_DISPATCH(O_cur->W, (lanczos_t<2>(H, O_prev, O_cur, b_prev, P, b_out)),
                          (lanczos_t<4>(H, O_prev, O_cur, b_prev, P, b_out)));
}

int trace_product(const pauli_sum* A, const pauli_sum* B, double* re, double* im) {
  return PS_WIDE_DISPATCH(A->W, (trace_t<2>(A, B, re, im)), (trace_t<4>(A, B, re, im)));
}

int norm2(const pauli_sum* O, double* out) {
  return PS_WIDE_DISPATCH(O->W, (norm2_t<2>(O, out)), (norm2_t<4>(O, out)));
}

}  // namespace wide_api
}  // namespace ps
