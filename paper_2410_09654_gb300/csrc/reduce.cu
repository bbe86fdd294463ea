// Exact reductions: sum |c|^2 (norm) and sum a_s b_s (trace product), each the
// exactly rounded value of the exact sum of exact products.
//
// Every product of two doubles is an integer (the product of the two 53-bit
// significands, 64x64->128 bit) times a power of two.  Each thread adds these
// integers into a 256-bit two's-complement register window anchored about 190 bits
// below the largest product's top bit (found by a first pass), so almost every
// term is an exact integer addition on the integer pipes (no FP64 arithmetic).
// Terms reaching below the window go, exactly, into a full-range accumulator of
// 32-bit digits held in 64-bit counters.  Integer addition is associative, so the
// result does not depend on the storage order or the scheduling; the host rounds
// the final integer once to the nearest double (ties to even).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "exact_sum.cuh"

namespace ps {

using namespace exact;

namespace {

// ---------------------------------------------------------------- norm
__global__ void k_norm_top(const Rec* __restrict__ d, int64_t n, int* top) {
  int m = -100000;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Rec r = d[i];
    m = max(m, max(prod_top(r.re, r.re), prod_top(r.im, r.im)));
    m = max(m, max(nonfinite_top(r.re), nonfinite_top(r.im)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(top, m);
}

// The same pass for a single-component sum whose Lanczos truncation ranks |x| (component
// cls): it also writes the rank key of every string (the bit pattern of |x|) and the
// histogram of its top 11 bits (warp-aggregated per bin).
__global__ void __launch_bounds__(kRedThreads) k_norm_top_key(const Rec* __restrict__ d, int64_t n, int* top, int cls,
                                                              uint64_t* __restrict__ ab, unsigned* __restrict__ hist0) {
  __shared__ unsigned s_hist[kKeyBins];
  for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  int m = -100000;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
    const int64_t i = b0 + lane;  // b0 is uniform across the warp
    uint32_t dgt = 0xFFFFFFFFu;
    if (i < n) {
      const Rec r = d[i];
      m = max(m, max(prod_top(r.re, r.re), prod_top(r.im, r.im)));
      m = max(m, max(nonfinite_top(r.re), nonfinite_top(r.im)));
      const uint64_t g = (uint64_t)__double_as_longlong(cls == kClsImag ? r.im : r.re) & ~(1ull << 63);
      ab[i] = g;
      dgt = (uint32_t)(g >> 53);
    }
    const unsigned mm = __match_any_sync(0xffffffffu, dgt);
    if (i < n && lane == __ffs(mm) - 1) atomicAdd(&s_hist[dgt], (unsigned)__popc(mm));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(top, m);
  __syncthreads();
  for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&hist0[i], s_hist[i]);
}

// TS: a translation-symmetric generator on a ring of `ring` sites; a string of period p
// stands for ring/p copies of each translate, so its |c|^2 is added ring/p times.
template <bool TS>
__global__ void __launch_bounds__(kRedThreads) k_norm_acc(const Rec* __restrict__ d, int64_t n, const int* top,
                                                          long long* gwin, long long* full, int* wlo_out, int ring,
                                                          uint64_t divmask) {
  int t = *top;
  if (t <= -100000 || t >= kTopInf) return;
  int wlo = ((t - 190 + kBias) & ~31) - kBias;  // 32-aligned: terms < 2^222, 33 bits of headroom
  if (blockIdx.x == 0 && threadIdx.x == 0) *wlo_out = wlo;
  Win acc{{0, 0, 0, 0}};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Rec r = d[i];
    const int m = TS ? ring / ts_period(r.v, r.w, ring, divmask) : 1;
    for (int j = 0; j < m; ++j) {
      add_product(acc, r.re, r.re, wlo, full);
      add_product(acc, r.im, r.im, wlo, full);
    }
  }
  block_flush(acc, gwin);
}

// The accumulation pass from rank keys: g = bit pattern of |x| of a single-component sum's
// non-zero component, so x^2 = |x|^2 is added exactly (the other component is zero); with
// HIST, the histogram of the keys' top 11 bits in the same read (shared-memory adds: measured
// a little faster than aggregating equal bins of a warp first).
template <bool HIST>
__global__ void __launch_bounds__(kRedThreads) k_norm_acc_keys(const uint64_t* __restrict__ ab, int64_t n,
                                                               const int* top, long long* gwin, long long* full,
                                                               int* wlo_out, unsigned* __restrict__ hist0) {
  __shared__ unsigned s_hist[HIST ? kKeyBins : 1];
  if constexpr (HIST) {
    for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
  }
  const int t = *top;
  const bool acc_on = !(t <= -100000 || t >= kTopInf);  // uniform over the grid
  const int wlo = ((t - 190 + kBias) & ~31) - kBias;
  if (acc_on && blockIdx.x == 0 && threadIdx.x == 0) *wlo_out = wlo;
  Win acc{{0, 0, 0, 0}};
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
    const int64_t i = b0 + lane;  // b0 is uniform across the warp
    uint32_t dgt = 0xFFFFFFFFu;
    if (i < n) {
      const uint64_t g = ab[i];
      const double x = __longlong_as_double((long long)g);
      if (acc_on) add_product(acc, x, x, wlo, full);
      dgt = (uint32_t)(g >> 53);
    }
    if constexpr (HIST) {
      if (i < n) atomicAdd(&s_hist[dgt], 1u);
    }
  }
  if (acc_on) block_flush(acc, gwin);
  if constexpr (HIST) {
    __syncthreads();
    for (int i = threadIdx.x; i < kKeyBins; i += blockDim.x)
      if (s_hist[i]) atomicAdd(&hist0[i], s_hist[i]);
  }
}

// ---------------------------------------------------------------- trace product
// Table of B's keys (empty = all ones; the all-ones key itself is kept aside in *ones_idx).
__global__ void k_tp_build(const Rec* __restrict__ B, int64_t n, ulonglong2* tkey, int64_t* tidx, uint64_t tmask,
                           long long* ones_idx) {
  const ulonglong2 empty = make_ulonglong2(~0ull, ~0ull);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = make_ulonglong2(B[i].v, B[i].w);
    if (k.x == empty.x && k.y == empty.y) {
      *ones_idx = i;
      continue;
    }
    uint64_t slot = mix_key(k.x, k.y) & tmask;
    for (uint64_t p = 0; p <= tmask; ++p) {
      ulonglong2 old = cas128_g(&tkey[slot], empty, k);
      if (old.x == empty.x && old.y == empty.y) {
        tidx[slot] = i;
        break;
      }
      slot = (slot + 1) & tmask;
    }
  }
}

// ---------------------------------------------------------------- coefficient lookup
// out[j] = (re, im) of the O string equal to table key j (the table holds distinct keys;
// entries with no match keep their zero).
__global__ void k_coef_probe(const Rec* __restrict__ O, int64_t n, const ulonglong2* tkey, const int64_t* tidx,
                             uint64_t tmask, const long long* ones_idx, double2* __restrict__ out) {
  const long long oi = *ones_idx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Rec r = O[i];
    const int64_t j = tp_find(tkey, tidx, tmask, oi, r.v, r.w);
    if (j >= 0) out[j] = make_double2(r.re, r.im);
  }
}

// label[i] = 1 if X's i-th string is a key of the table, else 0.
__global__ void k_member(const Rec* __restrict__ X, int64_t n, const ulonglong2* tkey, const int64_t* tidx,
                         uint64_t tmask, const long long* ones_idx, float* __restrict__ label) {
  const long long oi = *ones_idx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Rec r = X[i];
    label[i] = tp_find(tkey, tidx, tmask, oi, r.v, r.w) >= 0 ? 1.0f : 0.0f;
  }
}

__global__ void k_tp_top(const Rec* __restrict__ A, int64_t n, const Rec* __restrict__ B, const ulonglong2* tkey,
                         const int64_t* tidx, uint64_t tmask, const long long* ones_idx, int* top) {
  int m = -100000;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Rec a = A[i];
    int64_t j = tp_find(tkey, tidx, tmask, *ones_idx, a.v, a.w);
    if (j < 0) continue;
    Rec b = B[j];
    m = max(m, max(max(prod_top(a.re, b.re), prod_top(a.im, b.im)), max(prod_top(a.re, b.im), prod_top(a.im, b.re))));
    // a non-finite factor in a matched pair makes both parts NaN
    if (nonfinite_top(a.re) > 0 || nonfinite_top(a.im) > 0 || nonfinite_top(b.re) > 0 || nonfinite_top(b.im) > 0)
      m = kTopNaN;
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) {
    atomicMax(top, m);
  }
}

__global__ void __launch_bounds__(kRedThreads) k_tp_acc(const Rec* __restrict__ A, int64_t n, const Rec* __restrict__ B,
                                                        const ulonglong2* tkey, const int64_t* tidx, uint64_t tmask,
                                                        const long long* ones_idx, const int* top, long long* gwin_re,
                                                        long long* full_re, long long* gwin_im, long long* full_im,
                                                        int* wlo_out) {
  int t = *top;
  if (t <= -100000 || t >= kTopInf) return;
  int wlo = ((t - 190 + kBias) & ~31) - kBias;
  if (blockIdx.x == 0 && threadIdx.x == 0) *wlo_out = wlo;
  Win ar{{0, 0, 0, 0}}, ai{{0, 0, 0, 0}};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Rec a = A[i];
    int64_t j = tp_find(tkey, tidx, tmask, *ones_idx, a.v, a.w);
    if (j < 0) continue;
    Rec b = B[j];
    add_product(ar, a.re, b.re, wlo, full_re);
    add_product(ar, -a.im, b.im, wlo, full_re);
    add_product(ai, a.re, b.im, wlo, full_im);
    add_product(ai, a.im, b.re, wlo, full_im);
  }
  block_flush(ar, gwin_re);
  __syncthreads();
  block_flush(ai, gwin_im);
}

}  // namespace

namespace {
int exact_norm2_impl(const Rec* d, int64_t n, cudaStream_t s, double* out, int ring, int cls, uint64_t* ab,
                     unsigned* hist) {
  *out = 0.0;
  if (n == 0) return PS_OK;
  Buf<long long> acc;  // [0..7] window, [8..8+kFullDigits) full
  Buf<int> ints;       // [0] top, [1] wlo
  PS_TRY(acc.alloc(kWinDigits + kFullDigits, s));
  PS_TRY(ints.alloc(2, s));
  PS_CUDA(cudaMemsetAsync(acc.p, 0, (kWinDigits + kFullDigits) * sizeof(long long), s));
  // top starts at 0x80808080 (far below any exponent; a memset, not a host copy, which would
  // synchronise the stream)
  PS_CUDA(cudaMemsetAsync(ints.p, 0x80, 2 * sizeof(int), s));
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kRedThreads), 4 * num_sms()));
  if (ab)
    PS_LAUNCH("k_norm_top", s, k_norm_top_key<<<blocks, kRedThreads, 0, s>>>(d, n, ints.p, cls, ab, hist));
  else
    PS_LAUNCH("k_norm_top", s, k_norm_top<<<blocks, kRedThreads, 0, s>>>(d, n, ints.p));
  PS_CUDA(cudaGetLastError());
  if (ring > 0)
    PS_LAUNCH("k_norm_acc", s, k_norm_acc<true><<<blocks, kRedThreads, 0, s>>>(d, n, ints.p, acc.p, acc.p + kWinDigits,
                                                                              ints.p + 1, ring, proper_divisor_mask(ring)));
  else
    PS_LAUNCH("k_norm_acc", s, k_norm_acc<false><<<blocks, kRedThreads, 0, s>>>(d, n, ints.p, acc.p, acc.p + kWinDigits,
                                                                               ints.p + 1, 0, 0ull));
  PS_CUDA(cudaGetLastError());
  std::vector<long long> h(kWinDigits + kFullDigits);
  int hi[2];
  PS_CUDA(cudaMemcpyAsync(h.data(), acc.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(hi, ints.p, sizeof(hi), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  if (hi[0] <= -100000) return PS_OK;
  if (hi[0] >= kTopInf) {
    *out = hi[0] == kTopNaN ? std::nan("") : HUGE_VAL;
    return PS_OK;
  }
  std::vector<long long> full(h.begin() + kWinDigits, h.end());
  *out = round_exact(full, h.data(), hi[1]);
  return PS_OK;
}
}  // namespace

int exact_norm2_keys_top(const uint64_t* ab, int64_t n, const int* top, cudaStream_t s, double* out, unsigned* hist) {
  *out = 0.0;
  if (hist) PS_CUDA(cudaMemsetAsync(hist, 0, kKeyBins * sizeof(unsigned), s));
  if (n == 0) return PS_OK;
  Buf<long long> acc;  // [0..7] window, [8..8+kFullDigits) full
  Buf<int> wlo;
  PS_TRY(acc.alloc(kWinDigits + kFullDigits, s));
  PS_TRY(wlo.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(acc.p, 0, (kWinDigits + kFullDigits) * sizeof(long long), s));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kRedThreads), 4 * num_sms()));
  if (hist)
    PS_LAUNCH("k_norm_acc", s, k_norm_acc_keys<true><<<blocks, kRedThreads, 0, s>>>(ab, n, top, acc.p, acc.p + kWinDigits, wlo.p, hist));
  else
    PS_LAUNCH("k_norm_acc", s, k_norm_acc_keys<false><<<blocks, kRedThreads, 0, s>>>(ab, n, top, acc.p, acc.p + kWinDigits, wlo.p, nullptr));
  PS_CUDA(cudaGetLastError());
  std::vector<long long> h(kWinDigits + kFullDigits);
  int hi[2];
  PS_CUDA(cudaMemcpyAsync(h.data(), acc.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&hi[0], top, sizeof(int), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&hi[1], wlo.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  if (hi[0] <= -100000) return PS_OK;
  if (hi[0] >= kTopInf) {
    *out = hi[0] == kTopNaN ? std::nan("") : HUGE_VAL;
    return PS_OK;
  }
  std::vector<long long> full(h.begin() + kWinDigits, h.end());
  *out = round_exact(full, h.data(), hi[1]);
  return PS_OK;
}

int key_first_digits(const uint64_t* ab, int64_t n, cudaStream_t s, unsigned* hist) {
  PS_CUDA(cudaMemsetAsync(hist, 0, kKeyBins * sizeof(unsigned), s));
  if (n == 0) return PS_OK;
  Buf<int> top;  // below every bound: the pass only counts
  PS_TRY(top.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(top.p, 0x80, sizeof(int), s));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kRedThreads), 4 * num_sms()));
  PS_LAUNCH("k_key_hist", s, k_norm_acc_keys<true><<<blocks, kRedThreads, 0, s>>>(ab, n, top.p, nullptr, nullptr, nullptr, hist));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int exact_norm2(const Rec* d, int64_t n, cudaStream_t s, double* out, int ring) {
  return exact_norm2_impl(d, n, s, out, ring, 0, nullptr, nullptr);
}

// ab: n rank keys; hist: kKeyBins counters, zeroed here.
int exact_norm2_keys(const Rec* d, int64_t n, cudaStream_t s, double* out, int cls, uint64_t* ab, unsigned* hist) {
  PS_CUDA(cudaMemsetAsync(hist, 0, kKeyBins * sizeof(unsigned), s));
  return exact_norm2_impl(d, n, s, out, 0, cls, ab, hist);
}

int exact_trace_product(const Rec* A, int64_t na, const Rec* B, int64_t nb, cudaStream_t s, double* re, double* im) {
  *re = 0.0;
  *im = 0.0;
  if (na == 0 || nb == 0) return PS_OK;
  // table over the smaller operand
  bool swap = nb > na;
  const Rec* P = swap ? B : A;  // probed
  const Rec* T = swap ? A : B;  // tabled
  int64_t np = swap ? nb : na, nt = swap ? na : nb;
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * nt)) slots <<= 1;
  Buf<ulonglong2> tkey;
  Buf<int64_t> tidx;
  Buf<long long> acc;  // re window, re full, im window, im full, ones_idx
  Buf<int> ints;
  const int span = kWinDigits + kFullDigits;
  PS_TRY(tkey.alloc(slots, s));
  PS_TRY(tidx.alloc(slots, s));
  PS_TRY(acc.alloc(2 * span + 1, s));
  PS_TRY(ints.alloc(2, s));
  PS_CUDA(cudaMemsetAsync(tkey.p, 0xFF, slots * sizeof(ulonglong2), s));
  PS_CUDA(cudaMemsetAsync(acc.p, 0, 2 * span * sizeof(long long), s));
  PS_CUDA(cudaMemsetAsync(acc.p + 2 * span, 0xFF, sizeof(long long), s));  // ones_idx = -1
  PS_CUDA(cudaMemsetAsync(ints.p, 0x80, 2 * sizeof(int), s));              // top far below any exponent
  int bt = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nt, 256), 4 * num_sms()));
  PS_LAUNCH("k_tp_build", s, k_tp_build<<<bt, 256, 0, s>>>(T, nt, tkey.p, tidx.p, slots - 1, acc.p + 2 * span));
  PS_CUDA(cudaGetLastError());
  int bp = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(np, kRedThreads), 4 * num_sms()));
  // a_s b_s is symmetric in (A, B): probing with either operand gives the same terms
  PS_LAUNCH("k_tp_top", s, k_tp_top<<<bp, kRedThreads, 0, s>>>(P, np, T, tkey.p, tidx.p, slots - 1, acc.p + 2 * span, ints.p));
  PS_CUDA(cudaGetLastError());
  PS_LAUNCH("k_tp_acc", s, k_tp_acc<<<bp, kRedThreads, 0, s>>>(P, np, T, tkey.p, tidx.p, slots - 1, acc.p + 2 * span, ints.p, acc.p,
                                      acc.p + kWinDigits, acc.p + span, acc.p + span + kWinDigits, ints.p + 1));
  PS_CUDA(cudaGetLastError());
  std::vector<long long> h(2 * span);
  int hi[2];
  PS_CUDA(cudaMemcpyAsync(h.data(), acc.p, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(hi, ints.p, sizeof(hi), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
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

}  // namespace ps

namespace ps {

// Coefficients of nq query strings (host arrays) in the device sum O.  Queries are
// deduplicated on the host, their table built on the device, O streamed once.
int coefficients(const Rec* O, int64_t n, const uint64_t* qv, const uint64_t* qw, int64_t nq, cudaStream_t s,
                 double* re, double* im) {
  for (int64_t j = 0; j < nq; ++j) re[j] = im[j] = 0.0;
  if (nq == 0 || n == 0) return PS_OK;
  std::vector<int64_t> ord((size_t)nq);
  for (int64_t j = 0; j < nq; ++j) ord[(size_t)j] = j;
  std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
    return qv[a] < qv[b] || (qv[a] == qv[b] && qw[a] < qw[b]);
  });
  std::vector<Rec> uq;
  std::vector<int64_t> slot_of((size_t)nq);
  for (int64_t r = 0; r < nq; ++r) {
    const int64_t j = ord[(size_t)r];
    if (uq.empty() || uq.back().v != qv[j] || uq.back().w != qw[j]) uq.push_back(Rec{qv[j], qw[j], 0.0, 0.0});
    slot_of[(size_t)j] = (int64_t)uq.size() - 1;
  }
  const int64_t nu = (int64_t)uq.size();
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * nu)) slots <<= 1;
  Buf<Rec> dq;
  Buf<ulonglong2> tkey;
  Buf<int64_t> tidx;
  Buf<long long> ones;
  Buf<double2> out;
  PS_TRY(dq.alloc(nu, s));
  PS_TRY(tkey.alloc(slots, s));
  PS_TRY(tidx.alloc(slots, s));
  PS_TRY(ones.alloc(1, s));
  PS_TRY(out.alloc(nu, s));
  PS_CUDA(cudaMemcpyAsync(dq.p, uq.data(), nu * sizeof(Rec), cudaMemcpyHostToDevice, s));
  PS_CUDA(cudaMemsetAsync(tkey.p, 0xFF, slots * sizeof(ulonglong2), s));
  PS_CUDA(cudaMemsetAsync(out.p, 0, nu * sizeof(double2), s));
  PS_CUDA(cudaMemsetAsync(ones.p, 0xFF, sizeof(long long), s));  // -1: no all-ones query
  const int nsm = num_sms();
  int bt = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nu, 256), 4 * nsm));
  PS_LAUNCH("k_tp_build", s, k_tp_build<<<bt, 256, 0, s>>>(dq.p, nu, tkey.p, tidx.p, slots - 1, ones.p));
  PS_CUDA(cudaGetLastError());
  int bp = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * nsm));
  PS_LAUNCH("k_coef_probe", s, k_coef_probe<<<bp, 256, 0, s>>>(O, n, tkey.p, tidx.p, slots - 1, ones.p, out.p));
  PS_CUDA(cudaGetLastError());
  std::vector<double2> h((size_t)nu);
  PS_CUDA(cudaMemcpyAsync(h.data(), out.p, nu * sizeof(double2), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  for (int64_t j = 0; j < nq; ++j) {
    re[j] = h[(size_t)slot_of[(size_t)j]].x;
    im[j] = h[(size_t)slot_of[(size_t)j]].y;
  }
  return PS_OK;
}

// Membership of X's strings in T (T's keys distinct): label[i] in {0, 1}, X's storage order.
int membership(const Rec* X, int64_t nx, const Rec* T, int64_t nt, cudaStream_t s, float* label) {
  if (nx == 0) return PS_OK;
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * std::max<int64_t>(nt, 1))) slots <<= 1;
  Buf<ulonglong2> tkey;
  Buf<int64_t> tidx;
  Buf<long long> ones;
  PS_TRY(tkey.alloc(slots, s));
  PS_TRY(tidx.alloc(slots, s));
  PS_TRY(ones.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(tkey.p, 0xFF, slots * sizeof(ulonglong2), s));
  PS_CUDA(cudaMemsetAsync(ones.p, 0xFF, sizeof(long long), s));  // -1: the all-ones key is absent
  const int nsm = num_sms();
  if (nt > 0) {
    int bt = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nt, 256), 4 * nsm));
    PS_LAUNCH("k_tp_build", s, k_tp_build<<<bt, 256, 0, s>>>(T, nt, tkey.p, tidx.p, slots - 1, ones.p));
  }
  int bp = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nx, 256), 8 * nsm));
  PS_LAUNCH("k_member", s, k_member<<<bp, 256, 0, s>>>(X, nx, tkey.p, tidx.p, slots - 1, ones.p, label));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace ps
