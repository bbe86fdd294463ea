// Truncation (paper: trim(O, M; keep), cutoff(O, eps), discarding long strings,
// add_noise(O, eps*dt)):
//   1. optional division by a real b (the Lanczos normalisation O = A/b);
//   2. depolarising transmission c *= exp(-(gamma*dt) * wt), wt = popcount(v|w);
//   3. drop wt > max_weight; drop exact zeros; drop |c|^2 < cutoff^2;
//   4. keep the top_k by |c|^2 = re*re + im*im, exact ties to the smaller key (v, then w),
//      never dropping a string of the keep set.
// Step 4 is a most-significant-digit radix select over the 192-bit rank key
// (|c|^2 bits, ~v, ~w): all rank keys are distinct, so exactly top_k strings
// outrank the selected threshold.  A caller-given score can take the place of |c|^2
// (the learned truncation ranks by ln|c| - gamma dt wt + z).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "select.cuh"

namespace ps {

namespace {


struct TruncArgs {
  int max_weight;
  double cut2;
  int use_cut;
  int use_gamma;
  int use_div;
  DivConst dc;
  double factor[65];     // exp(-(gamma*dt) w), w = 0..64 (passed by value: no host copy)
  int cls;               // coefficient class of the input: components that may be non-zero
  int round32;           // FP32 sum: round to FP32 after the division and dissipation
};

__device__ __forceinline__ double sq_sum(double re, double im) {
  double a = is_zero(re) ? 0.0 : __dmul_rn(re, re);
  double b = is_zero(im) ? 0.0 : __dmul_rn(im, im);
  return add_rn(a, b);
}

// re*re + im*im when only the components in `cls` can be non-zero (identical value).
__device__ __forceinline__ double sq_sum_cls(double re, double im, int cls) {
  if (cls == 1) return __dmul_rn(re, re);
  if (cls == 2) return __dmul_rn(im, im);
  return sq_sum(re, im);
}

// Tile compaction: a block handles tiles of kTile elements (kTI per thread), counts the
// kept ones per warp and item, and reserves their output range with one atomic per tile.
constexpr int kTT = 256;
constexpr int kTI = 4;
constexpr int kTile = kTT * kTI;

struct TileRes {
  uint32_t wcnt[kTT / 32][kTI];
  unsigned long long base;
};

__device__ __forceinline__ void tile_positions(const bool (&f)[kTI], TileRes& sm, unsigned long long* counter,
                                               unsigned long long (&pos)[kTI]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned m[kTI];
#pragma unroll
  for (int k = 0; k < kTI; ++k) {
    m[k] = __ballot_sync(0xffffffffu, f[k]);
    if (lane == 0) sm.wcnt[warp][k] = __popc(m[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < kTI; ++k)
      for (int w = 0; w < kTT / 32; ++w) {
        uint32_t c = sm.wcnt[w][k];
        sm.wcnt[w][k] = run;
        run += c;
      }
    sm.base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kTI; ++k) pos[k] = sm.base + sm.wcnt[warp][k] + __popc(m[k] & ((1u << lane) - 1));
  __syncthreads();
}

// Order-preserving map of a double score to 64 bits: larger score -> larger key; -0 and +0
// map alike; NaN maps to 0, below every number.
__device__ __forceinline__ uint64_t score_key(double x) {
  if (x != x) return 0ull;
  if (x == 0.0) x = 0.0;
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}

// Steps 1-3 with compaction (order of survivors is unspecified).  For a later top-k
// select it also stores each survivor's rank value (the |c|^2 bit pattern: non-negative
// doubles order like their bit patterns; or, with a score array, the score's key) and
// histograms its top kDigitBits bits.
__global__ void __launch_bounds__(kTT) k_filter(const Rec* __restrict__ in, int64_t n, TruncArgs a,
                                                const double* __restrict__ score, Rec* __restrict__ out,
                                                uint64_t* __restrict__ ab, unsigned* __restrict__ hist0,
                                                unsigned long long* __restrict__ n_out) {
  __shared__ unsigned s_hist[kBins];
  __shared__ TileRes s_res;
  if (hist0) {
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
  }
  const int64_t tiles = ceil_div_dev(n, kTile);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    bool keep[kTI];
    Rec r[kTI];
    uint64_t a2[kTI];
#pragma unroll
    for (int k = 0; k < kTI; ++k) {
      const int64_t i = tile * kTile + (int64_t)k * kTT + threadIdx.x;
      keep[k] = false;
      a2[k] = 0;
      if (i < n) {
        r[k] = in[i];
        if (a.use_div) {  // components outside the class are zero and stay zero
          if (a.cls & 1) r[k].re = div_const(r[k].re, a.dc);
          if (a.cls & 2) r[k].im = div_const(r[k].im, a.dc);
        }
        const int wt = __popcll(r[k].v | r[k].w);
        if (a.use_gamma) {
          const double f = a.factor[wt];
          if (a.cls & 1) r[k].re = __dmul_rn(r[k].re, f);
          if (a.cls & 2) r[k].im = __dmul_rn(r[k].im, f);
        }
        if (a.round32) {
          r[k].re = (double)__double2float_rn(r[k].re);
          r[k].im = (double)__double2float_rn(r[k].im);
        }
        keep[k] = !(a.max_weight >= 0 && wt > a.max_weight) && !(is_zero(r[k].re) && is_zero(r[k].im));
        if (keep[k] && (a.use_cut || ab)) {
          const double q = sq_sum_cls(r[k].re, r[k].im, a.cls);
          a2[k] = score ? score_key(score[i]) : (uint64_t)__double_as_longlong(q);
          if (a.use_cut) keep[k] = !(q < a.cut2);
        }
      }
    }
    unsigned long long pos[kTI];
    tile_positions(keep, s_res, n_out, pos);
#pragma unroll
    for (int k = 0; k < kTI; ++k) {
      if (!keep[k]) continue;
      out[pos[k]] = r[k];
      if (ab) {
        ab[pos[k]] = a2[k];
        atomicAdd(&s_hist[a2[k] >> (64 - kDigitBits)], 1u);
      }
    }
  }
  if (hist0) {
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
      if (s_hist[i]) atomicAdd(&hist0[i], s_hist[i]);
  }
}

__global__ void k_sel_init(SelState* st, unsigned long long need) {
  SelState z{};
  z.need = need;
  *st = z;
}

// After the first digit is fixed, only candidates with that top digit can decide the
// threshold: collect their indices once.
__global__ void __launch_bounds__(kTT) k_sel_narrow(const uint64_t* __restrict__ ab, int64_t n,
                                                    const SelState* __restrict__ st_p, uint32_t* __restrict__ list,
                                                    unsigned long long* __restrict__ n_list) {
  __shared__ TileRes s_res;
  const SelState st = *st_p;
  if (st.done) return;
  const uint64_t d0 = st.prefix[0] >> (64 - kDigitBits);
  const int64_t tiles = ceil_div_dev(n, kTile);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    bool f[kTI];
    int64_t idx[kTI];
#pragma unroll
    for (int k = 0; k < kTI; ++k) {
      idx[k] = tile * kTile + (int64_t)k * kTT + threadIdx.x;
      f[k] = idx[k] < n && (ab[idx[k]] >> (64 - kDigitBits)) == d0;
    }
    unsigned long long pos[kTI];
    tile_positions(f, s_res, n_list, pos);
#pragma unroll
    for (int k = 0; k < kTI; ++k)
      if (f[k]) list[pos[k]] = (uint32_t)idx[k];
  }
}

__global__ void k_sel_hist(const Rec* __restrict__ d, const uint64_t* __restrict__ ab,
                           const uint32_t* __restrict__ list, const unsigned long long* __restrict__ n_list,
                           const SelState* __restrict__ st_p, int pass, unsigned* __restrict__ hist) {
  __shared__ unsigned s_hist[kBins];
  const SelState st = *st_p;
  if (st.done) return;
  const int64_t n = (int64_t)*n_list;
  const bool need_key = (pass + 1) * kDigitBits > 64;  // this pass reads bits of ~v / ~w
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = list[j];
    uint64_t k[3];
    Rec r;
    if (need_key) r = d[i];
    rank_key(ab[i], need_key ? &r : nullptr, k);
    if (!matches_prefix(k, st, pass)) continue;
    atomicAdd(&s_hist[rank_digit(k, pass)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBins; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

// Pick the digit of the need-th largest key in the current prefix (one block of 256 threads).
__global__ void __launch_bounds__(256) k_sel_pick(SelState* st_p, int pass, unsigned* __restrict__ hist) {
  sel_pick_block(st_p, pass, hist);
}

// keep iff rank key >= threshold (prefix with zero low bits), or in the keep set (sorted keys)
__global__ void __launch_bounds__(kTT) k_sel_compact(const Rec* __restrict__ in, const uint64_t* __restrict__ ab,
                                                     int64_t n, const SelState* __restrict__ st_p,
                                                     const ulonglong2* __restrict__ keep, int64_t nkeep,
                                                     Rec* __restrict__ out, unsigned long long* __restrict__ n_out,
                                                     int use_div, DivConst dc, int cls) {
  __shared__ TileRes s_res;
  const SelState st = *st_p;
  const int64_t tiles = ceil_div_dev(n, kTile);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    bool kp[kTI];
    Rec r[kTI];
#pragma unroll
    for (int k = 0; k < kTI; ++k) {
      const int64_t i = tile * kTile + (int64_t)k * kTT + threadIdx.x;
      kp[k] = false;
      if (i < n) {
        const uint64_t a2 = ab[i];
        if (a2 > st.prefix[0]) {
          kp[k] = true;
          r[k] = in[i];
        } else if (a2 == st.prefix[0] || nkeep > 0) {
          r[k] = in[i];
          uint64_t key[3];
          rank_key(a2, &r[k], key);
          kp[k] = (key[0] > st.prefix[0]) ||
                  (key[0] == st.prefix[0] && (key[1] > st.prefix[1] || (key[1] == st.prefix[1] && key[2] >= st.prefix[2])));
          if (!kp[k] && nkeep > 0) {
            int64_t l = 0, h = nkeep;
            while (l < h) {
              int64_t m = (l + h) >> 1;
              ulonglong2 c = keep[m];
              if (c.x < r[k].v || (c.x == r[k].v && c.y < r[k].w)) l = m + 1; else h = m;
            }
            kp[k] = (l < nkeep && keep[l].x == r[k].v && keep[l].y == r[k].w);
          }
        }
      }
    }
    if (use_div) {  // the Lanczos division of the kept strings (rank values were taken before it)
#pragma unroll
      for (int k = 0; k < kTI; ++k) {
        if (!kp[k]) continue;
        if (cls & 1) r[k].re = div_const(r[k].re, dc);
        if (cls & 2) r[k].im = div_const(r[k].im, dc);
      }
    }
    unsigned long long pos[kTI];
    tile_positions(kp, s_res, n_out, pos);
#pragma unroll
    for (int k = 0; k < kTI; ++k)
      if (kp[k]) out[pos[k]] = r[k];
  }
}

// ---- Lanczos truncation without a division per candidate (single-component FP64 sums,
// top-k only).  The rank value |RN(x/b)|^2 (rounded square of the rounded quotient) is a
// non-decreasing function of |x|, so the top-k by it is found from |x| itself: an exact
// select on the bit pattern of |x| gives the k-th largest x_k; the host finds the interval
// [g_lo, g_hi] of |x| whose rank value equals that of x_k; the strings in the interval are
// tied and ordered by key (~v, ~w) exactly as in the plain truncation, those above it are
// kept.  Only the kept strings are divided (in the compaction).

// |x| of the non-zero component as a 64-bit rank value (non-negative doubles order like
// their bit patterns), with the histogram of its top digit (warp-aggregated per digit).
__global__ void __launch_bounds__(kTT) k_abskey(const Rec* __restrict__ in, int64_t n, int cls,
                                                uint64_t* __restrict__ ab, unsigned* __restrict__ hist0) {
  __shared__ unsigned s_hist[kBins];
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
    const int64_t i = b0 + lane;  // b0 is uniform across the warp
    uint32_t dgt = 0xFFFFFFFFu;
    if (i < n) {
      const double x = cls == 2 ? in[i].im : in[i].re;
      const uint64_t g = (uint64_t)__double_as_longlong(x) & ~(1ull << 63);
      ab[i] = g;
      dgt = (uint32_t)(g >> (64 - kDigitBits));
    }
    const unsigned m = __match_any_sync(0xffffffffu, dgt);
    if (i < n && lane == __ffs(m) - 1) atomicAdd(&s_hist[dgt], (unsigned)__popc(m));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBins; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&hist0[i], s_hist[i]);
}

__global__ void k_sel_init_ex(SelState* st, unsigned long long need, int exact, uint64_t prefix0) {
  SelState z{};
  z.need = need;
  z.exact = exact;
  z.prefix[0] = prefix0;
  *st = z;
}

// Strings whose rank value lies in [g_lo, g_hi] (tied with the k-th) take the common rank
// value g_hi and are listed; those above the interval are counted.
__global__ void __launch_bounds__(kTT) k_tie_prep(uint64_t* __restrict__ ab, int64_t n, uint64_t g_lo, uint64_t g_hi,
                                                  uint32_t* __restrict__ list, unsigned long long* __restrict__ n_list,
                                                  unsigned long long* __restrict__ n_above) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long above = 0;
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
    const int64_t i = b0 + lane;
    bool tie = false;
    if (i < n) {
      const uint64_t g = ab[i];
      if (g > g_hi) {
        ++above;
      } else if (g >= g_lo) {
        tie = true;
        ab[i] = g_hi;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, tie);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(n_list, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (tie) list[base + __popc(m & ((1u << lane) - 1))] = (uint32_t)i;
    }
  }
  for (int d = 16; d > 0; d >>= 1) above += __shfl_down_sync(0xffffffffu, above, d);
  if (lane == 0 && above) atomicAdd(n_above, above);
}

// Second narrowing: the listed candidates whose top `bits` bits of the rank value equal the
// threshold's (the prefix fixed so far).
__global__ void __launch_bounds__(kTT) k_sel_renarrow(const uint64_t* __restrict__ ab, const uint32_t* __restrict__ list,
                                                      const unsigned long long* __restrict__ n_list, int bits,
                                                      const SelState* __restrict__ st_p, uint32_t* __restrict__ out,
                                                      unsigned long long* __restrict__ n_out) {
  const int64_t n = (int64_t)*n_list;
  const uint64_t want = st_p->prefix[0] >> (64 - bits);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
    const int64_t j = b0 + lane;
    uint32_t i = 0;
    bool f = false;
    if (j < n) {
      i = list[j];
      f = (ab[i] >> (64 - bits)) == want;
    }
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(n_out, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (f) out[base + __popc(m & ((1u << lane) - 1))] = i;
    }
  }
}

// k_tie_prep over the listed candidates only (the interval lies inside their common prefix).
__global__ void __launch_bounds__(kTT) k_tie_prep_list(uint64_t* __restrict__ ab, const uint32_t* __restrict__ list,
                                                       const unsigned long long* __restrict__ n_list, uint64_t g_lo,
                                                       uint64_t g_hi, uint32_t* __restrict__ ties,
                                                       unsigned long long* __restrict__ n_ties,
                                                       unsigned long long* __restrict__ n_above) {
  const int64_t n = (int64_t)*n_list;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long above = 0;
  for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b0 < n; b0 += stride) {
    const int64_t j = b0 + lane;
    bool tie = false;
    uint32_t i = 0;
    if (j < n) {
      i = list[j];
      const uint64_t g = ab[i];
      if (g > g_hi) {
        ++above;
      } else if (g >= g_lo) {
        tie = true;
        ab[i] = g_hi;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, tie);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(n_ties, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (tie) ties[base + __popc(m & ((1u << lane) - 1))] = i;
    }
  }
  for (int d = 16; d > 0; d >>= 1) above += __shfl_down_sync(0xffffffffu, above, d);
  if (lane == 0 && above) atomicAdd(n_above, above);
}

// The tie-break digits for a small tie set in one block: the keys (~v, ~w) of the listed
// strings are held in shared memory and every remaining pass (histogram, pick) runs here.
constexpr int kTieSmem = 2048;
__global__ void __launch_bounds__(256) k_sel_tie_block(const Rec* __restrict__ d, const uint32_t* __restrict__ list,
                                                       const unsigned long long* __restrict__ n_list, uint64_t gkey,
                                                       SelState* st_p, int pass0) {
  __shared__ ulonglong2 s_key[kTieSmem];
  __shared__ unsigned s_hist[kBins];
  const int T = (int)min(*n_list, (unsigned long long)kTieSmem);  // the host checked T <= kTieSmem
  for (int j = threadIdx.x; j < T; j += blockDim.x) {
    const Rec r = d[list[j]];
    s_key[j] = make_ulonglong2(~r.v, ~r.w);
  }
  for (int pass = pass0; pass < kPasses; ++pass) {
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    const SelState st = *st_p;
    if (st.done) break;  // every thread reads the same state after the barrier
    for (int j = threadIdx.x; j < T; j += blockDim.x) {
      const uint64_t k[3] = {gkey, s_key[j].x, s_key[j].y};
      if (matches_prefix(k, st, pass)) atomicAdd(&s_hist[rank_digit(k, pass)], 1u);
    }
    __syncthreads();
    sel_pick_block(st_p, pass, s_hist);
    __syncthreads();
  }
}

__global__ void k_debug_divide(double* __restrict__ x, int64_t n, DivConst dc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = div_const(x[i], dc);
}

}  // namespace

static_assert(kBins == kKeyBins, "the norm's key histogram has the select's first-digit bins");
bool g_general_truncation = false;  // test hook: always take the general truncation path
bool lanczos_keys_eligible(const pauli_sum* A, const pauli_trunc_policy* P);

namespace {

// |RN(x/b)|^2 as the truncation computes it (the correctly rounded quotient, then the rounded
// square), in IEEE double arithmetic on the host; b > 0.
double sq_of_quotient(double x, double b) {
  volatile double q = x / b;
  volatile double r = q * q;
  return r;
}

double from_bits(uint64_t g) {
  double x;
  std::memcpy(&x, &g, sizeof(x));
  return x;
}

constexpr int kFallback = 1 << 20;  // not an error: the caller takes the general path

// Top-k after the Lanczos division for a single-component FP64 sum O of n > k strings,
// without dividing the candidates (see k_abskey): returns a status, or kFallback when the
// threshold's rank value is zero or not finite.
// ab_in / hist_in: the rank keys and their first-digit histogram when the norm's first pass
// has produced them (else computed here).
int truncate_div_top(pauli_sum* O, int64_t k, const TruncArgs& a, double divisor, uint64_t* ab_in = nullptr,
                     unsigned* hist_in = nullptr) {
  cudaStream_t s = O->stream;
  const int64_t n = O->n;
  const int nsm = num_sms();
  auto grid = [&](int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, kTT), 8 * nsm)); };
  Buf<uint64_t> ab;
  Buf<unsigned> hist;
  Buf<SelState> st;     // [0] stage 1, [1] stage 2, [2] stage 1 after its second digit
  Buf<uint32_t> list;   // [0, n): first-digit list, later the tied strings; [n, 2n): second narrowing
  Buf<unsigned long long> cnt;  // listed, tied, above the interval, kept, second narrowing
  if (!ab_in) {
    PS_TRY(ab.alloc((size_t)n, s));
    PS_TRY(hist.alloc(kBins, s));
  }
  uint64_t* abp = ab_in ? ab_in : ab.p;
  unsigned* histp = ab_in ? hist_in : hist.p;
  PS_TRY(st.alloc(3, s));
  PS_TRY(list.alloc((size_t)n * 2, s));
  PS_TRY(cnt.alloc(5, s));
  PS_CUDA(cudaMemsetAsync(cnt.p, 0, 5 * sizeof(unsigned long long), s));
  uint32_t* list2 = list.p + n;
  // stage 1: the exact rank value |x_k| of the k-th largest |x|; the candidates are narrowed
  // to those sharing the threshold's first digit, then its first two digits (22 bits)
  if (!ab_in) {
    PS_CUDA(cudaMemsetAsync(hist.p, 0, kBins * sizeof(unsigned), s));
    PS_LAUNCH("k_abskey", s, k_abskey<<<grid(n), kTT, 0, s>>>(O->d, n, a.cls, ab.p, hist.p));
  }
  PS_LAUNCH("k_sel_init", s, k_sel_init_ex<<<1, 1, 0, s>>>(st.p, (unsigned long long)k, 1, 0ull));
  PS_LAUNCH("k_sel_pick", s, k_sel_pick<<<1, 256, 0, s>>>(st.p, 0, histp));
  PS_LAUNCH("k_sel_narrow", s, k_sel_narrow<<<grid(n), kTT, 0, s>>>(abp, n, st.p, list.p, cnt.p));
  const int hb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4 * nsm));
  PS_LAUNCH("k_sel_hist", s, k_sel_hist<<<hb, 256, 0, s>>>(O->d, abp, list.p, cnt.p, st.p, 1, histp));
  PS_LAUNCH("k_sel_pick", s, k_sel_pick<<<1, 256, 0, s>>>(st.p, 1, histp));
  PS_CUDA(cudaMemcpyAsync(st.p + 2, st.p, sizeof(SelState), cudaMemcpyDeviceToDevice, s));
  constexpr int kBits2 = 2 * kDigitBits;
  PS_LAUNCH("k_sel_narrow", s, k_sel_renarrow<<<hb, kTT, 0, s>>>(abp, list.p, cnt.p, kBits2, st.p, list2, cnt.p + 4));
  for (int pass = 2; pass <= 5; ++pass) {  // pass 5 fixes the last bits of |x_k|
    PS_LAUNCH("k_sel_hist", s, k_sel_hist<<<hb, 256, 0, s>>>(O->d, abp, list2, cnt.p + 4, st.p, pass, histp));
    PS_LAUNCH("k_sel_pick", s, k_sel_pick<<<1, 256, 0, s>>>(st.p, pass, histp));
  }
  SelState hs[3];
  PS_CUDA(cudaMemcpyAsync(hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  const uint64_t gk = hs[0].prefix[0];
  const double b = std::fabs(divisor);
  const double fk = sq_of_quotient(from_bits(gk), b);
  if (!(fk > 0.0) || !std::isfinite(fk)) return kFallback;
  // the interval of |x| with the same rank value (the rank value is non-decreasing in |x|)
  uint64_t lo = gk, hi = 0x7FF0000000000000ull;  // rank value of +inf: inf > fk
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (sq_of_quotient(from_bits(mid), b) <= fk) lo = mid; else hi = mid;
  }
  const uint64_t g_hi = lo;
  lo = 0;  // rank value 0 < fk
  hi = gk;
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (sq_of_quotient(from_bits(mid), b) < fk) lo = mid; else hi = mid;
  }
  const uint64_t g_lo = hi;
  // stage 2: the tied strings by key.  When the interval shares the threshold's first two
  // digits, only the second list can hold tied strings or strings above the interval inside
  // that prefix; the strings above the prefix are counted by the select itself (k minus the
  // rank still needed after the second digit).
  const bool in_prefix = (g_lo >> (64 - kBits2)) == (gk >> (64 - kBits2)) && (g_hi >> (64 - kBits2)) == (gk >> (64 - kBits2));
  int64_t above_prefix = 0;
  if (in_prefix) {
    above_prefix = k - (int64_t)hs[2].need;
    PS_LAUNCH("k_tie_prep", s, k_tie_prep_list<<<hb, kTT, 0, s>>>(abp, list2, cnt.p + 4, g_lo, g_hi, list.p, cnt.p + 1, cnt.p + 2));
  } else {
    PS_LAUNCH("k_tie_prep", s, k_tie_prep<<<grid(n), kTT, 0, s>>>(abp, n, g_lo, g_hi, list.p, cnt.p + 1, cnt.p + 2));
  }
  unsigned long long hc[3];
  PS_CUDA(cudaMemcpyAsync(hc, cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  const int64_t T = (int64_t)hc[1], above = above_prefix + (int64_t)hc[2];
  const int64_t need = k - above;
  if (need < 1 || need > T) return kFallback;  // cannot happen for a non-decreasing rank value
  SelState* st2 = st.p + 1;
  const uint64_t fixed55 = g_hi & ~((1ull << (64 - 5 * kDigitBits)) - 1);  // the digits of passes 0-4
  PS_LAUNCH("k_sel_init", s, k_sel_init_ex<<<1, 1, 0, s>>>(st2, (unsigned long long)need, 0, fixed55));
  if (T <= kTieSmem) {
    PS_LAUNCH("k_sel_tie_block", s, k_sel_tie_block<<<1, 256, 0, s>>>(O->d, list.p, cnt.p + 1, g_hi, st2, 5));
  } else {
    for (int pass = 5; pass < kPasses; ++pass) {
      PS_LAUNCH("k_sel_hist", s, k_sel_hist<<<hb, 256, 0, s>>>(O->d, abp, list.p, cnt.p + 1, st2, pass, histp));
      PS_LAUNCH("k_sel_pick", s, k_sel_pick<<<1, 256, 0, s>>>(st2, pass, histp));
    }
  }
  // compaction: kept = above the interval, or tied and at or above the key threshold; the
  // kept strings are divided here
  const int64_t cap = above + T;
  Rec* outb = nullptr;
  PS_TRY(dev_alloc((void**)&outb, (size_t)std::max<int64_t>(cap, 1) * sizeof(Rec), s));
  const int cb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kTile), 8 * nsm));
  PS_LAUNCH("k_sel_compact", s, k_sel_compact<<<cb, kTT, 0, s>>>(O->d, abp, n, st2, nullptr, 0, outb, cnt.p + 3, 1, a.dc,
                                                                 a.cls));
  cudaError_t e = cudaGetLastError();
  unsigned long long nk = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nk, cnt.p + 3, sizeof(nk), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(outb, s);
    set_cuda_error(e, "truncate select");
    return PS_ERR_CUDA;
  }
  return sum_adopt(O, outb, std::max<int64_t>(cap, 1), (int64_t)nk);
}

}  // namespace

// Truncate O in place; `divisor` (if non-null) divides every coefficient first.
int truncate_run(pauli_sum* O, const pauli_trunc_policy* P, const pauli_sum* keep, double dt, const double* divisor,
                 const double* score) {
  cudaStream_t s = O->stream;
  const bool use_gamma = P && P->gamma != 0.0;
  const bool use_w = P && P->max_weight >= 0;
  const bool use_cut = P && P->cutoff > 0.0;
  const bool use_top = P && P->top_k > 0;
  if (!use_gamma && !use_w && !use_cut && !use_top && !divisor && !O->f32) return PS_OK;
  if (O->n == 0) return PS_OK;
  const int nsm = num_sms();

  Buf<unsigned long long> cnt;
  PS_TRY(cnt.alloc(2, s));
  PS_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s));
  TruncArgs a{};
  a.max_weight = use_w ? P->max_weight : -1;
  a.use_cut = use_cut;
  a.cut2 = use_cut ? P->cutoff * P->cutoff : 0.0;
  a.use_gamma = use_gamma;
  a.use_div = divisor != nullptr;
  a.dc = make_divconst(divisor ? *divisor : 1.0);
  a.cls = O->cls ? O->cls : kClsComplex;
  a.round32 = O->f32;
  if (use_gamma) {
    const double x = P->gamma * dt;
    for (int wt = 0; wt <= 64; ++wt) a.factor[wt] = std::exp(-(x * (double)wt));
  }
  // the Lanczos truncation (division, then top-k alone) of a single-component FP64 sum: ranked
  // without dividing every candidate
  if (divisor && !score && !(keep && keep->n > 0) && lanczos_keys_eligible(O, P) && *divisor != 0.0 &&
      std::isfinite(*divisor)) {
    const int rc = truncate_div_top(O, P->top_k, a, *divisor);
    if (rc != kFallback) return rc;
  }
  Rec* cand = nullptr;
  PS_TRY(dev_alloc((void**)&cand, (size_t)O->n * sizeof(Rec), s));
  Buf<uint64_t> ab;
  Buf<unsigned> hist;
  if (use_top && O->n > P->top_k) {
    PS_TRY(ab.alloc((size_t)O->n, s));
    PS_TRY(hist.alloc(kBins, s));
    PS_CUDA(cudaMemsetAsync(hist.p, 0, kBins * sizeof(unsigned), s));
  }
  auto tile_grid = [&](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kTile), 8 * nsm)); };
  PS_LAUNCH("k_filter", s, k_filter<<<tile_grid(O->n), kTT, 0, s>>>(O->d, O->n, a, score, cand, ab.p, hist.p, cnt.p));
  cudaError_t e = cudaGetLastError();
  unsigned long long nc = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nc, cnt.p, sizeof(nc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(cand, s);
    set_cuda_error(e, "truncate filter");
    return PS_ERR_CUDA;
  }
  if (!use_top || (int64_t)nc <= P->top_k) return sum_adopt(O, cand, O->n, (int64_t)nc);

  // ---- top-k select
  Buf<SelState> st;
  Buf<ulonglong2> keepk;
  PS_TRY(st.alloc(1, s));
  PS_LAUNCH("k_sel_init", s, k_sel_init<<<1, 1, 0, s>>>(st.p, (unsigned long long)P->top_k));
  int64_t nkeep = 0;
  if (keep && keep->n > 0) {
    std::vector<Rec> hk((size_t)keep->n);
    PS_CUDA(cudaMemcpyAsync(hk.data(), keep->d, hk.size() * sizeof(Rec), cudaMemcpyDeviceToHost, keep->stream));
    PS_CUDA(cudaStreamSynchronize(keep->stream));
    std::vector<ulonglong2> kk(hk.size());
    for (size_t i = 0; i < hk.size(); ++i) kk[i] = make_ulonglong2(hk[i].v, hk[i].w);
    std::sort(kk.begin(), kk.end(), [](const ulonglong2& x, const ulonglong2& y) { return x.x < y.x || (x.x == y.x && x.y < y.y); });
    nkeep = (int64_t)kk.size();
    PS_TRY(keepk.alloc(kk.size(), s));
    PS_CUDA(cudaMemcpyAsync(keepk.p, kk.data(), kk.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice, s));
  }
  int hb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)nc, 256), 4 * nsm));
  // first digit from the filter's histogram; then only candidates with that digit matter
  Buf<uint32_t> list;
  Buf<unsigned long long> n_list;
  PS_TRY(list.alloc((size_t)nc, s));
  PS_TRY(n_list.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(n_list.p, 0, sizeof(unsigned long long), s));
  PS_LAUNCH("k_sel_pick", s, k_sel_pick<<<1, 256, 0, s>>>(st.p, 0, hist.p));
  PS_LAUNCH("k_sel_narrow", s, k_sel_narrow<<<tile_grid((int64_t)nc), kTT, 0, s>>>(ab.p, (int64_t)nc, st.p, list.p, n_list.p));
  // |c|^2 digits first (6 passes); the key digits only matter for exact ties
  for (int pass = 1; pass < kPasses; ++pass) {
    PS_LAUNCH("k_sel_hist", s, k_sel_hist<<<hb, 256, 0, s>>>(cand, ab.p, list.p, n_list.p, st.p, pass, hist.p));
    PS_LAUNCH("k_sel_pick", s, k_sel_pick<<<1, 256, 0, s>>>(st.p, pass, hist.p));
    if (pass == 5 || pass == kPasses - 1) {
      SelState hs;
      PS_CUDA(cudaMemcpyAsync(&hs, st.p, sizeof(hs), cudaMemcpyDeviceToHost, s));
      PS_CUDA(cudaStreamSynchronize(s));
      if (hs.done) break;
    }
  }
  PS_CUDA(cudaGetLastError());
  Rec* outb = nullptr;
  int64_t ocap = (int64_t)nc;  // kept <= top_k + |keep| <= nc
  PS_TRY(dev_alloc((void**)&outb, (size_t)std::max<int64_t>(ocap, 1) * sizeof(Rec), s));
  PS_LAUNCH("k_sel_compact", s, k_sel_compact<<<tile_grid((int64_t)nc), kTT, 0, s>>>(cand, ab.p, (int64_t)nc, st.p, keepk.p, nkeep, outb, cnt.p + 1, 0, DivConst{}, 0));
  e = cudaGetLastError();
  unsigned long long nk = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nk, cnt.p + 1, sizeof(nk), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(cand, s);
  if (e != cudaSuccess) {
    dev_free(outb, s);
    set_cuda_error(e, "truncate select");
    return PS_ERR_CUDA;
  }
  return sum_adopt(O, outb, std::max<int64_t>(ocap, 1), (int64_t)nk);
}

// The conditions of the division-free Lanczos truncation, the divisor aside: top-k alone
// (no weight filter, cutoff or dissipation), FP64, single-component values, more strings than
// kept, 32-bit candidate indices.
bool lanczos_keys_eligible(const pauli_sum* A, const pauli_trunc_policy* P) {
  const int cls = A->cls ? A->cls : kClsComplex;
  return P && P->top_k > 0 && P->max_weight < 0 && !(P->cutoff > 0.0) && P->gamma == 0.0 && !A->f32 &&
         (cls == kClsReal || cls == kClsImag) && A->n > P->top_k && A->n < (int64_t)0xFFFFFFFF &&
         !g_general_truncation;
}

// The Lanczos truncation O = trunc(A / divisor) with rank keys already produced by the norm's
// first pass (exact_norm2_keys); the general path when the conditions do not hold.
int truncate_lanczos_keys(pauli_sum* A, const pauli_trunc_policy* P, double divisor, uint64_t* ab, unsigned* hist) {
  if (lanczos_keys_eligible(A, P) && divisor != 0.0 && std::isfinite(divisor)) {
    TruncArgs a{};
    a.max_weight = -1;
    a.use_div = 1;
    a.dc = make_divconst(divisor);
    a.cls = A->cls;
    const int rc = truncate_div_top(A, P->top_k, a, divisor, ab, hist);
    if (rc != kFallback) return rc;
  }
  return truncate_run(A, P, nullptr, 0.0, &divisor);
}

// Top-k alone (the RK4 stage trim) of a single-component sum from the rank keys |x| that its
// merge wrote: the division-free top-k above with divisor 1 (x / 1 = x, and RN(x^2) is the
// general path's |c|^2 of a single-component string), also for FP32 sums, whose stored values
// are FP32 numbers already; the general path when the conditions do not hold.
int truncate_top_keys(pauli_sum* A, const pauli_trunc_policy* P, uint64_t* ab, unsigned* hist) {
  const int cls = A->cls ? A->cls : kClsComplex;
  const bool ok = P && P->top_k > 0 && P->max_weight < 0 && !(P->cutoff > 0.0) && P->gamma == 0.0 &&
                  (cls == kClsReal || cls == kClsImag) && A->n > P->top_k && A->n < (int64_t)0xFFFFFFFF &&
                  !g_general_truncation && ab && hist;
  if (ok) {
    TruncArgs a{};
    a.max_weight = -1;
    a.use_div = 1;
    a.dc = make_divconst(1.0);
    a.cls = A->cls;
    const int rc = truncate_div_top(A, P->top_k, a, 1.0, ab, hist);
    if (rc != kFallback) return rc;
  }
  return truncate_run(A, P, nullptr, 0.0, nullptr);
}

int round_f32(pauli_sum* s) { return s->f32 ? truncate_run(s, nullptr, nullptr, 0.0, nullptr) : PS_OK; }

}  // namespace ps

extern "C" int pauli_debug_divide(double* x, int64_t n, double b, void* cuda_stream) {
  if (n < 0 || (n > 0 && !x)) return PS_ERR_INVALID;
  if (n == 0) return PS_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ps::ceil_div(n, 256), 4 * ps::num_sms()));
  PS_LAUNCH("k_debug_divide", s, ps::k_debug_divide<<<blocks, 256, 0, s>>>(x, n, ps::make_divconst(b)));
  PS_CUDA(cudaGetLastError());
  PS_CUDA(cudaStreamSynchronize(s));
  return PS_OK;
}

extern "C" int pauli_debug_general_truncation(int on) {
  ps::g_general_truncation = on != 0;
  return PS_OK;
}
