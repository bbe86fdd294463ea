// Most-significant-digit radix select over 192-bit rank keys (|c|^2 or score bits, ~v, ~w):
// shared by the truncation (one select) and the batched truncation (one per instance).
#pragma once

#include "common.cuh"

namespace ps {
namespace {

constexpr int kDigitBits = 11;
constexpr int kBins = 1 << kDigitBits;
constexpr int kPasses = (192 + kDigitBits - 1) / kDigitBits;  // 18

// Digit d (0 = most significant) of the 192-bit rank key (k0, k1, k2), kDigitBits wide.
__device__ __forceinline__ uint32_t rank_digit(const uint64_t k[3], int d) {
  int hi = 192 - d * kDigitBits;  // bits [lo, hi), bit 0 = LSB of k2
  int lo = max(hi - kDigitBits, 0);
  uint32_t out = 0;
  for (int b = hi - 1; b >= lo; --b) {
    uint64_t word = b >= 128 ? k[0] : (b >= 64 ? k[1] : k[2]);
    out = (out << 1) | (uint32_t)((word >> (b & 63)) & 1);
  }
  return out;
}

// Rank key: (|c|^2 bits, ~v, ~w); larger key = kept first (larger |c|, then smaller v, w).
__device__ __forceinline__ void rank_key(uint64_t a2, const Rec* r, uint64_t k[3]) {
  k[0] = a2;
  k[1] = r ? ~r->v : 0;
  k[2] = r ? ~r->w : 0;
}

// Select state: the digits fixed so far, the rank still needed inside the current prefix.
struct SelState {
  uint64_t prefix[3];   // fixed high bits of the threshold (others zero)
  unsigned long long need;
  int done;
  int pass;
  int exact;            // 1: never stop early (every digit of the need-th key is fixed)
};

__device__ __forceinline__ bool matches_prefix(const uint64_t k[3], const SelState& st, int pass) {
  int nbits = min(pass * kDigitBits, 192);  // high bits already fixed
  for (int w = 0; w < 3; ++w) {
    int wb = nbits - 64 * w;  // fixed bits in this word
    if (wb <= 0) break;
    uint64_t m = wb >= 64 ? ~0ull : (~0ull << (64 - wb));
    if ((k[w] & m) != (st.prefix[w] & m)) return false;
  }
  return true;
}

// Pick the digit of the need-th largest key in the current prefix (called by every thread of
// one block of 256): a block-wide scan of the histogram from the top bin down finds the one
// bin b with above(b) < need <= above(b) + hist(b); the histogram is cleared for the next
// pass.
__device__ __forceinline__ void sel_pick_block(SelState* st_p, int pass, unsigned* __restrict__ hist) {
  constexpr int per = kBins / 256;
  __shared__ unsigned long long s_w[8];
  __shared__ int s_sel;
  __shared__ unsigned long long s_above;
  const SelState st = *st_p;
  if (st.done) return;
  const int hi = 192 - pass * kDigitBits;
  const int width = min(kDigitBits, hi);
  const int top = (1 << width) - 1;
  const int t = threadIdx.x;
  // thread t owns ranks r = t*per .. t*per+per-1, rank r = bin (top - r)
  unsigned h[per];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    int b = top - (t * per + k);
    h[k] = b >= 0 ? hist[b] : 0u;
    sum += h[k];
  }
  __syncthreads();
  for (int i = t; i < kBins; i += 256) hist[i] = 0;  // ready for the next pass
  int lane = t & 31, warp = t >> 5;
  unsigned long long incl = sum;
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) s_w[warp] = incl;
  if (t == 0) s_sel = -1;
  __syncthreads();
  unsigned long long run = incl - sum;
  for (int k = 0; k < warp; ++k) run += s_w[k];
  for (int k = 0; k < per; ++k) {
    int b = top - (t * per + k);
    if (b >= 0 && run < st.need && st.need <= run + h[k]) {
      s_sel = b;
      s_above = run;
    }
    run += h[k];
  }
  __syncthreads();
  if (t == 0 && s_sel >= 0) {
    const int sel = s_sel;
    const int lo = hi - width;
    for (int j = 0; j < width; ++j) {
      int b = lo + j;  // bit index counted from LSB of k2
      if ((sel >> j) & 1) {
        int word = b >= 128 ? 0 : (b >= 64 ? 1 : 2);
        st_p->prefix[word] |= 1ull << (b & 63);
      }
    }
    st_p->need = st.need - s_above;
    st_p->pass = pass + 1;
  }
  __syncthreads();
  // the selected bin's count decides whether every key in it is kept
  for (int k = 0; k < per; ++k) {
    int b = top - (t * per + k);
    if (b >= 0 && b == s_sel) {
      const int lo = hi - width;
      if (lo == 0 || (!st.exact && h[k] == st.need - s_above)) st_p->done = 1;
    }
  }
}

// Order-keeping compaction of a tile of TT * TI elements (element k * TT + thread of the tile
// at f[k]): one output reservation per tile, positions in tile order, so runs of neighbouring
// strings stay neighbours in the output (the emission's slot reservations rely on it).
template <int TT, int TI>
struct TileSlots {
  uint32_t wcnt[TT / 32][TI];
  unsigned long long base;
};

template <int TT, int TI>
__device__ __forceinline__ void tile_slots(const bool (&f)[TI], TileSlots<TT, TI>& sm, unsigned long long* counter,
                                           unsigned long long (&pos)[TI]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned m[TI];
#pragma unroll
  for (int k = 0; k < TI; ++k) {
    m[k] = __ballot_sync(0xffffffffu, f[k]);
    if (lane == 0) sm.wcnt[warp][k] = __popc(m[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int k = 0; k < TI; ++k)
      for (int w = 0; w < TT / 32; ++w) {
        const uint32_t c = sm.wcnt[w][k];
        sm.wcnt[w][k] = run;
        run += c;
      }
    sm.base = run ? atomicAdd(counter, (unsigned long long)run) : 0ull;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TI; ++k) pos[k] = sm.base + sm.wcnt[warp][k] + __popc(m[k] & ((1u << lane) - 1));
  __syncthreads();
}

}  // namespace
}  // namespace ps
