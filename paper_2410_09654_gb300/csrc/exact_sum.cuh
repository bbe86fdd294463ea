// Exact summation of products of doubles with integer arithmetic (shared by the exact
// reductions and the allocation-free trace product).
//
// Every product of two doubles is an integer (the product of the two 53-bit significands,
// 64x64->128 bit) times a power of two.  A thread adds these integers into a 256-bit
// two's-complement register window anchored below the largest product's top bit; terms
// reaching below the window go, exactly, into a full-range accumulator of 32-bit digits
// held in 64-bit counters.  Integer addition is associative, so the result does not
// depend on the order of the terms; the host rounds the final integer once to the
// nearest double (ties to even).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ps {
namespace exact {

constexpr int kFullDigits = 160;   // digit i has weight 2^(32 i - kBias)
constexpr int kBias = 2368;        // multiple of 32; below the smallest product bit (2^-2252)
constexpr int kWinDigits = 8;      // 256-bit window as 8 signed 32-bit digits
constexpr int kRedThreads = 256;

struct Split {
  uint64_t m;  // significand (< 2^53), 0 for zero
  int e;       // value = m * 2^e
};

__device__ __forceinline__ Split split_double(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  uint64_t frac = b & ((1ull << 52) - 1);
  int ex = (int)((b >> 52) & 0x7FF);
  Split s;
  if (ex == 0) {
    s.m = frac;
    s.e = -1074;
  } else {
    s.m = frac | (1ull << 52);
    s.e = ex - 1075;
  }
  return s;
}

__device__ __forceinline__ bool neg_double(double x) { return __double_as_longlong(x) < 0; }

// Top bit position (exclusive bound) of the product x*y: e_x + e_y + 106, or INT_MIN if zero.
__device__ __forceinline__ int prod_top(double x, double y) {
  if (is_zero(x) || is_zero(y)) return -100000;
  Split a = split_double(x), b = split_double(y);
  return a.e + b.e + 106;
}

// Markers of the exponent bound for sums holding a non-finite coefficient (above every
// finite bound; NaN above Inf so that atomicMax keeps it): the result is then +Inf or NaN,
// as the IEEE sum would be, and the accumulation pass does nothing.
constexpr int kTopInf = 1 << 29, kTopNaN = (1 << 29) + 1;

__device__ __forceinline__ int nonfinite_top(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if (((b >> 52) & 0x7FF) != 0x7FF) return -100000;
  return (b & ((1ull << 52) - 1)) ? kTopNaN : kTopInf;
}

struct Win {
  uint64_t w[4];  // 256-bit two's complement
};

__device__ __forceinline__ void win_add(Win& acc, const uint64_t t[4]) {
  asm("add.cc.u64 %0, %0, %4;\n\t"
      "addc.cc.u64 %1, %1, %5;\n\t"
      "addc.cc.u64 %2, %2, %6;\n\t"
      "addc.u64 %3, %3, %7;"
      : "+l"(acc.w[0]), "+l"(acc.w[1]), "+l"(acc.w[2]), "+l"(acc.w[3])
      : "l"(t[0]), "l"(t[1]), "l"(t[2]), "l"(t[3]));
}

// Add +-(ma*mb) * 2^pos (pos relative to the full-range digit grid origin, i.e. absolute
// exponent + kBias) to the full-range accumulator.
__device__ __forceinline__ void full_add(long long* full, uint64_t lo, uint64_t hi, int pos, bool neg) {
  int d = pos >> 5, sh = pos & 31;
  // shift the 128-bit product left by sh into 160 bits, then cut 32-bit digits
  uint64_t l2 = lo << sh;
  uint64_t h2 = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
  uint64_t top = sh ? (hi >> (64 - sh)) : 0;
  uint32_t dig[5] = {(uint32_t)l2, (uint32_t)(l2 >> 32), (uint32_t)h2, (uint32_t)(h2 >> 32), (uint32_t)top};
#pragma unroll
  for (int k = 0; k < 5; ++k)
    if (dig[k]) atomicAdd((unsigned long long*)&full[d + k], neg ? (unsigned long long)(-(long long)dig[k]) : (unsigned long long)dig[k]);
}

// Add the exact product x*y (sign included) to the window (bit 0 at absolute exponent wlo)
// or, when it reaches below the window, to the full-range accumulator.
__device__ __forceinline__ void add_product(Win& acc, double x, double y, int wlo, long long* full) {
  if (is_zero(x) || is_zero(y)) return;
  Split a = split_double(x), b = split_double(y);
  bool neg = neg_double(x) != neg_double(y);
  uint64_t lo = a.m * b.m;
  uint64_t hi = __umul64hi(a.m, b.m);
  int off = a.e + b.e - wlo;
  if (off < 0) {
    full_add(full, lo, hi, a.e + b.e + kBias, neg);
    return;
  }
  // off + 106 <= 222 by the choice of the window, so the term spans words 0..2
  int word = off >> 6, sh = off & 63;
  uint64_t s0 = lo << sh;
  uint64_t s1 = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
  uint64_t s2 = sh ? (hi >> (64 - sh)) : 0;
  uint64_t t[4] = {0, 0, 0, 0};
  if (word == 0) { t[0] = s0; t[1] = s1; t[2] = s2; }
  else if (word == 1) { t[1] = s0; t[2] = s1; t[3] = s2; }
  else { t[2] = s0; t[3] = s1; }
  if (neg) {  // two's complement negate
    t[0] = ~t[0]; t[1] = ~t[1]; t[2] = ~t[2]; t[3] = ~t[3];
    uint64_t one[4] = {1, 0, 0, 0};
    Win tmp{{t[0], t[1], t[2], t[3]}};
    win_add(tmp, one);
    t[0] = tmp.w[0]; t[1] = tmp.w[1]; t[2] = tmp.w[2]; t[3] = tmp.w[3];
  }
  win_add(acc, t);
}

// Reduce the windows of a block and add them, as signed 32-bit digits, to the global window.
__device__ __forceinline__ void block_flush(Win acc, long long* gwin) {
  __shared__ long long s_dig[kWinDigits];
  if (threadIdx.x < kWinDigits) s_dig[threadIdx.x] = 0;
  __syncthreads();
  // warp reduce with carries (256-bit adds)
  for (int d = 16; d > 0; d >>= 1) {
    uint64_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = __shfl_down_sync(0xffffffffu, acc.w[k], d);
    win_add(acc, o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t lo = (uint32_t)acc.w[k], hi = (uint32_t)(acc.w[k] >> 32);
      long long dhi = (k == 3) ? (long long)(int32_t)hi : (long long)hi;  // top digit is signed
      atomicAdd((unsigned long long*)&s_dig[2 * k], (unsigned long long)(long long)lo);
      atomicAdd((unsigned long long*)&s_dig[2 * k + 1], (unsigned long long)dhi);
    }
  }
  __syncthreads();
  if (threadIdx.x < kWinDigits && s_dig[threadIdx.x])
    atomicAdd((unsigned long long*)&gwin[threadIdx.x], (unsigned long long)s_dig[threadIdx.x]);
}

__device__ __forceinline__ uint64_t mix_key(uint64_t v, uint64_t w) { return key_hash64(v, w); }

__device__ __forceinline__ ulonglong2 cas128_g(ulonglong2* p, ulonglong2 expect, ulonglong2 desired) {
  ulonglong2 old;
  asm volatile(
      "{\n\t.reg .b128 d, b, c;\n\t"
      "mov.b128 b, {%2, %3};\n\t"
      "mov.b128 c, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], b, c;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(old.x), "=l"(old.y)
      : "l"(expect.x), "l"(expect.y), "l"(desired.x), "l"(desired.y), "l"(p)
      : "memory");
  return old;
}

__device__ __forceinline__ int64_t tp_find(const ulonglong2* tkey, const int64_t* tidx, uint64_t tmask,
                                           long long ones_idx, uint64_t v, uint64_t w) {
  if (v == ~0ull && w == ~0ull) return ones_idx;
  uint64_t slot = mix_key(v, w) & tmask;
  for (uint64_t p = 0; p <= tmask; ++p) {
    ulonglong2 k = tkey[slot];
    if (k.x == v && k.y == w) return tidx[slot];
    if (k.x == ~0ull && k.y == ~0ull) return -1;
    slot = (slot + 1) & tmask;
  }
  return -1;
}

// ---------------------------------------------------------------- host rounding
// Combine window digits (weight 2^(wlo + 32 k)) and full-range digits (weight 2^(32 i - kBias))
// into one exact integer and round it to the nearest double, ties to even.
inline double round_exact(const std::vector<long long>& full_in, const long long* win, int wlo) {
  const int n = kFullDigits + 4;
  std::vector<__int128> dig(n, 0);
  for (int i = 0; i < kFullDigits; ++i) dig[i] = full_in[i];
  if (win) {
    int base = (wlo + kBias) / 32;
    for (int k = 0; k < kWinDigits; ++k) dig[base + k] += win[k];
  }
  // normalise to base 2^32 digits with a signed top
  for (int i = 0; i + 1 < n; ++i) {
    __int128 q = dig[i] >> 32;  // floor
    dig[i] -= q << 32;
    dig[i + 1] += q;
  }
  bool neg = dig[n - 1] < 0;
  if (neg) {
    for (int i = 0; i < n; ++i) dig[i] = -dig[i];
    for (int i = 0; i + 1 < n; ++i) {
      __int128 q = dig[i] >> 32;
      dig[i] -= q << 32;
      dig[i + 1] += q;
    }
  }
  // most significant set bit
  int msd = -1;
  for (int i = n - 1; i >= 0; --i)
    if (dig[i] != 0) { msd = i; break; }
  if (msd < 0) return 0.0;
  uint32_t top = (uint32_t)dig[msd];
  int topbit = msd * 32 + 31 - __builtin_clz(top);
  auto bit_at = [&](int b) -> uint32_t { return b < 0 ? 0u : (uint32_t)((uint64_t)dig[b >> 5] >> (b & 31)) & 1u; };
  int lsb = topbit - 52;
  if (lsb < kBias - 1074) lsb = kBias - 1074;  // subnormal spacing
  uint64_t mant = 0;
  for (int b = topbit; b >= lsb; --b) mant = (mant << 1) | bit_at(b);
  uint32_t half = bit_at(lsb - 1);
  bool rest = false;
  for (int b = lsb - 2; b >= 0 && !rest; --b) {
    if ((b & 31) == 31 && dig[b >> 5] == 0) { b -= 31; continue; }
    rest = bit_at(b) != 0;
  }
  if (half && (rest || (mant & 1))) ++mant;
  double r = std::ldexp((double)mant, lsb - kBias);
  return neg ? -r : r;
}


}  // namespace exact
}  // namespace ps
