// Learned truncation scorer: a two-layer ReLU network on string features, trained and
// evaluated with hand-written BF16 tensor-core kernels (FP32 accumulation), with an FP32
// Adam update.  The paper's conclusion proposes predicting the importance of strings with
// machine learning rather than ranking them by |c| alone; the model is this library's:
//
//   features (80): x0 = wt/N (wt = popcount(v|w)), x1 = extent/N (last - first + 1 over the
//     non-identity sites, 0 for the identity), x2 = ln(max(|c|, 1e-300))/16, and for each
//     of 16 site bins (site j in bin floor(16 j / N)) the fractions of its sites holding
//     I, X, Y, Z (x[3 + 4b + t]); x[67..79] = 0.
//   z = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, W1 128x80, W2 128x128 (rows = outputs).
//   loss: mean binary cross-entropy on z; update: bias-corrected Adam.
//   truncation score: ln|c| - gamma dt wt + z (ln|c| after the dissipation factor), ranked
//     through the order-equivalent rank value |c|^2 e^(2 (z - gamma dt wt)), which is |c|^2
//     itself when the exponent is zero.
//
// Only the rank value's |c|^2 and one product are FP64 (the FP64 rate of this part is low):
// ln|c| for the feature is FP32 from the exponent and leading mantissa bits of the larger
// component, and the rescaling factor is a power of two times exp2 of a fraction in FP32.
//
// Inference (the scorer inside the RK4 step) runs on tcgen05.mma with TMEM accumulators
// (k_mlp_fwd_tc).  Training runs on mma.sync m16n8k16 (bf16 in, fp32 accumulate): each warp
// owns 16 rows; the accumulator of one layer is repacked in registers as the A operand of the
// next (the m16n8 C layout of two adjacent column tiles is the m16k16 A layout).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "exact_sum.cuh"

namespace ps {
namespace {

constexpr int kF = 80;
constexpr int kHid = 128;
constexpr int oW1 = 0, oB1 = kHid * kF, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kHid;
constexpr int kParams = oB3 + 1;  // 27009
constexpr int kSF = kF + 8;       // shared row stride (bf16) of K = 80 rows: 44 words, conflict-free fragments
constexpr int kSH = kHid + 8;     // of K = 128 rows: 68 words
constexpr int kTrainRows = 64;    // rows per training tile (4 warps x 16)
constexpr int kSR = kTrainRows + 8;  // stride of the transposed (row-contiguous) tiles: 36 words

struct FeatConst {
  uint64_t bin_mask[16];
  int bin_size[16];
  float inv_size[16];  // 1 / bin size (0 for an empty bin)
  float inv_n;         // 1 / N
  int n_sites;
  float x2_floor;  // ln(1e-300) / 16
  float ln2;       // ln 2
  float log2e;     // log2(e)
};

FeatConst make_featconst(int n) {
  FeatConst f{};
  f.n_sites = n;
  f.x2_floor = (float)(std::log(1e-300) / 16.0);
  f.ln2 = (float)std::log(2.0);
  f.log2e = (float)(1.0 / std::log(2.0));
  for (int j = 0; j < n; ++j) {
    const int b = (16 * j) / n;
    f.bin_mask[b] |= 1ull << j;
    f.bin_size[b] += 1;
  }
  for (int b = 0; b < 16; ++b) f.inv_size[b] = f.bin_size[b] ? (float)(1.0 / f.bin_size[b]) : 0.0f;
  f.inv_n = (float)(1.0 / n);
  return f;
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}

__device__ __forceinline__ bool bf16_pos(uint32_t pair, int half) {
  const uint32_t h = (pair >> (16 * half)) & 0xFFFFu;
  return h != 0 && (h & 0x8000u) == 0;
}

// ln(max(|c|, 1e-300)) / 16 in FP32: with a = max(|re|, |im|) = m 2^e (m in [1, 2), from the
// leading 23 mantissa bits) and b the other component, ln|c| = e ln 2 + ln m + ln(1 + (b/a)^2)/2.
// Integer and FP32 operations only.
__device__ __forceinline__ float feature_lnc(double re, double im, const FeatConst& fc) {
  const uint64_t ua = (uint64_t)__double_as_longlong(re) & 0x7FFFFFFFFFFFFFFFull;
  const uint64_t ub = (uint64_t)__double_as_longlong(im) & 0x7FFFFFFFFFFFFFFFull;
  const uint64_t hi = ua > ub ? ua : ub, lo = ua > ub ? ub : ua;  // non-negative doubles order like bits
  if (hi < 0x01A56E1FC2F8F359ull) return fc.x2_floor;              // below 1e-300 (and zeros)
  const int ea = (int)(hi >> 52), el = (int)(lo >> 52);
  const float mh = __int_as_float(0x3F800000 | (int)((hi >> 29) & 0x7FFFFF));
  float r = 0.0f;
  if (el > 0 && ea - el < 60) {
    const float ml = __int_as_float(0x3F800000 | (int)((lo >> 29) & 0x7FFFFF));
    r = ldexpf(__fdiv_rn(ml, mh), el - ea);
  }
  const float lnc = (float)(ea - 1023) * fc.ln2 + logf(mh) + 0.5f * log1pf(r * r);
  return lnc * 0.0625f;
}

// Rank value |c|^2 e^(2 (z - gdt wt)): exactly q = |c|^2 when the exponent is zero; otherwise
// q * exp2(f) * 2^k with t = 2 (z - gdt wt) log2(e) = k + f, k integer, f in [0, 1).  FP64
// work: the squares of the non-zero components and one product (the FP32 factor in [1, 2)
// is widened and the power of two applied on the integer pipe when the result stays normal).
__device__ __forceinline__ double rank_value(double re, double im, float z, float gdt_wt, const FeatConst& fc) {
  const bool zr = ((uint64_t)__double_as_longlong(re) << 1) == 0, zi = ((uint64_t)__double_as_longlong(im) << 1) == 0;
  if (zr && zi) return 0.0;
  const double q = zi ? __dmul_rn(re, re) : (zr ? __dmul_rn(im, im) : __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)));
  float t = 2.0f * (z - gdt_wt);
  if (t == 0.0f) return q;
  t = fminf(fmaxf(t * fc.log2e, -2000.0f), 2000.0f);
  const float kf = floorf(t);
  const int k = (int)kf;
  const uint32_t fb = (uint32_t)__float_as_int(exp2f(t - kf));  // in [1, 2]
  double mul;
  if ((fb >> 23) == 127u) {
    mul = __longlong_as_double((long long)((0x3FFull << 52) | ((uint64_t)(fb & 0x7FFFFF) << 29)));
  } else {
    mul = (double)__int_as_float((int)fb);  // exp2f rounded up to exactly 2
  }
  const double p = __dmul_rn(q, mul);
  const uint64_t pb = (uint64_t)__double_as_longlong(p);
  const int e = (int)((pb >> 52) & 0x7FF);
  if (e > 0 && e + k >= 1 && e + k <= 2046) return __longlong_as_double((long long)(pb + ((uint64_t)(int64_t)k << 52)));
  return scalbn(p, k);
}

// Feature k of a string (0 <= k < 80); k is a compile-time constant at every call, so the
// branches fold.  Fractions are products with the reciprocal (within one FP32 unit of the
// quotient, below BF16 resolution).
__device__ __forceinline__ float feature(const Rec& r, const FeatConst& fc, int k) {
  const uint64_t s = r.v | r.w;
  if (k == 0) return (float)__popcll(s) * fc.inv_n;
  if (k == 1) {
    const int ext = s ? (63 - __clzll((long long)s)) - (__ffsll((long long)s) - 1) + 1 : 0;
    return (float)ext * fc.inv_n;
  }
  if (k == 2) return feature_lnc(r.re, r.im, fc);
  if (k >= 67) return 0.0f;
  const int b = (k - 3) >> 2, t = (k - 3) & 3;
  const uint64_t m = fc.bin_mask[b];
  int c;
  if (t == 1) c = __popcll(r.w & ~r.v & m);
  else if (t == 2) c = __popcll(r.v & r.w & m);
  else if (t == 3) c = __popcll(r.v & ~r.w & m);
  else c = fc.bin_size[b] - __popcll(s & m);
  return (float)c * fc.inv_size[b];
}

// Features [44 HALF, 44 HALF + 44) (HALF 0) or [44, 80) (HALF 1) of one string, stored as
// BF16 pairs into a shared row (and optionally a global row and a transposed shared tile).
template <int HALF>
__device__ __forceinline__ void store_features(const Rec& r, bool valid, const FeatConst& fc, uint16_t* xs_row,
                                               uint16_t* x_glob, uint16_t* xT, int sr, int row) {
  constexpr int k0 = HALF ? 44 : 0, k1 = HALF ? 80 : 44;
#pragma unroll
  for (int k = k0; k < k1; k += 2) {
    const float f0 = valid ? feature(r, fc, k) : 0.0f, f1 = valid ? feature(r, fc, k + 1) : 0.0f;
    const uint32_t pr = pack_bf16(f0, f1);
    *reinterpret_cast<uint32_t*>(xs_row + k) = pr;
    if (x_glob) *reinterpret_cast<uint32_t*>(x_glob + k) = pr;
    if (xT) {
      xT[k * sr + row] = (uint16_t)(pr & 0xFFFFu);
      xT[(k + 1) * sr + row] = (uint16_t)(pr >> 16);
    }
  }
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragment (16 x 16) of a row-major bf16 tile with row stride S.
template <int S>
__device__ __forceinline__ void load_a(const uint16_t* base, int r0, int k0, int g, int t, uint32_t (&a)[4]) {
  a[0] = ld32(base + (r0 + g) * S + k0 + 2 * t);
  a[1] = ld32(base + (r0 + g + 8) * S + k0 + 2 * t);
  a[2] = ld32(base + (r0 + g) * S + k0 + 2 * t + 8);
  a[3] = ld32(base + (r0 + g + 8) * S + k0 + 2 * t + 8);
}

// B fragment (16 x 8) from an [n][k] tile (k contiguous) with row stride S.
template <int S>
__device__ __forceinline__ void load_b(const uint16_t* base, int n0, int k0, int g, int t, uint32_t& b0,
                                       uint32_t& b1) {
  b0 = ld32(base + (n0 + g) * S + k0 + 2 * t);
  b1 = ld32(base + (n0 + g) * S + k0 + 2 * t + 8);
}

// B fragments of two adjacent n tiles (n0..n0+7 and n0+8..n0+15) at k0 with one ldmatrix.x4:
// lane L supplies the row address of matrix L/8 (tile (L/16), k half (L/8)&1), 16-byte
// aligned (S even multiples of 8 elements, k0 a multiple of 8).
template <int S>
__device__ __forceinline__ void load_b2(const uint16_t* base, int n0, int k0, int lane, uint32_t& b0a, uint32_t& b1a,
                                        uint32_t& b0b, uint32_t& b1b) {
  const int mtx = lane >> 3, row = lane & 7;
  const uint16_t* p = base + (n0 + ((mtx >> 1) << 3) + row) * S + k0 + ((mtx & 1) << 3);
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(b0a), "=r"(b1a), "=r"(b0b), "=r"(b1b)
               : "r"(addr));
}

// Copy a dense [rows][cols] bf16 matrix into shared memory with row stride S.
template <int S>
__device__ __forceinline__ void stage(uint16_t* dst, const uint16_t* __restrict__ src, int rows, int cols) {
  const int words = cols / 2;
  for (int i = threadIdx.x; i < rows * words; i += blockDim.x) {
    const int r = i / words, c = i - r * words;
    reinterpret_cast<uint32_t*>(dst + r * S)[c] = reinterpret_cast<const uint32_t*>(src + r * cols)[c];
  }
}

// Layer 1 and 2 of one warp's 16 rows: returns relu(layer 2) in acc2 (fp32, C layout) and
// relu(layer 1) packed as bf16 A fragments in h1.
__device__ __forceinline__ void forward_rows(const uint16_t* xs, int r0, const uint16_t* W1s, const uint16_t* W2s,
                                             const float* fb1, const float* fb2, int g, int t, uint32_t (&h1)[8][4],
                                             float (&acc2)[16][4]) {
  float acc[16][4];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int ks = 0; ks < kF / 16; ++ks) {
    uint32_t a[4];
    load_a<kSF>(xs, r0, 16 * ks, g, t, a);
#pragma unroll
    for (int np = 0; np < 8; ++np) {
      uint32_t b0, b1, b2, b3;
      load_b2<kSF>(W1s, 16 * np, 16 * ks, lane, b0, b1, b2, b3);
      mma_bf16(acc[2 * np], a, b0, b1);
      mma_bf16(acc[2 * np + 1], a, b2, b3);
    }
  }
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nt = 2 * ks + h, c = 8 * nt + 2 * t;
      const float e0 = fmaxf(acc[nt][0] + fb1[c], 0.0f), e1 = fmaxf(acc[nt][1] + fb1[c + 1], 0.0f);
      const float e2 = fmaxf(acc[nt][2] + fb1[c], 0.0f), e3 = fmaxf(acc[nt][3] + fb1[c + 1], 0.0f);
      h1[ks][2 * h] = pack_bf16(e0, e1);
      h1[ks][2 * h + 1] = pack_bf16(e2, e3);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) acc2[j][0] = acc2[j][1] = acc2[j][2] = acc2[j][3] = 0.0f;
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {
#pragma unroll
    for (int np = 0; np < 8; ++np) {
      uint32_t b0, b1, b2, b3;
      load_b2<kSH>(W2s, 16 * np, 16 * ks, lane, b0, b1, b2, b3);
      mma_bf16(acc2[2 * np], h1[ks], b0, b1);
      mma_bf16(acc2[2 * np + 1], h1[ks], b2, b3);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    const int c = 8 * nt + 2 * t;
    acc2[nt][0] = fmaxf(acc2[nt][0] + fb2[c], 0.0f);
    acc2[nt][1] = fmaxf(acc2[nt][1] + fb2[c + 1], 0.0f);
    acc2[nt][2] = fmaxf(acc2[nt][2] + fb2[c], 0.0f);
    acc2[nt][3] = fmaxf(acc2[nt][3] + fb2[c + 1], 0.0f);
  }
}

// z for rows g and g+8 (every lane of the quad gets both).
__device__ __forceinline__ void output_rows(const float (&h2)[16][4], const float* fw3, float b3, int t, float& zg,
                                            float& zg8) {
  float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    const int c = 8 * nt + 2 * t;
    s0 += h2[nt][0] * fw3[c] + h2[nt][1] * fw3[c + 1];
    s1 += h2[nt][2] * fw3[c] + h2[nt][3] * fw3[c + 1];
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  zg = s0 + b3;
  zg8 = s1 + b3;
}

struct MlpDev {
  const uint16_t* w1b;   // [128][80] bf16
  const uint16_t* w2b;   // [128][128] bf16 (rows = outputs)
  const uint16_t* w2tb;  // [128][128] bf16, transposed
  const float* p;        // FP32 master parameters
};

// ---------------------------------------------------------------- inference on tcgen05
// The same network on the fifth-generation tensor cores: per tile of 128 strings, the BF16
// operands sit in shared memory in the no-swizzle K-major layout of tcgen05.mma (8-row x
// 16-byte core matrices: core (r/8, k/8) of a [rows][K] tile at ((r/8)(K/8) + k/8) 128 bytes,
// row r%8 at 16 (r%8), element k%8 at 2 (k%8); descriptors: leading offset 128 bytes between
// cores along K, stride offset (K/8) 128 bytes between cores along M or N), one thread issues
// the M = N = 128 products (K = 80 in five steps of 16, then K = 128 in eight), the FP32
// accumulators live in tensor memory (columns 0..127 layer 1, 128..255 layer 2, one lane per
// string), and every thread reads its string's row back with tcgen05.ld for the bias, ReLU and
// output epilogues.  Completion goes through an mbarrier whose waits are bounded: a wait that
// gives up sets *err and the kernel stops cleanly.
constexpr int kTcRows = 128;
constexpr uint32_t kTcCols = 256;                   // tensor-memory columns per block
constexpr int kTcA1 = kTcRows * kF * 2;             // bytes: features tile [128][80]
constexpr int kTcA2 = kTcRows * kHid * 2;           // h1 tile [128][128]
constexpr int kTcW1 = kHid * kF * 2;                // W1 [128][80]
constexpr int kTcW2 = kHid * kHid * 2;              // W2 [128][128]
constexpr int kTcOffA1 = 0, kTcOffA2 = kTcOffA1 + kTcA1, kTcOffW1 = kTcOffA2 + kTcA2, kTcOffW2 = kTcOffW1 + kTcW1,
              kTcOffF = kTcOffW2 + kTcW2;
constexpr size_t kTcSmem = (size_t)kTcOffF + 3 * kHid * 4 + 2 * kTcRows * 4 + 64 + 1024;  // + alignment slack
constexpr long long kTcWaitLimit = 1ll << 26;       // try_wait rounds before a wait gives up

__device__ __forceinline__ uint32_t core_off(int r, int k, int K) {  // byte offset in a core-matrix tile
  return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // version 1, no swizzle
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N = 128, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
               ::"r"(dtm), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc)
               : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Wait for the mbarrier phase with the given parity; false when the bounded wait gave up.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Features [k0, k1) of one string as BF16 pairs into its row of the core-matrix feature tile.
template <int HALF>
__device__ __forceinline__ void store_features_tc(const Rec& r, bool valid, const FeatConst& fc, unsigned char* a1,
                                                  int row, uint16_t* x_glob) {
  constexpr int k0 = HALF ? 44 : 0, k1 = HALF ? 80 : 44;
#pragma unroll
  for (int k = k0; k < k1; k += 2) {
    const float f0 = valid ? feature(r, fc, k) : 0.0f, f1 = valid ? feature(r, fc, k + 1) : 0.0f;
    const uint32_t pr = pack_bf16(f0, f1);
    *reinterpret_cast<uint32_t*>(a1 + core_off(row, k, kF)) = pr;
    if (x_glob) *reinterpret_cast<uint32_t*>(x_glob + k) = pr;
  }
}

__global__ void __launch_bounds__(256, 2) k_mlp_fwd_tc(const Rec* __restrict__ d, int64_t n, FeatConst fc, MlpDev m,
                                                    double gamma_dt, uint16_t* __restrict__ x_out,
                                                    float* __restrict__ z_out, double* __restrict__ score_out,
                                                    int* __restrict__ err, int no_products, long long wait_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* a1 = sm + kTcOffA1;
  unsigned char* a2 = sm + kTcOffA2;
  unsigned char* w1 = sm + kTcOffW1;
  unsigned char* w2 = sm + kTcOffW2;
  float* fb1 = reinterpret_cast<float*>(sm + kTcOffF);
  float* fb2 = fb1 + kHid;
  float* fw3 = fb2 + kHid;
  float* zpart = fw3 + kHid;                                   // [2][128] partial output sums
  uint64_t* mbar = reinterpret_cast<uint64_t*>(zpart + 2 * kTcRows);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // weights into the core-matrix layout (B operands: [n][k], K contiguous), biases, w3
  for (int i = tid; i < kHid * kF / 2; i += blockDim.x) {
    const int nn = (2 * i) / kF, k = (2 * i) % kF;
    *reinterpret_cast<uint32_t*>(w1 + core_off(nn, k, kF)) = reinterpret_cast<const uint32_t*>(m.w1b)[i];
  }
  for (int i = tid; i < kHid * kHid / 2; i += blockDim.x) {
    const int nn = (2 * i) / kHid, k = (2 * i) % kHid;
    *reinterpret_cast<uint32_t*>(w2 + core_off(nn, k, kHid)) = reinterpret_cast<const uint32_t*>(m.w2b)[i];
  }
  for (int i = tid; i < kHid; i += blockDim.x) {
    fb1[i] = m.p[oB1 + i];
    fb2[i] = m.p[oB2 + i];
    fw3[i] = m.p[oW3 + i];
  }
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(mbar);
  if (tid == 0) {
    *s_err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // tensor memory: 256 columns (two accumulators of 128 x 128 FP32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(tmem_slot)), "r"(kTcCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sa1 = (uint32_t)__cvta_generic_to_shared(a1), sa2 = (uint32_t)__cvta_generic_to_shared(a2);
  const uint32_t sw1 = (uint32_t)__cvta_generic_to_shared(w1), sw2 = (uint32_t)__cvta_generic_to_shared(w2);
  const float b3 = m.p[oB3];
  const float gdt_f = (float)gamma_dt;
  const int row = 32 * (warp & 3) + lane;   // this thread's string (tensor-memory lane) in the tile
  const int half = warp >> 2;                 // accumulator columns [64 half, 64 half + 64)
  const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
  uint32_t parity = 0;
  const int64_t tiles = ceil_div_dev(n, kTcRows);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t base = tile * kTcRows;
    {  // features: two warps per 32 strings (the even warp 0..43, the odd one 44..79)
      const int frow = (warp >> 1) * 32 + lane;
      const int64_t i = base + frow;
      Rec r{0, 0, 0.0, 0.0};
      const bool valid = i < n;
      if (valid) r = d[i];
      uint16_t* xg = (x_out && valid) ? x_out + i * kF : nullptr;
      if (warp & 1) store_features_tc<1>(r, valid, fc, a1, frow, xg);
      else store_features_tc<0>(r, valid, fc, a1, frow, xg);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0 && !no_products) {  // layer 1: D1 = X W1^T, K = 80
#pragma unroll
      for (int ks = 0; ks < kF / 16; ++ks)
        tc_mma(tmem, umma_desc(sa1 + ks * 256, 128, (kF / 8) * 128), umma_desc(sw1 + ks * 256, 128, (kF / 8) * 128),
               ks > 0);
      tc_commit(mbar_a);
    }
    if (!tc_wait(mbar_a, parity, wait_limit)) atomicOr(s_err, 1);
    parity ^= 1u;
    tc_after_sync();
    tc_before_sync();
    __syncthreads();  // every thread has seen the wait's outcome
    tc_after_sync();
    if (*s_err) break;
    {  // epilogue 1: relu(D1 + b1) as BF16 into the h1 tile (this thread's row, 64 columns)
      for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
        float v[16];
        tc_ld16(tmem + lane_addr + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const float e0 = fmaxf(v[j] + fb1[c0 + j], 0.0f), e1 = fmaxf(v[j + 1] + fb1[c0 + j + 1], 0.0f);
          *reinterpret_cast<uint32_t*>(a2 + core_off(row, c0 + j, kHid)) = pack_bf16(e0, e1);
        }
      }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (*s_err) break;
    if (tid == 0) {  // layer 2: D2 = H1 W2^T, K = 128
#pragma unroll
      for (int ks = 0; ks < kHid / 16; ++ks)
        tc_mma(tmem + 128, umma_desc(sa2 + ks * 256, 128, (kHid / 8) * 128),
               umma_desc(sw2 + ks * 256, 128, (kHid / 8) * 128), ks > 0);
      tc_commit(mbar_a);
    }
    if (!tc_wait(mbar_a, parity, wait_limit)) atomicOr(s_err, 1);
    parity ^= 1u;
    tc_after_sync();
    {  // epilogue 2: relu(D2 + b2) . w3 over this thread's 64 columns
      float acc = 0.0f;
      for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
        float v[16];
        tc_ld16(tmem + lane_addr + 128u + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc += fmaxf(v[j] + fb2[c0 + j], 0.0f) * fw3[c0 + j];
      }
      zpart[half * kTcRows + row] = acc;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (*s_err) break;
    if (half == 0) {
      const int64_t i = base + row;
      if (i < n) {
        const float z = zpart[row] + zpart[kTcRows + row] + b3;
        if (z_out) z_out[i] = z;
        if (score_out) {
          const Rec r = d[i];
          score_out[i] = rank_value(r.re, r.im, z, gdt_f * (float)__popcll(r.v | r.w), fc);
        }
      }
    }
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (tid == 0 && *s_err) atomicOr(err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// ---------------------------------------------------------------- training
// Fused forward + backward over tiles of 64 rows [i0, i0 + nb) of X with labels y:
// gradients of the mean BCE are added (fp32 atomics) into grad; the loss sum (already
// divided by nb) into *loss.
__global__ void __launch_bounds__(128, 1) k_mlp_train(const Rec* __restrict__ d, int64_t nb, FeatConst fc, MlpDev m,
                                                      const float* __restrict__ y, float inv_n,
                                                      float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* W1s = reinterpret_cast<uint16_t*>(smem);
  uint16_t* W2s = W1s + kHid * kSF;
  uint16_t* W2Ts = W2s + kHid * kSH;
  uint16_t* xs = W2Ts + kHid * kSH;
  uint16_t* xT = xs + kTrainRows * kSF;
  uint16_t* h1T = xT + kF * kSR;
  uint16_t* dh2T = h1T + kHid * kSR;
  uint16_t* dh1T = dh2T + kHid * kSR;
  float* fb1 = reinterpret_cast<float*>(dh1T + kHid * kSR);
  float* fb2 = fb1 + kHid;
  float* fw3 = fb2 + kHid;
  float* sdb1 = fw3 + kHid;
  float* sdb2 = sdb1 + kHid;
  float* sdw3 = sdb2 + kHid;
  float* sdb3 = sdw3 + kHid;  // [1]
  stage<kSF>(W1s, m.w1b, kHid, kF);
  stage<kSH>(W2s, m.w2b, kHid, kHid);
  stage<kSH>(W2Ts, m.w2tb, kHid, kHid);
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    fb1[i] = m.p[oB1 + i];
    fb2[i] = m.p[oB2 + i];
    fw3[i] = m.p[oW3 + i];
    sdb1[i] = sdb2[i] = sdw3[i] = 0.0f;
  }
  if (threadIdx.x == 0) sdb3[0] = 0.0f;
  const float b3 = m.p[oB3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * warp;
  double wloss = 0.0;
  const int64_t tiles = ceil_div_dev(nb, kTrainRows);
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t base = tile * kTrainRows;
    __syncthreads();
    {  // features: two warps per 32 rows (even warp features 0..43, odd warp 44..79)
      const int row = (warp >> 1) * 32 + lane;
      const int64_t i = base + row;
      Rec r{0, 0, 0.0, 0.0};
      const bool valid = i < nb;
      if (valid) r = d[i];
      if (warp & 1) store_features<1>(r, valid, fc, xs + row * kSF, nullptr, xT, kSR, row);
      else store_features<0>(r, valid, fc, xs + row * kSF, nullptr, xT, kSR, row);
    }
    __syncthreads();
    uint32_t h1[8][4];
    float h2[16][4];
    forward_rows(xs, r0, W1s, W2s, fb1, fb2, g, t, h1, h2);
    // h1 transposed for the weight gradient of layer 2
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 16 * ks + 8 * h + 2 * t;
        const uint32_t lo = h1[ks][2 * h], hi = h1[ks][2 * h + 1];
        h1T[c * kSR + r0 + g] = (uint16_t)(lo & 0xFFFFu);
        h1T[(c + 1) * kSR + r0 + g] = (uint16_t)(lo >> 16);
        h1T[c * kSR + r0 + g + 8] = (uint16_t)(hi & 0xFFFFu);
        h1T[(c + 1) * kSR + r0 + g + 8] = (uint16_t)(hi >> 16);
      }
    float zg, zg8;
    output_rows(h2, fw3, b3, t, zg, zg8);
    const int64_t ig = base + r0 + g, ig8 = ig + 8;
    const bool vg = ig < nb, vg8 = ig8 < nb;
    const float yg = vg ? y[ig] : 0.0f, yg8 = vg8 ? y[ig8] : 0.0f;
    const float dzg = vg ? (1.0f / (1.0f + expf(-zg)) - yg) * inv_n : 0.0f;
    const float dzg8 = vg8 ? (1.0f / (1.0f + expf(-zg8)) - yg8) * inv_n : 0.0f;
    if (t == 0) {
      if (vg) wloss += (double)(fmaxf(zg, 0.0f) - zg * yg + log1pf(expf(-fabsf(zg))));
      if (vg8) wloss += (double)(fmaxf(zg8, 0.0f) - zg8 * yg8 + log1pf(expf(-fabsf(zg8))));
    }
    // output layer: dW3, db3; dh2 = dz w3 (h2 > 0); db2
    float pw[16][2], pb[16][2];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int c = 8 * nt + 2 * t;
      pw[nt][0] = dzg * h2[nt][0] + dzg8 * h2[nt][2];
      pw[nt][1] = dzg * h2[nt][1] + dzg8 * h2[nt][3];
      h2[nt][0] = h2[nt][0] > 0.0f ? dzg * fw3[c] : 0.0f;
      h2[nt][1] = h2[nt][1] > 0.0f ? dzg * fw3[c + 1] : 0.0f;
      h2[nt][2] = h2[nt][2] > 0.0f ? dzg8 * fw3[c] : 0.0f;
      h2[nt][3] = h2[nt][3] > 0.0f ? dzg8 * fw3[c + 1] : 0.0f;
      pb[nt][0] = h2[nt][0] + h2[nt][2];
      pb[nt][1] = h2[nt][1] + h2[nt][3];
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int sh = 4; sh < 32; sh <<= 1) {
          pw[nt][e] += __shfl_xor_sync(0xffffffffu, pw[nt][e], sh);
          pb[nt][e] += __shfl_xor_sync(0xffffffffu, pb[nt][e], sh);
        }
    if (g == 0) {
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        const int c = 8 * nt + 2 * t;
        atomicAdd(&sdw3[c], pw[nt][0]);
        atomicAdd(&sdw3[c + 1], pw[nt][1]);
        atomicAdd(&sdb2[c], pb[nt][0]);
        atomicAdd(&sdb2[c + 1], pb[nt][1]);
      }
    }
    {
      float s = (t == 0) ? dzg + dzg8 : 0.0f;
#pragma unroll
      for (int sh = 1; sh < 32; sh <<= 1) s += __shfl_xor_sync(0xffffffffu, s, sh);
      if (lane == 0) atomicAdd(sdb3, s);
    }
    // dh2 (bf16): transposed copy for dW2 and A fragments for dh1
    uint32_t da[8][4];
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int nt = 2 * ks + h, c = 8 * nt + 2 * t;
        da[ks][2 * h] = pack_bf16(h2[nt][0], h2[nt][1]);
        da[ks][2 * h + 1] = pack_bf16(h2[nt][2], h2[nt][3]);
        dh2T[c * kSR + r0 + g] = (uint16_t)(da[ks][2 * h] & 0xFFFFu);
        dh2T[(c + 1) * kSR + r0 + g] = (uint16_t)(da[ks][2 * h] >> 16);
        dh2T[c * kSR + r0 + g + 8] = (uint16_t)(da[ks][2 * h + 1] & 0xFFFFu);
        dh2T[(c + 1) * kSR + r0 + g + 8] = (uint16_t)(da[ks][2 * h + 1] >> 16);
      }
    // dh1 = (dh2 W2) * (h1 > 0)
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
#pragma unroll
      for (int np = 0; np < 8; ++np) {
        uint32_t b0, b1, b2, b3;
        load_b2<kSH>(W2Ts, 16 * np, 16 * ks, lane, b0, b1, b2, b3);
        mma_bf16(acc[2 * np], da[ks], b0, b1);
        mma_bf16(acc[2 * np + 1], da[ks], b2, b3);
      }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int ks = nt >> 1, h = nt & 1, c = 8 * nt + 2 * t;
      const uint32_t lo = h1[ks][2 * h], hi = h1[ks][2 * h + 1];
      const float e0 = bf16_pos(lo, 0) ? acc[nt][0] : 0.0f, e1 = bf16_pos(lo, 1) ? acc[nt][1] : 0.0f;
      const float e2 = bf16_pos(hi, 0) ? acc[nt][2] : 0.0f, e3 = bf16_pos(hi, 1) ? acc[nt][3] : 0.0f;
      const uint32_t plo = pack_bf16(e0, e1), phi = pack_bf16(e2, e3);
      dh1T[c * kSR + r0 + g] = (uint16_t)(plo & 0xFFFFu);
      dh1T[(c + 1) * kSR + r0 + g] = (uint16_t)(plo >> 16);
      dh1T[c * kSR + r0 + g + 8] = (uint16_t)(phi & 0xFFFFu);
      dh1T[(c + 1) * kSR + r0 + g + 8] = (uint16_t)(phi >> 16);
      pb[nt][0] = e0 + e2;
      pb[nt][1] = e1 + e3;
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int sh = 4; sh < 32; sh <<= 1) pb[nt][e] += __shfl_xor_sync(0xffffffffu, pb[nt][e], sh);
    if (g == 0) {
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        const int c = 8 * nt + 2 * t;
        atomicAdd(&sdb1[c], pb[nt][0]);
        atomicAdd(&sdb1[c + 1], pb[nt][1]);
      }
    }
    __syncthreads();
    // weight gradients over the tile's rows: dW2 = dh2^T h1, dW1 = dh1^T x (K = 64 rows)
    const int o0 = 32 * warp;
#pragma unroll 1
    for (int nc = 0; nc < 4; ++nc) {
      float wa[2][4][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < 4; ++j) wa[mt][j][0] = wa[mt][j][1] = wa[mt][j][2] = wa[mt][j][3] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < kTrainRows / 16; ++ks) {
        uint32_t a0[4], a1[4];
        load_a<kSR>(dh2T, o0, 16 * ks, g, t, a0);
        load_a<kSR>(dh2T, o0 + 16, 16 * ks, g, t, a1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t b0, b1;
          load_b<kSR>(h1T, 32 * nc + 8 * j, 16 * ks, g, t, b0, b1);
          mma_bf16(wa[0][j], a0, b0, b1);
          mma_bf16(wa[1][j], a1, b0, b1);
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int o = o0 + 16 * mt + g, i = 32 * nc + 8 * j + 2 * t;
          atomicAdd(&grad[oW2 + o * kHid + i], wa[mt][j][0]);
          atomicAdd(&grad[oW2 + o * kHid + i + 1], wa[mt][j][1]);
          atomicAdd(&grad[oW2 + (o + 8) * kHid + i], wa[mt][j][2]);
          atomicAdd(&grad[oW2 + (o + 8) * kHid + i + 1], wa[mt][j][3]);
        }
    }
#pragma unroll 1
    for (int nc = 0; nc < 2; ++nc) {
      float wa[2][5][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < 5; ++j) wa[mt][j][0] = wa[mt][j][1] = wa[mt][j][2] = wa[mt][j][3] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < kTrainRows / 16; ++ks) {
        uint32_t a0[4], a1[4];
        load_a<kSR>(dh1T, o0, 16 * ks, g, t, a0);
        load_a<kSR>(dh1T, o0 + 16, 16 * ks, g, t, a1);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          uint32_t b0, b1;
          load_b<kSR>(xT, 40 * nc + 8 * j, 16 * ks, g, t, b0, b1);
          mma_bf16(wa[0][j], a0, b0, b1);
          mma_bf16(wa[1][j], a1, b0, b1);
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const int o = o0 + 16 * mt + g, f = 40 * nc + 8 * j + 2 * t;
          atomicAdd(&grad[oW1 + o * kF + f], wa[mt][j][0]);
          atomicAdd(&grad[oW1 + o * kF + f + 1], wa[mt][j][1]);
          atomicAdd(&grad[oW1 + (o + 8) * kF + f], wa[mt][j][2]);
          atomicAdd(&grad[oW1 + (o + 8) * kF + f + 1], wa[mt][j][3]);
        }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    atomicAdd(&grad[oB1 + i], sdb1[i]);
    atomicAdd(&grad[oB2 + i], sdb2[i]);
    atomicAdd(&grad[oW3 + i], sdw3[i]);
  }
  if (threadIdx.x == 0) atomicAdd(&grad[oB3], sdb3[0]);
#pragma unroll
  for (int sh = 1; sh < 32; sh <<= 1) wloss += __shfl_xor_sync(0xffffffffu, wloss, sh);
  if (lane == 0 && wloss != 0.0) atomicAdd(loss, wloss * (double)inv_n);
}

// Adam on the FP32 master parameters (the gradient buffer is cleared for the next step),
// then the BF16 copies the products read.
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float beta1, float beta2, float eps, float bc1,
                           float bc2, int update, uint16_t* __restrict__ w1b, uint16_t* __restrict__ w2b,
                           uint16_t* __restrict__ w2tb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += gridDim.x * blockDim.x) {
    float x = p[i];
    if (update) {
      const float g = grad[i];
      const float a = beta1 * m1[i] + (1.0f - beta1) * g;
      const float b = beta2 * m2[i] + (1.0f - beta2) * g * g;
      m1[i] = a;
      m2[i] = b;
      x -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
      p[i] = x;
      grad[i] = 0.0f;
    }
    if (i < oB1) {
      w1b[i] = bf16_bits(x);
    } else if (i >= oW2 && i < oB2) {
      const int k = i - oW2, o = k / kHid, j = k - o * kHid;
      w2b[k] = bf16_bits(x);
      w2tb[j * kHid + o] = bf16_bits(x);
    }
  }
}

constexpr size_t kTrainSmem =
    (size_t)(kHid * kSF + 2 * kHid * kSH + kTrainRows * kSF + kF * kSR + 3 * kHid * kSR) * 2 + (6 * kHid + 4) * 4;

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double gauss(uint64_t& s) {  // Box-Muller on two uniforms from the top 53 bits
  const double u1 = ((double)(splitmix(s) >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(splitmix(s) >> 11) * 0x1.0p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace
}  // namespace ps

struct pauli_mlp {
  int n_sites;
  cudaStream_t stream;
  float* p;   // parameters
  float* g;   // gradient accumulator
  float* m1;  // Adam moments
  float* m2;
  uint16_t* w1b;
  uint16_t* w2b;
  uint16_t* w2tb;
  double* loss;
  int64_t t;  // Adam steps taken
};

namespace ps {

namespace {

MlpDev dev_view(const pauli_mlp* m) { return MlpDev{m->w1b, m->w2b, m->w2tb, m->p}; }

int refresh_bf16(pauli_mlp* m) {  // BF16 copies from the FP32 parameters, no update
  PS_LAUNCH("k_mlp_adam", m->stream,
            k_mlp_adam<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, 0.f, 0.f, 0.f, 0.f,
                                                                     1.f, 1.f, 0, m->w1b, m->w2b, m->w2tb));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

int smem_attr() {
  static int done = 0;
  if (done) return PS_OK;
  PS_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  PS_CUDA(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem));
  done = 1;
  return PS_OK;
}

// Test hook (pauli_debug_mlp_wait): the scorer issues no products and gives up its first wait
// after `limit` polls, so that the timeout path runs without any tensor-core work in flight.
int g_mlp_no_products = 0;
long long g_mlp_wait_limit = kTcWaitLimit;

int fwd_run(const pauli_mlp* m, const Rec* d, int64_t n, cudaStream_t s, double gamma_dt, uint16_t* x, float* z,
            double* score) {
  if (n == 0) return PS_OK;
  PS_TRY(smem_attr());
  Buf<int> err;
  PS_TRY(err.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kTcRows), 2 * num_sms()));
  PS_LAUNCH("k_mlp_fwd", s,
            k_mlp_fwd_tc<<<grid, 256, kTcSmem, s>>>(d, n, make_featconst(m->n_sites), dev_view(m), gamma_dt, x, z,
                                                     score, err.p, g_mlp_no_products, g_mlp_wait_limit));
  PS_CUDA(cudaGetLastError());
  int herr = 0;
  PS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  return herr ? PS_ERR_TIMEOUT : PS_OK;
}

// Gradient of the mean BCE over X's records [i0, i0 + nb) into m->g (added), loss into m->loss.
int grad_run(pauli_mlp* m, const pauli_sum* X, const float* y, int64_t i0, int64_t nb) {
  cudaStream_t s = m->stream;
  if (X->stream != s) PS_CUDA(cudaStreamSynchronize(X->stream));
  PS_TRY(smem_attr());
  PS_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), s));
  if (nb == 0) return PS_OK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb, kTrainRows), num_sms()));
  PS_LAUNCH("k_mlp_train", s,
            k_mlp_train<<<grid, 128, kTrainSmem, s>>>(X->d + i0, nb, make_featconst(m->n_sites), dev_view(m), y + i0,
                                                      1.0f / (float)nb, m->g, m->loss));
  PS_CUDA(cudaGetLastError());
  return PS_OK;
}

}  // namespace

int mlp_scores(const pauli_mlp* m, const Rec* d, int64_t n, double gamma_dt, cudaStream_t s, double* score) {
  return fwd_run(m, d, n, s, gamma_dt, nullptr, nullptr, score);
}
int mlp_n_sites(const pauli_mlp* m) { return m->n_sites; }
cudaStream_t mlp_stream(const pauli_mlp* m) { return m->stream; }

}  // namespace ps

using namespace ps;

extern "C" {

int64_t pauli_mlp_param_count(void) { return kParams; }

int pauli_mlp_create(int n_sites, uint64_t seed, void* cuda_stream, pauli_mlp** out) {
  if (!out || n_sites < 1 || n_sites > 64) return PS_ERR_INVALID;
  *out = nullptr;
  pauli_mlp* m = new pauli_mlp{};
  m->n_sites = n_sites;
  m->stream = (cudaStream_t)cuda_stream;
  cudaStream_t s = m->stream;
  auto fail = [&](int st) {
    dev_free(m->p, s);
    dev_free(m->g, s);
    dev_free(m->m1, s);
    dev_free(m->m2, s);
    dev_free(m->w1b, s);
    dev_free(m->w2b, s);
    dev_free(m->w2tb, s);
    dev_free(m->loss, s);
    delete m;
    return st;
  };
  int st = PS_OK;
  if ((st = dev_alloc((void**)&m->p, kParams * sizeof(float), s)) != PS_OK ||
      (st = dev_alloc((void**)&m->g, kParams * sizeof(float), s)) != PS_OK ||
      (st = dev_alloc((void**)&m->m1, kParams * sizeof(float), s)) != PS_OK ||
      (st = dev_alloc((void**)&m->m2, kParams * sizeof(float), s)) != PS_OK ||
      (st = dev_alloc((void**)&m->w1b, (size_t)kHid * kF * 2, s)) != PS_OK ||
      (st = dev_alloc((void**)&m->w2b, (size_t)kHid * kHid * 2, s)) != PS_OK ||
      (st = dev_alloc((void**)&m->w2tb, (size_t)kHid * kHid * 2, s)) != PS_OK ||
      (st = dev_alloc((void**)&m->loss, sizeof(double), s)) != PS_OK)
    return fail(st);
  // He-style initialisation: W1 ~ N(0, 2/80), W2 ~ N(0, 2/128), w3 ~ N(0, 1/128), biases 0
  std::vector<float> h(kParams, 0.0f);
  uint64_t state = seed;
  for (int i = oW1; i < oB1; ++i) h[i] = (float)(gauss(state) * std::sqrt(2.0 / kF));
  for (int i = oW2; i < oB2; ++i) h[i] = (float)(gauss(state) * std::sqrt(2.0 / kHid));
  for (int i = oW3; i < oB3; ++i) h[i] = (float)(gauss(state) * std::sqrt(1.0 / kHid));
  cudaError_t e = cudaMemcpyAsync(m->p, h.data(), kParams * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->g, 0, kParams * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, kParams * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, kParams * sizeof(float), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_cuda_error(e, "pauli_mlp_create");
    return fail(PS_ERR_CUDA);
  }
  if ((st = refresh_bf16(m)) != PS_OK) return fail(st);
  *out = m;
  return PS_OK;
}

int pauli_debug_mlp_wait(int no_products, int64_t wait_limit) {
  if (wait_limit < 1) return PS_ERR_INVALID;
  g_mlp_no_products = no_products ? 1 : 0;
  g_mlp_wait_limit = wait_limit;
  return PS_OK;
}

int pauli_mlp_destroy(pauli_mlp* m) {
  if (!m) return PS_OK;
  cudaStream_t s = m->stream;
  dev_free(m->p, s);
  dev_free(m->g, s);
  dev_free(m->m1, s);
  dev_free(m->m2, s);
  dev_free(m->w1b, s);
  dev_free(m->w2b, s);
  dev_free(m->w2tb, s);
  dev_free(m->loss, s);
  delete m;
  return PS_OK;
}

int pauli_mlp_get_params(const pauli_mlp* m, float* params, int64_t n) {
  if (!m || !params || n != kParams) return PS_ERR_INVALID;
  PS_CUDA(cudaMemcpyAsync(params, m->p, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  PS_CUDA(cudaStreamSynchronize(m->stream));
  return PS_OK;
}

int pauli_mlp_set_params(pauli_mlp* m, const float* params, int64_t n) {
  if (!m || !params || n != kParams) return PS_ERR_INVALID;
  std::vector<float> h(params, params + kParams);
  PS_CUDA(cudaMemcpyAsync(m->p, h.data(), kParams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
  PS_CUDA(cudaMemsetAsync(m->g, 0, kParams * sizeof(float), m->stream));
  PS_CUDA(cudaMemsetAsync(m->m1, 0, kParams * sizeof(float), m->stream));
  PS_CUDA(cudaMemsetAsync(m->m2, 0, kParams * sizeof(float), m->stream));
  PS_CUDA(cudaStreamSynchronize(m->stream));
  m->t = 0;
  return refresh_bf16(m);
}

int pauli_mlp_features(const pauli_mlp* m, const pauli_sum* O, uint16_t* x) {
  PS_NARROW(O);
  if (!m || !O || O->n_sites != m->n_sites || (O->n > 0 && !x)) return PS_ERR_INVALID;
  if (O->stream != m->stream) PS_CUDA(cudaStreamSynchronize(O->stream));
  PS_TRY(fwd_run(m, O->d, O->n, m->stream, 0.0, x, nullptr, nullptr));
  PS_CUDA(cudaStreamSynchronize(m->stream));
  return PS_OK;
}

int pauli_mlp_logits(const pauli_mlp* m, const pauli_sum* O, float* z) {
  PS_NARROW(O);
  if (!m || !O || O->n_sites != m->n_sites || (O->n > 0 && !z)) return PS_ERR_INVALID;
  if (O->stream != m->stream) PS_CUDA(cudaStreamSynchronize(O->stream));
  PS_TRY(fwd_run(m, O->d, O->n, m->stream, 0.0, nullptr, z, nullptr));
  PS_CUDA(cudaStreamSynchronize(m->stream));
  return PS_OK;
}

int pauli_mlp_scores(const pauli_mlp* m, const pauli_sum* O, double gamma_dt, double* score) {
  PS_NARROW(O);
  NvtxRange nvtx("pauli_mlp_scores");
  if (!m || !O || O->n_sites != m->n_sites || (O->n > 0 && !score) || !std::isfinite(gamma_dt))
    return PS_ERR_INVALID;
  if (O->stream != m->stream) PS_CUDA(cudaStreamSynchronize(O->stream));
  PS_TRY(fwd_run(m, O->d, O->n, m->stream, gamma_dt, nullptr, nullptr, score));
  PS_CUDA(cudaStreamSynchronize(m->stream));
  return PS_OK;
}

int pauli_mlp_gradient(pauli_mlp* m, const pauli_sum* X, const float* labels, int64_t i0, int64_t nb, float* grad,
                       double* loss) {
  PS_NARROW(X);
  if (!m || !X || X->n_sites != m->n_sites || !grad || i0 < 0 || nb < 0 || i0 + nb > X->n || (nb > 0 && !labels))
    return PS_ERR_INVALID;
  PS_CUDA(cudaMemsetAsync(m->g, 0, kParams * sizeof(float), m->stream));
  PS_TRY(grad_run(m, X, labels, i0, nb));
  PS_CUDA(cudaMemcpyAsync(grad, m->g, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  double l = 0.0;
  PS_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PS_CUDA(cudaMemsetAsync(m->g, 0, kParams * sizeof(float), m->stream));
  PS_CUDA(cudaStreamSynchronize(m->stream));
  if (loss) *loss = l;
  return PS_OK;
}

int pauli_mlp_train_step(pauli_mlp* m, const pauli_sum* X, const float* labels, int64_t i0, int64_t nb, float lr,
                         double* loss) {
  PS_NARROW(X);
  NvtxRange nvtx("pauli_mlp_train_step");
  if (!m || !X || X->n_sites != m->n_sites || i0 < 0 || nb < 1 || i0 + nb > X->n || !labels || !(lr >= 0.0f))
    return PS_ERR_INVALID;
  PS_TRY(grad_run(m, X, labels, i0, nb));
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->t)), bc2 = (float)(1.0 - std::pow(0.999, (double)m->t));
  PS_LAUNCH("k_mlp_adam", m->stream,
            k_mlp_adam<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, lr, b1, b2, 1e-8f,
                                                                     bc1, bc2, 1, m->w1b, m->w2b, m->w2tb));
  PS_CUDA(cudaGetLastError());
  if (loss) {
    PS_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    PS_CUDA(cudaStreamSynchronize(m->stream));
  }
  return PS_OK;
}

int pauli_mlp_labels(const pauli_sum* X, const pauli_sum* target, float* labels) {
  PS_NARROW(X);
  if (!X || !target || X->n_sites != target->n_sites || (X->n > 0 && !labels)) return PS_ERR_INVALID;
  if (target->stream != X->stream) PS_CUDA(cudaStreamSynchronize(target->stream));
  PS_TRY(membership(X->d, X->n, target->d, target->n, X->stream, labels));
  PS_CUDA(cudaStreamSynchronize(X->stream));
  return PS_OK;
}

}  // extern "C"
