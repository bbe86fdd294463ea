// Internal definitions shared by the CUDA translation units of libpaulistr.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstddef>
#include <cstring>
#include <string>

#include "../../include/paulistr.h"

namespace ps {

// One string with its complex FP64 coefficient: 32 bytes, one DRAM sector.
struct __align__(16) Rec {
  uint64_t v, w;
  double re, im;
};

struct Cx {
  double re, im;
};

// ----------------------------------------------------------------------------- errors
void set_cuda_error(cudaError_t e, const char* where);
#define PS_CUDA(call)                                 \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) {                          \
      ::ps::set_cuda_error(_e, #call);                \
      return PS_ERR_CUDA;                             \
    }                                                 \
  } while (0)
#define PS_TRY(expr)               \
  do {                             \
    int _s = (expr);               \
    if (_s != PS_OK) return _s;    \
  } while (0)

// ----------------------------------------------------------------------------- memory
// Stream-ordered device allocation (cudaMallocAsync on the stream's pool).  The
// test hook pauli_debug_fail_alloc_after makes a chosen allocation fail on the host.
int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// RAII scratch buffer freed in stream order.
template <class T>
struct Buf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { reset(); }
  int alloc(size_t count, cudaStream_t stream) {
    reset();
    s = stream;
    n = count;
    if (count == 0) return PS_OK;
    return dev_alloc((void**)&p, count * sizeof(T), stream);
  }
  void reset() {
    if (p) dev_free(p, s);
    p = nullptr;
    n = 0;
  }
  // take ownership of a buffer from dev_alloc
  void adopt(T* q, size_t count, cudaStream_t stream) {
    reset();
    p = q;
    n = count;
    s = stream;
  }
};

}  // namespace ps

// The opaque sum (device resident).  `n` is the authoritative size; it is kept
// current on the host after every call (calls that change it synchronise).
struct pauli_sum {
  int n_sites;
  cudaStream_t stream;
  ps::Rec* d;
  int64_t cap;
  int64_t n;
  int cls;  // coefficient class: bit 0 = real parts may be non-zero, bit 1 = imaginary parts may be
  int f32;  // FP32 coefficients: every result written into the sum is rounded to FP32
  int W;    // 64-bit words per mask: 1 (n_sites <= 64), 2 (<= 128) or 4 (<= 256)
};

namespace ps {

// ----------------------------------------------------------------------------- coefficient classes
// A class is the set of components that may be non-zero: 0 (no terms), 1 (real),
// 2 (imaginary), 3 (complex).  Hermitian strings with real coefficients stay real or
// imaginary through the whole commutator path, which lets the merge use one real
// product per contribution.
constexpr int kClsReal = 1, kClsImag = 2, kClsComplex = 3;
inline int cls_swap(int c) { return ((c & 1) << 1) | ((c >> 1) & 1); }        // times i
inline int cls_mul(int a, int b) {                                               // product of values
  if (!a || !b) return 0;
  if (a == kClsComplex || b == kClsComplex) return kClsComplex;
  return a == b ? kClsReal : kClsImag;
}
inline int cls_of(double re, double im) { return (re != 0.0 ? 1 : 0) | (im != 0.0 ? 2 : 0); }

// Words per mask and bytes per record for a site count: one word up to 64 sites (the 32-byte
// record {v, w, re, im}), else 2 or 4 words per mask (records of 16 W + 16 bytes).
inline int words_for(int n_sites) { return n_sites <= 64 ? 1 : (n_sites <= 128 ? 2 : 4); }
inline size_t rec_bytes(int W) { return W == 1 ? sizeof(Rec) : (size_t)(16 * W + 16); }
// Entry points that exist only for one-word masks reject wider sums.
#define PS_NARROW(s)                                    \
  do {                                                  \
    if ((s) && (s)->W > 1) return PS_ERR_INVALID;       \
  } while (0)

int sum_reserve(pauli_sum* s, int64_t cap, bool keep_contents);
int sum_adopt(pauli_sum* s, Rec* d, int64_t cap, int64_t n);  // take ownership of a buffer
uint64_t key_mask(int n_sites);

// ----------------------------------------------------------------------------- output hash
// F: a GF(2)-linear map from a 128-bit key to 32 bits, F_j(v,w) = parity((v & A_j) ^ (w & B_j)).
// Linearity gives F(a ^ b) = F(a) ^ F(b): the bin of a product string is the XOR of the
// bins of its factors, so products can be routed to bins without forming the key first.
constexpr int kHashRows = 32;
uint32_t host_hash(uint64_t v, uint64_t w, int bits);
void host_hash_rows(const uint64_t** a, const uint64_t** b);
// A key whose hash (low `bits` bits) is exactly `target`; the map has full rank.
void host_key_with_hash(uint32_t target, int bits, uint64_t* v, uint64_t* w);
int upload_hash_tables();  // merge.cu: copies the rows to its __constant__ tables

// ----------------------------------------------------------------------------- Pauli algebra
// Strings a, b anticommute iff popcount(wa&vb) + popcount(va&wb) is odd (eq. eps_com);
// the parity of a sum of popcounts is the popcount parity of the XOR.
__device__ __forceinline__ bool anticommute(uint64_t va, uint64_t wa, uint64_t vb, uint64_t wb) {
  return (__popcll((wa & vb) ^ (va & wb)) & 1) != 0;
}

// P_a P_b = i^k P_{a^b} in the Hermitian basis P(v,w) = (-i)^{pop(v&w)} Z^v X^w:
// k = pop(vc&wc) - pop(va&wa) - pop(vb&wb) + 2 pop(wa&vb) (mod 4)  (eq. eps12 rewritten).
__device__ __forceinline__ int product_phase(uint64_t va, uint64_t wa, uint64_t vb, uint64_t wb) {
  uint64_t vc = va ^ vb, wc = wa ^ wb;
  int k = __popcll(vc & wc) - __popcll(va & wa) - __popcll(vb & wb) + 2 * __popcll(wa & vb);
  return k & 3;
}

// Translation on a ring of n sites (site j -> j + k mod n): a rotation of both masks by k
// within their low n bits.
__host__ __device__ __forceinline__ uint64_t rotl_ring(uint64_t x, int k, int n) {
  const uint64_t mask = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  return k == 0 ? (x & mask) : (((x << k) | (x >> (n - k))) & mask);
}

// Representative of the translation orbit of (v, w) on a ring of n sites: the smallest
// translate in (v, then w) unsigned order, and the smallest shift r reaching it.
__device__ __forceinline__ void ts_canonical(uint64_t v, uint64_t w, int n, uint64_t& cv, uint64_t& cw, int& r) {
  cv = v;
  cw = w;
  r = 0;
  for (int k = 1; k < n; ++k) {
    const uint64_t tv = rotl_ring(v, k, n), tw = rotl_ring(w, k, n);
    if (tv < cv || (tv == cv && tw < cw)) {
      cv = tv;
      cw = tw;
      r = k;
    }
  }
}

// Smallest period d of (v, w) on a ring of n sites; divmask has bit d set for each proper
// divisor d of n (the only candidates).
__device__ __forceinline__ int ts_period(uint64_t v, uint64_t w, int n, uint64_t divmask) {
  while (divmask) {
    const int d = __ffsll((long long)divmask) - 1;
    divmask &= divmask - 1;
    if (rotl_ring(v, d, n) == v && rotl_ring(w, d, n) == w) return d;
  }
  return n;
}

inline uint64_t proper_divisor_mask(int n) {
  uint64_t m = 0;
  for (int d = 1; d < n; ++d)
    if (n % d == 0) m |= 1ull << d;
  return m;
}

// Exactly-rounded FP64 operations without contraction into FMA.
__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }

// Slot hash of a string key for the open-addressing tables (global and shared memory):
// MurmurHash3's 64-bit finaliser (Appleby; invertible, every input bit reaches every output
// bit) applied to w, XORed into v, and applied again.  A plain product by an odd constant is
// not enough here: it carries bits upward only, so strings that differ only in the top bits
// of a mask word (sites 57-64, for instance) would share most of their hash.
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xFF51AFD7ED558CCDull;
  x ^= x >> 33;
  x *= 0xC4CEB9FE1A85EC53ull;
  x ^= x >> 33;
  return x;
}
__device__ __forceinline__ uint64_t key_hash64(uint64_t v, uint64_t w) {
  return fmix64(v ^ fmix64(w ^ 0x9E3779B97F4A7C15ull));
}

// 2*x, exact (exponent increment); falls back to x+x for zero, subnormal, huge or non-finite x.
__device__ __forceinline__ double twice(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  if (e != 0u && e < 0x7FEu) return __longlong_as_double((long long)(b + (1ull << 52)));
  return __dadd_rn(x, x);
}

// (a.re b.re - a.im b.im, a.re b.im + a.im b.re) with separately rounded products and sums.
// Products with an exactly-zero factor are skipped: they are +-0 and do not change a
// non-zero partial result, so every non-zero component is bit-identical to the full formula.
__device__ __forceinline__ Cx cmul(Cx a, Cx b) {
  double rr = (is_zero(a.re) || is_zero(b.re)) ? 0.0 : __dmul_rn(a.re, b.re);
  double ii = (is_zero(a.im) || is_zero(b.im)) ? 0.0 : __dmul_rn(a.im, b.im);
  double ri = (is_zero(a.re) || is_zero(b.im)) ? 0.0 : __dmul_rn(a.re, b.im);
  double ir = (is_zero(a.im) || is_zero(b.re)) ? 0.0 : __dmul_rn(a.im, b.re);
  Cx r;
  r.re = is_zero(ii) ? rr : (is_zero(rr) ? -ii : __dsub_rn(rr, ii));
  r.im = is_zero(ir) ? ri : (is_zero(ri) ? ir : __dadd_rn(ri, ir));
  return r;
}

__device__ __forceinline__ Cx rot(Cx a, int k) {  // multiply by i^k (exact)
  switch (k & 3) {
    case 0: return a;
    case 1: return Cx{-a.im, a.re};
    case 2: return Cx{-a.re, -a.im};
    default: return Cx{a.im, -a.re};
  }
}

// ----------------------------------------------------------------------------- division by a constant
// a / b correctly rounded (round to nearest even) for a fixed b, with one FP64 multiply and
// one FMA instead of a full division: Q = RN(|a| * RN(1/|b|)) is within 1.5 ulp of
// t = |a|/|b|; the remainder rho = |a| - Q|b| is exact (one FMA); comparing rho with the exact
// products |b| * (half gaps to Q's neighbours), powers of two times |b|, decides RN(t) among
// Q and its two neighbours.  Whenever an operand or result leaves the normal range, or Q is
// more than one ulp away, it falls back to the IEEE division.  The exact FMA remainder and the
// rounding decision from it are those of Markstein's correction step for division (P. Markstein,
// IA-64 and Elementary Functions, 2000); the remainder's exactness when Q is within an ulp is
// Boldo and Daumas' result (Representable correcting terms for possibly underflowing floating
// point operations, ARITH 2003).
struct DivConst {
  double b;       // divisor
  double rabs;    // RN(1 / |b|)
  double babs;    // |b|
  int ok;         // |b| normal and RN(1/|b|) normal
};

__host__ inline DivConst make_divconst(double b) {
  DivConst d;
  d.b = b;
  d.babs = b < 0 ? -b : b;
  d.rabs = 1.0 / d.babs;
  d.ok = (d.babs >= 2.2250738585072014e-308 && d.babs <= 8.98846567431158e307 && d.rabs >= 2.2250738585072014e-308) ? 1 : 0;
  return d;
}

// x * 2^k for a normal x when the result stays normal; ok = false otherwise.
__device__ __forceinline__ double ldexp_exact(double x, int k, bool& ok) {
  unsigned long long bx = (unsigned long long)__double_as_longlong(x);
  int E = (int)((bx >> 52) & 0x7FF);
  int E2 = E + k;
  ok = (E != 0 && E != 0x7FF && E2 >= 1 && E2 <= 2046);
  return ok ? __longlong_as_double((long long)(bx + ((unsigned long long)(long long)k << 52))) : 0.0;
}

__device__ __forceinline__ double div_const(double a, const DivConst& d) {
  if (!d.ok) return __ddiv_rn(a, d.b);
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long sign = (ua ^ (unsigned long long)__double_as_longlong(d.b)) & (1ull << 63);
  const int Ea = (int)((ua >> 52) & 0x7FF);
  if (Ea < 128 || Ea > 1900) return __ddiv_rn(a, d.b);  // zeros, tiny, huge, non-finite
  const double A = __longlong_as_double((long long)(ua & ~(1ull << 63)));
  const double Q = __dmul_rn(A, d.rabs);
  const unsigned long long uq = (unsigned long long)__double_as_longlong(Q);
  const int Eq = (int)((uq >> 52) & 0x7FF);
  if (Eq < 64 || Eq > 2000) return __ddiv_rn(a, d.b);
  const double rho = __fma_rn(-Q, d.babs, A);  // A - Q |b|, exact
  const bool pow2 = (uq & ((1ull << 52) - 1)) == 0;
  bool ok1, ok2;
  const double eu = ldexp_exact(d.babs, Eq - 1076, ok1);                 // |b| * ulp(Q)/2
  const double el = pow2 ? ldexp_exact(d.babs, Eq - 1077, ok2) : eu;     // |b| * (gap below Q)/2
  if (!ok1 || (pow2 && !ok2)) return __ddiv_rn(a, d.b);
  const long long ir = __double_as_longlong(rho);
  const long long ieu = __double_as_longlong(eu), iel = __double_as_longlong(el);
  unsigned long long r = uq;
  if (ir > 0) {  // t above Q: compare rho with |b| ulp/2 (positive doubles order like their bits)
    if (ir >= ieu + (1ll << 52)) return __ddiv_rn(a, d.b);  // rho >= 2 eu: more than one ulp away
    if (ir > ieu || (ir == ieu && (uq & 1))) r = uq + 1;
  } else if (ir < 0) {
    const long long mr = ir & 0x7FFFFFFFFFFFFFFFll;  // |rho|
    if (mr >= iel + (1ll << 52)) return __ddiv_rn(a, d.b);
    if (mr > iel || (mr == iel && (uq & 1))) r = uq - 1;
  }
  return __longlong_as_double((long long)(r | sign));
}

__device__ __forceinline__ double add_rn(double a, double b) {
  if (is_zero(b)) return a;
  if (is_zero(a)) return b;
  return __dadd_rn(a, b);
}

// ----------------------------------------------------------------------------- profiling
// Scoped around one kernel launch: counts the launch and, when profiling is enabled,
// records CUDA events on the launching stream before and after it.
class KTimer {
 public:
  KTimer(const char* name, cudaStream_t s);
  ~KTimer();
  KTimer(const KTimer&) = delete;
  KTimer& operator=(const KTimer&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  void* a_;
};
#define PS_LAUNCH(name, stream, ...) \
  do {                               \
    ::ps::KTimer _kt(name, stream);  \
    __VA_ARGS__;                     \
  } while (0)

// ----------------------------------------------------------------------------- tracing
// An NVTX range for the scope of one library call (header-only NVTX: a no-op unless a
// profiler is attached), so that timelines show steps and their phases by name.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ----------------------------------------------------------------------------- misc
__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__device__ __forceinline__ int64_t ceil_div_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }
int num_sms();

// Exclusive prefix sum of n unsigned values into out[0..n]; out[n] = total (device only).
int scan_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s);
int scan_u32_to_u64(const uint32_t* in, uint64_t* out, int64_t n, cudaStream_t s);

// Merge engine (merge.cu).  For every output string c the engine forms
//   acc(c) = sequential sum, in order, of: the products 2 i^(k+rot) h x for each H term h
//            (H order) with x in X and h^x = c, anticommuting; then alpha_s * y_s(c) for
//            each extra source s in order;
// and returns out(c) = acc(c)                    (no post scale), or
//              out(c) = pre(c) + post * acc(c)    (with post; absent terms are zero).
// Exact zeros are dropped.  This covers [H,X], A + alpha B, the Lanczos combination
// [H,O] - b O_prev and the RK4 stage combinations.
struct MergeSource {
  const Rec* rec;
  int64_t n;
  Cx alpha;
  int cls = kClsComplex;  // coefficient class of rec
  int ts = 0;             // translation symmetry: 0 none; kTsCanon each string to its orbit
                          // representative (order code = shift); kTsExpand each string to all
                          // ring translates (order code = shift)
};
constexpr int kTsCanon = 1, kTsExpand = 2;
struct MergeSpec {
  const Rec* H = nullptr;
  int nH = 0;
  const Rec* X = nullptr;
  int64_t nX = 0;
  int rot = 0;
  bool product = false;
  int ring = 0;  // ring length of translation-symmetric sources (their order codes are 0..ring-1)  // X pairs: every (h, x) with i^k h x (operator product); else the commutator's
                         // anticommuting pairs with 2 i^(k + rot) h x
  MergeSource src[4];
  int nsrc = 0;
  const Rec* pre = nullptr;
  int64_t npre = 0;
  bool has_post = false;
  Cx post{1.0, 0.0};
  int clsH = kClsComplex, clsX = kClsComplex, clsPre = kClsComplex;  // coefficient classes of the operands
  // Batched instances (optional): the coefficient of H term h for a string x of instance
  // b = x.v >> hb_shift is hbatch[b * nH + h] (the real factor of H's component); H's own
  // coefficients only fix the class.  Needs the table emission of full records.
  const double* hbatch = nullptr;
  int hb_shift = 0;
  // With hbatch (optional): per H term, the coefficient shared by every instance, or NaN when
  // the instances differ; shared terms skip the per-instance table.
  const double* hbatch_uniform = nullptr;
  // Rank keys of a single-component output (optional): when keys_out is set and the merge runs
  // in single-component mode on a ranked merge, its output stage also writes, per output
  // string in storage order, the bit pattern of |x| of its non-zero component into a device
  // array it allocates (*keys_out; the caller frees it with dev_free), and raises *keys_top
  // (device int, set to a value below every bound beforehand) to the exponent bound of the
  // exact norm, max prod_top(x, x) (kTopInf / kTopNaN for a non-finite x).  *keys_out stays
  // null when the merge cannot provide them.
  uint64_t** keys_out = nullptr;
  int* keys_top = nullptr;
};
int merge_run(const MergeSpec& spec, cudaStream_t s, pauli_sum* out);
int autotune_commutator(const MergeSpec& sp, pauli_sum* out, int reps, int* best_bin, int* best_quota,
                        double* best_ms, double* default_ms);
void autotune_reset();
int merge_geometry_fix(int bin_target, int quota);
int ts_translates(const Rec* G, int64_t n, int ring, cudaStream_t s, Rec* out);
void record_merge_stats(const pauli_merge_stats& st);

// truncate.cu / reduce.cu
// score (optional): a ranking value per record of O (storage order) that replaces |c|^2 in
// the top-k select (higher kept first, exact ties to the smaller key, NaN lowest).
int truncate_run(pauli_sum* O, const pauli_trunc_policy* P, const pauli_sum* keep, double dt, const double* divisor,
                 const double* score = nullptr);
int exact_norm2(const Rec* d, int64_t n, cudaStream_t s, double* out, int ring = 0);
// The exact norm of a single-component sum from its rank keys (bit patterns of |x|, see
// MergeSpec::keys_out) and the exponent bound top (device int); with hist non-null, the keys'
// first-digit histogram (kKeyBins counters, zeroed here) in the same pass.
int exact_norm2_keys_top(const uint64_t* ab, int64_t n, const int* top, cudaStream_t s, double* out, unsigned* hist);
// The first-digit histogram (kKeyBins counters, zeroed here) of n rank keys, without a norm.
int key_first_digits(const uint64_t* ab, int64_t n, cudaStream_t s, unsigned* hist);
// The Lanczos truncation of a single-component FP64 sum by top-k alone ranks the undivided
// values |x| (truncate.cu).  Its rank keys (bit patterns of |x|) and their first-digit
// histogram (kKeyBins counters) can be produced by the first pass of the norm.
constexpr int kKeyBins = 2048;
bool lanczos_keys_eligible(const pauli_sum* A, const pauli_trunc_policy* P);
int exact_norm2_keys(const Rec* d, int64_t n, cudaStream_t s, double* out, int cls, uint64_t* ab, unsigned* hist);
int truncate_lanczos_keys(pauli_sum* A, const pauli_trunc_policy* P, double divisor, uint64_t* ab, unsigned* hist);
// Top-k alone from the merge's rank keys (the RK4 stage trim); the general path otherwise.
int truncate_top_keys(pauli_sum* A, const pauli_trunc_policy* P, uint64_t* ab, unsigned* hist);
int exact_trace_product(const Rec* A, int64_t na, const Rec* B, int64_t nb, cudaStream_t s, double* re, double* im);
int coefficients(const Rec* O, int64_t n, const uint64_t* qv, const uint64_t* qw, int64_t nq, cudaStream_t s,
                 double* re, double* im);
int membership(const Rec* X, int64_t nx, const Rec* T, int64_t nt, cudaStream_t s, float* label);
// FP32 sums: round every coefficient to FP32 and drop the strings that become zero (no-op
// for FP64 sums).
int round_f32(pauli_sum* s);

// wide.cu: the path for masks of 2 or 4 words (n_sites 65..256); masks are passed as
// row-major arrays of W words per string (word k holds sites 64k+1 .. 64k+64).
namespace wide_api {
int upload(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re, const double* im, int64_t n,
           bool host);
int download(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im);
int download_device(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im);
int commutator(const pauli_sum* H, const pauli_sum* O, int rot, pauli_sum* out);
int add(const pauli_sum* A, Cx alpha, const pauli_sum* B, pauli_sum* out);
int truncate(pauli_sum* O, const pauli_trunc_policy* P, const pauli_sum* keep, double dt, const double* divisor);
int rk4_step(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* P, const pauli_sum* keep);
int lanczos_step(const pauli_sum* H, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev, const pauli_trunc_policy* P,
                 double* b_out);
int trace_product(const pauli_sum* A, const pauli_sum* B, double* re, double* im);
int norm2(const pauli_sum* O, double* out);
}  // namespace wide_api

// mlp.cu: learned truncation score ln|c| - gamma_dt wt + z of every record (storage order)
int mlp_scores(const pauli_mlp* m, const Rec* d, int64_t n, double gamma_dt, cudaStream_t s, double* score);
int mlp_n_sites(const pauli_mlp* m);
cudaStream_t mlp_stream(const pauli_mlp* m);

}  // namespace ps
