// Allocation-free trace product: pauli_trace_product_noalloc.
//
// Some callers cannot allocate device memory: code running inside another framework's
// memory budget or allocator, code that must not call cudaMalloc while a CUDA graph is
// being captured elsewhere in the process, or plug-ins handed only pre-allocated
// buffers.  This entry point computes the same exactly rounded Tr(AB)/2^N as
// pauli_trace_product, but from caller-provided device arrays and with its scratch (a
// key table and the exact accumulators) in one file-scope device array, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
#include <mutex>

#include "common.cuh"
#include "exact_sum.cuh"

namespace ps {

using namespace exact;

namespace {

constexpr int kNaLogSlots = 18;
constexpr int64_t kNaSlots = (int64_t)1 << kNaLogSlots;  // key table slots
constexpr int64_t kNaMaxTabled = kNaSlots / 2;            // largest smaller operand: 131072 strings
constexpr int kNaSpan = kWinDigits + kFullDigits;

struct NaScratch {
  ulonglong2 key[kNaSlots];              // 4 MiB: keys of the smaller operand (empty = all ones)
  int64_t idx[kNaSlots];                 // 2 MiB: their indices
  long long acc[2 * kNaSpan];            // re window + digits, im window + digits
  long long ones_idx;                    // index of the all-ones key in the tabled operand, or -1
  int top;                               // largest product exponent bound
  int wlo[2];                            // window origins (re, im)
};

// The scratch: a fixed array of sizeof(NaScratch) bytes (about 6 MiB); every GPU that
// loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_na_scratch[sizeof(NaScratch)];

// In host code g_na_scratch names a host-side stand-in, not device memory: its device
// address is looked up once per device (with that device current) and passed to the kernels.
std::mutex g_na_mu;
NaScratch* g_na_ptr[128] = {};

int na_scratch(NaScratch** out) {
  int dev = 0;
  PS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return PS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      set_cuda_error(e, "cudaGetSymbolAddress(g_na_scratch)");
      return PS_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<NaScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return PS_OK;
}

// Operand as four device arrays.
struct SoA {
  const uint64_t* v;
  const uint64_t* w;
  const double* re;
  const double* im;
};

__global__ void k_na_build(SoA T, int64_t n, NaScratch* s, uint64_t tmask) {
  const ulonglong2 empty = make_ulonglong2(~0ull, ~0ull);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ulonglong2 k = make_ulonglong2(T.v[i], T.w[i]);
    if (k.x == empty.x && k.y == empty.y) {
      s->ones_idx = i;
      continue;
    }
    uint64_t slot = mix_key(k.x, k.y) & tmask;
    for (uint64_t p = 0; p <= tmask; ++p) {
      ulonglong2 old = cas128_g(&s->key[slot], empty, k);
      if (old.x == empty.x && old.y == empty.y) {
        s->idx[slot] = i;
        break;
      }
      slot = (slot + 1) & tmask;
    }
  }
}

__global__ void k_na_top(SoA P, int64_t n, SoA T, NaScratch* s, uint64_t tmask) {
  int m = -100000;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = tp_find(s->key, s->idx, tmask, s->ones_idx, P.v[i], P.w[i]);
    if (j < 0) continue;
    double ar = P.re[i], ai = P.im[i], br = T.re[j], bi = T.im[j];
    m = max(m, max(max(prod_top(ar, br), prod_top(ai, bi)), max(prod_top(ar, bi), prod_top(ai, br))));
    // a non-finite factor in a matched pair makes both parts NaN (as pauli_trace_product)
    if (nonfinite_top(ar) > 0 || nonfinite_top(ai) > 0 || nonfinite_top(br) > 0 || nonfinite_top(bi) > 0) m = kTopNaN;
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&s->top, m);
}

__global__ void __launch_bounds__(kRedThreads) k_na_acc(SoA P, int64_t n, SoA T, NaScratch* s, uint64_t tmask) {
  const int t = s->top;
  if (t <= -100000 || t >= kTopInf) return;
  const int wlo = ((t - 190 + kBias) & ~31) - kBias;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->wlo[0] = wlo;
    s->wlo[1] = wlo;
  }
  Win ar{{0, 0, 0, 0}}, ai{{0, 0, 0, 0}};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = tp_find(s->key, s->idx, tmask, s->ones_idx, P.v[i], P.w[i]);
    if (j < 0) continue;
    double pr = P.re[i], pi = P.im[i], qr = T.re[j], qi = T.im[j];
    add_product(ar, pr, qr, wlo, s->acc + kWinDigits);
    add_product(ar, -pi, qi, wlo, s->acc + kWinDigits);
    add_product(ai, pr, qi, wlo, s->acc + kNaSpan + kWinDigits);
    add_product(ai, pi, qr, wlo, s->acc + kNaSpan + kWinDigits);
  }
  block_flush(ar, s->acc);
  __syncthreads();
  block_flush(ai, s->acc + kNaSpan);
}

}  // namespace

}  // namespace ps

using namespace ps;

extern "C" int pauli_trace_product_noalloc(const uint64_t* av, const uint64_t* aw, const double* are,
                                           const double* aim, int64_t na, const uint64_t* bv, const uint64_t* bw,
                                           const double* bre, const double* bim, int64_t nb, void* cuda_stream,
                                           double* re, double* im) {
  if (!re || !im || na < 0 || nb < 0) return PS_ERR_INVALID;
  if ((na > 0 && (!av || !aw || !are || !aim)) || (nb > 0 && (!bv || !bw || !bre || !bim))) return PS_ERR_INVALID;
  *re = 0.0;
  *im = 0.0;
  if (na == 0 || nb == 0) return PS_OK;
  // the key table holds the smaller operand
  const bool swap = nb > na;
  const SoA A{av, aw, are, aim}, B{bv, bw, bre, bim};
  const SoA P = swap ? B : A, T = swap ? A : B;
  const int64_t np = swap ? nb : na, nt = swap ? na : nb;
  if (nt > kNaMaxTabled) return PS_ERR_CAPACITY;  // the smaller operand exceeds the fixed scratch
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (s) {  // the scratch address is the current device's: the stream must belong to it
    int cur = 0, sdev = 0;
    PS_CUDA(cudaGetDevice(&cur));
    PS_CUDA(cudaStreamGetDevice(s, &sdev));
    if (sdev != cur) return PS_ERR_INVALID;
  }
  NaScratch* sc = nullptr;
  PS_TRY(na_scratch(&sc));
  uint64_t slots = 1;
  while (slots < (uint64_t)(2 * nt)) slots <<= 1;
  // clear the part of the scratch this call reads: the used table slots and the accumulators
  PS_CUDA(cudaMemsetAsync(sc->key, 0xFF, slots * sizeof(ulonglong2), s));
  PS_CUDA(cudaMemsetAsync(sc->acc, 0, sizeof(sc->acc), s));
  // ones_idx = -1 (all bytes 0xFF); top = 0x80808080, below the -100000 "no product" mark
  // (memsets: no host copy from pageable memory)
  PS_CUDA(cudaMemsetAsync(&sc->ones_idx, 0xFF, sizeof(sc->ones_idx), s));
  PS_CUDA(cudaMemsetAsync(&sc->top, 0x80, sizeof(sc->top), s));
  const int nsm = num_sms();
  int bt = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nt, 256), 4 * nsm));
  int bp = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(np, kRedThreads), 4 * nsm));
  PS_LAUNCH("k_na_build", s, k_na_build<<<bt, 256, 0, s>>>(T, nt, sc, slots - 1));
  PS_CUDA(cudaGetLastError());
  PS_LAUNCH("k_na_top", s, k_na_top<<<bp, kRedThreads, 0, s>>>(P, np, T, sc, slots - 1));
  PS_CUDA(cudaGetLastError());
  PS_LAUNCH("k_na_acc", s, k_na_acc<<<bp, kRedThreads, 0, s>>>(P, np, T, sc, slots - 1));
  PS_CUDA(cudaGetLastError());
  std::vector<long long> h(2 * kNaSpan);
  int top = 0, wlo[2] = {0, 0};
  PS_CUDA(cudaMemcpyAsync(h.data(), sc->acc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&top, &sc->top, sizeof(int), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(wlo, sc->wlo, sizeof(wlo), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  if (top <= -100000) return PS_OK;
  if (top >= kTopInf) {
    *re = *im = std::nan("");
    return PS_OK;
  }
  std::vector<long long> fre(h.begin() + kWinDigits, h.begin() + kNaSpan);
  std::vector<long long> fim(h.begin() + kNaSpan + kWinDigits, h.end());
  *re = round_exact(fre, h.data(), wlo[0]);
  *im = round_exact(fim, h.data() + kNaSpan, wlo[1]);
  return PS_OK;
}
