// Batched instances: many independent problems (for example disorder realisations of one
// chain, H_b = sum of common terms + sum_i h_i^(b) Z_i) evolved together in one sum.  A
// string of instance b carries b in its high v bits, as Z letters on sites above the
// chain (key = (v | b << tag_shift, w)).  Those bits are transparent to the method: the
// common H strings have no bits there, so the anticommutation test, the product phase
// and the XOR of the masks leave the tag of x unchanged in every product, and sums and
// merges never mix instances.  What differs per instance is supplied per instance: the
// coefficient of each H term (read by the emission from a table indexed by the tag) and
// the truncation cap (a top-k per instance, selected in one pass sequence for all).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "select.cuh"

struct pauli_batch {
  int n_inst;
  int tag_shift;
  int nH;
  cudaStream_t stream;
  double* hcoef;             // device [n_inst][nH]
  double* huni;              // device [nH]: a term's coefficient when every instance has it, else NaN
  std::vector<int64_t> cap;  // per-instance cap (<= 0: none)
};

namespace ps {
namespace {

constexpr int kBT = 256;

__device__ __forceinline__ uint32_t inst_of(const Rec& r, int shift) { return (uint32_t)(r.v >> shift); }

// Strings per instance; *bad = 1 for a string whose tag is out of range or whose w has bits
// at or above the tag position.
__global__ void __launch_bounds__(kBT) k_bcount(const Rec* __restrict__ d, int64_t n, int shift, int n_inst,
                                                unsigned long long* __restrict__ cnt, int* __restrict__ bad) {
  extern __shared__ unsigned long long s_cnt[];
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Rec r = d[i];
    const uint64_t b = r.v >> shift;
    if (b >= (uint64_t)n_inst || (r.w >> shift) != 0) {
      *bad = 1;
      continue;
    }
    atomicAdd(&s_cnt[b], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
}

// sum |c|^2 per instance (FP64 atomics: the order of the additions is not fixed).
__global__ void __launch_bounds__(kBT) k_bnorm(const Rec* __restrict__ d, int64_t n, int shift, int n_inst,
                                               double* __restrict__ acc) {
  extern __shared__ double s_acc[];
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) s_acc[i] = 0.0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const Rec r = d[i];
    const uint32_t b = inst_of(r, shift);
    if (b < (uint32_t)n_inst) atomicAdd(&s_acc[b], __dadd_rn(__dmul_rn(r.re, r.re), __dmul_rn(r.im, r.im)));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x)
    if (s_acc[i] != 0.0) atomicAdd(&acc[i], s_acc[i]);
}

// Rank keys (|c|^2 bit patterns: non-negative doubles order like their bits), instance tags
// and per-instance string counts in one read of the records (the tags of the library's own merges are in range: every step validates them first).
__global__ void __launch_bounds__(kBT) k_bkeys_tags(const Rec* __restrict__ d, int64_t n, int shift, int n_inst,
                                                    uint64_t* __restrict__ ab, uint16_t* __restrict__ tag,
                                                    unsigned long long* __restrict__ cnt) {
  extern __shared__ unsigned long long s_cnt[];
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) s_cnt[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    uint32_t b = 0xFFFFFFFFu;
    if (i < n) {
      const Rec r = d[i];
      const double x = is_zero(r.re) ? 0.0 : __dmul_rn(r.re, r.re);
      const double y = is_zero(r.im) ? 0.0 : __dmul_rn(r.im, r.im);
      ab[i] = (uint64_t)__double_as_longlong(add_rn(x, y));
      b = inst_of(r, shift);
      tag[i] = (uint16_t)b;
    }
    // one shared-memory add per instance present in the warp (few instances: hot counters)
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (i < n && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[b], (unsigned long long)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x)
    if (s_cnt[i]) atomicAdd(&cnt[i], s_cnt[i]);
}

// One digit pass for every instance still selecting: hist[b][digit] over the strings whose
// rank key matches b's prefix; over all strings (list null) or over a candidate list.  The
// record is read only for the digits beyond the |c|^2 bits.  One global add per distinct
// (instance, digit) in the warp: with few instances and clustered exponents the plain adds
// pile up on a few counters.
__global__ void __launch_bounds__(kBT) k_bhist(const Rec* __restrict__ d, const uint64_t* __restrict__ ab,
                                               const uint16_t* __restrict__ tag, int64_t n,
                                               const uint32_t* __restrict__ list,
                                               const unsigned long long* __restrict__ nlist,
                                               const SelState* __restrict__ st, const int* __restrict__ act, int pass,
                                               unsigned* __restrict__ hist) {
  const bool need_key = (pass + 1) * kDigitBits > 64;
  const int64_t m = list ? (int64_t)*nlist : n;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; j0 < m; j0 += stride) {
    const int64_t j = j0 + lane;
    uint32_t code = 0xFFFFFFFFu, b = 0, dg = 0;
    if (j < m) {
      const int64_t i = list ? (int64_t)list[j] : j;
      b = tag[i];
      if (act[b] && !st[b].done) {
        uint64_t k[3];
        const uint64_t g = ab[i];
        if (need_key) {
          const Rec r = d[i];
          rank_key(g, &r, k);
        } else {
          rank_key(g, nullptr, k);
        }
        if (matches_prefix(k, st[b], pass)) {
          dg = rank_digit(k, pass);
          code = (b << kDigitBits) | dg;
        }
      }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, code);
    if (code != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
      atomicAdd(&hist[(size_t)b * kBins + dg], (unsigned)__popc(peers));
  }
}

// The candidates still selecting after the first digits: every string of a selecting instance
// whose rank key matches the instance's prefix (warp-aggregated appends).
__global__ void __launch_bounds__(kBT) k_bnarrow(const uint64_t* __restrict__ ab, const uint16_t* __restrict__ tag,
                                                 int64_t n, const SelState* __restrict__ st,
                                                 const int* __restrict__ act, int pass, uint32_t* __restrict__ list,
                                                 unsigned long long* __restrict__ nlist) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~(int64_t)31; i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    bool keep = false;
    if (i < n) {
      const uint32_t b = tag[i];
      if (act[b] && !st[b].done) {
        uint64_t k[3];
        rank_key(ab[i], nullptr, k);
        keep = matches_prefix(k, st[b], pass);
      }
    }
    const unsigned mk = __ballot_sync(0xffffffffu, keep);
    unsigned long long base = 0;
    if (lane == 0 && mk) base = atomicAdd(nlist, (unsigned long long)__popc(mk));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) list[base + __popc(mk & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

// One block per instance: pick the digit; count the instances that finished.
__global__ void __launch_bounds__(256) k_bpick(SelState* st, const int* __restrict__ act, int pass,
                                               unsigned* __restrict__ hist, unsigned* __restrict__ n_done) {
  const int b = blockIdx.x;
  if (!act[b]) return;
  const int was = st[b].done;
  if (was) return;
  sel_pick_block(&st[b], pass, hist + (size_t)b * kBins);
  __syncthreads();
  if (threadIdx.x == 0 && st[b].done) atomicAdd(n_done, 1u);
}

// Keep a string iff its instance is not capped or its rank key reaches the instance's
// threshold.  Tiles of kBT * kBTI strings, one output reservation per tile: the kept strings
// keep their order within a tile (the merge's bin order, on which the next emission's slot
// reservations rely).
constexpr int kBTI = 4;
__global__ void __launch_bounds__(kBT) k_bcompact(const Rec* __restrict__ d, const uint64_t* __restrict__ ab,
                                                  const uint16_t* __restrict__ tag, int64_t n,
                                                  const SelState* __restrict__ st, const int* __restrict__ act,
                                                  Rec* __restrict__ out, unsigned long long* __restrict__ n_out) {
  __shared__ TileSlots<kBT, kBTI> s_res;
  const int64_t tile_n = (int64_t)kBT * kBTI;
  const int64_t tiles = (n + tile_n - 1) / tile_n;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    bool kp[kBTI];
    Rec r[kBTI];
#pragma unroll
    for (int k = 0; k < kBTI; ++k) {
      const int64_t i = tile * tile_n + (int64_t)k * kBT + threadIdx.x;
      kp[k] = false;
      if (i < n) {
        r[k] = d[i];
        const uint32_t b = tag[i];
        if (!act[b]) {
          kp[k] = true;
        } else {
          uint64_t key[3];
          rank_key(ab[i], &r[k], key);
          const SelState& s = st[b];
          kp[k] = key[0] > s.prefix[0] ||
                  (key[0] == s.prefix[0] && (key[1] > s.prefix[1] || (key[1] == s.prefix[1] && key[2] >= s.prefix[2])));
        }
      }
    }
    unsigned long long pos[kBTI];
    tile_slots<kBT, kBTI>(kp, s_res, n_out, pos);
#pragma unroll
    for (int k = 0; k < kBTI; ++k)
      if (kp[k]) out[pos[k]] = r[k];
  }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kBT), 8 * num_sms())); }

int counts_run(const pauli_batch* B, const pauli_sum* O, std::vector<unsigned long long>& h) {
  cudaStream_t s = O->stream;
  h.assign((size_t)B->n_inst, 0ull);
  if (O->n == 0) return PS_OK;
  Buf<unsigned long long> cnt;
  Buf<int> bad;
  PS_TRY(cnt.alloc((size_t)B->n_inst, s));
  PS_TRY(bad.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)B->n_inst * sizeof(unsigned long long), s));
  PS_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  PS_LAUNCH("k_bcount", s,
            k_bcount<<<grid_of(O->n), kBT, (size_t)B->n_inst * sizeof(unsigned long long), s>>>(
                O->d, O->n, B->tag_shift, B->n_inst, cnt.p, bad.p));
  PS_CUDA(cudaGetLastError());
  int hbad = 0;
  PS_CUDA(cudaMemcpyAsync(h.data(), cnt.p, (size_t)B->n_inst * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  return hbad ? PS_ERR_INVALID : PS_OK;
}

// Per-instance top-k by |c|^2 (ties to the smaller key) for every instance over its cap: one
// read of the records gives the rank keys, the instance tags and the counts; the first two
// digit passes run over keys and tags (10 bytes per string); the strings still tied with
// their instance's threshold after them are listed, and the remaining passes run over the list.
int batch_truncate(const pauli_batch* B, pauli_sum* O) {
  cudaStream_t s = O->stream;
  if (O->n == 0) return PS_OK;
  Buf<uint64_t> ab;
  Buf<uint16_t> tag;
  Buf<unsigned long long> dcnt;
  PS_TRY(ab.alloc((size_t)O->n, s));
  PS_TRY(tag.alloc((size_t)O->n, s));
  PS_TRY(dcnt.alloc((size_t)B->n_inst, s));
  PS_CUDA(cudaMemsetAsync(dcnt.p, 0, (size_t)B->n_inst * sizeof(unsigned long long), s));
  PS_LAUNCH("k_bkeys", s,
            k_bkeys_tags<<<grid_of(O->n), kBT, (size_t)B->n_inst * sizeof(unsigned long long), s>>>(
                O->d, O->n, B->tag_shift, B->n_inst, ab.p, tag.p, dcnt.p));
  PS_CUDA(cudaGetLastError());
  std::vector<unsigned long long> cnt((size_t)B->n_inst);
  PS_CUDA(cudaMemcpyAsync(cnt.data(), dcnt.p, cnt.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  PS_CUDA(cudaStreamSynchronize(s));
  std::vector<int> act((size_t)B->n_inst, 0);
  std::vector<SelState> st((size_t)B->n_inst);
  int n_act = 0;
  for (int b = 0; b < B->n_inst; ++b) {
    st[(size_t)b] = SelState{};
    const int64_t cap = B->cap[(size_t)b];
    if (cap > 0 && (int64_t)cnt[(size_t)b] > cap) {
      act[(size_t)b] = 1;
      st[(size_t)b].need = (unsigned long long)cap;
      ++n_act;
    }
  }
  if (n_act == 0) return PS_OK;
  Buf<int> dact;
  Buf<SelState> dst;
  Buf<unsigned> hist, ndone;
  Buf<uint32_t> list;
  Buf<unsigned long long> nlist;
  PS_TRY(dact.alloc((size_t)B->n_inst, s));
  PS_TRY(dst.alloc((size_t)B->n_inst, s));
  PS_TRY(hist.alloc((size_t)B->n_inst * kBins, s));
  PS_TRY(ndone.alloc(1, s));
  PS_TRY(nlist.alloc(1, s));
  const bool narrow = O->n <= (int64_t)0xFFFFFFFF;  // 32-bit candidate indices
  if (narrow) PS_TRY(list.alloc((size_t)O->n, s));
  PS_CUDA(cudaMemcpyAsync(dact.p, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  PS_CUDA(cudaMemcpyAsync(dst.p, st.data(), st.size() * sizeof(SelState), cudaMemcpyHostToDevice, s));
  PS_CUDA(cudaMemsetAsync(hist.p, 0, (size_t)B->n_inst * kBins * sizeof(unsigned), s));
  PS_CUDA(cudaMemsetAsync(ndone.p, 0, sizeof(unsigned), s));
  PS_CUDA(cudaMemsetAsync(nlist.p, 0, sizeof(unsigned long long), s));
  constexpr int kNarrowAt = 2;  // digits fixed over all strings before the candidates are listed
  for (int pass = 0; pass < kPasses; ++pass) {
    if (narrow && pass == kNarrowAt)
      PS_LAUNCH("k_bnarrow", s,
                k_bnarrow<<<grid_of(O->n), kBT, 0, s>>>(ab.p, tag.p, O->n, dst.p, dact.p, pass, list.p, nlist.p));
    const bool listed = narrow && pass >= kNarrowAt;
    PS_LAUNCH("k_bhist", s,
              k_bhist<<<grid_of(O->n), kBT, 0, s>>>(O->d, ab.p, tag.p, O->n, listed ? list.p : nullptr,
                                                    listed ? nlist.p : nullptr, dst.p, dact.p, pass, hist.p));
    PS_LAUNCH("k_bpick", s, k_bpick<<<B->n_inst, 256, 0, s>>>(dst.p, dact.p, pass, hist.p, ndone.p));
    if (pass == 4 || pass == 8 || pass == 12) {  // every instance usually settles within the |c|^2 digits
      unsigned nd = 0;
      PS_CUDA(cudaMemcpyAsync(&nd, ndone.p, sizeof(nd), cudaMemcpyDeviceToHost, s));
      PS_CUDA(cudaStreamSynchronize(s));
      if ((int)nd == n_act) break;
    }
  }
  PS_CUDA(cudaGetLastError());
  Rec* outb = nullptr;
  Buf<unsigned long long> nout;
  PS_TRY(nout.alloc(1, s));
  PS_CUDA(cudaMemsetAsync(nout.p, 0, sizeof(unsigned long long), s));
  PS_TRY(dev_alloc((void**)&outb, (size_t)O->n * sizeof(Rec), s));
  PS_LAUNCH("k_bcompact", s,
            k_bcompact<<<grid_of(O->n), kBT, 0, s>>>(O->d, ab.p, tag.p, O->n, dst.p, dact.p, outb, nout.p));
  cudaError_t e = cudaGetLastError();
  unsigned long long nk = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nk, nout.p, sizeof(nk), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(outb, s);
    set_cuda_error(e, "batch truncate");
    return PS_ERR_CUDA;
  }
  return sum_adopt(O, outb, O->n, (int64_t)nk);
}

struct BTmp {
  pauli_sum s;
  explicit BTmp(const pauli_sum* like) : s{like->n_sites, like->stream, nullptr, 0, 0, 0, like->f32, like->W} {}
  ~BTmp() { dev_free(s.d, s.stream); }
  BTmp(const BTmp&) = delete;
  BTmp& operator=(const BTmp&) = delete;
};

int merge_r(const MergeSpec& sp, pauli_sum* out) { return merge_run(sp, out->stream, out); }

MergeSource src_of(const pauli_sum* p, double a) {
  MergeSource m{p->d, p->n, Cx{a, 0.0}};
  m.cls = p->cls;
  return m;
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" {

int pauli_batch_create(const pauli_sum* H, const double* hcoef, int n_inst, int tag_shift, const int64_t* caps,
                       pauli_batch** out) {
  PS_NARROW(H);
  if (!out) return PS_ERR_INVALID;
  *out = nullptr;
  if (!H || !hcoef || n_inst < 1 || n_inst > 4096 || tag_shift < 1 || tag_shift > 63) return PS_ERR_INVALID;
  if (H->n < 1 || H->n > 256 || (H->cls & kClsImag)) return PS_ERR_INVALID;
  int tbits = 0;  // bits of the largest tag
  while ((1ll << tbits) < (long long)n_inst) ++tbits;
  if (tag_shift + tbits > H->n_sites) return PS_ERR_INVALID;  // tagged keys must be keys of the sums
  // H's strings must lie below the tag bits
  std::vector<Rec> hh((size_t)H->n);
  PS_CUDA(cudaMemcpyAsync(hh.data(), H->d, hh.size() * sizeof(Rec), cudaMemcpyDeviceToHost, H->stream));
  PS_CUDA(cudaStreamSynchronize(H->stream));
  for (const Rec& r : hh)
    if ((r.v >> tag_shift) || (r.w >> tag_shift)) return PS_ERR_INVALID;
  const size_t nc = (size_t)n_inst * (size_t)H->n;
  for (size_t i = 0; i < nc; ++i)
    if (!std::isfinite(hcoef[i])) return PS_ERR_INVALID;
  pauli_batch* b = new pauli_batch{};
  b->n_inst = n_inst;
  b->tag_shift = tag_shift;
  b->nH = (int)H->n;
  b->stream = H->stream;
  b->cap.assign((size_t)n_inst, 0);
  if (caps)
    for (int i = 0; i < n_inst; ++i) b->cap[(size_t)i] = caps[i];
  // terms whose coefficient is the same (bit for bit) in every instance
  std::vector<double> uni((size_t)H->n);
  for (size_t h = 0; h < (size_t)H->n; ++h) {
    uni[h] = hcoef[h];
    for (int i = 1; i < n_inst; ++i)
      if (std::memcmp(&hcoef[(size_t)i * (size_t)H->n + h], &uni[h], sizeof(double)) != 0) {
        uni[h] = std::nan("");
        break;
      }
  }
  int st = dev_alloc((void**)&b->hcoef, nc * sizeof(double), b->stream);
  if (st == PS_OK) st = dev_alloc((void**)&b->huni, uni.size() * sizeof(double), b->stream);
  if (st != PS_OK) {
    dev_free(b->hcoef, b->stream);
    delete b;
    return st;
  }
  cudaError_t e = cudaMemcpyAsync(b->hcoef, hcoef, nc * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->huni, uni.data(), uni.size() * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    dev_free(b->hcoef, b->stream);
    dev_free(b->huni, b->stream);
    delete b;
    set_cuda_error(e, "pauli_batch_create");
    return PS_ERR_CUDA;
  }
  *out = b;
  return PS_OK;
}

int pauli_batch_destroy(pauli_batch* b) {
  if (!b) return PS_OK;
  dev_free(b->hcoef, b->stream);
  dev_free(b->huni, b->stream);
  delete b;
  return PS_OK;
}

int pauli_batch_counts(const pauli_batch* b, const pauli_sum* O, int64_t* counts) {
  PS_NARROW(O);
  if (!b || !O || !counts) return PS_ERR_INVALID;
  std::vector<unsigned long long> h;
  PS_TRY(counts_run(b, O, h));
  for (int i = 0; i < b->n_inst; ++i) counts[i] = (int64_t)h[(size_t)i];
  return PS_OK;
}

int pauli_batch_norms(const pauli_batch* b, const pauli_sum* O, double* norms) {
  PS_NARROW(O);
  if (!b || !O || !norms) return PS_ERR_INVALID;
  cudaStream_t s = O->stream;
  std::vector<double> h((size_t)b->n_inst, 0.0);
  if (O->n > 0) {
    Buf<double> acc;
    PS_TRY(acc.alloc((size_t)b->n_inst, s));
    PS_CUDA(cudaMemsetAsync(acc.p, 0, (size_t)b->n_inst * sizeof(double), s));
    PS_LAUNCH("k_bnorm", s,
              k_bnorm<<<grid_of(O->n), kBT, (size_t)b->n_inst * sizeof(double), s>>>(O->d, O->n, b->tag_shift,
                                                                                       b->n_inst, acc.p));
    PS_CUDA(cudaGetLastError());
    PS_CUDA(cudaMemcpyAsync(h.data(), acc.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
  }
  for (int i = 0; i < b->n_inst; ++i) norms[i] = std::sqrt(h[(size_t)i]);
  return PS_OK;
}

int pauli_batch_rk4_steps(const pauli_batch* b, const pauli_sum* H, pauli_sum* O, double dt, int trim_stages,
                          int n_steps, int* steps_done) {
  if (steps_done) *steps_done = 0;
  if (n_steps < 0) return PS_ERR_INVALID;
  for (int k = 0; k < n_steps; ++k) {
    PS_TRY(pauli_batch_rk4_step(b, H, O, dt, trim_stages));
    if (steps_done) *steps_done = k + 1;
  }
  return PS_OK;
}

int pauli_batch_truncate(const pauli_batch* b, pauli_sum* O) {
  PS_NARROW(O);
  if (!b || !O) return PS_ERR_INVALID;
  return batch_truncate(b, O);
}

int pauli_batch_rk4_step(const pauli_batch* b, const pauli_sum* H, pauli_sum* O, double dt, int trim_stages) {
  PS_NARROW(O);
  NvtxRange nvtx("pauli_batch_rk4_step");
  if (!b || !H || !O || H == O || H->n != b->nH || H->n_sites != O->n_sites || !std::isfinite(dt))
    return PS_ERR_INVALID;
  if ((O->cls & kClsImag) || (H->cls & kClsImag)) return PS_ERR_INVALID;  // real coefficients (single-component products)
  if (H->stream != O->stream) PS_CUDA(cudaStreamSynchronize(H->stream));
  std::vector<unsigned long long> cnt;
  PS_TRY(counts_run(b, O, cnt));  // every tag in range before the emission reads the table by tag
  const double h2 = dt / 2.0, h6 = dt / 6.0;
  BTmp k1(O), k2(O), k3(O), k4(O), X(O);
  auto L = [&](const pauli_sum* in, pauli_sum* k) -> int {
    MergeSpec sp;
    sp.H = H->d;
    sp.nH = (int)H->n;
    sp.X = in->d;
    sp.nX = in->n;
    sp.rot = 1;
    sp.clsH = H->cls;
    sp.clsX = in->cls;
    sp.hbatch = b->hcoef;
    sp.hbatch_uniform = b->huni;
    sp.hb_shift = b->tag_shift;
    PS_TRY(merge_r(sp, k));
    if (trim_stages) PS_TRY(batch_truncate(b, k));
    return PS_OK;
  };
  auto stage_input = [&](const pauli_sum* k, double a) -> int {
    MergeSpec sp;
    sp.src[0] = src_of(O, 1.0);
    sp.src[1] = src_of(k, a);
    sp.nsrc = 2;
    return merge_r(sp, &X.s);
  };
  PS_TRY(L(O, &k1.s));
  PS_TRY(stage_input(&k1.s, h2));
  PS_TRY(L(&X.s, &k2.s));
  PS_TRY(stage_input(&k2.s, h2));
  PS_TRY(L(&X.s, &k3.s));
  PS_TRY(stage_input(&k3.s, dt));
  PS_TRY(L(&X.s, &k4.s));
  MergeSpec sp;
  sp.src[0] = src_of(&k1.s, 1.0);
  sp.src[1] = src_of(&k2.s, 2.0);
  sp.src[2] = src_of(&k3.s, 2.0);
  sp.src[3] = src_of(&k4.s, 1.0);
  sp.nsrc = 4;
  sp.pre = O->d;
  sp.npre = O->n;
  sp.clsPre = O->cls;
  sp.has_post = true;
  sp.post = Cx{h6, 0.0};
  PS_TRY(merge_r(sp, &X.s));
  PS_TRY(batch_truncate(b, &X.s));
  std::swap(O->d, X.s.d);
  std::swap(O->cap, X.s.cap);
  std::swap(O->n, X.s.n);
  std::swap(O->cls, X.s.cls);
  return PS_OK;
}

}  // extern "C"
