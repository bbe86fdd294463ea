// C ABI entry points: commutator, add, truncate, RK4 step, Lanczos step, trace product, norm.
#include <algorithm>
#include <cmath>
#include <utility>

#include "common.cuh"

using namespace ps;

namespace {

// The merge (into an FP32 sum it rounds every output coefficient once to FP32 itself).
int merge_into(const MergeSpec& sp, cudaStream_t s, pauli_sum* out) { return merge_run(sp, s, out); }

bool same_sites(const pauli_sum* a, const pauli_sum* b) { return !a || !b || a->n_sites == b->n_sites; }

// A library-internal temporary sum on a given stream.
struct Tmp {
  pauli_sum s;
  explicit Tmp(const pauli_sum* like) : s{like->n_sites, like->stream, nullptr, 0, 0, 0, like->f32, like->W} {}
  ~Tmp() { dev_free(s.d, s.stream); }
  Tmp(const Tmp&) = delete;
  Tmp& operator=(const Tmp&) = delete;
};

void swap_contents(pauli_sum* a, pauli_sum* b) {
  std::swap(a->d, b->d);
  std::swap(a->cap, b->cap);
  std::swap(a->n, b->n);
  std::swap(a->cls, b->cls);
}

MergeSource source(const pauli_sum* p, Cx alpha) {
  MergeSource m{p->d, p->n, alpha};
  m.cls = p->cls;
  return m;
}

// k = i[H, X] (rot = 1) or [H, X] (rot = 0) into out.
// keys (optional): receives the output's rank keys |x| when the merge can write them (see
// MergeSpec::keys_out; null otherwise), owned by the caller.
int commutator_into(const pauli_sum* H, const pauli_sum* X, int rot, pauli_sum* out, uint64_t** keys = nullptr) {
  MergeSpec sp;
  sp.H = H->d;
  sp.nH = (int)H->n;
  sp.X = X->d;
  sp.nX = X->n;
  sp.rot = rot;
  sp.clsH = H->cls;
  sp.clsX = X->cls;
  Buf<int> top;
  if (keys) {
    PS_TRY(top.alloc(1, out->stream));
    PS_CUDA(cudaMemsetAsync(top.p, 0x80, sizeof(int), out->stream));
    sp.keys_out = keys;
    sp.keys_top = top.p;
  }
  return merge_into(sp, out->stream, out);
}

bool policy_valid(const pauli_trunc_policy* p, const pauli_sum* O = nullptr) {
  if (!p) return true;
  return std::isfinite(p->cutoff) && std::isfinite(p->gamma) && p->max_weight <= (O ? 64 * O->W : 64);
}

// translation symmetry

int ts_merge(const pauli_sum* X, int mode, pauli_sum* out) {
  MergeSpec sp;
  sp.src[0] = source(X, Cx{1.0, 0.0});
  sp.src[0].ts = mode;
  sp.nsrc = 1;
  sp.ring = X->n_sites;
  return merge_into(sp, out->stream, out);
}

// H written out as the list of H0's translates T_0(H0), T_1(H0), ... (not merged).
int ts_translates_into(const pauli_sum* H0, pauli_sum* out) {
  const int64_t n = H0->n * H0->n_sites;
  if (n > 0xEFFF) return PS_ERR_INVALID;
  PS_TRY(sum_reserve(out, n, false));
  PS_TRY(ts_translates(H0->d, H0->n, H0->n_sites, out->stream, out->d));
  out->n = n;
  out->cls = H0->cls;
  return PS_OK;
}

// Generator of [H, O] (ts_commutator of the oracle): [translates of H0, O_0] moved to
// representatives.
int ts_commutator_into(const pauli_sum* H0, const pauli_sum* O0, pauli_sum* out) {
  Tmp Hf(O0), C(O0);
  PS_TRY(ts_translates_into(H0, &Hf.s));
  PS_TRY(commutator_into(&Hf.s, O0, 0, &C.s));
  return ts_merge(&C.s, kTsCanon, out);
}

bool ts_ok(const pauli_sum* s) { return s && s->n_sites >= 2; }

}  // namespace

extern "C" {

int pauli_commutator(const pauli_sum* H, const pauli_sum* O, pauli_sum* out) {
  NvtxRange nvtx("pauli_commutator");
  if (!H || !O || !out || out == H || out == O) return PS_ERR_INVALID;
  if (!same_sites(H, O) || !same_sites(O, out)) return PS_ERR_INVALID;
  if (H->n > 0xEFFF) return PS_ERR_INVALID;
  if (H->stream != out->stream) PS_CUDA(cudaStreamSynchronize(H->stream));
  if (O->stream != out->stream) PS_CUDA(cudaStreamSynchronize(O->stream));
  if (O->W > 1) return wide_api::commutator(H, O, 0, out);
  return commutator_into(H, O, 0, out);
}

int pauli_multiply(const pauli_sum* A, const pauli_sum* B, pauli_sum* out) {
  NvtxRange nvtx("pauli_multiply");
  if (!A || !B || !out || out == A || out == B) return PS_ERR_INVALID;
  if (!same_sites(A, B) || !same_sites(B, out)) return PS_ERR_INVALID;
  PS_NARROW(A);
  if (A->n > 0xEFFF) return PS_ERR_INVALID;
  if (A->stream != out->stream) PS_CUDA(cudaStreamSynchronize(A->stream));
  if (B->stream != out->stream) PS_CUDA(cudaStreamSynchronize(B->stream));
  MergeSpec sp;
  sp.H = A->d;
  sp.nH = (int)A->n;
  sp.X = B->d;
  sp.nX = B->n;
  sp.product = true;
  sp.clsH = A->cls;
  sp.clsX = B->cls;
  return merge_into(sp, out->stream, out);
}


int pauli_ts_expand(const pauli_sum* G, pauli_sum* out) {
  PS_NARROW(G);
  if (!ts_ok(G) || !out || out == G || !same_sites(G, out)) return PS_ERR_INVALID;
  if (G->stream != out->stream) PS_CUDA(cudaStreamSynchronize(G->stream));
  return ts_merge(G, kTsExpand, out);
}

int pauli_ts_canonicalize(const pauli_sum* X, pauli_sum* out) {
  PS_NARROW(X);
  if (!ts_ok(X) || !out || out == X || !same_sites(X, out)) return PS_ERR_INVALID;
  if (X->stream != out->stream) PS_CUDA(cudaStreamSynchronize(X->stream));
  return ts_merge(X, kTsCanon, out);
}

int pauli_ts_commutator(const pauli_sum* H0, const pauli_sum* O0, pauli_sum* out) {
  PS_NARROW(H0);
  PS_NARROW(O0);
  if (!ts_ok(H0) || !ts_ok(O0) || !out || out == H0 || out == O0) return PS_ERR_INVALID;
  if (!same_sites(H0, O0) || !same_sites(O0, out)) return PS_ERR_INVALID;
  if (H0->stream != out->stream) PS_CUDA(cudaStreamSynchronize(H0->stream));
  if (O0->stream != out->stream) PS_CUDA(cudaStreamSynchronize(O0->stream));
  return ts_commutator_into(H0, O0, out);
}

int pauli_ts_norm(const pauli_sum* O0, double* out) {
  PS_NARROW(O0);
  if (!ts_ok(O0) || !out) return PS_ERR_INVALID;
  double n2 = 0.0;
  PS_TRY(exact_norm2(O0->d, O0->n, O0->stream, &n2, O0->n_sites));
  *out = std::sqrt(n2);
  return PS_OK;
}

int pauli_ts_lanczos_step(const pauli_sum* H0, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev,
                          const pauli_trunc_policy* policy, double* b_out) {
  PS_NARROW(H0);
  PS_NARROW(O_cur);
  if (!ts_ok(H0) || !O_prev || !O_cur || !b_out || O_prev == O_cur || H0 == O_prev || H0 == O_cur)
    return PS_ERR_INVALID;
  if (!same_sites(H0, O_cur) || !same_sites(O_prev, O_cur) || !policy_valid(policy) || !std::isfinite(b_prev))
    return PS_ERR_INVALID;
  *b_out = 0.0;
  Tmp Hf(O_cur), C(O_cur), A(O_cur);
  PS_TRY(ts_translates_into(H0, &Hf.s));
  PS_TRY(commutator_into(&Hf.s, O_cur, 0, &C.s));
  // A_0 = C_0 - b_prev O_prev (representatives in shift order, then the O_prev term)
  MergeSpec sp;
  sp.src[0] = source(&C.s, Cx{1.0, 0.0});
  sp.src[0].ts = kTsCanon;
  sp.nsrc = 1;
  if (O_prev->n > 0) {
    sp.src[1] = source(O_prev, Cx{-b_prev, 0.0});
    sp.nsrc = 2;
  }
  sp.ring = O_cur->n_sites;
  PS_TRY(merge_into(sp, O_cur->stream, &A.s));
  double n2 = 0.0;
  PS_TRY(exact_norm2(A.s.d, A.s.n, A.s.stream, &n2, O_cur->n_sites));
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
  PS_TRY(truncate_run(&A.s, &p, nullptr, 0.0, &b));
  swap_contents(O_prev, O_cur);
  swap_contents(O_cur, &A.s);
  return PS_OK;
}

int pauli_add(const pauli_sum* A, double alpha_re, double alpha_im, const pauli_sum* B, pauli_sum* out) {
  if (!A || !B || !out || out == A || out == B) return PS_ERR_INVALID;
  if (!same_sites(A, B) || !same_sites(A, out)) return PS_ERR_INVALID;
  if (A->W > 1) return wide_api::add(A, Cx{alpha_re, alpha_im}, B, out);
  MergeSpec sp;
  sp.src[0] = source(A, Cx{1.0, 0.0});
  sp.src[1] = source(B, Cx{alpha_re, alpha_im});
  sp.nsrc = 2;
  return merge_into(sp, out->stream, out);
}

int pauli_truncate(pauli_sum* O, const pauli_trunc_policy* policy, const pauli_sum* keep, double dt) {
  NvtxRange nvtx("pauli_truncate");
  if (!O || !same_sites(O, keep) || !policy_valid(policy, O) || !std::isfinite(dt)) return PS_ERR_INVALID;
  if (O->W > 1) return wide_api::truncate(O, policy, keep, dt, nullptr);
  return truncate_run(O, policy, keep, dt, nullptr);
}

int pauli_autotune_commutator(const pauli_sum* H, const pauli_sum* O, int reps, int* best_bin_target,
                              int* best_quota, double* best_ms, double* default_ms) {
  PS_NARROW(O);
  if (!H || !O || H == O || !same_sites(H, O) || H->n > 0xEFFF || reps < 1) return PS_ERR_INVALID;
  if (H->stream != O->stream) PS_CUDA(cudaStreamSynchronize(H->stream));
  Tmp out(O);
  MergeSpec sp;
  sp.H = H->d;
  sp.nH = (int)H->n;
  sp.X = O->d;
  sp.nX = O->n;
  sp.clsH = H->cls;
  sp.clsX = O->cls;
  return autotune_commutator(sp, &out.s, reps, best_bin_target, best_quota, best_ms, default_ms);
}

int pauli_autotune_reset(void) {
  autotune_reset();
  return PS_OK;
}

int pauli_merge_geometry_fix(int bin_target, int quota) { return merge_geometry_fix(bin_target, quota); }

int pauli_truncate_scored(pauli_sum* O, const pauli_trunc_policy* policy, const pauli_sum* keep, double dt,
                          const double* score) {
  PS_NARROW(O);
  if (!O || !same_sites(O, keep) || !policy_valid(policy) || !std::isfinite(dt)) return PS_ERR_INVALID;
  if (O->n > 0 && !score) return PS_ERR_INVALID;
  return truncate_run(O, policy, keep, dt, nullptr, score);
}

}  // extern "C"

namespace {

// One RK4 step; the final truncation ranks by the learned score when a model is given;
// cand (optional) receives the step's result before that truncation.
int rk4_impl(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* policy, const pauli_sum* keep,
             const pauli_mlp* model, pauli_sum* cand) {
  NvtxRange nvtx(model ? "rk4_step (learned truncation)" : "rk4_step");
  const double h2 = dt / 2.0, h6 = dt / 6.0;
  const bool trim = policy && policy->trim_stages && policy->top_k > 0;
  pauli_trunc_policy stage{-1, 0.0, policy ? policy->top_k : 0, 0.0, 0};
  Tmp k1(O), k2(O), k3(O), k4(O), X(O);
  auto L = [&](const pauli_sum* in, pauli_sum* k) -> int {
    NvtxRange r("k_j = i[H, X]");
    if (!trim) return commutator_into(H, in, 1, k);
    // the stage trim is top-k alone: on a single-component k_j it ranks the rank keys |x| that
    // the merge writes (the division-free top-k of the Lanczos step with divisor 1, which keeps
    // the same strings as the general path), else the general path
    uint64_t* keys = nullptr;
    PS_TRY(commutator_into(H, in, 1, k, &keys));
    Buf<uint64_t> kb;
    if (keys) kb.adopt(keys, (size_t)k->n, k->stream);
    if (kb.p && k->n > stage.top_k) {
      Buf<unsigned> hist;
      PS_TRY(hist.alloc(kKeyBins, k->stream));
      PS_TRY(key_first_digits(kb.p, k->n, k->stream, hist.p));
      return truncate_top_keys(k, &stage, kb.p, hist.p);
    }
    return truncate_run(k, &stage, nullptr, dt, nullptr);
  };
  auto stage_input = [&](const pauli_sum* k, double a) -> int {  // X = O + a k
    NvtxRange r("stage input");
    MergeSpec sp;
    sp.src[0] = source(O, Cx{1.0, 0.0});
    sp.src[1] = source(k, Cx{a, 0.0});
    sp.nsrc = 2;
    return merge_into(sp, O->stream, &X.s);
  };
  PS_TRY(L(O, &k1.s));
  PS_TRY(stage_input(&k1.s, h2));
  PS_TRY(L(&X.s, &k2.s));
  PS_TRY(stage_input(&k2.s, h2));
  PS_TRY(L(&X.s, &k3.s));
  PS_TRY(stage_input(&k3.s, dt));
  PS_TRY(L(&X.s, &k4.s));
  // S = ((k1 + 2 k2) + 2 k3) + k4;  O' = O + (dt/6) S
  MergeSpec sp;
  sp.src[0] = source(&k1.s, Cx{1.0, 0.0});
  sp.src[1] = source(&k2.s, Cx{2.0, 0.0});
  sp.src[2] = source(&k3.s, Cx{2.0, 0.0});
  sp.src[3] = source(&k4.s, Cx{1.0, 0.0});
  sp.nsrc = 4;
  sp.pre = O->d;
  sp.npre = O->n;
  sp.clsPre = O->cls;
  sp.has_post = true;
  sp.post = Cx{h6, 0.0};
  PS_TRY(merge_into(sp, O->stream, &X.s));
  if (cand) {
    PS_TRY(sum_reserve(cand, X.s.n, false));
    if (X.s.n > 0)
      PS_CUDA(cudaMemcpyAsync(cand->d, X.s.d, (size_t)X.s.n * sizeof(Rec), cudaMemcpyDeviceToDevice, O->stream));
    cand->n = X.s.n;
    cand->cls = X.s.cls;
    if (cand->stream != O->stream) PS_CUDA(cudaStreamSynchronize(O->stream));
  }
  if (model && policy && policy->top_k > 0 && X.s.n > policy->top_k) {
    Buf<double> score;
    PS_TRY(score.alloc((size_t)X.s.n, O->stream));
    const double gdt = policy->gamma != 0.0 ? policy->gamma * dt : 0.0;
    PS_TRY(mlp_scores(model, X.s.d, X.s.n, gdt, O->stream, score.p));
    PS_TRY(truncate_run(&X.s, policy, keep, dt, nullptr, score.p));
  } else {
    PS_TRY(truncate_run(&X.s, policy, keep, dt, nullptr));
  }
  swap_contents(O, &X.s);
  return PS_OK;
}

}  // namespace

extern "C" {

int pauli_rk4_step(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* policy,
                   const pauli_sum* keep) {
  if (!H || !O || H == O || !same_sites(H, O) || !same_sites(O, keep)) return PS_ERR_INVALID;
  if (!policy_valid(policy, O) || !std::isfinite(dt) || H->n > 0xEFFF) return PS_ERR_INVALID;
  if (O->W > 1) return wide_api::rk4_step(H, O, dt, policy, keep);
  return rk4_impl(H, O, dt, policy, keep, nullptr, nullptr);
}

int pauli_rk4_step_mlp(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* policy,
                       const pauli_sum* keep, const pauli_mlp* model, pauli_sum* cand_out) {
  PS_NARROW(O);
  if (!H || !O || H == O || !same_sites(H, O) || !same_sites(O, keep) || !same_sites(O, cand_out)) return PS_ERR_INVALID;
  if (cand_out == O || cand_out == H) return PS_ERR_INVALID;
  if (!policy_valid(policy) || !std::isfinite(dt) || H->n > 0xEFFF) return PS_ERR_INVALID;
  if (model && mlp_n_sites(model) != O->n_sites) return PS_ERR_INVALID;
  if (model && mlp_stream(model) != O->stream) PS_CUDA(cudaStreamSynchronize(mlp_stream(model)));
  return rk4_impl(H, O, dt, policy, keep, model, cand_out);
}

int pauli_lanczos_step(const pauli_sum* H, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev,
                       const pauli_trunc_policy* policy, double* b_out) {
  NvtxRange nvtx("pauli_lanczos_step");
  if (!H || !O_prev || !O_cur || !b_out || O_prev == O_cur || H == O_prev || H == O_cur) return PS_ERR_INVALID;
  if (!same_sites(H, O_cur) || !same_sites(O_prev, O_cur) || !policy_valid(policy, O_cur) || !std::isfinite(b_prev))
    return PS_ERR_INVALID;
  if (H->n > 0xEFFF) return PS_ERR_INVALID;
  *b_out = 0.0;
  if (O_cur->W > 1) return wide_api::lanczos_step(H, O_prev, O_cur, b_prev, policy, b_out);
  Tmp A(O_cur);
  MergeSpec sp;
  sp.H = H->d;
  sp.nH = (int)H->n;
  sp.X = O_cur->d;
  sp.nX = O_cur->n;
  sp.clsH = H->cls;
  sp.clsX = O_cur->cls;
  if (O_prev->n > 0) {
    sp.src[0] = source(O_prev, Cx{-b_prev, 0.0});
    sp.nsrc = 1;
  }
  // A = [H, O_n] - b_{n-1} O_{n-1}; a single-component merge also writes the rank keys |x| of
  // A and the exact norm's exponent bound from its output stage
  Buf<int> ktop;
  PS_TRY(ktop.alloc(1, O_cur->stream));
  PS_CUDA(cudaMemsetAsync(ktop.p, 0x80, sizeof(int), O_cur->stream));  // below every bound
  uint64_t* mkeys = nullptr;
  sp.keys_out = &mkeys;
  sp.keys_top = ktop.p;
  PS_TRY(merge_into(sp, O_cur->stream, &A.s));
  Buf<uint64_t> ab;
  if (mkeys) ab.adopt(mkeys, (size_t)A.s.n, A.s.stream);
  pauli_trunc_policy p{-1, 0.0, 0, 0.0, 0};
  if (policy) {
    p.max_weight = policy->max_weight;
    p.cutoff = policy->cutoff;
    p.top_k = policy->top_k;
  }
  // b_n = ||A||: from the merge's keys (one read of 8 bytes per string, which also gives the
  // division-free truncation its first-digit histogram), else from the records, where the
  // norm's first pass writes the keys when the truncation can use them
  const bool keys = lanczos_keys_eligible(&A.s, &p);
  Buf<unsigned> hist;
  double n2 = 0.0;
  if (keys) PS_TRY(hist.alloc(kKeyBins, A.s.stream));
  if (ab.p) {
    PS_TRY(exact_norm2_keys_top(ab.p, A.s.n, ktop.p, A.s.stream, &n2, keys ? hist.p : nullptr));
  } else if (keys) {
    PS_TRY(ab.alloc((size_t)A.s.n, A.s.stream));
    PS_TRY(exact_norm2_keys(A.s.d, A.s.n, A.s.stream, &n2, A.s.cls, ab.p, hist.p));
  } else {
    PS_TRY(exact_norm2(A.s.d, A.s.n, A.s.stream, &n2));
  }
  double b = std::sqrt(n2);
  *b_out = b;
  if (!std::isfinite(b)) return PS_ERR_NONFINITE;
  if (b == 0.0) return PS_ERR_KRYLOV_EXHAUSTED;
  if (keys)
    PS_TRY(truncate_lanczos_keys(&A.s, &p, b, ab.p, hist.p));
  else
    PS_TRY(truncate_run(&A.s, &p, nullptr, 0.0, &b));
  // rotate: O_prev <- O_cur, O_cur <- O_n
  swap_contents(O_prev, O_cur);
  swap_contents(O_cur, &A.s);
  return PS_OK;
}

int pauli_trace_product(const pauli_sum* A, const pauli_sum* B, double* re, double* im) {
  if (!A || !B || !re || !im || !same_sites(A, B)) return PS_ERR_INVALID;
  if (A->stream != B->stream) PS_CUDA(cudaStreamSynchronize(B->stream));
  if (A->W > 1) return wide_api::trace_product(A, B, re, im);
  return exact_trace_product(A->d, A->n, B->d, B->n, A->stream, re, im);
}

int pauli_coefficients(const pauli_sum* O, const uint64_t* qv, const uint64_t* qw, int64_t nq, double* re,
                       double* im) {
  if (!O || nq < 0 || (nq > 0 && (!qv || !qw || !re || !im))) return PS_ERR_INVALID;
  PS_NARROW(O);
  const uint64_t inv = O->n_sites >= 64 ? 0ull : ~((1ull << O->n_sites) - 1ull);
  for (int64_t j = 0; j < nq; ++j)
    if ((qv[j] | qw[j]) & inv) return PS_ERR_INVALID;
  return coefficients(O->d, O->n, qv, qw, nq, O->stream, re, im);
}

int pauli_norm(const pauli_sum* O, double* out) {
  if (!O || !out) return PS_ERR_INVALID;
  double n2 = 0.0;
  if (O->W > 1) {
    PS_TRY(wide_api::norm2(O, &n2));
    *out = std::sqrt(n2);
    return PS_OK;
  }
  PS_TRY(exact_norm2(O->d, O->n, O->stream, &n2));
  *out = std::sqrt(n2);
  return PS_OK;
}

}  // extern "C"
