/* paulistr.h -- C ABI of the GB300 (sm_103a) Pauli-string commutator library.
 *
 * The library implements the hot path of the binary Pauli-string method
 * (Loizeau, Peacock, Sels, "Quantum many-body simulations with
 * PauliStrings.jl", arXiv:2410.09654): the commutator [H, O] of two Pauli
 * sums with duplicate merging (Alg. 1 adapted with eq. eps_com), truncation
 * (trim / cutoff / long-string discarding / depolarising noise), one RK4 step
 * of the Heisenberg equation dO/dt = i[H, O] and one Lanczos step of the
 * recursion method, plus the trace products and norms they need.
 *
 * Conventions (paper, Methods, eqs. v12, w12, eps12, eps_com):
 *   - A Pauli string on n_sites <= 64 sites is a pair of uint64 masks (v, w).
 *     Bit i-1 is site i; v is the Z bit and w the X bit (tau table).  Bits at or
 *     above n_sites must be zero.
 *   - Wider registers (the paper's masks have any length): for 65 <= n_sites <= 256 each
 *     mask is W = 2 (n_sites <= 128) or W = 4 (n_sites <= 256) uint64 words, and every
 *     array of masks a call reads or writes holds W words per string, row-major (string i
 *     at [i*W, i*W + W)); word k holds sites 64k+1 .. 64k+64.  Canonical order compares v,
 *     then w, as unsigned W-word integers.  Sums of this width support uploads, downloads,
 *     copies, pauli_commutator, pauli_add, pauli_truncate, pauli_rk4_step,
 *     pauli_lanczos_step, pauli_trace_product and pauli_norm (the same results as the
 *     one-word path: same summation order, same truncation rules; H at most 61439 strings);
 *     every other entry point returns PS_ERR_INVALID for them.
 *   - A coefficient multiplies the Hermitian string
 *     P(v,w) = (-i)^{popcount(v & w)} Z^v X^w  (site letters I, X, Y, Z).
 *   - Coefficients are complex FP64, passed as separate real and imaginary arrays.
 *
 * Memory and streams:
 *   - A pauli_sum is device resident and owned by the library (stream-ordered
 *     allocations on the sum's stream).  Host arrays passed in or out are owned
 *     by the caller and are only read or written during the call.
 *   - Every call is ordered on the stream given at creation (a cudaStream_t,
 *     e.g. PyTorch's current stream; NULL is the legacy default stream).  Calls
 *     that return a host value (sizes, norms, b_n, trace products) synchronise
 *     that stream; the others may synchronise it to size their outputs.
 *   - All sums passed to one call must share n_sites and should share the stream.
 *
 * Errors: every entry point returns a status (PS_OK = 0).  On error, output
 * sums are left empty or unchanged and nothing aborts; no device code traps.
 *
 * Non-finite values: uploads reject NaN and +-Inf coefficients (PS_ERR_INVALID).  Arithmetic
 * that overflows follows IEEE rules (a merge may produce +-Inf or NaN coefficients; a NaN
 * coefficient ranks lowest in truncation).  pauli_norm then returns +Inf (NaN if any
 * coefficient is NaN), pauli_trace_product returns NaN in both parts when a matched pair holds
 * a non-finite factor, and the Lanczos steps return PS_ERR_NONFINITE without rotating.
 * pauli_status_string() gives a description.
 *
 * Determinism: for every string, the contributions to its coefficient are added
 * in the same order as in Alg. 1 with H in the outer loop (H's term order as
 * uploaded), with separately rounded FP64 products and sums and no FMA; norms
 * and trace products are the exactly rounded values of the exact sums.  The
 * results are therefore independent of the storage order of the strings and of
 * the GPU scheduling, and equal those of a plain sequential implementation.
 * Storage order inside a sum is unspecified; pauli_sum_download returns the
 * canonical order (v ascending, then w ascending, unsigned).
 */
#ifndef PAULISTR_H
#define PAULISTR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define PS_OK 0
#define PS_ERR_INVALID 1          /* bad argument: null, n_sites out of range, key bits >= n_sites, ... */
#define PS_ERR_CAPACITY 2         /* a caller-provided capacity is too small (download) */
#define PS_ERR_TABLE_FULL 3       /* a merge table could not be resolved even after splitting */
#define PS_ERR_CUDA 4             /* a CUDA runtime call failed; see pauli_last_cuda_error() */
#define PS_ERR_TIMEOUT 5          /* a bounded device-side wait gave up (the learned scorer's wait on its tensor-core products) */
#define PS_ERR_KRYLOV_EXHAUSTED 6 /* Lanczos: b_n == 0 (the Krylov space closed); b_out is 0 */
#define PS_ERR_NOMEM 7            /* device allocation failed */
#define PS_ERR_UNCERTAIN 8        /* reserved */
#define PS_ERR_IO 9               /* a checkpoint file could not be written or read, or is not one */
#define PS_ERR_NONFINITE 10       /* Lanczos: b_n is +Inf or NaN (a coefficient overflowed); b_out holds it */

const char* pauli_status_string(int status);
/* Text of the last CUDA error seen by the library on this thread ("" if none). */
const char* pauli_last_cuda_error(void);

/* ------------------------------------------------------------------ sums */
typedef struct pauli_sum pauli_sum; /* opaque, device resident */

/* Create an empty sum on n_sites (1..256) sites.  capacity is a hint (strings);
 * sums grow as needed.  cuda_stream: cudaStream_t the sum's work is ordered on. */
int pauli_sum_create(int n_sites, int64_t capacity, void* cuda_stream, pauli_sum** out);
int pauli_sum_destroy(pauli_sum* s);

/* Replace the contents of s with n strings from HOST arrays v, w, re, im
 * (caller-owned, read during the call).  Strings must be distinct (a repeated
 * string is PS_ERR_INVALID) and have no bits at or above n_sites.  The given
 * order is kept; for a sum used as the left operand H of a commutator this is
 * the order of the outer loop of Alg. 1.  Exact-zero coefficients are kept.
 * Arrays in pinned host memory mapped into the device's address space are read by the
 * packing kernel directly over the host link; other host arrays go through a staging copy. */
int pauli_sum_upload(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re,
                     const double* im, int64_t n);

/* Same as pauli_sum_upload but v, w, re, im are DEVICE pointers (n elements each) on the
 * current device, or pinned host memory mapped into its address space; any other pointer
 * (pageable host memory, another device's memory) is PS_ERR_INVALID.  Only the bit-range
 * check is done (on the device); distinctness is the caller's responsibility. */
int pauli_sum_upload_device(pauli_sum* s, const uint64_t* v, const uint64_t* w, const double* re,
                            const double* im, int64_t n);

/* Number of strings (synchronises the stream). */
int pauli_sum_size(const pauli_sum* s, int64_t* n);
int pauli_sum_n_sites(const pauli_sum* s, int* n_sites);

/* Coefficient precision of a sum (FP64 by default).  In an FP32 sum every stored
 * coefficient is an FP32 number: uploads, copies and every result a call writes into the
 * sum are rounded to FP32 (round to nearest even) and strings that round to zero are
 * dropped.  A merge forms each output from the exact products of its inputs (products of
 * FP32 numbers are exact in FP64), accumulated in FP64 in the FP64 path's order - no less
 * accurate than a compensated FP32 sum - and rounds once; truncation rounds after the
 * division and the dissipation factor, before its decisions.  Norms, trace products and
 * b_n stay FP64 (exact sums of the FP32 values).  Temporaries of RK4 and Lanczos steps take
 * the precision of the operator being evolved; H's coefficients are used as stored (set H
 * to FP32 too for an all-FP32 computation).  Setting PS_COEF_F32 rounds the current
 * contents.  The records keep the 32-byte layout. */
#define PS_COEF_F64 0
#define PS_COEF_F32 1
/* FP32 arithmetic with compensated sums: like PS_COEF_F32 for storage, truncation, norms and
 * b_n, but a merge computes every term in FP32 (product terms 2 i^(k+rot) RN32(h x), source
 * terms RN32(alpha y), with h, x, alpha rounded to FP32 first) and adds a string's terms in
 * Alg. 1's order with the compensated sum Sum2 of Ogita, Rump and Oishi (Knuth's TwoSum on the
 * running sum, the errors summed in FP32, one final rounding); with a post factor the output is
 * RN32(pre + RN32(post acc)).  The sums must be single-component (real or imaginary
 * coefficients throughout) and H at most 508 terms (ranked merges); other merges return
 * PS_ERR_INVALID.  A merge writing into such a sum uses this arithmetic. */
#define PS_COEF_F32C 2
int pauli_sum_set_precision(pauli_sum* s, int coef_dtype);
int pauli_sum_precision(const pauli_sum* s, int* coef_dtype);

/* Copy the sum to HOST arrays of capacity cap in canonical order (v, then w,
 * ascending).  *n receives the size; PS_ERR_CAPACITY (nothing written) if cap < size. */
int pauli_sum_download(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im,
                       int64_t cap, int64_t* n);

/* Copy the sum to DEVICE arrays in storage order (unspecified order), ordered on the sum's
 * stream (not synchronised).  The arrays may also be pinned host memory mapped into the
 * device's address space: the unpacking kernel then writes them over the host link, and they
 * are complete once the stream has run it.  Any other pointer (pageable host memory, another
 * device's memory) is PS_ERR_INVALID. */
int pauli_sum_download_device(const pauli_sum* s, uint64_t* v, uint64_t* w, double* re, double* im,
                              int64_t cap, int64_t* n);

int pauli_sum_copy(const pauli_sum* src, pauli_sum* dst);

/* Reorder the storage of s (contents unchanged) so that strings in the same bucket of the
 * merge's output hash are adjacent: the order in which merges already return their results.
 * An operand in that order lets the emission of [H, s] reserve output slots for a warp's
 * neighbouring strings in few bins; an operand uploaded in canonical (sorted) order runs
 * about a quarter slower at the Lanczos benchmark size.  Results never depend on storage
 * order, but the order of a sum used as H (the left operand) is Alg. 1's outer-loop order:
 * do not reorder such a sum.  Asynchronous on s's stream. */
int pauli_sum_sort_by_hash(pauli_sum* s);

/* Checkpoint / resume of long runs.  pauli_sum_save writes the sum to a file: an 8-byte
 * magic "PSUMCKP1", u32 version (1), u32 n_sites, u32 precision (PS_COEF_*), u32 n_meta,
 * u64 string count, n_meta f64 caller values (for example t, the step, the b_n so far),
 * the records {u64 v, u64 w, f64 re, f64 im} in canonical order (v, then w), and a u64
 * FNV-1a checksum of everything before it; all little-endian.  pauli_sum_load replaces the
 * contents of s (which must have the file's n_sites) and its precision, and copies up to
 * meta_cap caller values into meta (*n_meta receives the stored count).  Errors: PS_ERR_IO
 * (cannot open or write, short or corrupt file, wrong magic, version or checksum),
 * PS_ERR_INVALID (bad arguments, n_sites mismatch).  Both synchronise the sum's stream. */
int pauli_sum_save(const pauli_sum* s, const char* path, const double* meta, int64_t n_meta);
int pauli_sum_load(pauli_sum* s, const char* path, double* meta, int64_t meta_cap, int64_t* n_meta);

/* ------------------------------------------------------------------ algebra */

/* out = [H, O] = H O - O H  (Alg. 1 with eq. eps_com): all-pairs string
 * products (XOR of the masks, eqs. v12/w12), anticommutation test and popcount
 * phase, coefficient 2 i^k h o for anticommuting pairs, duplicates merged,
 * exact zeros dropped.  out must be distinct from H and O. */
int pauli_commutator(const pauli_sum* H, const pauli_sum* O, pauli_sum* out);

/* out = A B, the operator product (Alg. 1 proper): every pair of strings a in A,
 * b in B contributes i^k a b to the string with masks (va ^ vb, wa ^ wb), k the
 * popcount phase of eq. eps12 in the Hermitian basis; duplicates are merged with the
 * contributions to each output string added in A's order, exact zeros dropped.
 * A is the outer operand and may hold at most 61439 strings (PS_ERR_INVALID beyond);
 * B any number.  The identity coefficient of A B is Tr(AB)/2^N (pauli_trace_product
 * gives it exactly rounded without forming the product).  out must be distinct from A
 * and B; all three must have the same number of sites. */
int pauli_multiply(const pauli_sum* A, const pauli_sum* B, pauli_sum* out);

/* out = A + alpha * B over the union of supports (absent strings are zero),
 * exact zeros dropped.  out must be distinct from A and B. */
int pauli_add(const pauli_sum* A, double alpha_re, double alpha_im, const pauli_sum* B, pauli_sum* out);

/* Truncation policy (paper: trim(O, M; keep), cutoff(O, eps), discarding long
 * strings, add_noise(O, eps*dt)). */
typedef struct {
  int max_weight;   /* drop strings of Pauli weight > max_weight; < 0: off */
  double cutoff;    /* drop |c| < cutoff, tested as re*re + im*im < cutoff*cutoff; <= 0: off */
  int64_t top_k;    /* keep the top_k strings by |c|^2, exact ties to the smaller (v, w); <= 0: off */
  double gamma;     /* depolarising transmission exp(-(gamma*dt) * weight); 0: off */
  int trim_stages;  /* RK4 only: also cut each stage derivative k_j to its top_k */
} pauli_trunc_policy;

/* In place: (1) c *= exp(-(gamma*dt)*wt), wt = popcount(v|w); (2) drop wt > max_weight;
 * (3) drop |c|^2 < cutoff^2; (4) keep the top_k by |c|^2 (ties: smaller key), never
 * dropping a string that is present in keep (keep may be NULL; only its strings
 * matter).  Exact zeros are dropped. */
int pauli_truncate(pauli_sum* O, const pauli_trunc_policy* policy, const pauli_sum* keep, double dt);

/* One classical RK4 step of dO/dt = i[H, O] (paper, Heisenberg time evolution):
 *   k1 = i[H,O]; k2 = i[H, O + dt/2 k1]; k3 = i[H, O + dt/2 k2]; k4 = i[H, O + dt k3];
 *   S = k1 + 2 k2; S = S + 2 k3; S = S + k4;  O <- O + (dt/6) S;
 * then pauli_truncate(O, policy, keep, dt).  policy may be NULL (no truncation). */
int pauli_rk4_step(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* policy,
                   const pauli_sum* keep);

/* One step of the Lanczos recursion (paper, Krylov subspace expansion):
 *   A = [H, O_cur] - b_prev O_prev;  b_n = ||A|| = sqrt(sum |c|^2);  O_n = trunc(A / b_n)
 * and the sums rotate: O_prev <- O_cur, O_cur <- O_n.  For the first step pass an
 * empty O_prev (and b_prev = 0): then b_1 = ||[H, O_0]||.  *b_out receives b_n.
 * If b_n == 0 the sums are left unchanged and PS_ERR_KRYLOV_EXHAUSTED is returned.
 * policy may be NULL (no truncation); its gamma and trim_stages are ignored. */
int pauli_lanczos_step(const pauli_sum* H, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev,
                       const pauli_trunc_policy* policy, double* b_out);

/* Tr(A B) / 2^N = sum over strings present in both of a_s b_s (eq. correlator with
 * the Hermitian, trace-orthonormal strings); each component exactly rounded. */
int pauli_trace_product(const pauli_sum* A, const pauli_sum* B, double* re, double* im);

/* ||O|| = sqrt(sum |c|^2) = sqrt(Tr(O^dag O) / 2^N) (the norm of the Krylov section,
 * read with the square root), from the exactly rounded sum of squares. */
int pauli_norm(const pauli_sum* O, double* out);

/* ------------------------------------------------------- translation symmetry
 * A translation-symmetric operator on a periodic chain of n = n_sites sites (2..64),
 * O = sum_{i<n} T_i(O_0) with T_i the translation by i sites (site j -> j + i mod n),
 * is stored as its generator O_0: one representative string per translation orbit, the
 * orbit's smallest translate in (v, then w) unsigned order (the Methods' translation-
 * symmetric encoding and Alg. 2, whose Shiftleft picks a representative per orbit).
 * These calls need single-component coefficients (all real or all imaginary; the
 * Lanczos recursion of a real H keeps them so) and return PS_ERR_INVALID otherwise. */

/* out = sum_{k<n} T_k(G) as a plain sum (G any strings). */
int pauli_ts_expand(const pauli_sum* G, pauli_sum* out);

/* out = X with every string moved to its orbit representative; the contributions to one
 * representative are added in increasing shift (the smallest k with T_k(x) = rep). */
int pauli_ts_canonicalize(const pauli_sum* X, pauli_sum* out);

/* out = generator of [H, O] for generators H0, O0: [sum_k T_k(H0), O0] moved to
 * representatives (H is translation invariant, so [H, O] = sum_j T_j([H, O0])).  H0
 * expanded may hold at most 61439 strings. */
int pauli_ts_commutator(const pauli_sum* H0, const pauli_sum* O0, pauli_sum* out);

/* *out = ||O|| / sqrt(n) for O = sum_i T_i(O0): sqrt(sum_r (n/d_r) |c_r|^2), d_r the period
 * of representative r; the sum exact, rounded once. */
int pauli_ts_norm(const pauli_sum* O0, double* out);

/* One Lanczos step on generators, as pauli_lanczos_step with the calls above:
 * A_0 = TS commutator(H0, O_cur) - b_prev O_prev, b = pauli_ts_norm(A_0),
 * O_cur <- trunc(A_0 / b) (policy as in pauli_lanczos_step), O_prev <- old O_cur.
 * b_n equal those of the expanded periodic chain (the norm's constant factor cancels). */
int pauli_ts_lanczos_step(const pauli_sum* H0, pauli_sum* O_prev, pauli_sum* O_cur, double b_prev,
                          const pauli_trunc_policy* policy, double* b_out);

/* Coefficients of given strings in O, for two-point correlators such as
 * Tr(O(t) Z_j)/2^N over all sites j (section "Heisenberg time evolution"; the
 * Hermitian strings are trace-orthonormal, so Tr(O P_q)/2^N is O's coefficient of q).
 *   qv, qw: HOST arrays of nq query strings (caller-owned; duplicates allowed; bits at
 *     or above n_sites give PS_ERR_INVALID);
 *   re, im: HOST arrays of nq doubles receiving each coefficient (0 for strings absent
 *     from O).  O is read once on the device; the call synchronises O's stream. */
int pauli_coefficients(const pauli_sum* O, const uint64_t* qv, const uint64_t* qw, int64_t nq, double* re,
                       double* im);

/* Allocation-free variant of pauli_trace_product, for callers that cannot allocate
 * device memory (code running under another framework's allocator or memory budget,
 * plug-ins handed only pre-allocated buffers, code that must not call cudaMalloc while
 * a CUDA graph is being captured elsewhere in the process).  The paper has no
 * counterpart; it computes the same exactly rounded Tr(AB)/2^N.
 *   av, aw, are, aim: DEVICE arrays of A's na strings (masks and coefficients);
 *   bv, bw, bre, bim: DEVICE arrays of B's nb strings; both caller-owned, read only;
 *     strings within each operand must be distinct;
 *   cuda_stream: the cudaStream_t the work is ordered on (NULL: legacy default stream);
 *     it must belong to the current device (the scratch is looked up per device);
 *     a stream of another device gives PS_ERR_INVALID;
 *   re, im: HOST doubles receiving the result; the call synchronises the stream.
 * Scratch lives in one fixed device array of about 6 MiB inside the library (held by
 * every GPU that loads it, until exit): no cudaMalloc, cudaFree or allocating library
 * routine is called.  The smaller of na, nb may be at most 131072 strings; larger
 * inputs return PS_ERR_CAPACITY without launching anything.  The first call on a device
 * looks up the scratch address on that device (make that first call before any stream
 * capture).  Every call reuses the same scratch, so calls that overlap on the GPU (on
 * different streams, or from different host threads) race: serialise them. */
int pauli_trace_product_noalloc(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim,
                                int64_t na, const uint64_t* bv, const uint64_t* bw, const double* bre,
                                const double* bim, int64_t nb, void* cuda_stream, double* re, double* im);

/* ------------------------------------------------------------------ statistics */
/* Counters of the last pauli_commutator / merge on this sum's stream: pair tests
 * (|H|*|O|), anticommuting contributions, merged output strings. */
typedef struct {
  int64_t pair_tests;
  int64_t contributions;
  int64_t merged;
  int64_t groups;
  int64_t split_groups;
} pauli_merge_stats;
int pauli_last_merge_stats(pauli_merge_stats* out);

/* ------------------------------------------------------------------ learned truncation
 * The paper's conclusion proposes predicting the importance of strings with machine
 * learning instead of ranking them by |c| alone.  This library's scorer is a small
 * network on string features, trained and run with BF16 tensor-core kernels (FP32
 * accumulation, FP32 master weights, Adam):
 *   features x (80): x0 = wt/N (wt = popcount(v|w)); x1 = extent/N (last - first + 1 over
 *     the non-identity sites; 0 for the identity); x2 = ln(max(|c|, 1e-300))/16; for each
 *     of 16 site bins (site j, 0-based, in bin floor(16 j / N)) the fractions of the bin's
 *     sites holding I, X, Y, Z at x[3 + 4b + 0..3] (zeros for an empty bin); x[67..79] = 0;
 *   z = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 (W1 128x80, W2 128x128, rows = outputs);
 *   truncation score = ln|c| - gamma dt wt + z (ln|c| after the dissipation factor), ranked
 *     through the equivalent rank value |c|^2 e^(2 (z - gamma dt wt)) = e^(2 score), which is
 *     |c|^2 bit for bit when z - gamma dt wt = 0: a network that outputs 0 ranks exactly as
 *     |c| does (without dissipation).
 * Flat FP32 parameter layout (pauli_mlp_param_count() = 27009 floats): W1 (row-major),
 * b1 (128), W2 (row-major), b2 (128), w3 (128), b3 (1).
 * All calls are ordered on the model's stream; sums on another stream are synchronised
 * first.  Record order ("storage order") is that of pauli_sum_download_device. */
typedef struct pauli_mlp pauli_mlp; /* opaque: device-resident parameters and Adam state */

int64_t pauli_mlp_param_count(void);
/* New model on n_sites sites (features depend on N): weights drawn from N(0, 2/fan_in)
 * (w3: N(0, 1/128)) with a splitmix64 stream seeded by seed, biases 0, Adam state 0. */
int pauli_mlp_create(int n_sites, uint64_t seed, void* cuda_stream, pauli_mlp** out);
int pauli_mlp_destroy(pauli_mlp* m);
/* FP32 parameters to / from HOST arrays of exactly pauli_mlp_param_count() floats
 * (PS_ERR_INVALID otherwise); set_params also clears the Adam state. */
int pauli_mlp_get_params(const pauli_mlp* m, float* params, int64_t n);
int pauli_mlp_set_params(pauli_mlp* m, const float* params, int64_t n);
/* Per string of O in storage order, into DEVICE arrays (caller-owned):
 *   features: x[80 * i + k] as BF16 bit patterns (round to nearest even);
 *   logits:   z[i] (FP32);
 *   scores:   rank[i] = |c_i|^2 e^(2 (z_i - gamma_dt wt_i)) (FP64; 0 for c = 0), the values
 *             the learned truncation ranks by (pass them to pauli_truncate_scored).
 * O must have the model's n_sites.  Each call synchronises the model's stream. */
int pauli_mlp_features(const pauli_mlp* m, const pauli_sum* O, uint16_t* x);
int pauli_mlp_logits(const pauli_mlp* m, const pauli_sum* O, float* z);
int pauli_mlp_scores(const pauli_mlp* m, const pauli_sum* O, double gamma_dt, double* score);
/* Gradient (HOST array of pauli_mlp_param_count() floats) and *loss (may be NULL) of the
 * mean binary cross-entropy of z over records [i0, i0 + nb) of X against DEVICE labels
 * (labels[i] in [0, 1], indexed like X's storage order).  The parameters are unchanged. */
int pauli_mlp_gradient(pauli_mlp* m, const pauli_sum* X, const float* labels, int64_t i0, int64_t nb, float* grad,
                       double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on that batch's
 * gradient, nb >= 1.  *loss (if loss is not NULL; this synchronises) receives the batch
 * loss before the update. */
int pauli_mlp_train_step(pauli_mlp* m, const pauli_sum* X, const float* labels, int64_t i0, int64_t nb, float lr,
                         double* loss);
/* labels[i] = 1 if the i-th string of X (storage order) is present in target, else 0
 * (DEVICE array of X's size).  The training label of a candidate string is whether a
 * run at a larger cap keeps it. */
int pauli_mlp_labels(const pauli_sum* X, const pauli_sum* target, float* labels);

/* pauli_truncate with the top-k ranked by score[i] (DEVICE array, one FP64 value per
 * string of O in storage order, read during the call) instead of |c|^2: higher scores
 * are kept first, exact ties keep the smaller key (v, then w), a NaN score ranks below
 * every number, -0 equals +0.  Dissipation, the weight filter, exact-zero removal, the
 * cutoff (on |c|) and the keep set are as in pauli_truncate. */
int pauli_truncate_scored(pauli_sum* O, const pauli_trunc_policy* policy, const pauli_sum* keep, double dt,
                          const double* score);

/* pauli_rk4_step whose final truncation ranks the top_k by the learned score of model
 * (model NULL: by |c|, as pauli_rk4_step).  Stage trims (trim_stages) stay by |c|.
 * cand_out (may be NULL; distinct from H and O) receives the step's result before that
 * final truncation: the candidates the truncation chose from. */
int pauli_rk4_step_mlp(const pauli_sum* H, pauli_sum* O, double dt, const pauli_trunc_policy* policy,
                       const pauli_sum* keep, const pauli_mlp* model, pauli_sum* cand_out);

/* ------------------------------------------------------------------ autotuner
 * The merge's geometry has two free sizes: the target number of entries per output hash
 * bin (which sets the number of bins, 2^4..2^20) and the group quota (entries a merge block
 * takes per group).  Results do not depend on them (the merge is exact in any geometry);
 * the time does.  pauli_autotune_commutator times [H, O] (CUDA events, best of reps after
 * one warm-up run) with bin targets 1024, 2048, 4096 and quotas 1024, 1536, and keeps the
 * fastest for every later merge of the same size class (log2 of the merge's entry bound) in
 * this process.  Outputs (may be NULL): the chosen pair, its time and the default's
 * (2048, 1536) time in ms.  pauli_autotune_reset returns every class to the defaults. */
int pauli_autotune_commutator(const pauli_sum* H, const pauli_sum* O, int reps, int* best_bin_target,
                              int* best_quota, double* best_ms, double* default_ms);
int pauli_autotune_reset(void);
/* Use one geometry for every merge until pauli_autotune_reset (bin target 64..65536 entries,
 * quota 64..4096); for tests that run the merge in each geometry. */
int pauli_merge_geometry_fix(int bin_target, int quota);

/* ------------------------------------------------------------------ batched instances
 * Many independent problems with the same H strings but their own H coefficients (for
 * example disorder realisations of a chain, H_b = common terms + sum_i h_i^(b) Z_i) and
 * their own truncation caps, evolved together in one sum.  A string of instance b carries
 * b in its v bits from tag_shift up (Z letters on sites above the physical ones):
 * key = (v | b << tag_shift, w).  These bits are transparent to the method (H's strings
 * have none, so every product keeps the tag of its O string) and no result mixes
 * instances.  Results equal those of each instance run alone. */
typedef struct pauli_batch pauli_batch; /* opaque */

/* H: the common strings (1..256 of them, real coefficients; the values are not used),
 * no bits at or above tag_shift.  hcoef: HOST array [n_inst][H size] (row b = the
 * coefficients of instance b's H, in H's string order; read during the call).  caps:
 * HOST array [n_inst] of per-instance top-k sizes (<= 0 or caps NULL: no cap).
 * 1 <= n_inst <= 4096; the tags must fit below H's n_sites (tag_shift + bits(n_inst - 1)
 * <= n_sites). */
int pauli_batch_create(const pauli_sum* H, const double* hcoef, int n_inst, int tag_shift, const int64_t* caps,
                       pauli_batch** out);
int pauli_batch_destroy(pauli_batch* b);
/* One RK4 step (as pauli_rk4_step) of every instance of O: the products use each string's
 * instance coefficients; with trim_stages each k_j is cut to its instance's cap; the new O
 * is cut to the caps (top-k by |c|^2, ties to the smaller key, per instance).  O must hold
 * real coefficients and only valid tags (PS_ERR_INVALID otherwise); O's precision applies. */
int pauli_batch_rk4_step(const pauli_batch* b, const pauli_sum* H, pauli_sum* O, double dt, int trim_stages);
/* n_steps (>= 0) such steps in a row, the same as n_steps calls of pauli_batch_rk4_step.  On
 * an error the steps already taken stay applied and *steps_done (nullable) says how many. */
int pauli_batch_rk4_steps(const pauli_batch* b, const pauli_sum* H, pauli_sum* O, double dt, int trim_stages,
                          int n_steps, int* steps_done);
/* Per-instance top-k of O to the caps. */
int pauli_batch_truncate(const pauli_batch* b, pauli_sum* O);
/* Strings per instance (HOST [n_inst]); PS_ERR_INVALID if a string has a tag >= n_inst or
 * w bits at or above tag_shift. */
int pauli_batch_counts(const pauli_batch* b, const pauli_sum* O, int64_t* counts);
/* ||O_b|| = sqrt(sum |c|^2) per instance (HOST [n_inst]); FP64 sums whose addition order is
 * not fixed (the last bits may differ between runs). */
int pauli_batch_norms(const pauli_batch* b, const pauli_sum* O, double* norms);

/* ------------------------------------------------------------------ profiling */
/* Enable (1) or disable (0) per-kernel timing: every kernel launch of the library is
 * bracketed by CUDA events recorded on its launching stream.  Enabling clears the totals. */
int pauli_profile_enable(int on);
/* Write the totals as JSON {"kernel": [launches, total_ms], ...} into buf (len bytes,
 * NUL-terminated); waits for the recorded events.  *needed receives the size required;
 * PS_ERR_CAPACITY if len is too small. */
int pauli_profile_report(char* buf, int64_t len, int64_t* needed);
/* Number of kernels the library has launched since it was loaded. */
int64_t pauli_launch_count(void);

/* ------------------------------------------------------------------ testing hooks */
/* Make the next n-th device allocation of the library fail (n >= 1; 0 disables).
 * Host-side fault injection for tests; it never touches the GPU. */
int pauli_debug_fail_alloc_after(int64_t n);
/* The merge's 32-bit output hash F(v, w) (a GF(2)-linear map of the 128 key bits; a
 * merge bins strings by its low bits and splits crowded bins by the next ones) of n HOST
 * strings into the HOST array out.  Host-only; for tests that build colliding inputs. */
int pauli_debug_output_hash(const uint64_t* v, const uint64_t* w, int64_t n, uint32_t* out);
/* Divide n DEVICE doubles in place by b with the division used by the Lanczos
 * normalisation (correctly rounded, equal to the IEEE quotient); synchronises the stream.
 * For tests of that arithmetic. */
int pauli_debug_divide(double* x, int64_t n, double b, void* cuda_stream);
/* The learned scorer's bounded wait on its tensor-core products: with no_products != 0 the
 * scorer issues no products (so its wait can only run out), and every wait gives up after
 * wait_limit polls (default 2^26).  For tests of the PS_ERR_TIMEOUT path; it never leaves work
 * in flight. */
int pauli_debug_mlp_wait(int no_products, int64_t wait_limit);
/* on != 0: every truncation takes the general path (division of every candidate before the
 * ranking).  By default the Lanczos truncation of a single-component FP64 sum by top-k alone
 * ranks the undivided values (the rank value |RN(x/b)|^2 is non-decreasing in |x|: the k-th
 * value and its ties are found exactly) and divides only the kept strings; both paths give
 * the same strings and coefficients.  For tests comparing the two. */
int pauli_debug_general_truncation(int on);

#ifdef __cplusplus
}
#endif
#endif /* PAULISTR_H */
