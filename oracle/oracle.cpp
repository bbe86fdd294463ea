// CPU oracle for the binary Pauli-string commutator path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library or its
// Python binding) may link, load or call this file; only the tests, the
// package's smoke entry and the benchmark's CPU-baseline leg do.  It shares no
// code, header, table or helper with the CUDA path.
//
// It is deliberately plain and slow: a hash map keyed by the (v,w) pair, FP64
// coefficients, loops in the order the paper states them.  Built with
// -ffp-contract=off so that every product and sum is a separately rounded IEEE
// operation.
//
// Conventions (paper, "Methods / Pauli strings", eqs. v12, w12, eps12, eps_com):
//   * a string is a pair of bit masks (v, w); bit i-1 of each mask is site i;
//     v is the Z bit and w the X bit of the tau table (tau_00 = 1, tau_01 = X,
//     tau_10 = Z, tau_11 = ZX = iY);
//   * coefficients multiply the HERMITIAN string P(v,w) = (-i)^{pop(v&w)} Z^v X^w
//     (so site (1,1) is Y, not iY); the product and commutator phases below are
//     the paper's eqs. eps12 / eps_com rewritten for this basis;
//   * the product string of a and b has masks (va ^ vb, wa ^ wb)  (eqs. v12, w12).
//
// Parity status of each entry point is stated beside it.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

struct Key {
  uint64_t v, w;
  bool operator==(const Key& o) const { return v == o.v && w == o.w; }
  bool operator<(const Key& o) const { return v < o.v || (v == o.v && w < o.w); }
};

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = k.v * 0x9E3779B97F4A7C15ull;
    h ^= (k.w + 0x632BE59BD9B4E019ull) + (h << 6) + (h >> 2);
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    return (size_t)(h ^ (h >> 32));
  }
};

struct Cx {
  double re, im;
};

using Dict = std::unordered_map<Key, Cx, KeyHash>;

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

// Complex product written out: four rounded products, two rounded sums.
inline Cx cmul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Multiply by i^k (exact: a swap and sign changes).
inline Cx rot(Cx a, int k) {
  switch (k & 3) {
    case 0: return a;
    case 1: return {-a.im, a.re};
    case 2: return {-a.re, -a.im};
    default: return {a.im, -a.re};
  }
}

// Phase of a string product in the Hermitian basis:
//   P_a P_b = i^k P_{a^b},
//   k = pop(vc&wc) - pop(va&wa) - pop(vb&wb) + 2 pop(wa&vb)   (mod 4).
// Derivation: P = (-i)^{pop(v&w)} Z^v X^w and X^{wa} Z^{vb} = (-1)^{pop(wa&vb)} Z^{vb} X^{wa},
// which is the paper's eq. eps12 with the sign moved to the (Z-first) ordering used here.
inline int product_phase(uint64_t va, uint64_t wa, uint64_t vb, uint64_t wb) {
  uint64_t vc = va ^ vb, wc = wa ^ wb;
  int k = popc(vc & wc) - popc(va & wa) - popc(vb & wb) + 2 * popc(wa & vb);
  return ((k % 4) + 4) % 4;
}

// Two Hermitian strings commute iff pop(wa&vb) + pop(va&wb) is even (eq. eps_com:
// alpha = (-1)^{pop(v1&w2)} - (-1)^{pop(w1&v2)} vanishes exactly then).  When they
// anticommute, [P_a, P_b] = 2 P_a P_b = 2 i^k P_{a^b}.
inline bool anticommute(uint64_t va, uint64_t wa, uint64_t vb, uint64_t wb) {
  return ((popc(wa & vb) + popc(va & wb)) & 1) != 0;
}

struct Term {
  Key k;
  Cx c;
};

// Canonical key order (v, then w, both unsigned ascending), exact zeros dropped.
std::vector<Term> canonical(const Dict& d) {
  std::vector<Term> out;
  out.reserve(d.size());
  for (const auto& kv : d)
    if (kv.second.re != 0.0 || kv.second.im != 0.0) out.push_back({kv.first, kv.second});
  std::sort(out.begin(), out.end(), [](const Term& a, const Term& b) { return a.k < b.k; });
  return out;
}

std::vector<Term> from_arrays(const uint64_t* v, const uint64_t* w, const double* re,
                              const double* im, int64_t n) {
  std::vector<Term> t((size_t)n);
  for (int64_t i = 0; i < n; ++i) t[(size_t)i] = {{v[i], w[i]}, {re[i], im[i]}};
  return t;
}

// Alg. 1 proper, the operator product: C = A B = sum_{a in A} sum_{b in B} A_a B_b P_a P_b
// with P_a P_b = i^k P_{a^b} (eqs. v12, w12, eps12 in the Hermitian basis).  Same visiting
// order as the commutator below: A outer, B inner, contributions added in that order.
std::vector<Term> product(const std::vector<Term>& A, const std::vector<Term>& B) {
  Dict C;
  C.reserve(A.size() * B.size() + 16);
  for (const Term& a : A) {
    for (const Term& b : B) {
      int k = product_phase(a.k.v, a.k.w, b.k.v, b.k.w);
      Cx t = rot(cmul(a.c, b.c), k);
      Key c{a.k.v ^ b.k.v, a.k.w ^ b.k.w};
      auto it = C.find(c);
      if (it == C.end()) {
        C.emplace(c, t);
      } else {
        it->second.re += t.re;
        it->second.im += t.im;
      }
    }
  }
  return canonical(C);
}

// Alg. 1 adapted with eq. eps_com: C = [A, B] = sum_{a in A} sum_{b in B} A_a B_b [P_a, P_b].
// A's terms are visited in the order given (outer loop), B's in the order given (inner
// loop); every contribution is added to the dictionary entry in that visiting order.
// Because a fixed string a maps distinct b to distinct products, the contributions to
// one output string arrive in A's order.
std::vector<Term> commutator(const std::vector<Term>& A, const std::vector<Term>& B) {
  Dict C;
  C.reserve(A.size() * B.size() / 2 + 16);
  for (const Term& a : A) {
    for (const Term& b : B) {
      if (!anticommute(a.k.v, a.k.w, b.k.v, b.k.w)) continue;  // alpha = 0
      int k = product_phase(a.k.v, a.k.w, b.k.v, b.k.w);
      Cx p = cmul(a.c, b.c);
      Cx t = rot({2.0 * p.re, 2.0 * p.im}, k);
      Key c{a.k.v ^ b.k.v, a.k.w ^ b.k.w};
      auto it = C.find(c);
      if (it == C.end()) {
        C.emplace(c, t);
      } else {
        it->second.re += t.re;
        it->second.im += t.im;
      }
    }
  }
  return canonical(C);
}

// R = A + alpha * B over the union of the supports (absent entries are zero):
// for a string in both, A_s + (alpha * B_s); only in A, A_s; only in B, alpha * B_s.
std::vector<Term> axpy(const std::vector<Term>& A, Cx alpha, const std::vector<Term>& B) {
  Dict R;
  R.reserve(A.size() + B.size() + 16);
  for (const Term& a : A) {
    auto it = R.find(a.k);
    if (it == R.end()) R.emplace(a.k, a.c);
    else { it->second.re += a.c.re; it->second.im += a.c.im; }
  }
  for (const Term& b : B) {
    Cx t = cmul(alpha, b.c);
    auto it = R.find(b.k);
    if (it == R.end()) R.emplace(b.k, t);
    else { it->second.re += t.re; it->second.im += t.im; }
  }
  return canonical(R);
}

// Real scaling written per component: (re * s, im * s).
std::vector<Term> scale(const std::vector<Term>& A, double s) {
  Dict R;
  for (const Term& a : A) R[a.k] = {a.c.re * s, a.c.im * s};
  return canonical(R);
}

// Division by a real: (re / b, im / b)  (the "/b" of the Lanczos listing).
std::vector<Term> divide(const std::vector<Term>& A, double b) {
  Dict R;
  for (const Term& a : A) R[a.k] = {a.c.re / b, a.c.im / b};
  return canonical(R);
}

// ---------------------------------------------------------------------------
// Exact accumulation of sums of products of doubles (plain big-integer fixed point).
// Each product x*y is exact as an integer mantissa product times a power of two; the
// accumulator holds the exact sum and converts it once, rounding to nearest even.
// ---------------------------------------------------------------------------
struct ExactSum {
  // digit i has weight 2^(32*i - BIAS); products of doubles lie in [2^-2252, 2^2048).
  static constexpr int BIAS = 2304;        // multiple of 32, below the smallest product bit
  static constexpr int NDIG = 144;         // 144*32 = 4608 bits: up to 2^2304, with headroom
  std::vector<int64_t> d = std::vector<int64_t>(NDIG, 0);

  static void split(double x, int64_t& m, int& e) {  // x = m * 2^e exactly, |m| < 2^53
    int ex;
    double f = std::frexp(x, &ex);
    m = (int64_t)std::ldexp(f, 53);
    e = ex - 53;
  }

  void add_product(double x, double y) {
    if (x == 0.0 || y == 0.0) return;
    int64_t mx, my;
    int ex, ey;
    split(x, mx, ex);
    split(y, my, ey);
    bool neg = (mx < 0) != (my < 0);
    unsigned __int128 mag = (unsigned __int128)(uint64_t)(mx < 0 ? -mx : mx) *
                            (unsigned __int128)(uint64_t)(my < 0 ? -my : my);
    int pos = ex + ey + BIAS;  // absolute bit index of the product's bit 0
    int base = pos / 32, sh = pos % 32;
    // spread mag << sh over 32-bit digits starting at `base`
    unsigned __int128 lo = mag << sh;                      // low 128 bits
    uint64_t hi = sh ? (uint64_t)(mag >> (128 - sh)) : 0;  // bits above 128
    uint32_t dig[5] = {(uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)(lo >> 64),
                       (uint32_t)(lo >> 96), (uint32_t)hi};
    for (int i = 0; i < 5; ++i) d[base + i] += neg ? -(int64_t)dig[i] : (int64_t)dig[i];
  }

  // Round the exact value to the nearest double (ties to even).
  double value() const {
    std::vector<int64_t> t = d;
    for (int i = 0; i + 1 < NDIG; ++i) {  // carry-propagate to base-2^32 digits
      int64_t c = t[i] >> 32;             // arithmetic shift: floor division
      t[i] -= c * ((int64_t)1 << 32);
      t[i + 1] += c;
    }
    bool neg = t[NDIG - 1] < 0;
    if (neg) {  // negate the two's-complement digit string
      for (int i = 0; i < NDIG; ++i) t[i] = -t[i];
      for (int i = 0; i + 1 < NDIG; ++i) {
        int64_t c = t[i] >> 32;
        t[i] -= c * ((int64_t)1 << 32);
        t[i + 1] += c;
      }
    }
    int top = -1;
    for (int i = NDIG - 1; i >= 0 && top < 0; --i)
      if (t[i]) top = i * 32 + 63 - __builtin_clzll((uint64_t)t[i]);
    if (top < 0) return 0.0;
    auto bit = [&](int i) -> int { return i < 0 ? 0 : (int)((t[i / 32] >> (i % 32)) & 1); };
    int lsb = std::max(top - 52, -1074 + BIAS);
    uint64_t M = 0;
    for (int i = top; i >= lsb; --i) M = (M << 1) | (uint64_t)bit(i);
    int rnd = bit(lsb - 1);
    bool sticky = false;
    for (int i = lsb - 2; i >= 0 && !sticky; --i) sticky = bit(i) != 0;
    if (rnd && (sticky || (M & 1))) M += 1;
    double r = std::ldexp((double)M, lsb - BIAS);
    return neg ? -r : r;
  }
};

// Sum of |c|^2 over all terms, exact then rounded once.
double norm2_exact(const std::vector<Term>& A) {
  ExactSum s;
  for (const Term& a : A) {
    s.add_product(a.c.re, a.c.re);
    s.add_product(a.c.im, a.c.im);
  }
  return s.value();
}

// sum over strings present in both of A_s * B_s  (= Tr(AB)/2^N in the Hermitian basis),
// each component summed exactly then rounded once.
Cx trace_product(const std::vector<Term>& A, const std::vector<Term>& B) {
  Dict b;
  for (const Term& t : B) b[t.k] = t.c;
  ExactSum sr, si;
  for (const Term& a : A) {
    auto it = b.find(a.k);
    if (it == b.end()) continue;
    Cx c = it->second;
    sr.add_product(a.c.re, c.re);
    sr.add_product(-a.c.im, c.im);
    si.add_product(a.c.re, c.im);
    si.add_product(a.c.im, c.re);
  }
  return {sr.value(), si.value()};
}

struct Policy {
  int max_weight;   // < 0: off
  double cutoff;    // <= 0: off
  int64_t top_k;    // <= 0: off
  double gamma;     // 0: off
};

// Truncation after a step (paper: add_noise, trim, cutoff; "discarding long strings"):
//   1. depolarising transmission: c <- c * exp(-(gamma*dt) * wt), wt = pop(v|w);
//   2. Pauli-weight filter: drop wt > max_weight;
//   3. cutoff: drop |c|^2 < cutoff^2, |c|^2 = re*re + im*im;
//   4. top-k: keep the top_k strings by |c|^2, exact ties ranked by the smaller key;
//      strings of `keep` are never dropped by this step.
// Exact zeros are dropped.
std::vector<Term> truncate(const std::vector<Term>& O, const Policy& P, const std::vector<Term>& keep,
                           double dt) {
  std::vector<double> factor(129, 1.0);
  if (P.gamma != 0.0) {
    double x = P.gamma * dt;
    for (int wt = 0; wt <= 128; ++wt) factor[wt] = std::exp(-(x * (double)wt));
  }
  double cut2 = P.cutoff * P.cutoff;
  std::vector<Term> cand;
  cand.reserve(O.size());
  for (const Term& t : O) {
    int wt = popc(t.k.v | t.k.w);
    Cx c = t.c;
    if (P.gamma != 0.0) c = {c.re * factor[wt], c.im * factor[wt]};
    if (P.max_weight >= 0 && wt > P.max_weight) continue;
    if (c.re == 0.0 && c.im == 0.0) continue;
    if (P.cutoff > 0.0) {
      double a2 = c.re * c.re + c.im * c.im;
      if (a2 < cut2) continue;
    }
    cand.push_back({t.k, c});
  }
  if (P.top_k > 0 && (int64_t)cand.size() > P.top_k) {
    std::vector<std::pair<double, size_t>> r(cand.size());
    for (size_t i = 0; i < cand.size(); ++i)
      r[i] = {cand[i].c.re * cand[i].c.re + cand[i].c.im * cand[i].c.im, i};
    std::sort(r.begin(), r.end(), [&](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) {
      if (a.first != b.first) return a.first > b.first;
      return cand[a.second].k < cand[b.second].k;
    });
    std::vector<char> kept(cand.size(), 0);
    for (int64_t i = 0; i < P.top_k; ++i) kept[r[(size_t)i].second] = 1;
    if (!keep.empty()) {
      Dict kd;
      for (const Term& t : keep) kd[t.k] = t.c;
      for (size_t i = 0; i < cand.size(); ++i)
        if (kd.count(cand[i].k)) kept[i] = 1;
    }
    std::vector<Term> out;
    for (size_t i = 0; i < cand.size(); ++i)
      if (kept[i]) out.push_back(cand[i]);
    cand.swap(out);
  }
  std::sort(cand.begin(), cand.end(), [](const Term& a, const Term& b) { return a.k < b.k; });
  return cand;
}

// i * X (exact rotation of every coefficient).
std::vector<Term> times_i(const std::vector<Term>& X) {
  std::vector<Term> r = X;
  for (Term& t : r) t.c = rot(t.c, 1);
  return r;
}

// One classical RK4 step of dO/dt = i[H, O] (paper, "Heisenberg time evolution"):
//   k1 = i[H,O];  k2 = i[H, O + (dt/2) k1];  k3 = i[H, O + (dt/2) k2];  k4 = i[H, O + dt k3];
//   S = k1 + 2 k2;  S = S + 2 k3;  S = S + k4;  O' = O + (dt/6) S;
// then the truncation above.  With trim_stages, each k_j is cut to the top top_k strings
// right after its commutator (no keep set there).
std::vector<Term> rk4_step(const std::vector<Term>& H, const std::vector<Term>& O, double dt,
                           const Policy& P, const std::vector<Term>& keep, int trim_stages) {
  const double h2 = dt / 2.0, h6 = dt / 6.0;
  Policy stage{-1, 0.0, P.top_k, 0.0};
  std::vector<Term> none;
  auto L = [&](const std::vector<Term>& X) {
    std::vector<Term> k = times_i(commutator(H, X));
    if (trim_stages && P.top_k > 0) k = truncate(k, stage, none, dt);
    return k;
  };
  std::vector<Term> k1 = L(O);
  std::vector<Term> k2 = L(axpy(O, {h2, 0.0}, k1));
  std::vector<Term> k3 = L(axpy(O, {h2, 0.0}, k2));
  std::vector<Term> k4 = L(axpy(O, {dt, 0.0}, k3));
  std::vector<Term> S = axpy(k1, {2.0, 0.0}, k2);
  S = axpy(S, {2.0, 0.0}, k3);
  S = axpy(S, {1.0, 0.0}, k4);
  std::vector<Term> On = axpy(O, {h6, 0.0}, S);
  return truncate(On, P, keep, dt);
}

// ---------------------------------------------------------------------------
// Translation-symmetric operators on a periodic chain of n sites (Methods, the
// translation-symmetric encoding and Alg. 2).  Such an operator is O = sum_{i<n} T_i(O_0),
// T_i the translation by i sites (site j -> j + i mod n, a rotation of both masks), and is
// stored as its generator O_0: one representative string per translation orbit.
// ---------------------------------------------------------------------------
inline uint64_t rotl_n(uint64_t x, int k, int n) {
  const uint64_t mask = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  k %= n;
  if (k == 0) return x & mask;
  return ((x << k) | (x >> (n - k))) & mask;
}

inline Key translate(Key s, int k, int n) { return {rotl_n(s.v, k, n), rotl_n(s.w, k, n)}; }

// Representative of the orbit of s: its smallest translate in (v, then w) unsigned order;
// *r receives the smallest shift with T_r(s) equal to it.  (The paper's Shiftleft moves a
// string to start on the first site; any fixed choice of one string per orbit serves, and
// this one is also defined for strings that wrap around the ring.)
inline Key ts_canonical(Key s, int n, int* r) {
  Key best = s;
  int br = 0;
  for (int k = 1; k < n; ++k) {
    Key t = translate(s, k, n);
    if (t < best) {
      best = t;
      br = k;
    }
  }
  if (r) *r = br;
  return best;
}

// Smallest d > 0 with T_d(s) = s (a divisor of n).
inline int ts_period(Key s, int n) {
  for (int d = 1; d < n; ++d)
    if (translate(s, d, n) == s) return d;
  return n;
}

// sum_{k<n} T_k(G) as a plain sum: the translates T_0(G), T_1(G), ... added in turn (k outer,
// then G), so the contributions to one string arrive in increasing shift (one string of G
// per shift reaches a given string).
std::vector<Term> ts_expand(const std::vector<Term>& G, int n) {
  Dict C;
  for (int k = 0; k < n; ++k)
    for (const Term& g : G) {
      Key s = translate(g.k, k, n);
      auto it = C.find(s);
      if (it == C.end()) {
        C.emplace(s, g.c);
      } else {
        it->second.re += g.c.re;
        it->second.im += g.c.im;
      }
    }
  return canonical(C);
}

// Every string of X moved to its orbit's representative; the contributions to one
// representative are added in increasing shift r (distinct strings of one orbit need
// distinct smallest shifts, so the order is total).  Exact zeros dropped.
std::vector<Term> ts_canonical_merge(const std::vector<Term>& X, int n) {
  struct E {
    Key k;
    int r;
    Cx c;
  };
  std::vector<E> e;
  e.reserve(X.size());
  for (const Term& x : X) {
    int r = 0;
    Key k = ts_canonical(x.k, n, &r);
    e.push_back({k, r, x.c});
  }
  std::sort(e.begin(), e.end(), [](const E& a, const E& b) { return a.k < b.k || (a.k == b.k && a.r < b.r); });
  std::vector<Term> out;
  for (size_t i = 0; i < e.size();) {
    Cx acc = e[i].c;
    size_t j = i + 1;
    for (; j < e.size() && e[j].k == e[i].k; ++j) {
      acc.re += e[j].c.re;
      acc.im += e[j].c.im;
    }
    if (acc.re != 0.0 || acc.im != 0.0) out.push_back({e[i].k, acc});
    i = j;
  }
  return out;
}

// The translates of G as a list, not merged: T_0(G), T_1(G), ..., T_{n-1}(G) in turn.
std::vector<Term> ts_translates(const std::vector<Term>& G, int n) {
  std::vector<Term> out;
  out.reserve(G.size() * (size_t)n);
  for (int k = 0; k < n; ++k)
    for (const Term& g : G) out.push_back({translate(g.k, k, n), g.c});
  return out;
}

// [H, O] of translation-symmetric operators: H = sum_i T_i(H_0) is translation invariant,
// so [H, O] = sum_j T_j([H, O_0]) and its generator is [H, O_0] with H written out as the
// list of H_0's translates (Alg. 1's outer loop over that list), moved to representatives.
// Alg. 2 forms the same sums, A_0 against every translate of B_0; the loop order and the
// representative order above fix the rounding.
std::vector<Term> ts_commutator(const std::vector<Term>& H0, const std::vector<Term>& O0, int n) {
  return ts_canonical_merge(commutator(ts_translates(H0, n), O0), n);
}

// ||O||^2 / n for O = sum_i T_i(O_0): a representative of period d stands for n/d copies of
// each of its d distinct translates, so ||O||^2 = n sum_r (n/d_r) |c_r|^2.  The sum is exact,
// rounded once.
double ts_norm2_exact(const std::vector<Term>& O0, int n) {
  ExactSum s;
  for (const Term& t : O0) {
    const int m = n / ts_period(t.k, n);
    for (int j = 0; j < m; ++j) {
      s.add_product(t.c.re, t.c.re);
      s.add_product(t.c.im, t.c.im);
    }
  }
  return s.value();
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI for the Python test harness.  Results are returned through an opaque
// handle that owns its arrays (canonical key order).
// ---------------------------------------------------------------------------
struct or_result {
  std::vector<Term> t;
  std::vector<double> scalars;
};

extern "C" {

int64_t or_result_size(const or_result* r) { return (int64_t)r->t.size(); }

void or_result_copy(const or_result* r, uint64_t* v, uint64_t* w, double* re, double* im) {
  for (size_t i = 0; i < r->t.size(); ++i) {
    v[i] = r->t[i].k.v;
    w[i] = r->t[i].k.w;
    re[i] = r->t[i].c.re;
    im[i] = r->t[i].c.im;
  }
}

int64_t or_result_nscalars(const or_result* r) { return (int64_t)r->scalars.size(); }

void or_result_scalars(const or_result* r, double* out) {
  for (size_t i = 0; i < r->scalars.size(); ++i) out[i] = r->scalars[i];
}

void or_result_free(or_result* r) { delete r; }

// Single-string product P_a P_b = i^k P_c: returns k, writes c.
int or_string_product(uint64_t va, uint64_t wa, uint64_t vb, uint64_t wb, uint64_t* vc, uint64_t* wc) {
  *vc = va ^ vb;
  *wc = wa ^ wb;
  return product_phase(va, wa, vb, wb);
}

int or_anticommute(uint64_t va, uint64_t wa, uint64_t vb, uint64_t wb) {
  return anticommute(va, wa, vb, wb) ? 1 : 0;
}

// [A, B] by Alg. 1 (A outer in the given order).  Parity: pinned by the single-site
// Pauli table, dense 2^N matrices and the printed Lanczos example.
or_result* or_commutator(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim,
                         int64_t na, const uint64_t* bv, const uint64_t* bw, const double* bre,
                         const double* bim, int64_t nb) {
  return new or_result{commutator(from_arrays(av, aw, are, aim, na), from_arrays(bv, bw, bre, bim, nb)), {}};
}

// A B by Alg. 1 (A outer in the given order).  Parity: pinned by dense matrix products,
// the single-site Pauli table, AB - BA = [A, B] and exact associativity on dyadic sums.
or_result* or_product(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim,
                      int64_t na, const uint64_t* bv, const uint64_t* bw, const double* bre,
                      const double* bim, int64_t nb) {
  return new or_result{product(from_arrays(av, aw, are, aim, na), from_arrays(bv, bw, bre, bim, nb)), {}};
}

// Translation-symmetric operators (n = ring length).  Parity: pinned by brute-force orbit
// checks, dense matrices of the expanded operators, expand(C_0) = [expand(H_0), expand(O_0)]
// bit for bit on dyadic sums, and b_n equal to the plain Lanczos of the expanded chain.
or_result* or_ts_expand(const uint64_t* gv, const uint64_t* gw, const double* gre, const double* gim, int64_t ng,
                        int n) {
  return new or_result{ts_expand(from_arrays(gv, gw, gre, gim, ng), n), {}};
}

or_result* or_ts_canonical_merge(const uint64_t* xv, const uint64_t* xw, const double* xre, const double* xim,
                                 int64_t nx, int n) {
  return new or_result{ts_canonical_merge(from_arrays(xv, xw, xre, xim, nx), n), {}};
}

int or_ts_canonical(uint64_t v, uint64_t w, int n, uint64_t* cv, uint64_t* cw) {
  int r = 0;
  Key k = ts_canonical({v, w}, n, &r);
  *cv = k.v;
  *cw = k.w;
  return r;
}

int or_ts_period(uint64_t v, uint64_t w, int n) { return ts_period({v, w}, n); }

or_result* or_ts_commutator(const uint64_t* hv, const uint64_t* hw, const double* hre, const double* him,
                            int64_t nh, const uint64_t* ov, const uint64_t* ow, const double* ore,
                            const double* oim, int64_t no, int n) {
  return new or_result{ts_commutator(from_arrays(hv, hw, hre, him, nh), from_arrays(ov, ow, ore, oim, no), n), {}};
}

double or_ts_norm2(const uint64_t* ov, const uint64_t* ow, const double* ore, const double* oim, int64_t no, int n) {
  return ts_norm2_exact(from_arrays(ov, ow, ore, oim, no), n);
}

// One Lanczos step of translation-symmetric operators, as the plain step with the TS
// commutator and norm: A_0 = C_0 - b_prev O_prev,0, b = ||A||, O_0 = trunc(A_0 / b).
or_result* or_ts_lanczos_step(const uint64_t* hv, const uint64_t* hw, const double* hre, const double* him,
                              int64_t nh, const uint64_t* pv, const uint64_t* pw, const double* pre,
                              const double* pim, int64_t np, const uint64_t* cv, const uint64_t* cw,
                              const double* cre, const double* cim, int64_t nc, double b_prev, int max_weight,
                              double cutoff, int64_t top_k, int n) {
  std::vector<Term> H0 = from_arrays(hv, hw, hre, him, nh);
  std::vector<Term> Op = from_arrays(pv, pw, pre, pim, np);
  std::vector<Term> Oc = from_arrays(cv, cw, cre, cim, nc);
  std::vector<Term> A = ts_commutator(H0, Oc, n);
  if (!Op.empty()) A = axpy(A, {-b_prev, 0.0}, Op);
  const double b = std::sqrt(ts_norm2_exact(A, n));
  or_result* r = new or_result;
  r->scalars.push_back(b);
  if (b == 0.0) return r;
  Policy P{max_weight, cutoff, top_k, 0.0};
  std::vector<Term> none;
  r->t = truncate(divide(A, b), P, none, 0.0);
  return r;
}

// A + alpha B.  Parity: pinned by dense matrices and by brute force on small inputs.
or_result* or_axpy(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim, int64_t na,
                   double alpha_re, double alpha_im, const uint64_t* bv, const uint64_t* bw, const double* bre,
                   const double* bim, int64_t nb) {
  return new or_result{axpy(from_arrays(av, aw, are, aim, na), {alpha_re, alpha_im},
                            from_arrays(bv, bw, bre, bim, nb)), {}};
}

or_result* or_scale(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim, int64_t na,
                    double s) {
  return new or_result{scale(from_arrays(av, aw, are, aim, na), s), {}};
}

or_result* or_divide(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim, int64_t na,
                     double b) {
  return new or_result{divide(from_arrays(av, aw, are, aim, na), b), {}};
}

// sum |c|^2, exact then rounded once.  Parity: pinned against exact rational arithmetic.
double or_norm2(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim, int64_t na) {
  return norm2_exact(from_arrays(av, aw, are, aim, na));
}

void or_trace_product(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim, int64_t na,
                      const uint64_t* bv, const uint64_t* bw, const double* bre, const double* bim, int64_t nb,
                      double* out_re, double* out_im) {
  Cx c = trace_product(from_arrays(av, aw, are, aim, na), from_arrays(bv, bw, bre, bim, nb));
  *out_re = c.re;
  *out_im = c.im;
}

or_result* or_truncate(const uint64_t* av, const uint64_t* aw, const double* are, const double* aim, int64_t na,
                       int max_weight, double cutoff, int64_t top_k, double gamma, double dt,
                       const uint64_t* kv, const uint64_t* kw, int64_t nk) {
  std::vector<Term> keep;
  for (int64_t i = 0; i < nk; ++i) keep.push_back({{kv[i], kw[i]}, {1.0, 0.0}});
  return new or_result{truncate(from_arrays(av, aw, are, aim, na), {max_weight, cutoff, top_k, gamma}, keep, dt), {}};
}

// One RK4 step with truncation.  Parity: pinned by dense RK4 and the closed form for H = hZ_1.
or_result* or_rk4_step(const uint64_t* hv, const uint64_t* hw, const double* hre, const double* him, int64_t nh,
                       const uint64_t* ov, const uint64_t* ow, const double* ore, const double* oim, int64_t no,
                       double dt, int max_weight, double cutoff, int64_t top_k, double gamma, int trim_stages,
                       const uint64_t* kv, const uint64_t* kw, int64_t nk) {
  std::vector<Term> keep;
  for (int64_t i = 0; i < nk; ++i) keep.push_back({{kv[i], kw[i]}, {1.0, 0.0}});
  return new or_result{rk4_step(from_arrays(hv, hw, hre, him, nh), from_arrays(ov, ow, ore, oim, no), dt,
                                {max_weight, cutoff, top_k, gamma}, keep, trim_stages), {}};
}

// Lanczos recursion (paper, "Krylov subspace expansion"; eqs. for O_1, b_1, O_n', O_n, b_n):
//   b_1 = ||[H,O_0]||, O_1 = trunc([H,O_0] / b_1);
//   A = [H,O_{n-1}] - b_{n-1} O_{n-2},  b_n = ||A||,  O_n = trunc(A / b_n),
// with ||X|| = sqrt(sum |c|^2) (the normalised Frobenius norm) and trunc the
// cutoff / top-k truncation.  Runs n_steps coefficients (stops early when b_n = 0).
// scalars = b_1..b_n; terms = the last O_n (and O_{n-1} follows it when want_prev).
or_result* or_lanczos(const uint64_t* hv, const uint64_t* hw, const double* hre, const double* him, int64_t nh,
                      const uint64_t* ov, const uint64_t* ow, const double* ore, const double* oim, int64_t no,
                      int n_steps, int max_weight, double cutoff, int64_t top_k) {
  std::vector<Term> H = from_arrays(hv, hw, hre, him, nh);
  std::vector<Term> Oprev = from_arrays(ov, ow, ore, oim, no);
  Policy P{max_weight, cutoff, top_k, 0.0};
  std::vector<Term> none;
  or_result* r = new or_result;
  std::vector<Term> A = commutator(H, Oprev);
  double b = std::sqrt(norm2_exact(A));
  r->scalars.push_back(b);
  if (b == 0.0) { r->t = Oprev; return r; }
  std::vector<Term> Ocur = truncate(divide(A, b), P, none, 0.0);
  for (int n = 2; n <= n_steps; ++n) {
    A = axpy(commutator(H, Ocur), {-b, 0.0}, Oprev);
    double bn = std::sqrt(norm2_exact(A));
    r->scalars.push_back(bn);
    if (bn == 0.0) break;
    std::vector<Term> On = truncate(divide(A, bn), P, none, 0.0);
    Oprev.swap(Ocur);
    Ocur.swap(On);
    b = bn;
  }
  r->t = Ocur;
  return r;
}

}  // extern "C"
