// Plain CPU oracle for the sparse-wavefunction UCC path.
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the entry module's smoke check
// and the benchmark's CPU-baseline leg may load this library.  It shares no
// code, header, table or helper with the CUDA library; both read the same
// seeded inputs and nothing else.
//
// What it computes, in the paper's order and notation (Mullinax & Tubman,
// "Large-scale sparse wavefunction circuit simulator ..."):
//   * the factorised UCC state of Eq. 3, U_K ... U_1 |Psi_0>, with each factor
//     U_k = exp(theta_k (tau_k - tau_k^+)) (Eqs. 4-5) applied to a sparse map
//     determinant -> amplitude (Results section; Methods section);
//   * after each factor, amplitudes with |c| < eps are discarded (Methods
//     section), optionally followed by the N_MAX / N_CUT rule of the Methods
//     section (sort by |c|, keep N_CUT when more than N_MAX remain);
//   * the energy <psi|H|psi>/<psi|psi> of the second-quantised Hamiltonian
//     built from the one- and two-electron integrals (Methods section) with
//     the Slater-Condon rules;
//   * dE/dtheta for every factor by a checkpointed reverse (adjoint) sweep.
//
// Readings where the paper is silent (each is listed in the design notes):
//   * the factor's closed form (the paper cites Chen, Cheng and Freericks but
//     does not print it): with A = tau - tau^+ and tau|E> = s|D>, A acts on
//     span{E, D} as the generator of a plane rotation, so
//         c_E' = cos(theta) c_E - s sin(theta) c_D
//         c_D' = cos(theta) c_D + s sin(theta) c_E
//     and as zero on determinants that tau and tau^+ both annihilate;
//   * tau = a+_a a+_b a_j a_i for row (i, j, a, b); a single is a+_a a_i;
//   * Jordan-Wigner: a_p and a+_p pick up (-1)^(number of occupied
//     spin-orbitals with index below p);
//   * a missing partner enters the rotation with amplitude +0.0 and is
//     created; the eps test is strict (|c| < eps is dropped) and applies to the
//     two members of every rotated pair;
//   * no renormalisation: E = <psi|H|psi>/<psi|psi>.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off (no fused multiply-add, so each
// rotation is two rounded products and one rounded sum), once with
// ORC_KEY_BITS=64 (determinant keys in one 64-bit word, up to 64
// spin-orbitals; entry points orc_*) and once with ORC_KEY_BITS=128 (keys in a
// 128-bit integer, up to 128 spin-orbitals; entry points orc128_*, keys passed
// as (low, high) pairs of 64-bit words), both linked into one library.  The
// two builds are the same source: only the key type and the entry-point
// names differ.
// Parity: pinned by the tests in tests/test_oracle_*.py (dense state-vector
// brute force, closed forms, invariants, finite differences and the exact
// parameter-shift rule).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#ifndef ORC_KEY_BITS
#define ORC_KEY_BITS 64
#endif

namespace {

#if ORC_KEY_BITS == 64
typedef uint64_t Key;
typedef std::hash<uint64_t> KeyHash;
#define ORC(name) orc_##name
// Keys at the C boundary: one 64-bit word each.
Key load_key(const uint64_t* a, long long t) { return a[t]; }
void store_key(uint64_t* a, long long t, Key k) { a[t] = k; }
#elif ORC_KEY_BITS == 128
typedef unsigned __int128 Key;
struct KeyHash {
  size_t operator()(Key k) const {
    const uint64_t lo = (uint64_t)k, hi = (uint64_t)(k >> 64);
    return std::hash<uint64_t>()(lo ^ (hi * 0x9E3779B97F4A7C15ULL));
  }
};
#define ORC(name) orc128_##name
// Keys at the C boundary: two 64-bit words each, low word first.
Key load_key(const uint64_t* a, long long t) { return ((Key)a[2 * t + 1] << 64) | (Key)a[2 * t]; }
void store_key(uint64_t* a, long long t, Key k) {
  a[2 * t] = (uint64_t)k;
  a[2 * t + 1] = (uint64_t)(k >> 64);
}
#else
#error "ORC_KEY_BITS must be 64 or 128"
#endif

constexpr int kKeyBits = ORC_KEY_BITS;
Key bit(int p) { return (Key)1 << p; }

typedef std::unordered_map<Key, double, KeyHash> Psi;

struct Excitation {
  int i, j, a, b;  // j = b = -1 for a single
};

struct Problem {
  int n_spatial = 0, n_alpha = 0, n_beta = 0;
  std::vector<double> h;  // n_spatial^2, row-major
  std::vector<double> g;  // n_spatial^4, chemist (pq|rs)
  std::vector<Excitation> exc;
  int n_so() const { return 2 * n_spatial; }
  Key reference() const {
    Key det = 0;
    for (int s = 0; s < n_alpha; ++s) det |= bit(2 * s);
    for (int s = 0; s < n_beta; ++s) det |= bit(2 * s + 1);
    return det;
  }
};

struct Counts {
  long long rotations = 0;       // linked pairs updated (det-rotations)
  long long created = 0;         // partners that entered the map
  long long dropped_new = 0;     // partners computed but below eps
  long long dropped_old = 0;     // existing entries that fell below eps
  long long cut = 0;             // entries removed by the N_MAX/N_CUT rule
};

// ------------------------------------------------------------------------
// Jordan-Wigner second quantisation on determinant keys (bit p = spin-orbital p).
// ------------------------------------------------------------------------
bool is_occupied(Key det, int p) { return ((det >> p) & 1) != 0; }

int occupied_below(Key det, int p) {
  int count = 0;
  for (int q = 0; q < p; ++q)
    if (is_occupied(det, q)) ++count;
  return count;
}

bool annihilate(Key& det, int p, int& sign) {
  if (!is_occupied(det, p)) return false;
  if (occupied_below(det, p) % 2 == 1) sign = -sign;
  det &= ~bit(p);
  return true;
}

bool create(Key& det, int p, int& sign) {
  if (is_occupied(det, p)) return false;
  if (occupied_below(det, p) % 2 == 1) sign = -sign;
  det |= bit(p);
  return true;
}

// tau |det> = sign |out>, operators applied right to left: a_i, a_j, a+_b, a+_a.
bool apply_tau(const Excitation& e, Key det, Key* out, int* sign) {
  int s = 1;
  Key d = det;
  if (!annihilate(d, e.i, s)) return false;
  if (e.j >= 0 && !annihilate(d, e.j, s)) return false;
  if (e.b >= 0 && !create(d, e.b, s)) return false;
  if (!create(d, e.a, s)) return false;
  *out = d;
  *sign = s;
  return true;
}

// tau^+ |det> = sign |out>, tau^+ = a+_i a+_j a_b a_a, applied right to left.
bool apply_tau_dagger(const Excitation& e, Key det, Key* out, int* sign) {
  int s = 1;
  Key d = det;
  if (!annihilate(d, e.a, s)) return false;
  if (e.b >= 0 && !annihilate(d, e.b, s)) return false;
  if (e.j >= 0 && !create(d, e.j, s)) return false;
  if (!create(d, e.i, s)) return false;
  *out = d;
  *sign = s;
  return true;
}

// A linked pair of factor k: E is the member tau excites, D = tau E up to sign.
struct Pair {
  Key E, D;
  int sign;  // tau|E> = sign |D>
};

// Classify det under factor k.  Returns false if tau and tau^+ both kill it.
bool pair_of(const Excitation& e, Key det, Pair* out) {
  Key other;
  int sign;
  if (apply_tau(e, det, &other, &sign)) {
    *out = Pair{det, other, sign};
    return true;
  }
  if (apply_tau_dagger(e, det, &other, &sign)) {
    Key back;
    int s2;
    apply_tau(e, other, &back, &s2);  // the sign is defined from the excited side
    *out = Pair{other, det, s2};
    return true;
  }
  return false;
}

double value_or_zero(const Psi& psi, Key key) {
  auto it = psi.find(key);
  return it == psi.end() ? 0.0 : it->second;
}

// ------------------------------------------------------------------------
// One factor of Eq. 3 (Eqs. 4-5 in the rotation form) plus the eps rule.
// ------------------------------------------------------------------------
void store_or_drop(Psi& out, Key key, double v, double eps, bool existed, Counts& cnt) {
  if (std::fabs(v) < eps) {
    if (existed) {
      out.erase(key);
      ++cnt.dropped_old;
    } else {
      ++cnt.dropped_new;
    }
  } else {
    out[key] = v;
    if (!existed) ++cnt.created;
  }
}

Psi apply_factor(const Excitation& e, double c, double s, double eps, const Psi& before, Counts& cnt) {
  Psi after = before;
  for (const auto& kv : before) {
    Pair p;
    if (!pair_of(e, kv.first, &p)) continue;
    // Each pair is rotated once: from its excited member E when E is in the
    // map, otherwise from D.
    if (kv.first == p.D && before.count(p.E)) continue;
    bool hasE = before.count(p.E) != 0, hasD = before.count(p.D) != 0;
    double cE = value_or_zero(before, p.E);
    double cD = value_or_zero(before, p.D);
    double ss = p.sign > 0 ? s : -s;
    double newE = c * cE - ss * cD;
    double newD = c * cD + ss * cE;
    ++cnt.rotations;
    store_or_drop(after, p.E, newE, eps, hasE, cnt);
    store_or_drop(after, p.D, newD, eps, hasD, cnt);
  }
  return after;
}

// Methods-section wavefunction truncation: if more than n_max determinants
// remain, keep the n_cut of largest |c| (ties: smaller key first).
void truncate_top(Psi& psi, long long n_max, long long n_cut, Counts& cnt) {
  if (n_max <= 0 || (long long)psi.size() <= n_max) return;
  std::vector<std::pair<Key, double>> all(psi.begin(), psi.end());
  std::sort(all.begin(), all.end(), [](const std::pair<Key, double>& x, const std::pair<Key, double>& y) {
    double ax = std::fabs(x.second), ay = std::fabs(y.second);
    if (ax != ay) return ax > ay;
    return x.first < y.first;
  });
  cnt.cut += (long long)all.size() - n_cut;
  all.resize((size_t)n_cut);
  psi.clear();
  for (const auto& kv : all) psi[kv.first] = kv.second;
}

// Eq. 6: S = - sum_I |c_I|^2 ln |c_I|^2 over the map (0 ln 0 = 0).
double entropy(const Psi& psi) {
  double s = 0.0, comp = 0.0;  // Neumaier
  for (const auto& kv : psi) {
    const double p = kv.second * kv.second;
    if (p == 0.0) continue;
    const double x = -p * std::log(p);
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      comp += (s - t) + x;
    else
      comp += (x - t) + s;
    s = t;
  }
  return s + comp;
}

Psi run_factors(const Problem& P, const double* theta, int k0, int k1, double eps, long long n_max,
                long long n_cut, Psi psi, Counts& cnt, double* entropy_out = nullptr) {
  for (int k = k0; k < k1; ++k) {
    psi = apply_factor(P.exc[k], std::cos(theta[k]), std::sin(theta[k]), eps, psi, cnt);
    truncate_top(psi, n_max, n_cut, cnt);
    if (entropy_out) entropy_out[k] = entropy(psi);
  }
  return psi;
}

// ------------------------------------------------------------------------
// Hamiltonian: spin-orbital integrals from the spatial ones, Slater-Condon.
//   h_pq   = h(p/2, q/2) if spin p == spin q
//   <pq|rs> = (pr|qs) if spin p == spin r and spin q == spin s
//   <pq||rs> = <pq|rs> - <pq|sr>
//   H = sum h_pq a+_p a_q + 1/4 sum <pq||rs> a+_p a+_q a_s a_r
// ------------------------------------------------------------------------
double h_so(const Problem& P, int p, int q) {
  if ((p & 1) != (q & 1)) return 0.0;
  return P.h[(size_t)(p >> 1) * P.n_spatial + (q >> 1)];
}

double chem(const Problem& P, int p, int q, int r, int s) {
  const size_t n = (size_t)P.n_spatial;
  return P.g[((p * n + q) * n + r) * n + s];
}

double phys(const Problem& P, int p, int q, int r, int s) {
  if ((p & 1) != (r & 1) || (q & 1) != (s & 1)) return 0.0;
  return chem(P, p >> 1, r >> 1, q >> 1, s >> 1);
}

double anti(const Problem& P, int p, int q, int r, int s) { return phys(P, p, q, r, s) - phys(P, p, q, s, r); }

// The set bits of a key, ascending.
struct Bits {
  int n = 0;
  int p[kKeyBits];
};

Bits bits_of(Key x) {
  Bits out;
  for (int q = 0; q < kKeyBits; ++q)
    if (is_occupied(x, q)) out.p[out.n++] = q;
  return out;
}

// <J|H|I>
double hmat(const Problem& P, Key I, Key J) {
  Bits holes = bits_of(I & ~J);      // occupied in I, empty in J
  Bits particles = bits_of(J & ~I);  // empty in I, occupied in J
  if (holes.n != particles.n || holes.n > 2) return 0.0;
  Bits occ = bits_of(I);
  if (holes.n == 0) {
    double v = 0.0;
    for (int x = 0; x < occ.n; ++x) v += h_so(P, occ.p[x], occ.p[x]);
    for (int x = 0; x < occ.n; ++x)
      for (int y = 0; y < occ.n; ++y) v += 0.5 * anti(P, occ.p[x], occ.p[y], occ.p[x], occ.p[y]);
    return v;
  }
  if (holes.n == 1) {
    int i = holes.p[0], a = particles.p[0];
    int sign = 1;
    Key d = I;
    annihilate(d, i, sign);
    create(d, a, sign);
    double v = h_so(P, a, i);
    for (int x = 0; x < occ.n; ++x)
      if (occ.p[x] != i) v += anti(P, a, occ.p[x], i, occ.p[x]);
    return sign * v;
  }
  int i = holes.p[0], j = holes.p[1], a = particles.p[0], b = particles.p[1];
  int sign = 1;
  Key d = I;
  annihilate(d, i, sign);
  annihilate(d, j, sign);
  create(d, b, sign);
  create(d, a, sign);
  return sign * anti(P, a, b, i, j);
}

// Neumaier's compensated summation.
struct Sum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// sigma_I = sum_{J in psi} <I|H|J> c_J for one I (psi's keys only), by
// generating every determinant one spin-conserving single or double away from
// I and looking it up.
double sigma_one(const Problem& P, const Psi& psi, Key I) {
  Bits occ = bits_of(I);
  Bits emp;
  for (int p = 0; p < P.n_so(); ++p)
    if (!is_occupied(I, p)) emp.p[emp.n++] = p;
  Sum acc;
  acc.add(hmat(P, I, I) * value_or_zero(psi, I));
  for (int x = 0; x < occ.n; ++x)
    for (int u = 0; u < emp.n; ++u) {
      int p = occ.p[x], q = emp.p[u];
      if ((p & 1) != (q & 1)) continue;
      Key J = (I & ~bit(p)) | bit(q);
      auto it = psi.find(J);
      if (it != psi.end()) acc.add(hmat(P, I, J) * it->second);
    }
  for (int x = 0; x < occ.n; ++x)
    for (int y = x + 1; y < occ.n; ++y)
      for (int u = 0; u < emp.n; ++u)
        for (int v = u + 1; v < emp.n; ++v) {
          int p = occ.p[x], q = occ.p[y], r = emp.p[u], s = emp.p[v];
          if ((p & 1) + (q & 1) != (r & 1) + (s & 1)) continue;
          Key J = (I & ~bit(p) & ~bit(q)) | bit(r) | bit(s);
          auto it = psi.find(J);
          if (it != psi.end()) acc.add(hmat(P, I, J) * it->second);
        }
  return acc.value();
}

Psi sigma_lookup(const Problem& P, const Psi& psi) {
  Psi sigma;
  for (const auto& kv : psi) sigma[kv.first] = sigma_one(P, psi, kv.first);
  return sigma;
}

// The same sigma from every pair of map entries (O(N^2)).
Psi sigma_pairwise(const Problem& P, const Psi& psi) {
  Psi sigma;
  for (const auto& a : psi) {
    Sum acc;
    for (const auto& b : psi) acc.add(hmat(P, a.first, b.first) * b.second);
    sigma[a.first] = acc.value();
  }
  return sigma;
}

void energy_from_sigma(const Psi& psi, const Psi& sigma, double* E, double* norm2) {
  Sum num, den;
  for (const auto& kv : psi) {
    num.add(kv.second * sigma.at(kv.first));
    den.add(kv.second * kv.second);
  }
  *norm2 = den.value();
  *E = num.value() / den.value();
}

// ------------------------------------------------------------------------
// Adjoint gradient.  With the prune sets held fixed, psi_k = P_k U_k psi_{k-1}
// (P_k keeps the map's keys after factor k).  For
//   E = <psi|H|psi>/<psi|psi>,  dE/dtheta_k = 2 <lambda_{k-1}| A_k psi_{k-1}>
// with mu_K = P_K (H psi - E psi)/<psi|psi>, lambda_{k-1} = U_k^T mu_k and
// mu_{k-1} = P_{k-1} lambda_{k-1}.  On a pair (E, D), A psi has D-component
// s psi_E and E-component -s psi_D, and U^T rotates by -theta.  Intermediate
// states come from checkpoints every `stride` factors and a forward
// recomputation of each segment.
// ------------------------------------------------------------------------
void gradient(const Problem& P, const double* theta, double eps, long long n_max, long long n_cut, int stride,
              double* E_out, double* grad) {
  const int K = (int)P.exc.size();
  if (stride <= 0) stride = std::max(1, (int)std::ceil(std::sqrt((double)K)));
  Counts cnt;
  std::vector<Psi> checkpoints;
  Psi psi;
  psi[P.reference()] = 1.0;
  for (int k = 0; k < K; ++k) {
    if (k % stride == 0) checkpoints.push_back(psi);
    psi = run_factors(P, theta, k, k + 1, eps, n_max, n_cut, psi, cnt);
  }
  Psi sigma = sigma_lookup(P, psi);
  double E, norm2;
  energy_from_sigma(psi, sigma, &E, &norm2);
  *E_out = E;
  Psi mu;
  for (const auto& kv : psi) mu[kv.first] = (sigma.at(kv.first) - E * kv.second) / norm2;

  for (int seg = (int)checkpoints.size() - 1; seg >= 0; --seg) {
    int k0 = seg * stride, k1 = std::min(K, k0 + stride);
    std::vector<Psi> states;  // states[t] = psi before factor k0 + t
    states.push_back(checkpoints[seg]);
    for (int k = k0; k < k1 - 1; ++k) states.push_back(run_factors(P, theta, k, k + 1, eps, n_max, n_cut, states.back(), cnt));
    for (int k = k1 - 1; k >= k0; --k) {
      const Psi& before = states[k - k0];
      const Excitation& e = P.exc[k];
      double c = std::cos(theta[k]), s = std::sin(theta[k]);
      // lambda = U_k^T mu on every pair touching mu's support; elsewhere lambda = mu.
      Psi lambda = mu;
      std::unordered_set<Key, KeyHash> candidates;
      for (const auto& kv : mu) candidates.insert(kv.first);
      for (const auto& kv : before) candidates.insert(kv.first);
      std::unordered_set<Key, KeyHash> done;
      Sum gk;
      for (Key key : candidates) {
        Pair p;
        if (!pair_of(e, key, &p)) continue;
        if (done.count(p.E)) continue;
        done.insert(p.E);
        double ss = p.sign > 0 ? s : -s;
        double muE = value_or_zero(mu, p.E), muD = value_or_zero(mu, p.D);
        double lamE = c * muE + ss * muD;
        double lamD = c * muD - ss * muE;
        lambda[p.E] = lamE;
        lambda[p.D] = lamD;
        double psiE = value_or_zero(before, p.E), psiD = value_or_zero(before, p.D);
        gk.add(p.sign * (lamD * psiE - lamE * psiD));
      }
      grad[k] = 2.0 * gk.value();
      Psi restricted;
      for (const auto& kv : before) {
        auto it = lambda.find(kv.first);
        restricted[kv.first] = it == lambda.end() ? 0.0 : it->second;
      }
      mu.swap(restricted);
    }
  }
}

struct WF {
  std::vector<Key> keys;
  std::vector<double> amps;
};

WF export_sorted(const Psi& psi) {
  std::vector<std::pair<Key, double>> all(psi.begin(), psi.end());
  std::sort(all.begin(), all.end());
  WF w;
  for (const auto& kv : all) {
    w.keys.push_back(kv.first);
    w.amps.push_back(kv.second);
  }
  return w;
}

Psi from_arrays(long long n, const uint64_t* keys, const double* amps) {
  Psi psi;
  for (long long t = 0; t < n; ++t) psi[load_key(keys, t)] = amps[t];
  return psi;
}

Psi from_wf(const WF& w) {
  Psi psi;
  for (size_t t = 0; t < w.keys.size(); ++t) psi[w.keys[t]] = w.amps[t];
  return psi;
}

}  // namespace

extern "C" {

struct orc_counts {
  long long rotations, created, dropped_new, dropped_old, cut;
};

void* ORC(problem_new)(int n_spatial, int n_alpha, int n_beta, const double* h, const double* g, int n_exc,
                      const int* exc) {
  Problem* P = new Problem;
  P->n_spatial = n_spatial;
  P->n_alpha = n_alpha;
  P->n_beta = n_beta;
  size_t n = (size_t)n_spatial;
  P->h.assign(h, h + n * n);
  P->g.assign(g, g + n * n * n * n);
  for (int k = 0; k < n_exc; ++k) P->exc.push_back(Excitation{exc[4 * k], exc[4 * k + 1], exc[4 * k + 2], exc[4 * k + 3]});
  return P;
}

void ORC(problem_free)(void* p) { delete static_cast<Problem*>(p); }

// Apply factors [0, n_factors) to the reference; returns a wavefunction handle.
// entropy_out (optional, n_factors doubles): Eq. 6 after each factor.
void* ORC(apply)(const void* prob, const double* theta, int n_factors, double eps, long long n_max, long long n_cut,
                orc_counts* counts, double* entropy_out) {
  const Problem& P = *static_cast<const Problem*>(prob);
  Counts cnt;
  Psi psi;
  psi[P.reference()] = 1.0;
  psi = run_factors(P, theta, 0, n_factors, eps, n_max, n_cut, psi, cnt, entropy_out);
  if (counts) *counts = orc_counts{cnt.rotations, cnt.created, cnt.dropped_new, cnt.dropped_old, cnt.cut};
  return new WF(export_sorted(psi));
}

// keys: n keys at the C boundary (see load_key).
void* ORC(wf_from_arrays)(long long n, const uint64_t* keys, const double* amps) {
  return new WF(export_sorted(from_arrays(n, keys, amps)));
}

long long ORC(wf_size)(const void* wf) { return (long long)static_cast<const WF*>(wf)->keys.size(); }

void ORC(wf_export)(const void* wf, uint64_t* keys, double* amps) {
  const WF& w = *static_cast<const WF*>(wf);
  for (size_t t = 0; t < w.keys.size(); ++t) store_key(keys, (long long)t, w.keys[t]);
  if (!w.amps.empty()) std::memcpy(amps, w.amps.data(), w.amps.size() * sizeof(double));
}

void ORC(wf_free)(void* wf) { delete static_cast<WF*>(wf); }

// sigma over the wavefunction's keys (sorted by key), route 0 = generate and
// look up, route 1 = all pairs.
void ORC(sigma)(const void* prob, const void* wf, int route, double* sigma_out) {
  const Problem& P = *static_cast<const Problem*>(prob);
  const WF& w = *static_cast<const WF*>(wf);
  Psi psi = from_wf(w);
  Psi sigma = route == 1 ? sigma_pairwise(P, psi) : sigma_lookup(P, psi);
  for (size_t t = 0; t < w.keys.size(); ++t) sigma_out[t] = sigma.at(w.keys[t]);
}

// sigma_I for the n query keys I (each must be a key of the wavefunction or
// not: sigma is P_S H psi evaluated at I either way).
void ORC(sigma_at)(const void* prob, const void* wf, long long n, const uint64_t* query, double* out) {
  const Problem& P = *static_cast<const Problem*>(prob);
  const WF& w = *static_cast<const WF*>(wf);
  Psi psi = from_wf(w);
  for (long long t = 0; t < n; ++t) out[t] = sigma_one(P, psi, load_key(query, t));
}

void ORC(energy)(const void* prob, const void* wf, int route, double* E, double* norm2) {
  const Problem& P = *static_cast<const Problem*>(prob);
  const WF& w = *static_cast<const WF*>(wf);
  Psi psi = from_wf(w);
  Psi sigma = route == 1 ? sigma_pairwise(P, psi) : sigma_lookup(P, psi);
  energy_from_sigma(psi, sigma, E, norm2);
}

// <J|H|I> and tau_k |det> (which = 0) or tau_k^+ |det> (which = 1; returns
// the sign, or 0 when the operator annihilates det).  The 64-bit build takes
// keys by value; the 128-bit build takes pointers to (low, high) pairs.
#if ORC_KEY_BITS == 64
double ORC(hmat)(const void* prob, uint64_t I, uint64_t J) {
  return hmat(*static_cast<const Problem*>(prob), I, J);
}

int ORC(tau)(const void* prob, int k, int which, uint64_t det, uint64_t* out) {
  const Problem& P = *static_cast<const Problem*>(prob);
  int sign = 0;
  Key o = 0;
  bool ok = which == 0 ? apply_tau(P.exc[k], det, &o, &sign) : apply_tau_dagger(P.exc[k], det, &o, &sign);
  *out = o;
  return ok ? sign : 0;
}
#else
double ORC(hmat)(const void* prob, const uint64_t* I, const uint64_t* J) {
  return hmat(*static_cast<const Problem*>(prob), load_key(I, 0), load_key(J, 0));
}

int ORC(tau)(const void* prob, int k, int which, const uint64_t* det, uint64_t* out) {
  const Problem& P = *static_cast<const Problem*>(prob);
  int sign = 0;
  Key o = 0;
  const Key d = load_key(det, 0);
  bool ok = which == 0 ? apply_tau(P.exc[k], d, &o, &sign) : apply_tau_dagger(P.exc[k], d, &o, &sign);
  store_key(out, 0, o);
  return ok ? sign : 0;
}
#endif

void ORC(gradient)(const void* prob, const double* theta, double eps, long long n_max, long long n_cut, int stride,
                  double* E, double* grad) {
  gradient(*static_cast<const Problem*>(prob), theta, eps, n_max, n_cut, stride, E, grad);
}

}  // extern "C"
