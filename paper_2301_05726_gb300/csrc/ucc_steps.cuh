// Per-entry bodies of the factor steps, shared by the single-problem kernels
// and the batched (many-job) kernels so both run the same arithmetic.
#pragma once

#include "ucc_device.cuh"

namespace ucc {

// Bit-pattern tests and sign flips of doubles.  They are written in inline
// PTX on 32/64-bit integer registers: as plain C++ the compiler recognises
// the patterns and turns them back into FP64 negations and compares, which
// run on the GPU's narrow FP64 pipe.

// |v| < eps for finite v and eps >= 0 (non-negative doubles order like their
// bit patterns).
__device__ __forceinline__ bool below_eps(double v, double eps) {
  unsigned int r;
  asm("{\n\t.reg .pred q;\n\t.reg .b64 m;\n\t"
      "and.b64 m, %1, 0x7FFFFFFFFFFFFFFF;\n\t"
      "setp.lt.u64 q, m, %2;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "l"(__double_as_longlong(v)), "l"(__double_as_longlong(eps)));
  return r != 0u;
}

// -v when flip is 1, else v: the sign bit flipped by an integer xor (the
// same bits as a multiply by -1.0).
__device__ __forceinline__ double neg_if(double v, int flip) {
  unsigned int hi;
  asm("xor.b32 %0, %1, %2;" : "=r"(hi) : "r"(__double2hiint(v)), "r"((unsigned int)(flip & 1) << 31));
  return __hiloint2double((int)hi, __double2loint(v));
}

// v != 0.0 (either zero) on the bit pattern.
__device__ __forceinline__ bool nonzero(double v) {
  unsigned int r;
  asm("{\n\t.reg .b32 h;\n\tand.b32 h, %1, 0x7FFFFFFF;\n\tor.b32 %0, h, %2;\n\t}"
      : "=r"(r)
      : "r"(__double2hiint(v)), "r"(__double2loint(v)));
  return r != 0u;
}

// Per-thread counts of one launch (32 bits: a thread handles far fewer than
// 2^32 entries per launch; blocks sum them in 64 bits).
struct StepCounts {
  unsigned int rot = 0, cre = 0, dnew = 0, dold = 0;
  int dead_delta = 0;
  double dS = 0.0;  // change of the Eq. 6 entropy (when recorded)
};

// The Eq. 6 summand -|c|^2 ln|c|^2 (zero at c = 0).
__device__ __forceinline__ double entropy_term(double c) {
  const double p = c * c;
  return p > 0.0 ? -p * log(p) : 0.0;
}

template <class KT>
__device__ __forceinline__ void record_kill(const TableT<KT>& t, const TapeT<KT>& tape, KT key, double val,
                                            unsigned int born) {
  unsigned long long ti = aggregated_add(&t.cnt->tape_n);
  if (ti < tape.cap) {
    TapeRecT<KT>& rec = tape_at(tape, ti);
    rec.key = key;
    rec.val = val;
    rec.born = born;
  } else {
    raise_error(t.cnt, ERR_TAPE_FULL);
  }
}

// One stored entry i of a factor step U_k (Eq. 3 with the eps rule).  Each
// linked pair (E, D = tau E) is rotated exactly once: by the thread of E when
// E is stored and live at the start of the step, otherwise by the thread of D.
// Entries dropped during this step carry this step's stamp, so a D-thread can
// tell "E was live when the step began" (live or DEAD_NOW) from "E absent"
// (ABSENT or DEAD_OLD).  Every lane of the warp calls this (findG votes across
// lanes); in_range is false for lanes past the end of the table.
// The rotation, creation and eps rule for one linked entry i (key X, live
// amplitude cX, ex = X is the excited member) whose partner lookup is r.
// Append a created entry without hashing it: within a factor step no thread
// looks a created key up (its only partner is the creating entry), so the
// slot is claimed after the step (link_appended) and the claim's round trip
// stays off the step's critical path.
template <class KT>
__device__ __forceinline__ void append_unlinked(const TableT<KT>& t, KT key, double amp, unsigned int born,
                                                bool with_born) {
  const unsigned long long idx = aggregated_add(&t.cnt->n_tail);
  if (idx >= t.cap_n) {
    raise_error(t.cnt, ERR_CAPACITY);
    return;
  }
  t.keys[idx] = key;
  t.amps[idx] = amp;
  if (with_born) t.born[idx] = born;
}

// Give appended entry idx its hash slot unless its key already has one (a
// revived key, whose slot the step repointed).
template <class KT>
__device__ __forceinline__ void link_appended(const TableT<KT>& t, KT key, unsigned long long idx) {
  unsigned long long h = home_slot(t, key);
  for (int step = 0; step < MAX_PROBE; ++step) {
    const KT prev = key_cas(&t.slots[h].key, KeyOps<KT>::zero(), key);
    if (KeyOps<KT>::is_zero(prev)) {
      t.slots[h].idx = idx;
      filter_add(t, key);
      return;
    }
    if (prev == key) return;
    h = (h + 1) & t.slot_mask;
  }
  raise_error(t.cnt, ERR_PROBE_BOUND);
}

// link_appended from slot `start` on (the hash's probe sequence for key passes
// through start with every slot before it full).
template <class KT>
__device__ __forceinline__ void link_from_slot(const TableT<KT>& t, KT key, unsigned long long idx,
                                               unsigned long long start) {
  unsigned long long h = start & t.slot_mask;
  for (int step = 0; step < MAX_PROBE; ++step) {
    const KT prev = key_cas(&t.slots[h].key, KeyOps<KT>::zero(), key);
    if (KeyOps<KT>::is_zero(prev)) {
      t.slots[h].idx = idx;
      filter_add(t, key);
      return;
    }
    if (prev == key) return;
    h = (h + 1) & t.slot_mask;
  }
  raise_error(t.cnt, ERR_PROBE_BOUND);
}

// DEFER: created entries are appended unlinked (link_appended runs after the
// step); otherwise they are hashed at once.
template <bool RECORD, bool DEFER = false, class KT>
__device__ __forceinline__ void forward_resolve(const TableT<KT>& t, const FactorT<KT>& f, int k, double eps,
                                                unsigned int stamp, const TapeT<KT>& tape, unsigned long long i, KT X,
                                                double cX, bool ex, const Lookup& r, StepCounts& sc) {
  const KT Y = X ^ (f.occ | f.vir);
  const bool partner_live = (r.state == ALIVE);
  if (!ex && (partner_live || r.state == DEAD_NOW)) return;  // E's thread owns the pair
  if (ex && r.state == DEAD_NOW) {
    raise_consistency(t.cnt, SITE_PAIR_OWNER);
    return;
  }
  const KT E = ex ? X : Y;
  const int parity = (KeyOps<KT>::popc(E & f.pmask) + f.pconst) & 1;
  const double ss = neg_if(f.s, parity);  // s * sin(theta), exact
  const double cE = ex ? cX : 0.0;
  const double cD = ex ? (partner_live ? r.amp : 0.0) : cX;
  // c_E' = cos c_E - s sin c_D ;  c_D' = cos c_D + s sin c_E  (no contraction)
  double nE, nD;
  if (!partner_live) {
    // One member is +0.0: its two products are zeros, and adding or
    // subtracting a zero leaves a nonzero product unchanged, so two products
    // give the same bits as the full formula whenever both are nonzero.
    const double pa = __dmul_rn(f.c, cX), pb = __dmul_rn(ss, cX);
    if (nonzero(pa) && nonzero(pb)) {
      nE = ex ? pa : neg_if(pb, 1);
      nD = ex ? pb : pa;
    } else {
      nE = __dsub_rn(__dmul_rn(f.c, cE), __dmul_rn(ss, cD));
      nD = __dadd_rn(__dmul_rn(f.c, cD), __dmul_rn(ss, cE));
    }
  } else {
    nE = __dsub_rn(__dmul_rn(f.c, cE), __dmul_rn(ss, cD));
    nD = __dadd_rn(__dmul_rn(f.c, cD), __dmul_rn(ss, cE));
  }
  const double nX = ex ? nE : nD;
  const double nY = ex ? nD : nE;
  ++sc.rot;
  if (t.entropy) {
    // Eq. 6 changes only on the pair: new terms (zero if dropped) minus old.
    const double kX = below_eps(nX, eps) ? 0.0 : nX;
    const double kY = below_eps(nY, eps) ? 0.0 : nY;
    sc.dS += entropy_term(kX) + entropy_term(kY) - entropy_term(cX) - (partner_live ? entropy_term(r.amp) : 0.0);
  }
  // The thread's own entry.
  if (below_eps(nX, eps)) {
    if (RECORD) record_kill(t, tape, X, nX, t.born[i]);
    t.amps[i] = dead_value(stamp);
    ++sc.dold;
    ++sc.dead_delta;
  } else {
    t.amps[i] = nX;
  }
  // The partner.
  if (partner_live) {
    if (below_eps(nY, eps)) {
      if (RECORD) record_kill(t, tape, Y, nY, t.born[r.idx]);
      t.amps[r.idx] = dead_value(stamp);
      ++sc.dold;
      ++sc.dead_delta;
    } else {
      t.amps[r.idx] = nY;
    }
  } else if (below_eps(nY, eps)) {
    ++sc.dnew;
  } else if (r.state == DEAD_OLD) {
    // Revive a dropped key as a fresh entry past the scan range and point
    // its slot there.  (Reviving in place would let the old index's scan
    // thread, if it runs later in this step, see a live entry that was
    // not live when the step began and rotate the pair a second time.)
    const unsigned long long idx = aggregated_add(&t.cnt->n_tail);
    if (idx < t.cap_n) {
      t.keys[idx] = Y;
      t.amps[idx] = nY;
      if (RECORD) t.born[idx] = (unsigned int)k;
      t.slots[r.slot].idx = idx;
    } else {
      raise_error(t.cnt, ERR_CAPACITY);
    }
    ++sc.cre;
  } else {
    if (DEFER)
      append_unlinked(t, Y, nY, (unsigned int)k, RECORD);
    else
      insert_new(t, Y, nY, (unsigned int)k, r.slot, RECORD, false, SITE_CREATE_DUP);
    ++sc.cre;
  }
}

// Scan half of a factor step: whether stored entry i (in_range false past the
// end of the table) is a live member of one of the factor's linked pairs.  X
// is its key, cX its amplitude, ex whether it is the excited member E.
template <class KT>
__device__ __forceinline__ bool linked_entry(const TableT<KT>& t, const FactorT<KT>& f, unsigned long long i,
                                             bool in_range, KT& X, double& cX, bool& ex) {
  X = KeyOps<KT>::zero();
  cX = 0.0;
  ex = false;
  if (!in_range) return false;
  X = t.keys[i];
  const KT tX = X & (f.occ | f.vir);  // occ and vir are disjoint
  ex = tX == f.occ;
  if (!(ex || tX == f.vir)) return false;
  cX = t.amps[i];
  return !is_dead(cX);
}

template <int G, bool RECORD, class KT>
__device__ __forceinline__ void forward_entry(const TableT<KT>& t, const FactorT<KT>& f, int k, double eps,
                                              unsigned int stamp, const TapeT<KT>& tape, unsigned long long i,
                                              bool in_range, StepCounts& sc) {
  KT X;
  double cX;
  bool ex;
  const bool act = linked_entry(t, f, i, in_range, X, cX, ex);
  Lookup r = findG<G>(t, X ^ (f.occ | f.vir), act, stamp);
  if (!act) return;
  forward_resolve<RECORD>(t, f, k, eps, stamp, tape, i, X, cX, ex, r, sc);
}

// One stored entry i of the reverse step for factor k: psi_k -> psi_{k-1} in
// place (inverse rotation on a stored pair, cos(theta) divided out of a lone
// member), lambda_{k-1} = U_k^T mu_k, and this pair's share of
// dE/dtheta_k / 2 = sum_pairs s (lam_D psi_E - lam_E psi_D) added to acc.
// Entries created by factor k (born == k) leave the table.  Every lane of the
// warp calls this.
// The reverse step for one linked entry i (key X, live amplitude cX, ex = X
// is the excited member) whose partner lookup is r.
template <class KT>
__device__ __forceinline__ void reverse_resolve(const TableT<KT>& t, const FactorT<KT>& f, int k, unsigned int stamp,
                                                unsigned long long i, KT X, double cX, double muX, bool ex,
                                                const Lookup& r, double& acc, unsigned int& pairs,
                                                unsigned int& kills) {
  const KT Y = X ^ (f.occ | f.vir);
  const bool partner_live = (r.state == ALIVE);
  if (!ex && (partner_live || r.state == DEAD_NOW)) return;  // E's thread owns the pair
  const KT E = ex ? X : Y;
  const int parity = (KeyOps<KT>::popc(E & f.pmask) + f.pconst) & 1;
  const double ss = neg_if(f.s, parity);
  ++pairs;
  if (partner_live) {
    // Both members stored: (e, d) = U^T (e', d'), (lamE, lamD) = U^T (muE, muD).
    // The reverse sweep feeds only the gradient (no eps decision rests on
    // it), so it contracts to fused multiply-adds: fewer FP64 instructions,
    // and each result rounded once.
    const double e1 = cX, d1 = r.amp;
    const double muE = muX, muD = t.lam[r.idx];
    const double e0 = fma(f.c, e1, ss * d1);
    const double d0 = fma(f.c, d1, -(ss * e1));
    const double lE = fma(f.c, muE, ss * muD);
    const double lD = fma(f.c, muD, -(ss * muE));
    // acc += s (lam_D psi_E - lam_E psi_D)
    acc = fma(neg_if(lD, parity), e0, acc);
    acc = fma(neg_if(lE, parity ^ 1), d0, acc);
    if (t.born[i] == (unsigned int)k) {
      t.amps[i] = dead_value(stamp);
      ++kills;
    } else {
      t.amps[i] = e0;
      t.lam[i] = lE;
    }
    if (t.born[r.idx] == (unsigned int)k) {
      t.amps[r.idx] = dead_value(stamp);
      ++kills;
    } else {
      t.amps[r.idx] = d0;
      t.lam[r.idx] = lD;
    }
  } else {
    // X alone: its partner was absent before the factor (and is not stored
    // after it), so c_X' = cos c_X.  For X = E the partner's adjoint is
    // lam_D = -s mu_E and the term s lam_D psi_E; for X = D it is
    // lam_E = s mu_D and the term -s lam_E psi_D: both are -s (ss mu_X) psi_X.
    const double x0 = __dmul_rn(cX, f.ic);
    acc = fma(neg_if(__dmul_rn(ss, muX), parity ^ 1), x0, acc);
    t.amps[i] = x0;
    t.lam[i] = __dmul_rn(f.c, muX);
  }
}

template <int G, class KT>
__device__ __forceinline__ void reverse_entry(const TableT<KT>& t, const FactorT<KT>& f, int k, unsigned int stamp,
                                              unsigned long long i, bool in_range, double& acc, unsigned int& pairs,
                                              unsigned int& kills) {
  KT X;
  double cX;
  bool ex;
  const bool act = linked_entry(t, f, i, in_range, X, cX, ex);
  Lookup r = findG<G>(t, X ^ (f.occ | f.vir), act, stamp);
  if (!act) return;
  reverse_resolve(t, f, k, stamp, i, X, cX, t.lam[i], ex, r, acc, pairs, kills);
}

// Per-warp queues of linked entries in shared memory.  Only a fraction of
// the stored determinants belong to a given factor's pairs, and for most of
// those the existence filter proves the partner absent.  A warp that resolved
// its 32 scanned entries in place would run the pair arithmetic (on the narrow
// FP64 pipe, where a warp instruction costs the same with one lane as with 32)
// and the partner probes on mostly idle lanes, and every lane would wait for
// the slowest lane's probe chain.  Instead the lanes append the linked entries
// they find to a queue; each 32 taken from it test their partners' filter
// bits together, the lanes whose partner is proved absent resolve at once
// (no slot probe), and the rest move to a probe queue that is resolved, slot
// probe first, 32 at a time.  The order in which a step's pairs are resolved
// does not matter: ownership and the dropped-entry stamps decide everything
// from the state at the start of the step.
//
// The keys and amplitudes of a warp's next round of kScanTiles tiles (and,
// with AUX, a third per-entry array: the adjoint in the reverse sweep) are
// copied into shared memory (cp.async, two buffers per warp) while it works on
// the current one, so the scan's load latency overlaps the pair work and a
// linked entry's own values never need a load of their own.
constexpr int kScanTiles = 2;
constexpr int kRound = 32 * kScanTiles;
constexpr int kQueue = 64;
// Queue entries keep the entry index in 31 bits and the excited-member flag in
// the top bit: the host keeps every table below kMaxEntries entries.
constexpr unsigned int kExBit = 1u << 31;
static_assert(kMaxEntries <= (1ull << 31), "queue indices are 31-bit");

template <class KT, bool AUX>
struct LinkQueueT {
  unsigned int i[kQueue];  // entry index, kExBit set for the excited member
  KT X[kQueue];
  double c[kQueue];
  double m[AUX ? kQueue : 1];
};

template <class KT, bool AUX>
struct __align__(16) ScanStageT {
  KT X[kRound];
  double c[kRound];
  double m[AUX ? kRound : 2];
};

// Per-warp shared memory of for_each_linked.
template <class KT, bool AUX>
struct LinkScratchT {
  ScanStageT<KT, AUX> stage[2];
  LinkQueueT<KT, AUX> linked;  // linked entries, before the filter test
  LinkQueueT<KT, AUX> probe;   // linked entries whose partner may be stored
};
template <class KT>
using LinkScratch = LinkScratchT<KT, false>;

// Threads per block of the kernels built on for_each_linked: with four warps
// per block, the eight blocks an SM holds at 64 registers per thread also fit
// its shared memory with their LinkScratch.
constexpr int kStepThreads = 128;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_last() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// The staged scan copies 16-byte pieces starting at even entries, so keys and
// amps (and lam) must start on a 16-byte boundary (device allocations do).
template <class KT>
inline bool scan_aligned(const TableT<KT>& t) {
  return ((reinterpret_cast<uintptr_t>(t.keys) | reinterpret_cast<uintptr_t>(t.amps) |
           reinterpret_cast<uintptr_t>(t.lam)) & 15u) == 0u;
}

// Copy entries [base, min(base + kRound, n)) of keys and amps (and aux) into a
// stage: 16-byte pieces of two entries (of one entry for two-word keys); the
// piece holding entry n - 1 alone copies 8 bytes (the rest zero-filled) and
// pieces past n are not issued.
template <class KT, bool AUX>
__device__ __forceinline__ void stage_round(const TableT<KT>& t, const double* aux, ScanStageT<KT, AUX>& st,
                                            unsigned long long base, unsigned long long n, unsigned int lane) {
#pragma unroll
  for (int h = 0; h < kRound / 64; ++h) {
    const int e = 2 * (int)(lane + 32u * h);  // first entry of the piece, relative to base
    const unsigned long long g = base + (unsigned long long)e;
    if (g < n) {
      const int bytes = g + 1ull < n ? 16 : 8;
      if (sizeof(KT) == 8) cp_async16(&st.X[e], t.keys + g, bytes);
      cp_async16(&st.c[e], t.amps + g, bytes);
      if (AUX) cp_async16(&st.m[e], aux + g, bytes);
    }
  }
  if (sizeof(KT) == 16) {
#pragma unroll
    for (int h = 0; h < kRound / 32; ++h) {
      const int e = (int)(lane + 32u * h);
      const unsigned long long g = base + (unsigned long long)e;
      if (g < n) cp_async16(&st.X[e], t.keys + g, 16);
    }
  }
}

// A lookup result for a key the existence filter proved absent.
__device__ __forceinline__ Lookup absent_lookup() {
  Lookup r;
  r.state = ABSENT;
  r.slot = 0ull;
  r.idx = 0ull;
  r.amp = 0.0;
  return r;
}

// Append (i, X, c, ex, m) of the active lanes (ballot mk) to queue q at qn.
template <class KT, bool AUX>
__device__ __forceinline__ void enqueue(LinkQueueT<KT, AUX>& q, int qn, unsigned int mk, unsigned int below_me,
                                        bool act, unsigned long long i, KT X, double c, bool ex, double m) {
  if (act) {
    const int p = qn + __popc(mk & below_me);
    q.i[p] = (unsigned int)i | (ex ? kExBit : 0u);
    q.X[p] = X;
    q.c[p] = c;
    if (AUX) q.m[p] = m;
  }
}

// Pop the last 32 entries of a queue holding qn >= 32 into the lanes and call
// f(i, X, c, ex, m, true).
template <class KT, bool AUX, class F>
__device__ __forceinline__ void drain32(LinkQueueT<KT, AUX>& q, int& qn, unsigned int lane, F& f) {
  __syncwarp();
  const int p = qn - 32 + (int)lane;
  const unsigned int qi = q.i[p];
  const KT qX = q.X[p];
  const double qc = q.c[p];
  const double qm = AUX ? q.m[p] : 0.0;
  __syncwarp();
  qn -= 32;
  f((unsigned long long)(qi & ~kExBit), qX, qc, (qi & kExBit) != 0u, qm, true);
}

// The qn < 32 entries left in a queue (lanes past qn inactive); empties it.
template <class KT, bool AUX, class F>
__device__ __forceinline__ void drain_rest(LinkQueueT<KT, AUX>& q, int& qn, unsigned int lane, F& f) {
  __syncwarp();
  const bool a = (int)lane < qn;
  unsigned int qi = 0u;
  KT qX = KeyOps<KT>::zero();
  double qc = 0.0, qm = 0.0;
  if (a) {
    qi = q.i[lane];
    qX = q.X[lane];
    qc = q.c[lane];
    if (AUX) qm = q.m[lane];
  }
  __syncwarp();
  qn = 0;
  f((unsigned long long)(qi & ~kExBit), qX, qc, (qi & kExBit) != 0u, qm, a);
}

// Scan entries [0, n) in warp-strided rounds of kRound entries and resolve
// every live linked entry: lone(i, X, cX, ex, m, active) when the filter
// proves its partner absent, probe(i, X, cX, ex, m, active) otherwise, where m
// is the entry's value in aux (AUX: staged with the scan) or, without AUX,
// pre(i, active) for lone entries (loaded together with the filter word, so a
// lone entry waits for a single round trip) and 0 for probed ones.  Every lane
// of the warp calls this; lone and probe are called by all lanes together.
// hint(i) is called for each live linked entry i when it is queued (a
// prefetch of what its resolution will load).
template <bool AUX, class KT, class Pre, class Lone, class Probe, class Hint>
__device__ __forceinline__ void for_each_linked(const TableT<KT>& t, const FactorT<KT>& f, unsigned long long n,
                                                LinkScratchT<KT, AUX>& w, const double* aux, Pre pre, Lone lone,
                                                Probe probe, Hint hint) {
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int below_me = (1u << lane) - 1u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long step = nwarps * (unsigned long long)kRound;
  const KT m = f.occ | f.vir;
  int nl = 0, np = 0;  // warp-uniform lengths of the linked and probe queues
  // Up to 32 linked entries: the partner's filter bit sends each lane to lone
  // at once or onto the probe queue.
  auto split = [&](unsigned long long i, KT X, double c, bool ex, double mu, bool act) {
    if (!AUX) mu = pre(i, act);
    bool maybe = act;
    if (act && t.filt) {
      const unsigned long long h = KeyOps<KT>::filt_hash(X ^ m);
      maybe = filter_hit(t, t.filt[filter_word(t, h)], h);
    }
    const bool pr = act && maybe;
    const unsigned int mp = __ballot_sync(0xFFFFFFFFu, pr);
    enqueue<KT, AUX>(w.probe, np, mp, below_me, pr, i, X, c, ex, mu);
    np += __popc(mp);
    lone(i, X, c, ex, mu, act && !maybe);
    if (np >= 32) drain32<KT, AUX>(w.probe, np, lane, probe);
  };
  unsigned long long base = warp * (unsigned long long)kRound;
  if (base < n) stage_round<KT, AUX>(t, aux, w.stage[0], base, n, lane);
  cp_async_commit();
  for (int r = 0; base < n; base += step, ++r) {
    // Next round's copy into the other buffer (its last reader was round r - 1).
    if (base + step < n) stage_round<KT, AUX>(t, aux, w.stage[(r + 1) & 1], base + step, n, lane);
    cp_async_commit();
    cp_async_wait_all_but_last();  // this round's copy has landed (this lane's pieces)
    __syncwarp();                  // ... and every other lane's
    const ScanStageT<KT, AUX>& st = w.stage[r & 1];
    // Not unrolled: the body inlines the resolve paths (instruction cache).
#pragma unroll 1
    for (int u = 0; u < kScanTiles; ++u) {
      const int e = 32 * u + (int)lane;
      const unsigned long long i = base + (unsigned long long)e;
      bool act = false, ex = false;
      KT X = KeyOps<KT>::zero();
      double cX = 0.0, mu = 0.0;
      if (i < n) {
        X = st.X[e];
        // occ and vir are disjoint: E holds exactly occ of the factor's
        // orbitals, D exactly vir
        const KT tX = X & m;
        ex = tX == f.occ;
        if (ex || tX == f.vir) {
          cX = st.c[e];
          act = !is_dead(cX);
          if (AUX) mu = st.m[e];
        }
      }
      const unsigned int ml = __ballot_sync(0xFFFFFFFFu, act);
      if (act) hint(i);
      enqueue<KT, AUX>(w.linked, nl, ml, below_me, act, i, X, cX, ex, mu);
      nl += __popc(ml);
      if (nl >= 32) drain32<KT, AUX>(w.linked, nl, lane, split);
    }
    __syncwarp();  // every lane is done with this buffer before it is refilled
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // nothing left in flight
  if (nl > 0) drain_rest<KT, AUX>(w.linked, nl, lane, split);
  if (np > 0) drain_rest<KT, AUX>(w.probe, np, lane, probe);
}

template <bool AUX, class KT, class Pre, class Lone, class Probe>
__device__ __forceinline__ void for_each_linked(const TableT<KT>& t, const FactorT<KT>& f, unsigned long long n,
                                                LinkScratchT<KT, AUX>& w, const double* aux, Pre pre, Lone lone,
                                                Probe probe) {
  for_each_linked<AUX>(t, f, n, w, aux, pre, lone, probe, [](unsigned long long) {});
}

// Bring the line holding p into L2 (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// (ab|cd) in chemist notation over spatial orbitals.
__device__ __forceinline__ double chem(const Integrals& in, int a, int b, int c, int d) {
  const int n = in.n;
  return __ldg(&in.g[((a * n + b) * n + c) * n + d]);
}

// <rs||pq> over spin-orbitals.
__device__ __forceinline__ double anti(const Integrals& in, int r, int s, int p, int q) {
  double v = 0.0;
  if (((r ^ p) & 1) == 0 && ((s ^ q) & 1) == 0) v += chem(in, r >> 1, p >> 1, s >> 1, q >> 1);
  if (((r ^ q) & 1) == 0 && ((s ^ p) & 1) == 0) v -= chem(in, r >> 1, q >> 1, s >> 1, p >> 1);
  return v;
}

__device__ __forceinline__ double h_so(const Integrals& in, int p, int q) {
  if ((p ^ q) & 1) return 0.0;
  return __ldg(&in.h[(p >> 1) * in.n + (q >> 1)]);
}

// Sign of a+_r a+_s a_q a_p |I> (p, q occupied; r, s empty; all distinct).
template <class KT>
__device__ __forceinline__ int double_parity(KT I, int p, int q, int r, int s) {
  using K = KeyOps<KT>;
  const KT msk = K::below(p) ^ K::below(q) ^ K::below(r) ^ K::below(s);
  return (K::popc(I & msk) + (p < q) + (p < s) + (q < s) + (p < r) + (q < r) + (s < r)) & 1;
}

// Sign of a+_r a_p |I>.
template <class KT>
__device__ __forceinline__ int single_parity(KT I, int p, int r) {
  using K = KeyOps<KT>;
  return (K::popc(I & (K::below(p) ^ K::below(r))) + (p < r)) & 1;
}

// Connections a lane tests per round of the energy pass (filter words in flight).
constexpr int kV = 2;

// Slot probe for a key the filter did not exclude: whether it is stored and
// live, with its amplitude and entry index.
template <class KT>
__device__ __forceinline__ bool probe_live_at(const TableT<KT>& t, KT key, double* amp, unsigned long long* idx) {
  unsigned long long h = home_slot(t, key);
  for (int step = 0; step < MAX_PROBE; ++step) {
    const SlotT<KT> s = t.slots[h];
    if (s.key == key) {
      const double a = t.amps[s.idx];
      if (is_dead(a)) return false;
      *amp = a;
      *idx = s.idx;
      return true;
    }
    if (KeyOps<KT>::is_zero(s.key)) return false;
    h = (h + 1) & t.slot_mask;
  }
  raise_error(t.cnt, ERR_PROBE_BOUND);
  return false;
}

// Per-warp lists of one determinant I for the lower-triangle sigma; NS =
// spin-orbitals of one spin a key holds.  Spin-orbital p has spin p & 1.
template <class KT>
struct LowerLists {
  static constexpr int NS = KeyOps<KT>::kBits / 2;
  static constexpr int kPairs = NS * (NS - 1) / 2;
  unsigned char occ[2][NS];
  unsigned char emp[2][NS];
  int n_occ[2], n_emp[2];
  unsigned short pairs[2][kPairs];      // same-spin empty pairs (r | s << 8), r < s, ordered by s
  unsigned short opp[NS * NS];          // (r alpha | s beta << 8), ordered by max(r, s)
  KT hitJ[32 * (kV + 1)];               // connections whose filter word holds all their bits
  unsigned int hitCode[32 * (kV + 1)];  // and their excitation (connection_code)
  unsigned long long mulBit[2 * NS];    // filter-hash term of spin-orbital x
};

// An excitation of I packed in 30 bits: kind (0 single p -> r, 1 double
// p, q -> r, s) and the four spin-orbital indices, 7 bits each.
__device__ __forceinline__ unsigned int connection_code(int kind, int p, int q, int r, int s) {
  return (unsigned int)kind | ((unsigned int)p << 2) | ((unsigned int)q << 9) | ((unsigned int)r << 16) |
         ((unsigned int)s << 23);
}

// The connections J < I of the lower-triangle energy pass, with the warp in
// lock step (count is warp-uniform): the lanes test kV filter words each and
// queue the connections whose word holds all their bits (hash_of(u) gives
// J's filter hash, key_of(u) J itself, code_of(u) its excitation); whenever
// 32 or more are queued after a round, resolve_hits takes them 32 at a time,
// so the slot probes of rare hits run on full warps instead of stalling the
// loop once per hit.  The queue holds fewer than 32 between rounds.
template <class KT, class HashOf, class KeyOf, class CodeOf, class Resolve>
__device__ __forceinline__ void probe_lower(const TableT<KT>& t, LowerLists<KT>& L, int& qn, int count, int lane,
                                            HashOf hash_of, KeyOf key_of, CodeOf code_of, Resolve resolve_hits,
                                            unsigned long long& probes) {
  const unsigned int below_me = (1u << lane) - 1u;
  for (int u0 = 0; u0 < count; u0 += 32 * kV) {
    bool w[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const int u = u0 + 32 * v + lane;
      w[v] = false;
      if (u < count) {
        ++probes;
        if (t.filt) {
          const unsigned long long h = hash_of(u);
          w[v] = filter_hit(t, t.filt[filter_word(t, h)], h);
        } else {
          w[v] = true;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) {
      const int u = u0 + 32 * v + lane;
      const unsigned int m = __ballot_sync(0xFFFFFFFFu, w[v]);
      if (w[v]) {
        const int p = qn + __popc(m & below_me);
        L.hitJ[p] = key_of(u);
        L.hitCode[p] = code_of(u);
      }
      qn += __popc(m);
    }
    while (qn >= 32) resolve_hits(32);
  }
}

// Lower-triangle sigma for one stored determinant I: the lane's share of
// sum_{J in S, J < I} <I|H|J> c_J (returned) and of the diagonal <I|H|I>
// (in diag), with every hit's transposed term sent to sigma_J.  Over all
// stored I this covers each connected stored pair once, from its larger key.
// J = I with holes P and particles Q set/cleared is below I exactly when the
// highest changed spin-orbital is a hole, max(P) > max(Q), so every list
// below is cut to a prefix by counting the empty orbitals under max(P): no
// connection J > I is generated.  Every lane of the warp calls this.
template <class KT>
__device__ __forceinline__ double sigma_lower(const TableT<KT>& t, const Integrals& in, LowerLists<KT>& L, KT I,
                                              double cI, int lane, double& diag, unsigned long long& probes,
                                              unsigned long long& hits) {
  using K = KeyOps<KT>;
  const KT alpha = K::alpha(), beta = ~K::alpha();
  const KT all = K::below(in.n_so);
  const KT emask = ~I & all;
  // empty spin-orbitals of spin sp below orbital m
  auto empty_below = [&](int sp, int m) { return K::popc(emask & (sp ? beta : alpha) & K::below(m)); };
  // Occupied and empty lists by spin, ascending: lanes over the orbitals, each
  // placed at the count of same-kind, same-spin orbitals below it.
  for (int p = lane; p < in.n_so; p += 32) {
    const int sp = p & 1;
    const KT spin = sp ? beta : alpha;
    if (K::test(I, p))
      L.occ[sp][K::popc(I & spin & K::below(p))] = (unsigned char)p;
    else
      L.emp[sp][K::popc(emask & spin & K::below(p))] = (unsigned char)p;
  }
  if (lane < 2) {
    const KT spin = lane ? beta : alpha;
    L.n_occ[lane] = K::popc(I & all & spin);
    L.n_emp[lane] = K::popc(emask & spin);
  }
  __syncwarp();
  for (int sp = 0; sp < 2; ++sp) {
    const int m = L.n_emp[sp];
    const int np = m * (m - 1) / 2;
    for (int u = lane; u < np; u += 32) {
      // u -> (x, y), x < y, column by column: u = y (y - 1) / 2 + x
      int y = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)u)) * 0.5f);
      while (y * (y - 1) / 2 > u) --y;
      while ((y + 1) * y / 2 <= u) ++y;
      const int x = u - y * (y - 1) / 2;
      L.pairs[sp][u] = (unsigned short)(L.emp[sp][x] | (L.emp[sp][y] << 8));
    }
  }
  // Filter-hash terms: J = (I with the holes cleared) + 2^r + 2^s exactly (the
  // particles are empty in I), so hash(J) = base + mulBit[r] + mulBit[s]
  // modulo 2^64, with one base per hole set.
  for (int x = lane; x < 2 * LowerLists<KT>::NS; x += 32) L.mulBit[x] = K::filt_bit(x);
  // Opposite-spin empty pairs grouped by their larger orbital o: the pairs
  // with max < o number (alpha empties below o) * (beta empties below o).
  for (int o = lane; o < in.n_so; o += 32) {
    if (!K::test(emask, o)) continue;
    const int ra = empty_below(0, o), sb = empty_below(1, o);
    const int st = ra * sb;
    if ((o & 1) == 0) {
      for (int j = 0; j < sb; ++j) L.opp[st + j] = (unsigned short)(o | (L.emp[1][j] << 8));
    } else {
      for (int j = 0; j < ra; ++j) L.opp[st + j] = (unsigned short)(L.emp[0][j] | (o << 8));
    }
  }
  __syncwarp();

  // Diagonal: lanes over the first index p.
  double d = 0.0;
  for (int sp = 0; sp < 2; ++sp)
    for (int x = lane; x < L.n_occ[sp]; x += 32) {
      const int p = L.occ[sp][x];
      d += h_so(in, p, p);
      for (int sq = 0; sq < 2; ++sq)
        for (int y = 0; y < L.n_occ[sq]; ++y) {
          const int q = L.occ[sq][y];
          if (q != p) d += 0.5 * anti(in, p, q, p, q);
        }
    }
  diag = d;

  double part = 0.0;
  int qn = 0;  // warp-uniform length of the hit queue
  // <J|H|I> for the queued excitation code of J = tau I.
  auto elem = [&](unsigned int code) {
    const int p = (code >> 2) & 127, q = (code >> 9) & 127, r = (code >> 16) & 127, s = (code >> 23) & 127;
    if ((code & 3u) == 0u) {
      double v = h_so(in, r, p);
      for (int sk = 0; sk < 2; ++sk)
        for (int y = 0; y < L.n_occ[sk]; ++y) {
          const int kk = L.occ[sk][y];
          if (kk != p) v += anti(in, r, kk, p, kk);
        }
      return single_parity(I, p, r) ? -v : v;
    }
    const double v = anti(in, r, s, p, q);
    return double_parity(I, p, q, r, s) ? -v : v;
  };
  // The last `take` queued connections, one per lane: probe the slot array;
  // on a live hit add <I|H|J> c_J here and the transposed term to sigma_J.
  auto resolve_hits = [&](int take) {
    __syncwarp();
    const bool a = lane < take;
    const int pidx = qn - take + lane;
    const KT J = a ? L.hitJ[pidx] : K::zero();
    const unsigned int code = a ? L.hitCode[pidx] : 0u;
    __syncwarp();
    qn -= take;
    double cJ;
    unsigned long long j;
    if (a && probe_live_at(t, J, &cJ, &j)) {
      ++hits;
      const double h = elem(code);
      part += h * cJ;
      atomicAdd(&t.sigma[j], h * cI);
    }
  };
  // Singles p -> r, same spin, r < p.
  for (int sp = 0; sp < 2; ++sp)
    for (int x = 0; x < L.n_occ[sp]; ++x) {
      const int p = L.occ[sp][x];
      const unsigned long long base = K::filt_hash(I ^ K::bit(p));
      probe_lower(
          t, L, qn, empty_below(sp, p), lane, [&](int u) { return base + L.mulBit[L.emp[sp][u]]; },
          [&](int u) { return I ^ (K::bit(p) | K::bit(L.emp[sp][u])); },
          [&](int u) { return connection_code(0, p, 0, L.emp[sp][u], 0); }, resolve_hits, probes);
    }
  // Doubles, same spin: holes p < q, particles r < s < q.
  for (int sp = 0; sp < 2; ++sp) {
    const int no = L.n_occ[sp];
    for (int x = 0; x < no; ++x)
      for (int y = x + 1; y < no; ++y) {
        const int p = L.occ[sp][x], q = L.occ[sp][y];
        const KT hole = K::bit(p) | K::bit(q);
        const unsigned long long base = K::filt_hash(I ^ hole);
        const int y0 = empty_below(sp, q);
        probe_lower(
            t, L, qn, y0 * (y0 - 1) / 2, lane,
            [&](int u) {
              const unsigned short pr = L.pairs[sp][u];
              return base + L.mulBit[pr & 0xFF] + L.mulBit[pr >> 8];
            },
            [&](int u) {
              const unsigned short pr = L.pairs[sp][u];
              return I ^ (hole | K::bit(pr & 0xFF) | K::bit(pr >> 8));
            },
            [&](int u) {
              const unsigned short pr = L.pairs[sp][u];
              return connection_code(1, p, q, pr & 0xFF, pr >> 8);
            },
            resolve_hits, probes);
      }
  }
  // Doubles, opposite spin: holes p alpha, q beta; particles r alpha, s beta
  // both below max(p, q).
  for (int x = 0; x < L.n_occ[0]; ++x)
    for (int y = 0; y < L.n_occ[1]; ++y) {
      const int p = L.occ[0][x], q = L.occ[1][y];
      const int m = p > q ? p : q;
      const KT hole = K::bit(p) | K::bit(q);
      const unsigned long long base = K::filt_hash(I ^ hole);
      probe_lower(
          t, L, qn, empty_below(0, m) * empty_below(1, m), lane,
          [&](int u) {
            const unsigned short pr = L.opp[u];
            return base + L.mulBit[pr & 0xFF] + L.mulBit[pr >> 8];
          },
          [&](int u) {
            const unsigned short pr = L.opp[u];
            return I ^ (hole | K::bit(pr & 0xFF) | K::bit(pr >> 8));
          },
          [&](int u) {
            const unsigned short pr = L.opp[u];
            return connection_code(1, p, q, pr & 0xFF, pr >> 8);
          },
          resolve_hits, probes);
    }
  if (qn > 0) resolve_hits(qn);
  __syncwarp();  // the lists of I are read until here
  return part;
}


}  // namespace ucc
