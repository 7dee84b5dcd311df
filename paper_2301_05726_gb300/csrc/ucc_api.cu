// Host runtime behind include/ucc.h: validation, device buffers, capacity
// management and the launch sequences of apply / energy / gradient.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ucc.h"
#include "ucc_internal.h"

using namespace ucc;

namespace {

thread_local std::string g_last_error;

ucc_status fail(ucc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

}  // namespace

void ucc::set_last_error(const char* msg) { g_last_error = msg; }

namespace {

#define CUDA_TRY(expr)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? UCC_ENOMEM : UCC_ECUDA,                              \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                                   \
  } while (0)

#define UCC_TRY(expr)              \
  do {                             \
    ucc_status s_ = (expr);        \
    if (s_ != UCC_OK) return s_;   \
  } while (0)

template <class T>
ucc_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(UCC_ENOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  return UCC_OK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

unsigned long long next_pow2(unsigned long long x) {
  unsigned long long p = 1;
  while (p < x) p <<= 1;
  return p;
}

// One set of table arrays; a rebuild writes into a second set and swaps.
// Keys take kw 64-bit words each and slots kw 16-byte units (kw = 2 above 64
// spin-orbitals); the kernels see them through TableT<KT>.
struct Arrays {
  unsigned long long cap_n = 0, n_slots = 0;
  int kw = 1;
  unsigned long long* keys = nullptr;
  double* amps = nullptr;
  unsigned int* born = nullptr;
  double* lam = nullptr;
  double* sigma = nullptr;
  Slot* slots = nullptr;
  unsigned int* filt = nullptr;  // one 32-bit word per 4 slots
  bool slots_clean = false;      // the slot array is known to be all empty
  void release() {
    dfree(filt);
    dfree(keys);
    dfree(amps);
    dfree(born);
    dfree(lam);
    dfree(sigma);
    dfree(slots);
    cap_n = n_slots = 0;
    slots_clean = false;
  }
  ucc_status allocate(unsigned long long cn, unsigned long long ns) {
    release();
    UCC_TRY(dalloc(&keys, cn * kw));
    UCC_TRY(dalloc(&amps, cn));
    UCC_TRY(dalloc(&born, cn));
    UCC_TRY(dalloc(&lam, cn));
    UCC_TRY(dalloc(&sigma, cn));
    UCC_TRY(dalloc(&slots, ns * kw));
    UCC_TRY(dalloc(&filt, ns / 4));
    cap_n = cn;
    n_slots = ns;
    return UCC_OK;
  }
};

// A wavefunction table: entry arrays (current, and a spare for rebuilds) and
// its device counters with a pinned host mirror.
struct TableSet {
  Arrays cur, spare;
  Counters* d_cnt = nullptr;
  Counters* h_cnt = nullptr;
  // The spare's slot array and filter are cleared on a side stream right
  // after it is swapped out, overlapping the factor steps that follow; the
  // next rebuild waits for `clean` instead of clearing on the main stream.
  cudaEvent_t clean = nullptr;
  bool clean_pending = false;
  void release() {
    cur.release();
    spare.release();
    dfree(d_cnt);
    if (h_cnt) cudaFreeHost(h_cnt);
    h_cnt = nullptr;
    if (clean) cudaEventDestroy(clean);
    clean = nullptr;
    clean_pending = false;
  }
  ucc_status init() {
    if (cudaEventCreateWithFlags(&clean, cudaEventDisableTiming) != cudaSuccess) {
      clean = nullptr;
      return fail(UCC_ECUDA, "event creation failed");
    }
    UCC_TRY(dalloc(&d_cnt, 1));
    if (cudaMallocHost((void**)&h_cnt, sizeof(Counters)) != cudaSuccess) {
      h_cnt = nullptr;
      return fail(UCC_ENOMEM, "pinned host allocation failed");
    }
    std::memset(h_cnt, 0, sizeof(Counters));
    return UCC_OK;
  }
};

// psi (live keys and amplitudes) at the start of a gradient segment; keys of
// kw words each.
struct Snapshot {
  unsigned long long n = 0;
  unsigned long long* keys = nullptr;
  double* amps = nullptr;
  void release() {
    dfree(keys);
    dfree(amps);
    n = 0;
  }
};

}  // namespace

struct ucc_ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;   // clears spare hash arrays off the critical path
  int n_spatial = 0, n_alpha = 0, n_beta = 0, n_so = 0;
  double e_nuc = 0.0;
  int K = 0;
  std::vector<int> rows;         // K x 4
  std::vector<double> theta;     // K
  bool wide = false;             // more than 64 spin-orbitals: two-word keys
  int kw = 1;                    // key words
  std::vector<Factor> factors;   // host copy (one-word keys)
  std::vector<FactorT<Key128>> factors_w;  // host copy (two-word keys)
  ucc_options opt{};

  void* d_factors = nullptr;     // FactorT<KT>[K]
  double* d_h = nullptr;
  double* d_g = nullptr;
  double* d_grad = nullptr;
  double* d_partials = nullptr;
  int partial_cap = 0;
  // Bucketed energy: per-partition counts, fill counters and offsets, and the
  // record buffer (kept between evaluations).
  unsigned int* d_sb_cnt = nullptr;
  unsigned int* d_sb_fill = nullptr;
  unsigned long long* d_sb_off = nullptr;
  unsigned long long sb_parts = 0;
  unsigned char* d_sb_rec = nullptr;
  size_t sb_rec_cap = 0;  // bytes
  RehashScratch rs;       // hash builds by regions
  SelectState* d_sel = nullptr;
  void* d_cand = nullptr;  // SelectCandT<KT>[kSelectCandCap]: candidates of the cut's last selection passes
  double* d_entropy = nullptr;  // [K] Eq. 6 after each factor of the last apply
  bool entropy_on = false;
  bool have_entropy = false;
  TableSet ts[2];  // ts[main] holds psi; the other is the gradient's work table
  int main = 0;
  std::vector<Snapshot> snaps;
  // kill tape (paged) of the segment being reversed
  std::vector<void*> t_pages;
  void** d_pages = nullptr;             // [kTapeMaxPages] TapeRecT<KT> pages
  unsigned long long* t_off = nullptr;  // K + 1
  unsigned long long tape_cap = 0;
  unsigned long long tape_budget = 0;   // bytes the tape may take in this call
  bool tape_over_budget = false;
  bool force_segments = false;

  bool have_psi = false;
  bool have_sigma = false;
  cudaEvent_t ev[6] = {};
  cudaEvent_t kev[2] = {};  // around each chunk of factor launches
  // Event pairs around cuts and rebuilds, read without waiting for them: the
  // elapsed times are added to their totals when a pass ends (or the pool
  // is full), so timing a cut costs the host no round trip.
  std::vector<cudaEvent_t> tev;  // two per pair
  std::vector<double*> tev_acc;  // the total each recorded pair adds to
  size_t tev_used = 0;           // pairs recorded since the last flush
  ucc_stats stats{};
  int probe_width = 1;
  long long launches = 0;
  long long cut_total = 0;

  template <class KT>
  TableT<KT> table(const TableSet& s) const {
    TableT<KT> t;
    t.keys = reinterpret_cast<KT*>(s.cur.keys);
    t.amps = s.cur.amps;
    t.born = s.cur.born;
    t.lam = s.cur.lam;
    t.sigma = s.cur.sigma;
    t.slots = reinterpret_cast<SlotT<KT>*>(s.cur.slots);
    t.slot_mask = s.cur.n_slots - 1;
    t.slot_shift = 64 - __builtin_ctzll(s.cur.n_slots);
    t.filt = s.cur.filt;
    t.filt_shift = 32 - (__builtin_ctzll(s.cur.n_slots) - 2);
    t.cap_n = s.cur.cap_n;
    t.cnt = s.d_cnt;
    t.partials = d_partials;
    t.entropy = entropy_on ? d_entropy : nullptr;
    return t;
  }
  template <class KT>
  TapeT<KT> tape() const {
    TapeT<KT> tp;
    tp.pages = reinterpret_cast<TapeRecT<KT>* const*>(d_pages);
    tp.off = t_off;
    tp.cap = tape_cap;
    return tp;
  }
  template <class KT>
  FactorT<KT>* dfactors() const {
    return static_cast<FactorT<KT>*>(d_factors);
  }
  template <class KT>
  SelectCandT<KT>* dcand() const {
    return static_cast<SelectCandT<KT>*>(d_cand);
  }
  size_t tape_rec_bytes() const { return wide ? sizeof(TapeRecT<Key128>) : sizeof(TapeRec); }
  int full_grid(int per_sm = 8) const { return std::max(1, num_sms * per_sm); }
};

namespace {

// Jordan-Wigner sign mask of tau = a+_a a+_b a_j a_i acting on a determinant
// E that it excites: the four operators count occupied modes below i, j, b, a
// in the running determinant; relative to E those counts shift by the index
// comparisons below, so parity = popc(E & pmask) + pconst (mod 2).
template <class KT>
FactorT<KT> make_factor(int i, int j, int a, int b, double th) {
  using K = KeyOps<KT>;
  FactorT<KT> f{};
  if (j < 0) {
    f.occ = K::bit(i);
    f.vir = K::bit(a);
    f.pmask = K::below(i) ^ K::below(a);
    f.pconst = (i < a) ? 1 : 0;
    f.is_double = 0;
  } else {
    f.occ = K::bit(i) | K::bit(j);
    f.vir = K::bit(a) | K::bit(b);
    f.pmask = K::below(i) ^ K::below(j) ^ K::below(a) ^ K::below(b);
    f.pconst = ((i < j) + (i < b) + (j < b) + (i < a) + (j < a) + (b < a)) & 1;
    f.is_double = 1;
  }
  f.c = std::cos(th);
  f.s = std::sin(th);
  f.ic = 1.0 / f.c;
  return f;
}

ucc_status check_device_error(const Counters& h) {
  int err = h.error;
  if (!err) return UCC_OK;
  std::string msg = "device error word:";
  if (err & ERR_PROBE_BOUND) msg += " probe-bound";
  if (err & ERR_CONSISTENCY)
    msg += " consistency (site " + std::to_string(h.err_site) + ", key " + std::to_string(h.err_key) + ")";
  if (err & ERR_TAPE_FULL) msg += " tape-full";
  if (err & ERR_CAPACITY) msg += " capacity";
  return fail((err & (ERR_CAPACITY | ERR_TAPE_FULL)) ? UCC_ECAPACITY : UCC_ECUDA, msg);
}

ucc_status read_counters(ucc_ctx* c, TableSet& s) {
  CUDA_TRY(cudaMemcpyAsync(s.h_cnt, s.d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return check_device_error(*s.h_cnt);
}

ucc_status ensure_partials(ucc_ctx* c, int grid) {
  if (grid * 2 <= c->partial_cap) return UCC_OK;
  dfree(c->d_partials);
  UCC_TRY(dalloc(&c->d_partials, (size_t)grid * 2));
  c->partial_cap = grid * 2;
  return UCC_OK;
}

unsigned long long slots_for(unsigned long long cap_n) {
  // at most cap_n / 2 entries before a step, 2x that after: keep <= 75% full
  return next_pow2(std::max<unsigned long long>(64, (cap_n * 4 + 2) / 3));
}

// Whether a hash of n_slots slots receiving `entries` keys is built region by
// region: one-word keys, at least 2^20 slots, and the entries filling at least
// a quarter of the slots (a region build writes every slot, a direct rehash
// claims one random slot per entry; on the 64-so workload's 2^25-slot table
// with 6.25e6 entries after a cut the direct rehash is faster).  entries =
// ~0 when not known: direct.  The test option forces either way.
bool regions_ok(const ucc_ctx* c, unsigned long long n_slots, unsigned long long entries) {
  if (c->wide || c->opt.rebuild_test_regions == 1) return false;
  if (c->opt.rebuild_test_regions == 2) return n_slots >= (1ull << kRegionBits);
  return n_slots >= (1ull << 20) && entries != ~0ull && 4 * entries >= n_slots;
}

// Scratch of the region build for a table of cap entries and n_slots slots.
ucc_status ensure_rehash_scratch(ucc_ctx* c, unsigned long long cap, unsigned long long n_slots) {
  RehashScratch& r = c->rs;
  const unsigned long long regions = n_slots >> kRegionBits;
  if (r.regions < regions) {
    dfree(r.rcnt);
    dfree(r.rfill);
    dfree(r.roff);
    r.regions = 0;
    UCC_TRY(dalloc(&r.rcnt, regions));
    UCC_TRY(dalloc(&r.rfill, regions));
    UCC_TRY(dalloc(&r.roff, regions + 1));
    r.regions = regions;
  }
  if (!r.over_n) UCC_TRY(dalloc(&r.over_n, 1));
  if (r.cap < cap) {
    dfree(r.pairs);
    dfree(r.over);
    r.cap = 0;
    UCC_TRY(dalloc(&r.pairs, 2 * cap));
    UCC_TRY(dalloc(&r.over, 2 * cap));
    r.cap = cap;
  }
  return UCC_OK;
}

// The spare arrays of table s, sized for new_cap entries and cleared, as the
// target of a compaction; finish_rebuild hashes them and swaps them in.
template <class KT>
ucc_status prepare_spare(ucc_ctx* c, TableSet& s, unsigned long long new_cap, TableT<KT>* out) {
  if (new_cap >= kMaxEntries)
    return fail(UCC_ECAPACITY, "the wavefunction needs more than 2^31 stored entries (" + std::to_string(new_cap) +
                                   ")");
  unsigned long long ns = slots_for(new_cap);
  bool cleared = false;
  if (s.clean_pending) {
    // the side stream's clearing of these arrays must finish first (also when
    // they are released below: their memory may be handed out again)
    CUDA_TRY(cudaStreamWaitEvent(c->stream, s.clean, 0));
    s.clean_pending = false;
    cleared = true;
  }
  if (s.spare.cap_n != new_cap || s.spare.n_slots != ns) {
    s.spare.release();
    cleared = false;
    ucc_status st = s.spare.allocate(new_cap, ns);
    if (st != UCC_OK) {
      s.spare.release();
      return fail(UCC_ECAPACITY, "cannot allocate " + std::to_string(new_cap) + " entries: " + g_last_error);
    }
  }
  TableT<KT> to = c->template table<KT>(s);
  to.keys = reinterpret_cast<KT*>(s.spare.keys);
  to.amps = s.spare.amps;
  to.born = s.spare.born;
  to.lam = s.spare.lam;
  to.sigma = s.spare.sigma;
  to.slots = reinterpret_cast<SlotT<KT>*>(s.spare.slots);
  to.slot_mask = ns - 1;
  to.slot_shift = 64 - __builtin_ctzll(ns);
  to.filt = s.spare.filt;
  to.filt_shift = 32 - (__builtin_ctzll(ns) - 2);
  to.cap_n = new_cap;
  CUDA_TRY(cudaMemsetAsync(&s.d_cnt->new_n, 0, sizeof(unsigned long long), c->stream));
  if (!cleared) {
    CUDA_TRY(cudaMemsetAsync(to.slots, 0, ns * sizeof(SlotT<KT>), c->stream));
    CUDA_TRY(cudaMemsetAsync(to.filt, 0, ns / 4 * sizeof(unsigned int), c->stream));
    s.spare.slots_clean = true;
  }
  *out = to;
  return UCC_OK;
}

// After a swap: clear the arrays just swapped out (the new spare) on the side
// stream once the main stream has finished with them.
ucc_status clear_spare_async(ucc_ctx* c, TableSet& s) {
  if (!c->side || s.spare.cap_n == 0) return UCC_OK;
  CUDA_TRY(cudaEventRecord(s.clean, c->stream));
  CUDA_TRY(cudaStreamWaitEvent(c->side, s.clean, 0));
  CUDA_TRY(cudaMemsetAsync(s.spare.slots, 0, s.spare.n_slots * s.spare.kw * sizeof(Slot), c->side));
  s.spare.slots_clean = true;
  CUDA_TRY(cudaMemsetAsync(s.spare.filt, 0, s.spare.n_slots / 4 * sizeof(unsigned int), c->side));
  CUDA_TRY(cudaEventRecord(s.clean, c->side));
  s.clean_pending = true;
  return UCC_OK;
}

// Wait (on the main stream) for a pending side-stream clearing of the spare.
ucc_status settle_spare(ucc_ctx* c, TableSet& s) {
  if (!s.clean_pending) return UCC_OK;
  CUDA_TRY(cudaStreamWaitEvent(c->stream, s.clean, 0));
  s.clean_pending = false;
  return UCC_OK;
}

// Hash the compacted spare arrays `to` and make them the current ones.
template <class KT>
ucc_status finish_rebuild(ucc_ctx* c, TableSet& s, const TableT<KT>& to, unsigned long long expect = ~0ull,
                          unsigned long long entries = ~0ull) {
  const int grid = c->full_grid();
  const unsigned long long ns = to.slot_mask + 1ull;
  bool by_regions = false;
  if constexpr (sizeof(KT) == 8) {
    if (regions_ok(c, ns, entries)) {
      if (ensure_rehash_scratch(c, to.cap_n, ns) == UCC_OK) {
        CUDA_TRY(launch_rehash_regions(to, c->rs, grid, c->num_sms, c->stream));
        c->launches += 5;
        by_regions = true;
      } else {
        cudaGetLastError();  // a failed scratch allocation: the direct rehash below
      }
    }
  }
  if (!by_regions) {
    // the direct rehash claims slots in a cleared array
    if (!s.spare.slots_clean) CUDA_TRY(cudaMemsetAsync(to.slots, 0, ns * sizeof(SlotT<KT>), c->stream));
    CUDA_TRY(launch_rehash(to, grid, c->stream));
    c->launches++;
  }
  CUDA_TRY(launch_finish_rebuild(to, expect, c->stream));
  c->launches += 1;
  std::swap(s.cur, s.spare);
  s.cur.slots_clean = false;  // the live hash
  s.spare.slots_clean = false;  // the previous live hash, until cleared
  // After growth the old, smaller arrays are not reused: free them now.
  if (s.spare.cap_n != s.cur.cap_n)
    s.spare.release();
  else
    UCC_TRY(clear_spare_async(c, s));
  c->stats.rebuilds++;
  return UCC_OK;
}

// Copy live entries into arrays of capacity new_cap (dropping dead entries) and
// rebuild the hash.  Counters are updated on the device.
// Device time between the two events, added to *acc after the stream reaches
// the second one.
constexpr size_t kTimingPairs = 256;

// Stats are about to be reset: pairs a failed call left pending are dropped.
void drop_timings(ucc_ctx* c) {
  c->tev_used = 0;
  c->tev_acc.clear();
}

// Add the elapsed times of the recorded pairs to their totals (waits for the
// last one, which the stream reaches after all the others).
ucc_status flush_timings(ucc_ctx* c) {
  if (c->tev_used == 0) return UCC_OK;
  CUDA_TRY(cudaEventSynchronize(c->tev[2 * c->tev_used - 1]));
  for (size_t x = 0; x < c->tev_used; ++x) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->tev[2 * x], c->tev[2 * x + 1]));
    *c->tev_acc[x] += ms;
  }
  c->tev_used = 0;
  c->tev_acc.clear();
  return UCC_OK;
}

ucc_status timed_begin(ucc_ctx* c) {
  if (c->tev_used == kTimingPairs) UCC_TRY(flush_timings(c));
  while (c->tev.size() < 2 * (c->tev_used + 1)) {
    cudaEvent_t e = nullptr;
    CUDA_TRY(cudaEventCreate(&e));
    c->tev.push_back(e);
  }
  CUDA_TRY(cudaEventRecord(c->tev[2 * c->tev_used], c->stream));
  return UCC_OK;
}

ucc_status timed_end(ucc_ctx* c, double* acc) {
  CUDA_TRY(cudaEventRecord(c->tev[2 * c->tev_used + 1], c->stream));
  c->tev_acc.push_back(acc);
  ++c->tev_used;
  return UCC_OK;
}

// entries: the live entries the compaction keeps, when the host knows them.
template <class KT>
ucc_status rebuild(ucc_ctx* c, TableSet& s, unsigned long long new_cap, bool with_lam = false,
                   unsigned long long entries = ~0ull) {
  TableT<KT> to;
  UCC_TRY(timed_begin(c));
  UCC_TRY(prepare_spare(c, s, new_cap, &to));
  CUDA_TRY(launch_compact(c->template table<KT>(s), to, with_lam ? 2 : 1, c->full_grid(), c->stream));
  c->launches++;
  UCC_TRY(finish_rebuild(c, s, to, ~0ull, entries));
  return timed_end(c, &c->stats.rebuild_ms);
}

// The Methods-section cut after factor k: select the N_CUT-th entry, then one
// pass keeps the entries above it in the spare arrays (dropping the ε-dropped
// ones too) and records the cut ones on the tape, and the spare arrays are
// hashed and swapped in.
template <class KT>
ucc_status cut_rebuild(ucc_ctx* c, TableSet& s, bool record, int k) {
  const int grid = c->full_grid();
  UCC_TRY(timed_begin(c));
  CUDA_TRY(launch_select_threshold(c->template table<KT>(s), c->d_sel, c->template dcand<KT>(),
                                   (unsigned long long)c->opt.n_cut, grid, c->stream, &c->launches));
  TableT<KT> to;
  UCC_TRY(prepare_spare(c, s, s.cur.cap_n, &to));
  CUDA_TRY(launch_cut_compact(c->template table<KT>(s), to, c->d_sel, record ? 1 : 0, c->template tape<KT>(), k,
                              grid, c->stream));
  c->launches++;
  // the kept count must be N_CUT (checked on the device: no round trip here)
  UCC_TRY(finish_rebuild(c, s, to, (unsigned long long)c->opt.n_cut, (unsigned long long)c->opt.n_cut));
  return timed_end(c, &c->stats.cut_ms);
}

// Grow the paged tape to hold `need` records (pages are added, never moved).
// Past the call's budget it stops with tape_over_budget set; the gradient
// then falls back to segment checkpoints.
ucc_status ensure_tape(ucc_ctx* c, unsigned long long need) {
  while (c->tape_cap < need) {
    if ((int)c->t_pages.size() >= kTapeMaxPages) return fail(UCC_ECAPACITY, "kill tape page table full");
    const unsigned long long bytes = (c->tape_cap + kTapePageRecs) * c->tape_rec_bytes();
    if (c->tape_budget && bytes > c->tape_budget) {
      c->tape_over_budget = true;
      return fail(UCC_ECAPACITY, "kill tape over its memory budget");
    }
    unsigned char* page = nullptr;
    UCC_TRY(dalloc(&page, kTapePageRecs * c->tape_rec_bytes()));
    void* pv = page;
    CUDA_TRY(cudaMemcpyAsync(c->d_pages + c->t_pages.size(), &pv, sizeof(void*), cudaMemcpyHostToDevice,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->t_pages.push_back(pv);
    c->tape_cap += kTapePageRecs;
  }
  return UCC_OK;
}

void release_tape(ucc_ctx* c) {
  for (auto& p : c->t_pages) dfree(p);
  c->t_pages.clear();
  c->tape_cap = 0;
}

template <class KT>
KT reference_key(const ucc_ctx* c) {
  KT hf = KeyOps<KT>::zero();
  for (int s = 0; s < c->n_alpha; ++s) hf = hf | KeyOps<KT>::bit(2 * s);
  for (int s = 0; s < c->n_beta; ++s) hf = hf | KeyOps<KT>::bit(2 * s + 1);
  return hf;
}

// psi = {reference: 1.0} in table s.
template <class KT>
ucc_status reset_table(ucc_ctx* c, TableSet& s) {
  if (s.cur.cap_n == 0) UCC_TRY(s.cur.allocate(1 << 12, slots_for(1 << 12)));
  CUDA_TRY(cudaMemsetAsync(s.d_cnt, 0, sizeof(Counters), c->stream));
  CUDA_TRY(cudaMemsetAsync(s.cur.slots, 0, s.cur.n_slots * sizeof(SlotT<KT>), c->stream));
  CUDA_TRY(cudaMemsetAsync(s.cur.filt, 0, s.cur.n_slots / 4 * sizeof(unsigned int), c->stream));
  CUDA_TRY(launch_reset(c->template table<KT>(s), reference_key<KT>(c), c->stream));
  c->launches++;
  return UCC_OK;
}

// Start the kill tape of a segment that begins at factor k0.
ucc_status reset_tape(ucc_ctx* c, TableSet& s, int k0) {
  UCC_TRY(ensure_tape(c, 1));
  CUDA_TRY(cudaMemsetAsync(&s.d_cnt->tape_n, 0, sizeof(unsigned long long), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->t_off + k0, 0, sizeof(unsigned long long), c->stream));
  return UCC_OK;
}

// Load a snapshot into table s (its previous contents are discarded).
template <class KT>
ucc_status load_snapshot(ucc_ctx* c, TableSet& s, const Snapshot& snap) {
  const unsigned long long cap = std::max<unsigned long long>(4 * snap.n, 1 << 12);
  if (cap >= kMaxEntries) return fail(UCC_ECAPACITY, "snapshot too large for one table");
  if (s.cur.cap_n < cap) UCC_TRY(s.cur.allocate(cap, slots_for(cap)));
  CUDA_TRY(cudaMemsetAsync(s.d_cnt, 0, sizeof(Counters), c->stream));
  CUDA_TRY(cudaMemsetAsync(s.cur.slots, 0, s.cur.n_slots * sizeof(SlotT<KT>), c->stream));
  CUDA_TRY(cudaMemsetAsync(s.cur.filt, 0, s.cur.n_slots / 4 * sizeof(unsigned int), c->stream));
  const int grid = c->full_grid();
  CUDA_TRY(launch_restore(c->template table<KT>(s), reinterpret_cast<const KT*>(snap.keys), snap.amps, snap.n, grid,
                          c->stream));
  CUDA_TRY(launch_rehash(c->template table<KT>(s), grid, c->stream));
  c->launches += 2;
  return read_counters(c, s);
}

// Copy the live entries of table s into a new snapshot.
template <class KT>
ucc_status take_snapshot(ucc_ctx* c, TableSet& s, Snapshot* out) {
  UCC_TRY(read_counters(c, s));
  const unsigned long long live = s.h_cnt->n_tail - s.h_cnt->n_dead;
  out->release();
  UCC_TRY(dalloc(&out->keys, live * c->kw));
  UCC_TRY(dalloc(&out->amps, live));
  out->n = live;
  CUDA_TRY(cudaMemsetAsync(&s.d_cnt->new_n, 0, sizeof(unsigned long long), c->stream));
  CUDA_TRY(launch_export(c->template table<KT>(s), live, reinterpret_cast<KT*>(out->keys), out->amps, nullptr,
                         c->full_grid(), c->stream));
  c->launches++;
  UCC_TRY(read_counters(c, s));
  if (s.h_cnt->new_n != live) return fail(UCC_ECUDA, "snapshot count mismatch");
  return UCC_OK;
}

// Host copy of factor k in the context's key width.
template <class KT>
FactorT<KT> host_factor(const ucc_ctx* c, int k);
template <>
Factor host_factor<unsigned long long>(const ucc_ctx* c, int k) {
  return c->factors[k];
}
template <>
FactorT<Key128> host_factor<Key128>(const ucc_ctx* c, int k) {
  return c->factors_w[k];
}

int pick_probe_width(ucc_ctx* c) {
  int pw = c->opt.probe_width;
  if (pw == 1 || pw == 2 || pw == 4 || pw == 8) return pw;
  return c->probe_width;
}

// Probe-width autotuner: per (spin-orbitals, floor(log2 stored entries)) the
// fastest of 1, 2, 4 and 8 lanes per lookup, timed on the live table by a
// read-only replay of the next factor's partner lookups.  Results are kept
// for the life of the process.
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, int> g_tuned;

template <class KT>
ucc_status autotune(ucc_ctx* c, TableSet& s, int k, unsigned long long n) {
  if (c->opt.probe_width != 0 || n < (1ull << 16) || k >= c->K) return UCC_OK;
  int bucket = 0;
  while ((2ull << bucket) <= n) ++bucket;
  const std::pair<int, int> key(c->n_so, bucket);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      c->probe_width = it->second;
      return UCC_OK;
    }
  }
  unsigned long long* sink = nullptr;
  UCC_TRY(dalloc(&sink, 1));
  const int widths[4] = {1, 2, 4, 8};
  float best_ms = 0.f;
  int best = 1;
  ucc_status st = UCC_OK;
  for (int rep = 0; rep < 2 && st == UCC_OK; ++rep)
    for (int w : widths) {
      if (cudaEventRecord(c->kev[0], c->stream) != cudaSuccess ||
          launch_probe_bench(c->template table<KT>(s), host_factor<KT>(c, k), w, sink, c->full_grid(), c->stream) !=
              cudaSuccess ||
          cudaEventRecord(c->kev[1], c->stream) != cudaSuccess || cudaEventSynchronize(c->kev[1]) != cudaSuccess) {
        st = fail(UCC_ECUDA, "probe-width autotuning failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->kev[0], c->kev[1]);
      if (rep == 1 && (w == 1 || ms < best_ms)) {
        best_ms = ms;
        best = w;
      }
      c->launches++;
    }
  dfree(sink);
  UCC_TRY(st);
  c->probe_width = best;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned[key] = best;
  return UCC_OK;
}

// Make room for the next factor: it may append one entry per stored entry
// (and, in gradient runs, drop as many onto the tape).  Compacts when a
// quarter of the stored entries are dropped ones.
// Room for the next factor of table s, whose counters the host knows (*h,
// updated here): grow or compact when the next factor might not fit or a
// quarter of the stored entries are dropped; more kill tape when recording.
template <class KT>
ucc_status ensure_room_known(ucc_ctx* c, TableSet& s, bool record, Counters* h) {
  const unsigned long long live = h->n_tail - h->n_dead;
  if (c->opt.max_entries > 0 && live > (unsigned long long)c->opt.max_entries)
    return fail(UCC_ECAPACITY, "wavefunction exceeds max_entries (" + std::to_string(live) + " live)");
  const bool room = 2 * h->n_tail <= s.cur.cap_n && 8 * h->n_tail <= 3 * s.cur.n_slots;
  const bool sparse = h->n_dead > 4096 && h->n_dead * 4 > h->n_tail;
  if (record) UCC_TRY(ensure_tape(c, h->tape_n + 2 * live + (1 << 12)));
  if (!room || sparse) {
    unsigned long long cap = s.cur.cap_n;
    if (2 * live > cap || 8 * live > 3 * s.cur.n_slots) cap = std::max<unsigned long long>(5 * live / 2, 1 << 12);
    UCC_TRY(rebuild<KT>(c, s, cap, false, live));
    h->n_tail = live;  // a compaction keeps exactly the live entries
    h->n_dead = 0;
  }
  return UCC_OK;
}

template <class KT>
ucc_status ensure_room(ucc_ctx* c, TableSet& s, bool record) {
  UCC_TRY(read_counters(c, s));
  Counters h = *s.h_cnt;  // copy: later reads overwrite the mirror
  return ensure_room_known<KT>(c, s, record, &h);
}

// Factors [k0, k1) on table s.  The last block of each factor flags a stop
// when the next factor might not fit or when the Methods-section cut is due;
// later launches in the chunk then skip, and the host cuts / grows and
// resumes at the flagged factor.  Chunks shrink when stops come often.
template <class KT>
ucc_status run_factors(ucc_ctx* c, TableSet& s, double eps, bool record, int k0, int k1) {
  const unsigned long long n_max = c->opt.n_max > 0 ? (unsigned long long)c->opt.n_max : 0ull;
  UCC_TRY(read_counters(c, s));
  unsigned long long n_known = s.h_cnt->n_tail;
  int chunk = 64;
  int k = k0;
  // Growth per factor of the live entries and of the table's tail, from the
  // last chunk: a chunk is sized to end just past the factor expected to
  // stop it (a cut or a table that needs room), so few launches after a stop
  // are skipped and few chunks end early.
  double g_live = 0.0, g_tail = 0.0;
  auto predicted_chunk = [&](const Counters& h, unsigned long long cap, unsigned long long slots) {
    double f = 64.0;
    const double live = (double)(h.n_tail - h.n_dead);
    if (n_max > 0 && g_live > 0.0) f = std::min(f, ((double)n_max - live) / g_live);
    const double nt_lim = std::min((double)cap / 2.0, 3.0 * (double)slots / 8.0);
    if (g_tail > 0.0) f = std::min(f, (nt_lim - (double)h.n_tail) / g_tail);
    return (int)std::max(2.0, std::min(64.0, std::floor(f) + 2.0));
  };
  while (k < k1) {
    const int end = std::min(k1, k + chunk);
    const unsigned long long live0 = s.h_cnt->n_tail - s.h_cnt->n_dead, tail0 = s.h_cnt->n_tail;
    // Grid sized from the last known count (grid-stride loops stay correct if
    // the table grew since).
    const unsigned long long est = std::min<unsigned long long>(n_known * 4, s.cur.cap_n);
    int grid = (int)std::min<unsigned long long>((unsigned long long)c->full_grid(), (est + 255) / 256);
    grid = std::max(grid, std::min(c->full_grid(), 4));
    if (k < 0 || end > c->K) return fail(UCC_ECUDA, "factor index out of range");
    const int pw = pick_probe_width(c);
    CUDA_TRY(cudaEventRecord(c->kev[0], c->stream));
    for (int kk = k; kk < end; ++kk) {
      CUDA_TRY(launch_forward(c->template table<KT>(s), c->template dfactors<KT>(), kk, eps, (unsigned int)(kk + 1),
                              record ? 1 : 0, c->template tape<KT>(), n_max, pw, grid, c->stream));
      c->launches += 2;  // the step and the linking of its appended entries
      c->stats.forward_launches++;
    }
    CUDA_TRY(cudaEventRecord(c->kev[1], c->stream));
    UCC_TRY(read_counters(c, s));
    {
      float kms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&kms, c->kev[0], c->kev[1]));
      c->stats.forward_kernel_ms += kms;
    }
    const Counters h = *s.h_cnt;  // copy: later reads overwrite the mirror
    n_known = h.n_tail;
    c->stats.peak_entries = std::max<long long>(c->stats.peak_entries, (long long)h.n_tail);
    {
      const int applied = h.stop_k >= 0 ? h.stop_k - k : end - k;
      if (applied > 0) {
        g_live = ((double)(h.n_tail - h.n_dead) - (double)live0) / applied;
        g_tail = ((double)h.n_tail - (double)tail0) / applied;
      }
    }
    if (h.stop_k >= 0) {
      const int resume = h.stop_k;
      if (resume <= k || resume > end) return fail(UCC_ECUDA, "invalid resume factor");
      // The host follows the table's counters through the cut and any growth
      // without reading them back: the cut keeps exactly N_CUT entries with
      // none dropped (the device checks the count) and records the other live
      // ones on the tape.
      Counters known = h;
      if (h.cut_pending) {
        const unsigned long long before = h.n_tail - h.n_dead, kept = (unsigned long long)c->opt.n_cut;
        UCC_TRY(cut_rebuild<KT>(c, s, record, resume - 1));
        known.n_tail = kept;
        known.n_dead = 0;
        if (record) known.tape_n = h.tape_n + (before - kept);
        c->cut_total += (long long)(before - kept);
      }
      UCC_TRY(ensure_room_known<KT>(c, s, record, &known));
      CUDA_TRY(cudaMemsetAsync(&s.d_cnt->stop_k, 0xFF, sizeof(int), c->stream));  // -1
      CUDA_TRY(cudaMemsetAsync(&s.d_cnt->cut_pending, 0, sizeof(int), c->stream));
      known.stop_k = -1;
      known.cut_pending = 0;
      *s.h_cnt = known;
      n_known = known.n_tail;
      chunk = predicted_chunk(known, s.cur.cap_n, s.cur.n_slots);
      k = resume;
      continue;
    }
    UCC_TRY(autotune<KT>(c, s, end, h.n_tail));
    // Compact when a quarter of the stored entries are dropped ones.
    if (h.n_dead > 4096 && h.n_dead * 4 > h.n_tail) {
      UCC_TRY(rebuild<KT>(c, s, s.cur.cap_n, false, h.n_tail - h.n_dead));
      s.h_cnt->n_tail = h.n_tail - h.n_dead;  // a compaction keeps exactly the live entries
      s.h_cnt->n_dead = 0;
    }
    chunk = predicted_chunk(*s.h_cnt, s.cur.cap_n, s.cur.n_slots);
    k = end;
  }
  return UCC_OK;
}

void fill_forward_stats(ucc_ctx* c, const Counters& h) {
  c->stats.n_det = (long long)(h.n_tail - h.n_dead);
  c->stats.rotations = (long long)h.rotations;
  c->stats.created = (long long)h.created;
  c->stats.dropped_new = (long long)h.dropped_new;
  c->stats.dropped_old = (long long)h.dropped_old;
  c->stats.cut = c->cut_total;
  c->stats.scanned = (long long)h.scanned;
  c->stats.probe_width = pick_probe_width(c);
}

// Factors per gradient segment.  One segment (the whole run on one tape) when
// the tape fits its memory budget; otherwise ~sqrt(K)-long segments:
// snapshots at their starts, one recomputation each, and a tape that covers
// one segment.
int segment_stride(const ucc_ctx* c) {
  if (c->opt.checkpoint_stride > 0) return std::min(c->opt.checkpoint_stride, std::max(1, c->K));
  if (c->force_segments) return std::max(1, (int)std::ceil(std::sqrt((double)std::max(1, c->K))));
  return std::max(1, c->K);
}

template <class KT>
ucc_status run_forward(ucc_ctx* c, double eps, bool record) {
  if (!(eps >= 0.0) || std::isinf(eps)) return fail(UCC_EINVAL, "eps must be finite and >= 0");
  TableSet& s = c->ts[c->main];
  c->cut_total = 0;
  c->entropy_on = !record && c->opt.record_entropy != 0;
  c->have_entropy = false;
  UCC_TRY(reset_table<KT>(c, s));
  CUDA_TRY(cudaEventRecord(c->ev[0], c->stream));
  if (!record) {
    UCC_TRY(run_factors<KT>(c, s, eps, false, 0, c->K));
    c->have_entropy = c->entropy_on;
    c->entropy_on = false;
  } else {
    const int S = segment_stride(c);
    const int nseg = c->K == 0 ? 0 : (c->K + S - 1) / S;
    for (auto& sn : c->snaps) sn.release();
    c->snaps.assign(std::max(0, nseg), Snapshot());
    for (int j = 0; j < nseg; ++j) {
      const int k0 = j * S, k1 = std::min(c->K, k0 + S);
      if (j > 0) UCC_TRY(take_snapshot<KT>(c, s, &c->snaps[j]));
      UCC_TRY(reset_tape(c, s, k0));
      UCC_TRY(run_factors<KT>(c, s, eps, true, k0, k1));
    }
  }
  CUDA_TRY(cudaEventRecord(c->ev[1], c->stream));
  UCC_TRY(read_counters(c, s));
  UCC_TRY(flush_timings(c));
  fill_forward_stats(c, *s.h_cnt);
  c->stats.tape_entries = (long long)s.h_cnt->tape_n;
  c->stats.capacity_entries = (long long)s.cur.cap_n;
  c->stats.hash_slots = (long long)s.cur.n_slots;
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  c->stats.apply_ms = ms;
  c->have_psi = true;
  return UCC_OK;
}

// Record buffer of the bucketed energy: at most this much device memory, and
// at most this share of what is free.
constexpr size_t kSbBudgetBytes = size_t(32) << 30;
constexpr double kSbBudgetShare = 0.4;

// sigma, E and <psi|psi> by buckets of shared cores (records of partitions in
// rounds that fit the record buffer).  *done = false, with nothing launched,
// when the buffers cannot be had and the route allows the per-connection pass.
template <class KT>
ucc_status energy_by_buckets(ucc_ctx* c, TableSet& s, const Integrals& in, bool* done, unsigned long long* records) {
  *done = false;
  const bool must = c->opt.energy_route == 2;
  const Counters h = *s.h_cnt;
  const unsigned long long n = h.n_tail, live = h.n_tail - h.n_dead;
  const unsigned long long ne = (unsigned long long)(c->n_alpha + c->n_beta);
  const unsigned long long est = live * (ne + ne * (ne - 1) / 2);
  if (est == 0) {
    if (must) return fail(UCC_ESTATE, "no stored determinant to bucket");
    return UCC_OK;
  }
  int log2p = 0;
  if (c->opt.energy_test_partitions > 0)
    while ((1 << log2p) < c->opt.energy_test_partitions) ++log2p;
  else
    while (log2p < 24 && (est >> log2p) > (unsigned long long)sb_partition_target()) ++log2p;
  const unsigned long long P = 1ull << log2p;
  auto unavailable = [&](const char* what) -> ucc_status {
    if (must) return fail(UCC_ENOMEM, std::string("bucketed energy: ") + what);
    cudaGetLastError();  // clear a failed allocation
    return UCC_OK;
  };
  if (c->sb_parts < P) {
    dfree(c->d_sb_cnt);
    dfree(c->d_sb_fill);
    dfree(c->d_sb_off);
    c->sb_parts = 0;
    if (dalloc(&c->d_sb_cnt, P) != UCC_OK || dalloc(&c->d_sb_fill, P) != UCC_OK ||
        dalloc(&c->d_sb_off, P + 1) != UCC_OK) {
      dfree(c->d_sb_cnt);
      dfree(c->d_sb_fill);
      dfree(c->d_sb_off);
      return unavailable("partition arrays");
    }
    c->sb_parts = P;
  }
  const size_t rec_bytes = sb_record_bytes(c->wide ? 2 : 1);
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const size_t want = std::min<size_t>(kSbBudgetBytes, (size_t)est * rec_bytes);
  if (c->sb_rec_cap < want && c->sb_rec_cap < (size_t)(kSbBudgetShare * (double)(free_b + c->sb_rec_cap))) {
    dfree(c->d_sb_rec);
    c->sb_rec_cap = 0;
    size_t bytes = std::min(want, (size_t)(kSbBudgetShare * (double)free_b));
    bytes -= bytes % 32;
    if (bytes < 32 * rec_bytes || dalloc(&c->d_sb_rec, bytes) != UCC_OK) return unavailable("record buffer");
    c->sb_rec_cap = bytes;
  }
  unsigned long long cap_recs = c->sb_rec_cap / rec_bytes;
  if (c->opt.energy_test_buffer_records > 0)
    cap_recs = std::min<unsigned long long>(cap_recs, (unsigned long long)c->opt.energy_test_buffer_records);
  const int grid = (int)std::max<unsigned long long>(
      1ull, std::min<unsigned long long>((unsigned long long)c->full_grid(8), (n + 255) / 256));
  const int pair_grid = std::max(1, c->num_sms * std::max(1, sb_blocks_per_sm(c->wide ? 2 : 1)));
  const TableT<KT> t = c->template table<KT>(s);
  SigRecT<KT>* rec = reinterpret_cast<SigRecT<KT>*>(c->d_sb_rec);
  CUDA_TRY(cudaMemsetAsync(c->d_sb_cnt, 0, P * sizeof(unsigned int), c->stream));
  CUDA_TRY(cudaMemsetAsync(t.sigma, 0, n * sizeof(double), c->stream));
  CUDA_TRY(launch_sb_count(t, c->d_sb_cnt, log2p, grid, c->stream));
  CUDA_TRY(launch_sb_scan(c->d_sb_cnt, c->d_sb_off, P, c->stream));
  c->launches += 2;
  auto off_at = [&](unsigned long long p, unsigned long long* v) -> ucc_status {
    CUDA_TRY(cudaMemcpyAsync(v, c->d_sb_off + p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return UCC_OK;
  };
  unsigned long long total = 0;
  UCC_TRY(off_at(P, &total));
  *records = total;
  // Rounds: partition ranges whose records fit the buffer, halved until they do.
  std::vector<std::pair<unsigned long long, unsigned long long>> todo;
  {
    const unsigned long long rounds = std::max<unsigned long long>(1ull, (total + cap_recs - 1) / cap_recs);
    unsigned long long width = P;
    while (width > 1 && P / width < rounds) width >>= 1;
    for (unsigned long long p = P; p > 0; p -= width) todo.push_back({p - width, p});
  }
  while (!todo.empty()) {
    const auto [p0, p1] = todo.back();
    todo.pop_back();
    unsigned long long a = 0, b = 0;
    UCC_TRY(off_at(p0, &a));
    UCC_TRY(off_at(p1, &b));
    if (b - a > cap_recs) {
      if (p1 - p0 == 1) return fail(UCC_ECAPACITY, "one core partition outgrew the record buffer");
      const unsigned long long mid = p0 + (p1 - p0) / 2;
      todo.push_back({mid, p1});
      todo.push_back({p0, mid});
      continue;
    }
    if (b == a) continue;
    CUDA_TRY(cudaMemsetAsync(c->d_sb_fill + p0, 0, (p1 - p0) * sizeof(unsigned int), c->stream));
    CUDA_TRY(launch_sb_scatter(t, c->d_sb_off, c->d_sb_fill, rec, log2p, p0, p1, a, grid, c->stream));
    CUDA_TRY(launch_sb_pairs(t, in, rec, c->d_sb_off, log2p, p0, p1, a,
                             (int)std::min<unsigned long long>((unsigned long long)pair_grid, p1 - p0), c->stream));
    c->launches += 2;
  }
  CUDA_TRY(launch_sb_finish(t, in, grid, c->stream));
  c->launches++;
  *done = true;
  return UCC_OK;
}

template <class KT>
ucc_status run_energy(ucc_ctx* c, double* E, double* norm2) {
  TableSet& s = c->ts[c->main];
  Integrals in;
  in.h = c->d_h;
  in.g = c->d_g;
  in.n = c->n_spatial;
  in.n_so = c->n_so;
  UCC_TRY(read_counters(c, s));
  const unsigned long long n = s.h_cnt->n_tail;
  int grid = (int)std::min<unsigned long long>((unsigned long long)c->full_grid(), (n + 7) / 8);
  grid = std::max(grid, 1);
  UCC_TRY(ensure_partials(c, c->full_grid()));
  CUDA_TRY(cudaMemsetAsync(&s.d_cnt->sig_probes, 0, 2 * sizeof(unsigned long long), c->stream));
  CUDA_TRY(cudaEventRecord(c->ev[2], c->stream));
  bool bucketed = false;
  unsigned long long records = 0;
  if (c->opt.energy_route != 1) UCC_TRY(energy_by_buckets<KT>(c, s, in, &bucketed, &records));
  if (!bucketed) {
    CUDA_TRY(launch_sigma(c->template table<KT>(s), in, grid, c->stream));
    c->launches += 2;
  }
  CUDA_TRY(cudaEventRecord(c->ev[3], c->stream));
  UCC_TRY(read_counters(c, s));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
  c->stats.energy_ms = ms;
  c->stats.energy_route = bucketed ? 2 : 1;
  // probes: hash lookups (per connection) or core records (by buckets); hits:
  // connected stored pairs, each counted once
  c->stats.sigma_probes = bucketed ? (long long)records : (long long)s.h_cnt->sig_probes;
  c->stats.sigma_hits = bucketed ? (long long)(s.h_cnt->sig_hits / 2) : (long long)s.h_cnt->sig_hits;
  const double n2 = s.h_cnt->norm2;
  if (norm2) *norm2 = n2;
  if (E) *E = s.h_cnt->e_num / n2 + c->e_nuc;
  c->have_sigma = true;
  return UCC_OK;
}

// The reverse sweep over factors [k0, k1) on table s, which holds psi_{k1}
// and mu_{k1} (in lam), with the tape recorded for this segment.  Step k
// appends at most its own tape records; the host keeps an upper bound of the
// stored count and compacts (keeping lam) or grows before a step could pass
// the table's room.
// Reverse steps between reads of the dropped-entry count.
constexpr int kDeadCheck = 16;

template <class KT>
ucc_status reverse_segment(ucc_ctx* c, TableSet& s, int k0, int k1) {
  if (k1 <= k0) return UCC_OK;
  std::vector<unsigned long long> off(k1 - k0 + 1);
  CUDA_TRY(cudaMemcpyAsync(off.data(), c->t_off + k0, off.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, c->stream));
  UCC_TRY(read_counters(c, s));
  const int grid_full = c->full_grid();
  unsigned long long bound = s.h_cnt->n_tail;
  int grid = (int)std::min<unsigned long long>((unsigned long long)grid_full, (bound * 2 + 255) / 256);
  grid = std::max(grid, std::min(grid_full, 4));
  CUDA_TRY(cudaEventRecord(c->kev[0], c->stream));
  float kernel_ms = 0.f;
  int since_check = 0;
  for (int k = k1 - 1; k >= k0; --k) {
    const unsigned int stamp = 0x80000000u | (unsigned int)k;
    const unsigned long long lo = off[k - k0], hi = off[k - k0 + 1];
    if (hi > c->tape_cap || lo > hi) return fail(UCC_ECUDA, "tape offsets out of range");
    const unsigned long long rec = hi - lo;
    // Every kDeadCheck steps, read the counters: when a third of the stored
    // entries are dropped (entries the sweep removed, and those the forward
    // pass dropped since its last rebuild), compact, since every step scans
    // them all.
    bool compact = false;
    if (++since_check >= kDeadCheck) {
      since_check = 0;
      UCC_TRY(read_counters(c, s));
      compact = s.h_cnt->n_dead > 4096 && 3ull * s.h_cnt->n_dead > s.h_cnt->n_tail;
    }
    if (compact || bound + rec > s.cur.cap_n || 4ull * (bound + rec) > 3ull * s.cur.n_slots) {
      CUDA_TRY(cudaEventRecord(c->kev[1], c->stream));
      UCC_TRY(read_counters(c, s));
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, c->kev[0], c->kev[1]));
      kernel_ms += ms;
      // Live entries now: stored minus those the sweep or the forward dropped.
      UCC_TRY(rebuild<KT>(c, s, s.cur.cap_n, true, s.h_cnt->n_tail - s.h_cnt->n_dead));
      c->stats.reverse_compactions++;
      UCC_TRY(read_counters(c, s));
      bound = s.h_cnt->n_tail;
      if (bound + rec > s.cur.cap_n || 4ull * (bound + rec) > 3ull * s.cur.n_slots) {
        UCC_TRY(rebuild<KT>(c, s, std::max<unsigned long long>(2 * s.cur.cap_n, 2 * (bound + rec) + 64), true,
                            s.h_cnt->n_tail - s.h_cnt->n_dead));
        UCC_TRY(read_counters(c, s));
        bound = s.h_cnt->n_tail;
      }
      grid = (int)std::min<unsigned long long>((unsigned long long)grid_full, (bound * 2 + 255) / 256);
      grid = std::max(grid, std::min(grid_full, 4));
      CUDA_TRY(cudaEventRecord(c->kev[0], c->stream));
    }
    if (rec) {
      const int g2 = (int)std::min<unsigned long long>((unsigned long long)grid_full, (rec + 255) / 256);
      // A bulk re-insertion of at least one record per eight slots (a cut's
      // records) into a large one-word table is hashed region by region: the
      // regions are read and written whole, which beats one random claim per
      // record only when most regions receive many records.
      const bool by_regions = (8 * rec >= s.cur.n_slots || c->opt.rebuild_test_regions == 2) &&
                              regions_ok(c, s.cur.n_slots, s.cur.n_slots) &&
                              ensure_rehash_scratch(c, s.cur.cap_n, s.cur.n_slots) == UCC_OK;
      if (!by_regions) cudaGetLastError();
      CUDA_TRY(launch_tape_reinsert(c->template table<KT>(s), c->template tape<KT>(), k, rec, std::max(g2, 1),
                                    c->stream, &c->launches, by_regions ? &c->rs : nullptr, c->num_sms));
    }
    CUDA_TRY(launch_reverse(c->template table<KT>(s), c->template dfactors<KT>(), k, stamp, c->d_grad,
                            pick_probe_width(c), grid, c->stream));
    c->launches++;
    c->stats.reverse_launches++;
    bound += rec;
  }
  CUDA_TRY(cudaEventRecord(c->kev[1], c->stream));
  UCC_TRY(read_counters(c, s));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->kev[0], c->kev[1]));
  c->stats.reverse_kernel_ms += kernel_ms + ms;
  c->stats.reverse_pairs += (long long)s.h_cnt->rev_pairs;
  c->stats.reverse_scanned += (long long)s.h_cnt->rev_scanned;
  return UCC_OK;
}

template <class KT>
ucc_status run_gradient_once(ucc_ctx* c, double eps, double* E, double* grad_out, int on_device);

// dE/dtheta: first on one tape; if the tape would pass its budget, again with
// segment checkpoints.
template <class KT>
ucc_status run_gradient(ucc_ctx* c, double eps, double* E, double* grad_out, int on_device) {
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  const unsigned long long held = (unsigned long long)c->tape_cap * c->tape_rec_bytes();
  c->tape_budget = c->opt.tape_budget_mb > 0 ? (unsigned long long)c->opt.tape_budget_mb << 20
                                             : (unsigned long long)(0.6 * (double)(free_b + held));
  c->force_segments = false;
  c->tape_over_budget = false;
  ucc_status s = run_gradient_once<KT>(c, eps, E, grad_out, on_device);
  if (s == UCC_ECAPACITY && c->tape_over_budget && c->opt.checkpoint_stride <= 0) {
    release_tape(c);
    c->force_segments = true;
    c->tape_over_budget = false;
    c->tape_budget = 0;
    s = run_gradient_once<KT>(c, eps, E, grad_out, on_device);
  }
  return s;
}

template <class KT>
ucc_status run_gradient_once(ucc_ctx* c, double eps, double* E, double* grad_out, int on_device) {
  c->launches = 0;
  drop_timings(c);
  c->stats = ucc_stats{};
  c->main = 0;
  UCC_TRY(run_forward<KT>(c, eps, true));
  TableSet& s0 = c->ts[c->main];
  double e = 0.0, n2 = 0.0;
  UCC_TRY(run_energy<KT>(c, &e, &n2));
  if (E) *E = e;
  const int grid_full = c->full_grid();
  UCC_TRY(ensure_partials(c, grid_full));
  CUDA_TRY(cudaEventRecord(c->ev[4], c->stream));
  CUDA_TRY(launch_lambda_init(c->template table<KT>(s0), grid_full, c->stream));
  c->launches++;
  const int S = segment_stride(c);
  const int nseg = c->K == 0 ? 0 : (c->K + S - 1) / S;
  long long tape_peak = c->stats.tape_entries;
  for (int j = nseg - 1; j >= 0; --j) {
    const int k0 = j * S, k1 = std::min(c->K, k0 + S);
    if (j < nseg - 1) {
      // Recompute segment j forward from its snapshot on the other table,
      // recording its tape; carry mu over by key; swap the tables' roles.
      TableSet& from = c->ts[c->main];
      TableSet& work = c->ts[1 - c->main];
      if (j == 0) {
        UCC_TRY(reset_table<KT>(c, work));
      } else {
        UCC_TRY(load_snapshot<KT>(c, work, c->snaps[j]));
      }
      UCC_TRY(reset_tape(c, work, k0));
      UCC_TRY(run_factors<KT>(c, work, eps, true, k0, k1));
      UCC_TRY(read_counters(c, work));
      c->stats.recompute_scanned += (long long)work.h_cnt->scanned;
      c->stats.recompute_rotations += (long long)work.h_cnt->rotations;
      c->stats.recompute_created += (long long)work.h_cnt->created;
      tape_peak = std::max<long long>(tape_peak, (long long)work.h_cnt->tape_n);
      CUDA_TRY(launch_transfer_lambda(c->template table<KT>(work), c->template table<KT>(from), grid_full, c->stream));
      c->launches++;
      c->main = 1 - c->main;
    }
    UCC_TRY(reverse_segment<KT>(c, c->ts[c->main], k0, k1));
  }
  CUDA_TRY(cudaEventRecord(c->ev[5], c->stream));
  if (grad_out && c->K) {
    CUDA_TRY(cudaMemcpyAsync(grad_out, c->d_grad, c->K * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  UCC_TRY(read_counters(c, c->ts[c->main]));
  UCC_TRY(flush_timings(c));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
  c->stats.reverse_ms = ms;
  c->stats.tape_entries = tape_peak;
  c->stats.kernel_launches = c->launches;
  for (auto& sn : c->snaps) sn.release();
  c->have_psi = false;
  c->have_sigma = false;
  c->main = 0;
  return UCC_OK;
}

ucc_status validate_problem(const ucc_hamiltonian* ham, const ucc_ansatz* an) {
  if (!ham || !an) return fail(UCC_EINVAL, "null hamiltonian or ansatz");
  const int n = ham->n_spatial;
  if (n < 1 || n > 64) return fail(UCC_EINVAL, "n_spatial must be in [1, 64] (128-bit determinant keys)");
  if (ham->n_alpha < 0 || ham->n_beta < 0 || ham->n_alpha > n || ham->n_beta > n || ham->n_alpha + ham->n_beta < 1)
    return fail(UCC_EINVAL, "electron counts out of range");
  if (!ham->h || !ham->g) return fail(UCC_EINVAL, "null integrals");
  if (an->n_exc < 0 || (an->n_exc > 0 && !an->idx)) return fail(UCC_EINVAL, "bad excitation list");
  if (!std::isfinite(ham->e_nuc)) return fail(UCC_EINVAL, "e_nuc not finite");
  const size_t n4 = (size_t)n * n * n * n;
  for (size_t x = 0; x < (size_t)n * n; ++x)
    if (!std::isfinite(ham->h[x])) return fail(UCC_EINVAL, "h has a non-finite entry");
  for (size_t x = 0; x < n4; ++x)
    if (!std::isfinite(ham->g[x])) return fail(UCC_EINVAL, "g has a non-finite entry");
  const int nso = 2 * n;
  for (int k = 0; k < an->n_exc; ++k) {
    const int* r = an->idx + 4 * k;
    const int i = r[0], j = r[1], a = r[2], b = r[3];
    const bool single = (j == -1 && b == -1);
    if (!single && (j < 0 || b < 0)) return fail(UCC_EINVAL, "row " + std::to_string(k) + ": malformed");
    int ids[4] = {i, j, a, b};
    int cnt = single ? 2 : 4;
    int used[2] = {i, a};
    for (int x = 0; x < cnt; ++x) {
      int v = single ? used[x] : ids[x];
      if (v < 0 || v >= nso) return fail(UCC_EINVAL, "row " + std::to_string(k) + ": index out of range");
    }
    if (single) {
      if (i == a) return fail(UCC_EINVAL, "row " + std::to_string(k) + ": repeated index");
      if ((i & 1) != (a & 1)) return fail(UCC_EINVAL, "row " + std::to_string(k) + ": spin not conserved");
    } else {
      for (int x = 0; x < 4; ++x)
        for (int y = x + 1; y < 4; ++y)
          if (ids[x] == ids[y]) return fail(UCC_EINVAL, "row " + std::to_string(k) + ": repeated index");
      if (((i & 1) + (j & 1)) != ((a & 1) + (b & 1)))
        return fail(UCC_EINVAL, "row " + std::to_string(k) + ": spin not conserved");
    }
    if (an->theta && !std::isfinite(an->theta[k])) return fail(UCC_EINVAL, "theta is not finite");
  }
  return UCC_OK;
}

ucc_status upload_factors(ucc_ctx* c) {
  for (int k = 0; k < c->K; ++k) {
    const int* r = &c->rows[4 * k];
    if (c->wide)
      c->factors_w[k] = make_factor<Key128>(r[0], r[1], r[2], r[3], c->theta[k]);
    else
      c->factors[k] = make_factor<unsigned long long>(r[0], r[1], r[2], r[3], c->theta[k]);
  }
  if (c->K && c->wide)
    CUDA_TRY(cudaMemcpyAsync(c->d_factors, c->factors_w.data(), c->K * sizeof(FactorT<Key128>),
                             cudaMemcpyHostToDevice, c->stream));
  else if (c->K)
    CUDA_TRY(cudaMemcpyAsync(c->d_factors, c->factors.data(), c->K * sizeof(Factor), cudaMemcpyHostToDevice,
                             c->stream));
  // The host vector must outlive the copy.
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return UCC_OK;
}

void destroy(ucc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
    c->side = nullptr;
  }
  c->ts[0].release();
  c->ts[1].release();
  for (auto& sn : c->snaps) sn.release();
  dfree(c->d_factors);
  dfree(c->d_h);
  dfree(c->d_g);
  dfree(c->d_grad);
  dfree(c->d_partials);
  dfree(c->d_sb_cnt);
  dfree(c->d_sb_fill);
  dfree(c->d_sb_off);
  dfree(c->d_sb_rec);
  dfree(c->rs.rcnt);
  dfree(c->rs.rfill);
  dfree(c->rs.roff);
  dfree(c->rs.pairs);
  dfree(c->rs.over);
  dfree(c->rs.over_n);
  dfree(c->d_sel);
  dfree(c->d_cand);
  release_tape(c);
  dfree(c->d_entropy);
  dfree(c->d_pages);
  dfree(c->t_off);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->kev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->tev)
    if (e) cudaEventDestroy(e);
  delete c;
}

// Determinants in a job's sector (fixed alpha and beta electron counts).
unsigned long long sector_size(const ucc_ctx* c) {
  auto comb = [](int n, int k) {
    unsigned long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (unsigned long long)(n - k + i) / (unsigned long long)i;
    return r;
  };
  return comb(c->n_spatial, c->n_alpha) * comb(c->n_spatial, c->n_beta);
}

// Entry capacity a job of the persistent batch is given up front: three times
// its sector (a table holds at most the sector live plus a quarter dropped,
// and a step may double what it holds), or three times N_MAX when its cut can
// fire.  0 when the job cannot be sized (no cut and a sector too large).
unsigned long long batch_capacity(const ucc_ctx* c) {
  if (c->wide) return 0;  // the persistent batched kernels take one-word keys
  const unsigned long long sector = sector_size(c);
  const unsigned long long n_max = c->opt.n_max > 0 ? (unsigned long long)c->opt.n_max : 0ull;
  unsigned long long cap = (n_max > 0 && sector > n_max) ? 3 * n_max : 3 * sector;
  cap = std::max<unsigned long long>(cap, 4096);
  if (c->opt.max_entries > 0 && cap > 3ull * (unsigned long long)c->opt.max_entries) return 0;
  // A job's cuts and compactions run on one block: larger tables take the
  // one-job path, whose kernels spread a table over the whole GPU.
  if (cap > (1ull << 22)) return 0;
  return cap;
}

// A graph holding the one launch that `launch` enqueues on st, or nullptr when
// the launch cannot be captured (the caller then launches it directly).
template <class F>
cudaGraphExec_t capture_one(cudaStream_t st, F launch) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const cudaError_t le = launch();
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  if (le == cudaSuccess && ce == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ex;
}

// Persistent-batch tuning: (probe width, tiles per warp visit) per batch shape,
// chosen by timing the first steps of the forward pass with each candidate.
std::mutex g_btune_mutex;
std::map<std::pair<int, int>, std::pair<int, int>> g_btuned;

// The batched path: one cooperative launch runs the whole forward pass of every
// job, one launch the energy, one the whole reverse pass.
ucc_status batch_persistent(const std::vector<int>& idx, ucc_ctx* const* jobs, double eps, double* E,
                            double* const* grads) {
  const int n = (int)idx.size();
  ucc_ctx* c0 = jobs[idx[0]];
  cudaStream_t st = c0->stream;
  bool record = false;
  for (int x = 0; x < n; ++x) record |= grads && grads[idx[x]];
  JobView* d_jobs = nullptr;
  JobState* d_js = nullptr;
  BatchHeader* d_bh = nullptr;
  UCC_TRY(dalloc(&d_jobs, n));
  UCC_TRY(dalloc(&d_js, n));
  UCC_TRY(dalloc(&d_bh, 1));
  std::vector<JobView> hv(n);
  std::vector<JobState> hs(n);
  BatchHeader hb{};
  cudaGraphExec_t g_fwd = nullptr, g_rev = nullptr;
  auto release = [&]() {
    if (g_fwd) cudaGraphExecDestroy(g_fwd);
    if (g_rev) cudaGraphExecDestroy(g_rev);
    dfree(d_jobs);
    dfree(d_js);
    dfree(d_bh);
  };
  auto view_of = [&](int x) {
    ucc_ctx* c = jobs[idx[x]];
    JobView v{};
    v.t = c->template table<unsigned long long>(c->ts[0]);
    v.factors = c->template dfactors<unsigned long long>();
    v.tape = c->template tape<unsigned long long>();
    v.in.h = c->d_h;
    v.in.g = c->d_g;
    v.in.n = c->n_spatial;
    v.in.n_so = c->n_so;
    v.grad = c->d_grad;
    v.eps = eps;
    v.K = c->K;
    const Arrays& sp = c->ts[0].spare;
    v.sp = SpareArrays{sp.keys, sp.amps, sp.born, sp.lam, sp.slots, sp.filt};
    v.n_max = c->opt.n_max;
    v.n_cut = c->opt.n_cut;
    return v;
  };
  // Bring each host-side table in line with the device view: the persistent
  // kernels swap a job's two array sets.
  auto sync_swaps = [&]() -> ucc_status {
    std::vector<JobView> dv(n);
    CUDA_TRY(cudaMemcpyAsync(dv.data(), d_jobs, n * sizeof(JobView), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int x = 0; x < n; ++x) {
      TableSet& ts = jobs[idx[x]]->ts[0];
      if (dv[x].t.keys == ts.spare.keys) std::swap(ts.cur, ts.spare);
      if (dv[x].t.keys != ts.cur.keys) return fail(UCC_ECUDA, "batched job arrays out of step");
      // the kernels swap every array but sigma, which stays where it was
      if (dv[x].t.sigma != ts.cur.sigma) std::swap(ts.cur.sigma, ts.spare.sigma);
      hv[x] = dv[x];
    }
    return UCC_OK;
  };
  auto upload = [&]() -> ucc_status {
    for (int x = 0; x < n; ++x) hv[x] = view_of(x);
    CUDA_TRY(cudaMemcpyAsync(d_jobs, hv.data(), n * sizeof(JobView), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d_js, hs.data(), n * sizeof(JobState), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return UCC_OK;
  };
  auto fetch = [&]() -> ucc_status {
    CUDA_TRY(cudaMemcpyAsync(hs.data(), d_js, n * sizeof(JobState), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hb, d_bh, sizeof(BatchHeader), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return UCC_OK;
  };
  // Header for a (re)launch: barrier words cleared, error cleared.
  const unsigned long long wait_ns =
      c0->opt.batch_wait_ms > 0 ? 1000000ull * (unsigned long long)c0->opt.batch_wait_ms : 2000000000ull;
  auto reset_header = [&](int skip_block) -> ucc_status {
    BatchHeader h{};
    h.skip_block = skip_block;
    h.wait_ns = wait_ns;
    h.steps = hb.steps;
    CUDA_TRY(cudaMemcpyAsync(d_bh, &h, sizeof(BatchHeader), cudaMemcpyHostToDevice, st));
    return UCC_OK;
  };
  // Every job back to psi = {reference: 1.0} with its tables sized up front.
  auto reset_all = [&]() -> ucc_status {
    for (int x = 0; x < n; ++x) {
      ucc_ctx* c = jobs[idx[x]];
      const unsigned long long cap = batch_capacity(c);
      const unsigned long long ns = slots_for(cap);
      TableSet& ts = c->ts[0];
      UCC_TRY(settle_spare(c, ts));  // the kernels use the spare arrays directly
      ts.cur.slots_clean = false;     // ... and write both slot arrays
      ts.spare.slots_clean = false;
      if (ts.cur.cap_n != cap || ts.cur.n_slots != ns) UCC_TRY(ts.cur.allocate(cap, ns));
      if (ts.spare.cap_n != cap || ts.spare.n_slots != ns) UCC_TRY(ts.spare.allocate(cap, ns));
      c->main = 0;
      UCC_TRY(reset_table<unsigned long long>(c, ts));
      if (record) UCC_TRY(reset_tape(c, ts, 0));
      hs[x] = JobState{};
      hs[x].stop = -1;
    }
    hb = BatchHeader{};
    UCC_TRY(upload());
    return reset_header(-1);
  };
  auto run = [&]() -> ucc_status {
    for (int x = 0; x < n; ++x) {
      ucc_ctx* c = jobs[idx[x]];
      c->launches = 0;
      drop_timings(c);
      c->stats = ucc_stats{};
      c->cut_total = 0;
      c->tape_budget = 0;
      if (record) UCC_TRY(ensure_tape(c, 1));
    }
    // Probe width and tiles per warp visit: tuned once per batch shape.
    int maxK = 0, max_so = 0;
    for (int x = 0; x < n; ++x) {
      maxK = std::max(maxK, jobs[idx[x]]->K);
      max_so = std::max(max_so, jobs[idx[x]]->n_so);
    }
    int pw = c0->opt.probe_width > 0 ? c0->opt.probe_width : 0, tiles = c0->opt.batch_tiles;
    if (pw == 8) pw = 4;
    const std::pair<int, int> key((n + 15) / 16 * 16, max_so * 2 + (record ? 1 : 0));
    if (!tiles || !pw) {
      std::lock_guard<std::mutex> lock(g_btune_mutex);
      auto it = g_btuned.find(key);
      if (it != g_btuned.end()) {
        if (!pw) pw = it->second.first;
        if (!tiles) tiles = it->second.second;
      }
    }
    if (!tiles) {
      // Coordinate search on the first 64 steps: tiles with one-lane probes,
      // then the probe width with the best tile count.
      auto trial = [&](int w, int tl, float* ms) -> ucc_status {
        UCC_TRY(reset_all());
        CUDA_TRY(cudaEventRecord(c0->kev[0], st));
        CUDA_TRY(launch_persist_forward(d_jobs, d_js, n, d_bh, record ? 1 : 0, w, tl, 64, st));
        CUDA_TRY(cudaEventRecord(c0->kev[1], st));
        CUDA_TRY(cudaEventSynchronize(c0->kev[1]));
        CUDA_TRY(cudaEventElapsedTime(ms, c0->kev[0], c0->kev[1]));
        UCC_TRY(fetch());
        if (hb.error) return fail(hb.error & 1 ? UCC_ETIMEOUT : UCC_ECAPACITY, "persistent batch trial failed");
        for (int x = 0; x < n; ++x) jobs[idx[x]]->launches++;
        return UCC_OK;
      };
      float best = 0.f;
      int bw = pw ? pw : 1, bt = 1;
      for (int tl : {1, 2, 4, 8}) {
        float ms = 0.f;
        UCC_TRY(trial(bw, tl, &ms));
        if (tl == 1 || ms < best) {
          best = ms;
          bt = tl;
        }
      }
      if (!pw) {
        for (int w : {2, 4}) {
          float ms = 0.f;
          UCC_TRY(trial(w, bt, &ms));
          if (ms < best) {
            best = ms;
            bw = w;
          }
        }
      }
      pw = bw;
      tiles = bt;
      std::lock_guard<std::mutex> lock(g_btune_mutex);
      g_btuned[key] = std::make_pair(pw, tiles);
    }
    if (!pw) pw = 1;
    UCC_TRY(reset_all());
    // The forward pass: one persistent launch (a captured graph), relaunched
    // only when jobs wait for more tape.
    g_fwd = capture_one(st, [&]() {
      return launch_persist_forward(d_jobs, d_js, n, d_bh, record ? 1 : 0, pw, tiles, 1 << 30, st);
    });
    UCC_TRY(reset_header(c0->opt.batch_test_skip_block > 0 ? c0->opt.batch_test_skip_block - 1 : -1));
    CUDA_TRY(cudaEventRecord(c0->ev[0], st));
    for (int round = 0;; ++round) {
      if (g_fwd)
        CUDA_TRY(cudaGraphLaunch(g_fwd, st));
      else
        CUDA_TRY(launch_persist_forward(d_jobs, d_js, n, d_bh, record ? 1 : 0, pw, tiles, 1 << 30, st));
      UCC_TRY(fetch());
      for (int x = 0; x < n; ++x) jobs[idx[x]]->launches++;
      if (hb.error & 1) return fail(UCC_ETIMEOUT, "a grid barrier of the persistent batch timed out");
      if (hb.error) return fail(UCC_ECAPACITY, "a batched job outgrew the table it was given");
      bool waiting = false, done = true;
      for (int x = 0; x < n; ++x) {
        ucc_ctx* c = jobs[idx[x]];
        if (hs[x].k < c->K) done = false;
        if (hs[x].stop >= 0) {
          waiting = true;
          UCC_TRY(read_counters(c, c->ts[0]));
          const Counters h = *c->ts[0].h_cnt;
          UCC_TRY(ensure_tape(c, 2 * (h.tape_n + 2 * h.n_tail) + (1 << 12)));
          hs[x].stop = -1;
        }
      }
      if (done) break;
      if (!waiting || round > 4096) return fail(UCC_ECUDA, "persistent batch made no progress");
      UCC_TRY(sync_swaps());
      for (int x = 0; x < n; ++x) hv[x].tape = jobs[idx[x]]->template tape<unsigned long long>();
      CUDA_TRY(cudaMemcpyAsync(d_jobs, hv.data(), n * sizeof(JobView), cudaMemcpyHostToDevice, st));
      CUDA_TRY(cudaMemcpyAsync(d_js, hs.data(), n * sizeof(JobState), cudaMemcpyHostToDevice, st));
      UCC_TRY(reset_header(-1));
    }
    CUDA_TRY(cudaEventRecord(c0->ev[1], st));
    UCC_TRY(sync_swaps());
    for (int x = 0; x < n; ++x) {
      ucc_ctx* c = jobs[idx[x]];
      UCC_TRY(read_counters(c, c->ts[0]));
      c->cut_total = hs[x].cut;
      fill_forward_stats(c, *c->ts[0].h_cnt);
      c->stats.tape_entries = (long long)c->ts[0].h_cnt->tape_n;
      c->stats.forward_launches = 1;
      c->stats.probe_width = pw;
      c->stats.capacity_entries = (long long)c->ts[0].cur.cap_n;
      c->stats.hash_slots = (long long)c->ts[0].cur.n_slots;
    }
    // Energy of every job in one launch.
    for (int x = 0; x < n; ++x) hs[x].e_num = hs[x].norm2 = hs[x].gacc = 0.0;
    CUDA_TRY(cudaMemcpyAsync(d_js, hs.data(), n * sizeof(JobState), cudaMemcpyHostToDevice, st));
    for (int x = 0; x < n; ++x)
      CUDA_TRY(cudaMemsetAsync(&jobs[idx[x]]->ts[0].d_cnt->sig_probes, 0, 2 * sizeof(unsigned long long), st));
    CUDA_TRY(launch_batch_layout(d_jobs, d_js, n, d_bh, st));
    CUDA_TRY(cudaEventRecord(c0->ev[2], st));
    CUDA_TRY(launch_sigma_batch(d_jobs, d_js, n, d_bh, c0->full_grid(), st));
    CUDA_TRY(cudaEventRecord(c0->ev[3], st));
    UCC_TRY(fetch());
    for (int x = 0; x < n; ++x) {
      ucc_ctx* c = jobs[idx[x]];
      E[idx[x]] = hs[x].e_num / hs[x].norm2 + c->e_nuc;
      c->launches += 3;
    }
    if (record) {
      CUDA_TRY(launch_lambda_init_batch(d_jobs, d_js, n, d_bh, c0->full_grid(), st));
      for (int x = 0; x < n; ++x) {
        hs[x].k = jobs[idx[x]]->K - 1;
        hs[x].gacc = 0.0;
      }
      CUDA_TRY(cudaMemcpyAsync(d_js, hs.data(), n * sizeof(JobState), cudaMemcpyHostToDevice, st));
      g_rev = capture_one(st, [&]() { return launch_persist_reverse(d_jobs, d_js, n, d_bh, pw, tiles, st); });
      UCC_TRY(reset_header(-1));
      CUDA_TRY(cudaEventRecord(c0->ev[4], st));
      if (g_rev)
        CUDA_TRY(cudaGraphLaunch(g_rev, st));
      else
        CUDA_TRY(launch_persist_reverse(d_jobs, d_js, n, d_bh, pw, tiles, st));
      CUDA_TRY(cudaEventRecord(c0->ev[5], st));
      UCC_TRY(fetch());
      if (hb.error & 1) return fail(UCC_ETIMEOUT, "a grid barrier of the persistent batch timed out");
      if (hb.error) return fail(UCC_ECAPACITY, "a batched job outgrew the table it was given");
      UCC_TRY(sync_swaps());
      for (int x = 0; x < n; ++x) {
        ucc_ctx* c = jobs[idx[x]];
        if (hs[x].k != -1) return fail(UCC_ECUDA, "batched reverse sweep did not finish");
        if (c->K && grads[idx[x]])
          CUDA_TRY(cudaMemcpyAsync(grads[idx[x]], c->d_grad, c->K * sizeof(double), cudaMemcpyDeviceToHost, st));
        c->launches += 2;
        c->stats.reverse_launches = 1;
      }
    }
    float ms = 0.f;
    for (int x = 0; x < n; ++x) {
      ucc_ctx* c = jobs[idx[x]];
      UCC_TRY(read_counters(c, c->ts[0]));
      c->stats.sigma_probes = (long long)c->ts[0].h_cnt->sig_probes;
      c->stats.sigma_hits = (long long)c->ts[0].h_cnt->sig_hits;
      c->stats.reverse_pairs = (long long)c->ts[0].h_cnt->rev_pairs;
      c->stats.reverse_scanned = (long long)c->ts[0].h_cnt->rev_scanned;
      c->stats.kernel_launches = c->launches;
      c->have_psi = !record;
      c->have_sigma = !record;
    }
    CUDA_TRY(cudaEventElapsedTime(&ms, c0->ev[0], c0->ev[1]));
    c0->stats.apply_ms = ms;
    CUDA_TRY(cudaEventElapsedTime(&ms, c0->ev[2], c0->ev[3]));
    c0->stats.energy_ms = ms;
    if (record) {
      CUDA_TRY(cudaEventElapsedTime(&ms, c0->ev[4], c0->ev[5]));
      c0->stats.reverse_ms = ms;
    }
    c0->stats.probe_width = pw;
    for (int x = 0; x < n; ++x) jobs[idx[x]]->stats.batch_tiles = tiles;
    return UCC_OK;
  };
  ucc_status s = run();
  if (s != UCC_OK) {
    // leave the host view consistent with the device arrays
    std::string msg = g_last_error;
    sync_swaps();
    g_last_error = msg;
  }
  release();
  return s;
}

// The batch runs on a private stream (graph capture needs one that is not
// the legacy default stream), ordered after and before the caller's stream.
ucc_status batch_together(const std::vector<int>& idx, ucc_ctx* const* jobs, double eps, double* E,
                          double* const* grads) {
  cudaStream_t caller = jobs[idx[0]]->stream;
  cudaStream_t bs = nullptr;
  cudaEvent_t e_in = nullptr, e_out = nullptr;
  CUDA_TRY(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  if (cudaEventCreateWithFlags(&e_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaStreamDestroy(bs);
    return fail(UCC_ECUDA, "event creation failed");
  }
  cudaEventRecord(e_in, caller);
  cudaStreamWaitEvent(bs, e_in, 0);
  for (int j : idx) jobs[j]->stream = bs;
  ucc_status s = batch_persistent(idx, jobs, eps, E, grads);
  for (int j : idx) jobs[j]->stream = caller;
  cudaEventRecord(e_out, bs);
  cudaStreamWaitEvent(caller, e_out, 0);
  cudaStreamSynchronize(bs);
  cudaEventDestroy(e_in);
  cudaEventDestroy(e_out);
  cudaStreamDestroy(bs);
  return s;
}

}  // namespace

extern "C" {

ucc_status ucc_create(const ucc_hamiltonian* ham, const ucc_ansatz* an, void* cuda_stream, ucc_ctx** out) {
  if (!out) return fail(UCC_EINVAL, "null out pointer");
  *out = nullptr;
  UCC_TRY(validate_problem(ham, an));
  ucc_ctx* c = new ucc_ctx;
  auto bail = [&](ucc_status s) {
    std::string msg = g_last_error;
    destroy(c);
    g_last_error = msg;
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(fail(UCC_ECUDA, "no CUDA device"));
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return bail(fail(UCC_ECUDA, "device query failed"));
  c->num_sms = prop.multiProcessorCount;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess) {
    c->side = nullptr;
    return bail(fail(UCC_ECUDA, "stream creation failed"));
  }
  c->n_spatial = ham->n_spatial;
  c->n_alpha = ham->n_alpha;
  c->n_beta = ham->n_beta;
  c->n_so = 2 * ham->n_spatial;
  c->e_nuc = ham->e_nuc;
  c->K = an->n_exc;
  c->rows.assign(an->idx, an->idx + 4 * (size_t)c->K);
  c->theta.assign(c->K, 0.0);
  if (an->theta) std::copy(an->theta, an->theta + c->K, c->theta.begin());
  c->wide = c->n_so > 64;
  c->kw = c->wide ? 2 : 1;
  for (auto& t : c->ts) t.cur.kw = t.spare.kw = c->kw;
  if (c->wide)
    c->factors_w.resize(c->K);
  else
    c->factors.resize(c->K);
  const size_t n = (size_t)c->n_spatial;
  ucc_status s;
  const size_t fbytes = c->wide ? sizeof(FactorT<Key128>) : sizeof(Factor);
  const size_t cbytes = c->wide ? sizeof(SelectCandT<Key128>) : sizeof(SelectCand);
  unsigned char* fb = nullptr;
  unsigned char* cb = nullptr;
  if ((s = dalloc(&fb, fbytes * (size_t)std::max(1, c->K))) != UCC_OK) return bail(s);
  c->d_factors = fb;
  if ((s = dalloc(&cb, cbytes * kSelectCandCap)) != UCC_OK) return bail(s);
  c->d_cand = cb;
  if ((s = dalloc(&c->d_h, n * n)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_g, n * n * n * n)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_grad, std::max(1, c->K))) != UCC_OK) return bail(s);
  if ((s = c->ts[0].init()) != UCC_OK) return bail(s);
  if ((s = c->ts[1].init()) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_sel, 1)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->t_off, (size_t)c->K + 1)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_pages, kTapeMaxPages)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_entropy, std::max(1, c->K))) != UCC_OK) return bail(s);
  if ((s = ensure_partials(c, c->full_grid())) != UCC_OK) return bail(s);
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(UCC_ECUDA, "event creation failed"));
  for (auto& e : c->kev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(fail(UCC_ECUDA, "event creation failed"));
  if (cudaMemcpyAsync(c->d_h, ham->h, n * n * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->d_g, ham->g, n * n * n * n * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess)
    return bail(fail(UCC_ECUDA, "integral upload failed"));
  if ((s = upload_factors(c)) != UCC_OK) return bail(s);
  *out = c;
  return UCC_OK;
}

ucc_status ucc_set_theta(ucc_ctx* c, const double* theta, int on_device) {
  if (!c || !theta) return fail(UCC_EINVAL, "null argument");
  if (c->K == 0) return UCC_OK;
  if (on_device) {
    CUDA_TRY(cudaMemcpyAsync(c->theta.data(), theta, c->K * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  } else {
    std::copy(theta, theta + c->K, c->theta.begin());
  }
  for (int k = 0; k < c->K; ++k)
    if (!std::isfinite(c->theta[k])) return fail(UCC_EINVAL, "theta is not finite");
  UCC_TRY(upload_factors(c));
  c->have_psi = false;
  return UCC_OK;
}

ucc_status ucc_set_options(ucc_ctx* c, const ucc_options* opt) {
  if (!c) return fail(UCC_EINVAL, "null context");
  ucc_options o{};
  if (opt) o = *opt;
  if (o.n_max < 0 || o.n_cut < 0 || o.max_entries < 0) return fail(UCC_EINVAL, "negative option");
  if (o.n_max > 0 && (o.n_cut <= 0 || o.n_cut > o.n_max)) return fail(UCC_EINVAL, "need 0 < n_cut <= n_max");
  if (o.probe_width != 0 && o.probe_width != 1 && o.probe_width != 2 && o.probe_width != 4 && o.probe_width != 8)
    return fail(UCC_EINVAL, "probe_width must be 0, 1, 2, 4 or 8");
  if (o.batch_wait_ms < 0 || o.batch_test_skip_block < 0) return fail(UCC_EINVAL, "negative option");
  if (o.batch_tiles != 0 && o.batch_tiles != 1 && o.batch_tiles != 2 && o.batch_tiles != 4 && o.batch_tiles != 8)
    return fail(UCC_EINVAL, "batch_tiles must be 0, 1, 2, 4 or 8");
  if (o.energy_route < 0 || o.energy_route > 2) return fail(UCC_EINVAL, "energy_route must be 0, 1 or 2");
  if (o.energy_test_partitions < 0 || (o.energy_test_partitions & (o.energy_test_partitions - 1)) != 0 ||
      o.energy_test_partitions > (1 << 24))
    return fail(UCC_EINVAL, "energy_test_partitions must be 0 or a power of two up to 2^24");
  if (o.energy_test_buffer_records < 0) return fail(UCC_EINVAL, "negative option");
  if (o.rebuild_test_regions < 0 || o.rebuild_test_regions > 2)
    return fail(UCC_EINVAL, "rebuild_test_regions must be 0, 1 or 2");
  c->opt = o;
  return UCC_OK;
}

ucc_status ucc_apply(ucc_ctx* c, double eps) {
  if (!c) return fail(UCC_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  c->launches = 0;
  drop_timings(c);
  c->stats = ucc_stats{};
  UCC_TRY(c->wide ? run_forward<Key128>(c, eps, false) : run_forward<unsigned long long>(c, eps, false));
  c->stats.kernel_launches = c->launches;
  return UCC_OK;
}

ucc_status ucc_energy(ucc_ctx* c, double* E, double* norm2) {
  if (!c) return fail(UCC_EINVAL, "null context");
  if (!c->have_psi) return fail(UCC_ESTATE, "no wavefunction held: call ucc_apply first");
  CUDA_TRY(cudaSetDevice(c->device));
  long long before = c->launches;
  UCC_TRY(c->wide ? run_energy<Key128>(c, E, norm2) : run_energy<unsigned long long>(c, E, norm2));
  c->stats.kernel_launches = c->launches - before;
  return UCC_OK;
}

ucc_status ucc_gradient(ucc_ctx* c, double eps, double* E, double* grad, int on_device) {
  if (!c) return fail(UCC_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  return c->wide ? run_gradient<Key128>(c, eps, E, grad, on_device)
                 : run_gradient<unsigned long long>(c, eps, E, grad, on_device);
}

ucc_status ucc_get_wavefunction(ucc_ctx* c, size_t cap, size_t* n, uint64_t* keys, double* amps, double* sigma,
                                int on_device) {
  if (!c || !n) return fail(UCC_EINVAL, "null argument");
  if (!c->have_psi) return fail(UCC_ESTATE, "no wavefunction held: call ucc_apply first");
  if (sigma && !c->have_sigma) return fail(UCC_ESTATE, "no sigma held: call ucc_energy first");
  CUDA_TRY(cudaSetDevice(c->device));
  TableSet& tab = c->ts[c->main];
  UCC_TRY(read_counters(c, tab));
  const unsigned long long live = tab.h_cnt->n_tail - tab.h_cnt->n_dead;
  *n = (size_t)live;
  if (cap < live) return fail(UCC_ECAPACITY, "buffer smaller than the wavefunction");
  if (live == 0) return UCC_OK;
  if (!keys || !amps) return fail(UCC_EINVAL, "null output buffer");
  unsigned long long* dk = (unsigned long long*)keys;
  double* da = amps;
  double* ds = sigma;
  unsigned long long* tk = nullptr;
  double* ta = nullptr;
  double* tsig = nullptr;
  if (!on_device) {
    UCC_TRY(dalloc(&tk, live * c->kw));
    UCC_TRY(dalloc(&ta, live));
    if (sigma) UCC_TRY(dalloc(&tsig, live));
    dk = tk;
    da = ta;
    ds = tsig;
  }
  CUDA_TRY(cudaMemsetAsync(&tab.d_cnt->new_n, 0, sizeof(unsigned long long), c->stream));
  if (c->wide)
    CUDA_TRY(launch_export(c->template table<Key128>(tab), live, reinterpret_cast<Key128*>(dk), da, ds,
                           c->full_grid(), c->stream));
  else
    CUDA_TRY(launch_export(c->template table<unsigned long long>(tab), live, dk, da, ds, c->full_grid(), c->stream));
  if (!on_device) {
    CUDA_TRY(cudaMemcpyAsync(keys, tk, live * c->kw * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(amps, ta, live * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (sigma) CUDA_TRY(cudaMemcpyAsync(sigma, tsig, live * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  ucc_status s = read_counters(c, tab);
  dfree(tk);
  dfree(ta);
  dfree(tsig);
  UCC_TRY(s);
  if (tab.h_cnt->new_n != live) return fail(UCC_ECUDA, "export count mismatch");
  return UCC_OK;
}

ucc_status ucc_get_entropy(ucc_ctx* c, double* S, int32_t n) {
  if (!c || (!S && n > 0)) return fail(UCC_EINVAL, "null argument");
  if (n != c->K) return fail(UCC_EINVAL, "n must equal the number of factors");
  if (!c->have_entropy) return fail(UCC_ESTATE, "no entropy recorded: set record_entropy and call ucc_apply");
  if (n == 0) return UCC_OK;
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaMemcpyAsync(S, c->d_entropy, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return UCC_OK;
}

ucc_status ucc_get_stats(const ucc_ctx* c, ucc_stats* out) {
  if (!c || !out) return fail(UCC_EINVAL, "null argument");
  *out = c->stats;
  return UCC_OK;
}

ucc_status ucc_batch_run(int n_jobs, ucc_ctx* const* jobs, double eps, double* E, double* const* grads) {
  if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !E))) return fail(UCC_EINVAL, "bad batch arguments");
  if (n_jobs == 0) return UCC_OK;
  if (!(eps >= 0.0) || std::isinf(eps)) return fail(UCC_EINVAL, "eps must be finite and >= 0");
  for (int j = 0; j < n_jobs; ++j) {
    if (!jobs[j]) return fail(UCC_EINVAL, "null job");
    if (jobs[j]->device != jobs[0]->device || jobs[j]->stream != jobs[0]->stream)
      return fail(UCC_EINVAL, "batched jobs must share one device and one stream");
  }
  CUDA_TRY(cudaSetDevice(jobs[0]->device));
  // Jobs whose table cannot be sized up front (no cut and a large sector)
  // run one by one; the rest share the persistent launches.
  std::vector<int> together;
  for (int j = 0; j < n_jobs; ++j) {
    ucc_ctx* c = jobs[j];
    if (batch_capacity(c) == 0 || together.size() >= (size_t)kMaxBatchJobs) {
      if (grads && grads[j]) {
        UCC_TRY(c->wide ? run_gradient<Key128>(c, eps, &E[j], grads[j], 0)
                        : run_gradient<unsigned long long>(c, eps, &E[j], grads[j], 0));
      } else {
        c->launches = 0;
        drop_timings(c);
        c->stats = ucc_stats{};
        if (c->wide) {
          UCC_TRY(run_forward<Key128>(c, eps, false));
          UCC_TRY(run_energy<Key128>(c, &E[j], nullptr));
        } else {
          UCC_TRY(run_forward<unsigned long long>(c, eps, false));
          UCC_TRY(run_energy<unsigned long long>(c, &E[j], nullptr));
        }
      }
    } else {
      together.push_back(j);
    }
  }
  if (together.empty()) return UCC_OK;
  return batch_together(together, jobs, eps, E, grads);
}

const char* ucc_last_error(void) { return g_last_error.c_str(); }

void ucc_destroy(ucc_ctx* c) { destroy(c); }

}  // extern "C"
