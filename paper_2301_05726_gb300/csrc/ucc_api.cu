// Host runtime behind include/ucc.h: validation, device buffers, capacity
// management and the launch sequences of apply / energy / gradient.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
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
struct Arrays {
  unsigned long long cap_n = 0, n_slots = 0;
  unsigned long long* keys = nullptr;
  double* amps = nullptr;
  unsigned int* born = nullptr;
  double* lam = nullptr;
  double* sigma = nullptr;
  Slot* slots = nullptr;
  void release() {
    dfree(keys);
    dfree(amps);
    dfree(born);
    dfree(lam);
    dfree(sigma);
    dfree(slots);
    cap_n = n_slots = 0;
  }
  ucc_status allocate(unsigned long long cn, unsigned long long ns) {
    release();
    UCC_TRY(dalloc(&keys, cn));
    UCC_TRY(dalloc(&amps, cn));
    UCC_TRY(dalloc(&born, cn));
    UCC_TRY(dalloc(&lam, cn));
    UCC_TRY(dalloc(&sigma, cn));
    UCC_TRY(dalloc(&slots, ns));
    cap_n = cn;
    n_slots = ns;
    return UCC_OK;
  }
};

}  // namespace

struct ucc_ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  int n_spatial = 0, n_alpha = 0, n_beta = 0, n_so = 0;
  double e_nuc = 0.0;
  int K = 0;
  std::vector<int> rows;         // K x 4
  std::vector<double> theta;     // K
  std::vector<Factor> factors;   // host copy
  ucc_options opt{};

  Factor* d_factors = nullptr;
  double* d_h = nullptr;
  double* d_g = nullptr;
  double* d_grad = nullptr;
  double* d_partials = nullptr;
  int partial_cap = 0;
  Counters* d_cnt = nullptr;
  Counters* h_cnt = nullptr;  // pinned mirror
  SelectState* d_sel = nullptr;
  Arrays cur, spare;
  // kill tape
  unsigned long long* t_key = nullptr;
  double* t_val = nullptr;
  unsigned int* t_born = nullptr;
  unsigned long long* t_off = nullptr;  // K + 1
  unsigned long long tape_cap = 0;

  bool have_psi = false;
  bool have_sigma = false;
  cudaEvent_t ev[6] = {};
  ucc_stats stats{};
  int probe_width = 1;
  long long launches = 0;

  Table table() const {
    Table t;
    t.keys = cur.keys;
    t.amps = cur.amps;
    t.born = cur.born;
    t.lam = cur.lam;
    t.sigma = cur.sigma;
    t.slots = cur.slots;
    t.slot_mask = cur.n_slots - 1;
    t.cap_n = cur.cap_n;
    t.cnt = d_cnt;
    t.partials = d_partials;
    return t;
  }
  Tape tape() const {
    Tape tp;
    tp.key = t_key;
    tp.val = t_val;
    tp.born = t_born;
    tp.off = t_off;
    tp.cap = tape_cap;
    return tp;
  }
  int full_grid(int per_sm = 8) const { return std::max(1, num_sms * per_sm); }
};

namespace {

// Jordan-Wigner sign mask of tau = a+_a a+_b a_j a_i acting on a determinant
// E that it excites: the four operators count occupied modes below i, j, b, a
// in the running determinant; relative to E those counts shift by the index
// comparisons below, so parity = popc(E & pmask) + pconst (mod 2).
Factor make_factor(int i, int j, int a, int b, double th) {
  auto below = [](int p) { return p <= 0 ? 0ull : ((1ull << p) - 1ull); };
  Factor f{};
  if (j < 0) {
    f.occ = 1ull << i;
    f.vir = 1ull << a;
    f.pmask = below(i) ^ below(a);
    f.pconst = (i < a) ? 1 : 0;
    f.is_double = 0;
  } else {
    f.occ = (1ull << i) | (1ull << j);
    f.vir = (1ull << a) | (1ull << b);
    f.pmask = below(i) ^ below(j) ^ below(a) ^ below(b);
    f.pconst = ((i < j) + (i < b) + (j < b) + (i < a) + (j < a) + (b < a)) & 1;
    f.is_double = 1;
  }
  f.c = std::cos(th);
  f.s = std::sin(th);
  return f;
}

ucc_status check_device_error(ucc_ctx* c) {
  int err = c->h_cnt->error;
  if (!err) return UCC_OK;
  std::string msg = "device error word:";
  if (err & ERR_PROBE_BOUND) msg += " probe-bound";
  if (err & ERR_CONSISTENCY) msg += " consistency";
  if (err & ERR_TAPE_FULL) msg += " tape-full";
  if (err & ERR_CAPACITY) msg += " capacity";
  return fail((err & (ERR_CAPACITY | ERR_TAPE_FULL)) ? UCC_ECAPACITY : UCC_ECUDA, msg);
}

ucc_status read_counters(ucc_ctx* c) {
  CUDA_TRY(cudaMemcpyAsync(c->h_cnt, c->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
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

// Copy live entries into arrays of capacity new_cap (dropping dead entries) and
// rebuild the hash.  Counters are updated on the device.
ucc_status rebuild(ucc_ctx* c, unsigned long long new_cap) {
  if (c->opt.max_entries > 0 && new_cap > 2ull * (unsigned long long)c->opt.max_entries)
    new_cap = std::max<unsigned long long>(2ull * (unsigned long long)c->opt.max_entries, 64);
  unsigned long long ns = slots_for(new_cap);
  if (c->spare.cap_n != new_cap || c->spare.n_slots != ns) {
    c->spare.release();
    ucc_status s = c->spare.allocate(new_cap, ns);
    if (s != UCC_OK) {
      c->spare.release();
      return fail(UCC_ECAPACITY, "cannot allocate " + std::to_string(new_cap) + " entries: " + g_last_error);
    }
  }
  Table from = c->table();
  Table to = from;
  to.keys = c->spare.keys;
  to.amps = c->spare.amps;
  to.born = c->spare.born;
  to.lam = c->spare.lam;
  to.sigma = c->spare.sigma;
  to.slots = c->spare.slots;
  to.slot_mask = ns - 1;
  to.cap_n = new_cap;
  CUDA_TRY(cudaMemsetAsync(&c->d_cnt->new_n, 0, sizeof(unsigned long long), c->stream));
  CUDA_TRY(cudaMemsetAsync(to.slots, 0, ns * sizeof(Slot), c->stream));
  int grid = c->full_grid();
  CUDA_TRY(launch_compact(from, to, 1, grid, c->stream));
  CUDA_TRY(launch_rehash(to, grid, c->stream));
  CUDA_TRY(launch_finish_rebuild(to, c->stream));
  c->launches += 3;
  std::swap(c->cur, c->spare);
  c->stats.rebuilds++;
  return UCC_OK;
}

ucc_status ensure_tape(ucc_ctx* c, unsigned long long need) {
  if (need <= c->tape_cap) return UCC_OK;
  unsigned long long cap = std::max<unsigned long long>(need, 2 * c->tape_cap);
  cap = std::max<unsigned long long>(cap, 1 << 16);
  unsigned long long* nk = nullptr;
  double* nv = nullptr;
  unsigned int* nb = nullptr;
  UCC_TRY(dalloc(&nk, cap));
  UCC_TRY(dalloc(&nv, cap));
  UCC_TRY(dalloc(&nb, cap));
  if (c->tape_cap) {
    CUDA_TRY(cudaMemcpyAsync(nk, c->t_key, c->tape_cap * sizeof(*nk), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(nv, c->t_val, c->tape_cap * sizeof(*nv), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(nb, c->t_born, c->tape_cap * sizeof(*nb), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  }
  dfree(c->t_key);
  dfree(c->t_val);
  dfree(c->t_born);
  c->t_key = nk;
  c->t_val = nv;
  c->t_born = nb;
  c->tape_cap = cap;
  return UCC_OK;
}

ucc_status reset_state(ucc_ctx* c, bool record) {
  if (c->cur.cap_n == 0) UCC_TRY(c->cur.allocate(1 << 12, slots_for(1 << 12)));
  CUDA_TRY(cudaMemsetAsync(c->d_cnt, 0, sizeof(Counters), c->stream));
  CUDA_TRY(cudaMemsetAsync(c->cur.slots, 0, c->cur.n_slots * sizeof(Slot), c->stream));
  unsigned long long hf = 0;
  for (int s = 0; s < c->n_alpha; ++s) hf |= 1ull << (2 * s);
  for (int s = 0; s < c->n_beta; ++s) hf |= 1ull << (2 * s + 1);
  CUDA_TRY(launch_reset(c->table(), hf, c->stream));
  c->launches++;
  if (record) {
    UCC_TRY(ensure_tape(c, 1 << 16));
    CUDA_TRY(cudaMemsetAsync(c->t_off, 0, sizeof(unsigned long long), c->stream));
  }
  c->have_psi = false;
  c->have_sigma = false;
  return UCC_OK;
}

int pick_probe_width(ucc_ctx* c) {
  int pw = c->opt.probe_width;
  if (pw == 1 || pw == 2 || pw == 4 || pw == 8) return pw;
  return c->probe_width;
}

// Make room for the next factor: it may append one entry per stored entry
// (and, in gradient runs, drop as many onto the tape).  Compacts when a
// quarter of the stored entries are dropped ones.
ucc_status ensure_room(ucc_ctx* c, bool record) {
  UCC_TRY(read_counters(c));
  const Counters h = *c->h_cnt;  // copy: later reads overwrite the mirror
  const unsigned long long live = h.n_tail - h.n_dead;
  if (c->opt.max_entries > 0 && live > (unsigned long long)c->opt.max_entries)
    return fail(UCC_ECAPACITY, "wavefunction exceeds max_entries (" + std::to_string(live) + " live)");
  const bool room = 2 * h.n_tail <= c->cur.cap_n && 8 * h.n_tail <= 3 * c->cur.n_slots;
  const bool sparse = h.n_dead > 4096 && h.n_dead * 4 > h.n_tail;
  if (record) UCC_TRY(ensure_tape(c, h.tape_n + 2 * live + (1 << 12)));
  if (!room || sparse) {
    unsigned long long cap = c->cur.cap_n;
    if (2 * live > cap || 8 * live > 3 * c->cur.n_slots) cap = std::max<unsigned long long>(4 * live, 1 << 12);
    UCC_TRY(rebuild(c, cap));
    UCC_TRY(read_counters(c));
  }
  return UCC_OK;
}

// Factors [0, K) on the reference.  The last block of each factor flags a
// stop when the next factor might not fit or when the Methods-section cut is
// due; later launches in the chunk then skip, and the host cuts / grows and
// resumes at the flagged factor.
ucc_status run_forward(ucc_ctx* c, double eps, bool record) {
  if (!(eps >= 0.0) || std::isinf(eps)) return fail(UCC_EINVAL, "eps must be finite and >= 0");
  UCC_TRY(reset_state(c, record));
  const int pw = pick_probe_width(c);
  const int chunk = 64;
  const unsigned long long n_max = c->opt.n_max > 0 ? (unsigned long long)c->opt.n_max : 0ull;
  int k = 0;
  unsigned long long n_known = 1;
  long long cut_total = 0;
  CUDA_TRY(cudaEventRecord(c->ev[0], c->stream));
  while (k < c->K) {
    int end = std::min(c->K, k + chunk);
    // Grid sized from the last known count (grid-stride loops stay correct if
    // the table grew since).
    unsigned long long est = std::min<unsigned long long>(n_known * 4, c->cur.cap_n);
    int grid = (int)std::min<unsigned long long>((unsigned long long)c->full_grid(), (est + 255) / 256);
    grid = std::max(grid, std::min(c->full_grid(), 4));
    if (k < 0 || end > c->K) return fail(UCC_ECUDA, "factor index out of range");
    for (int kk = k; kk < end; ++kk) {
      CUDA_TRY(launch_forward(c->table(), c->d_factors, kk, eps, (unsigned int)(kk + 1), record ? 1 : 0, c->tape(),
                              n_max, pw, grid, c->stream));
      c->launches++;
    }
    UCC_TRY(read_counters(c));
    const Counters h = *c->h_cnt;  // copy: later reads overwrite the mirror
    n_known = h.n_tail;
    c->stats.peak_entries = std::max<long long>(c->stats.peak_entries, (long long)h.n_tail);
    if (h.stop_k >= 0) {
      const int resume = h.stop_k;
      if (resume <= k || resume > end) return fail(UCC_ECUDA, "invalid resume factor");
      if (h.cut_pending) {
        const unsigned long long before = h.n_tail - h.n_dead;
        CUDA_TRY(launch_select_cut(c->table(), c->d_sel, (unsigned long long)c->opt.n_cut, (unsigned int)resume,
                                   record ? 1 : 0, c->tape(), resume - 1, c->full_grid(), c->stream, &c->launches));
        UCC_TRY(read_counters(c));
        const unsigned long long after = c->h_cnt->n_tail - c->h_cnt->n_dead;
        if (after != (unsigned long long)c->opt.n_cut)
          return fail(UCC_ECUDA, "truncation kept " + std::to_string(after) + " entries, expected " +
                                     std::to_string(c->opt.n_cut));
        cut_total += (long long)(before - after);
      }
      UCC_TRY(ensure_room(c, record));
      const int minus_one = -1, zero = 0;
      CUDA_TRY(cudaMemcpyAsync(&c->d_cnt->stop_k, &minus_one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
      CUDA_TRY(cudaMemcpyAsync(&c->d_cnt->cut_pending, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
      UCC_TRY(read_counters(c));
      n_known = c->h_cnt->n_tail;
      k = resume;
      continue;
    }
    // Compact when a quarter of the stored entries are dropped ones.
    if (h.n_dead > 4096 && h.n_dead * 4 > h.n_tail) UCC_TRY(rebuild(c, c->cur.cap_n));
    k = end;
  }
  CUDA_TRY(cudaEventRecord(c->ev[1], c->stream));
  UCC_TRY(read_counters(c));
  const Counters h = *c->h_cnt;  // copy: later reads overwrite the mirror
  c->stats.n_det = (long long)(h.n_tail - h.n_dead);
  c->stats.rotations = (long long)h.rotations;
  c->stats.created = (long long)h.created;
  c->stats.dropped_new = (long long)h.dropped_new;
  c->stats.dropped_old = (long long)h.dropped_old;
  c->stats.cut = cut_total;
  c->stats.tape_entries = (long long)h.tape_n;
  c->stats.scanned = (long long)h.scanned;
  c->stats.capacity_entries = (long long)c->cur.cap_n;
  c->stats.hash_slots = (long long)c->cur.n_slots;
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  c->stats.apply_ms = ms;
  c->have_psi = true;
  return UCC_OK;
}

ucc_status run_energy(ucc_ctx* c, double* E, double* norm2) {
  Integrals in;
  in.h = c->d_h;
  in.g = c->d_g;
  in.n = c->n_spatial;
  in.n_so = c->n_so;
  unsigned long long n = c->h_cnt->n_tail;
  int grid = (int)std::min<unsigned long long>((unsigned long long)c->full_grid(), (n + 7) / 8);
  grid = std::max(grid, 1);
  UCC_TRY(ensure_partials(c, c->full_grid()));
  CUDA_TRY(cudaMemsetAsync(&c->d_cnt->sig_probes, 0, 2 * sizeof(unsigned long long), c->stream));
  CUDA_TRY(cudaEventRecord(c->ev[2], c->stream));
  CUDA_TRY(launch_sigma(c->table(), in, grid, c->stream));
  c->launches++;
  CUDA_TRY(cudaEventRecord(c->ev[3], c->stream));
  UCC_TRY(read_counters(c));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
  c->stats.energy_ms = ms;
  c->stats.sigma_probes = (long long)c->h_cnt->sig_probes;
  c->stats.sigma_hits = (long long)c->h_cnt->sig_hits;
  const double n2 = c->h_cnt->norm2;
  if (norm2) *norm2 = n2;
  if (E) *E = c->h_cnt->e_num / n2 + c->e_nuc;
  c->have_sigma = true;
  return UCC_OK;
}

ucc_status run_gradient(ucc_ctx* c, double eps, double* E, double* grad_out, int on_device) {
  c->launches = 0;
  c->stats = ucc_stats{};
  UCC_TRY(run_forward(c, eps, true));
  {
    // The reverse sweep re-inserts up to tape_n entries: make room now, before
    // sigma and lambda are laid out against the entry indices.
    const Counters h = *c->h_cnt;  // copy: later reads overwrite the mirror
    const unsigned long long live = h.n_tail - h.n_dead;
    const unsigned long long need = h.n_tail + h.tape_n;
    if (need > c->cur.cap_n || 4ull * need > 3ull * c->cur.n_slots) {
      UCC_TRY(rebuild(c, std::max<unsigned long long>(c->cur.cap_n, 2 * (live + h.tape_n) + 64)));
      UCC_TRY(read_counters(c));
    }
  }
  double e = 0.0, n2 = 0.0;
  UCC_TRY(run_energy(c, &e, &n2));
  if (E) *E = e;
  const int grid_full = c->full_grid();
  CUDA_TRY(cudaEventRecord(c->ev[4], c->stream));
  CUDA_TRY(launch_lambda_init(c->table(), grid_full, c->stream));
  c->launches++;
  // Tape offsets of every factor.
  std::vector<unsigned long long> off(c->K + 1);
  CUDA_TRY(cudaMemcpyAsync(off.data(), c->t_off, (c->K + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int pw = pick_probe_width(c);
  unsigned long long n_now = c->h_cnt->n_tail;
  int grid = (int)std::min<unsigned long long>((unsigned long long)grid_full, (n_now * 2 + 255) / 256);
  grid = std::max(grid, std::min(grid_full, 4));
  UCC_TRY(ensure_partials(c, grid_full));
  for (int k = c->K - 1; k >= 0; --k) {
    const unsigned int stamp = 0x80000000u | (unsigned int)k;
    if (off[k + 1] > off[k]) {
      int g2 = (int)std::min<unsigned long long>((unsigned long long)grid_full, (off[k + 1] - off[k] + 255) / 256);
      CUDA_TRY(launch_tape_reinsert(c->table(), c->tape(), k, std::max(g2, 1), c->stream));
      c->launches++;
    }
    CUDA_TRY(launch_reverse(c->table(), c->d_factors, k, stamp, c->d_grad, pw, grid, c->stream));
    c->launches++;
  }
  CUDA_TRY(cudaEventRecord(c->ev[5], c->stream));
  if (grad_out) {
    CUDA_TRY(cudaMemcpyAsync(grad_out, c->d_grad, c->K * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  UCC_TRY(read_counters(c));
  float ms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
  c->stats.reverse_ms = ms;
  c->stats.reverse_pairs = (long long)c->h_cnt->rev_pairs;
  c->stats.kernel_launches = c->launches;
  c->have_psi = false;
  c->have_sigma = false;
  return UCC_OK;
}

ucc_status validate_problem(const ucc_hamiltonian* ham, const ucc_ansatz* an) {
  if (!ham || !an) return fail(UCC_EINVAL, "null hamiltonian or ansatz");
  const int n = ham->n_spatial;
  if (n < 1 || n > 32) return fail(UCC_EINVAL, "n_spatial must be in [1, 32] (64-bit determinant keys)");
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
    c->factors[k] = make_factor(r[0], r[1], r[2], r[3], c->theta[k]);
  }
  if (c->K)
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
  c->cur.release();
  c->spare.release();
  dfree(c->d_factors);
  dfree(c->d_h);
  dfree(c->d_g);
  dfree(c->d_grad);
  dfree(c->d_partials);
  dfree(c->d_cnt);
  dfree(c->d_sel);
  dfree(c->t_key);
  dfree(c->t_val);
  dfree(c->t_born);
  dfree(c->t_off);
  if (c->h_cnt) cudaFreeHost(c->h_cnt);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  delete c;
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
  c->n_spatial = ham->n_spatial;
  c->n_alpha = ham->n_alpha;
  c->n_beta = ham->n_beta;
  c->n_so = 2 * ham->n_spatial;
  c->e_nuc = ham->e_nuc;
  c->K = an->n_exc;
  c->rows.assign(an->idx, an->idx + 4 * (size_t)c->K);
  c->theta.assign(c->K, 0.0);
  if (an->theta) std::copy(an->theta, an->theta + c->K, c->theta.begin());
  c->factors.resize(c->K);
  const size_t n = (size_t)c->n_spatial;
  ucc_status s;
  if ((s = dalloc(&c->d_factors, std::max(1, c->K))) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_h, n * n)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_g, n * n * n * n)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_grad, std::max(1, c->K))) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_cnt, 1)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->d_sel, 1)) != UCC_OK) return bail(s);
  if ((s = dalloc(&c->t_off, (size_t)c->K + 1)) != UCC_OK) return bail(s);
  if ((s = ensure_partials(c, c->full_grid())) != UCC_OK) return bail(s);
  if (cudaMallocHost((void**)&c->h_cnt, sizeof(Counters)) != cudaSuccess)
    return bail(fail(UCC_ENOMEM, "pinned host allocation failed"));
  std::memset(c->h_cnt, 0, sizeof(Counters));
  for (auto& e : c->ev)
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
  c->opt = o;
  return UCC_OK;
}

ucc_status ucc_apply(ucc_ctx* c, double eps) {
  if (!c) return fail(UCC_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  c->launches = 0;
  c->stats = ucc_stats{};
  UCC_TRY(run_forward(c, eps, false));
  c->stats.kernel_launches = c->launches;
  return UCC_OK;
}

ucc_status ucc_energy(ucc_ctx* c, double* E, double* norm2) {
  if (!c) return fail(UCC_EINVAL, "null context");
  if (!c->have_psi) return fail(UCC_ESTATE, "no wavefunction held: call ucc_apply first");
  CUDA_TRY(cudaSetDevice(c->device));
  long long before = c->launches;
  UCC_TRY(run_energy(c, E, norm2));
  c->stats.kernel_launches = c->launches - before;
  return UCC_OK;
}

ucc_status ucc_gradient(ucc_ctx* c, double eps, double* E, double* grad, int on_device) {
  if (!c) return fail(UCC_EINVAL, "null context");
  CUDA_TRY(cudaSetDevice(c->device));
  return run_gradient(c, eps, E, grad, on_device);
}

ucc_status ucc_get_wavefunction(ucc_ctx* c, size_t cap, size_t* n, uint64_t* keys, double* amps, double* sigma,
                                int on_device) {
  if (!c || !n) return fail(UCC_EINVAL, "null argument");
  if (!c->have_psi) return fail(UCC_ESTATE, "no wavefunction held: call ucc_apply first");
  if (sigma && !c->have_sigma) return fail(UCC_ESTATE, "no sigma held: call ucc_energy first");
  CUDA_TRY(cudaSetDevice(c->device));
  UCC_TRY(read_counters(c));
  const unsigned long long live = c->h_cnt->n_tail - c->h_cnt->n_dead;
  *n = (size_t)live;
  if (cap < live) return fail(UCC_ECAPACITY, "buffer smaller than the wavefunction");
  if (live == 0) return UCC_OK;
  if (!keys || !amps) return fail(UCC_EINVAL, "null output buffer");
  unsigned long long* dk = (unsigned long long*)keys;
  double* da = amps;
  double* ds = sigma;
  unsigned long long* tk = nullptr;
  double* ta = nullptr;
  double* ts = nullptr;
  if (!on_device) {
    UCC_TRY(dalloc(&tk, live));
    UCC_TRY(dalloc(&ta, live));
    if (sigma) UCC_TRY(dalloc(&ts, live));
    dk = tk;
    da = ta;
    ds = ts;
  }
  CUDA_TRY(cudaMemsetAsync(&c->d_cnt->new_n, 0, sizeof(unsigned long long), c->stream));
  CUDA_TRY(launch_export(c->table(), live, dk, da, ds, c->full_grid(), c->stream));
  if (!on_device) {
    CUDA_TRY(cudaMemcpyAsync(keys, tk, live * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(amps, ta, live * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (sigma) CUDA_TRY(cudaMemcpyAsync(sigma, ts, live * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  ucc_status s = read_counters(c);
  dfree(tk);
  dfree(ta);
  dfree(ts);
  UCC_TRY(s);
  if (c->h_cnt->new_n != live) return fail(UCC_ECUDA, "export count mismatch");
  return UCC_OK;
}

ucc_status ucc_get_stats(const ucc_ctx* c, ucc_stats* out) {
  if (!c || !out) return fail(UCC_EINVAL, "null argument");
  *out = c->stats;
  return UCC_OK;
}

ucc_status ucc_batch_run(int n_jobs, ucc_ctx* const* jobs, double eps, double* E, double* const* grads) {
  if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !E))) return fail(UCC_EINVAL, "bad batch arguments");
  for (int j = 0; j < n_jobs; ++j) {
    ucc_ctx* c = jobs[j];
    if (!c) return fail(UCC_EINVAL, "null job");
    if (grads && grads[j]) {
      UCC_TRY(ucc_gradient(c, eps, &E[j], grads[j], 0));
    } else {
      UCC_TRY(ucc_apply(c, eps));
      UCC_TRY(ucc_energy(c, &E[j], nullptr));
    }
  }
  return UCC_OK;
}

const char* ucc_last_error(void) { return g_last_error.c_str(); }

void ucc_destroy(ucc_ctx* c) { destroy(c); }

}  // extern "C"
