// Internal types shared by the CUDA translation units of libucc.so.
// Not part of the public ABI (include/ucc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ucc_keys.cuh"

namespace ucc {

// One factor U_k of Eq. 3 as the kernels need it.  tau_k = a+_a a+_b a_j a_i.
//   occ, vir : bit masks of {i, j} and {a, b};
//   pmask, pconst : the Jordan-Wigner sign of tau_k|E> is
//                   (-1)^(popc(E & pmask) + pconst) for every E that tau_k
//                   excites (the four annihilate/create steps each count the
//                   occupied modes below their index; the counts differ from
//                   popc(E & below(x)) only by index comparisons, folded into
//                   pconst);
//   c, s : cos(theta_k), sin(theta_k) from the host's libm;
//   ic   : 1/cos(theta_k), used by the reverse sweep to undo a lone member.
template <class KT>
struct FactorT {
  KT occ, vir, pmask;
  double c, s, ic;
  int pconst, is_double;
};
using Factor = FactorT<unsigned long long>;
static_assert(sizeof(Factor) == 56, "Factor layout");

// Open-addressing hash slot: key 0 = empty (no valid determinant has zero
// electrons); idx = position of the entry in the compacted arrays.
template <class KT>
struct __align__(16) SlotT {
  KT key;
  unsigned long long idx;
};
using Slot = SlotT<unsigned long long>;
static_assert(sizeof(Slot) == 16 && sizeof(SlotT<Key128>) == 32, "slot layout");

// Device-resident counters of one run, zeroed at reset.
struct Counters {
  unsigned long long n_tail;  // entries appended to the compacted arrays (incl. dropped)
  unsigned long long n_scan;  // entries the current step scans (fixed per step)
  unsigned long long n_dead;  // entries dropped since the last rebuild
  unsigned long long tape_n;  // kill-tape records
  unsigned long long rotations, created, dropped_new, dropped_old;
  unsigned long long new_n;   // output count of compaction / export
  unsigned long long scanned; // keys read by forward steps (sum of n_scan)
  unsigned long long sig_probes, sig_hits;  // hash probes / hits of the energy pass
  unsigned long long rev_pairs;             // pairs handled by the reverse sweep
  unsigned long long rev_scanned;           // entries scanned by reverse steps (sum of n_tail)
  unsigned long long link_from, link_to;    // entries the last forward step appended without a hash slot
  unsigned int done;          // last-block arrival counter
  int stop_k;                 // first factor skipped: no room, or a cut is due (-1: none)
  int error;                  // device error word (bit flags below)
  int cut_pending;            // more than n_max live entries after factor stop_k - 1
  int err_site;               // where the first consistency error was raised (ErrSite)
  unsigned long long err_key; // the key involved in it
  double e_num, norm2;        // <psi|H|psi>, <psi|psi> of the last energy pass
  double entropy;             // running Eq. 6 entropy of the stored state (when recorded)
};

// Where a consistency error was raised (Counters::err_site, first one wins).
enum ErrSite : int {
  SITE_PAIR_OWNER = 1,    // a factor step found the excited member's partner dropped in the same step
  SITE_DUP_CLAIM = 2,     // a slot claim met its own key already hashed
  SITE_REHASH_DUP = 3,    // a rehash met a key twice
  SITE_TAPE_ALIVE = 4,    // a kill-tape record's key was live when re-inserted
  SITE_BULK_ALIVE = 5,    // the same, bulk re-insertion
  SITE_BATCH_ALIVE = 6,   // the same, persistent batched reverse
  SITE_CREATE_DUP = 7,    // a created partner's key was already hashed
  SITE_REINSERT_DUP = 8,  // a re-inserted record's key was already hashed
  SITE_REBUILD_DUP = 9,   // a compaction kept a key twice
  SITE_CUT_COUNT = 10     // a cut kept other than N_CUT entries (err_key: the count kept)
};

enum DeviceError : int {
  ERR_PROBE_BOUND = 1,   // a probe ran past its step bound (table too full)
  ERR_CONSISTENCY = 2,   // a state the algorithm excludes was observed
  ERR_TAPE_FULL = 4,     // kill tape capacity exceeded
  ERR_CAPACITY = 8       // entry allocation past capacity
};

// Everything a kernel needs to address the wavefunction table.
template <class KT>
struct TableT {
  KT* keys;                  // [cap_n] determinant keys
  double* amps;              // [cap_n] amplitudes; a dropped entry holds a tagged NaN
  unsigned int* born;        // [cap_n] factor that created the entry (gradient runs)
  double* lam;               // [cap_n] adjoint vector (gradient runs)
  double* sigma;             // [cap_n] P_S H psi (energy runs)
  SlotT<KT>* slots;          // [slot_mask + 1], a power of two
  unsigned long long slot_mask;
  int slot_shift;            // 64 - log2(slot_mask + 1): home slot = (key * phi64) >> slot_shift
  int filt_shift;            // 32 - log2(filter words)
  unsigned int* filt;        // existence filter, one 32-bit word per 4 slots (nullptr: none)
  unsigned long long cap_n;
  Counters* cnt;
  double* partials;          // [grid] per-block partial sums
  double* entropy;           // [K] Eq. 6 after each factor (nullptr: not recorded)
};
using Table = TableT<unsigned long long>;

// Kill-tape record: a stored entry that fell below eps or was cut, with its
// value just before the drop and the factor that created it.
template <class KT>
struct TapeRecT {
  KT key;
  double val;
  unsigned int born;
  unsigned int pad;
};
using TapeRec = TapeRecT<unsigned long long>;

// The tape is paged so it can grow to tens of GB without copying: record x
// lives in pages[x >> kTapePageBits][x & (kTapePageRecs - 1)].
constexpr int kTapePageBits = 20;
constexpr unsigned long long kTapePageRecs = 1ull << kTapePageBits;  // 1M records, 24 MB
constexpr int kTapeMaxPages = 65536;                                 // up to 1.6 TB

template <class KT>
struct TapeT {
  TapeRecT<KT>* const* pages;  // [kTapeMaxPages] device array of page pointers
  unsigned long long* off;     // [K + 1] tape_n at the start of factor k
  unsigned long long cap;      // records in the allocated pages
};
using Tape = TapeT<unsigned long long>;

// Spatial integrals for the energy kernel.
struct Integrals {
  const double* h;  // [n^2]
  const double* g;  // [n^4] chemist (pq|rs)
  int n;            // spatial orbitals
  int n_so;
};

// One record of the bucketed energy: a core K (a stored determinant with one
// or two electrons removed), the determinant's amplitude and entry index, and
// the removed spin-orbitals p | q << 8 (q = 0xFF for one).  32 bytes for
// either key width, 32-byte aligned: a record is one DRAM sector, written by
// one 256-bit store.
template <class KT>
struct __align__(32) SigRecT {
  KT K;
  double c;
  unsigned int i;
  unsigned short pq;
  unsigned short pad;
};
static_assert(sizeof(SigRecT<unsigned long long>) == 32, "record is one sector");

// Radix-selection state of the N_MAX / N_CUT truncation.
struct SelectState {
  unsigned long long prefix, target;          // |c| bits of the threshold, rank left inside it
  unsigned long long key_prefix, key_target;  // key tie-break among |c| == threshold (low word)
  unsigned long long key_prefix_hi;           // its high word (two-word keys)
  unsigned long long count_eq, cut_total;
  unsigned long long n_cand;                  // entries gathered into the candidate buffer
  int need_keys, pad;
  unsigned long long hist[2048];
};

// A candidate of the selection's last passes: |c| as its IEEE bit pattern and the key.
template <class KT>
struct SelectCandT {
  unsigned long long mag;
  KT key;
};
using SelectCand = SelectCandT<unsigned long long>;
constexpr unsigned long long kSelectCandCap = 1ull << 16;  // candidates the buffer holds

// A second set of table arrays of a job (same sizes as its current ones): the
// target of the job's compactions and cuts inside the persistent batched
// kernels, which swap the two sets on the device.
struct SpareArrays {
  unsigned long long* keys;
  double* amps;
  unsigned int* born;
  double* lam;
  Slot* slots;
  unsigned int* filt;
};

// One job of a batch, as the batched kernels see it (uploaded by the host;
// the persistent kernels swap t's arrays with sp's on the device).
struct JobView {
  Table t;
  const Factor* factors;
  Tape tape;
  Integrals in;
  double* grad;  // [K] dE/dtheta of this job
  double eps;
  int K;
  int pad;
  SpareArrays sp;
  long long n_max, n_cut;  // the Methods-section cut of this job (n_max 0: none)
};

// Per-job progress, written by the batched kernels and read back by the host.
struct JobState {
  int k;                      // forward: next factor; reverse: next factor to undo (-1 when done)
  int stop;                   // forward: factor the job waits at for host action (-1: none)
  unsigned long long base;    // this step's padded offset of the job in the batch index space
  unsigned long long n;       // entries of the job this step covers
  unsigned long long n_tail, n_dead, tape_n;  // mirror of the job's counters after the step
  double e_num, norm2, gacc;  // energy sums; gradient accumulator of the current factor
  unsigned long long rbase, rn;  // reverse: this step's tape records of the job in the record index space
  long long cut;              // entries the job's cuts removed
  int swapped;                // the job's current arrays are its spare set (odd number of swaps)
  int pad2;
};

struct BatchHeader {
  unsigned long long total;   // size of the batch index space of the next step
  unsigned int done;          // last-block arrival counter
  int pad;
  unsigned long long rtotal;  // reverse: size of the tape-record index space of the next step
  unsigned int bar_count, bar_gen;  // grid barrier of the persistent kernels
  int active;                 // jobs still stepping after the last layout
  int error;                  // persistent kernels: 1 = a grid barrier timed out, 2 = a job ran out of room
  int skip_block;             // test hook: this block leaves before the first grid barrier (-1: none)
  int steps;                  // steps the persistent kernel ran (all launches of the call)
  unsigned long long wait_ns; // bound of one grid-barrier wait
};

constexpr int kMaxBatchJobs = 1024;

// Largest entry capacity of one table (the factor steps' queues index entries
// in 31 bits): 2^31 entries, about 120 GB of table.
constexpr unsigned long long kMaxEntries = 1ull << 31;

constexpr unsigned int BORN_INITIAL = 0xFFFFFFFFu;  // the reference determinant

// --- launch wrappers (each returns the launch's cudaError_t) ---------------
// The single-problem path is built for one-word keys (KT = unsigned long
// long, up to 64 spin-orbitals) and two-word keys (KT = Key128, up to 128).
template <class KT>
cudaError_t launch_reset(const TableT<KT>& t, KT hf, cudaStream_t st);
template <class KT>
cudaError_t launch_forward(const TableT<KT>& t, const FactorT<KT>* factors, int k, double eps, unsigned int stamp,
                           int record, const TapeT<KT>& tape, unsigned long long n_max, int probe_width, int grid,
                           cudaStream_t st);
// The N_CUT-th entry by (|c| descending, key ascending) into sel: prefix (its |c| bits), need_keys and
// key_prefix (the largest kept key among entries with that |c|).
template <class KT>
cudaError_t launch_select_threshold(const TableT<KT>& t, SelectState* sel, SelectCandT<KT>* cand,
                                    unsigned long long n_cut, int grid, cudaStream_t st, long long* launches);
// Copy the entries the threshold keeps into `to` (live entries only, unordered, counted in new_n) and
// record the ones it drops on the tape as factor k's (record) or account their entropy.
template <class KT>
cudaError_t launch_cut_compact(const TableT<KT>& from, const TableT<KT>& to, const SelectState* sel, int record,
                               const TapeT<KT>& tape, int k, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_compact(const TableT<KT>& from, const TableT<KT>& to, int with_born, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_rehash(const TableT<KT>& t, int grid, cudaStream_t st);

// Scratch of the hash build by regions (one-word keys): per region of
// 2^kRegionBits slots its entry count, fill counter and offset, the (key,
// index) pairs bucketed by region, and the pairs whose probe runs past their
// region's end.
constexpr int kRegionBits = 13;
struct RehashScratch {
  unsigned int* rcnt = nullptr;         // [regions]
  unsigned int* rfill = nullptr;        // [regions]
  unsigned long long* roff = nullptr;   // [regions + 1]
  unsigned long long* pairs = nullptr;  // [2 * cap]
  unsigned long long* over = nullptr;   // [2 * cap]
  unsigned long long* over_n = nullptr; // [1]
  unsigned long long cap = 0, regions = 0;
};
// Hash the first new_n entries of t (a cleared slot array is not needed: every
// slot is written) by regions: count, prefix sum, bucket, build each region in
// shared memory, then claim slots for the overflow.  With merge, hash instead
// the entries appended since k_mark_tail into the existing hash (insert if
// absent).  Needs t.slot_mask + 1 >= 2^kRegionBits and scratch for t.cap_n
// entries.
cudaError_t launch_rehash_regions(const TableT<unsigned long long>& t, const RehashScratch& rs, int grid,
                                  int num_sms, cudaStream_t st, bool merge = false);
template <class KT>
cudaError_t launch_finish_rebuild(const TableT<KT>& t, unsigned long long expect, cudaStream_t st);
template <class KT>
cudaError_t launch_export(const TableT<KT>& t, unsigned long long cap, KT* keys, double* amps, double* sigma,
                          int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_sigma(const TableT<KT>& t, const Integrals& in, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_lambda_init(const TableT<KT>& t, int grid, cudaStream_t st);
// Bucketed energy: records per core partition, their prefix sum, the records
// of partitions [p0, p1) (fill: per-partition counters, zeroed per round),
// the pair sums into sigma, and the diagonal with E and <psi|psi>.
template <class KT>
cudaError_t launch_sb_count(const TableT<KT>& t, unsigned int* cnt, int log2p, int grid, cudaStream_t st);
cudaError_t launch_sb_scan(const unsigned int* cnt, unsigned long long* off, unsigned long long n, cudaStream_t st);
template <class KT>
cudaError_t launch_sb_scatter(const TableT<KT>& t, const unsigned long long* off, unsigned int* fill,
                              SigRecT<KT>* rec, int log2p, unsigned long long p0, unsigned long long p1,
                              unsigned long long base, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_sb_pairs(const TableT<KT>& t, const Integrals& in, const SigRecT<KT>* rec,
                            const unsigned long long* off, int log2p, unsigned long long p0, unsigned long long p1,
                            unsigned long long base, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_sb_finish(const TableT<KT>& t, const Integrals& in, int grid, cudaStream_t st);
size_t sb_record_bytes(int key_words);
int sb_blocks_per_sm(int key_words);
int sb_partition_target();  // mean records per partition the host aims for
// rs (may be null): scratch of a hash build by regions, used to hash a bulk
// re-insertion's appended range into a large one-word table.
template <class KT>
cudaError_t launch_tape_reinsert(const TableT<KT>& t, const TapeT<KT>& tape, int k, unsigned long long records,
                                 int grid, cudaStream_t st, long long* launches, const RehashScratch* rs = nullptr,
                                 int num_sms = 0);
template <class KT>
cudaError_t launch_reverse(const TableT<KT>& t, const FactorT<KT>* factors, int k, unsigned int stamp, double* grad,
                           int probe_width, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_restore(const TableT<KT>& t, const KT* keys, const double* amps, unsigned long long n, int grid,
                           cudaStream_t st);
template <class KT>
cudaError_t launch_transfer_lambda(const TableT<KT>& dst, const TableT<KT>& src, int grid, cudaStream_t st);
template <class KT>
cudaError_t launch_probe_bench(const TableT<KT>& t, const FactorT<KT>& f, int probe_width, unsigned long long* sink,
                               int grid, cudaStream_t st);
// Batched (many-job) energy: the layout of every job's stored entries, then
// sigma and the energy sums of every job in one launch.
cudaError_t launch_batch_layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, cudaStream_t st);
cudaError_t launch_sigma_batch(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int grid,
                               cudaStream_t st);
cudaError_t launch_lambda_init_batch(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int grid,
                                     cudaStream_t st);
// Persistent batched passes: one cooperative launch runs every job's factor
// steps (forward: up to max_steps steps, or until no job can step) with
// bounded grid barriers.  probe_width 1/2/4/8, tiles = 32-entry tiles a warp
// takes per visit of a job (1, 2, 4 or 8).  Returns the launch's error.
cudaError_t launch_persist_forward(JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int record,
                                   int probe_width, int tiles, int max_steps, cudaStream_t st);
cudaError_t launch_persist_reverse(JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int probe_width,
                                   int tiles, cudaStream_t st);
// The persistent kernels' grid (blocks resident at once) on the current device.
int persist_grid(int record, int probe_width, int reverse);
// Message returned by ucc_last_error() on the calling thread.
void set_last_error(const char* msg);

}  // namespace ucc
