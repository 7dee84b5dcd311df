/*
 * ucc.h - C ABI of the GB300 sparse-wavefunction UCC library (libucc.so).
 *
 * The library implements the data-parallel hot path of the sparse
 * wavefunction circuit simulator of Mullinax & Tubman (arXiv 2301.05726):
 * the factorised unitary-coupled-cluster state of Eq. 3,
 *     |psi> = U_K ... U_2 U_1 |Psi_0>,   U_k = exp(theta_k (tau_k - tau_k^+))
 * (Eqs. 4-5), held as a sparse map from determinant bit strings to
 * FP64 amplitudes, with amplitudes below eps discarded after every factor
 * (Methods section), the energy <psi|H|psi>/<psi|psi> of the molecular
 * Hamiltonian built from one- and two-electron integrals (Methods section),
 * and dE/dtheta for every factor by one reverse (adjoint) sweep.
 *
 * Conventions shared by every call:
 *   - spin-orbital p = 2*spatial + spin (0 = alpha, 1 = beta); bit p of a
 *     determinant key is the Jordan-Wigner qubit of spin-orbital p; a key is
 *     one 64-bit word up to 64 spin-orbitals (the paper's 32-orbital
 *     restriction, Methods section) and two words, low word first, up to 128
 *     (the larger spaces the paper's Conclusion points to);
 *   - the reference |Psi_0> occupies spatial orbitals 0..n_alpha-1 (alpha)
 *     and 0..n_beta-1 (beta);
 *   - excitation row k = (i, j, a, b) is tau_k = a+_a a+_b a_j a_i; a single
 *     is (i, -1, a, -1), tau_k = a+_a a_i; row 0 is applied first (it is the
 *     rightmost factor of Eq. 3);
 *   - a_p and a+_p carry the Jordan-Wigner sign (-1)^(occupied modes below p);
 *   - on a linked pair tau|E> = s|D> a factor rotates
 *         c_E' = cos(t) c_E - s sin(t) c_D,   c_D' = cos(t) c_D + s sin(t) c_E
 *     (two rounded products and one rounded sum each, no fused multiply-add),
 *     a missing member enters as +0.0 and is created, and afterwards both
 *     members are dropped if |c| < eps (strict);
 *   - cos(theta) and sin(theta) are evaluated once on the host (libm).
 *
 * Ownership: the caller owns every pointer it passes; inputs are copied during
 * the call.  The library owns its device state (allocated with cudaMalloc on
 * the device current at ucc_create) and frees it in ucc_destroy.  All device
 * work is enqueued on the caller's stream (a cudaStream_t passed as void*;
 * NULL = legacy default stream).  A call that returns host values
 * synchronises that stream before returning.
 *
 * Errors: every call returns a ucc_status; nothing aborts, traps or exits.
 * ucc_last_error() returns a thread-local message for the last failing call
 * of the calling thread.  Device-side failures (a hash probe that exceeds its
 * bound, an internal inconsistency) are reported through a device error word
 * and returned as UCC_ECUDA or UCC_ECAPACITY by the next synchronising call.
 */
#ifndef UCC_H_
#define UCC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ucc_ctx ucc_ctx; /* opaque, library-owned */

typedef enum {
  UCC_OK = 0,
  UCC_EINVAL = 1,    /* malformed argument (sizes, indices, spin, NaN theta) */
  UCC_ENOMEM = 2,    /* a device or pinned-host allocation failed */
  UCC_ECAPACITY = 3, /* the wavefunction outgrew max_entries or device memory */
  UCC_ETIMEOUT = 4,  /* a bounded device wait gave up */
  UCC_ECUDA = 5,     /* a CUDA runtime error or a device error word */
  UCC_ESTATE = 6     /* call out of order (e.g. energy before apply) */
} ucc_status;

/* One- and two-electron integrals in the spatial-orbital basis (Methods
 * section: the paper takes them from PySCF).  h: n_spatial^2 row-major,
 * symmetric.  g: n_spatial^4 row-major chemist notation (pq|rs) with 8-fold
 * symmetry.  Host pointers.  e_nuc is added to every returned energy. */
typedef struct {
  int32_t n_spatial, n_alpha, n_beta;
  double e_nuc;
  const double* h;
  const double* g;
} ucc_hamiltonian;

/* The factor list of Eq. 3 (Eq. 2's singles and doubles, already ordered and
 * truncated as the Methods section describes).  idx: n_exc x 4 int32 host
 * array of spin-orbital rows (i, j, a, b), singles (i, -1, a, -1); the four
 * indices of a row must be distinct, < 2*n_spatial, and spin-conserving.
 * theta: n_exc host doubles (NULL = all zero). */
typedef struct {
  int32_t n_exc;
  const int32_t* idx;
  const double* theta;
} ucc_ansatz;

/* Run options.  Zero-initialise and set what you need. */
typedef struct {
  int64_t n_max, n_cut; /* Methods-section truncation: if more than n_max
                           determinants remain after a factor keep the n_cut of
                           largest |c| (ties: smaller key).  0 = off. */
  int64_t max_entries;  /* hard cap on stored determinants, 0 = device memory */
  int32_t probe_width;  /* lanes per hash probe: 1, 2, 4 or 8; 0 = autotuned */
  int32_t checkpoint_stride; /* gradient: factors between snapshots of psi; 0 =
                                one segment while the kill tape fits its
                                budget, else ceil(sqrt(K)) */
  int32_t tape_budget_mb;    /* kill-tape budget in MiB; 0 = 60% of free memory */
  int32_t record_entropy;    /* ucc_apply records Eq. 6 after every factor */
  int32_t batch_wait_ms;     /* ucc_batch_run: bound of one grid-barrier wait of
                                its persistent launches, in ms; 0 = 2000.  Read
                                from the first job. */
  int32_t batch_test_skip_block; /* test only: block (1-based) of the batch's
                                    persistent forward launch that leaves
                                    before its first grid barrier, so that the
                                    others' bounded waits run out and the call
                                    returns UCC_ETIMEOUT; 0 = none */
  int32_t batch_tiles;       /* ucc_batch_run: 32-entry tiles a warp takes per
                                visit of a job (1, 2, 4 or 8); 0 = autotuned.
                                Read from the first job. */
  int32_t energy_route;      /* ucc_energy / ucc_gradient: 0 = by buckets of
                                shared cores when their records fit device
                                memory, else per connection; 1 = per
                                connection (every single and double excitation
                                of each stored determinant looked up in the
                                hash); 2 = by buckets (UCC_ENOMEM if the
                                record buffer cannot be allocated) */
  int32_t energy_test_partitions;     /* test only: core partitions of the
                                         bucketed energy (a power of two;
                                         0 = sized by the library) */
  int32_t energy_test_buffer_records; /* test only: cap on the records one
                                         round of the bucketed energy holds
                                         (0 = sized by the library) */
  int32_t rebuild_test_regions; /* test only: hash builds by regions (one-word
                                   keys): 0 = for tables of at least 2^20
                                   slots (and bulk re-insertions of at least
                                   one record per eight slots), 1 = never,
                                   2 = for every table of at least 8,192 slots
                                   and every bulk re-insertion */
  int32_t pad_;
} ucc_options;

/* Counters of the last apply / gradient call. */
typedef struct {
  int64_t n_det;            /* live determinants after the last factor */
  int64_t rotations;        /* linked pairs rotated (det-rotations), forward */
  int64_t created;          /* partners that entered the map */
  int64_t dropped_new;      /* partners computed below eps, never stored */
  int64_t dropped_old;      /* stored entries that fell below eps */
  int64_t cut;              /* entries removed by the n_max/n_cut rule */
  int64_t peak_entries;     /* largest stored count (incl. dropped slots) */
  int64_t capacity_entries; /* current entry capacity */
  int64_t hash_slots;       /* current hash-table size */
  int64_t rebuilds;         /* compactions / growths during the last run */
  int64_t tape_entries;     /* adjoint kill-tape records (gradient only) */
  int64_t kernel_launches;  /* kernels this library launched in the last call */
  int64_t scanned;          /* determinant keys read by the forward factor steps */
  int64_t sigma_probes;     /* last energy evaluation: hash lookups (per
                               connection) or core records (by buckets) */
  int64_t sigma_hits;       /* connected pairs of stored determinants found,
                               each pair counted once */
  int64_t reverse_pairs;    /* linked pairs handled by the reverse sweep */
  int64_t recompute_scanned;   /* gradient: keys read while recomputing segments */
  int64_t recompute_rotations; /* gradient: pairs rotated while recomputing segments */
  int64_t recompute_created;   /* gradient: entries created while recomputing segments */
  int64_t forward_launches;    /* forward factor launches (incl. recomputation) */
  int64_t reverse_launches;    /* reverse factor launches */
  int64_t probe_width;         /* lanes per hash probe in use (fixed or autotuned) */
  int64_t reverse_scanned;     /* entries scanned by the reverse sweep's factor steps */
  int64_t reverse_compactions; /* compactions of the table during the reverse sweep */
  double apply_ms;          /* device time of the last forward pass */
  double energy_ms;         /* device time of the last energy evaluation */
  double reverse_ms;        /* device time of the last reverse sweep */
  double forward_kernel_ms; /* device time of the forward factor launches alone */
  double reverse_kernel_ms; /* device time of the reverse factor launches alone */
  int64_t batch_tiles;      /* ucc_batch_run: 32-entry tiles a warp takes per
                               visit of a job (fixed by the autotuner) */
  double cut_ms;            /* device time of the Methods-section cuts (selection,
                               compaction, rehash) of the last forward pass */
  double rebuild_ms;        /* device time of the other compactions and growths */
  int64_t energy_route;     /* route of the last energy evaluation: 1 per
                               connection, 2 by buckets of shared cores */
} ucc_stats;

/* Create a context: validate and upload the problem (h, g, the factor table
 * with host-evaluated cos/sin).  The stream is stored and used by every later
 * call on this context.  Returns UCC_EINVAL for n_spatial > 64 or < 1,
 * electron counts out of range, a malformed or spin-violating excitation row,
 * or a NaN/inf theta. */
ucc_status ucc_create(const ucc_hamiltonian* ham, const ucc_ansatz* ansatz, void* cuda_stream, ucc_ctx** out);

/* Replace all n_exc angles.  theta is a host pointer (on_device = 0) or a
 * device pointer on the context's device (on_device = 1). */
ucc_status ucc_set_theta(ucc_ctx* ctx, const double* theta, int on_device);

/* Set run options (copied).  NULL restores the defaults (no cut, autotuned
 * probe width, no entry cap). */
ucc_status ucc_set_options(ucc_ctx* ctx, const ucc_options* opt);

/* Build psi = U_K ... U_1 |Psi_0> on the device, dropping |c| < eps after
 * every factor (Eq. 3; Methods section).  eps >= 0.  Synchronises the stream
 * at chunk boundaries to size the table (it grows on demand). */
ucc_status ucc_apply(ucc_ctx* ctx, double eps);

/* E = <psi|H|psi>/<psi|psi> + e_nuc and norm2 = <psi|psi> of the last
 * applied state (Results section's UCCSD energy; Slater-Condon rules).
 * UCC_ESTATE if no state is held.  Synchronises. */
ucc_status ucc_energy(ucc_ctx* ctx, double* E, double* norm2);

/* Apply, energy and the adjoint sweep in one call: E and dE/dtheta_k for all
 * n_exc factors.  grad is a host (on_device = 0) or device (on_device = 1)
 * array of n_exc doubles.  With eps > 0 (or a cut) the derivative is that of
 * the truncated map with the kept sets held fixed.  The sweep leaves no
 * usable state (a later ucc_energy returns UCC_ESTATE).  Synchronises. */
ucc_status ucc_gradient(ucc_ctx* ctx, double eps, double* E, double* grad, int on_device);

/* Copy the live determinants of the held state (unordered) into caller
 * buffers of capacity cap: keys (one uint64 per determinant up to 64
 * spin-orbitals, two -- low word first -- above, so 2*cap words), amps, and
 * optionally sigma = P_S H psi from the last energy evaluation (NULL to
 * skip).  Host or device pointers (on_device).  *n receives the count;
 * UCC_ECAPACITY (and *n set) if cap is too small.  Synchronises. */
ucc_status ucc_get_wavefunction(ucc_ctx* ctx, size_t cap, size_t* n, uint64_t* keys, double* amps, double* sigma,
                                int on_device);

/* The Eq. 6 entropy S_k = -sum_I |c_I|^2 ln|c_I|^2 of the stored state after
 * each factor k of the last ucc_apply (after its eps rule and cut), the
 * quantity the paper plots per factor index (Figs. 3b and 4).  Needs
 * ucc_options.record_entropy; S is a host array of n = n_exc doubles.
 * UCC_ESTATE if the last apply did not record it.  Synchronises. */
ucc_status ucc_get_entropy(ucc_ctx* ctx, double* S, int32_t n);

/* Counters of the last call.  Does not synchronise beyond what that call did. */
ucc_status ucc_get_stats(const ucc_ctx* ctx, ucc_stats* out);

/* Energies and gradients of n_jobs independent contexts (molecules or theta
 * vectors of uneven size): E[j] and grads[j][0..n_exc_j) (host pointers;
 * grads may be NULL for energy only).  Every job whose table can be sized up
 * front (three times its determinant sector, or three times its n_max when
 * its Methods-section cut can fire; at most 2^22 entries; keys of one word)
 * runs in one cooperative
 * persistent launch per pass (forward, energy, reverse) inside a captured CUDA
 * graph: each step applies one factor of every job, and each job's cut and
 * compactions run on the device.  The forward launch is repeated only when
 * jobs wait for more kill tape.  Probe width and tiles per warp are tuned on
 * the first call for a batch shape.  The other jobs run one by one in the
 * same call.  Grid barriers wait at most batch_wait_ms (first job's options);
 * a wait that runs out returns UCC_ETIMEOUT and leaves the contexts usable.
 * All contexts must live on the same device and use the same stream as
 * jobs[0].  Synchronises. */
ucc_status ucc_batch_run(int n_jobs, ucc_ctx* const* jobs, double eps, double* E, double* const* grads);

/* Largest wavefunction ucc_energy_static accepts. */
#define UCC_STATIC_MAX_DETS 262144

/* The energy pass (the same kernel as ucc_energy) over a wavefunction the
 * caller holds, for callers that cannot allocate device memory at the point
 * of the call: cudaMalloc/cudaFree may synchronise the whole device, the
 * device memory may all belong to another allocator, or the device may be out
 * of memory.  The paper has no counterpart; this is a service entry point.
 *
 * Inputs (device pointers on the current device, owned by the caller): h
 * (n_spatial^2) and g (n_spatial^4, chemist order) as in ucc_hamiltonian;
 * keys[n_det] distinct determinants with n_alpha electrons on the even
 * (alpha) and n_beta on the odd (beta) spin-orbitals below 2*n_spatial,
 * amps[n_det] finite amplitudes.  Outputs:
 * sigma[n_det] (device) = P_S H psi at each key, *E = <psi|H|psi>/<psi|psi>
 * + e_nuc and *norm2 (host; norm2 may be NULL).  Work is enqueued on
 * cuda_stream and the call synchronises it before returning.
 *
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its
 * scratch (hash slots over the keys, partial sums, counters, about 8.4 MB) is
 * one file-scope device array that every device loading the library holds
 * until the process exits.  The first call on a device, with that device
 * current, looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the library.  Resetting the device
 * (cudaDeviceReset) after that call is not supported: the module reloads and
 * the kept address goes stale.  Every call reuses the array
 * and clears it first, so calls whose work overlaps on the GPU race: do not
 * run two at once on one device.  n_det above UCC_STATIC_MAX_DETS, or 0,
 * returns UCC_EINVAL; malformed keys or amplitudes return UCC_EINVAL. */
ucc_status ucc_energy_static(int32_t n_spatial, int32_t n_alpha, int32_t n_beta, double e_nuc, const double* h,
                             const double* g, size_t n_det, const uint64_t* keys, const double* amps, double* sigma,
                             double* E, double* norm2, void* cuda_stream);

/* Thread-local message of the last failing call on this thread. */
const char* ucc_last_error(void);

/* Free a context (NULL is a no-op).  Synchronises its stream first. */
void ucc_destroy(ucc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* UCC_H_ */
