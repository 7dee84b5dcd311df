// Reverse (adjoint) sweep: dE/dtheta_k for every factor in one pass K..1.
//
// With the prune sets held fixed, psi_k = P_k U_k psi_{k-1} and
//   dE/dtheta_k = 2 <lambda_{k-1}| A_k psi_{k-1}>,
//   mu_K = P_K (H psi - E psi)/<psi|psi>,
//   lambda_{k-1} = U_k^T mu_k,  mu_{k-1} = P_{k-1} lambda_{k-1},
// where A_k = tau_k - tau_k^+ maps a linked pair (E, D = s tau E) as
// A|E> = s|D>, A|D> = -s|E>, so  <lambda|A psi> = sum_pairs s (lam_D psi_E - lam_E psi_D).
//
// psi_{k-1} is recovered from psi_k in place: both members of a pair by the
// inverse rotation, a lone member by dividing out cos(theta) (its partner was
// absent before the factor and fell below eps after it).  The only values the
// forward pass destroys are those of stored entries that fell below eps; the
// forward pass records them (the kill tape) and step k re-inserts its records
// before the pair sweep.  Entries created by factor k (born[] == k) leave the
// table when the sweep passes k.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

constexpr int kThreads = 256;

// Re-insert the entries factor k dropped, with their values just before the
// drop, a zero adjoint, and their original birth factor.
__global__ void __launch_bounds__(kThreads) k_tape_reinsert(Table t, Tape tape, int k) {
  const unsigned long long hi = min(tape.off[k + 1], tape.cap);
  const unsigned long long lo = min(tape.off[k], hi);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long x = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < hi; x += stride) {
    const TapeRec rec = tape_at(tape, x);
    const unsigned long long key = rec.key;
    const double val = rec.val;
    const unsigned int born = rec.born;
    Lookup r = find1(t, key, 0u);
    if (r.state == ALIVE) {
      raise_error(t.cnt, ERR_CONSISTENCY);
    } else if (r.state == DEAD_OLD || r.state == DEAD_NOW) {
      t.amps[r.idx] = val;
      t.lam[r.idx] = 0.0;
      t.born[r.idx] = born;
      // one dropped entry fewer (a warp-aggregated decrement)
      cg::coalesced_group g = cg::coalesced_threads();
      if (g.thread_rank() == 0) atomicAdd(&t.cnt->n_dead, 0ull - (unsigned long long)g.size());
    } else {
      insert_new(t, key, val, born, r.slot, true, true);
    }
  }
}

template <int G>
__global__ void __launch_bounds__(kStepThreads, 8) k_reverse(Table t, const Factor* __restrict__ factors, int k,
                                                             unsigned int stamp, double* grad) {
  __shared__ LinkScratch s_w[kStepThreads / 32];
  const Factor f = factors[k];
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  double acc = 0.0;
  unsigned int pairs = 0, kills = 0;
  for_each_linked(
      t, f, n, s_w[threadIdx.x >> 5], [&](unsigned long long i, bool act) { return act ? t.lam[i] : 0.0; },
      [&](unsigned long long i, unsigned long long X, double cX, bool ex, double mu, bool act) {
        if (act) reverse_resolve(t, f, k, stamp, i, X, cX, mu, ex, absent_lookup(), acc, pairs, kills);
      },
      [&](unsigned long long i, unsigned long long X, double cX, bool ex, bool act) {
        const double mu = act ? t.lam[i] : 0.0;
        Lookup r = findG<G>(t, X ^ (f.occ | f.vir), act, stamp);
        if (act) reverse_resolve(t, f, k, stamp, i, X, cX, mu, ex, r, acc, pairs, kills);
      });
  {
    // Entries this step removed (born at factor k) count as dropped, so the
    // host can compact the table when they pile up.
    __shared__ unsigned long long s_pairs, s_kills;
    if (threadIdx.x == 0) s_pairs = s_kills = 0;
    __syncthreads();
    if (pairs) atomicAdd(&s_pairs, (unsigned long long)pairs);
    if (kills) atomicAdd(&s_kills, (unsigned long long)kills);
    __syncthreads();
    if (threadIdx.x == 0 && s_pairs) atomicAdd(&t.cnt->rev_pairs, s_pairs);
    if (threadIdx.x == 0 && s_kills) atomicAdd(&t.cnt->n_dead, s_kills);
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) t.partials[blockIdx.x] = b;
  if (last_block_arrive(t.cnt)) {
    double s = 0.0;
    for (unsigned int x = threadIdx.x; x < gridDim.x; x += blockDim.x) s += ld_cg(&t.partials[x]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
      grad[k] = 2.0 * s;
      t.cnt->rev_scanned += n;
      t.cnt->done = 0u;
    }
  }
}

}  // namespace

cudaError_t launch_tape_reinsert(const Table& t, const Tape& tape, int k, int grid, cudaStream_t st) {
  k_tape_reinsert<<<grid, kThreads, 0, st>>>(t, tape, k);
  return cudaGetLastError();
}

cudaError_t launch_reverse(const Table& t, const Factor* factors, int k, unsigned int stamp, double* grad,
                           int probe_width, int grid, cudaStream_t st) {
  if (!scan_aligned(t)) return cudaErrorMisalignedAddress;
  switch (probe_width) {
    case 2:
      k_reverse<2><<<one_wave<k_reverse<2>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp, grad);
      break;
    case 4:
      k_reverse<4><<<one_wave<k_reverse<4>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp, grad);
      break;
    case 8:
      k_reverse<8><<<one_wave<k_reverse<8>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp, grad);
      break;
    default:
      k_reverse<1><<<one_wave<k_reverse<1>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp, grad);
      break;
  }
  return cudaGetLastError();
}

}  // namespace ucc
