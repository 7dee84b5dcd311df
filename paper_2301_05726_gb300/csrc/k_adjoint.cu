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
// Records from which a factor's re-insertion takes the bulk path.
constexpr unsigned long long kBulkRecords = 1024;

// Re-insert the entries factor k dropped, with their values just before the
// drop, a zero adjoint, and their original birth factor.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_tape_reinsert(TableT<KT> t, TapeT<KT> tape, int k) {
  const unsigned long long hi = min(tape.off[k + 1], tape.cap);
  const unsigned long long lo = min(tape.off[k], hi);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long x = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < hi; x += stride) {
    const TapeRecT<KT> rec = tape_at(tape, x);
    const KT key = rec.key;
    const double val = rec.val;
    const unsigned int born = rec.born;
    Lookup r = find1(t, key, 0u);
    if (r.state == ALIVE) {
      raise_consistency(t.cnt, SITE_TAPE_ALIVE);
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

// Bulk re-insertion (a cut's records): each warp takes 128 records per round,
// four per lane, tests their filter words together, revives in place the few
// whose key is still stored (dropped), and appends the rest without a hash
// slot, one reservation per warp and round; k_link_tail then hashes the
// appended range.  This replaces a per-record chain of filter load, slot
// claim and tail reservation.
template <class KT>
__global__ void k_mark_tail(TableT<KT> t) {
  if (threadIdx.x == 0) t.cnt->link_from = *((volatile unsigned long long*)&t.cnt->n_tail);
}

template <class KT>
__global__ void __launch_bounds__(kThreads) k_tape_append(TableT<KT> t, TapeT<KT> tape, int k) {
  const unsigned long long hi = min(tape.off[k + 1], tape.cap);
  const unsigned long long lo = min(tape.off[k], hi);
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int below_me = (1u << lane) - 1u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long revived = 0;
  for (unsigned long long base = lo + warp * 128ull; base < hi; base += nwarps * 128ull) {  // warp-uniform
    TapeRecT<KT> rec[4];
    bool add[4], maybe[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned long long x = base + 32ull * j + lane;
      add[j] = x < hi;
      if (add[j]) rec[j] = tape_at(tape, x);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) maybe[j] = add[j] && filter_maybe(t, rec[j].key);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!maybe[j]) continue;
      const Lookup r = find1(t, rec[j].key, 0u);
      if (r.state == ALIVE) {
        raise_consistency(t.cnt, SITE_BULK_ALIVE);
        add[j] = false;
      } else if (r.state == DEAD_OLD || r.state == DEAD_NOW) {
        t.amps[r.idx] = rec[j].val;
        t.lam[r.idx] = 0.0;
        t.born[r.idx] = rec[j].born;
        ++revived;
        add[j] = false;
      }
    }
    unsigned int m[4];
    int total = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      m[j] = __ballot_sync(0xFFFFFFFFu, add[j]);
      total += __popc(m[j]);
    }
    if (total == 0) continue;  // warp-uniform
    unsigned long long at = 0;
    if (lane == 0) at = atomicAdd(&t.cnt->n_tail, (unsigned long long)total);
    at = __shfl_sync(0xFFFFFFFFu, at, 0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (add[j]) {
        const unsigned long long idx = at + __popc(m[j] & below_me);
        if (idx < t.cap_n) {
          t.keys[idx] = rec[j].key;
          t.amps[idx] = rec[j].val;
          t.born[idx] = rec[j].born;
          t.lam[idx] = 0.0;
        } else {
          raise_error(t.cnt, ERR_CAPACITY);
        }
      }
      at += __popc(m[j]);
    }
  }
  revived = warp_sum_u64(revived);
  if (lane == 0 && revived) atomicAdd(&t.cnt->n_dead, 0ull - revived);  // dropped entries revived
}

// Hash slots for the entries appended since k_mark_tail.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_link_tail(TableT<KT> t) {
  const unsigned long long lo = *((volatile unsigned long long*)&t.cnt->link_from);
  const unsigned long long hi = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < hi; j += stride)
    link_appended(t, t.keys[j], j);
}

template <class KT, int G>
__global__ void __launch_bounds__(kStepThreads, 8) k_reverse(TableT<KT> t, const FactorT<KT>* __restrict__ factors,
                                                             int k, unsigned int stamp, double* grad) {
  // The adjoint of a linked entry is prefetched into L2 when the entry is
  // queued and loaded with its partner's filter word (staging it with every
  // scanned entry costs more than it saves).
  __shared__ LinkScratch<KT> s_w[kStepThreads / 32];
  const FactorT<KT> f = factors[k];
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  double acc = 0.0;
  unsigned int pairs = 0, kills = 0;
  for_each_linked<false>(
      t, f, n, s_w[threadIdx.x >> 5], nullptr, [&](unsigned long long i, bool act) { return act ? t.lam[i] : 0.0; },
      [&](unsigned long long i, KT X, double cX, bool ex, double mu, bool act) {
        if (act) reverse_resolve(t, f, k, stamp, i, X, cX, mu, ex, absent_lookup(), acc, pairs, kills);
      },
      [&](unsigned long long i, KT X, double cX, bool ex, double, bool act) {
        const double mu = act ? t.lam[i] : 0.0;
        Lookup r = findG<G>(t, X ^ (f.occ | f.vir), act, stamp);
        if (act) reverse_resolve(t, f, k, stamp, i, X, cX, mu, ex, r, acc, pairs, kills);
      },
      // the adjoint of a queued entry moves towards L2 while the scan goes on
      [&](unsigned long long i) { prefetch_l2(&t.lam[i]); });
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

template <class KT>
cudaError_t launch_tape_reinsert(const TableT<KT>& t, const TapeT<KT>& tape, int k, unsigned long long records,
                                 int grid, cudaStream_t st, long long* launches, const RehashScratch* rs,
                                 int num_sms) {
  if (records < kBulkRecords) {
    k_tape_reinsert<KT><<<grid, kThreads, 0, st>>>(t, tape, k);
    *launches += 1;
  } else {
    k_mark_tail<KT><<<1, 32, 0, st>>>(t);
    k_tape_append<KT><<<grid, kThreads, 0, st>>>(t, tape, k);
    bool merged = false;
    if constexpr (sizeof(KT) == 8) {
      if (rs != nullptr) {
        // the appended range hashed region by region into the existing hash
        const cudaError_t e = launch_rehash_regions(t, *rs, grid, num_sms, st, true);
        if (e != cudaSuccess) return e;
        *launches += 7;
        merged = true;
      }
    }
    if (!merged) {
      k_link_tail<KT><<<grid, kThreads, 0, st>>>(t);
      *launches += 3;
    }
  }
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_reverse(const TableT<KT>& t, const FactorT<KT>* factors, int k, unsigned int stamp, double* grad,
                           int probe_width, int grid, cudaStream_t st) {
  if (!scan_aligned(t)) return cudaErrorMisalignedAddress;
  switch (probe_width) {
    case 2:
      k_reverse<KT, 2><<<one_wave<k_reverse<KT, 2>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp,
                                                                                                 grad);
      break;
    case 4:
      k_reverse<KT, 4><<<one_wave<k_reverse<KT, 4>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp,
                                                                                                 grad);
      break;
    case 8:
      k_reverse<KT, 8><<<one_wave<k_reverse<KT, 8>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp,
                                                                                                 grad);
      break;
    default:
      k_reverse<KT, 1><<<one_wave<k_reverse<KT, 1>, kStepThreads>(grid), kStepThreads, 0, st>>>(t, factors, k, stamp,
                                                                                                 grad);
      break;
  }
  return cudaGetLastError();
}

#define UCC_ADJOINT_INSTANTIATE(KT)                                                                               \
  template cudaError_t launch_tape_reinsert<KT>(const TableT<KT>&, const TapeT<KT>&, int, unsigned long long, int, \
                                                cudaStream_t, long long*, const RehashScratch*, int);            \
  template cudaError_t launch_reverse<KT>(const TableT<KT>&, const FactorT<KT>*, int, unsigned int, double*, int,  \
                                          int, cudaStream_t);
UCC_ADJOINT_INSTANTIATE(unsigned long long)
UCC_ADJOINT_INSTANTIATE(Key128)

}  // namespace ucc
