// Forward kernels: one factor of Eq. 3 per launch, plus table maintenance.
//
// Data layout (HBM): compacted structure-of-arrays keys[] (uint64) and
// amps[] (fp64) scanned with coalesced loads, an open-addressing hash of
// 16-byte slots {key, index} for partner lookups, and (gradient runs) born[]
// (uint32, the factor that created each entry) plus an append-only kill tape.

#include <algorithm>

#include "ucc_steps.cuh"

namespace ucc {

namespace {

constexpr int kThreads = 256;

// Block totals of the step counters: a warp reduction, then one shared
// atomic per warp and one global atomic per block and counter.
__device__ __forceinline__ void block_add_counts(Counters* c, unsigned long long rot, unsigned long long cre,
                                                 unsigned long long dnew, unsigned long long dold,
                                                 long long dead_delta) {
  __shared__ unsigned long long s_v[5];
  if (threadIdx.x < 5) s_v[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long v[5] = {rot, cre, dnew, dold, (unsigned long long)dead_delta};
#pragma unroll
  for (int x = 0; x < 5; ++x) v[x] = warp_sum_u64(v[x]);
  if ((threadIdx.x & 31u) == 0) {
#pragma unroll
    for (int x = 0; x < 5; ++x)
      if (v[x]) atomicAdd(&s_v[x], v[x]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_v[0]) atomicAdd(&c->rotations, s_v[0]);
    if (s_v[1]) atomicAdd(&c->created, s_v[1]);
    if (s_v[2]) atomicAdd(&c->dropped_new, s_v[2]);
    if (s_v[3]) atomicAdd(&c->dropped_old, s_v[3]);
    if (s_v[4]) atomicAdd(&c->n_dead, s_v[4]);
  }
}

// One factor U_k on every stored determinant.  Each linked pair (E, D = tau E)
// is rotated exactly once: by the thread of E when E is stored and live at the
// start of the step, otherwise by the thread of D.  Entries dropped during
// this step carry this step's stamp, so a D-thread can tell "E was live when
// the step began" (live or DEAD_NOW) from "E absent" (ABSENT or DEAD_OLD).
template <class KT, int G, bool RECORD>
__global__ void __launch_bounds__(kStepThreads, 8) k_forward(TableT<KT> t, const FactorT<KT>* __restrict__ factors,
                                                             int k, double eps, unsigned int stamp, TapeT<KT> tape,
                                                             unsigned long long n_max) {
  __shared__ int s_skip;
  __shared__ LinkScratch<KT> s_w[kStepThreads / 32];
  if (threadIdx.x == 0) s_skip = *((volatile int*)&t.cnt->stop_k) >= 0;
  __syncthreads();
  // An earlier factor of this chunk stopped it: every block of the launch
  // reads the same flag (only this launch's last block could change it, after
  // every other block has read it), so the whole launch leaves at once.
  if (s_skip != 0) return;
  StepCounts sc;
  {
    const FactorT<KT> f = factors[k];
    const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_scan), t.cap_n);
    for_each_linked<false>(
        t, f, n, s_w[threadIdx.x >> 5], nullptr, [](unsigned long long, bool) { return 0.0; },
        [&](unsigned long long i, KT X, double cX, bool ex, double, bool act) {
          if (act) forward_resolve<RECORD, true>(t, f, k, eps, stamp, tape, i, X, cX, ex, absent_lookup(), sc);
        },
        [&](unsigned long long i, KT X, double cX, bool ex, double, bool act) {
          Lookup r = findG<G>(t, X ^ (f.occ | f.vir), act, stamp);
          if (act) forward_resolve<RECORD, true>(t, f, k, eps, stamp, tape, i, X, cX, ex, r, sc);
        });
  }
  block_add_counts(t.cnt, sc.rot, sc.cre, sc.dnew, sc.dold, sc.dead_delta);
  if (t.entropy) {
    const double b = block_sum(sc.dS);
    if (threadIdx.x == 0) t.partials[blockIdx.x] = b;
  }
  const bool last = last_block_arrive(t.cnt);
  if (last && t.entropy) {
    // Fixed-order sum of the block changes, added once to the running total.
    double s = 0.0;
    for (unsigned int x = threadIdx.x; x < gridDim.x; x += blockDim.x) s += ld_cg(&t.partials[x]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
      t.cnt->entropy += s;
      t.entropy[k] = t.cnt->entropy;
    }
  }
  if (last && threadIdx.x == 0) {
    Counters* c = t.cnt;
    c->done = 0u;
    {
      const unsigned long long nt = ld_cg(&c->n_tail);
      c->link_from = ld_cg(&c->n_scan);  // this step's appended entries, linked next
      c->link_to = nt;
      c->scanned += ld_cg(&c->n_scan);
      c->n_scan = nt;
      unsigned long long tn = 0;
      if (RECORD) {
        tn = ld_cg(&c->tape_n);
        tape.off[k + 1] = tn;
      }
      // Room for factor k+1: it can append at most nt entries and drop at
      // most nt; the hash must stay at most 75% full afterwards.
      const unsigned long long slots = t.slot_mask + 1ull;
      const bool room = 2ull * nt <= t.cap_n && 8ull * nt <= 3ull * slots && (!RECORD || tn + nt <= tape.cap);
      // Methods-section truncation is due when more than n_max entries live.
      const bool cut = n_max > 0 && nt - ld_cg(&c->n_dead) > n_max;
      if (cut) c->cut_pending = 1;
      if (!room || cut) c->stop_k = k + 1;
    }
  }
}

// Hash slots for the entries factor k's step appended (k_forward defers
// them); skipped with the step itself when an earlier factor stopped the chunk.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_link(TableT<KT> t, int k) {
  const int stop = *((volatile int*)&t.cnt->stop_k);
  if (stop >= 0 && stop <= k) return;
  const unsigned long long lo = *((volatile unsigned long long*)&t.cnt->link_from);
  const unsigned long long hi = min(*((volatile unsigned long long*)&t.cnt->link_to), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < hi; j += stride)
    link_appended(t, t.keys[j], j);
}

// Copy the live entries of `from` into `to` (unordered), counting in new_n.
// with_born: 0 keys and amplitudes, 1 also born, 2 also born and lam.
// Each warp takes four tiles of 32 entries per round: their amplitudes are
// loaded together and one reservation per round places the live ones.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_compact(TableT<KT> from, TableT<KT> to, int with_born) {
  const unsigned long long n = min(*((volatile unsigned long long*)&from.cnt->n_tail), from.cap_n);
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned int below_me = (1u << lane) - 1u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long base = warp * 128ull; base < n; base += nwarps * 128ull) {  // warp-uniform
    double a[4];
    bool live[4];
    unsigned int m[4];
    int total = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned long long i = base + 32ull * u + lane;
      a[u] = i < n ? from.amps[i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      live[u] = base + 32ull * u + lane < n && !is_dead(a[u]);
      m[u] = __ballot_sync(0xFFFFFFFFu, live[u]);
      total += __popc(m[u]);
    }
    if (total == 0) continue;  // warp-uniform
    unsigned long long at = 0;
    if (lane == 0) at = atomicAdd(&from.cnt->new_n, (unsigned long long)total);
    at = __shfl_sync(0xFFFFFFFFu, at, 0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (live[u]) {
        const unsigned long long i = base + 32ull * u + lane;
        const unsigned long long j = at + __popc(m[u] & below_me);
        if (j < to.cap_n) {
          to.keys[j] = from.keys[i];
          to.amps[j] = a[u];
          if (with_born) to.born[j] = from.born[i];
          if (with_born > 1) to.lam[j] = from.lam[i];  // mid reverse sweep: keep the adjoint
        } else {
          raise_error(from.cnt, ERR_CAPACITY);
        }
      }
      at += __popc(m[u]);
    }
  }
}

// Insert entries [0, new_n) into an empty slot array.
// Four entries per thread and round: their keys are loaded and their home
// slots claimed together (the home slot is usually free), and only the
// entries whose home slot was taken probe on.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_rehash(TableT<KT> t) {
  using K = KeyOps<KT>;
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->new_n), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    KT key[4], prev[4];
    unsigned long long h[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned long long i = i0 + u * stride;
      key[u] = i < n ? t.keys[i] : K::zero();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h[u] = home_slot(t, key[u]);
      prev[u] = !K::is_zero(key[u]) ? key_cas(&t.slots[h[u]].key, K::zero(), key[u]) : K::bit(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (K::is_zero(key[u])) continue;
      const unsigned long long i = i0 + u * stride;
      unsigned long long s = h[u];
      if (K::is_zero(prev[u])) {
        filter_add(t, key[u]);
      } else {
        if (prev[u] == key[u]) raise_consistency(t.cnt, SITE_REHASH_DUP, K::lo(key[u]));
        s = claim_slot(t, key[u], h[u] + 1);
      }
      if (s != ~0ull) t.slots[s].idx = i;
    }
  }
}

template <class KT>
__global__ void k_finish_rebuild(TableT<KT> t, unsigned long long expect) {
  Counters* c = t.cnt;
  const unsigned long long n = min(*((volatile unsigned long long*)&c->new_n), t.cap_n);
  if (expect != ~0ull && n != expect) raise_consistency(c, SITE_CUT_COUNT, n);
  c->n_tail = n;
  c->n_scan = n;
  c->n_dead = 0;
  c->new_n = 0;
  const unsigned long long slots = t.slot_mask + 1ull;
  if (c->stop_k >= 0 && 2ull * n <= t.cap_n && 8ull * n <= 3ull * slots) c->stop_k = -1;
}

// Hash build by regions.  Inserting entries in table order claims one random
// slot each (a DRAM sector read and written per entry); bucketing the entries
// by the region of 2^kRegionBits slots their home slot falls in first lets one
// block build each region in shared memory and write it out whole.  Linear
// probing that runs past a region's end continues, after every region is
// written, at the next region's first slot (all slots it passed are full).
constexpr int kRegionSlots = 1 << kRegionBits;
constexpr int kRegionThreads = 512;

__device__ __forceinline__ unsigned long long region_of(const Table& t, unsigned long long key) {
  return home_slot(t, key) >> kRegionBits;
}

// The entries a build hashes: a rebuild's [0, new_n), or (merge) the range
// appended since k_mark_tail, [link_from, n_tail), into the existing hash.
__device__ __forceinline__ void rr_range(const Table& t, bool merge, unsigned long long* lo, unsigned long long* hi) {
  if (merge) {
    *hi = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
    *lo = min(*((volatile unsigned long long*)&t.cnt->link_from), *hi);
  } else {
    *lo = 0ull;
    *hi = min(*((volatile unsigned long long*)&t.cnt->new_n), t.cap_n);
  }
}

__global__ void __launch_bounds__(kThreads) k_rr_count(Table t, unsigned int* __restrict__ rcnt, bool merge) {
  unsigned long long lo, n;
  rr_range(t, merge, &lo, &n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(&rcnt[region_of(t, t.keys[i])], 1u);
}

__global__ void __launch_bounds__(kThreads) k_rr_scatter(Table t, const unsigned long long* __restrict__ roff,
                                                         unsigned int* __restrict__ rfill,
                                                         unsigned long long* __restrict__ pairs, bool merge) {
  unsigned long long lo, n;
  rr_range(t, merge, &lo, &n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = lo + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long key = t.keys[i];
    const unsigned long long r = region_of(t, key);
    const unsigned long long at = roff[r] + atomicAdd(&rfill[r], 1u);
    if (at >= roff[r + 1]) {  // more entries than counted: never written past the region's share
      raise_error(t.cnt, ERR_CAPACITY);
      continue;
    }
    *reinterpret_cast<ulonglong2*>(pairs + 2 * at) = make_ulonglong2(key, i);
  }
}

// One block per region (grid-stride): the region's slots in shared memory
// (empty, or with merge the hash's current slots), its pairs inserted by
// linear probing with shared-memory CAS (each new key added to the filter),
// then every slot of the region written back.  A probe that reaches the
// region's end goes to the overflow list.  A key met twice is an error in a
// rebuild and left as it is in a merge (insert-if-absent).  With merge a
// region without new pairs is left untouched.
__global__ void __launch_bounds__(kRegionThreads) k_rr_build(Table t, const unsigned long long* __restrict__ roff,
                                                             const unsigned long long* __restrict__ pairs,
                                                             unsigned long long* __restrict__ over,
                                                             unsigned long long* __restrict__ over_n,
                                                             unsigned long long regions, bool merge) {
  extern __shared__ __align__(16) unsigned char rr_smem[];
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(rr_smem);
  unsigned int* si = reinterpret_cast<unsigned int*>(sk + kRegionSlots);
  for (unsigned long long r = blockIdx.x; r < regions; r += gridDim.x) {
    const unsigned long long lo = roff[r], hi = roff[r + 1];
    if (merge && lo == hi) continue;
    Slot* out = t.slots + (r << kRegionBits);
    for (int x = (int)threadIdx.x; x < kRegionSlots; x += kRegionThreads) {
      if (merge) {
        const Slot sl = out[x];
        sk[x] = sl.key;
        si[x] = (unsigned int)sl.idx;
      } else {
        sk[x] = 0ull;
      }
    }
    __syncthreads();
    for (unsigned long long p = lo + threadIdx.x; p < hi; p += kRegionThreads) {
      const ulonglong2 kv = *reinterpret_cast<const ulonglong2*>(pairs + 2 * p);
      int h = (int)(home_slot(t, kv.x) & (unsigned long long)(kRegionSlots - 1));
      for (;;) {
        const unsigned long long prev = atomicCAS(&sk[h], 0ull, kv.x);
        if (prev == 0ull) {
          si[h] = (unsigned int)kv.y;
          filter_add(t, kv.x);
          break;
        }
        if (prev == kv.x) {
          if (!merge) raise_consistency(t.cnt, SITE_REHASH_DUP, kv.x);
          break;
        }
        if (++h == kRegionSlots) {
          const unsigned long long o = atomicAdd(over_n, 1ull);
          *reinterpret_cast<ulonglong2*>(over + 2 * o) = kv;
          break;
        }
      }
    }
    __syncthreads();
    for (int x = (int)threadIdx.x; x < kRegionSlots; x += kRegionThreads) {
      const unsigned long long key = sk[x];
      Slot sl;
      sl.key = key;
      sl.idx = key ? (unsigned long long)si[x] : 0ull;
      out[x] = sl;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_rr_overflow(Table t, const unsigned long long* __restrict__ over,
                                                          const unsigned long long* __restrict__ over_n, bool merge) {
  const unsigned long long n = *over_n;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long o = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += stride) {
    const ulonglong2 kv = *reinterpret_cast<const ulonglong2*>(over + 2 * o);
    const unsigned long long next = (region_of(t, kv.x) + 1ull) << kRegionBits;
    if (merge) {
      link_from_slot(t, kv.x, kv.y, next);
    } else {
      const unsigned long long s = claim_slot(t, kv.x, next, SITE_REHASH_DUP);
      if (s != ~0ull) t.slots[s].idx = kv.y;
    }
  }
}

// Gather live entries into caller buffers (unordered).
template <class KT>
__global__ void __launch_bounds__(kThreads) k_export(TableT<KT> t, unsigned long long cap, KT* keys, double* amps,
                                                      double* sigma) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long j = aggregated_add(&t.cnt->new_n);
    if (j < cap) {
      keys[j] = t.keys[i];
      amps[j] = a;
      if (sigma) sigma[j] = t.sigma[i];
    }
  }
}

// psi = {HF: 1.0}; the slots are already zero.
template <class KT>
__global__ void k_reset(TableT<KT> t, KT hf) {
  Counters* c = t.cnt;
  t.keys[0] = hf;
  t.amps[0] = 1.0;
  if (t.born) t.born[0] = BORN_INITIAL;
  const unsigned long long s = home_slot(t, hf);
  t.slots[s].key = hf;
  t.slots[s].idx = 0;
  filter_add(t, hf);
  c->n_tail = 1;
  c->n_scan = 1;
  c->stop_k = -1;
}

}  // namespace

template <class KT>
cudaError_t launch_reset(const TableT<KT>& t, KT hf, cudaStream_t st) {
  k_reset<KT><<<1, 1, 0, st>>>(t, hf);
  return cudaGetLastError();
}

template <class KT, bool RECORD>
static cudaError_t forward_g(const TableT<KT>& t, const FactorT<KT>* factors, int k, double eps, unsigned int stamp,
                             const TapeT<KT>& tape, unsigned long long n_max, int pw, int grid, cudaStream_t st) {
  switch (pw) {
    case 2:
      k_forward<KT, 2, RECORD><<<one_wave<k_forward<KT, 2, RECORD>, kStepThreads>(grid), kStepThreads, 0, st>>>(
          t, factors, k, eps, stamp, tape, n_max);
      break;
    case 4:
      k_forward<KT, 4, RECORD><<<one_wave<k_forward<KT, 4, RECORD>, kStepThreads>(grid), kStepThreads, 0, st>>>(
          t, factors, k, eps, stamp, tape, n_max);
      break;
    case 8:
      k_forward<KT, 8, RECORD><<<one_wave<k_forward<KT, 8, RECORD>, kStepThreads>(grid), kStepThreads, 0, st>>>(
          t, factors, k, eps, stamp, tape, n_max);
      break;
    default:
      k_forward<KT, 1, RECORD><<<one_wave<k_forward<KT, 1, RECORD>, kStepThreads>(grid), kStepThreads, 0, st>>>(
          t, factors, k, eps, stamp, tape, n_max);
      break;
  }
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_forward(const TableT<KT>& t, const FactorT<KT>* factors, int k, double eps, unsigned int stamp,
                           int record, const TapeT<KT>& tape, unsigned long long n_max, int probe_width, int grid,
                           cudaStream_t st) {
  if (!scan_aligned(t)) return cudaErrorMisalignedAddress;
  const cudaError_t e = record ? forward_g<KT, true>(t, factors, k, eps, stamp, tape, n_max, probe_width, grid, st)
                               : forward_g<KT, false>(t, factors, k, eps, stamp, tape, n_max, probe_width, grid, st);
  if (e != cudaSuccess) return e;
  k_link<KT><<<one_wave<k_link<KT>, kThreads>(grid), kThreads, 0, st>>>(t, k);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_compact(const TableT<KT>& from, const TableT<KT>& to, int with_born, int grid, cudaStream_t st) {
  k_compact<KT><<<grid, kThreads, 0, st>>>(from, to, with_born);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_rehash(const TableT<KT>& t, int grid, cudaStream_t st) {
  k_rehash<KT><<<grid, kThreads, 0, st>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_rehash_regions(const Table& t, const RehashScratch& rs, int grid, int num_sms, cudaStream_t st,
                                  bool merge) {
  constexpr size_t smem = (size_t)kRegionSlots * (sizeof(unsigned long long) + sizeof(unsigned int));
  {
    // per device (the current one): set on every launch
    const cudaError_t e = cudaFuncSetAttribute(k_rr_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned long long regions = (t.slot_mask + 1ull) >> kRegionBits;
  if (regions == 0 || regions > rs.regions) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = cudaMemsetAsync(rs.rcnt, 0, regions * sizeof(unsigned int), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(rs.rfill, 0, regions * sizeof(unsigned int), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(rs.over_n, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  k_rr_count<<<grid, kThreads, 0, st>>>(t, rs.rcnt, merge);
  if ((e = launch_sb_scan(rs.rcnt, rs.roff, regions, st)) != cudaSuccess) return e;
  k_rr_scatter<<<grid, kThreads, 0, st>>>(t, rs.roff, rs.rfill, rs.pairs, merge);
  const int bgrid = (int)std::min<unsigned long long>(regions, (unsigned long long)(2 * num_sms));
  k_rr_build<<<bgrid, kRegionThreads, smem, st>>>(t, rs.roff, rs.pairs, rs.over, rs.over_n, regions, merge);
  k_rr_overflow<<<std::max(1, num_sms), kThreads, 0, st>>>(t, rs.over, rs.over_n, merge);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_finish_rebuild(const TableT<KT>& t, unsigned long long expect, cudaStream_t st) {
  k_finish_rebuild<KT><<<1, 1, 0, st>>>(t, expect);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_export(const TableT<KT>& t, unsigned long long cap, KT* keys, double* amps, double* sigma,
                          int grid, cudaStream_t st) {
  k_export<KT><<<grid, kThreads, 0, st>>>(t, cap, keys, amps, sigma);
  return cudaGetLastError();
}

#define UCC_APPLY_INSTANTIATE(KT)                                                                                  \
  template cudaError_t launch_reset<KT>(const TableT<KT>&, KT, cudaStream_t);                                      \
  template cudaError_t launch_forward<KT>(const TableT<KT>&, const FactorT<KT>*, int, double, unsigned int, int,   \
                                          const TapeT<KT>&, unsigned long long, int, int, cudaStream_t);           \
  template cudaError_t launch_compact<KT>(const TableT<KT>&, const TableT<KT>&, int, int, cudaStream_t);           \
  template cudaError_t launch_rehash<KT>(const TableT<KT>&, int, cudaStream_t);                                    \
  template cudaError_t launch_finish_rebuild<KT>(const TableT<KT>&, unsigned long long, cudaStream_t);                                 \
  template cudaError_t launch_export<KT>(const TableT<KT>&, unsigned long long, KT*, double*, double*, int,        \
                                         cudaStream_t);
UCC_APPLY_INSTANTIATE(unsigned long long)
UCC_APPLY_INSTANTIATE(Key128)

}  // namespace ucc

namespace ucc {

namespace {

// Load a snapshot (live keys and amplitudes, unordered) as entries [0, n).
template <class KT>
__global__ void __launch_bounds__(256) k_restore(TableT<KT> t, const KT* keys, const double* amps,
                                                  unsigned long long n) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n && i < t.cap_n;
       i += stride) {
    t.keys[i] = keys[i];
    t.amps[i] = amps[i];
    t.born[i] = BORN_INITIAL;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Counters* c = t.cnt;
    const unsigned long long m = n < t.cap_n ? n : t.cap_n;
    c->n_tail = m;
    c->n_scan = m;
    c->new_n = m;
    c->n_dead = 0;
    c->stop_k = -1;
  }
}

// Copy the adjoint vector of `src` onto the live entries of `dst` by key
// (zero where src has no live entry).
template <class KT>
__global__ void __launch_bounds__(256) k_transfer_lambda(TableT<KT> dst, TableT<KT> src) {
  const unsigned long long n = min(*((volatile unsigned long long*)&dst.cnt->n_tail), dst.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (is_dead(dst.amps[i])) continue;
    Lookup r = find1(src, dst.keys[i], 0u);
    dst.lam[i] = (r.state == ALIVE) ? src.lam[r.idx] : 0.0;
  }
}

}  // namespace

template <class KT>
cudaError_t launch_restore(const TableT<KT>& t, const KT* keys, const double* amps, unsigned long long n, int grid,
                           cudaStream_t st) {
  k_restore<KT><<<grid, 256, 0, st>>>(t, keys, amps, n);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_transfer_lambda(const TableT<KT>& dst, const TableT<KT>& src, int grid, cudaStream_t st) {
  k_transfer_lambda<KT><<<grid, 256, 0, st>>>(dst, src);
  return cudaGetLastError();
}

template cudaError_t launch_restore<unsigned long long>(const Table&, const unsigned long long*, const double*,
                                                        unsigned long long, int, cudaStream_t);
template cudaError_t launch_restore<Key128>(const TableT<Key128>&, const Key128*, const double*, unsigned long long,
                                            int, cudaStream_t);
template cudaError_t launch_transfer_lambda<unsigned long long>(const Table&, const Table&, int, cudaStream_t);
template cudaError_t launch_transfer_lambda<Key128>(const TableT<Key128>&, const TableT<Key128>&, int,
                                                    cudaStream_t);

}  // namespace ucc

namespace ucc {

namespace {

// Read-only replay of factor f's partner lookups on the live table with
// G-lane probes (the autotuner times it); the result only feeds a checksum.
template <class KT, int G>
__global__ void __launch_bounds__(kStepThreads) k_probe_bench(TableT<KT> t, FactorT<KT> f, unsigned long long* sink) {
  __shared__ LinkScratch<KT> s_w[kStepThreads / 32];
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const KT m = f.occ | f.vir;
  unsigned long long acc = 0;
  for_each_linked<false>(
      t, f, n, s_w[threadIdx.x >> 5], nullptr, [](unsigned long long, bool) { return 0.0; },
      [&](unsigned long long, KT, double, bool, double, bool) {},
      [&](unsigned long long, KT X, double, bool, double, bool act) {
        Lookup r = findG<G>(t, X ^ m, act, 0u);
        if (act) acc += r.idx + (unsigned long long)r.state;
      });
  acc = warp_sum_u64(acc);
  if ((threadIdx.x & 31u) == 0 && acc) atomicAdd(sink, acc);
}

}  // namespace

template <class KT>
cudaError_t launch_probe_bench(const TableT<KT>& t, const FactorT<KT>& f, int probe_width, unsigned long long* sink,
                               int grid, cudaStream_t st) {
  if (!scan_aligned(t)) return cudaErrorMisalignedAddress;
  switch (probe_width) {
    case 2:
      k_probe_bench<KT, 2><<<grid, kStepThreads, 0, st>>>(t, f, sink);
      break;
    case 4:
      k_probe_bench<KT, 4><<<grid, kStepThreads, 0, st>>>(t, f, sink);
      break;
    case 8:
      k_probe_bench<KT, 8><<<grid, kStepThreads, 0, st>>>(t, f, sink);
      break;
    default:
      k_probe_bench<KT, 1><<<grid, kStepThreads, 0, st>>>(t, f, sink);
      break;
  }
  return cudaGetLastError();
}

template cudaError_t launch_probe_bench<unsigned long long>(const Table&, const Factor&, int, unsigned long long*, int,
                                                            cudaStream_t);
template cudaError_t launch_probe_bench<Key128>(const TableT<Key128>&, const FactorT<Key128>&, int,
                                                unsigned long long*, int, cudaStream_t);

}  // namespace ucc
