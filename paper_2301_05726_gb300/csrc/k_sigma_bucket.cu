// Energy by buckets of shared cores: sigma_I = sum_{J in S} <I|H|J> c_J over
// the stored set S with work proportional to the connected pairs inside S.
//
// Two determinants I != J of S are connected by a double excitation exactly
// when they share the (n_e - 2)-electron core K2 = I minus two electrons =
// J minus two other electrons, and then K2 = I & J is unique; by a single
// excitation exactly when they share the (n_e - 1)-electron core K1 = I & J.
// So every stored I emits one record per removed set (n_e singles and
// n_e (n_e - 1) / 2 doubles, with c_I and its entry index); the records are
// hashed on the core into partitions that fit one block's shared memory, and
// within a partition the records of one core form a group whose pairs are
// exactly the connections (Slater-Condon rules; for doubles only the pairs
// whose removed sets are disjoint: the others are singles, counted in their
// K1 group, or the determinant itself).  The diagonal is added per entry.
// E = <psi|H|psi> / <psi|psi> (Results section) follows from sigma.
//
// Layout: records are 32 bytes (one DRAM sector, one 256-bit store) for
// either key width in HBM, written partition by partition in rounds whose
// records fit a fixed buffer; a partition's records are counted into bins on
// 11 further bits of the core's hash (a core's records share a bin), placed
// into shared memory in bin order, and the ordered pairs of every bin are
// split evenly over the block's threads.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

// Removed spin-orbitals of a record: p | q << 8, q = kSingle for a single.
constexpr unsigned int kSingle = 0xFFu;
// Records per partition held in shared memory, and the counting-sort bins.
constexpr int kSbCap = 3072;
constexpr int kSbBins = 2048;  // a multiple of kSbThreads
constexpr int kSbBinBits = 11;
constexpr int kSbThreads = 512;

template <class KT>
__device__ __forceinline__ unsigned long long core_hash(KT K) {
  return KeyOps<KT>::slot_hash(K);
}

__device__ __forceinline__ unsigned long long partition_of(unsigned long long h, int log2p) {
  return log2p == 0 ? 0ull : (h >> (64 - log2p));
}

__device__ __forceinline__ int bin_of(unsigned long long h, int log2p) {
  return (int)((h >> (64 - log2p - kSbBinBits)) & (unsigned long long)(kSbBins - 1));
}

// f(p) for every set bit p of k, ascending.
template <class F>
__device__ __forceinline__ void for_each_bit(unsigned long long k, int offset, F f) {
  for (unsigned long long x = k; x != 0ull; x &= x - 1ull) f(__ffsll((long long)x) - 1 + offset);
}
template <class F>
__device__ __forceinline__ void for_each_bit(Key128 k, int, F f) {
  for_each_bit(k.lo, 0, f);
  for_each_bit(k.hi, 64, f);
}

// f(core, removed) for the n_e single and n_e (n_e - 1) / 2 double cores of I.
template <class KT, class F>
__device__ __forceinline__ void for_each_core(KT I, F f) {
  using K = KeyOps<KT>;
  for_each_bit(I, 0, [&](int p) {
    const KT Ip = I ^ K::bit(p);
    f(Ip, (unsigned int)p | (kSingle << 8));
    // q > p: the bits of I above p
    for_each_bit(I & ~K::below(p + 1), 0, [&](int q) { f(Ip ^ K::bit(q), (unsigned int)p | ((unsigned int)q << 8)); });
  });
}

// Records per core partition.
template <class KT>
__global__ void __launch_bounds__(256) k_sb_count(TableT<KT> t, unsigned int* __restrict__ cnt, int log2p) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (is_dead(t.amps[i])) continue;
    for_each_core(t.keys[i], [&](KT core, unsigned int) { atomicAdd(&cnt[partition_of(core_hash(core), log2p)], 1u); });
  }
}

// Exclusive prefix sum of n counts into off[0..n] by one block (the counts
// of one energy evaluation: at most a few million partitions).
__global__ void __launch_bounds__(1024) k_sb_scan(const unsigned int* __restrict__ cnt,
                                                  unsigned long long* __restrict__ off, unsigned long long n) {
  __shared__ unsigned long long s_part[1024];
  const unsigned long long per = (n + blockDim.x - 1) / blockDim.x;
  const unsigned long long lo = min(n, (unsigned long long)threadIdx.x * per), hi = min(n, lo + per);
  unsigned long long sum = 0;
  for (unsigned long long x = lo; x < hi; ++x) sum += cnt[x];
  s_part[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan of the thread sums.
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned int)d ? s_part[threadIdx.x - d] : 0ull;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x ? s_part[threadIdx.x - 1] : 0ull;
  for (unsigned long long x = lo; x < hi; ++x) {
    off[x] = run;
    run += cnt[x];
  }
  if (threadIdx.x == blockDim.x - 1) off[n] = s_part[threadIdx.x];
}

// A record as one 256-bit store (a whole 32-byte sector: no partial-sector
// write for the memory to merge).
__device__ __forceinline__ void store_words(void* at, unsigned long long a, unsigned long long b, unsigned long long c,
                                            unsigned long long d) {
  asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(at), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}
__device__ __forceinline__ void store_record(SigRecT<unsigned long long>* at, unsigned long long K, double c,
                                             unsigned int i, unsigned int pq) {
  store_words(at, K, (unsigned long long)__double_as_longlong(c), (unsigned long long)i | ((unsigned long long)pq << 32),
              0ull);
}
__device__ __forceinline__ void store_record(SigRecT<Key128>* at, Key128 K, double c, unsigned int i,
                                             unsigned int pq) {
  store_words(at, K.lo, K.hi, (unsigned long long)__double_as_longlong(c),
              (unsigned long long)i | ((unsigned long long)pq << 32));
}

// The records of partitions [p0, p1), at rec[off[p] - base + fill[p]++].
template <class KT>
__global__ void __launch_bounds__(256) k_sb_scatter(TableT<KT> t, const unsigned long long* __restrict__ off,
                                                    unsigned int* __restrict__ fill, SigRecT<KT>* __restrict__ rec,
                                                    int log2p, unsigned long long p0, unsigned long long p1,
                                                    unsigned long long base) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double c = t.amps[i];
    if (is_dead(c)) continue;
    for_each_core(t.keys[i], [&](KT core, unsigned int removed) {
      const unsigned long long p = partition_of(core_hash(core), log2p);
      if (p < p0 || p >= p1) return;
      const unsigned long long f = atomicAdd(&fill[p], 1u);
      if (off[p] + f >= off[p + 1]) {  // more records than counted: never written past
        raise_error(t.cnt, ERR_CAPACITY);
        return;
      }
      store_record(rec + (off[p] - base + f), core, c, (unsigned int)i, removed);
    });
  }
}

// <I|H|J> for I = K + removed rx and J = K + removed rw (records of one core
// group, I != J), in *h; false when the pair is not an excitation of the
// group's kind (two doubles whose removed sets overlap: a single, counted in
// its own group).  Conventions as in the probe route: a single p -> r is
// h_rp + sum_{k in K} <rk||pk> with the sign of a+_r a_p |I>; a double
// p, q -> r, s is <rs||pq> with the sign of a+_r a+_s a_q a_p |I>.
template <class KT>
__device__ __forceinline__ bool pair_element(const Integrals& in, KT K, unsigned int rx, unsigned int rw, double* h) {
  using Ko = KeyOps<KT>;
  const int p = (int)(rx & 0xFFu), q = (int)(rx >> 8), r = (int)(rw & 0xFFu), s = (int)(rw >> 8);
  if ((unsigned int)q == kSingle) {
    double v = h_so(in, r, p);
    for_each_bit(K, 0, [&](int k) { v += anti(in, r, k, p, k); });
    *h = neg_if(v, single_parity(K | Ko::bit(p), p, r));
    return true;
  }
  if (p == r || p == s || q == r || q == s) return false;
  // <rs||pq> = (rp|sq) [spins of r, p and of s, q agree] - (rq|sp) [spins of
  // r, q and of s, p agree]: one term for opposite spins, two for equal ones.
  // FP64 is a narrow pipe on this GPU, so the zero start, the negations and
  // the sign are not FP64 operations (same values as anti()).
  const bool t1 = ((r ^ p) & 1) == 0 && ((s ^ q) & 1) == 0;
  const bool t2 = ((r ^ q) & 1) == 0 && ((s ^ p) & 1) == 0;
  double v = 0.0;
  if (t1 && t2)
    v = __dsub_rn(chem(in, r >> 1, p >> 1, s >> 1, q >> 1), chem(in, r >> 1, q >> 1, s >> 1, p >> 1));
  else if (t1)
    v = chem(in, r >> 1, p >> 1, s >> 1, q >> 1);
  else if (t2)
    v = neg_if(chem(in, r >> 1, q >> 1, s >> 1, p >> 1), 1);
  *h = neg_if(v, double_parity(K | Ko::bit(p) | Ko::bit(q), p, q, r, s));
  return true;
}

// A partition too large for shared memory: every record walks the whole
// partition in global memory (quadratic, for rare oversized partitions).
template <class KT>
__device__ unsigned long long pairs_in_global(const TableT<KT>& t, const Integrals& in, const SigRecT<KT>* r,
                                              unsigned long long m) {
  unsigned long long pairs = 0;
  for (unsigned long long x = threadIdx.x; x < m; x += blockDim.x) {
    const SigRecT<KT> a = r[x];
    double acc = 0.0;
    for (unsigned long long z = 0; z < m; ++z) {
      if (z == x) continue;
      const KT Kz = r[z].K;
      if (!(Kz == a.K)) continue;
      double h;
      if (pair_element(in, a.K, a.pq, r[z].pq, &h)) {
        acc += h * r[z].c;
        ++pairs;
      }
    }
    if (nonzero(acc)) atomicAdd(&t.sigma[a.i], acc);
  }
  return pairs;
}

template <class KT>
constexpr size_t sb_smem_bytes() {
  return (size_t)kSbCap * (sizeof(KT) + sizeof(double) + sizeof(unsigned int) + sizeof(unsigned short)) +
         (size_t)(3 * kSbBins + 2) * sizeof(unsigned int);
}

// Exclusive scans over the bins of n_b records (into sa) and of n_b (n_b - 1)
// ordered pairs (into sb), kSbBins + 1 entries each with the totals last; cnt
// is overwritten with sa (the placement cursors).  Warp-shuffle scans, two
// block barriers.  Every thread of the block calls this.
__device__ __forceinline__ void scan_bins(unsigned int* cnt, unsigned int* sa, unsigned int* sb, unsigned int* s_wa,
                                          unsigned int* s_wb) {
  constexpr int kPer = kSbBins / kSbThreads;
  constexpr int kWarps = kSbThreads / 32;
  const unsigned int tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
  unsigned int n[kPer], ta = 0u, tb = 0u;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    n[u] = cnt[tid * kPer + u];
    ta += n[u];
    tb += n[u] * (n[u] ? n[u] - 1u : 0u);
  }
  unsigned int ia = ta, ib = tb;  // inclusive within the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned int ya = __shfl_up_sync(0xFFFFFFFFu, ia, d), yb = __shfl_up_sync(0xFFFFFFFFu, ib, d);
    if (lane >= (unsigned int)d) {
      ia += ya;
      ib += yb;
    }
  }
  if (lane == 31u) {
    s_wa[wid] = ia;
    s_wb[wid] = ib;
  }
  __syncthreads();
  if (wid == 0) {
    unsigned int va = lane < (unsigned int)kWarps ? s_wa[lane] : 0u, vb = lane < (unsigned int)kWarps ? s_wb[lane] : 0u;
    unsigned int xa = va, xb = vb;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int ya = __shfl_up_sync(0xFFFFFFFFu, xa, d), yb = __shfl_up_sync(0xFFFFFFFFu, xb, d);
      if (lane >= (unsigned int)d) {
        xa += ya;
        xb += yb;
      }
    }
    if (lane < (unsigned int)kWarps) {
      s_wa[lane] = xa - va;  // exclusive prefix of the warp totals
      s_wb[lane] = xb - vb;
    }
    if (lane == (unsigned int)kWarps - 1u) {
      sa[kSbBins] = xa;
      sb[kSbBins] = xb;
    }
  }
  __syncthreads();
  unsigned int ra = s_wa[wid] + ia - ta, rb = s_wb[wid] + ib - tb;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    sa[tid * kPer + u] = ra;
    sb[tid * kPer + u] = rb;
    cnt[tid * kPer + u] = ra;
    ra += n[u];
    rb += n[u] * (n[u] ? n[u] - 1u : 0u);
  }
}

// One block per partition of [p0, p1) (grid-stride).  The partition's records
// are counted by core-hash bin (a core's records share a bin), placed into
// shared memory in bin order, and then the ordered pairs (x, w), x != w, of
// every bin are split evenly over the threads: each walks its contiguous share
// of pair indices, evaluates <I_x|H|J_w> c_w where the cores agree, and adds
// the sum of a record to sigma when its walk leaves that record.
template <class KT>
__global__ void __launch_bounds__(kSbThreads) k_sb_pairs(TableT<KT> t, Integrals in, const SigRecT<KT>* __restrict__ rec,
                                                         const unsigned long long* __restrict__ off, int log2p,
                                                         unsigned long long p0, unsigned long long p1,
                                                         unsigned long long base) {
  extern __shared__ __align__(16) unsigned char sb_smem[];
  KT* sK = reinterpret_cast<KT*>(sb_smem);
  double* sc = reinterpret_cast<double*>(sK + kSbCap);
  unsigned int* si = reinterpret_cast<unsigned int*>(sc + kSbCap);
  unsigned short* sp = reinterpret_cast<unsigned short*>(si + kSbCap);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(sp + kSbCap);  // counts, then placement cursors
  unsigned int* start = cnt + kSbBins;                                // kSbBins + 1: records before each bin
  unsigned int* pst = start + kSbBins + 1;                            // kSbBins + 1: ordered pairs before each bin
  __shared__ unsigned int s_a[kSbThreads / 32], s_b[kSbThreads / 32];
  const unsigned int tid = threadIdx.x;
  unsigned long long pairs = 0;
  for (unsigned long long p = p0 + blockIdx.x; p < p1; p += gridDim.x) {
    const unsigned long long lo = off[p] - base, m = off[p + 1] - off[p];
    if (m == 0) continue;
    if (m > (unsigned long long)kSbCap) {
      pairs += pairs_in_global(t, in, rec + lo, m);
      continue;
    }
    const int mi = (int)m;
    for (int b = (int)tid; b < kSbBins; b += kSbThreads) cnt[b] = 0u;
    __syncthreads();
    for (int x = (int)tid; x < mi; x += kSbThreads) atomicAdd(&cnt[bin_of(core_hash(rec[lo + x].K), log2p)], 1u);
    __syncthreads();
    scan_bins(cnt, start, pst, s_a, s_b);
    __syncthreads();
    for (int x = (int)tid; x < mi; x += kSbThreads) {
      const SigRecT<KT> r = rec[lo + (unsigned long long)x];
      const unsigned int at = atomicAdd(&cnt[bin_of(core_hash(r.K), log2p)], 1u);
      sK[at] = r.K;
      sc[at] = r.c;
      si[at] = r.i;
      sp[at] = r.pq;
    }
    __syncthreads();
    const unsigned int T = pst[kSbBins];
    const unsigned int per = (T + kSbThreads - 1u) / kSbThreads;
    unsigned int j = tid * per;
    const unsigned int j_end = min(T, j + per);
    if (j < j_end) {
      // the bin holding pair index j: the last b with pst[b] <= j
      int lo_b = 0, hi_b = kSbBins;
      while (hi_b - lo_b > 1) {
        const int mid = (lo_b + hi_b) >> 1;
        if (pst[mid] <= j)
          lo_b = mid;
        else
          hi_b = mid;
      }
      int b = lo_b;
      unsigned int mb = start[b + 1] - start[b];
      unsigned int loc = j - pst[b];
      unsigned int u = loc / (mb - 1u), v = loc % (mb - 1u);
      v += (v >= u) ? 1u : 0u;
      unsigned int x = start[b] + u;
      KT K = sK[x];
      unsigned int rx = sp[x];
      double acc = 0.0;
      for (; j < j_end; ++j) {
        const unsigned int w = start[b] + v;
        if (sK[w] == K) {
          double h;
          if (pair_element(in, K, rx, sp[w], &h)) {
            acc += h * sc[w];
            ++pairs;
          }
        }
        // next pair: (u, v + 1) skipping v == u; then the next record; then
        // the next bin holding a pair
        if (++v == u) ++v;
        if (v >= mb) {
          if (nonzero(acc)) atomicAdd(&t.sigma[si[x]], acc);
          acc = 0.0;
          if (++u >= mb) {
            if (j + 1u >= j_end) break;
            do {
              ++b;
            } while (pst[b + 1] == pst[b]);
            mb = start[b + 1] - start[b];
            u = 0u;
          }
          v = (u == 0u) ? 1u : 0u;
          x = start[b] + u;
          K = sK[x];
          rx = sp[x];
        }
      }
      if (nonzero(acc)) atomicAdd(&t.sigma[si[x]], acc);
    }
    __syncthreads();  // shared arrays are refilled for the next partition
  }
  pairs = warp_sum_u64(pairs);
  if ((tid & 31u) == 0 && pairs) atomicAdd(&t.cnt->sig_hits, pairs);
}

// sigma_I += <I|H|I> c_I on every live entry, then E's numerator
// sum c_I sigma_I and <psi|psi> (block partials, summed in a fixed order by
// the last block).
template <class KT>
__global__ void __launch_bounds__(256) k_sb_finish(TableT<KT> t, Integrals in) {
  using Ko = KeyOps<KT>;
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  double acc_e = 0.0, acc_n = 0.0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double c = t.amps[i];
    if (is_dead(c)) continue;
    const KT I = t.keys[i];
    double d = 0.0;
    for_each_bit(I, 0, [&](int p) {
      d += h_so(in, p, p);
      for_each_bit(I & ~Ko::below(p + 1), 0, [&](int q) { d += anti(in, p, q, p, q); });
    });
    const double s = t.sigma[i] + d * c;
    t.sigma[i] = s;
    acc_e += c * s;
    acc_n += c * c;
  }
  const double be = block_sum(acc_e);
  const double bn = block_sum(acc_n);
  if (threadIdx.x == 0) {
    t.partials[2 * blockIdx.x] = be;
    t.partials[2 * blockIdx.x + 1] = bn;
  }
  if (last_block_arrive(t.cnt)) {
    double se = 0.0, sn = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
      se += ld_cg(&t.partials[2 * b]);
      sn += ld_cg(&t.partials[2 * b + 1]);
    }
    se = block_sum(se);
    sn = block_sum(sn);
    if (threadIdx.x == 0) {
      t.cnt->e_num = se;
      t.cnt->norm2 = sn;
      t.cnt->done = 0u;
    }
  }
}

}  // namespace

size_t sb_record_bytes(int key_words) { return key_words == 2 ? sizeof(SigRecT<Key128>) : sizeof(SigRecT<unsigned long long>); }

template <class KT>
cudaError_t launch_sb_count(const TableT<KT>& t, unsigned int* cnt, int log2p, int grid, cudaStream_t st) {
  k_sb_count<KT><<<grid, 256, 0, st>>>(t, cnt, log2p);
  return cudaGetLastError();
}

cudaError_t launch_sb_scan(const unsigned int* cnt, unsigned long long* off, unsigned long long n, cudaStream_t st) {
  k_sb_scan<<<1, 1024, 0, st>>>(cnt, off, n);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_sb_scatter(const TableT<KT>& t, const unsigned long long* off, unsigned int* fill,
                              SigRecT<KT>* rec, int log2p, unsigned long long p0, unsigned long long p1,
                              unsigned long long base, int grid, cudaStream_t st) {
  k_sb_scatter<KT><<<grid, 256, 0, st>>>(t, off, fill, rec, log2p, p0, p1, base);
  return cudaGetLastError();
}

// The pairs kernel's dynamic shared memory is above the default 48 KB limit:
// raised (for the current device) before every launch and occupancy query.
template <class KT>
cudaError_t sb_allow_smem() {
  return cudaFuncSetAttribute(k_sb_pairs<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb_smem_bytes<KT>());
}

template <class KT>
cudaError_t launch_sb_pairs(const TableT<KT>& t, const Integrals& in, const SigRecT<KT>* rec,
                            const unsigned long long* off, int log2p, unsigned long long p0, unsigned long long p1,
                            unsigned long long base, int grid, cudaStream_t st) {
  const cudaError_t e = sb_allow_smem<KT>();
  if (e != cudaSuccess) return e;
  k_sb_pairs<KT><<<grid, kSbThreads, sb_smem_bytes<KT>(), st>>>(t, in, rec, off, log2p, p0, p1, base);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_sb_finish(const TableT<KT>& t, const Integrals& in, int grid, cudaStream_t st) {
  k_sb_finish<KT><<<grid, 256, 0, st>>>(t, in);
  return cudaGetLastError();
}

int sb_blocks_per_sm(int key_words) {
  int nb = 0;
  cudaError_t e;
  if (key_words == 2) {
    e = sb_allow_smem<Key128>();
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sb_pairs<Key128>, kSbThreads, sb_smem_bytes<Key128>());
  } else {
    e = sb_allow_smem<unsigned long long>();
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sb_pairs<unsigned long long>, kSbThreads,
                                                        sb_smem_bytes<unsigned long long>());
  }
  return e == cudaSuccess ? nb : 0;
}

int sb_partition_target() { return kSbCap / 2; }

#define UCC_SB_INSTANTIATE(KT)                                                                                      \
  template cudaError_t launch_sb_count<KT>(const TableT<KT>&, unsigned int*, int, int, cudaStream_t);             \
  template cudaError_t launch_sb_scatter<KT>(const TableT<KT>&, const unsigned long long*, unsigned int*,         \
                                             SigRecT<KT>*, int, unsigned long long, unsigned long long,            \
                                             unsigned long long, int, cudaStream_t);                               \
  template cudaError_t launch_sb_pairs<KT>(const TableT<KT>&, const Integrals&, const SigRecT<KT>*,               \
                                           const unsigned long long*, int, unsigned long long, unsigned long long, \
                                           unsigned long long, int, cudaStream_t);                                 \
  template cudaError_t launch_sb_finish<KT>(const TableT<KT>&, const Integrals&, int, cudaStream_t);
UCC_SB_INSTANTIATE(unsigned long long)
UCC_SB_INSTANTIATE(Key128)

}  // namespace ucc
