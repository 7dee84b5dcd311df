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
// Layout: records are 24 bytes for one-word keys (32 for two-word ones) in
// HBM, written partition by partition in rounds whose records fit a fixed
// buffer; a partition's records are read once into shared memory, grouped by
// a counting sort on 11 further bits of the core's hash, and each record's
// group is walked from shared memory.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

// Removed spin-orbitals of a record: p | q << 8, q = kSingle for a single.
constexpr unsigned int kSingle = 0xFFu;
// Records per partition held in shared memory, and the counting-sort bins.
constexpr int kSbCap = 3072;
constexpr int kSbBins = 2048;
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
      const unsigned long long at = off[p] - base + f;
      SigRecT<KT> r;
      r.K = core;
      r.c = c;
      r.i = (unsigned int)i;
      r.pq = (unsigned short)removed;
      r.pad = 0;
      rec[at] = r;
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
    *h = single_parity(K | Ko::bit(p), p, r) ? -v : v;
    return true;
  }
  if (p == r || p == s || q == r || q == s) return false;
  const double v = anti(in, r, s, p, q);
  *h = double_parity(K | Ko::bit(p) | Ko::bit(q), p, q, r, s) ? -v : v;
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
    if (acc != 0.0) atomicAdd(&t.sigma[a.i], acc);
  }
  return pairs;
}

template <class KT>
constexpr size_t sb_smem_bytes() {
  return (size_t)kSbCap * (sizeof(KT) + sizeof(double) + sizeof(unsigned int) + 2 * sizeof(unsigned short) +
                           sizeof(unsigned short)) +
         (size_t)(2 * kSbBins + 1) * sizeof(unsigned int);
}

// One block per partition of [p0, p1) (grid-stride): the partition's records
// into shared memory, a counting sort by core-hash bin, then every record sums
// <I|H|J> c_J over the records of its core (found within its bin) and adds the
// sum to sigma_I.
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
  unsigned short* sb = sp + kSbCap;
  unsigned short* perm = sb + kSbCap;
  unsigned int* cursor = reinterpret_cast<unsigned int*>(perm + kSbCap);
  unsigned int* start = cursor + kSbBins;  // kSbBins + 1 entries
  __shared__ unsigned int s_sum[kSbThreads];
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
    for (int b = (int)tid; b < kSbBins; b += kSbThreads) cursor[b] = 0u;
    __syncthreads();
    for (int x = (int)tid; x < mi; x += kSbThreads) {
      const SigRecT<KT> r = rec[lo + (unsigned long long)x];
      sK[x] = r.K;
      sc[x] = r.c;
      si[x] = r.i;
      sp[x] = r.pq;
      const int b = bin_of(core_hash(r.K), log2p);
      sb[x] = (unsigned short)b;
      atomicAdd(&cursor[b], 1u);
    }
    __syncthreads();
    // Exclusive scan of the bin counts: four bins per thread, then the
    // thread sums (Hillis-Steele).
    constexpr int kPer = kSbBins / kSbThreads;
    unsigned int v[kPer], tot = 0u;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      v[u] = cursor[tid * kPer + u];
      tot += v[u];
    }
    s_sum[tid] = tot;
    __syncthreads();
    for (int d = 1; d < kSbThreads; d <<= 1) {
      const unsigned int a = tid >= (unsigned int)d ? s_sum[tid - d] : 0u;
      __syncthreads();
      s_sum[tid] += a;
      __syncthreads();
    }
    unsigned int run = tid ? s_sum[tid - 1] : 0u;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      start[tid * kPer + u] = run;
      cursor[tid * kPer + u] = run;
      run += v[u];
    }
    if (tid == 0) start[kSbBins] = (unsigned int)mi;
    __syncthreads();
    for (int x = (int)tid; x < mi; x += kSbThreads) perm[atomicAdd(&cursor[sb[x]], 1u)] = (unsigned short)x;
    __syncthreads();
    // Sorted positions: the lanes of a warp mostly share a bin and a core.
    for (int y = (int)tid; y < mi; y += kSbThreads) {
      const int x = perm[y];
      const KT K = sK[x];
      const unsigned int rx = sp[x];
      const int b = sb[x];
      double acc = 0.0;
      for (int z = (int)start[b]; z < (int)start[b + 1]; ++z) {
        const int w = perm[z];
        if (w == x || !(sK[w] == K)) continue;
        double h;
        if (pair_element(in, K, rx, sp[w], &h)) {
          acc += h * sc[w];
          ++pairs;
        }
      }
      if (acc != 0.0) atomicAdd(&t.sigma[si[x]], acc);
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

template <class KT>
cudaError_t launch_sb_pairs(const TableT<KT>& t, const Integrals& in, const SigRecT<KT>* rec,
                            const unsigned long long* off, int log2p, unsigned long long p0, unsigned long long p1,
                            unsigned long long base, int grid, cudaStream_t st) {
  constexpr size_t smem = sb_smem_bytes<KT>();
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_sb_pairs<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_sb_pairs<KT><<<grid, kSbThreads, smem, st>>>(t, in, rec, off, log2p, p0, p1, base);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_sb_finish(const TableT<KT>& t, const Integrals& in, int grid, cudaStream_t st) {
  k_sb_finish<KT><<<grid, 256, 0, st>>>(t, in);
  return cudaGetLastError();
}

int sb_blocks_per_sm(int key_words) {
  int nb = 0;
  const cudaError_t e =
      key_words == 2
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sb_pairs<Key128>, kSbThreads, sb_smem_bytes<Key128>())
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sb_pairs<unsigned long long>, kSbThreads,
                                                          sb_smem_bytes<unsigned long long>());
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
