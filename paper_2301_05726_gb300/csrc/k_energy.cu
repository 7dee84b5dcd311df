// Energy: sigma = P_S H psi and <psi|H|psi>, <psi|psi> (Results section's
// UCCSD energy; the Hamiltonian of the Methods section's integrals).
//
// One warp per stored determinant I.  The warp builds I's occupied and empty
// spin-orbital lists by spin in shared memory, then its lanes walk the
// spin-conserving singles and doubles J = tau I with J < I, look J up in the
// hash table and, on a hit, add <I|H|J> c_J to sigma_I and <J|H|I> c_I to
// sigma_J (H is real symmetric, so each connected stored pair is visited once,
// from its larger key), by the Slater-Condon rules:
//   <I|H|I>   = sum_{p in I} h_pp + 1/2 sum_{p,q in I} <pq||pq>
//   <J|H|I>   = sgn (h_rp + sum_{k in I, k != p} <rk||pk>)     J = a+_r a_p I
//   <J|H|I>   = sgn <rs||pq>                                  J = a+_r a+_s a_q a_p I
// with <pq|rs> = (pr|qs) delta(spin p, spin r) delta(spin q, spin s) and
// <pq||rs> = <pq|rs> - <pq|sr>.  sgn is the Jordan-Wigner sign of the
// operator string on I.  <psi|H|psi> = sum_I c_I^2 <I|H|I> + 2 sum_{J<I} c_I
// <I|H|J> c_J is summed alongside.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

// Warps per block of the energy kernel: the warps' connection lists fill the
// static shared memory (two-word keys have four times the pair lists).
template <class KT>
__host__ __device__ constexpr int sigma_warps() {
  return sizeof(KT) == 8 ? 8 : 2;
}
// Blocks per SM that the lists allow (47 KB a block for one-word keys, 39 KB
// for two-word ones, of 228 KB); the register budget is held to match.
template <class KT>
__host__ __device__ constexpr int sigma_min_blocks() {
  return sizeof(KT) == 8 ? 4 : 5;
}
// sigma[0, n_tail) = 0 before the lower-triangle pass accumulates into it.
template <class KT>
__global__ void __launch_bounds__(256) k_sigma_zero(TableT<KT> t) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    t.sigma[i] = 0.0;
}

template <class KT>
__global__ void __launch_bounds__(sigma_warps<KT>() * 32, sigma_min_blocks<KT>()) k_sigma(TableT<KT> t, Integrals in) {
  constexpr int kWarps = sigma_warps<KT>();
  __shared__ LowerLists<KT> lists[kWarps];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  LowerLists<KT>& L = lists[w];
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long gw = (unsigned long long)blockIdx.x * kWarps + w;
  const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
  double acc_e = 0.0, acc_n = 0.0;  // lane 0 only
  unsigned long long probes = 0, hits = 0;
  for (unsigned long long e = gw; e < n; e += nw) {
    const double cI = t.amps[e];
    if (is_dead(cI)) continue;  // warp-uniform
    const KT I = t.keys[e];
    double d;
    double part = sigma_lower(t, in, L, I, cI, lane, d, probes, hits);
    d = warp_sum(d);
    part = warp_sum(part);
    if (lane == 0) {
      const double dc = d * cI;
      atomicAdd(&t.sigma[e], dc + part);
      acc_e += cI * (dc + 2.0 * part);
      acc_n += cI * cI;
    }
    __syncwarp();
  }
  {
    __shared__ unsigned long long s_pr, s_hi;
    if (threadIdx.x == 0) s_pr = s_hi = 0;
    __syncthreads();
    if (probes) atomicAdd(&s_pr, probes);
    if (hits) atomicAdd(&s_hi, hits);
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(&t.cnt->sig_probes, s_pr);
      atomicAdd(&t.cnt->sig_hits, s_hi);
    }
  }
  const double be = block_sum(acc_e);
  const double bn = block_sum(acc_n);
  if (threadIdx.x == 0) {
    t.partials[2 * blockIdx.x] = be;
    t.partials[2 * blockIdx.x + 1] = bn;
  }
  if (last_block_arrive(t.cnt)) {
    // Fixed-order sum of the block partials.
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

// mu_K = (sigma - E psi) / <psi|psi> on the live entries; 0 on dropped ones.
template <class KT>
__global__ void __launch_bounds__(256) k_lambda_init(TableT<KT> t) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const double norm2 = *((volatile double*)&t.cnt->norm2);
  const double E = *((volatile double*)&t.cnt->e_num) / norm2;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    t.lam[i] = is_dead(a) ? 0.0 : (t.sigma[i] - E * a) / norm2;
  }
}

}  // namespace

template <class KT>
cudaError_t launch_sigma(const TableT<KT>& t, const Integrals& in, int grid, cudaStream_t st) {
  k_sigma_zero<KT><<<grid, 256, 0, st>>>(t);
  k_sigma<KT><<<grid, sigma_warps<KT>() * 32, 0, st>>>(t, in);
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_lambda_init(const TableT<KT>& t, int grid, cudaStream_t st) {
  k_lambda_init<KT><<<grid, 256, 0, st>>>(t);
  return cudaGetLastError();
}

template cudaError_t launch_sigma<unsigned long long>(const Table&, const Integrals&, int, cudaStream_t);
template cudaError_t launch_sigma<Key128>(const TableT<Key128>&, const Integrals&, int, cudaStream_t);
template cudaError_t launch_lambda_init<unsigned long long>(const Table&, int, cudaStream_t);
template cudaError_t launch_lambda_init<Key128>(const TableT<Key128>&, int, cudaStream_t);

}  // namespace ucc
