// Energy: sigma = P_S H psi and <psi|H|psi>, <psi|psi> (Results section's
// UCCSD energy; the Hamiltonian of the Methods section's integrals).
//
// One warp per stored determinant I.  The warp builds I's occupied and empty
// spin-orbital lists by spin in shared memory, then its lanes walk every
// spin-conserving single and double J = tau I, look J up in the hash table
// and, on a hit, add <I|H|J> c_J by the Slater-Condon rules:
//   <I|H|I>   = sum_{p in I} h_pp + 1/2 sum_{p,q in I} <pq||pq>
//   <J|H|I>   = sgn (h_rp + sum_{k in I, k != p} <rk||pk>)     J = a+_r a_p I
//   <J|H|I>   = sgn <rs||pq>                                  J = a+_r a+_s a_q a_p I
// with <pq|rs> = (pr|qs) delta(spin p, spin r) delta(spin q, spin s) and
// <pq||rs> = <pq|rs> - <pq|sr>.  sgn is the Jordan-Wigner sign of the
// operator string on I.

#include "ucc_device.cuh"

namespace ucc {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxSpin = 32;                          // spin-orbitals of one spin
constexpr int kMaxPairs = kMaxSpin * (kMaxSpin - 1) / 2;  // same-spin empty pairs

struct WarpLists {
  unsigned char occ[2][kMaxSpin];
  unsigned char emp[2][kMaxSpin];
  int n_occ[2], n_emp[2];
  unsigned short pairs[2][kMaxPairs];  // same-spin empty pairs (r | s << 8), r < s
  int n_pairs[2];
};

__device__ __forceinline__ unsigned long long below(int p) { return (1ull << p) - 1ull; }

// (ab|cd) in chemist notation over spatial orbitals.
__device__ __forceinline__ double chem(const Integrals& in, int a, int b, int c, int d) {
  const int n = in.n;
  return __ldg(&in.g[((a * n + b) * n + c) * n + d]);
}

// <rs||pq> over spin-orbitals.
__device__ __forceinline__ double anti(const Integrals& in, int r, int s, int p, int q) {
  double v = 0.0;
  if (((r ^ p) & 1) == 0 && ((s ^ q) & 1) == 0) v += chem(in, r >> 1, p >> 1, s >> 1, q >> 1);
  if (((r ^ q) & 1) == 0 && ((s ^ p) & 1) == 0) v -= chem(in, r >> 1, q >> 1, s >> 1, p >> 1);
  return v;
}

__device__ __forceinline__ double h_so(const Integrals& in, int p, int q) {
  if ((p ^ q) & 1) return 0.0;
  return __ldg(&in.h[(p >> 1) * in.n + (q >> 1)]);
}

// Sign of a+_r a+_s a_q a_p |I> (p, q occupied; r, s empty; all distinct).
__device__ __forceinline__ int double_parity(unsigned long long I, int p, int q, int r, int s) {
  const unsigned long long msk = below(p) ^ below(q) ^ below(r) ^ below(s);
  return (__popcll(I & msk) + (p < q) + (p < s) + (q < s) + (p < r) + (q < r) + (s < r)) & 1;
}

// Sign of a+_r a_p |I>.
__device__ __forceinline__ int single_parity(unsigned long long I, int p, int r) {
  return (__popcll(I & (below(p) ^ below(r))) + (p < r)) & 1;
}

__device__ __forceinline__ bool lookup_live(const Table& t, unsigned long long key, double* amp) {
  unsigned long long h = mix64(key) & t.slot_mask;
  for (int step = 0; step < MAX_PROBE; ++step) {
    const Slot s = t.slots[h];
    if (s.key == key) {
      const double a = t.amps[s.idx];
      if (is_dead(a)) return false;
      *amp = a;
      return true;
    }
    if (s.key == 0ull) return false;
    h = (h + 1) & t.slot_mask;
  }
  raise_error(t.cnt, ERR_PROBE_BOUND);
  return false;
}

__global__ void __launch_bounds__(kThreads) k_sigma(Table t, Integrals in) {
  __shared__ WarpLists lists[kWarps];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  WarpLists& L = lists[w];
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long gw = (unsigned long long)blockIdx.x * kWarps + w;
  const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
  double acc_e = 0.0, acc_n = 0.0;  // lane 0 only
  unsigned long long probes = 0, hits = 0;
  for (unsigned long long e = gw; e < n; e += nw) {
    const double cI = t.amps[e];
    if (is_dead(cI)) continue;  // warp-uniform
    const unsigned long long I = t.keys[e];
    if (lane == 0) {
      for (int sp = 0; sp < 2; ++sp) L.n_occ[sp] = L.n_emp[sp] = 0;
      for (int p = 0; p < in.n_so; ++p) {
        const int sp = p & 1;
        if ((I >> p) & 1ull)
          L.occ[sp][L.n_occ[sp]++] = (unsigned char)p;
        else
          L.emp[sp][L.n_emp[sp]++] = (unsigned char)p;
      }
    }
    __syncwarp();
    for (int sp = 0; sp < 2; ++sp) {
      const int m = L.n_emp[sp];
      const int np = m * (m - 1) / 2;
      for (int u = lane; u < np; u += 32) {
        // u -> (x, y), x < y, row-major over the strict upper triangle
        int x = 0, rem = u;
        while (rem >= m - 1 - x) {
          rem -= m - 1 - x;
          ++x;
        }
        const int y = x + 1 + rem;
        L.pairs[sp][u] = (unsigned short)(L.emp[sp][x] | (L.emp[sp][y] << 8));
      }
      if (lane == 0) L.n_pairs[sp] = np;
    }
    __syncwarp();

    double part = 0.0;
    // Diagonal: lanes over the first index p.
    {
      double d = 0.0;
      for (int sp = 0; sp < 2; ++sp)
        for (int x = lane; x < L.n_occ[sp]; x += 32) {
          const int p = L.occ[sp][x];
          d += h_so(in, p, p);
          for (int sq = 0; sq < 2; ++sq)
            for (int y = 0; y < L.n_occ[sq]; ++y) {
              const int q = L.occ[sq][y];
              if (q != p) d += 0.5 * anti(in, p, q, p, q);
            }
        }
      part += d * cI;
    }
    // Singles p -> r, same spin.
    for (int sp = 0; sp < 2; ++sp) {
      const int no = L.n_occ[sp], ne = L.n_emp[sp];
      for (int u = lane; u < no * ne; u += 32) {
        const int p = L.occ[sp][u / ne];
        const int r = L.emp[sp][u % ne];
        const unsigned long long J = I ^ ((1ull << p) | (1ull << r));
        double cJ;
        ++probes;
        if (!lookup_live(t, J, &cJ)) continue;
        ++hits;
        double v = h_so(in, r, p);
        for (int sk = 0; sk < 2; ++sk)
          for (int y = 0; y < L.n_occ[sk]; ++y) {
            const int kk = L.occ[sk][y];
            if (kk != p) v += anti(in, r, kk, p, kk);
          }
        part += (single_parity(I, p, r) ? -v : v) * cJ;
      }
    }
    // Doubles: same-spin (p < q from one spin, r < s from the same spin).
    for (int sp = 0; sp < 2; ++sp) {
      const int no = L.n_occ[sp];
      const int np = L.n_pairs[sp];
      for (int x = 0; x < no; ++x)
        for (int y = x + 1; y < no; ++y) {
          const int p = L.occ[sp][x], q = L.occ[sp][y];
          const unsigned long long hole = (1ull << p) | (1ull << q);
          for (int u = lane; u < np; u += 32) {
            const unsigned short pr = L.pairs[sp][u];
            const int r = pr & 0xFF, s = pr >> 8;
            const unsigned long long J = I ^ (hole | (1ull << r) | (1ull << s));
            double cJ;
            ++probes;
            if (!lookup_live(t, J, &cJ)) continue;
            ++hits;
            const double v = anti(in, r, s, p, q);
            part += (double_parity(I, p, q, r, s) ? -v : v) * cJ;
          }
        }
    }
    // Doubles: opposite spin (p alpha, q beta -> r alpha, s beta).
    {
      const int noa = L.n_occ[0], nob = L.n_occ[1], nea = L.n_emp[0], neb = L.n_emp[1];
      const int nE = nea * neb;
      for (int x = 0; x < noa; ++x)
        for (int y = 0; y < nob; ++y) {
          const int p = L.occ[0][x], q = L.occ[1][y];
          const unsigned long long hole = (1ull << p) | (1ull << q);
          for (int u = lane; u < nE; u += 32) {
            const int r = L.emp[0][u / neb], s = L.emp[1][u % neb];
            const unsigned long long J = I ^ (hole | (1ull << r) | (1ull << s));
            double cJ;
            ++probes;
            if (!lookup_live(t, J, &cJ)) continue;
            ++hits;
            const double v = anti(in, r, s, p, q);
            part += (double_parity(I, p, q, r, s) ? -v : v) * cJ;
          }
        }
    }
    const double sig = warp_sum(part);
    if (lane == 0) {
      t.sigma[e] = sig;
      acc_e += cI * sig;
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
__global__ void __launch_bounds__(256) k_lambda_init(Table t) {
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

int sigma_smem_bytes(int) { return (int)sizeof(WarpLists) * kWarps; }

cudaError_t launch_sigma(const Table& t, const Integrals& in, int grid, cudaStream_t st) {
  k_sigma<<<grid, kThreads, 0, st>>>(t, in);
  return cudaGetLastError();
}

cudaError_t launch_lambda_init(const Table& t, int grid, cudaStream_t st) {
  k_lambda_init<<<grid, 256, 0, st>>>(t);
  return cudaGetLastError();
}

}  // namespace ucc
