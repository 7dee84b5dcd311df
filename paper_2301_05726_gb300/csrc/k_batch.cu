// Batched (many-job) kernels: one launch advances every job of a batch by one
// factor (forward or reverse), or evaluates every job's energy.
//
// Index space of a step: the jobs' stored entries laid end to end, each job's
// range padded to a multiple of 32 so that a warp never straddles two jobs.
// A warp finds its job by binary search over the step's offsets (kept in
// shared memory) and runs the same per-entry body as the single-problem
// kernels on that job's table.  Uneven jobs therefore share every launch: 256
// jobs of 16-36 spin-orbitals need max_j K_j launches per pass, not sum_j K_j,
// and a large job spreads over the whole GPU instead of one block.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

constexpr int kThreads = 256;
// The energy kernel's blocks: four warps keep the job table and the warps'
// connection lists within the static shared-memory limit.
constexpr int kSigmaWarps = 4;

__device__ __forceinline__ int job_of(const unsigned long long* base, int n_jobs, unsigned long long g) {
  int lo = 0, hi = n_jobs - 1;  // largest j with base[j] <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void load_bases(const JobState* js, int n_jobs, const BatchHeader* bh,
                                           unsigned long long* s_base) {
  for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) s_base[j] = js[j].base;
  if (threadIdx.x == 0) s_base[n_jobs] = *((volatile const unsigned long long*)&bh->total);
  __syncthreads();
}

// Sizes of this step's job ranges.  mode 0: forward (n_scan of jobs still
// applying factors, padded), 1: energy (n_tail of every job, unpadded, one warp
// per entry), 2: reverse (n_tail of jobs still undoing factors, padded), 3: the
// tape records of each job's current reverse factor (unpadded).
__device__ void layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int mode) {
  if (threadIdx.x != 0) return;
  unsigned long long total = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const JobView& jv = jobs[j];
    const Counters* c = jv.t.cnt;
    unsigned long long n = 0, w = 0;
    const int k = js[j].k;
    if (mode == 0) {
      if (k < jv.K && js[j].stop < 0) n = min(*((volatile const unsigned long long*)&c->n_scan), jv.t.cap_n);
      w = (n + 31ull) & ~31ull;
    } else if (mode == 1) {
      n = min(*((volatile const unsigned long long*)&c->n_tail), jv.t.cap_n);
      w = n;
    } else if (mode == 2) {
      if (k >= 0) n = min(*((volatile const unsigned long long*)&c->n_tail), jv.t.cap_n);
      w = (n + 31ull) & ~31ull;
    } else {
      if (k >= 0) {
        const unsigned long long hi = min(jv.tape.off[k + 1], jv.tape.cap);
        const unsigned long long lo = min(jv.tape.off[k], hi);
        n = hi - lo;
      }
      w = n;
    }
    js[j].base = total;
    js[j].n = n;
    total += w;
  }
  bh->total = total;
}

__global__ void k_batch_layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int mode) {
  layout(jobs, js, n_jobs, bh, mode);
}

__device__ __forceinline__ void flush_counts(Counters* c, StepCounts& sc) {
  const unsigned int lane = threadIdx.x & 31u;
  unsigned long long v[4] = {sc.rot, sc.cre, sc.dnew, sc.dold};
  long long dd = sc.dead_delta;
  for (int o = 16; o > 0; o >>= 1) {
    for (int x = 0; x < 4; ++x) v[x] += __shfl_xor_sync(0xFFFFFFFFu, v[x], o);
    dd += __shfl_xor_sync(0xFFFFFFFFu, dd, o);
  }
  if (lane == 0) {
    if (v[0]) atomicAdd(&c->rotations, v[0]);
    if (v[1]) atomicAdd(&c->created, v[1]);
    if (v[2]) atomicAdd(&c->dropped_new, v[2]);
    if (v[3]) atomicAdd(&c->dropped_old, v[3]);
    if (dd) atomicAdd(&c->n_dead, (unsigned long long)dd);
  }
  sc = StepCounts();
}

template <bool RECORD>
__global__ void __launch_bounds__(kThreads) k_forward_batch(const JobView* jobs, JobState* js, int n_jobs,
                                                             BatchHeader* bh) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  StepCounts sc;
  int cur = -1;
  for (unsigned long long g = warp * 32ull; g < total; g += nwarps * 32ull) {
    const int j = job_of(s_base, n_jobs, g);  // warp-uniform
    if (j != cur) {
      if (cur >= 0) flush_counts(jobs[cur].t.cnt, sc);
      cur = j;
    }
    const JobView& jv = jobs[j];
    const int k = js[j].k;
    const Factor f = jv.factors[k];
    const unsigned long long i = g - s_base[j] + lane;
    forward_entry<1, RECORD>(jv.t, f, k, jv.eps, (unsigned int)(k + 1), jv.tape, i, i < js[j].n, sc);
  }
  if (cur >= 0) flush_counts(jobs[cur].t.cnt, sc);
  // Last block: each job's end-of-factor bookkeeping, then the next layout.
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&bh->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) {
    if (js[j].n == 0) continue;  // not stepped this launch
    const JobView& jv = jobs[j];
    Counters* c = jv.t.cnt;
    const int k = js[j].k;
    const unsigned long long nt = ld_cg(&c->n_tail);
    c->scanned += ld_cg(&c->n_scan);
    c->n_scan = nt;
    unsigned long long tn = 0;
    if (RECORD) {
      tn = ld_cg(&c->tape_n);
      jv.tape.off[k + 1] = tn;
    }
    const unsigned long long slots = jv.t.slot_mask + 1ull;
    const bool room = 2ull * nt <= jv.t.cap_n && 8ull * nt <= 3ull * slots && (!RECORD || tn + nt <= jv.tape.cap);
    js[j].k = k + 1;
    if (!room && k + 1 < jv.K) js[j].stop = k + 1;
    js[j].n_tail = nt;
    js[j].n_dead = ld_cg(&c->n_dead);
    js[j].tape_n = tn;
  }
  __syncthreads();
  layout(jobs, js, n_jobs, bh, 0);
  if (threadIdx.x == 0) bh->done = 0u;
}

// sigma[0, n) = 0 in every job before the lower-triangle pass.
__global__ void __launch_bounds__(kThreads) k_sigma_zero_batch(const JobView* jobs, JobState* js, int n_jobs,
                                                                BatchHeader* bh) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int j = job_of(s_base, n_jobs, g);
    jobs[j].t.sigma[g - s_base[j]] = 0.0;
  }
}

// sigma and the energy sums of every job; one warp per stored entry, each
// connected stored pair of a job visited once from its larger key (the
// single-problem energy kernel's lower-triangle pass).
__global__ void __launch_bounds__(kSigmaWarps * 32) k_sigma_batch(const JobView* jobs, JobState* js,
                                                                   int n_jobs, BatchHeader* bh) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  __shared__ LowerLists lists[kSigmaWarps];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  LowerLists& L = lists[w];
  const unsigned long long gw = (unsigned long long)blockIdx.x * kSigmaWarps + w;
  const unsigned long long nw = (unsigned long long)gridDim.x * kSigmaWarps;
  int cur = -1;
  double se = 0.0, sn = 0.0;
  unsigned long long probes = 0, hits = 0;
  auto flush = [&](int j) {
    const unsigned long long p = warp_sum_u64(probes), h = warp_sum_u64(hits);
    if (lane == 0) {
      if (se != 0.0) atomicAdd(&js[j].e_num, se);
      if (sn != 0.0) atomicAdd(&js[j].norm2, sn);
      if (p) atomicAdd(&jobs[j].t.cnt->sig_probes, p);
      if (h) atomicAdd(&jobs[j].t.cnt->sig_hits, h);
    }
    se = sn = 0.0;
    probes = hits = 0;
  };
  for (unsigned long long g = gw; g < total; g += nw) {
    const int j = job_of(s_base, n_jobs, g);
    if (j != cur) {
      if (cur >= 0) flush(cur);
      cur = j;
    }
    const JobView& jv = jobs[j];
    const unsigned long long e = g - s_base[j];
    const double cI = jv.t.amps[e];
    if (is_dead(cI)) continue;
    double d;
    double part = sigma_lower(jv.t, jv.in, L, jv.t.keys[e], cI, lane, d, probes, hits);
    d = warp_sum(d);
    part = warp_sum(part);
    if (lane == 0) {
      const double dc = d * cI;
      atomicAdd(&jv.t.sigma[e], dc + part);
      se += cI * (dc + 2.0 * part);
      sn += cI * cI;
    }
    __syncwarp();
  }
  if (cur >= 0) flush(cur);
}

// mu_K = (sigma - E psi)/<psi|psi> for every job (E from its energy sums).
__global__ void __launch_bounds__(kThreads) k_lambda_init_batch(const JobView* jobs, JobState* js, int n_jobs,
                                                                 BatchHeader* bh) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int j = job_of(s_base, n_jobs, g);
    const JobView& jv = jobs[j];
    const unsigned long long e = g - s_base[j];
    const double norm2 = js[j].norm2;
    const double E = js[j].e_num / norm2;
    const double a = jv.t.amps[e];
    jv.t.lam[e] = is_dead(a) ? 0.0 : (jv.t.sigma[e] - E * a) / norm2;
  }
}

// Tape re-insertion of every job's current reverse factor (layout mode 3).
__global__ void __launch_bounds__(kThreads) k_tape_reinsert_batch(const JobView* jobs, JobState* js, int n_jobs,
                                                                   BatchHeader* bh) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int j = job_of(s_base, n_jobs, g);
    const JobView& jv = jobs[j];
    const int k = js[j].k;
    const unsigned long long x = min(jv.tape.off[k], jv.tape.cap) + (g - s_base[j]);
    const TapeRec rec = tape_at(jv.tape, x);
    const unsigned long long key = rec.key;
    Lookup r = find1(jv.t, key, 0u);
    if (r.state == ALIVE) {
      raise_error(jv.t.cnt, ERR_CONSISTENCY);
    } else if (r.state == DEAD_OLD || r.state == DEAD_NOW) {
      jv.t.amps[r.idx] = rec.val;
      jv.t.lam[r.idx] = 0.0;
      jv.t.born[r.idx] = rec.born;
    } else {
      insert_new(jv.t, key, rec.val, rec.born, r.slot, true, true);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_reverse_batch(const JobView* jobs, JobState* js, int n_jobs,
                                                             BatchHeader* bh) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  int cur = -1;
  double acc = 0.0;
  unsigned int pairs = 0, kills = 0;  // kills: not used by the batched sweep
  auto flush = [&](int j) {
    const double a = warp_sum(acc);
    const unsigned long long p = warp_sum_u64(pairs);
    if (lane == 0) {
      if (a != 0.0) atomicAdd(&js[j].gacc, a);
      if (p) atomicAdd(&jobs[j].t.cnt->rev_pairs, p);
    }
    acc = 0.0;
    pairs = 0;
  };
  for (unsigned long long g = warp * 32ull; g < total; g += nwarps * 32ull) {
    const int j = job_of(s_base, n_jobs, g);
    if (j != cur) {
      if (cur >= 0) flush(cur);
      cur = j;
    }
    const JobView& jv = jobs[j];
    const int k = js[j].k;
    const Factor f = jv.factors[k];
    const unsigned long long i = g - s_base[j] + lane;
    reverse_entry<1>(jv.t, f, k, 0x80000000u | (unsigned int)k, i, i < js[j].n, acc, pairs, kills);
  }
  if (cur >= 0) flush(cur);
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&bh->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) {
    const int k = js[j].k;
    if (k < 0) continue;
    jobs[j].grad[k] = 2.0 * ld_cg(&js[j].gacc);
    js[j].gacc = 0.0;
    js[j].k = k - 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) bh->done = 0u;
}

}  // namespace

cudaError_t launch_batch_layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int mode,
                                cudaStream_t st) {
  k_batch_layout<<<1, 32, 0, st>>>(jobs, js, n_jobs, bh, mode);
  return cudaGetLastError();
}

cudaError_t launch_forward_batch(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int record,
                                 int grid, cudaStream_t st) {
  if (record)
    k_forward_batch<true><<<grid, kThreads, 0, st>>>(jobs, js, n_jobs, bh);
  else
    k_forward_batch<false><<<grid, kThreads, 0, st>>>(jobs, js, n_jobs, bh);
  return cudaGetLastError();
}

cudaError_t launch_sigma_batch(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int grid,
                               cudaStream_t st) {
  k_sigma_zero_batch<<<grid, kThreads, 0, st>>>(jobs, js, n_jobs, bh);
  k_sigma_batch<<<2 * grid, kSigmaWarps * 32, 0, st>>>(jobs, js, n_jobs, bh);
  return cudaGetLastError();
}

cudaError_t launch_lambda_init_batch(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int grid,
                                     cudaStream_t st) {
  k_lambda_init_batch<<<grid, kThreads, 0, st>>>(jobs, js, n_jobs, bh);
  return cudaGetLastError();
}

cudaError_t launch_reverse_batch(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int grid,
                                 cudaStream_t st) {
  k_batch_layout<<<1, 32, 0, st>>>(jobs, js, n_jobs, bh, 3);
  k_tape_reinsert_batch<<<grid, kThreads, 0, st>>>(jobs, js, n_jobs, bh);
  k_batch_layout<<<1, 32, 0, st>>>(jobs, js, n_jobs, bh, 2);
  k_reverse_batch<<<grid, kThreads, 0, st>>>(jobs, js, n_jobs, bh);
  return cudaGetLastError();
}

}  // namespace ucc
