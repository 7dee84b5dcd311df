// Batched (many-job) kernels of the energy: one launch evaluates every job's
// sigma and energy sums, one initialises every job's adjoint.  (The factor
// steps of a batch run in the persistent kernels of k_persist.cu.)
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

// Every job's stored entries laid end to end (unpadded: the energy kernel
// takes one warp per entry), by one thread.
__device__ void layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh) {
  if (threadIdx.x != 0) return;
  unsigned long long total = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const JobView& jv = jobs[j];
    const unsigned long long n = min(*((volatile const unsigned long long*)&jv.t.cnt->n_tail), jv.t.cap_n);
    js[j].base = total;
    js[j].n = n;
    total += n;
  }
  bh->total = total;
}

__global__ void k_batch_layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh) {
  layout(jobs, js, n_jobs, bh);
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
  __shared__ LowerLists<unsigned long long> lists[kSigmaWarps];
  load_bases(js, n_jobs, bh, s_base);
  const unsigned long long total = s_base[n_jobs];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  LowerLists<unsigned long long>& L = lists[w];
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

}  // namespace

cudaError_t launch_batch_layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, cudaStream_t st) {
  k_batch_layout<<<1, 32, 0, st>>>(jobs, js, n_jobs, bh);
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

}  // namespace ucc
