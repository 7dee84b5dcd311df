// Persistent batched passes: many independent jobs (molecules or theta
// vectors of uneven size) advanced by ONE cooperative launch per pass.
//
// Every job's table is sized up front (its whole determinant sector, or four
// times its cut's N_MAX), so no job ever needs the host to grow it.  The
// launch loops over steps; each step is three phases separated by grid-wide
// barriers:
//
//   A  the factor step of every job that still has factors, over the jobs'
//      stored entries laid end to end (each job padded to a warp's visit of
//      `tiles` 32-entry tiles, so a visit never straddles two jobs);
//   C  one block per stepped job: end-of-step bookkeeping, then, if the job
//      holds more than N_MAX determinants, the Methods-section cut (exact
//      selection of the N_CUT of largest |c|, ties to the smaller key) fused
//      with a compaction into the job's spare arrays, which are hashed and
//      swapped in on the device; or a plain compaction when dropped entries
//      pile up;
//   L  one block lays out the next step.
//
// The reverse pass runs the same way: the tape re-insertion of each job's
// current factor, the reverse step, the per-job gradient entry and
// compactions (keeping the adjoint).
//
// The grid barriers wait with a bound (BatchHeader::wait_ns on %globaltimer):
// a block that waits longer sets the header's error word and every block
// leaves at its next barrier, so a barrier that can never complete ends the
// launch with an error status instead of a hang.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

constexpr int kPThreads = 256;
constexpr int kPWarps = kPThreads / 32;
constexpr int kCand = 512;  // candidates of a job's cut resolved by pairwise rank

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of
// the block) when the launch must end: a wait ran past wait_ns here or in
// another block, or a job ran out of room.
__device__ bool grid_sync(BatchHeader* bh) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &bh->bar_gen;
    const unsigned int g0 = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bh->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      bh->bar_count = 0u;
      __threadfence();
      atomicAdd(&bh->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      const unsigned long long limit = bh->wait_ns;
      while (*gen == g0) {
        if (*((volatile int*)&bh->error) != 0) break;
        if (global_ns() - t0 > limit) {
          atomicOr(&bh->error, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = *((volatile int*)&bh->error) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Loads of values other blocks wrote earlier in this launch (after a barrier).
template <class T>
__device__ __forceinline__ T ldv(const T* p) {
  return *((const volatile T*)p);
}

__device__ __forceinline__ int job_at(const unsigned long long* base, int n_jobs, unsigned long long g) {
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

// The job's current arrays (the device copy of its view, which phase C may
// have swapped).
__device__ __forceinline__ Table job_table(const JobView* jobs, int j) {
  Table t = jobs[j].t;
  const Table* src = &jobs[j].t;
  t.keys = ldv(&src->keys);
  t.amps = ldv(&src->amps);
  t.born = ldv(&src->born);
  t.lam = ldv(&src->lam);
  t.slots = ldv(&src->slots);
  t.filt = ldv(&src->filt);
  return t;
}

// Block-wide exclusive prefix of a per-thread count; returns the block total
// in *total (every thread).
__device__ __forceinline__ unsigned int block_prefix(unsigned int v, unsigned int* total) {
  __shared__ unsigned int s_w[kPWarps];
  __shared__ unsigned int s_tot;
  const unsigned int lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  unsigned int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  if (lane == 31) s_w[w] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int run = 0;
    for (int x = 0; x < kPWarps; ++x) {
      const unsigned int t = s_w[x];
      s_w[x] = run;
      run += t;
    }
    s_tot = run;
  }
  __syncthreads();
  const unsigned int r = s_w[w] + incl - v;
  *total = s_tot;
  __syncthreads();
  return r;
}

// Phase L: the step layout of every job (block 0).  mode 0: forward (n_scan
// of jobs with factors left and not stopped), 1: reverse (records of the
// current factor, and n_tail plus those records).  Pads each job's entry
// range to `pad` entries.
__device__ void layout(const JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int mode, int pad) {
  __shared__ unsigned long long s_run, s_rrun;
  __shared__ int s_active;
  if (threadIdx.x == 0) {
    s_run = 0;
    s_rrun = 0;
    s_active = 0;
  }
  __syncthreads();
  for (int j0 = 0; j0 < n_jobs; j0 += kPThreads) {
    const int j = j0 + (int)threadIdx.x;
    unsigned long long n = 0, w = 0, rn = 0;
    if (j < n_jobs) {
      const JobView& jv = jobs[j];
      const Counters* c = jv.t.cnt;
      const int k = ldv(&js[j].k);
      if (mode == 0) {
        if (k < jv.K && ldv(&js[j].stop) < 0) n = min(ldv(&c->n_scan), jv.t.cap_n);
      } else if (k >= 0) {
        const unsigned long long hi = min(ldv(&jv.tape.off[k + 1]), jv.tape.cap);
        const unsigned long long lo = min(ldv(&jv.tape.off[k]), hi);
        rn = hi - lo;
        n = min(ldv(&c->n_tail) + rn, jv.t.cap_n);
      }
      w = (n + (unsigned long long)pad - 1ull) / (unsigned long long)pad * (unsigned long long)pad;
    }
    // records are padded to whole warps too: a warp's lanes then re-insert
    // records of one job only (the warp-aggregated tail reservation of an
    // insertion must not mix two jobs' counters)
    const unsigned long long rw = (rn + 31ull) & ~31ull;
    // block prefix over (w, rn): 64-bit sums via shared running totals, 32 at a time per warp
    for (int x = 0; x < kPThreads; x += 32) {
      __syncthreads();
      if ((int)threadIdx.x >= x && (int)threadIdx.x < x + 32) {
        unsigned long long a = w, b = rw;
        const unsigned int lane = threadIdx.x & 31u;
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long ya = __shfl_up_sync(0xFFFFFFFFu, a, o);
          const unsigned long long yb = __shfl_up_sync(0xFFFFFFFFu, b, o);
          if ((int)lane >= o) {
            a += ya;
            b += yb;
          }
        }
        if (j < n_jobs) {
          js[j].base = s_run + a - w;
          js[j].n = n;
          js[j].rbase = s_rrun + b - rw;
          js[j].rn = rn;
        }
        const unsigned long long ta = __shfl_sync(0xFFFFFFFFu, a, 31);
        const unsigned long long tb = __shfl_sync(0xFFFFFFFFu, b, 31);
        const unsigned int act = __ballot_sync(0xFFFFFFFFu, n > 0 || (mode == 1 && j < n_jobs && ldv(&js[j].k) >= 0));
        if (lane == 0) {
          s_run += ta;
          s_rrun += tb;
          s_active += __popc(act);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bh->total = s_run;
    bh->rtotal = s_rrun;
    bh->active = s_active;
  }
}

__device__ __forceinline__ void flush_forward(Counters* c, StepCounts& sc) {
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

// ---------------------------------------------------------------------------
// Phase C helpers: one block rebuilds one job's table.
// ---------------------------------------------------------------------------

// Threshold of the job's cut: the N_CUT-th live entry by (|c| descending, key
// ascending) as (T, Kt); the entries kept are those with |c| > T, or |c| == T
// and key <= Kt.  Radix passes of 11 bits over |c| (then over the key among
// entries of equal |c|) narrow the current bin until it holds at most kCand
// entries; those are gathered and ranked pairwise.
__device__ void block_threshold(const Table& t, unsigned long long nt, unsigned long long live,
                                unsigned long long n_cut, unsigned long long* T_out, unsigned long long* Kt_out) {
  constexpr int kDigit = 11;
  __shared__ unsigned int h[1 << kDigit];
  __shared__ unsigned long long s_cm[kCand], s_ck[kCand];
  __shared__ unsigned long long s_pu, s_mu, s_pk, s_mk, s_target, s_bincnt;  // fixed bits and their masks
  __shared__ unsigned int s_nc;
  if (threadIdx.x == 0) {
    s_pu = s_mu = s_pk = s_mk = 0ull;
    s_target = n_cut;
    s_bincnt = live;
  }
  __syncthreads();
  auto mag = [](double a) { return (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull; };
  // Passes 0-5 fix |c| bits [63, 53], [52, 42], ..., [8, 0]; passes 6-11 the key's the same way.
  for (int pass = 0; pass < 12; ++pass) {
    const bool on_key = pass >= 6;
    if (s_bincnt <= (unsigned long long)kCand) break;  // block-uniform
    const int p = on_key ? pass - 6 : pass;
    const int top = 64 - kDigit * p;
    const int shift = top - kDigit > 0 ? top - kDigit : 0;
    const int nb = 1 << (top - shift);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long pu = s_pu, mu = s_mu, pk = s_pk, mk = s_mk;
    for (unsigned long long i = threadIdx.x; i < nt; i += blockDim.x) {
      const double a = t.amps[i];
      if (is_dead(a)) continue;
      const unsigned long long u = mag(a);
      if ((u & mu) != pu) continue;
      if (!on_key) {
        atomicAdd(&h[(u >> shift) & (unsigned long long)(nb - 1)], 1u);
      } else {
        const unsigned long long key = t.keys[i];
        if ((key & mk) == pk) atomicAdd(&h[(key >> shift) & (unsigned long long)(nb - 1)], 1u);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // |c| bins from the top (largest first), key bins from the bottom (smallest first)
      unsigned long long cum = 0;
      for (int o = 0; o < nb; ++o) {
        const int b = on_key ? o : nb - 1 - o;
        const unsigned long long cnt = h[b];
        if (cum + cnt >= s_target) {
          const unsigned long long digit_mask = (unsigned long long)(nb - 1) << shift;
          if (on_key) {
            s_pk |= (unsigned long long)b << shift;
            s_mk |= digit_mask;
          } else {
            s_pu |= (unsigned long long)b << shift;
            s_mu |= digit_mask;
          }
          s_target -= cum;
          s_bincnt = cnt;
          break;
        }
        cum += cnt;
      }
    }
    __syncthreads();
  }
  // Gather the current bin (at most kCand entries; the 64 key bits always
  // narrow it to one) and rank it pairwise.
  if (threadIdx.x == 0) s_nc = 0;
  __syncthreads();
  const unsigned long long pu = s_pu, mu = s_mu, pk = s_pk, mk = s_mk;
  for (unsigned long long i = threadIdx.x; i < nt; i += blockDim.x) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag(a);
    if ((u & mu) != pu) continue;
    const unsigned long long key = t.keys[i];
    if ((key & mk) != pk) continue;
    const unsigned int q = atomicAdd(&s_nc, 1u);
    if (q < (unsigned int)kCand) {
      s_cm[q] = u;
      s_ck[q] = key;
    }
  }
  __syncthreads();
  const unsigned int nc = min(s_nc, (unsigned int)kCand);
  for (unsigned int x = threadIdx.x; x < nc; x += blockDim.x) {
    unsigned long long before = 0;
    for (unsigned int y = 0; y < nc; ++y)
      before += (s_cm[y] > s_cm[x]) || (s_cm[y] == s_cm[x] && s_ck[y] < s_ck[x]);
    if (before + 1ull == s_target) {
      *T_out = s_cm[x];
      *Kt_out = s_ck[x];
    }
  }
  __syncthreads();
}

// Compact job table t (current arrays) into its spare arrays: live entries
// that keep(u, key) accepts go to the spare set (with born, and lam when
// with_lam); live entries it rejects are recorded on the tape (record) as
// factor k's.  Then the spare slots are cleared and hashed and the two sets
// swapped in the device view.  Returns the number of entries kept and the
// number dropped.
template <class Keep>
__device__ void block_rebuild(JobView* jobs, int j, const Table& t, unsigned long long nt, Keep keep, bool record,
                              bool with_lam, int k, unsigned long long* kept_out, unsigned long long* dropped_out) {
  JobView& jv = jobs[j];
  const SpareArrays sp = {ldv(&jv.sp.keys), ldv(&jv.sp.amps), ldv(&jv.sp.born),
                          ldv(&jv.sp.lam),  ldv(&jv.sp.slots), ldv(&jv.sp.filt)};
  __shared__ unsigned long long s_kept, s_drop, s_tape;
  if (threadIdx.x == 0) {
    s_kept = 0;
    s_drop = 0;
    s_tape = record ? ldv(&t.cnt->tape_n) : 0ull;
  }
  __syncthreads();
  // Four entries per thread and round (one prefix over the block per round):
  // entry base + u * blockDim.x + threadIdx.x for u < 4.
  constexpr int kPer = 4;
  for (unsigned long long base = 0; base < nt; base += kPer * (unsigned long long)blockDim.x) {
    unsigned int kp = 0, dp = 0;
    double a[kPer];
    unsigned long long key[kPer];
    int st[kPer];  // 0 none, 1 keep, 2 drop
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const unsigned long long i = base + (unsigned long long)u * blockDim.x + threadIdx.x;
      st[u] = 0;
      a[u] = 0.0;
      key[u] = 0ull;
      if (i < nt) {
        a[u] = t.amps[i];
        if (!is_dead(a[u])) {
          key[u] = t.keys[i];
          st[u] = keep(a[u], key[u]) ? 1 : 2;
          kp += st[u] == 1;
          dp += st[u] == 2;
        }
      }
    }
    unsigned int tk, td;
    unsigned int pk = block_prefix(kp, &tk);
    unsigned int pd = block_prefix(dp, &td);
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      if (st[u] == 0) continue;
      const unsigned long long i = base + (unsigned long long)u * blockDim.x + threadIdx.x;
      if (st[u] == 1) {
        const unsigned long long at = s_kept + pk++;
        if (at < t.cap_n) {
          sp.keys[at] = key[u];
          sp.amps[at] = a[u];
          sp.born[at] = t.born[i];
          if (with_lam) sp.lam[at] = t.lam[i];
        } else {
          raise_error(t.cnt, ERR_CAPACITY);
        }
      } else if (record) {
        const unsigned long long at = s_tape + pd++;
        if (at < jv.tape.cap) {
          TapeRec& rec = tape_at(jv.tape, at);
          rec.key = key[u];
          rec.val = a[u];
          rec.born = t.born[i];
        } else {
          raise_error(t.cnt, ERR_TAPE_FULL);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_kept += tk;
      s_drop += td;
      if (record) s_tape += td;
    }
    __syncthreads();
  }
  // clear the spare slots and filter, then hash the kept entries into them
  const unsigned long long ns = t.slot_mask + 1ull;
  uint4* const slot16 = reinterpret_cast<uint4*>(sp.slots);  // one 16-byte store per slot
  for (unsigned long long x = threadIdx.x; x < ns; x += blockDim.x) slot16[x] = make_uint4(0u, 0u, 0u, 0u);
  uint4* const filt16 = reinterpret_cast<uint4*>(sp.filt);  // four filter words per store (ns / 4 is a multiple of 4)
  for (unsigned long long x = threadIdx.x; x < ns / 16; x += blockDim.x) filt16[x] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  Table tt = t;
  tt.keys = sp.keys;
  tt.amps = sp.amps;
  tt.born = sp.born;
  tt.lam = sp.lam;
  tt.slots = sp.slots;
  tt.filt = sp.filt;
  const unsigned long long nk = min(s_kept, t.cap_n);
  for (unsigned long long i = threadIdx.x; i < nk; i += blockDim.x) {
    const unsigned long long s = claim_slot(tt, sp.keys[i], home_slot(tt, sp.keys[i]), SITE_REBUILD_DUP);
    if (s != ~0ull) tt.slots[s].idx = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // swap the two array sets in the device view
    const Table cur = job_table(jobs, j);
    jv.t.keys = sp.keys;
    jv.t.amps = sp.amps;
    jv.t.born = sp.born;
    jv.t.lam = sp.lam;
    jv.t.slots = sp.slots;
    jv.t.filt = sp.filt;
    jv.sp.keys = cur.keys;
    jv.sp.amps = cur.amps;
    jv.sp.born = cur.born;
    jv.sp.lam = cur.lam;
    jv.sp.slots = cur.slots;
    jv.sp.filt = cur.filt;
    Counters* c = t.cnt;
    c->n_tail = nk;
    c->n_scan = nk;
    c->n_dead = 0;
    if (record) c->tape_n = s_tape;
    *kept_out = nk;
    *dropped_out = s_drop;
    __threadfence();
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Forward pass
// ---------------------------------------------------------------------------
template <int G, bool RECORD>
__global__ void __launch_bounds__(kPThreads) k_persist_forward(JobView* jobs, JobState* js, int n_jobs,
                                                               BatchHeader* bh, int tiles, int max_steps) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  if ((int)blockIdx.x == bh->skip_block) return;  // test hook: this block never reaches a barrier
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long span = 32ull * (unsigned long long)tiles;
  if (blockIdx.x == 0) layout(jobs, js, n_jobs, bh, 0, (int)span);
  if (!grid_sync(bh)) return;
  for (int step = 0; step < max_steps; ++step) {
    if (ldv(&bh->active) == 0) return;
    for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) s_base[j] = ldv(&js[j].base);
    if (threadIdx.x == 0) s_base[n_jobs] = ldv(&bh->total);
    __syncthreads();
    const unsigned long long total = s_base[n_jobs];
    // Phase A: every job's factor step.
    {
      StepCounts sc;
      int cur = -1;
      for (unsigned long long g = warp * span; g < total; g += nwarps * span) {
        const int j = job_at(s_base, n_jobs, g);  // warp-uniform
        if (j != cur) {
          if (cur >= 0) flush_forward(jobs[cur].t.cnt, sc);
          cur = j;
        }
        const JobView& jv = jobs[j];
        const Table t = job_table(jobs, j);
        const int k = ldv(&js[j].k);
        const Factor f = jv.factors[k];
        const unsigned long long n = ldv(&js[j].n);
        for (int u = 0; u < tiles; ++u) {
          const unsigned long long i = g - s_base[j] + 32ull * u + lane;
          forward_entry<G, RECORD>(t, f, k, jv.eps, (unsigned int)(k + 1), jv.tape, i, i < n, sc);
        }
      }
      if (cur >= 0) flush_forward(jobs[cur].t.cnt, sc);
    }
    if (!grid_sync(bh)) return;
    // Phase C: one block per stepped job.
    for (int j = blockIdx.x; j < n_jobs; j += gridDim.x) {
      if (ldv(&js[j].n) == 0) continue;  // block-uniform
      JobView& jv = jobs[j];
      const Table t = job_table(jobs, j);
      Counters* c = t.cnt;
      const int k = ldv(&js[j].k);
      __shared__ unsigned long long s_nt, s_dead, s_T, s_Kt, s_kept, s_drop;
      if (threadIdx.x == 0) {
        const unsigned long long nt = ldv(&c->n_tail);
        c->scanned += ldv(&c->n_scan);
        c->n_scan = nt;
        if (RECORD) jv.tape.off[k + 1] = ldv(&c->tape_n);
        s_nt = nt;
        s_dead = ldv(&c->n_dead);
        s_T = 0;
        s_Kt = 0;
      }
      __syncthreads();
      const unsigned long long nt = s_nt, live = nt - s_dead;
      const unsigned long long n_max = (unsigned long long)jv.n_max;
      if (n_max > 0 && live > n_max) {
        block_threshold(t, nt, live, (unsigned long long)jv.n_cut, &s_T, &s_Kt);
        __syncthreads();
        const unsigned long long T = s_T, Kt = s_Kt;
        block_rebuild(
            jobs, j, t, nt,
            [&](double a, unsigned long long key) {
              const unsigned long long u = (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
              return u > T || (u == T && key <= Kt);
            },
            RECORD, false, k, &s_kept, &s_drop);
        if (threadIdx.x == 0) {
          js[j].cut += (long long)s_drop;
          if (RECORD) jv.tape.off[k + 1] = ldv(&c->tape_n);
        }
      } else if (s_dead > 0 &&
                 (4ull * s_dead > nt || 2ull * nt > t.cap_n || 8ull * nt > 3ull * (t.slot_mask + 1ull))) {
        // compact when a quarter of the stored entries are dropped ones, or
        // when the next step would not have room
        block_rebuild(
            jobs, j, t, nt, [](double, unsigned long long) { return true; }, false, false, k, &s_kept, &s_drop);
      }
      if (threadIdx.x == 0) {
        const unsigned long long n2 = ldv(&c->n_tail);
        const unsigned long long slots = t.slot_mask + 1ull;
        if (!(2ull * n2 <= t.cap_n && 8ull * n2 <= 3ull * slots)) {
          atomicOr(&bh->error, 2);  // the table was sized too small
        }
        js[j].k = k + 1;
        // tape room for the next factor's drops and a cut after it
        if (RECORD && k + 1 < jv.K && ldv(&c->tape_n) + 2ull * n2 + 64ull > jv.tape.cap) js[j].stop = k + 1;
        js[j].n_tail = n2;
        js[j].n_dead = ldv(&c->n_dead);
        js[j].tape_n = ldv(&c->tape_n);
      }
      __syncthreads();
    }
    if (!grid_sync(bh)) return;
    if (blockIdx.x == 0) {
      layout(jobs, js, n_jobs, bh, 0, (int)span);
      if (threadIdx.x == 0) bh->steps += 1;
    }
    if (!grid_sync(bh)) return;
  }
}

// ---------------------------------------------------------------------------
// Reverse pass
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kPThreads) k_persist_reverse(JobView* jobs, JobState* js, int n_jobs,
                                                               BatchHeader* bh, int tiles) {
  __shared__ unsigned long long s_base[kMaxBatchJobs + 1];
  if ((int)blockIdx.x == bh->skip_block) return;  // test hook
  const unsigned int lane = threadIdx.x & 31u;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long span = 32ull * (unsigned long long)tiles;
  if (blockIdx.x == 0) layout(jobs, js, n_jobs, bh, 1, (int)span);
  if (!grid_sync(bh)) return;
  for (;;) {
    if (ldv(&bh->active) == 0) return;
    // Phase R1: re-insert each job's records of its current factor (warp-
    // strided over the jobs' record ranges, each padded to whole warps).
    for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) s_base[j] = ldv(&js[j].rbase);
    if (threadIdx.x == 0) s_base[n_jobs] = ldv(&bh->rtotal);
    __syncthreads();
    {
      const unsigned long long rtotal = s_base[n_jobs];
      for (unsigned long long g = warp * 32ull + lane; g < rtotal; g += nwarps * 32ull) {
        const int j = job_at(s_base, n_jobs, g);  // warp-uniform
        const unsigned long long roff = g - s_base[j];
        if (roff >= ldv(&js[j].rn)) continue;
        const JobView& jv = jobs[j];
        const Table t = job_table(jobs, j);
        const int k = ldv(&js[j].k);
        const unsigned long long x = min(ldv(&jv.tape.off[k]), jv.tape.cap) + roff;
        const TapeRec rec = tape_at(jv.tape, x);
        Lookup r = find1(t, rec.key, 0u);
        if (r.state == ALIVE) {
          raise_consistency(t.cnt, SITE_BATCH_ALIVE);
        } else if (r.state == DEAD_OLD || r.state == DEAD_NOW) {
          t.amps[r.idx] = rec.val;
          t.lam[r.idx] = 0.0;
          t.born[r.idx] = rec.born;
          atomicAdd(&t.cnt->n_dead, 0ull - 1ull);
        } else {
          insert_new(t, rec.key, rec.val, rec.born, r.slot, true, true, SITE_REINSERT_DUP);
        }
      }
    }
    if (!grid_sync(bh)) return;
    // Phase R2: the reverse step of every job.
    for (int j = threadIdx.x; j < n_jobs; j += blockDim.x) s_base[j] = ldv(&js[j].base);
    if (threadIdx.x == 0) s_base[n_jobs] = ldv(&bh->total);
    __syncthreads();
    {
      const unsigned long long total = s_base[n_jobs];
      int cur = -1;
      double acc = 0.0;
      unsigned int pairs = 0, kills = 0;
      auto flush = [&](int j) {
        const double a = warp_sum(acc);
        const unsigned long long p = warp_sum_u64(pairs), kl = warp_sum_u64(kills);
        if (lane == 0) {
          if (a != 0.0) atomicAdd(&js[j].gacc, a);
          if (p) atomicAdd(&jobs[j].t.cnt->rev_pairs, p);
          if (kl) atomicAdd(&jobs[j].t.cnt->n_dead, kl);
        }
        acc = 0.0;
        pairs = 0;
        kills = 0;
      };
      for (unsigned long long g = warp * span; g < total; g += nwarps * span) {
        const int j = job_at(s_base, n_jobs, g);
        if (j != cur) {
          if (cur >= 0) flush(cur);
          cur = j;
        }
        const JobView& jv = jobs[j];
        const Table t = job_table(jobs, j);
        const int k = ldv(&js[j].k);
        const Factor f = jv.factors[k];
        const unsigned long long n = min(ldv(&t.cnt->n_tail), t.cap_n);
        for (int u = 0; u < tiles; ++u) {
          const unsigned long long i = g - s_base[j] + 32ull * u + lane;
          reverse_entry<G>(t, f, k, 0x80000000u | (unsigned int)k, i, i < n, acc, pairs, kills);
        }
      }
      if (cur >= 0) flush(cur);
    }
    if (!grid_sync(bh)) return;
    // Phase R3: gradient entry, next factor, compaction when needed.
    for (int j = blockIdx.x; j < n_jobs; j += gridDim.x) {
      const int k = ldv(&js[j].k);
      if (k < 0) continue;  // block-uniform
      JobView& jv = jobs[j];
      const Table t = job_table(jobs, j);
      Counters* c = t.cnt;
      __shared__ unsigned long long s_nt, s_dead, s_next, s_kept, s_drop;
      __shared__ int s_compact;
      if (threadIdx.x == 0) {
        jv.grad[k] = 2.0 * ldv(&js[j].gacc);
        js[j].gacc = 0.0;
        js[j].k = k - 1;
        c->rev_scanned += ldv(&c->n_tail);
        s_nt = ldv(&c->n_tail);
        s_dead = ldv(&c->n_dead);
        unsigned long long rec = 0;
        if (k - 1 >= 0) {
          const unsigned long long hi = min(ldv(&jv.tape.off[k]), jv.tape.cap);
          rec = hi - min(ldv(&jv.tape.off[k - 1]), hi);
        }
        s_next = rec;
        const unsigned long long need = s_nt + rec;
        const unsigned long long slots = t.slot_mask + 1ull;
        const bool room = need <= t.cap_n && 4ull * need <= 3ull * slots;
        s_compact = k - 1 >= 0 && (!room || (s_dead > 1024 && 3ull * s_dead > s_nt));
      }
      __syncthreads();
      if (s_compact) {
        block_rebuild(
            jobs, j, t, s_nt, [](double, unsigned long long) { return true; }, false, true, k, &s_kept, &s_drop);
        if (threadIdx.x == 0) {
          const unsigned long long n2 = ldv(&c->n_tail) + s_next;
          const unsigned long long slots = t.slot_mask + 1ull;
          if (!(n2 <= t.cap_n && 4ull * n2 <= 3ull * slots)) atomicOr(&bh->error, 2);
        }
      }
      __syncthreads();
    }
    if (!grid_sync(bh)) return;
    if (blockIdx.x == 0) {
      layout(jobs, js, n_jobs, bh, 1, (int)span);
      if (threadIdx.x == 0) bh->steps += 1;
    }
    if (!grid_sync(bh)) return;
  }
}

template <auto Kernel>
int resident_grid() {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, Kernel, kPThreads, 0) != cudaSuccess || occ < 1)
    return 0;
  return sms * occ;
}

template <auto Kernel, class... Args>
cudaError_t launch_coop(cudaStream_t st, Args... args) {
  const int grid = resident_grid<Kernel>();
  if (grid <= 0) return cudaErrorLaunchFailure;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, Kernel, args...);
}

}  // namespace

cudaError_t launch_persist_forward(JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int record,
                                   int probe_width, int tiles, int max_steps, cudaStream_t st) {
  if (n_jobs < 1 || n_jobs > kMaxBatchJobs) return cudaErrorInvalidValue;
  if (tiles != 1 && tiles != 2 && tiles != 4 && tiles != 8) return cudaErrorInvalidValue;
  if (record) {
    switch (probe_width) {
      case 2: return launch_coop<k_persist_forward<2, true>>(st, jobs, js, n_jobs, bh, tiles, max_steps);
      case 4: return launch_coop<k_persist_forward<4, true>>(st, jobs, js, n_jobs, bh, tiles, max_steps);
      default: return launch_coop<k_persist_forward<1, true>>(st, jobs, js, n_jobs, bh, tiles, max_steps);
    }
  }
  switch (probe_width) {
    case 2: return launch_coop<k_persist_forward<2, false>>(st, jobs, js, n_jobs, bh, tiles, max_steps);
    case 4: return launch_coop<k_persist_forward<4, false>>(st, jobs, js, n_jobs, bh, tiles, max_steps);
    default: return launch_coop<k_persist_forward<1, false>>(st, jobs, js, n_jobs, bh, tiles, max_steps);
  }
}

cudaError_t launch_persist_reverse(JobView* jobs, JobState* js, int n_jobs, BatchHeader* bh, int probe_width,
                                   int tiles, cudaStream_t st) {
  if (n_jobs < 1 || n_jobs > kMaxBatchJobs) return cudaErrorInvalidValue;
  if (tiles != 1 && tiles != 2 && tiles != 4 && tiles != 8) return cudaErrorInvalidValue;
  switch (probe_width) {
    case 2: return launch_coop<k_persist_reverse<2>>(st, jobs, js, n_jobs, bh, tiles);
    case 4: return launch_coop<k_persist_reverse<4>>(st, jobs, js, n_jobs, bh, tiles);
    default: return launch_coop<k_persist_reverse<1>>(st, jobs, js, n_jobs, bh, tiles);
  }
}

int persist_grid(int record, int probe_width, int reverse) {
  if (reverse) return resident_grid<k_persist_reverse<1>>();
  return record ? resident_grid<k_persist_forward<1, true>>() : resident_grid<k_persist_forward<1, false>>();
}

}  // namespace ucc
