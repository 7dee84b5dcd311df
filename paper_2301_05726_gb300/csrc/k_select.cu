// Methods-section wavefunction truncation on the device: when more than N_MAX
// determinants are stored after a factor, keep the N_CUT of largest |c|
// (ties: smaller key first) and drop the rest.
//
// Exact selection by radix passes over 11-bit digits, most significant first:
// |c| as its IEEE-754 bit pattern (monotone in |c| for non-negative values)
// from the top bin down, then, only if several entries share the threshold
// value, the determinant key from the bottom bin up.  Each pass is one kernel:
// every block histograms its share of the live entries in shared memory, and
// the last block to finish picks the bin that holds the target rank.

#include "ucc_steps.cuh"

namespace ucc {

namespace {

constexpr int kThreads = 256;
constexpr int kDigit = 11;
constexpr int kBins = 1 << kDigit;            // 2048
constexpr int kPasses = (64 + kDigit - 1) / kDigit;  // 6 (covers 64 bits)
static_assert(kBins <= sizeof(SelectState::hist) / sizeof(unsigned long long), "histogram size");

__device__ __forceinline__ unsigned long long mag_bits(double a) {
  return (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ int digit_shift(int pass) { return 64 - kDigit * (pass + 1) < 0 ? 0 : 64 - kDigit * (pass + 1); }
__device__ __forceinline__ unsigned long long digit_of(unsigned long long v, int pass) {
  const int top = 64 - kDigit * pass;          // bits [shift, top) form this digit
  const int shift = digit_shift(pass);
  const int width = top - shift;
  return (v >> shift) & ((1ull << width) - 1ull);
}
__device__ __forceinline__ unsigned long long high_mask(int pass) {
  // bits above this pass's digit, i.e. the digits already fixed
  const int top = 64 - kDigit * pass;
  return top >= 64 ? 0ull : (~0ull << top);
}

// The last block turns the global histogram into the next digit of the
// threshold: phase 0 walks bins from the top (largest |c| first), phase 1 from
// the bottom (smallest key first).
__device__ void pick_bin(SelectState* sel, int phase, int pass, int nbins) {
  __shared__ unsigned long long s_scan[kThreads];
  const int per = (nbins + kThreads - 1) / kThreads;
  unsigned long long local = 0;
  for (int j = 0; j < per; ++j) {
    const int o = threadIdx.x * per + j;  // visiting order
    if (o >= nbins) break;
    const int b = phase == 0 ? nbins - 1 - o : o;
    local += ld_cg(&sel->hist[b]);
  }
  s_scan[threadIdx.x] = local;
  __syncthreads();
  // inclusive scan (Hillis-Steele) over the 256 partial sums
  for (int off = 1; off < kThreads; off <<= 1) {
    unsigned long long v = threadIdx.x >= off ? s_scan[threadIdx.x - off] : 0ull;
    __syncthreads();
    s_scan[threadIdx.x] += v;
    __syncthreads();
  }
  const unsigned long long incl = s_scan[threadIdx.x];
  const unsigned long long before = incl - local;
  const unsigned long long target = phase == 0 ? sel->target : sel->key_target;
  if (before < target && target <= incl) {
    unsigned long long cum = before;
    for (int j = 0; j < per; ++j) {
      const int o = threadIdx.x * per + j;
      if (o >= nbins) break;
      const int b = phase == 0 ? nbins - 1 - o : o;
      const unsigned long long cnt = ld_cg(&sel->hist[b]);
      if (cum + cnt >= target) {
        const unsigned long long rest = target - cum;
        const int shift = digit_shift(pass);
        if (phase == 0) {
          sel->prefix |= (unsigned long long)b << shift;
          sel->target = rest;
          if (pass == kPasses - 1) {
            sel->count_eq = cnt;
            sel->need_keys = cnt > rest ? 1 : 0;
            sel->key_target = rest;
          }
        } else {
          sel->key_prefix |= (unsigned long long)b << shift;
          sel->key_target = rest;
        }
        break;
      }
      cum += cnt;
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) sel->hist[b] = 0;
}

// One radix pass: histogram of the pass's digit of |c| (phase 0) or of the
// key among |c| == threshold entries (phase 1), restricted to entries whose
// already-fixed digits match, then the pick in the last block.
__global__ void __launch_bounds__(kThreads) k_select_pass(Table t, SelectState* sel, int phase, int pass) {
  __shared__ unsigned int h[kBins];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (phase == 1 && !*((volatile int*)&sel->need_keys)) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;  // uniform over the grid: no tie to break
  const int top = 64 - kDigit * pass;
  const int nbins = 1 << (top - digit_shift(pass));
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long hm = high_mask(pass);
  const unsigned long long T = sel->prefix;
  const unsigned long long kp = sel->key_prefix;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag_bits(a);
    if (phase == 0) {
      if ((u & hm) != (T & hm)) continue;
      atomicAdd(&h[digit_of(u, pass)], 1u);
    } else {
      if (u != T) continue;
      const unsigned long long key = t.keys[i];
      if ((key & hm) != (kp & hm)) continue;
      atomicAdd(&h[digit_of(key, pass)], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (h[b]) atomicAdd(&sel->hist[b], (unsigned long long)h[b]);
  if (last_block_arrive(t.cnt)) {
    pick_bin(sel, phase, pass, nbins);
    if (threadIdx.x == 0) t.cnt->done = 0u;
  }
}

// Drop every live entry outside the kept set; record drops on the tape.
template <bool RECORD>
__global__ void __launch_bounds__(kThreads) k_select_mark(Table t, SelectState* sel, unsigned int stamp, Tape tape,
                                                          int k) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long T = sel->prefix;
  const bool keys = sel->need_keys != 0;
  const unsigned long long Kt = sel->key_prefix;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long dropped = 0;
  double dS = 0.0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag_bits(a);
    bool keep = u > T;
    if (u == T) keep = !keys || t.keys[i] <= Kt;
    if (keep) continue;
    if (t.entropy) dS -= entropy_term(a);
    if (RECORD) {
      const unsigned long long ti = aggregated_add(&t.cnt->tape_n);
      if (ti < tape.cap) {
        TapeRec& rec = tape_at(tape, ti);
        rec.key = t.keys[i];
        rec.val = a;
        rec.born = t.born[i];
      } else {
        raise_error(t.cnt, ERR_TAPE_FULL);
      }
    }
    t.amps[i] = dead_value(stamp);
    ++dropped;
  }
  __shared__ unsigned long long s_d;
  if (threadIdx.x == 0) s_d = 0;
  __syncthreads();
  if (dropped) atomicAdd(&s_d, dropped);
  __syncthreads();
  if (threadIdx.x == 0 && s_d) {
    atomicAdd(&t.cnt->n_dead, s_d);
    atomicAdd(&sel->cut_total, s_d);
  }
  if (t.entropy) {
    const double b = block_sum(dS);
    if (threadIdx.x == 0) t.partials[blockIdx.x] = b;
  }
  const bool last = last_block_arrive(t.cnt);
  if (last && t.entropy) {
    double s = 0.0;
    for (unsigned int x = threadIdx.x; x < gridDim.x; x += blockDim.x) s += ld_cg(&t.partials[x]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
      t.cnt->entropy += s;
      t.entropy[k] = t.cnt->entropy;
    }
  }
  if (last && threadIdx.x == 0) {
    t.cnt->done = 0u;
    if (RECORD) tape.off[k + 1] = ld_cg(&t.cnt->tape_n);
  }
}

__global__ void k_select_init(SelectState* sel, unsigned long long n_cut) {
  if (threadIdx.x == 0) {
    sel->prefix = 0;
    sel->target = n_cut;
    sel->key_prefix = 0;
    sel->key_target = 0;
    sel->need_keys = 0;
    sel->count_eq = 0;
  }
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) sel->hist[b] = 0;
}

}  // namespace

cudaError_t launch_select_cut(const Table& t, SelectState* sel, unsigned long long n_cut, unsigned int stamp,
                              int record, const Tape& tape, int k, int grid, cudaStream_t st, long long* launches) {
  k_select_init<<<1, kThreads, 0, st>>>(sel, n_cut);
  *launches += 1;
  for (int phase = 0; phase < 2; ++phase)
    for (int pass = 0; pass < kPasses; ++pass) {
      k_select_pass<<<grid, kThreads, 0, st>>>(t, sel, phase, pass);
      *launches += 1;
    }
  if (record)
    k_select_mark<true><<<grid, kThreads, 0, st>>>(t, sel, stamp, tape, k);
  else
    k_select_mark<false><<<grid, kThreads, 0, st>>>(t, sel, stamp, tape, k);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace ucc
