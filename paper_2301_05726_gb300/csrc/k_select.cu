// Methods-section wavefunction truncation on the device: when more than N_MAX
// determinants are stored after a factor, keep the N_CUT of largest |c|
// (ties: smaller key first) and drop the rest.
//
// Exact selection by radix passes over 8-bit digits, most significant first:
// |c| as its IEEE-754 bit pattern (monotone in |c| for non-negative values)
// from the top bin down, then, only if several entries share the threshold
// value, the determinant key from the bottom bin up.  Each pass is one
// histogram kernel over the live entries and one single-warp pick kernel.

#include "ucc_device.cuh"

namespace ucc {

namespace {

constexpr int kThreads = 256;
constexpr int kBins = 256;

__device__ __forceinline__ unsigned long long mag_bits(double a) {
  return (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
}

// Histogram of digit `d` of |c| (phase 0) or of the key among |c| == T
// entries (phase 1), restricted to entries whose higher digits equal the
// prefix chosen so far.
__global__ void __launch_bounds__(kThreads) k_select_hist(Table t, SelectState* sel, int phase, int d) {
  __shared__ unsigned int h[kBins];
  if (phase == 1 && !sel->need_keys) return;
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const int shift = 8 * d;
  const unsigned long long hi_mask = (d == 7) ? 0ull : (~0ull << (shift + 8));
  const unsigned long long T = sel->prefix;
  const unsigned long long kp = sel->key_prefix;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag_bits(a);
    if (phase == 0) {
      if ((u & hi_mask) != (T & hi_mask)) continue;
      atomicAdd(&h[(u >> shift) & 0xFF], 1u);
    } else {
      if (u != T) continue;
      const unsigned long long key = t.keys[i];
      if ((key & hi_mask) != (kp & hi_mask)) continue;
      atomicAdd(&h[(key >> shift) & 0xFF], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x)
    if (h[b]) atomicAdd(&sel->hist[b], (unsigned long long)h[b]);
}

// Pick the bin holding the target-th element.  phase 0 walks |c| bins from
// the top (largest first); phase 1 walks key bins from the bottom.
__global__ void k_select_pick(SelectState* sel, int phase, int d) {
  if (phase == 1 && !sel->need_keys) return;
  const int lane = threadIdx.x;  // one warp; lane owns 8 consecutive bins
  unsigned long long c[8];
  unsigned long long local = 0;
  for (int j = 0; j < 8; ++j) {
    // phase 0 visits bins 255..0, phase 1 visits 0..255
    const int b = phase == 0 ? (kBins - 1 - (lane * 8 + j)) : (lane * 8 + j);
    c[j] = sel->hist[b];
    local += c[j];
  }
  // inclusive scan over lanes
  unsigned long long incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned long long before = incl - local;
  const unsigned long long target = phase == 0 ? sel->target : sel->key_target;
  const bool mine = before < target && target <= incl;
  if (mine) {
    unsigned long long cum = before;
    for (int j = 0; j < 8; ++j) {
      if (cum + c[j] >= target) {
        const int b = phase == 0 ? (kBins - 1 - (lane * 8 + j)) : (lane * 8 + j);
        const unsigned long long rest = target - cum;  // rank inside the bin
        if (phase == 0) {
          sel->prefix |= (unsigned long long)b << (8 * d);
          sel->target = rest;
          if (d == 0) {
            sel->count_eq = c[j];
            sel->need_keys = c[j] > rest ? 1 : 0;
            sel->key_target = rest;
          }
        } else {
          sel->key_prefix |= (unsigned long long)b << (8 * d);
          sel->key_target = rest;
        }
        break;
      }
      cum += c[j];
    }
  }
  __syncwarp();
  for (int j = 0; j < 8; ++j) sel->hist[lane * 8 + j] = 0;
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
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag_bits(a);
    bool keep = u > T;
    if (u == T) keep = !keys || t.keys[i] <= Kt;
    if (keep) continue;
    if (RECORD) {
      const unsigned long long ti = aggregated_add(&t.cnt->tape_n);
      if (ti < tape.cap) {
        tape.key[ti] = t.keys[i];
        tape.val[ti] = a;
        tape.born[ti] = t.born[i];
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
  if (last_block_arrive(t.cnt) && threadIdx.x == 0) {
    t.cnt->done = 0u;
    if (RECORD) tape.off[k + 1] = ld_cg(&t.cnt->tape_n);
  }
}

__global__ void k_select_init(SelectState* sel, unsigned long long n_cut) {
  sel->prefix = 0;
  sel->target = n_cut;
  sel->key_prefix = 0;
  sel->key_target = 0;
  sel->need_keys = 0;
  sel->count_eq = 0;
  for (int b = 0; b < kBins; ++b) sel->hist[b] = 0;
}

}  // namespace

cudaError_t launch_select_cut(const Table& t, SelectState* sel, unsigned long long n_cut, unsigned int stamp,
                              int record, const Tape& tape, int k, int grid, cudaStream_t st, long long* launches) {
  k_select_init<<<1, 1, 0, st>>>(sel, n_cut);
  *launches += 1;
  for (int phase = 0; phase < 2; ++phase)
    for (int d = 7; d >= 0; --d) {
      k_select_hist<<<grid, kThreads, 0, st>>>(t, sel, phase, d);
      k_select_pick<<<1, 32, 0, st>>>(sel, phase, d);
      *launches += 2;
    }
  if (record)
    k_select_mark<true><<<grid, kThreads, 0, st>>>(t, sel, stamp, tape, k);
  else
    k_select_mark<false><<<grid, kThreads, 0, st>>>(t, sel, stamp, tape, k);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace ucc
