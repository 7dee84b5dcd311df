// Methods-section wavefunction truncation on the device: when more than N_MAX
// determinants are stored after a factor, keep the N_CUT of largest |c|
// (ties: smaller key first) and drop the rest.
//
// Exact selection by radix passes over 11-bit digits, most significant first:
// |c| as its IEEE-754 bit pattern (monotone in |c| for non-negative values)
// from the top bin down, then, only if several entries share the threshold
// value, the determinant key from the bottom bin up.  The first two digits of
// |c| are histogrammed over the whole table (one kernel each: every block
// histograms its share in shared memory, the last block to finish picks the
// bin that holds the target rank); the entries left in the picked bin (a
// relative window of about 2^-10 in |c|) are gathered into a small candidate
// buffer, and one block resolves the remaining digits of |c| and, for ties,
// of the key on that buffer.  When the bin holds more entries than the buffer
// (many exactly equal amplitudes), that block reads the table instead.
//
// The cut itself is fused with the compaction that follows it: one pass
// copies the kept entries into the spare arrays and records the dropped ones
// on the kill tape, so dropped entries are neither tagged nor scanned again.

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

// Turn a histogram of nbins bins (hist_at(b)) into the next digit of the
// threshold, NT threads of one block: phase 0 walks bins from the top (largest
// |c| first), phase 1 from the bottom (smallest key first).
template <int NT, class H>
__device__ void pick_bin(SelectState* sel, int phase, int pass, int nbins, H hist_at,
                         unsigned long long* key_word = nullptr) {
  __shared__ unsigned long long s_scan[NT];
  const int per = (nbins + NT - 1) / NT;
  unsigned long long local = 0;
  for (int j = 0; j < per; ++j) {
    const int o = threadIdx.x * per + j;  // visiting order
    if (o >= nbins) break;
    const int b = phase == 0 ? nbins - 1 - o : o;
    local += hist_at(b);
  }
  s_scan[threadIdx.x] = local;
  __syncthreads();
  // inclusive scan (Hillis-Steele) over the NT partial sums
  for (int off = 1; off < NT; off <<= 1) {
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
      const unsigned long long cnt = hist_at(b);
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
          *(key_word ? key_word : &sel->key_prefix) |= (unsigned long long)b << shift;
          sel->key_target = rest;
        }
        break;
      }
      cum += cnt;
    }
  }
  __syncthreads();
}

// One of the two full-table radix passes over |c| (pass 0: bits 63..53, pass
// 1: bits 52..42), restricted to live entries whose fixed digits match, then
// the pick in the last block.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_select_pass(TableT<KT> t, SelectState* sel, int pass) {
  __shared__ unsigned int h[kBins];
  const int top = 64 - kDigit * pass;
  const int nbins = 1 << (top - digit_shift(pass));
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long hm = high_mask(pass);
  const unsigned long long T = sel->prefix;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag_bits(a);
    if ((u & hm) != (T & hm)) continue;
    atomicAdd(&h[digit_of(u, pass)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (h[b]) atomicAdd(&sel->hist[b], (unsigned long long)h[b]);
  if (last_block_arrive(t.cnt)) {
    pick_bin<kThreads>(sel, 0, pass, nbins, [&](int b) { return ld_cg(&sel->hist[b]); });
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sel->hist[b] = 0;
    if (threadIdx.x == 0) t.cnt->done = 0u;
  }
}

// The live entries whose top 22 bits of |c| equal the threshold's so far.
template <class KT>
__global__ void __launch_bounds__(kThreads) k_select_gather(TableT<KT> t, SelectState* sel, SelectCandT<KT>* cand) {
  const unsigned long long n = min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  const unsigned long long hm = high_mask(2);
  const unsigned long long T = sel->prefix & hm;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a = t.amps[i];
    if (is_dead(a)) continue;
    const unsigned long long u = mag_bits(a);
    if ((u & hm) != T) continue;
    const unsigned long long j = aggregated_add(&sel->n_cand);
    if (j < kSelectCandCap) {
      cand[j].mag = u;
      cand[j].key = t.keys[i];
    }
  }
}

constexpr int kFinishThreads = 1024;

// The remaining digits of |c| (passes 2..5) and, when several entries share
// the threshold value, of the key (its high word first for two-word keys,
// each word in passes 0..5), by one block over the candidate buffer (or over
// the table when the buffer overflowed).
template <class KT>
__global__ void __launch_bounds__(kFinishThreads) k_select_finish(TableT<KT> t, SelectState* sel,
                                                                  const SelectCandT<KT>* cand) {
  using K = KeyOps<KT>;
  __shared__ unsigned int h[kBins];
  __shared__ unsigned long long s_mhi, s_mlo;  // key bits fixed so far (masks), high and low word
  const unsigned long long nc = sel->n_cand;
  const bool from_cand = nc <= kSelectCandCap;
  const unsigned long long n = from_cand ? nc : min(*((volatile unsigned long long*)&t.cnt->n_tail), t.cap_n);
  // entry x as (|c| bits, key), or false for a dropped table entry
  auto entry = [&](unsigned long long x, unsigned long long& u, KT& key) {
    if (from_cand) {
      u = cand[x].mag;
      key = cand[x].key;
      return true;
    }
    const double a = t.amps[x];
    if (is_dead(a)) return false;
    u = mag_bits(a);
    key = t.keys[x];
    return true;
  };
  // |c| digits
  for (int pass = 2; pass < kPasses; ++pass) {
    const int top = 64 - kDigit * pass;
    const int nbins = 1 << (top - digit_shift(pass));
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long hm = high_mask(pass);
    const unsigned long long T = sel->prefix;
    for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) {
      unsigned long long u;
      KT key;
      if (!entry(x, u, key)) continue;
      if ((u & hm) == (T & hm)) atomicAdd(&h[digit_of(u, pass)], 1u);
    }
    __syncthreads();
    pick_bin<kFinishThreads>(sel, 0, pass, nbins, [&](int b) { return (unsigned long long)h[b]; });
  }
  if (!sel->need_keys) return;  // block-uniform
  // key digits among the entries with |c| == T, smallest key first
  if (threadIdx.x == 0) {
    s_mhi = 0ull;
    s_mlo = 0ull;
    sel->key_prefix = 0ull;
    sel->key_prefix_hi = 0ull;
  }
  __syncthreads();
  for (int wp = 0; wp < K::kWords * kPasses; ++wp) {
    const bool hi_word = K::kWords == 2 && wp < kPasses;
    const int pass = wp % kPasses;
    const int top = 64 - kDigit * pass;
    const int nbins = 1 << (top - digit_shift(pass));
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long T = sel->prefix, phi = sel->key_prefix_hi, plo = sel->key_prefix;
    const unsigned long long mhi = s_mhi, mlo = s_mlo;
    for (unsigned long long x = threadIdx.x; x < n; x += blockDim.x) {
      unsigned long long u;
      KT key;
      if (!entry(x, u, key)) continue;
      if (u != T || (K::hi(key) & mhi) != phi || (K::lo(key) & mlo) != plo) continue;
      atomicAdd(&h[digit_of(hi_word ? K::hi(key) : K::lo(key), pass)], 1u);
    }
    __syncthreads();
    pick_bin<kFinishThreads>(sel, 1, pass, nbins, [&](int b) { return (unsigned long long)h[b]; },
                             hi_word ? &sel->key_prefix_hi : &sel->key_prefix);
    if (threadIdx.x == 0) {
      const int shift = digit_shift(pass);
      const unsigned long long dm = (unsigned long long)(nbins - 1) << shift;
      if (hi_word)
        s_mhi |= dm;
      else
        s_mlo |= dm;
    }
    __syncthreads();
  }
}

// The cut fused with the compaction that follows it.  Each block takes tiles
// of 4 x kThreads entries; a live entry above the threshold (|c| > T, or
// |c| == T and key <= key threshold when ties are broken) goes to the spare
// arrays, any other live entry is dropped: recorded on the tape with its value
// and birth factor (RECORD), its Eq. 6 term subtracted (entropy runs).
template <class KT, bool RECORD>
__global__ void __launch_bounds__(kThreads) k_cut_compact(TableT<KT> from, TableT<KT> to, const SelectState* sel,
                                                          TapeT<KT> tape, int k) {
  const unsigned long long n = min(*((volatile unsigned long long*)&from.cnt->n_tail), from.cap_n);
  const unsigned long long T = sel->prefix;
  const bool keys = sel->need_keys != 0;
  const KT Kt = KeyOps<KT>::from_words(sel->key_prefix, sel->key_prefix_hi);
  constexpr int kPer = 4;
  const unsigned long long tile = (unsigned long long)kPer * kThreads;
  unsigned long long dropped = 0;
  double dS = 0.0;
  for (unsigned long long base = (unsigned long long)blockIdx.x * tile; base < n;
       base += (unsigned long long)gridDim.x * tile) {  // block-uniform
    double a[kPer];
    KT key[kPer];
    int state[kPer];  // 0 none, 1 keep, 2 drop
    unsigned int nk = 0, nd = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const unsigned long long i = base + (unsigned long long)u * kThreads + threadIdx.x;
      a[u] = i < n ? from.amps[i] : dead_value(0u);
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      state[u] = 0;
      if (is_dead(a[u])) continue;
      const unsigned long long i = base + (unsigned long long)u * kThreads + threadIdx.x;
      key[u] = from.keys[i];
      const unsigned long long m = mag_bits(a[u]);
      const bool keep = m > T || (m == T && (!keys || !key_less(Kt, key[u])));
      state[u] = keep ? 1 : 2;
      nk += keep;
      nd += !keep;
    }
    // Places: per tile one reservation per counter for the block; inside it
    // the warps in order, and inside a warp tile u after tile u - 1 with the
    // lanes in order, so a warp's kept entries (and tape records) of one tile
    // land next to each other (coalesced stores).
    unsigned int mk[kPer], md[kPer], wk = 0, wd = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      mk[u] = __ballot_sync(0xFFFFFFFFu, state[u] == 1);
      md[u] = __ballot_sync(0xFFFFFFFFu, state[u] == 2);
      wk += __popc(mk[u]);
      wd += __popc(md[u]);
    }
    (void)nk;
    (void)nd;
    __shared__ unsigned int s_wk[kThreads / 32], s_wd[kThreads / 32];
    __shared__ unsigned long long s_bk, s_bd;
    const unsigned int lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const unsigned int below_me = (1u << lane) - 1u;
    if (lane == 0) {
      s_wk[w] = wk;
      s_wd[w] = wd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int rk = 0, rd = 0;
      for (int x = 0; x < kThreads / 32; ++x) {
        const unsigned int a = s_wk[x], b = s_wd[x];
        s_wk[x] = rk;
        s_wd[x] = rd;
        rk += a;
        rd += b;
      }
      s_bk = rk ? atomicAdd(&from.cnt->new_n, (unsigned long long)rk) : 0ull;
      s_bd = (RECORD && rd) ? atomicAdd(&from.cnt->tape_n, (unsigned long long)rd) : 0ull;
    }
    __syncthreads();
    unsigned long long pk = s_bk + s_wk[w], pd = s_bd + s_wd[w];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const unsigned long long i = base + (unsigned long long)u * kThreads + threadIdx.x;
      if (state[u] == 1) {
        const unsigned long long at = pk + __popc(mk[u] & below_me);
        if (at < to.cap_n) {
          to.keys[at] = key[u];
          to.amps[at] = a[u];
          if (to.born) to.born[at] = from.born[i];
        } else {
          raise_error(from.cnt, ERR_CAPACITY);
        }
      } else if (state[u] == 2) {
        ++dropped;
        if (from.entropy) dS -= entropy_term(a[u]);
        if (RECORD) {
          const unsigned long long at = pd + __popc(md[u] & below_me);
          if (at < tape.cap) {
            TapeRecT<KT>& rec = tape_at(tape, at);
            rec.key = key[u];
            rec.val = a[u];
            rec.born = from.born[i];
          } else {
            raise_error(from.cnt, ERR_TAPE_FULL);
          }
        }
      }
      pk += __popc(mk[u]);
      pd += __popc(md[u]);
    }
    __syncthreads();  // s_wk, s_wd, s_bk, s_bd are reused by the next tile
  }
  __shared__ unsigned long long s_d;
  if (threadIdx.x == 0) s_d = 0;
  __syncthreads();
  if (dropped) atomicAdd(&s_d, dropped);
  if (from.entropy) {
    const double b = block_sum(dS);
    if (threadIdx.x == 0) from.partials[blockIdx.x] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_d) atomicAdd(&const_cast<SelectState*>(sel)->cut_total, s_d);
  const bool last = last_block_arrive(from.cnt);
  if (last && from.entropy) {
    double s = 0.0;
    for (unsigned int x = threadIdx.x; x < gridDim.x; x += blockDim.x) s += ld_cg(&from.partials[x]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
      from.cnt->entropy += s;
      from.entropy[k] = from.cnt->entropy;
    }
  }
  if (last && threadIdx.x == 0) {
    from.cnt->done = 0u;
    if (RECORD) tape.off[k + 1] = ld_cg(&from.cnt->tape_n);
  }
}

__global__ void k_select_init(SelectState* sel, unsigned long long n_cut) {
  if (threadIdx.x == 0) {
    sel->prefix = 0;
    sel->target = n_cut;
    sel->key_prefix = 0;
    sel->key_prefix_hi = 0;
    sel->key_target = 0;
    sel->need_keys = 0;
    sel->count_eq = 0;
    sel->n_cand = 0;
  }
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) sel->hist[b] = 0;
}

}  // namespace

template <class KT>
cudaError_t launch_select_threshold(const TableT<KT>& t, SelectState* sel, SelectCandT<KT>* cand,
                                    unsigned long long n_cut, int grid, cudaStream_t st, long long* launches) {
  k_select_init<<<1, kThreads, 0, st>>>(sel, n_cut);
  k_select_pass<KT><<<grid, kThreads, 0, st>>>(t, sel, 0);
  k_select_pass<KT><<<grid, kThreads, 0, st>>>(t, sel, 1);
  k_select_gather<KT><<<grid, kThreads, 0, st>>>(t, sel, cand);
  k_select_finish<KT><<<1, kFinishThreads, 0, st>>>(t, sel, cand);
  *launches += 5;
  return cudaGetLastError();
}

template <class KT>
cudaError_t launch_cut_compact(const TableT<KT>& from, const TableT<KT>& to, const SelectState* sel, int record,
                               const TapeT<KT>& tape, int k, int grid, cudaStream_t st) {
  if (record)
    k_cut_compact<KT, true><<<grid, kThreads, 0, st>>>(from, to, sel, tape, k);
  else
    k_cut_compact<KT, false><<<grid, kThreads, 0, st>>>(from, to, sel, tape, k);
  return cudaGetLastError();
}

#define UCC_SELECT_INSTANTIATE(KT)                                                                                \
  template cudaError_t launch_select_threshold<KT>(const TableT<KT>&, SelectState*, SelectCandT<KT>*,             \
                                                   unsigned long long, int, cudaStream_t, long long*);           \
  template cudaError_t launch_cut_compact<KT>(const TableT<KT>&, const TableT<KT>&, const SelectState*, int,      \
                                              const TapeT<KT>&, int, int, cudaStream_t);
UCC_SELECT_INSTANTIATE(unsigned long long)
UCC_SELECT_INSTANTIATE(Key128)

}  // namespace ucc
