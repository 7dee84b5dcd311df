// Device helpers: hashing, probing, dropped-entry tags, reductions.
#pragma once

#include <cooperative_groups.h>
#include <stdint.h>

#include "ucc_internal.h"

namespace ucc {
namespace cg = cooperative_groups;

// Probe steps before a lookup gives up and raises ERR_PROBE_BOUND.  The host
// keeps the table at most 75% full, where linear probing needs a handful of
// steps; the bound only guarantees termination.
constexpr int MAX_PROBE = 1 << 14;

// Home slot of a key: Fibonacci hashing (Knuth, TAOCP vol. 3, 6.4) -- the
// top log2(slots) bits of key * 2^64/phi (KeyOps::slot_hash).  One 64-bit
// multiply per key word; on the workloads' determinant keys it gives the same
// linear-probing lengths as a full 64-bit finalizer.
template <class KT>
__device__ __forceinline__ unsigned long long home_slot(const TableT<KT>& t, KT key) {
  return KeyOps<KT>::slot_hash(key) >> t.slot_shift;
}

// Existence filter: a blocked Bloom filter of 32-bit words, 8 filter bits per
// hash slot (1/16 the size of the slot array, so it mostly stays in L2).  A
// key's filter hash h = key * kFilterMul (a second odd constant, the
// SplitMix64 finalizer's first multiplier, so it does not follow the slot)
// picks one word by its top bits and three bit positions in that word by the
// next 15 bits; the key sets all three.  Word and bits come from the high
// half of h and one funnel shift, so the test is 32-bit integer work.  A lookup is one load: a word missing
// any of the key's bits proves the key absent and saves the probe; a word
// holding all three (a stored key, or a collision) falls through to the
// probe.  Three bits in one word make collisions far rarer than one bit per
// key at the same size (the connection probes of the energy pass are mostly
// of absent keys).
template <class TT>
__device__ __forceinline__ unsigned int filter_word(const TT& t, unsigned long long h) {
  return (unsigned int)(h >> 32) >> t.filt_shift;  // the top log2(words) bits of h
}
template <class TT>
__device__ __forceinline__ unsigned int filter_bits(const TT& t, unsigned long long h) {
  // the 32 bits of h just below the word index
  const unsigned int r = __funnelshift_l((unsigned int)h, (unsigned int)(h >> 32), 32 - t.filt_shift);
  return (1u << (r >> 27)) | (1u << ((r >> 22) & 31u)) | (1u << ((r >> 17) & 31u));
}
// Whether filter word w holds every bit of the key with filter hash h.
template <class TT>
__device__ __forceinline__ bool filter_hit(const TT& t, unsigned int w, unsigned long long h) {
  const unsigned int m = filter_bits(t, h);
  return (w & m) == m;
}

template <class KT>
__device__ __forceinline__ bool filter_maybe(const TableT<KT>& t, KT key) {
  if (!t.filt) return true;
  const unsigned long long h = KeyOps<KT>::filt_hash(key);
  return filter_hit(t, t.filt[filter_word(t, h)], h);
}

template <class KT>
__device__ __forceinline__ void filter_add(const TableT<KT>& t, KT key) {
  if (!t.filt) return;
  const unsigned long long h = KeyOps<KT>::filt_hash(key);
  atomicOr(&t.filt[filter_word(t, h)], filter_bits(t, h));
}

// 16-byte compare-and-swap on a two-word key (sm_90 and later); returns the
// previous value.  One-word keys use the 8-byte atomicCAS.
__device__ __forceinline__ unsigned long long key_cas(unsigned long long* p, unsigned long long cmp,
                                                      unsigned long long val) {
  return atomicCAS(p, cmp, val);
}
__device__ __forceinline__ Key128 key_cas(Key128* p, Key128 cmp, Key128 val) {
  Key128 old;
  asm volatile(
      "{\n\t.reg .b128 c, v, d;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(old.lo), "=l"(old.hi)
      : "l"(cmp.lo), "l"(cmp.hi), "l"(val.lo), "l"(val.hi), "l"(p)
      : "memory");
  return old;
}

// A dropped entry keeps its key and slot; its amplitude becomes a quiet NaN
// whose low 32 bits name the step that dropped it.  Live amplitudes are never
// NaN (finite inputs, finite cos/sin).
constexpr unsigned int DEAD_TAG_HI = 0x7FFC0000u;

__device__ __forceinline__ double dead_value(unsigned int stamp) {
  return __longlong_as_double((long long)(((unsigned long long)DEAD_TAG_HI << 32) | stamp));
}
__device__ __forceinline__ bool is_dead(double v) {
  return (unsigned int)((unsigned long long)__double_as_longlong(v) >> 32) == DEAD_TAG_HI;
}
__device__ __forceinline__ unsigned int dead_stamp(double v) {
  return (unsigned int)((unsigned long long)__double_as_longlong(v) & 0xFFFFFFFFull);
}

__device__ __forceinline__ void raise_error(Counters* c, int bit) { atomicOr(&c->error, bit); }
__device__ __forceinline__ void raise_consistency(Counters* c, int site, unsigned long long key = 0ull) {
  atomicOr(&c->error, ERR_CONSISTENCY);
  if (atomicCAS(&c->err_site, 0, site) == 0) c->err_key = key;
}

// Result of looking a key up.
enum Found : int { ABSENT = 0, ALIVE = 1, DEAD_NOW = 2, DEAD_OLD = 3 };

struct Lookup {
  int state;                 // Found
  unsigned long long slot;   // slot of the key, or the first empty slot (ABSENT)
  unsigned long long idx;    // entry index (ALIVE / DEAD_*)
  double amp;                // amplitude (ALIVE)
};

template <class TT>
__device__ __forceinline__ void classify(const TT& t, unsigned long long idx, unsigned int stamp, Lookup& r) {
  r.idx = idx;
  double a = t.amps[idx];
  if (!is_dead(a)) {
    r.state = ALIVE;
    r.amp = a;
  } else {
    r.state = dead_stamp(a) == stamp ? DEAD_NOW : DEAD_OLD;
  }
}

// A lane's key broadcast from lane src.
__device__ __forceinline__ unsigned long long shfl_key(unsigned long long k, unsigned int src) {
  return __shfl_sync(0xFFFFFFFFu, k, src);
}
__device__ __forceinline__ Key128 shfl_key(Key128 k, unsigned int src) {
  return {__shfl_sync(0xFFFFFFFFu, k.lo, src), __shfl_sync(0xFFFFFFFFu, k.hi, src)};
}

// Single-lane linear probe.
template <class KT>
__device__ __forceinline__ Lookup find1(const TableT<KT>& t, KT key, unsigned int stamp) {
  Lookup r;
  r.state = ABSENT;
  r.idx = 0;
  r.amp = 0.0;
  unsigned long long h = home_slot(t, key);
  if (!filter_maybe(t, key)) {
    r.slot = h;  // absent: an insertion claims the first empty slot from home
    return r;
  }
  for (int step = 0; step < MAX_PROBE; ++step) {
    const SlotT<KT> s = t.slots[h];
    if (s.key == key) {
      r.slot = h;
      classify(t, s.idx, stamp, r);
      return r;
    }
    if (KeyOps<KT>::is_zero(s.key)) {
      r.slot = h;
      return r;
    }
    h = (h + 1) & t.slot_mask;
  }
  raise_error(t.cnt, ERR_PROBE_BOUND);
  r.slot = ~0ull;
  return r;
}

// Group-cooperative linear probe: the G lanes of a group read G consecutive
// slots in one step and vote.  Every lane of the warp must call it (inactive
// lanes pass active = false); each lane receives the result of its own query.
template <int G, class KT>
__device__ __forceinline__ Lookup findG(const TableT<KT>& t, KT key, bool active, unsigned int stamp) {
  if constexpr (G == 1) {
    Lookup r;
    r.state = ABSENT;
    r.idx = 0;
    r.amp = 0.0;
    r.slot = 0;
    if (active) r = find1(t, key, stamp);
    return r;
  } else {
    const unsigned int lane = threadIdx.x & 31u;
    const unsigned int gbase = lane & ~(unsigned)(G - 1);
    const unsigned int sub = lane - gbase;
    const unsigned int gmask = (G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << gbase));
    Lookup mine;
    mine.state = ABSENT;
    mine.idx = 0;
    mine.amp = 0.0;
    mine.slot = 0;
    for (int q = 0; q < G; ++q) {
      const unsigned int src = gbase + q;
      const KT qk = shfl_key(key, src);
      bool qa = __shfl_sync(0xFFFFFFFFu, active, src);
      // Group-uniform: every lane of the group sees the same qk / qa.
      unsigned long long res_slot = 0, res_idx = 0;
      int res_state = ABSENT;
      unsigned long long h = home_slot(t, qk);
      bool decided = !qa;
      if (qa && !filter_maybe(t, qk)) {  // group-uniform: absent without a probe
        decided = true;
        res_slot = h;
      }
      for (int step = 0; step < MAX_PROBE / G; ++step) {
        // All lanes of the warp run this loop in lock step (the trip count is
        // warp-uniform via the ballot below), so full-mask votes are safe.
        unsigned long long my = (h + sub) & t.slot_mask;
        SlotT<KT> s;
        s.key = KeyOps<KT>::bit(0);
        s.idx = 0;
        if (!decided) s = t.slots[my];
        unsigned int hit = __ballot_sync(0xFFFFFFFFu, !decided && s.key == qk) & gmask;
        unsigned int emp = __ballot_sync(0xFFFFFFFFu, !decided && KeyOps<KT>::is_zero(s.key)) & gmask;
        if (!decided) {
          if (hit) {
            int w = __ffs(hit) - 1;
            res_slot = __shfl_sync(gmask, my, w);
            res_idx = __shfl_sync(gmask, s.idx, w);
            res_state = ALIVE;  // refined by classify below
            decided = true;
          } else if (emp) {
            int w = __ffs(emp) - 1;
            res_slot = __shfl_sync(gmask, my, w);
            res_state = ABSENT;
            decided = true;
          } else {
            h = (h + G) & t.slot_mask;
          }
        }
        if (__all_sync(0xFFFFFFFFu, decided)) break;
        if (step == MAX_PROBE / G - 1 && !decided) raise_error(t.cnt, ERR_PROBE_BOUND);
      }
      if (lane == src && qa) {
        mine.slot = res_slot;
        if (res_state == ALIVE) {
          classify(t, res_idx, stamp, mine);
        } else {
          mine.state = ABSENT;
        }
      }
    }
    return mine;
  }
}

// Claim an empty slot for key, starting at the slot a failed lookup ended on.
// Only one lane ever inserts a given key during a step, so a lost CAS means
// another key took the slot and the probe moves on.
template <class KT>
__device__ __forceinline__ unsigned long long claim_slot(const TableT<KT>& t, KT key, unsigned long long start,
                                                         int site = SITE_DUP_CLAIM) {
  unsigned long long h = start & t.slot_mask;
  for (int step = 0; step < MAX_PROBE; ++step) {
    const KT prev = key_cas(&t.slots[h].key, KeyOps<KT>::zero(), key);
    if (KeyOps<KT>::is_zero(prev)) {
      filter_add(t, key);
      return h;
    }
    if (prev == key) {
      raise_consistency(t.cnt, site, KeyOps<KT>::lo(key));
      return h;
    }
    h = (h + 1) & t.slot_mask;
  }
  raise_error(t.cnt, ERR_PROBE_BOUND);
  return ~0ull;
}

// Warp-aggregated increment of a device counter: the lanes that reach this
// call together share one atomicAdd and receive consecutive values.
__device__ __forceinline__ unsigned long long aggregated_add(unsigned long long* counter) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  return base + g.thread_rank();
}

// Append (key, amp) as a new entry and point a slot at it.
template <class KT>
__device__ __forceinline__ bool insert_new(const TableT<KT>& t, KT key, double amp, unsigned int born,
                                           unsigned long long start_slot, bool with_born, bool with_lam,
                                           int site = SITE_DUP_CLAIM) {
  unsigned long long s = claim_slot(t, key, start_slot, site);
  unsigned long long idx = aggregated_add(&t.cnt->n_tail);
  if (idx >= t.cap_n || s == ~0ull) {
    raise_error(t.cnt, ERR_CAPACITY);
    return false;
  }
  t.keys[idx] = key;
  t.amps[idx] = amp;
  if (with_born) t.born[idx] = born;
  if (with_lam) t.lam[idx] = 0.0;
  t.slots[s].idx = idx;
  return true;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Block-wide sum; result valid in thread 0.  blockDim.x <= 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// "Last block" pattern: every block calls this once at its end; it returns
// true in exactly one block, after all other blocks' prior writes are visible.
__device__ __forceinline__ bool last_block_arrive(Counters* c) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(&c->done, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

template <class KT>
__device__ __forceinline__ TapeRecT<KT>& tape_at(const TapeT<KT>& tp, unsigned long long x) {
  return tp.pages[x >> kTapePageBits][x & (kTapePageRecs - 1ull)];
}

// Blocks of a kernel that are resident on the current device at once (one
// full wave), capped at grid: grid-strided kernels launched with this run in
// a single wave instead of a full wave plus a second one behind it.
template <auto Kernel, int Threads>
inline int one_wave(int grid) {
  static const int resident = [] {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, Kernel, Threads, 0) != cudaSuccess)
      return 0;
    return sms * occ;
  }();
  return resident > 0 && resident < grid ? resident : grid;
}

// Loads that bypass L1 (values other blocks wrote in this kernel).
__device__ __forceinline__ unsigned long long ld_cg(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }

}  // namespace ucc
