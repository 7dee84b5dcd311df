// Determinant keys: bit p is spin-orbital p (the Jordan-Wigner qubit).  One
// 64-bit word holds up to 64 spin-orbitals (the paper's 32-orbital limit,
// Methods section); a pair of words holds up to 128, the larger active spaces
// the paper's Conclusion says the method extends to.  Every kernel is written
// once over a key type KT and built for both.
#pragma once

#include <stdint.h>

namespace ucc {

struct __align__(16) Key128 {
  unsigned long long lo, hi;  // spin-orbitals 0-63, 64-127
};

__host__ __device__ __forceinline__ Key128 operator&(Key128 a, Key128 b) { return {a.lo & b.lo, a.hi & b.hi}; }
__host__ __device__ __forceinline__ Key128 operator|(Key128 a, Key128 b) { return {a.lo | b.lo, a.hi | b.hi}; }
__host__ __device__ __forceinline__ Key128 operator^(Key128 a, Key128 b) { return {a.lo ^ b.lo, a.hi ^ b.hi}; }
__host__ __device__ __forceinline__ Key128 operator~(Key128 a) { return {~a.lo, ~a.hi}; }
__host__ __device__ __forceinline__ bool operator==(Key128 a, Key128 b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ __forceinline__ bool operator!=(Key128 a, Key128 b) { return !(a == b); }
// Order of keys as 128-bit integers (high word first).
__host__ __device__ __forceinline__ bool key_less(Key128 a, Key128 b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ __forceinline__ bool key_less(unsigned long long a, unsigned long long b) { return a < b; }

// Fibonacci hashing (Knuth, TAOCP vol. 3, 6.4) of the slot: the top bits of
// lo * 2^64/phi + hi * (a second odd constant), mod 2^64; for one-word keys
// the plain product.
constexpr unsigned long long kFibonacci = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long kFibonacciHi = 0xD6E8FEB86659FD93ull;
// Filter hash: lo * C1 + hi * C2 mod 2^64 with two further odd constants.  It
// is additive in the key's set bits wherever adding a bit carries nothing
// (J = I with holes cleared + 2^r + 2^s), which the energy pass uses.
constexpr unsigned long long kFilterMul = 0xbf58476d1ce4e5b9ull;
constexpr unsigned long long kFilterMulHi = 0x94d049bb133111ebull;

template <class KT>
struct KeyOps;

template <>
struct KeyOps<unsigned long long> {
  static constexpr int kBits = 64;
  static constexpr int kWords = 1;
  __host__ __device__ static unsigned long long zero() { return 0ull; }
  __host__ __device__ static unsigned long long bit(int p) { return 1ull << p; }
  // bits 0 .. p-1 (p in [0, 64])
  __host__ __device__ static unsigned long long below(int p) { return p >= 64 ? ~0ull : ((1ull << p) - 1ull); }
  __host__ __device__ static bool test(unsigned long long k, int p) { return ((k >> p) & 1ull) != 0ull; }
  __host__ __device__ static bool is_zero(unsigned long long k) { return k == 0ull; }
  __host__ __device__ static unsigned long long slot_hash(unsigned long long k) { return k * kFibonacci; }
  __host__ __device__ static unsigned long long filt_hash(unsigned long long k) { return k * kFilterMul; }
  // filter-hash term of spin-orbital x
  __host__ __device__ static unsigned long long filt_bit(int x) { return kFilterMul << x; }
  __host__ __device__ static unsigned long long alpha() { return 0x5555555555555555ull; }
  __host__ __device__ static unsigned long long lo(unsigned long long k) { return k; }
  __host__ __device__ static unsigned long long hi(unsigned long long) { return 0ull; }
  __host__ __device__ static unsigned long long from_words(unsigned long long lo, unsigned long long) { return lo; }
#ifdef __CUDACC__
  __device__ static int popc(unsigned long long k) { return __popcll(k); }
#endif
};

template <>
struct KeyOps<Key128> {
  static constexpr int kBits = 128;
  static constexpr int kWords = 2;
  __host__ __device__ static Key128 zero() { return {0ull, 0ull}; }
  __host__ __device__ static Key128 bit(int p) {
    return p < 64 ? Key128{1ull << p, 0ull} : Key128{0ull, 1ull << (p - 64)};
  }
  __host__ __device__ static Key128 below(int p) {
    if (p >= 128) return {~0ull, ~0ull};
    if (p >= 64) return {~0ull, p == 64 ? 0ull : ((1ull << (p - 64)) - 1ull)};
    return {(1ull << p) - 1ull, 0ull};
  }
  __host__ __device__ static bool test(Key128 k, int p) {
    return p < 64 ? ((k.lo >> p) & 1ull) != 0ull : ((k.hi >> (p - 64)) & 1ull) != 0ull;
  }
  __host__ __device__ static bool is_zero(Key128 k) { return (k.lo | k.hi) == 0ull; }
  __host__ __device__ static unsigned long long slot_hash(Key128 k) { return k.lo * kFibonacci + k.hi * kFibonacciHi; }
  __host__ __device__ static unsigned long long filt_hash(Key128 k) { return k.lo * kFilterMul + k.hi * kFilterMulHi; }
  __host__ __device__ static unsigned long long filt_bit(int x) {
    return x < 64 ? (kFilterMul << x) : (kFilterMulHi << (x - 64));
  }
  __host__ __device__ static Key128 alpha() { return {0x5555555555555555ull, 0x5555555555555555ull}; }
  __host__ __device__ static unsigned long long lo(Key128 k) { return k.lo; }
  __host__ __device__ static unsigned long long hi(Key128 k) { return k.hi; }
  __host__ __device__ static Key128 from_words(unsigned long long lo, unsigned long long hi) { return {lo, hi}; }
#ifdef __CUDACC__
  __device__ static int popc(Key128 k) { return __popcll(k.lo) + __popcll(k.hi); }
#endif
};

}  // namespace ucc
