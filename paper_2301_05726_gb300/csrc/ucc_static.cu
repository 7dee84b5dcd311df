// ucc_energy_static: the energy pass over a caller-held wavefunction with
// all of its scratch memory in one fixed, file-scope device array, so the call
// allocates nothing.
//
// Who needs it: callers that cannot call cudaMalloc / cudaFree at this point
// -- because those calls can synchronise the whole device (a latency-critical
// loop cannot afford that), because every byte of device memory is already
// owned by another allocator (e.g. a framework's caching pool) with nothing
// left to carve, or because they run while the device is out of memory.  They
// still own and pass every input and output buffer; only the scratch (hash
// slots over the caller's keys, block partial sums, counters) comes from here.
//
// The array lives as long as the library stays loaded, on every device that
// loads it: sizeof(StaticScratch), about 8.4 MB per device.  Every call
// reuses it, so two calls whose work overlaps on the GPU (different streams,
// or different host threads on one device) race; serialise them.  Each call
// clears the slots and counters it needs before use.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/ucc.h"
#include "ucc_device.cuh"
#include "ucc_internal.h"

using namespace ucc;

namespace {

constexpr unsigned long long kStaticSlots = 1ull << 19;  // load <= 1/2 at the maximum
constexpr int kStaticGrid = 1216;                         // blocks of the energy kernel (<= this)

struct StaticScratch {
  Counters cnt;
  double partials[2 * kStaticGrid];
  Slot slots[kStaticSlots];
};

static_assert(UCC_STATIC_MAX_DETS * 2ull <= kStaticSlots, "slot array too small for the stated maximum");

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: host code must use the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[sizeof(StaticScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
StaticScratch* g_addr[kMaxDevices] = {};

// Checks the caller's keys (n_alpha electrons on the even spin-orbitals,
// n_beta on the odd ones, none past n_so) and amplitudes (finite) and records
// n in the counters.
__global__ void k_static_init(Counters* c, const unsigned long long* keys, const double* amps,
                              unsigned long long n, int n_alpha, int n_beta, int n_so) {
  constexpr unsigned long long kAlpha = 0x5555555555555555ull;  // spin-orbital p has spin p & 1
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long k = keys[i];
    const bool bad_key = __popcll(k & kAlpha) != n_alpha || __popcll(k & ~kAlpha) != n_beta ||
                         (n_so < 64 && (k >> n_so) != 0ull);
    if (bad_key || !isfinite(amps[i])) atomicOr(&c->error, ERR_CONSISTENCY);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->n_tail = n;
    c->new_n = n;
  }
}

}  // namespace

extern "C" ucc_status ucc_energy_static(int32_t n_spatial, int32_t n_alpha, int32_t n_beta, double e_nuc,
                                        const double* h, const double* g, size_t n_det, const uint64_t* keys,
                                        const double* amps, double* sigma, double* E, double* norm2,
                                        void* cuda_stream) {
  auto err = [](ucc_status s, const std::string& m) {
    set_last_error(m.c_str());
    return s;
  };
  if (!std::isfinite(e_nuc)) return err(UCC_EINVAL, "e_nuc not finite");
  if (n_spatial < 1 || n_spatial > 32 || n_alpha < 0 || n_beta < 0 || n_alpha > n_spatial || n_beta > n_spatial ||
      n_alpha + n_beta < 1)
    return err(UCC_EINVAL, "orbital or electron counts out of range");
  if (!h || !g || !keys || !amps || !sigma || !E) return err(UCC_EINVAL, "null pointer argument");
  if (n_det < 1 || n_det > (size_t)UCC_STATIC_MAX_DETS)
    return err(UCC_EINVAL, "n_det must be in [1, " + std::to_string(UCC_STATIC_MAX_DETS) + "]");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(UCC_ECUDA, "no usable current device");
  // Set-up, once per device, with that device current: the scratch's device
  // address.  The address is cached for the life of the library: a device
  // reset (cudaDeviceReset) unloads the module and would leave it stale, so
  // resetting a device that has called this entry point is not supported.
  StaticScratch* S = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) return err(UCC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = static_cast<StaticScratch*>(p);
    }
    S = g_addr[dev];
  }
  if (cudaMemsetAsync(&S->cnt, 0, sizeof(Counters), st) != cudaSuccess ||
      cudaMemsetAsync(S->slots, 0, sizeof(S->slots), st) != cudaSuccess)
    return err(UCC_ECUDA, "clearing the scratch failed");
  const int n_so = 2 * n_spatial;
  k_static_init<<<kStaticGrid, 256, 0, st>>>(&S->cnt, (const unsigned long long*)keys, amps,
                                             (unsigned long long)n_det, n_alpha, n_beta, n_so);
  Table t{};
  t.keys = const_cast<unsigned long long*>((const unsigned long long*)keys);
  t.amps = const_cast<double*>(amps);
  t.sigma = sigma;
  t.born = nullptr;
  t.lam = nullptr;
  t.slots = S->slots;
  t.slot_mask = kStaticSlots - 1;
  t.slot_shift = 64 - __builtin_ctzll(kStaticSlots);
  t.filt = nullptr;
  t.filt_shift = 32;
  t.cap_n = n_det;
  t.cnt = &S->cnt;
  t.partials = S->partials;
  Integrals in;
  in.h = h;
  in.g = g;
  in.n = n_spatial;
  in.n_so = n_so;
  if (cudaGetLastError() != cudaSuccess || launch_rehash(t, kStaticGrid, st) != cudaSuccess ||
      launch_sigma(t, in, kStaticGrid, st) != cudaSuccess)
    return err(UCC_ECUDA, "kernel launch failed");
  Counters host{};
  cudaError_t e = cudaMemcpyAsync(&host, &S->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(UCC_ECUDA, std::string("energy pass failed: ") + cudaGetErrorString(e));
  if (host.error & ERR_CONSISTENCY)
    return err(UCC_EINVAL, "keys must be distinct determinants with n_alpha electrons on the even and n_beta on "
                           "the odd spin-orbitals below 2*n_spatial, amplitudes finite");
  if (host.error) return err(UCC_ECUDA, "device error word " + std::to_string(host.error));
  if (!(host.norm2 > 0.0)) return err(UCC_EINVAL, "zero wavefunction");
  *E = host.e_num / host.norm2 + e_nuc;
  if (norm2) *norm2 = host.norm2;
  return UCC_OK;
}
