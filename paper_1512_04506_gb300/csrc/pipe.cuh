// Shared-memory pipeline helpers (mbarrier + cp.async.bulk) for the TMA-fed kernels.
#pragma once

#include "amg_internal.cuh"

namespace amgpipe {

__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ inline bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy completing on `bar`; dst, src 16-byte aligned, bytes % 16 == 0
__device__ inline void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// L2 policy for data streamed once (a coarse operator larger than L2): evict first, so that the
// small vectors around it (the Krylov basis of the coarse solve) stay resident.
__device__ inline uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// bulk_load with an L2 cache policy
__device__ inline void bulk_load_hint(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
__device__ inline void consumer_sync(int nthreads) { asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory"); }

constexpr long long kWaitCycles = 2000000000LL;  // about one second at GB300 clocks
constexpr int kMaxStages = 8;

struct Pipe {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  volatile int abort;
};
constexpr int kPipeBytes = 256;
static_assert(sizeof(Pipe) <= kPipeBytes, "pipe header");

// Waits for phase `parity` of `bar`; false when the CTA aborted or the wait ran out.
__device__ inline bool wait_phase(uint64_t* bar, unsigned parity, Pipe* pp) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (pp->abort) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}
__device__ inline void abort_cta(Pipe* pp, unsigned* err) {
  if (!pp->abort) {
    pp->abort = 1;
    atomicOr(err, AMG_EBIT_TIMEOUT);
  }
}
// Producer epilogue: every copy issued must have landed before the CTA may exit.
__device__ inline void drain(Pipe* pp, long long issued, int ns) {
  for (long long k = issued > ns ? issued - ns : 0; k < issued; ++k) {
    uint64_t* bar = &pp->full[k % ns];
    const unsigned par = (unsigned)((k / ns) & 1);
    const long long t0 = clock64();
    while (!mbar_test(bar, par) && clock64() - t0 < kWaitCycles) {
    }
  }
}


}  // namespace amgpipe
