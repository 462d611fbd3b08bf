// Device helpers shared by the kernels: acquire/release flags, bounded waits,
// mbarrier-tracked 1-D TMA bulk copies (cp.async.bulk) into shared memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace stiles {
namespace dev {

// Bound on waiting for a TMA copy that has been issued (copies always
// complete; the bound only guards against a hardware fault).  Independent of
// the user's spin limit, so that an aborting CTA never leaves a copy in flight.
constexpr long long kTmaWaitLimit = 1ll << 26;

// Control block of one persistent launch.
struct Ctl {
  int ticket;               // next ticket to hand out
  int status;               // 0 = ok, STILES_ERR_TIMEOUT when a wait gave up
  int abort;                // set on timeout: every CTA leaves at its next check
  int ticket2;              // next ticket of the second queue (critical-chain tasks)
  unsigned long long info;  // 1-based permuted column of the first bad pivot, ULLONG_MAX if none
  long long where;          // diagnostic: ticket that timed out
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Order this thread's earlier generic-proxy accesses with its later async-proxy
// (TMA) accesses to global memory, and vice versa.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared, completion counted on `bar` in bytes.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Wait until *flag == want; bounded by `limit` polls; gives up early when the
// launch is aborting.  Returns false on timeout/abort (the caller must stop).
// The first polls are back to back (the common case is a short wait on the
// critical path); later polls back off with __nanosleep.
__device__ __forceinline__ bool wait_flag(const int* flag, int want, long long limit, Ctl* ctl) {
  if (ld_acquire(flag) == want) return true;
  for (long long it = 0; it < limit; ++it) {
    if (it >= 2048) __nanosleep(256);
    if (ld_acquire(flag) == want) return true;
    if ((it & 255) == 255 && ld_volatile(&ctl->abort)) return false;
  }
  return false;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int smid() {
  int s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

__device__ __forceinline__ void raise_timeout(Ctl* ctl, long long where) {
  if (atomicCAS(&ctl->status, 0, 5 /* STILES_ERR_TIMEOUT */) == 0) ctl->where = where;
  atomicExch(&ctl->abort, 1);
}

// Reciprocal of a double on the pivot chain of the POTRFs, where the latency
// of an IEEE division is the cost that matters.  Newton-Raphson refinement of
// a single-precision seed, using the third-order member of the classical
// reciprocal iteration, y' = y (1 + e + e^2) with e = 1 - v y, which cubes the
// relative error (e' = e^3):
//   * the seed is rcp.approx.ftz.f32 (at most 1 ulp, i.e. 2^-23 relative) of
//     the mantissa of v as a float in [1, 2) (truncated to 23 bits, another
//     2^-23), rescaled by 2^-(exponent of v) with integer arithmetic, so the
//     seed error is below 2^-22 for every normal v without a float range limit;
//   * one third-order step leaves |e|^3 < 2^-66, below the final rounding, so
//     the result is within a few units in the last place of 1/v.
// Positive or negative normal v with a biased exponent in [1, 2044]; anything
// else (zero, subnormal, huge, inf, NaN) takes the IEEE division.
__device__ __forceinline__ double fast_rcp(double v) {
  const int hi = __double2hiint(v);
  const unsigned lo = static_cast<unsigned>(__double2loint(v));
  const int ex = (hi >> 20) & 0x7ff;
  if (ex < 1 || ex > 2044) return 1.0 / v;
  const float m = __int_as_float(0x3f800000 | ((hi & 0x000fffff) << 3) | int(lo >> 29));
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));  // r in (0.5, 1]
  const int rb = __float_as_int(r);
  // r = 2^(er - 127) * 1.f  ->  1/v ~ 2^(er - 127 - (ex - 1023)) * 1.f
  const int yex = ((rb >> 23) & 0xff) - 127 + 1023 - (ex - 1023);
  const int yhi = (hi & int(0x80000000u)) | (yex << 20) | ((rb & 0x7fffff) >> 3);
  double y = __hiloint2double(yhi, rb << 29);
  const double e = fma(-v, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

}  // namespace dev
}  // namespace stiles
