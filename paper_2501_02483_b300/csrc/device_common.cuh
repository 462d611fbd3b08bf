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
// Relaxed load: several can be in flight at once (an acquire load orders every
// later access after it, so a run of them costs one round trip each); a run of
// relaxed loads followed by fence_acq_rel_gpu() acquires them all together.
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
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

// Index of the first flag among ptr(first) .. ptr(n - 1) below its wanted
// value want(i) (n if none), read with up to 16 relaxed loads in flight (no
// acquire: the caller fences once it has advanced).  Flags only grow.
template <class P, class V>
__device__ __forceinline__ int count_set_flags(P ptr, V want, int first, int n) {
  constexpr int W = 16;
  while (first < n) {
    bool ok[W];
#pragma unroll
    for (int j = 0; j < W; ++j) ok[j] = (first + j < n) ? ld_relaxed(ptr(first + j)) >= want(first + j) : true;
    int adv = 0;
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (adv == j && ok[j]) ++adv;
    first = min(first + adv, n);
    if (adv < W) break;
  }
  return first;
}
template <class P>
__device__ __forceinline__ int count_set_flags(P ptr, int first, int n) {
  return count_set_flags(ptr, [](int) { return 1; }, first, n);
}

// Waits until every flag ptr(i), i < n, has reached want(i), polling them in
// batches; the final fence acquires every one of them.  Bounded like wait_flag.
template <class P, class V>
__device__ __forceinline__ bool wait_flags(P ptr, V want, int n, long long limit, Ctl* ctl) {
  int first = 0;
  for (long long it = 0;; ++it) {
    first = count_set_flags(ptr, want, first, n);
    if (first >= n) break;
    if (it >= limit) return false;
    if (it >= 2048) __nanosleep(256);
    if ((it & 255) == 255 && ld_volatile(&ctl->abort)) return false;
  }
  fence_acq_rel_gpu();
  return true;
}
template <class P>
__device__ __forceinline__ bool wait_flags(P ptr, int n, long long limit, Ctl* ctl) {
  return wait_flags(ptr, [](int) { return 1; }, n, limit, ctl);
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

}  // namespace dev
}  // namespace stiles
