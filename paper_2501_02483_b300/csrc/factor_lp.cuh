// Mixed-precision persistent tile Cholesky: the tile updates (SYRK/GEMM of
// Algorithm 1 and the tree partials of Algorithm 3) run on the tcgen05 tensor
// cores with BF16 or FP16 operands and FP32 accumulation in tensor memory; the
// triangular solves of off-diagonal tiles run in FP32; the diagonal tiles are
// factored in FP64.
//
// Tiles are B = 64 wide.  Every finished off-diagonal tile is stored twice:
// FP32 column-major (for the solves and the final answer) and in 16-bit form
// in the tensor cores' K-major core-matrix layout (8 x 8 blocks of 16 bytes,
// row blocks of 8 blocks), so one 1-D TMA bulk copy lands an operand in shared
// memory ready for the MMA.  The MMA is M = 128, N = 64, K = 16: the A operand
// buffer holds the 64-row tile followed by 64 zero rows, and only TMEM lanes
// 0..63 (warps 0 and 1) are read back.
//
// Scheduling is the same ticket / ready-flag scheme as the FP64 kernel.  One
// thread streams the operand tiles and issues the MMAs; the other threads wait
// for the accumulation and run the epilogue.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device_common.cuh"
#include "factor_f64.cuh"
#include "plan.h"

namespace stiles {
namespace dev {

constexpr int LP_B = 64;
constexpr int LP_TILE = LP_B * LP_B;
constexpr int LP_NSTAGE = 2;
constexpr uint32_t LP_OP_BYTES = LP_TILE * 2;       // one 16-bit operand tile
constexpr uint32_t LP_STAGE_BYTES = 3 * LP_OP_BYTES; // A (tile + 64 zero rows) + B
constexpr uint32_t LP_TMEM_COLS = 128;              // two 64-column FP32 accumulators (per slot)
constexpr int LP_SLOTS = 2;                         // task slots per CTA
constexpr int LP_THREADS = 128 * LP_SLOTS;

// shared memory: stages (also the POTRF's scratch) | sD (FP64 64x64) | sL (FP32 64x64) | sInv/sPiv/sRs
// (FP64 x 64 each) | barriers
constexpr size_t LP_SMEM = size_t(LP_NSTAGE) * LP_STAGE_BYTES + LP_TILE * 8 + LP_TILE * 4 + 3 * LP_B * 8 +
                           (LP_NSTAGE * 2 + 2) * 8 + 64;
constexpr size_t LP_SLOT_BYTES = (LP_SMEM + 1023) / 1024 * 1024;  // one slot's dynamic shared memory
constexpr size_t LP_KERNEL_SMEM = LP_SLOTS * LP_SLOT_BYTES;

struct LPMatCtx {
  float* tiles32;        // nsub * 64 * 64, column-major
  uint16_t* tiles16;     // nsub * 64 * 64, core-matrix layout, BF16 or FP16
  float* scratch;        // tree partials (negated sums), FP32 column-major
  float* invdiag32;      // nsb * 64: 1 / L_jj
  double* ldiag;         // nsb * 64: L_jj in FP64 (log-determinant)
  const DevTask* tasks;
  const int32_t* pairs;
  const int32_t* parts;
  int* flags;
  int* sflags;
  unsigned long long* info;
  long long* trace;
};

struct LPArgs {
  LPMatCtx single;       // the matrix of a one-matrix launch (mats == NULL)
  const LPMatCtx* mats;  // batched launch: one context per matrix (device memory)
  const int2* tickets;   // batched launch: (matrix, task) per ticket; NULL: one matrix
  int ntasks;
  Ctl* ctl;
  long long spin_limit;
  int fp16;              // 0: BF16 operands, 1: FP16 operands
};

__device__ __forceinline__ uint32_t lp_core_offset(int r, int k) {
  return uint32_t(((r >> 3) * (LP_B / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr >> 4) & 0x3FFF);
  d |= uint64_t((lbo >> 4) & 0x3FFF) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
  d |= uint64_t(1) << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 32 consecutive FP32 columns of TMEM lane (32 * warp + lane) into v
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  long long spins = 0;
  while (!mbar_try_wait(bar, parity))
    if (++spins > kTmaWaitLimit) return false;
  return true;
}

__device__ __forceinline__ uint16_t to_lp(float x, int fp16) {
  return fp16 ? __half_as_ushort(__float2half_rn(x)) : __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Store row `r` (64 FP32 values) of a finished tile: FP32 column-major and the
// 16-bit core-matrix copy (8 x 16-byte vectors).
__device__ __forceinline__ void lp_store_row(const LPMatCtx& mc, int fp16, int sub, int r, const float (&x)[LP_B]) {
  float* t32 = mc.tiles32 + size_t(sub) * LP_TILE;
#pragma unroll
  for (int c = 0; c < LP_B; ++c) t32[c * LP_B + r] = x[c];
  unsigned char* t16 = reinterpret_cast<unsigned char*>(mc.tiles16 + size_t(sub) * LP_TILE);
#pragma unroll
  for (int kb = 0; kb < LP_B / 8; ++kb) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h)
      w[h] = uint32_t(to_lp(x[kb * 8 + 2 * h], fp16)) | (uint32_t(to_lp(x[kb * 8 + 2 * h + 1], fp16)) << 16);
    *reinterpret_cast<uint4*>(t16 + lp_core_offset(r, kb * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__shared__ uint16_t lp_sElem16[PotrfDf<16>::NLIVE];  // element numbering of the 16-wide POTRF

// One task slot: 128 threads (4 warps) running the persistent task loop on
// their own shared-memory area, mbarriers, TMEM columns and ticket, with a
// named barrier for the slot's own synchronisation.

template <int SLOT>
__device__ __forceinline__ void lp_slot(const LPArgs& a, uint32_t tmem, int tid) {
  extern __shared__ __align__(1024) unsigned char lp_dyn[];
  __shared__ int sTicket, sAbort;  // one pair per instantiation, i.e. per slot
  unsigned char* smem_raw = lp_dyn + SLOT * LP_SLOT_BYTES;
  __builtin_assume(tid >= 0 && tid < 128);
  auto sync = []() { asm volatile("bar.sync %0, 128;" ::"n"(1 + SLOT) : "memory"); };
  auto publish = [&](int* flag) {
    sync();
    if (tid == 0) st_release(flag, 1);
  };
  unsigned char* sStage = smem_raw;                                    // LP_NSTAGE * LP_STAGE_BYTES
  double* sD = reinterpret_cast<double*>(sStage + LP_NSTAGE * LP_STAGE_BYTES);  // 64x64 FP64
  float* sL = reinterpret_cast<float*>(sD + LP_TILE);                 // 64x64 FP32
  double* sInv = reinterpret_cast<double*>(sL + LP_TILE);
  double* sPiv = sInv + LP_B;
  double* sRs = sPiv + LP_B;
  uint64_t* full = reinterpret_cast<uint64_t*>(sRs + LP_B);  // [LP_NSTAGE] operands landed
  uint64_t* empty = full + LP_NSTAGE;                         // [LP_NSTAGE] MMAs done with the stage
  uint64_t* accbar = empty + LP_NSTAGE;                       // all MMAs of the task done
  uint64_t* lbar = accbar + 1;                                // L_kk landed
  const int warp = tid >> 5, lane = tid & 31;
  (void)lane;
  if (tid == 0) {
    for (int s = 0; s < LP_NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accbar, 1);
    mbar_init(lbar, 1);
    mbar_fence_init();
  }
  // the 64 zero rows below each A operand tile (the MMA is M = 128)
  for (int s = 0; s < LP_NSTAGE; ++s) {
    uint4* z = reinterpret_cast<uint4*>(sStage + s * LP_STAGE_BYTES + LP_OP_BYTES);
    for (int i = tid; i < int(LP_OP_BYTES / 16); i += 128) z[i] = make_uint4(0, 0, 0, 0);
  }
  fence_proxy_async_shared();
  sync();
  const long long limit = a.spin_limit;
  // kind::f16 instruction descriptor: D = F32, A/B = BF16 (1) or F16 (0), both K-major,
  // N = 64 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24)
  const uint32_t fmt = a.fp16 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(64 >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  const uint32_t kLBO = 128, kSBO = (LP_B / 8) * 128;
  uint32_t ph_full = 0, ph_empty = 0, ph_acc = 0, ph_l = 0;  // parity bits
  uint32_t pending = 0;  // stage s has committed MMAs not yet waited on (thread 0 only)

  int next = 0;
  if (tid == 0) next = atomicAdd(&a.ctl->ticket, 1);
  bool aborted = false;
  while (!aborted) {
    // generic-proxy writes of the previous task to shared buffers that TMA
    // refills (sL, sRs) before the next copies
    fence_proxy_async_shared();
    if (tid == 0) {
      int cur = next;
      if (cur < a.ntasks && ld_volatile(&a.ctl->abort) == 0) next = atomicAdd(&a.ctl->ticket, 1);
      else cur = -1;
      sTicket = cur;
      sAbort = 0;
    }
    sync();
    const int t = sTicket;
    if (t < 0) break;
    int mi = 0, ti = t;
    if (a.tickets) {
      const int2 v = a.tickets[t];
      mi = v.x;
      ti = v.y;
    }
    const LPMatCtx mc = a.mats ? a.mats[mi] : a.single;
    const DevTask tk = mc.tasks[ti];
    long long* const trace = mc.trace ? mc.trace + 4 * size_t(ti) : nullptr;
    if (trace && tid == 0) {
      trace[0] = (long long)globaltimer();
      trace[3] = smid();
    }
    const bool chain = tk.type == TASK_CHAIN;
    const int nq = tk.qe - tk.qb, np = tk.pe - tk.pb;

    // ---- producer / MMA issuer: thread 0.  Item j uses stage j % 2; the copy of
    // item j + 1 is issued before the MMAs of item j when its tiles are ready. ----
    bool used[2] = {false, false};  // accumulator received at least one MMA
    if (tid == 0) {
      int issued = 0;
      auto issue = [&](int j, bool block) -> int {  // 1 issued, 0 not ready, -1 abort
        const int raw = mc.pairs[2 * (tk.pb + j)];
        const int pa = raw & kIndexMask, pb = mc.pairs[2 * (tk.pb + j) + 1];
        if (block) {
          if (!(wait_flag(mc.flags + pa, 1, limit, a.ctl) && (pb == pa || wait_flag(mc.flags + pb, 1, limit, a.ctl)))) {
            raise_timeout(a.ctl, t);
            return -1;
          }
        } else if (!(ld_acquire(mc.flags + pa) == 1 && (pb == pa || ld_acquire(mc.flags + pb) == 1))) {
          return 0;
        }
        const int st = j % LP_NSTAGE;
        if ((pending >> st) & 1u) {  // the MMAs that last read this stage must be done
          if (!mbar_wait_bounded(&empty[st], (ph_empty >> st) & 1u)) return -1;
          ph_empty ^= 1u << st;
          pending &= ~(1u << st);
        }
        unsigned char* sa = sStage + st * LP_STAGE_BYTES;
        fence_proxy_async_global();
        mbar_arrive_expect_tx(&full[st], (pb == pa ? 1u : 2u) * LP_OP_BYTES);
        tma_load_1d(sa, mc.tiles16 + size_t(pa) * LP_TILE, LP_OP_BYTES, &full[st]);
        if (pb != pa) tma_load_1d(sa + 2 * LP_OP_BYTES, mc.tiles16 + size_t(pb) * LP_TILE, LP_OP_BYTES, &full[st]);
        return 1;
      };
      for (int it = 0; it < np; ++it) {
        while (issued <= it) {
          const int rc = issue(issued, true);
          if (rc < 0) { aborted = true; break; }
          ++issued;
        }
        if (aborted) break;
        if (issued == it + 1 && issued < np) {
          const int rc = issue(issued, false);
          if (rc < 0) { aborted = true; break; }
          issued += rc;
        }
        const int st = it % LP_NSTAGE;
        if (!mbar_wait_bounded(&full[st], (ph_full >> st) & 1u)) { aborted = true; break; }
        ph_full ^= 1u << st;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int raw = mc.pairs[2 * (tk.pb + it)];
        const int pa = raw & kIndexMask, pb = mc.pairs[2 * (tk.pb + it) + 1];
        const int target = raw >> kTargetShift;
        unsigned char* sa = sStage + st * LP_STAGE_BYTES;
        const uint32_t a_addr = smem_addr(sa), b_addr = smem_addr(pb == pa ? sa : sa + 2 * LP_OP_BYTES);
        const uint32_t dcol = tmem + uint32_t(target) * 64;
#pragma unroll
        for (int ks = 0; ks < LP_B / 16; ++ks) {
          const uint32_t koff = uint32_t(ks) * 2 * 128;  // two core matrices of K per MMA
          umma_f16(dcol, umma_desc(a_addr + koff, kLBO, kSBO), umma_desc(b_addr + koff, kLBO, kSBO), idesc,
                   (used[target] || ks > 0) ? 1u : 0u);
        }
        used[target] = true;
        umma_commit(&empty[st]);
        pending |= 1u << st;
      }
      if (aborted) {
        // a flag timeout happens only while no copy is in flight; MMAs still in
        // flight are tracked by `pending` and waited for before the CTA leaves
        sAbort = 1;
      } else {
        umma_commit(accbar);  // fires once every MMA issued so far has completed
      }
      if (trace) trace[1] = (long long)globaltimer();
      sTicket = (used[0] ? 1 : 0) | (used[1] ? 2 : 0);
    }
    sync();
    if (sAbort) { aborted = true; break; }
    const int used_mask = sTicket;
    if (!mbar_wait_bounded(accbar, ph_acc & 1u)) { aborted = true; break; }
    ph_acc ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue: warps 0-1, one tile row per thread ----
    const int r = tid;  // valid for tid < 64
    float x1[LP_B], x2[LP_B];
    if (warp < 2) {
      // x = A (or 0 for a partial) - D + sum of partial tiles
      const bool from_tile = !(tk.type == TASK_PARTIAL || tk.type == TASK_COMBINE);
#pragma unroll
      for (int c = 0; c < LP_B; ++c) x1[c] = from_tile ? mc.tiles32[size_t(tk.out) * LP_TILE + c * LP_B + r] : 0.f;
      if (chain) {
#pragma unroll
        for (int c = 0; c < LP_B; ++c) x2[c] = mc.tiles32[size_t(tk.out2) * LP_TILE + c * LP_B + r];
      }
      for (int acc = 0; acc < 2; ++acc) {
        if (!((used_mask >> acc) & 1)) continue;
        float v[32];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          tmem_ld32(tmem + (uint32_t(warp * 32) << 16) + uint32_t(acc * 64 + h * 32), v);
          if (acc == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) x1[h * 32 + i] -= v[i];
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) x2[h * 32 + i] -= v[i];
          }
        }
      }
    }
    // partial tiles: acquire their flags (thread 0), then every row adds them
    for (int qi = 0; qi < nq; ++qi) {
      const int raw = mc.parts[tk.qb + qi];
      const int s = raw & kIndexMask;
      if (tid == 0 && !wait_flag(mc.sflags + s, 1, limit, a.ctl)) {
        raise_timeout(a.ctl, t);
        sAbort = 1;
      }
      sync();
      if (sAbort) { aborted = true; break; }
      if (warp < 2) {
        const float* src = mc.scratch + size_t(s) * LP_TILE;
        if ((raw >> kTargetShift) == 0) {
#pragma unroll
          for (int c = 0; c < LP_B; ++c) x1[c] += __ldcg(src + c * LP_B + r);
        } else {
#pragma unroll
          for (int c = 0; c < LP_B; ++c) x2[c] += __ldcg(src + c * LP_B + r);
        }
      }
    }
    if (aborted) break;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");

    if (tk.type == TASK_PARTIAL || tk.type == TASK_COMBINE) {
      if (warp < 2) {
        float* dst = mc.scratch + size_t(tk.out) * LP_TILE;
        // partials hold the negated sum: x1 = -D (+ children), as in the FP64 kernel
#pragma unroll
        for (int c = 0; c < LP_B; ++c) dst[c * LP_B + r] = x1[c];
      }
      publish(mc.sflags + tk.out);
      if (trace && tid == 0) trace[2] = (long long)globaltimer();
      continue;
    }

    if (tk.type == TASK_OFF || chain) {
      // ---- FP32 TRSM: x L_kk^T = s, row by row ----
      if (tid == 0) {
        if (!wait_flag(mc.flags + tk.diag, 1, limit, a.ctl)) {
          raise_timeout(a.ctl, t);
          sAbort = 1;
        } else {
          if (trace) trace[1] = (long long)globaltimer();
          fence_proxy_async_global();
          // L_kk and its 1/L_jj (into sRs, free until the POTRF) in one transaction
          mbar_arrive_expect_tx(lbar, LP_TILE * 4 + LP_B * 4);
          tma_load_1d(sL, mc.tiles32 + size_t(tk.diag) * LP_TILE, LP_TILE * 4, lbar);
          tma_load_1d(sRs, mc.invdiag32 + size_t(tk.col) * LP_B, LP_B * 4, lbar);
        }
      }
      sync();
      if (sAbort) { aborted = true; break; }
      if (!mbar_wait_bounded(lbar, ph_l & 1u)) { aborted = true; break; }
      ph_l ^= 1u;
      if (warp < 2) {
        const float* iv = reinterpret_cast<const float*>(sRs);
#pragma unroll
        for (int j = 0; j < LP_B; ++j) {
          float s = x1[j];
#pragma unroll
          for (int p = 0; p < j; ++p) s = fmaf(-x1[p], sL[j + p * LP_B], s);
          x1[j] = s * iv[j];
        }
        lp_store_row(mc, a.fp16, tk.out, r, x1);
      }
      if (!chain) {
        publish(mc.flags + tk.out);
        if (trace && tid == 0) trace[2] = (long long)globaltimer();
        continue;
      }
      // CHAIN: the SYRK term of the just-solved tile, in FP32 from shared memory
      sync();  // every row finished reading L_kk from sL
      if (warp < 2) {
#pragma unroll
        for (int c = 0; c < LP_B; ++c) sL[c * LP_B + r] = x1[c];
      }
      publish(mc.flags + tk.out);
      if (warp < 2) {
#pragma unroll 8
        for (int p = 0; p < LP_B; ++p) {
          const float xr = sL[r + p * LP_B];
#pragma unroll
          for (int c = 0; c < LP_B; ++c) x2[c] = fmaf(-xr, sL[c + p * LP_B], x2[c]);
        }
#pragma unroll
        for (int c = 0; c < LP_B; ++c) x1[c] = x2[c];
      }
    }

    // ---- FP64 POTRF of the diagonal tile (x1 holds it) ----
    const int out = chain ? tk.out2 : tk.out;
    const int col = chain ? tk.col2 : tk.col;
    if (warp < 2) {
#pragma unroll
      for (int c = 0; c < LP_B; ++c) sD[c * LP_B + r] = double(x1[c]);
    }
    sync();
    {
      // the stage area (every MMA of the task has completed) holds the POTRF's scratch
      const int bad = potrf_blocked<LP_B>(sD, LP_B, sInv, reinterpret_cast<double*>(sStage), lp_sElem16, tid, sync);
      if (bad >= 0 && tid == 0) atomicMin(mc.info, (unsigned long long)col * LP_B + bad + 1);
    }
    if (warp < 2) {
      float* t32 = mc.tiles32 + size_t(out) * LP_TILE;
#pragma unroll
      for (int c = 0; c < LP_B; ++c) t32[c * LP_B + r] = float(sD[c * LP_B + r]);
      mc.ldiag[size_t(col) * LP_B + r] = sD[r * LP_B + r];
      mc.invdiag32[size_t(col) * LP_B + r] = float(sInv[r]);
    }
    publish(mc.flags + out);
    if (trace && tid == 0) trace[2] = (long long)globaltimer();
  }

  // ---- leave: no MMA or copy may still target this slot's memory ----
  if (tid == 0) {
    for (int s = 0; s < LP_NSTAGE; ++s)
      if ((pending >> s) & 1u) mbar_wait_bounded(&empty[s], (ph_empty >> s) & 1u);
  }
}

// Two task slots per CTA: a kernel that allocates tensor memory runs one CTA
// per SM, so each CTA hosts two independent 128-thread slots (two tasks in
// flight per SM).  TMEM: LP_TMEM_COLS columns per slot, allocated once.
__global__ void __launch_bounds__(LP_THREADS) factor_lp_kernel(LPArgs a) {
  __shared__ uint32_t sTmem;
  const int slot = threadIdx.x >> 7, tid = threadIdx.x & 127;
  init_df_elements<16>(lp_sElem16, threadIdx.x, LP_THREADS);
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sTmem)),
                 "r"(LP_SLOTS * LP_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  static_assert(LP_SLOTS == 2, "one lp_slot instantiation per slot");
  if (slot == 0)
    lp_slot<0>(a, sTmem, tid);
  else
    lp_slot<1>(a, sTmem + LP_TMEM_COLS, tid);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sTmem), "r"(LP_SLOTS * LP_TMEM_COLS));
}

}  // namespace dev
}  // namespace stiles
