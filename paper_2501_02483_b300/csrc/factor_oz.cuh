// Persistent tile Cholesky with FP64-accurate tile updates on the tcgen05
// tensor cores (BF16 digit slices, exact FP32 accumulation in tensor memory).
//
// Algorithm 1 needs L_mk -= sum_n L_mn L_kn^T and A_kk -= sum_n L_kn L_kn^T in
// FP64.  Here every finished off-diagonal tile is also stored as four BF16
// digit slices: with a power-of-two scale 2^e_i per matrix row i, chosen so
// that |L_ij| < 2^e_i for every entry of the row (e_i from the original
// diagonal: sum_j L_ij^2 = a_ii, so |L_ij| <= sqrt(a_ii) < 2^e_i),
//     L_ij 2^-e_i = d0 2^-8 + d1 2^-16 + d2 2^-24 + d3 2^-32 + r,   |r| <= 2^-33,
// with integer digits |d0| <= 256, |d1|, |d2|, |d3| <= 128, each exact in
// BF16.  (The splitting of floating-point products into exact low-precision
// pieces follows Ozaki, Ogita and Oishi, 2012, and Ootomo, Ozaki and Yokota,
// 2024, for integer/low-precision tensor cores.)  The product of two tiles is
// then sum over slice pairs (s, t) of D_st = d_s(L_mn) d_t(L_kn)^T times
// 2^(e_i + e_c - 8 (s + t + 2)); each D_st is a sum of integer products and is
// exact in the FP32 accumulator:
//   - s = t = 0: by Cauchy-Schwarz over the whole row pair,
//     sum_j |d0_ij d0_cj| <~ 2^16 sqrt(a_ii a_cc) / 2^(e_i + e_c) < 2^16;
//   - other pairs: at most 2^15 sqrt(K) or K 2^14 in magnitude for K inner
//     terms, below 2^24 for the band widths here (and a level s + t >= 2 that
//     rounded would only perturb the result at 2^-40).
// The slices are stacked as one 128-row MMA operand (4 slices x 32 rows), so a
// tile pair costs four M = 128, N = 32, K = 32 MMAs (one per slice t of the
// second tile), and TMEM holds, for every slice pair, its own 32 x 32 block:
// lanes 32 s .. 32 s + 31, columns 32 t .. 32 t + 31 of the target's 128.  The
// epilogue reads them back, combines the 16 products exactly in 64-bit
// integers (V = sum D_st 2^(8 (3 - s - t)), the levels below 2^-40 rounded),
// and applies V 2^(e_i + e_c - 40) to the FP64 target: the update is exact up
// to the slices' representation error, 2^-33 of the row scales (a backward
// error of ~2^-32 sqrt(a_ii a_cc) per entry of A), far below what 16-bit
// updates give (2^-8 / 2^-11).
//
// Everything else is FP64 as in the FP64 kernel: tiles, tree partials, the
// diagonal POTRF (potrf_blocked) and the TRSM of off-diagonal tiles (rows
// against L_kk with pre-scaled columns).  The CHAIN task's SYRK term of the
// tile it just solved goes through the same slices (from shared memory) into
// the diagonal target's TMEM blocks: on this GPU an FP64 warp instruction
// (DFMA or DMMA) holds its sub-partition's FP64 pipe for 64 cycles, so the
// 32 x 32 x 32 SYRK costs ~7 us on the FP64 path against ~1 us of MMAs.
// The factor is an FP64 factor: log-determinant, solves and the selected
// inverse use it as they use the FP64 kernel's.
//
// Tiles are B = 32; two independent 128-thread task slots per CTA (a kernel
// that allocates TMEM runs one CTA per SM), each with its own stages,
// mbarriers, named barrier and 256 TMEM columns (two targets of a CHAIN task).
#pragma once

#include "device_common.cuh"
#include "factor_f64.cuh"
#include "factor_lp.cuh"
#include "plan.h"

namespace stiles {
namespace dev {

constexpr int OZ_B = 32;
constexpr int OZ_TILE = OZ_B * OZ_B;
constexpr int OZ_NSLICE = 4;
constexpr uint32_t OZ_SLICE_BYTES = OZ_TILE * 2;                // one 32 x 32 BF16 digit slice
constexpr uint32_t OZ_OP_BYTES = OZ_NSLICE * OZ_SLICE_BYTES;    // the four slices of a tile (8 KB)
constexpr int OZ_NSTAGE = 3;
constexpr uint32_t OZ_STAGE_BYTES = 2 * OZ_OP_BYTES;            // both operands of a pair
constexpr uint32_t OZ_TMEM_COLS = 256;                          // per slot: 2 targets x 4 x 32 columns
constexpr int OZ_SLOTS = 2;
constexpr int OZ_THREADS = 128 * OZ_SLOTS;
constexpr int OZ_SCALE_SHIFT = 40;                              // V is in units of 2^(e_i + e_c - 40)

// shared memory of one slot: stages (also the 64-bit reduction buffer and the
// POTRF's scratch) | sD, sL (FP64 32 x 32) | sSl (slices of a tile, 8 KB) |
// sInvL, sInv, sPiv, sRs (FP64 x 32) | sExpR, sExpC (int x 32) | barriers
constexpr size_t OZ_SMEM = size_t(OZ_NSTAGE) * OZ_STAGE_BYTES + 2 * OZ_TILE * 8 + OZ_OP_BYTES + 4 * OZ_B * 8 +
                           2 * OZ_B * 4 + (OZ_NSTAGE * 2 + 3) * 8 + 64;
constexpr size_t OZ_SLOT_BYTES = (OZ_SMEM + 1023) / 1024 * 1024;
constexpr size_t OZ_KERNEL_SMEM = OZ_SLOTS * OZ_SLOT_BYTES;
static_assert(size_t(OZ_NSTAGE) * OZ_STAGE_BYTES >= 4 * OZ_TILE * 8, "reduction buffer fits in the stages");

struct OZMatCtx {
  double* tiles;         // nsub * 32 * 32, column-major (A, then L)
  uint16_t* slices;      // nsub * 4 * 32 * 32: BF16 digit slices of every finished off-diagonal tile,
                         // core-matrix layout, slice s at s * 2 KB
  double* scratch;       // tree partials (negated sums), FP64 column-major
  double* invdiag;       // nsb * 32: 1 / L_jj
  const int* rowexp;     // nsb * 32: e_i of every (padded) row
  const DevTask* tasks;
  const int32_t* pairs;
  const int32_t* parts;
  int* flags;
  int* sflags;
  unsigned long long* info;
  long long* trace;
};

struct OZArgs {
  OZMatCtx single;       // the matrix of a one-matrix launch (mats == NULL)
  const OZMatCtx* mats;  // batched launch: one context per matrix (device memory)
  const int2* tickets;   // batched launch: (matrix, task) per ticket; NULL: one matrix
  int ntasks;
  Ctl* ctl;
  long long spin_limit;
  // Optional split of a one-matrix launch (as in the FP64 kernel): the diagonal
  // chain (DIAG and CHAIN tasks, `chain`) runs on slot 0 of the CTAs on the first
  // chain_sms SMs, alone on its SM (slot 1 there takes no work), so its FP64
  // TRSM and POTRF have the SM's FP64 pipes to themselves; every other task
  // (`bulk`) runs on the other SMs.  Both lists follow the one topological
  // ticket order.  chain_sms == 0: one queue, ticket = task.
  const int32_t* chain;
  const int32_t* bulk;
  int nchain, nbulk;
  int chain_sms;
  int* sm_claim;  // [chain_sms], zeroed per launch
};

// byte offset of element (r, k) of a 32-wide K-major core-matrix operand
__device__ __forceinline__ uint32_t oz_core_offset(int r, int k) {
  return uint32_t(((r >> 3) * (OZ_B / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ double oz_pow2(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// round(x 2^(32 - e)) as an integer (|x| < 2^e), from the bit pattern alone
// (integer pipes only); 0 for zeros, subnormals and anything at or above 2^e.
__device__ __forceinline__ long long oz_fixed32(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int ef = int((bits >> 52) & 0x7ff);
  const int sh = (e + 20 + 1023) - ef;  // right shift of the 53-bit significand
  if (ef == 0 || sh <= 0) return 0;
  if (sh >= 62) return 0;
  const long long mant = (bits & 0x000fffffffffffffLL) | (1LL << 52);
  const long long v = (mant + (1LL << (sh - 1))) >> sh;
  return bits < 0 ? -v : v;
}

// The four balanced base-256 digits of X (|X| <= 2^32): X = d0 2^24 + d1 2^16 + d2 2^8 + d3,
// as BF16 bit patterns (the digits are integers of magnitude <= 256, exact in BF16).
__device__ __forceinline__ void oz_digits(long long X, uint16_t (&d)[4]) {
  int r[4];
  long long v = X;
#pragma unroll
  for (int s = 3; s >= 1; --s) {
    const int lo = int(((v + 128) & 255) - 128);
    r[s] = lo;
    v = (v - lo) >> 8;
  }
  r[0] = int(v);
#pragma unroll
  for (int s = 0; s < 4; ++s) d[s] = uint16_t(__float_as_uint(float(r[s])) >> 16);
}

// role: 0 the single queue, 1 the chain queue, 2 the bulk queue, -1 no work
template <int SLOT>
__device__ __forceinline__ void oz_slot(const OZArgs& a, uint32_t tmem, int tid, int role) {
  using Cfg = FactorCfg<OZ_B>;
  constexpr int RPT = Cfg::RPT, CPT = Cfg::CPT;
  extern __shared__ __align__(1024) unsigned char oz_dyn[];
  __shared__ int sTicket, sAbort;  // one pair per instantiation, i.e. per slot
  __shared__ uint16_t sElem16[PotrfDf<16>::NLIVE];
  unsigned char* smem_raw = oz_dyn + SLOT * OZ_SLOT_BYTES;
  __builtin_assume(tid >= 0 && tid < 128);
  auto sync = []() { asm volatile("bar.sync %0, 128;" ::"n"(1 + SLOT) : "memory"); };
  auto publish = [&](int* flag) {
    sync();
    if (tid == 0) st_release(flag, 1);
  };
  unsigned char* sStage = smem_raw;
  long long* sV = reinterpret_cast<long long*>(sStage);          // [4 warps][32 columns][32 rows]
  double* sD = reinterpret_cast<double*>(sStage + OZ_NSTAGE * OZ_STAGE_BYTES);
  double* sL = sD + OZ_TILE;
  unsigned char* sSl = reinterpret_cast<unsigned char*>(sL + OZ_TILE);
  double* sInvL = reinterpret_cast<double*>(sSl + OZ_OP_BYTES);  // TMA target (16-byte aligned)
  double* sInv = sInvL + OZ_B;
  double* sPiv = sInv + OZ_B;
  double* sRs = sPiv + OZ_B;
  int* sExpR = reinterpret_cast<int*>(sRs + OZ_B);
  int* sExpC = sExpR + OZ_B;
  uint64_t* full = reinterpret_cast<uint64_t*>(sExpC + OZ_B);  // [OZ_NSTAGE] operands landed
  uint64_t* empty = full + OZ_NSTAGE;                           // [OZ_NSTAGE] MMAs done with the stage
  uint64_t* accbar = empty + OZ_NSTAGE;                         // every MMA of the task done
  uint64_t* lbar = accbar + 1;                                  // L_kk landed
  uint64_t* sbar = lbar + 1;                                    // the CHAIN's SYRK MMAs done
  const int warp = tid >> 5, lane = tid & 31;
  const int row = tid / RPT, q = tid % RPT;
  const int row_lane0 = lane - (lane % RPT);
  init_df_elements<16>(sElem16, tid, 128);
  if (tid == 0) {
    for (int s = 0; s < OZ_NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accbar, 1);
    mbar_init(lbar, 1);
    mbar_init(sbar, 1);
    mbar_fence_init();
  }
  sync();
  const long long limit = a.spin_limit;
  // kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = 32, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(32 >> 3) << 17) | (uint32_t(128 >> 4) << 24);
  const uint32_t kLBO = 128, kSBO = (OZ_B / 8) * 128;
  uint32_t ph_full = 0, ph_empty = 0, ph_acc = 0, ph_l = 0, ph_s = 0;
  uint32_t pending = 0;  // stage s has committed MMAs not yet waited on (thread 0 only)

  // the 16 slice products of one operand pair (stacked A slices x each B slice)
  auto issue_mmas = [&](uint32_t a_addr, uint32_t b_addr, uint32_t dcol, bool acc_in) {
#pragma unroll
    for (int t = 0; t < OZ_NSLICE; ++t)
#pragma unroll
      for (int ks = 0; ks < OZ_B / 16; ++ks) {
        const uint32_t koff = uint32_t(ks) * 2 * 128;
        umma_f16(dcol + uint32_t(t) * 32, umma_desc(a_addr + koff, kLBO, kSBO),
                 umma_desc(b_addr + uint32_t(t) * OZ_SLICE_BYTES + koff, kLBO, kSBO), idesc,
                 (acc_in || ks > 0) ? 1u : 0u);
      }
  };

  // V = sum over slice pairs of the target's TMEM blocks, exact in 64-bit
  // integers, reduced over the four lane groups through sV, then applied to
  // the FP64 accumulator (row, q + RPT m) with the scales of sExpR / sExpC.
  auto apply_tmem = [&](uint32_t tcol, double (&acc)[CPT]) {
    long long V[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) V[c] = 0;
#pragma unroll
    for (int t = 0; t < OZ_NSLICE; ++t) {
      float v[32];
      tmem_ld32(tmem + (uint32_t(warp * 32) << 16) + tcol + uint32_t(t) * 32, v);
      const int sh = 8 * (3 - warp - t);  // this warp holds the slice pairs (s = warp, t)
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const long long x = (long long)__float2int_rn(v[c]);
        V[c] += sh >= 0 ? (x << sh) : ((x + (1LL << (-sh - 1))) >> (-sh));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) sV[(warp * 32 + c) * 32 + lane] = V[c];
    sync();
    const int er = sExpR[row];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int c = q + RPT * m;
      const long long s = sV[(0 * 32 + c) * 32 + row] + sV[(1 * 32 + c) * 32 + row] +
                          sV[(2 * 32 + c) * 32 + row] + sV[(3 * 32 + c) * 32 + row];
      acc[m] = fma(-double(s), oz_pow2(er + sExpC[c] - OZ_SCALE_SHIFT), acc[m]);
    }
    sync();  // sV free again
  };

  // Slices of the finished tile held in acc (row, q + RPT m), row scales sExpR,
  // into sSl, then copied to the tile's slice array.
  auto make_slices = [&](const double (&acc)[CPT], uint16_t* gsl) {
    const int er = sExpR[row];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int c = q + RPT * m;
      uint16_t d[4];
      oz_digits(oz_fixed32(acc[m], er), d);
      const uint32_t off = oz_core_offset(row, c);
#pragma unroll
      for (int s = 0; s < 4; ++s) *reinterpret_cast<uint16_t*>(sSl + s * OZ_SLICE_BYTES + off) = d[s];
    }
    fence_proxy_async_shared();  // the CHAIN's SYRK MMAs read sSl through the async proxy
    sync();
    const uint4* src = reinterpret_cast<const uint4*>(sSl);
    uint4* dst = reinterpret_cast<uint4*>(gsl);
#pragma unroll
    for (int i = 0; i < int(OZ_OP_BYTES / 16 / 128); ++i) dst[tid + 128 * i] = src[tid + 128 * i];
  };

  auto load_exps = [&](const OZMatCtx& mc, int rblk, int cblk) {
    if (rblk < 0 || cblk < 0) return;
    if (tid < OZ_B) sExpR[tid] = mc.rowexp[size_t(rblk) * OZ_B + tid];
    else if (tid < 2 * OZ_B) sExpC[tid - OZ_B] = mc.rowexp[size_t(cblk) * OZ_B + tid - OZ_B];
  };

  int* const counter = (role == 1) ? &a.ctl->ticket2 : &a.ctl->ticket;
  const int nqueue = (role == 1) ? a.nchain : (role == 2 ? a.nbulk : (role == 0 ? a.ntasks : 0));
  int next = 0;
  if (tid == 0 && nqueue > 0) next = atomicAdd(counter, 1);
  bool aborted = false;
  while (!aborted) {
    fence_proxy_async_shared();
    if (tid == 0) {
      int cur = next;
      if (cur < nqueue && ld_volatile(&a.ctl->abort) == 0) next = atomicAdd(counter, 1);
      else cur = -1;
      sTicket = cur;
      sAbort = 0;
    }
    sync();
    const int t0 = sTicket;
    if (t0 < 0) break;
    const int t = (role == 1) ? a.chain[t0] : (role == 2 ? a.bulk[t0] : t0);  // task index (one matrix)
    int mi = 0, ti = t;
    if (a.tickets) {
      const int2 v = a.tickets[t];
      mi = v.x;
      ti = v.y;
    }
    const OZMatCtx mc = a.mats ? a.mats[mi] : a.single;
    const DevTask tk = mc.tasks[ti];
    long long* const trace = mc.trace ? mc.trace + 4 * size_t(ti) : nullptr;
    if (trace && tid == 0) {
      trace[0] = (long long)globaltimer();
      trace[3] = smid();
    }
    const bool chain = tk.type == TASK_CHAIN;
    const bool tree = tk.type == TASK_PARTIAL || tk.type == TASK_COMBINE;
    const int np = tk.pe - tk.pb, nq = tk.qe - tk.qb;
    load_exps(mc, tk.trow, tk.tcol);

    // ---- producer / MMA issuer: thread 0 ----
    bool used[2] = {false, false};
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
        const int st = j % OZ_NSTAGE;
        if ((pending >> st) & 1u) {
          if (!mbar_wait_bounded(&empty[st], (ph_empty >> st) & 1u)) return -1;
          ph_empty ^= 1u << st;
          pending &= ~(1u << st);
        }
        unsigned char* sa = sStage + st * OZ_STAGE_BYTES;
        fence_proxy_async_global();
        mbar_arrive_expect_tx(&full[st], (pb == pa ? 1u : 2u) * OZ_OP_BYTES);
        tma_load_1d(sa, mc.slices + size_t(pa) * (OZ_OP_BYTES / 2), OZ_OP_BYTES, &full[st]);
        if (pb != pa) tma_load_1d(sa + OZ_OP_BYTES, mc.slices + size_t(pb) * (OZ_OP_BYTES / 2), OZ_OP_BYTES, &full[st]);
        return 1;
      };
      for (int it = 0; it < np; ++it) {
        while (issued <= it) {
          const int rc = issue(issued, true);
          if (rc < 0) { aborted = true; break; }
          ++issued;
        }
        if (aborted) break;
        while (issued < np && issued < it + OZ_NSTAGE) {
          const int rc = issue(issued, false);
          if (rc < 0) { aborted = true; break; }
          if (rc == 0) break;
          ++issued;
        }
        if (aborted) break;
        const int st = it % OZ_NSTAGE;
        if (!mbar_wait_bounded(&full[st], (ph_full >> st) & 1u)) { aborted = true; break; }
        ph_full ^= 1u << st;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int raw = mc.pairs[2 * (tk.pb + it)];
        const int pa = raw & kIndexMask, pb = mc.pairs[2 * (tk.pb + it) + 1];
        const int target = raw >> kTargetShift;
        unsigned char* sa = sStage + st * OZ_STAGE_BYTES;
        issue_mmas(smem_addr(sa), smem_addr(pb == pa ? sa : sa + OZ_OP_BYTES), tmem + uint32_t(target) * 128,
                   used[target]);
        used[target] = true;
        umma_commit(&empty[st]);
        pending |= 1u << st;
      }
      if (aborted) {
        // a flag wait runs only when every issued copy has been consumed; MMAs
        // still in flight are tracked by `pending` and waited for before the slot leaves
        sAbort = 1;
      } else {
        umma_commit(accbar);
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

    // ---- epilogue: FP64 accumulators in the (row, q + RPT m) layout ----
    double acc1[CPT], acc2[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      acc1[m] = tree ? 0.0 : mc.tiles[size_t(tk.out) * OZ_TILE + (q + RPT * m) * OZ_B + row];
      acc2[m] = chain ? mc.tiles[size_t(tk.out2) * OZ_TILE + (q + RPT * m) * OZ_B + row] : 0.0;
    }
    if (used_mask & 1) apply_tmem(0, acc1);
    // tree partials (negated sums) of both targets: every flag polled together
    // (relaxed loads in flight, one acquire fence), then all loads issued
    // before the sums, two partials at a time
    if (nq > 0) {
      if (tid == 0 &&
          !wait_flags([&](int i) { return mc.sflags + (mc.parts[tk.qb + i] & kIndexMask); }, nq, limit, a.ctl)) {
        raise_timeout(a.ctl, t);
        sAbort = 1;
      }
      sync();
      if (sAbort) { aborted = true; break; }
      for (int qi = 0; qi < nq; qi += 2) {
        const int r0 = mc.parts[tk.qb + qi];
        const int r1 = (qi + 1 < nq) ? mc.parts[tk.qb + qi + 1] : -1;
        const double* s0 = mc.scratch + size_t(r0 & kIndexMask) * OZ_TILE;
        const double* s1 = mc.scratch + size_t(r1 < 0 ? 0 : (r1 & kIndexMask)) * OZ_TILE;
        double v0[CPT], v1[CPT];
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
          v0[m] = __ldcg(s0 + (q + RPT * m) * OZ_B + row);
          v1[m] = r1 < 0 ? 0.0 : __ldcg(s1 + (q + RPT * m) * OZ_B + row);
        }
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
          if ((r0 >> kTargetShift) == 0) acc1[m] += v0[m];
          else acc2[m] += v0[m];
          if (r1 >= 0) {
            if ((r1 >> kTargetShift) == 0) acc1[m] += v1[m];
            else acc2[m] += v1[m];
          }
        }
      }
    }

    if (tree) {
      double* dst = mc.scratch + size_t(tk.out) * OZ_TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * OZ_B + row] = acc1[m];
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      publish(mc.sflags + tk.out);
      if (trace && tid == 0) trace[2] = (long long)globaltimer();
      continue;
    }

    if (tk.type == TASK_OFF || chain) {
      // ---- FP64 TRSM: x L_kk^T = acc1, rows against L_kk with pre-scaled columns ----
      if (tid == 0) {
        if (!wait_flag(mc.flags + tk.diag, 1, limit, a.ctl)) {
          raise_timeout(a.ctl, t);
          sAbort = 1;
        } else {
          fence_proxy_async_global();
          mbar_arrive_expect_tx(lbar, uint32_t((OZ_TILE + OZ_B) * sizeof(double)));
          tma_load_1d(sL, mc.tiles + size_t(tk.diag) * OZ_TILE, OZ_TILE * sizeof(double), lbar);
          tma_load_1d(sInvL, mc.invdiag + size_t(tk.col) * OZ_B, OZ_B * sizeof(double), lbar);
        }
      }
      sync();
      if (sAbort) { aborted = true; break; }
      if (!mbar_wait_bounded(lbar, ph_l & 1u)) { aborted = true; break; }
      ph_l ^= 1u;
      double inv[CPT];
#pragma unroll
      for (int m = 0; m < CPT; ++m) inv[m] = sInvL[q + RPT * m];
      for (int e = tid; e < OZ_TILE; e += 128) {
        const int c = e % OZ_B, j = e / OZ_B;
        if (c > j) sL[e] *= sInvL[j];
      }
      sync();
      trsm_rows<OZ_B>(acc1, inv, sL, q, row_lane0);
      {
        double* dst = mc.tiles + size_t(tk.out) * OZ_TILE;
#pragma unroll
        for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * OZ_B + row] = acc1[m];
      }
      make_slices(acc1, mc.slices + size_t(tk.out) * (OZ_OP_BYTES / 2));
      if (!chain) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        publish(mc.flags + tk.out);
        if (trace && tid == 0) trace[2] = (long long)globaltimer();
        continue;
      }
      publish(mc.flags + tk.out);
      // CHAIN: the SYRK term L_{k,k-1} L_{k,k-1}^T from the slices in sSl into
      // the diagonal target's TMEM blocks (rows and columns of block k), on top
      // of the target's pair terms
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_mmas(smem_addr(sSl), smem_addr(sSl), tmem + 128u, (used_mask & 2) != 0);
        umma_commit(sbar);
      }
      if (tid < OZ_B) sExpC[tid] = mc.rowexp[size_t(tk.col2) * OZ_B + tid];  // rows: block k already
      if (!mbar_wait_bounded(sbar, ph_s & 1u)) { aborted = true; break; }
      ph_s ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      apply_tmem(128u, acc2);  // reads sExpC after its first barrier
#pragma unroll
      for (int m = 0; m < CPT; ++m) acc1[m] = acc2[m];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");

    // ---- FP64 POTRF of the diagonal tile (acc1 holds it) ----
    const int out = chain ? tk.out2 : tk.out;
    const int col = chain ? tk.col2 : tk.col;
#pragma unroll
    for (int m = 0; m < CPT; ++m) sD[(q + RPT * m) * OZ_B + row] = acc1[m];
    sync();
    {
      const int bad = potrf_blocked<OZ_B>(sD, OZ_B, sInv, reinterpret_cast<double*>(sStage), sElem16, tid, sync);
      if (bad >= 0 && tid == 0) atomicMin(mc.info, (unsigned long long)col * OZ_B + bad + 1);
    }
    {
      double* dst = mc.tiles + size_t(out) * OZ_TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * OZ_B + row] = sD[(q + RPT * m) * OZ_B + row];
      if (tid < OZ_B) mc.invdiag[size_t(col) * OZ_B + tid] = sInv[tid];
    }
    publish(mc.flags + out);
    if (trace && tid == 0) trace[2] = (long long)globaltimer();
  }

  // ---- leave: no MMA or copy may still target this slot's memory ----
  if (tid == 0) {
    for (int s = 0; s < OZ_NSTAGE; ++s)
      if ((pending >> s) & 1u) mbar_wait_bounded(&empty[s], (ph_empty >> s) & 1u);
  }
}

__global__ void __launch_bounds__(OZ_THREADS, 1) factor_oz_kernel(OZArgs a) {
  __shared__ uint32_t sTmem;
  const int slot = threadIdx.x >> 7, tid = threadIdx.x & 127;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sTmem)),
                 "r"(OZ_SLOTS * OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // queue of each slot: the single ticket order, or (split launch) the chain
  // queue for slot 0 of the first CTA on each reserved SM (slot 1 there and
  // any other CTA on a reserved SM take no work), the bulk queue elsewhere
  __shared__ int sRole;
  if (threadIdx.x == 0) {
    int role = 0;
    if (a.chain_sms > 0) {
      const int sm = smid();
      role = (sm < a.chain_sms) ? ((atomicAdd(a.sm_claim + sm, 1) == 0) ? 1 : -1) : 2;
    }
    sRole = role;
  }
  __syncthreads();
  const int role = sRole;
  static_assert(OZ_SLOTS == 2, "one oz_slot instantiation per slot");
  if (slot == 0)
    oz_slot<0>(a, sTmem, tid, role);
  else
    oz_slot<1>(a, sTmem + OZ_TMEM_COLS, tid, role == 1 ? -1 : role);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sTmem), "r"(OZ_SLOTS * OZ_TMEM_COLS));
}

// e_i of every padded row from the original diagonal a_ii (the scattered tiles):
// the smallest e with 2^(2e) > a_ii, i.e. ceil((E + 1) / 2) for a_ii in [2^E, 2^(E+1));
// 0 when a_ii is not a positive normal number (the POTRF reports that matrix).
__global__ void oz_rowexp_kernel(const double* tiles, const int32_t* diag_sub, int64_t nsb, int* rowexp) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= nsb * OZ_B) return;
  const int64_t k = g / OZ_B;
  const int r = int(g % OZ_B);
  const double v = tiles[size_t(diag_sub[k]) * OZ_TILE + size_t(r) * (OZ_B + 1)];
  const long long b = __double_as_longlong(v);
  int e = 0;
  if (b >= (1LL << 52) && b < (2047LL << 52)) {
    const int E = int(b >> 52) - 1023;
    e = (E + 2) >> 1;
  }
  rowexp[g] = e;
}

// batched form: descriptor per matrix (blockIdx.y)
struct OZRowexpDesc {
  const double* tiles;
  const int32_t* diag_sub;
  int64_t nsb;
  int* rowexp;
};
__global__ void oz_browexp_kernel(const OZRowexpDesc* d) {
  const OZRowexpDesc m = d[blockIdx.y];
  for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < m.nsb * OZ_B;
       g += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = g / OZ_B;
    const int r = int(g % OZ_B);
    const double v = m.tiles[size_t(m.diag_sub[k]) * OZ_TILE + size_t(r) * (OZ_B + 1)];
    const long long b = __double_as_longlong(v);
    int e = 0;
    if (b >= (1LL << 52) && b < (2047LL << 52)) e = (int(b >> 52) - 1023 + 2) >> 1;
    m.rowexp[g] = e;
  }
}

}  // namespace dev
}  // namespace stiles
