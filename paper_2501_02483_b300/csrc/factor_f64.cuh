// Persistent FP64 tile Cholesky (Algorithm 1, left-looking, on B x B sub-tiles).
//
// One launch runs the whole factorization.  Each CTA repeatedly takes the next
// ticket of a topologically ordered task list (the device analogue of the
// static scheduler's task table, Algorithm 2) and executes it:
//
//   DIAG     A_kk -= sum L_kn L_kn^T (+ tree partials), then POTRF
//   OFF      A_mk -= sum L_mn L_kn^T (+ tree partials), then TRSM with L_kk
//   CHAIN    OFF(k, k-1) and DIAG(k) together: TRSM of (k, k-1), publish it,
//            apply its SYRK term to (k, k) from shared memory, POTRF(k)
//   PARTIAL  S = -sum of a chunk of L_an L_bn^T       (tree leaf, Algorithm 3)
//   COMBINE  S = sum of child partials                 (tree node, GEADD)
//
// Dependencies are per-tile ready flags (the progress table of Algorithm 2)
// read with acquire loads; waits are bounded and end the launch with
// STILES_ERR_TIMEOUT instead of hanging.  Operand tiles are contiguous in HBM
// (CTSF) and are staged into shared memory by 1-D TMA bulk copies, NSTAGE
// pairs in flight.  The accumulator lives in registers: thread (i, q) owns row
// i and the columns q, q + RPT, q + 2 RPT, ... of the output tile.
#pragma once

#include <type_traits>

#include "device_common.cuh"
#include "plan.h"

namespace stiles {
namespace dev {

template <int B>
struct FactorCfg {
  static constexpr int NT = 128;
  static constexpr int RPT = NT / B;  // threads per tile row
  static constexpr int CPT = B / RPT; // columns per thread
  static constexpr int TILE = B * B;
  static constexpr int NSTAGE = (B == 64) ? 2 : 3;
  // stages | sC | sL | sInv, sPiv, sRs, sK (B ints in B doubles), sInvL (B each; sInvL is a TMA target)
  static constexpr size_t SMEM_DOUBLES = size_t(NSTAGE) * 2 * TILE + 2 * TILE + 5 * B;
  static constexpr size_t SMEM = SMEM_DOUBLES * sizeof(double) + (NSTAGE + 1) * sizeof(uint64_t) + 16;
};

// Bit 30 of a pair's first index / of a partial index selects the accumulator
// of a CHAIN task (0: the off-diagonal tile, 1: the diagonal tile).
constexpr int kTargetShift = 30;
constexpr int kIndexMask = (1 << 30) - 1;

// One matrix of a launch (a batched launch carries one per matrix).
struct MatCtx {
  double* tiles;    // nsub * B * B, sub-tile s at s * B * B, column-major
  double* scratch;  // nscratch * B * B (tree partials, stored negated)
  double* invdiag;  // nsb * B: 1 / L_jj of each diagonal sub-tile
  const DevTask* tasks;
  const int32_t* pairs;
  const int32_t* parts;
  int* flags;   // per sub-tile: 1 when final
  int* sflags;  // per scratch tile: 1 when final
  unsigned long long* info;  // first bad pivot column of this matrix (atomicMin)
  long long* trace;          // optional, 4 per task: start, dependencies ready, done, SM id
};

struct FactorArgs {
  MatCtx single;        // the matrix of a one-matrix launch (mats == NULL)
  const MatCtx* mats;   // batched launch: one context per matrix (device memory)
  const int2* tickets;  // batched launch: (matrix, task) per ticket; NULL: one matrix, ticket = task
  int ntasks;           // tickets in the launch
  Ctl* ctl;             // ticket counters, timeout status, abort flag of the launch
  long long spin_limit;
  // Optional split of a one-matrix launch into two queues: the diagonal chain
  // (DIAG and CHAIN tasks, `chain`) runs on `chain_sms` reserved SMs, one CTA
  // each; every other task (`bulk`) on the remaining SMs.  Both lists follow
  // the one topological ticket order, so each queue's first unfinished task
  // always has its inputs produced or in progress: no deadlock while each
  // queue keeps a CTA.  chain_sms == 0: one queue, ticket = task.
  const int32_t* chain;
  const int32_t* bulk;
  int nchain, nbulk;
  int chain_sms;
  int* sm_claim;        // [chain_sms], zeroed per launch: first CTA on a reserved SM takes the chain
};

// All threads have stored the tile; after the barrier, thread 0's release
// store makes the whole CTA's writes visible to any thread that acquires the
// flag (release cumulativity through bar.sync).
__device__ __forceinline__ void publish(int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) st_release(flag, 1);
}

template <int B>
struct PotrfDf {
  static constexpr int NLIVE = B * (B - 1) / 2;
  static constexpr int NE = (NLIVE + 127) / 128;  // elements per thread
};

template <int B>
__device__ __forceinline__ void init_df_elements(uint16_t* sElem, int tid, int nthreads) {
  for (int t = tid; t < PotrfDf<B>::NLIVE; t += nthreads) {
    int c = 1, off = 0;
    while (off + (B - c) <= t) {
      off += B - c;
      ++c;
    }
    sElem[t] = uint16_t(((c + t - off) << 8) | c);
  }
}

// POTRF of a B x B FP64 tile (B <= 32), division-free on the dependency chain.
//
// Right-looking elimination scaled so that no division is needed until the
// end: with the pivot a_jj = m_j 2^e_j (m_j in [1, 2)), step j replaces every
// trailing element (diagonal included) by
//     a_ic <- m_j a_ic - (a_ij 2^-e_j) a_cj          (j < c <= i),
// i.e. 2^-e_j (a_jj a_ic - a_ij a_cj): the trailing matrix stays the Schur
// complement times sigma_{j+1} = m_0 ... m_j, which grows by less than 2 per
// step.  A step is two multiplies and one FMA per element, with no reciprocal
// on the chain; at the end
//     L_ic = a_ic / sqrt(sigma_c a_cc),   L_cc = sqrt(a_cc / sigma_c).
// Beforehand the tile is equilibrated by powers of two, a_ic 2^-(k_i + k_c)
// with k_i = floor(log2(a_ii) / 2) (exact), so that the products stay in range
// whatever the tile's scale; L is scaled back by 2^k_i at the end.
//
// Every thread holds its elements (sElem) in registers and publishes an
// element to sC when it becomes final (column j+1 after step j; a diagonal one
// also as the next pivot, sPiv).  One barrier per step; every thread reads
// pivot j after the barrier that follows its publication and stops at the
// first bad one (not a positive normal number below 2^1022).  Returns that
// pivot (the tile is then NaN) or -1; sInv receives 1/L_jj.  Shared scratch:
// sC (B x B), sPiv, sRs, sInv (B each), sK (B ints), sElem.
template <int B, class Sync>
__device__ __forceinline__ int potrf_tile_df(double (&acc)[FactorCfg<B>::CPT], double* sC, double* sPiv,
                                             double* sInv, double* sRs, int* sK, const uint16_t* sElem, int row,
                                             int q, int tid, Sync sync) {
  static_assert(B <= 32, "one warp scans the pivots");
  constexpr int RPT = FactorCfg<B>::RPT, CPT = FactorCfg<B>::CPT;
  constexpr int NE = PotrfDf<B>::NE, NLIVE = PotrfDf<B>::NLIVE;
  auto pow2 = [](int e) { return __longlong_as_double((long long)(1023 + e) << 52); };  // 2^e, |e| <= 1022
  auto pivot_ok = [](double v) {
    const long long b = __double_as_longlong(v);
    return b >= (1LL << 52) && b < (2046LL << 52);
  };
#pragma unroll
  for (int m = 0; m < CPT; ++m) sC[(q + RPT * m) * B + row] = acc[m];
  sync();
  if (tid < B) {  // equilibration exponents
    const double v = sC[tid * (B + 1)];
    sK[tid] = pivot_ok(v) ? ((int(__double_as_longlong(v) >> 52) - 1023) >> 1) : 0;
  }
  sync();
  double a[NE];
  int ei[NE], ec[NE];
#pragma unroll
  for (int u = 0; u < NE; ++u) {
    const int t = tid + 128 * u;
    ei[u] = 0;
    ec[u] = B;  // no element: never live
    a[u] = 0.0;
    if (t < NLIVE) {
      const int v = sElem[t];
      ei[u] = v >> 8;
      ec[u] = v & 255;
      a[u] = sC[ei[u] + ec[u] * B] * pow2(-(sK[ei[u]] + sK[ec[u]]));
    }
  }
  if (tid < B) {  // column 0 is final from the start
    const double v = sC[tid] * pow2(-(sK[tid] + sK[0]));
    sC[tid] = v;
    if (tid == 0) sPiv[0] = v;
  }
  sync();

  int bad = -1;
  for (int j = 0; j + 1 < B; ++j) {
    // every thread reads the pivot (published before the barrier) and checks it
    const double piv = sPiv[j];
    if (!pivot_ok(piv)) {
      bad = j;
      break;
    }
    if (ec[NE - 1] > j) {  // this thread still has a live element (the last slot is the latest column)
      const long long pb = __double_as_longlong(piv);
      const double pj = __longlong_as_double((2046LL - (pb >> 52)) << 52);                 // 2^-e_j
      const double mj = __longlong_as_double((pb & 0x000fffffffffffffLL) | (1023LL << 52));  // m_j
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int i = ei[u], c = ec[u];
        if (c > j) {
          const double g = sC[i + j * B] * pj;
          a[u] = fma(-g, sC[c + j * B], mj * a[u]);
          if (c == j + 1) {  // final: publish (the diagonal one is the next pivot)
            sC[i + c * B] = a[u];
            if (i == c) sPiv[c] = a[u];
          }
        }
      }
    }
    sync();
  }
  if (bad < 0 && !pivot_ok(sPiv[B - 1])) bad = B - 1;

  if (bad >= 0) {
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = nanv;
    if (tid < B) sInv[tid] = nanv;
  } else {
    if (tid < 32) {
      // sigma_c = m_0 ... m_{c-1}: exclusive product scan over the pivots' mantissas
      const double pv = sPiv[tid < B ? tid : 0];
      const double mc = __longlong_as_double((__double_as_longlong(pv) & 0x000fffffffffffffLL) | (1023LL << 52));
      const double up = __shfl_up_sync(0xffffffffu, mc, 1);  // every lane takes part
      double sg = (tid >= 1 && tid < B) ? up : 1.0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double x = __shfl_up_sync(0xffffffffu, sg, o);
        if (tid >= o) sg *= x;
      }
      if (tid < B) {
        const double r = rsqrt(sg * pv);  // 1 / sqrt(sigma_c a_cc)
        const int k = sK[tid];
        sRs[tid] = r;
        sInv[tid] = sg * r * pow2(-k);  // 1 / L_cc
        sPiv[tid] = pv * r * pow2(k);   // L_cc
      }
    }
    sync();
    const double sr = pow2(sK[row]);
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int c = q + RPT * m;
      acc[m] = (c < row) ? sC[row + c * B] * sRs[c] * sr : ((c == row) ? sPiv[c] : 0.0);
    }
  }
  sync();
  return bad;
}

// X L^T = acc, column by column, with L's columns pre-scaled by 1/L_jj (sLs:
// L_cj / L_jj below the diagonal) so that the dependency chain of a column is
// a shuffle and one FMA: the unscaled y_j = x_j L_jj is broadcast to the row's
// RPT lanes, and x = y / L_jj is taken for every column at the end
// (inv = 1/L_jj of this thread's columns).
template <int B>
__device__ __forceinline__ void trsm_rows(double (&acc)[FactorCfg<B>::CPT], const double (&inv)[FactorCfg<B>::CPT],
                                          const double* sLs, int q, int row_lane0) {
  constexpr int RPT = FactorCfg<B>::RPT, CPT = FactorCfg<B>::CPT;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const int mj = j / RPT;
    const double y = __shfl_sync(0xffffffffu, acc[mj], row_lane0 + (j % RPT));
    // this thread's columns c = q + RPT m: those with m < j / RPT are all <= j and
    // those with m > j / RPT all > j, so only m = j / RPT needs the test (a masked
    // FP64 instruction still takes its issue slot)
#pragma unroll
    for (int m = mj; m < CPT; ++m) {
      const int c = q + RPT * m;
      if (m > mj || c > j) acc[m] = fma(-y, sLs[c + j * B], acc[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < CPT; ++m) acc[m] *= inv[m];
}

// Lower 8 x 8 blocks of X X^T (X: n rows of a column-major array with leading
// dimension ld, k columns) on the FP64 tensor path (mma.sync m8n8k4, 256 FMAs
// per warp instruction), block b to warp b % 4, into out (n x n, column-major;
// the upper blocks untouched); n a multiple of 8, k of 4.
__device__ __forceinline__ void syrk_mma(const double* X, int ld, int n, int k, double* out, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tq = lane & 3;  // fragment row / column group of this lane
  const int nb = n / 8;
  for (int bk = warp; bk < nb * (nb + 1) / 2; bk += 4) {
    int bi = 0;
    while ((bi + 1) * (bi + 2) / 2 <= bk) ++bi;
    const int bj = bk - bi * (bi + 1) / 2;  // block (bi, bj), bj <= bi, in 8-row units
    double d0 = 0.0, d1 = 0.0;
    for (int ks = 0; ks < k; ks += 4) {
      const double fa = X[(ks + tq) * ld + 8 * bi + g];  // A(g, tq) = X(8 bi + g, ks + tq)
      const double fb = X[(ks + tq) * ld + 8 * bj + g];  // B(tq, g) = X(8 bj + g, ks + tq)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(d0), "+d"(d1)
                   : "d"(fa), "d"(fb));
    }
    out[(8 * bi + g) + (8 * bj + 2 * tq) * n] = d0;
    out[(8 * bi + g) + (8 * bj + 2 * tq + 1) * n] = d1;
  }
}

// FP64 POTRF of the H x H block at S (column-major, leading dimension ld, lower
// triangle of the input read; H = 16, 32 or 64) in place.  H = 16: the
// division-free POTRF.  Larger H by H/2 x H/2 blocks:
//   L11 = chol(A11), L21 = A21 L11^{-T} (rows against L11 with its columns
//   pre-scaled by 1/L_jj), A22 -= L21 L21^T (FP64 tensor path), L22 = chol(A22),
// so every step keeps all 128 threads busy (a block row per 256 / H threads)
// where an H-wide elimination runs H dependent steps.  S receives L (zero
// strict upper triangle), inv the H values 1/L_jj.  Returns the first bad
// pivot (the block is then NaN) or -1.  sElem16: the 16-wide POTRF's element
// numbering (init_df_elements<16>).  Scratch: 1 KB + H^2 / 4 doubles per level.
// `tid` counts the 128 threads from 0; `sync` is their barrier.
template <int H, class Sync>
__device__ int potrf_blocked(double* S, int ld, double* inv, double* scratch, const uint16_t* sElem16, int tid,
                             Sync sync) {
  if constexpr (H == 16) {
    using C = FactorCfg<16>;
    constexpr int RPT = C::RPT, CPT = C::CPT;
    const int row = tid / RPT, q = tid % RPT;
    double* sW = scratch;  // 16 x 16
    double* sPiv = sW + H * H;
    double* sInv = sPiv + H;
    double* sRs = sInv + H;
    int* sK = reinterpret_cast<int*>(sRs + H);
    double acc[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = S[(q + RPT * m) * ld + row];
    const int bad = potrf_tile_df<16>(acc, sW, sPiv, sInv, sRs, sK, sElem16, row, q, tid, sync);
#pragma unroll
    for (int m = 0; m < CPT; ++m) S[(q + RPT * m) * ld + row] = acc[m];
    if (tid < H) inv[tid] = sInv[tid];
    sync();
    return bad;
  } else {
    constexpr int G = H / 2;
    using C = FactorCfg<G>;
    constexpr int RPT = C::RPT, CPT = C::CPT;
    const int row = tid / RPT, q = tid % RPT;
    double* sC = scratch;          // G x G: pre-scaled L11, then the A22 update
    double* sub = scratch + G * G;  // the half-size calls' scratch
    const int bad1 = potrf_blocked<G>(S, ld, inv, sub, sElem16, tid, sync);
    double iv[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int c = q + RPT * m;
      iv[m] = inv[c];
      S[(G + c) * ld + row] = 0.0;                             // upper right block
      if (row > c) sC[row + c * G] = S[c * ld + row] * iv[m];  // L11(row, c) / L11(c, c)
    }
    sync();
    // L21 = A21 L11^{-T}
    double acc[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = S[(q + RPT * m) * ld + G + row];
    trsm_rows<G>(acc, iv, sC, q, (tid & 31) - q);
#pragma unroll
    for (int m = 0; m < CPT; ++m) S[(q + RPT * m) * ld + G + row] = acc[m];
    sync();
    // A22 - L21 L21^T (lower triangle)
    syrk_mma(S + G, ld, G, G, sC, tid);
    sync();
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const int c = q + RPT * m;
      if (c <= row) S[(G + c) * ld + G + row] -= sC[row + c * G];
    }
    sync();
    const int bad2 = potrf_blocked<G>(S + G * ld + G, ld, inv + G, sub, sElem16, tid, sync);
    return bad1 >= 0 ? bad1 : (bad2 >= 0 ? G + bad2 : -1);
  }
}

// The tile POTRF of the FP64 kernel: the division-free form at B = 16; at
// B = 32 and 64 by halves down to 16 x 16 leaves (potrf_blocked), on the tile
// written to sC, with `scratch` (free shared memory) for the blocked steps.
template <int B>
__device__ __forceinline__ int potrf_any(double (&acc)[FactorCfg<B>::CPT], double* sC, double* sPiv, double* sInv,
                                         double* sRs, int* sK, const uint16_t* sElem16, double* scratch, int row,
                                         int q, int tid) {
  auto sync = []() { __syncthreads(); };
  if constexpr (B == 16) {
    return potrf_tile_df<16>(acc, sC, sPiv, sInv, sRs, sK, sElem16, row, q, tid, sync);
  } else {
    constexpr int RPT = FactorCfg<B>::RPT, CPT = FactorCfg<B>::CPT;
#pragma unroll
    for (int m = 0; m < CPT; ++m) sC[(q + RPT * m) * B + row] = acc[m];
    sync();
    const int bad = potrf_blocked<B>(sC, B, sInv, scratch, sElem16, tid, sync);
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = sC[(q + RPT * m) * B + row];
    sync();
    return bad;
  }
}

template <int B>
__global__ void __launch_bounds__(128) factor_f64_kernel(FactorArgs a) {
  using Cfg = FactorCfg<B>;
  constexpr int RPT = Cfg::RPT, CPT = Cfg::CPT, TILE = Cfg::TILE, NSTAGE = Cfg::NSTAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  double* sStage = reinterpret_cast<double*>(smem_raw);
  double* sC = sStage + NSTAGE * 2 * TILE;
  double* sL = sC + TILE;
  double* sInv = sL + TILE;
  double* sPiv = sInv + B;
  double* sRs = sPiv + B;
  int* sK = reinterpret_cast<int*>(sRs + B);  // equilibration exponents of the POTRF
  double* sInvL = sRs + 2 * B;                 // 1/L_jj of the diagonal tile a TRSM applies (16-byte aligned)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sInvL + B);
  __shared__ int sTicket, sAbort;
  __shared__ uint16_t sElem[PotrfDf<16>::NLIVE];  // the 16-wide division-free POTRF's elements

  const int tid = threadIdx.x;
  const int row = tid / RPT;
  const int q = tid % RPT;
  const int lane = tid & 31;
  const int row_lane0 = lane - (lane % RPT);  // first lane of this row inside the warp
  init_df_elements<16>(sElem, tid, 128);

  if (tid == 0) {
    for (int s = 0; s <= NSTAGE; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0;  // bit s: parity of the next completion of barrier s
  const long long limit = a.spin_limit;

  // queue of this CTA: the single ticket order, or (split launch) the chain
  // queue for the first CTA on each reserved SM, the bulk queue elsewhere; the
  // other CTAs on a reserved SM leave so the chain has the SM to itself
  __shared__ int sRole;
  if (tid == 0) {
    int role = 0;
    if (a.chain_sms > 0) {
      const int sm = int(smid());
      role = (sm < a.chain_sms) ? ((atomicAdd(a.sm_claim + sm, 1) == 0) ? 1 : -1) : 2;
    }
    sRole = role;
  }
  __syncthreads();
  const int role = sRole;
  if (role < 0) return;
  int* const counter = (role == 1) ? &a.ctl->ticket2 : &a.ctl->ticket;
  const int nqueue = (role == 1) ? a.nchain : (role == 2 ? a.nbulk : a.ntasks);

  int next = 0;
  if (tid == 0) next = atomicAdd(counter, 1);
  while (true) {
    // generic-proxy writes of the previous task to shared buffers that TMA
    // refills (in-place scaling, reused stage areas) before the next copies
    fence_proxy_async_shared();
    if (tid == 0) {
      int cur = next;
      if (cur < nqueue && ld_volatile(&a.ctl->abort) == 0) {
        next = atomicAdd(counter, 1);
      } else {
        cur = -1;
      }
      sTicket = cur;
      sAbort = 0;
    }
    __syncthreads();
    const int t0 = sTicket;
    if (t0 < 0) break;
    const int t = (role == 1) ? a.chain[t0] : (role == 2 ? a.bulk[t0] : t0);  // task index (one matrix)
    int mi = 0, ti = t;
    if (a.tickets) {
      const int2 v = a.tickets[t];
      mi = v.x;
      ti = v.y;
    }
    const MatCtx mc = a.mats ? a.mats[mi] : a.single;
    const DevTask tk = mc.tasks[ti];
    long long* const trace = mc.trace ? mc.trace + 4 * size_t(ti) : nullptr;
    unsigned long long t_ready = 0;
    if (trace && tid == 0) {
      t_ready = globaltimer();
      trace[0] = (long long)t_ready;
      trace[3] = smid();
    }
    const bool chain = tk.type == TASK_CHAIN;

    // accumulators: acc1 for `out`, acc2 for `out2` (CHAIN only)
    double acc1[CPT], acc2[CPT];
    if (tk.type == TASK_PARTIAL || tk.type == TASK_COMBINE) {
#pragma unroll
      for (int m = 0; m < CPT; ++m) acc1[m] = 0.0;
    } else {
      const double* src = mc.tiles + size_t(tk.out) * TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) acc1[m] = src[(q + RPT * m) * B + row];
    }
    if (chain) {
      const double* src = mc.tiles + size_t(tk.out2) * TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) acc2[m] = src[(q + RPT * m) * B + row];
    } else {
#pragma unroll
      for (int m = 0; m < CPT; ++m) acc2[m] = 0.0;
    }

    // ---- operand pipeline: partial tiles [qb, qe) (older sums) first, then pairs
    // [pb, pe) in the order their producers run; bit 30 of the first index names
    // the accumulator (acc2 = the diagonal tile of a CHAIN task) ----
    const int nq = tk.qe - tk.qb;
    const int nitems = nq + (tk.pe - tk.pb);
    int issued = 0, stop = nitems;
    bool aborted = false;
    for (int it = 0; it < nitems; ++it) {
      // producer (thread 0): keep up to NSTAGE items in flight; block only on item `it`
      if (tid == 0) {
        while (issued < nitems && issued < it + NSTAGE) {
          const int* f1;
          const int* f2 = nullptr;
          const double* g1;
          const double* g2 = nullptr;
          if (issued < nq) {
            const int s = mc.parts[tk.qb + issued] & kIndexMask;
            f1 = mc.sflags + s;
            g1 = mc.scratch + size_t(s) * TILE;
          } else {
            const int pidx = tk.pb + issued - nq;
            const int pa = mc.pairs[2 * pidx] & kIndexMask;
            const int pb = mc.pairs[2 * pidx + 1];
            f1 = mc.flags + pa;
            g1 = mc.tiles + size_t(pa) * TILE;
            if (pb != pa) {
              f2 = mc.flags + pb;
              g2 = mc.tiles + size_t(pb) * TILE;
            }
          }
          if (issued == it) {
            if (!(wait_flag(f1, 1, limit, a.ctl) && (f2 == nullptr || wait_flag(f2, 1, limit, a.ctl)))) {
              raise_timeout(a.ctl, t);
              sAbort = 1;
              break;
            }
          } else if (!(ld_acquire(f1) == 1 && (f2 == nullptr || ld_acquire(f2) == 1))) {
            break;
          }
          fence_proxy_async_global();
          const int st = issued % NSTAGE;
          double* dst = sStage + st * 2 * TILE;
          mbar_arrive_expect_tx(&bars[st], uint32_t((g2 ? 2 : 1) * TILE * sizeof(double)));
          tma_load_1d(dst, g1, TILE * sizeof(double), &bars[st]);
          if (g2) tma_load_1d(dst + TILE, g2, TILE * sizeof(double), &bars[st]);
          ++issued;
        }
        if (trace && it == nitems - 1) t_ready = globaltimer();
      }
      __syncthreads();  // the other warps sleep here while thread 0 waits on flags
      if (sAbort) { stop = it; aborted = true; break; }
      const int st = it % NSTAGE;
      {
        long long spins = 0;
        while (!mbar_try_wait(&bars[st], (phase >> st) & 1u)) {
          if (++spins > kTmaWaitLimit) { aborted = true; break; }
        }
      }
      if (aborted) { stop = it; break; }
      phase ^= (1u << st);
      const double* sA = sStage + st * 2 * TILE;
      if (it < nq) {
        if ((mc.parts[tk.qb + it] >> kTargetShift) == 0) {
#pragma unroll
          for (int m = 0; m < CPT; ++m) acc1[m] += sA[row + (q + RPT * m) * B];
        } else {
#pragma unroll
          for (int m = 0; m < CPT; ++m) acc2[m] += sA[row + (q + RPT * m) * B];
        }
      } else {
        const int pidx = tk.pb + it - nq;
        const int raw = mc.pairs[2 * pidx];
        const double* sB = ((raw & kIndexMask) == mc.pairs[2 * pidx + 1]) ? sA : sA + TILE;
        if ((raw >> kTargetShift) == 0) {
#pragma unroll 4
          for (int p = 0; p < B; ++p) {
            const double av = sA[row + p * B];
#pragma unroll
            for (int m = 0; m < CPT; ++m) acc1[m] = fma(-av, sB[q + RPT * m + p * B], acc1[m]);
          }
        } else {
#pragma unroll 4
          for (int p = 0; p < B; ++p) {
            const double av = sA[row + p * B];
#pragma unroll
            for (int m = 0; m < CPT; ++m) acc2[m] = fma(-av, sB[q + RPT * m + p * B], acc2[m]);
          }
        }
      }
      __syncthreads();  // stage `st` may be refilled
    }
    if (aborted) {
      // Drain copies that were issued but not consumed (items [stop, issued)),
      // so that no TMA write lands in shared memory after the CTA has exited.
      if (tid == 0) {
        for (int j = stop; j < issued; ++j) {
          const int st = j % NSTAGE;
          long long spins = 0;
          while (!mbar_try_wait(&bars[st], (phase >> st) & 1u) && ++spins < kTmaWaitLimit) {
          }
        }
      }
      break;
    }

    if (tk.type == TASK_PARTIAL || tk.type == TASK_COMBINE) {
      double* dst = mc.scratch + size_t(tk.out) * TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * B + row] = acc1[m];
      publish(mc.sflags + tk.out);
      if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
      continue;
    }

    if (tk.type == TASK_DIAG) {
      const int bad = potrf_any<B>(acc1, sC, sPiv, sInv, sRs, sK, sElem, sStage, row, q, tid);
      if (bad >= 0 && tid == 0) atomicMin(mc.info, (unsigned long long)tk.col * B + bad + 1);
      double* dst = mc.tiles + size_t(tk.out) * TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * B + row] = acc1[m];
      if (tid < B) mc.invdiag[size_t(tk.col) * B + tid] = sInv[tid];
      publish(mc.flags + tk.out);
      if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
      continue;
    }

    // ---- OFF and CHAIN: TRSM of `out` with L_kk once it is final ----
    if (tid == 0) {
      if (!wait_flag(mc.flags + tk.diag, 1, limit, a.ctl)) {
        raise_timeout(a.ctl, t);
        sAbort = 1;
      } else {
        if (trace) t_ready = globaltimer();
        fence_proxy_async_global();
        mbar_arrive_expect_tx(&bars[NSTAGE], uint32_t((TILE + B) * sizeof(double)));
        tma_load_1d(sL, mc.tiles + size_t(tk.diag) * TILE, TILE * sizeof(double), &bars[NSTAGE]);
        tma_load_1d(sInvL, mc.invdiag + size_t(tk.col) * B, B * sizeof(double), &bars[NSTAGE]);
      }
    }
    __syncthreads();
    if (sAbort) break;
    {
      long long spins = 0;
      while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u)) {
        if (++spins > kTmaWaitLimit) { aborted = true; break; }
      }
      if (aborted) break;
      phase ^= (1u << NSTAGE);
    }
    double inv[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) inv[m] = sInvL[q + RPT * m];
    // L_kk's columns scaled by 1/L_jj below the diagonal, in place
    for (int e = tid; e < TILE; e += 128) {
      const int c = e % B, j = e / B;
      if (c > j) sL[e] *= sInvL[j];
    }
    __syncthreads();
    trsm_rows<B>(acc1, inv, sL, q, row_lane0);
    {
      double* dst = mc.tiles + size_t(tk.out) * TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * B + row] = acc1[m];
    }
    if (!chain) {
      publish(mc.flags + tk.out);
      if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
      continue;
    }
    // CHAIN: publish L_{k,k-1} and keep it in shared memory for the SYRK term;
    // sL is reused once every warp has finished reading L_kk in the TRSM
    __syncthreads();
#pragma unroll
    for (int m = 0; m < CPT; ++m) sL[(q + RPT * m) * B + row] = acc1[m];
    publish(mc.flags + tk.out);  // includes the barrier that makes sL visible to the CTA
    if constexpr (B == 16) {
      // the SYRK term on the FP64 tensor cores (mma.sync m8n8k4, 256 FMAs per
      // warp instruction): the three lower 8 x 8 blocks of L_{k,k-1} L_{k,k-1}^T,
      // one per warp, into a free stage area, then subtracted row by row
      double* sS = sStage;  // 16 x 16, column-major
      const int warp = tid >> 5;
      if (warp < 3) {
        const int bi = (warp == 0) ? 0 : 8, bj = (warp == 2) ? 8 : 0;
        const int g = lane >> 2, tq = lane & 3;  // fragment row / column group of this lane
        double d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int ks = 0; ks < B; ks += 4) {
          const double fa = sL[(bi + g) + (ks + tq) * B];  // A(g, tq) = L(bi + g, ks + tq)
          const double fb = sL[(bj + g) + (ks + tq) * B];  // B(tq, g) = L(bj + g, ks + tq)
          asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                       : "+d"(d0), "+d"(d1)
                       : "d"(fa), "d"(fb));
        }
        sS[(bi + g) + (bj + 2 * tq) * B] = d0;
        sS[(bi + g) + (bj + 2 * tq + 1) * B] = d1;
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < CPT; ++m) {
        const int c = q + RPT * m;
        if (c <= row) acc2[m] -= sS[row + c * B];
      }
    } else {
#pragma unroll 4
      for (int p = 0; p < B; ++p) {
        const double av = sL[row + p * B];
#pragma unroll
        for (int m = 0; m < CPT; ++m) acc2[m] = fma(-av, sL[q + RPT * m + p * B], acc2[m]);
      }
    }
    const int bad = potrf_any<B>(acc2, sC, sPiv, sInv, sRs, sK, sElem, sStage, row, q, tid);
    if (bad >= 0 && tid == 0) atomicMin(mc.info, (unsigned long long)tk.col2 * B + bad + 1);
    {
      double* dst = mc.tiles + size_t(tk.out2) * TILE;
#pragma unroll
      for (int m = 0; m < CPT; ++m) dst[(q + RPT * m) * B + row] = acc2[m];
    }
    if (tid < B) mc.invdiag[size_t(tk.col2) * B + tid] = sInv[tid];
    publish(mc.flags + tk.out2);
    if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
  }
}

}  // namespace dev
}  // namespace stiles
