// Persistent forward (L y = P b) and backward (L^T x = y) tile sweeps.
//
// The sweeps compute in the factor's storage type TF: FP64 for an FP64 factor;
// FP32 for a mixed-precision factor (FP32 tiles), whose solves only feed the
// FP64 iterative refinement -- the factor's own error (BF16/FP16 updates)
// dominates FP32 rounding by orders of magnitude, and FP32 arithmetic runs at
// 64 times the FP64 rate on this part.
//
// Same scheduling scheme as the factorization: one task per B-row block of
// the right-hand sides, in ticket order, waiting on per-block ready flags.
// Long accumulations (the arrow rows, which see every body block) are split
// into tree leaves exactly like the factorization's arrow updates.
//
// Block layout: block k (rows k*B .. k*B+B-1 of the permuted system, nr
// right-hand sides) is contiguous, column-major B x nr, at Y + k * B * nr.
// Thread layout: W = min(B, 32) lanes hold one right-hand side column
// (RP = B / W rows each); the NT / W lane groups take columns g, g + G, ...
#pragma once

#include "aux_kernels.cuh"
#include "device_common.cuh"
#include "plan.h"

namespace stiles {
namespace dev {

constexpr int SOLVE_MAXR = 16;  // right-hand sides per launch

template <int B, typename TF>
struct SolveCfg {
  static constexpr int NT = 128;
  static constexpr int W = (B < 32) ? B : 32;
  static constexpr int RP = B / W;
  static constexpr int G = NT / W;
  static constexpr int U = (SOLVE_MAXR + G - 1) / G;
  static constexpr int TILE = B * B;
  static constexpr int BLK = B * SOLVE_MAXR;
  static constexpr int NSTAGE = 3;
  static constexpr size_t SMEM_ELEMS = size_t(NSTAGE) * (TILE + BLK) + TILE + size_t(B) * (B + 1) + B;
  static constexpr size_t SMEM = ((SMEM_ELEMS * sizeof(TF) + 15) / 16) * 16 + (NSTAGE + 1) * sizeof(uint64_t) + 16;
};



// One matrix of a solve launch (a batched launch carries one per matrix).
template <typename TF>
struct SolveCtx {
  const TF* tiles;        // factor sub-tiles (FP64, or FP32 for a mixed-precision factor)
  const TF* invdiag;      // nsb * B
  const TF* linv;         // nsb * B * B: L_kk^{-1} of every diagonal sub-tile
  TF* Y;                  // nsb blocks of B x nr
  TF* scratch;            // nscratch blocks
  const SolveTask* tasks;
  const int32_t* pairs;   // (L sub-tile, block)
  const int32_t* parts;
  int* flags;             // per block
  int* sflags;            // per scratch block
  long long* trace;       // optional, 4 per task: start, dependencies ready, done, SM id
  int nr;                 // right-hand sides (<= SOLVE_MAXR)
  int pad0;
};

template <typename TF>
struct SolveArgs {
  SolveCtx<TF> single;          // one-matrix launch (mats == NULL)
  const SolveCtx<TF>* mats;     // batched launch: one context per matrix
  const int2* tickets;          // batched launch: (matrix, task) per ticket
  int ntasks;
  Ctl* ctl;
  long long spin_limit;
};

template <int B, bool BACKWARD, typename TF>
__global__ void __launch_bounds__(128) solve_kernel(SolveArgs<TF> a) {
  using Cfg = SolveCfg<B, TF>;
  constexpr int W = Cfg::W, RP = Cfg::RP, G = Cfg::G, U = Cfg::U, TILE = Cfg::TILE, NSTAGE = Cfg::NSTAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TF* sStage = reinterpret_cast<TF*>(smem_raw);                    // NSTAGE * (TILE + BLK)
  TF* sL = sStage + NSTAGE * (TILE + Cfg::BLK);                     // TILE: L_kk^{-1}
  TF* sLt = sL + TILE;                                              // B x (B + 1): the accumulated block
  TF* sInv = sLt + B * (B + 1);                                     // B (unused)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + ((Cfg::SMEM_ELEMS * sizeof(TF) + 15) / 16) * 16);
  __shared__ int sTicket, sAbort;

  const int tid = threadIdx.x;
  const int li = tid % W;  // lane inside the column group
  const int grp = tid / W;
  const long long limit = a.spin_limit;

  if (tid == 0) {
    for (int s = 0; s <= NSTAGE; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0;

  int next = 0;
  if (tid == 0) next = atomicAdd(&a.ctl->ticket, 1);
  while (true) {
    if (tid == 0) {
      int cur = next;
      if (cur < a.ntasks && ld_volatile(&a.ctl->abort) == 0) next = atomicAdd(&a.ctl->ticket, 1);
      else cur = -1;
      sTicket = cur;
      sAbort = 0;
    }
    __syncthreads();
    const int t = sTicket;
    if (t < 0) break;
    int mi = 0, ti = t;
    if (a.tickets) {
      const int2 v = a.tickets[t];
      mi = v.x;
      ti = v.y;
    }
    const SolveCtx<TF> mc = a.mats ? a.mats[mi] : a.single;
    const SolveTask tk = mc.tasks[ti];
    const int nr = mc.nr;
    const int blk = B * nr;  // elements per block
    long long* const trace = mc.trace ? mc.trace + 4 * size_t(ti) : nullptr;
    unsigned long long t_ready = 0;
    if (trace && tid == 0) {
      t_ready = globaltimer();
      trace[0] = (long long)t_ready;
      trace[3] = smid();
    }

    TF acc[RP][U];
    if (tk.type == SOLVE_FINAL) {
      const TF* src = mc.Y + size_t(tk.out) * blk;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = grp + G * u;
#pragma unroll
        for (int s = 0; s < RP; ++s) acc[s][u] = (r < nr) ? src[r * B + li + W * s] : TF(0);
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int s = 0; s < RP; ++s) acc[s][u] = TF(0);
    }

    // the diagonal block's inverse does not depend on this sweep: fetch it first
    if (tk.type == SOLVE_FINAL && tid == 0) {
      mbar_arrive_expect_tx(&bars[NSTAGE], uint32_t(TILE * sizeof(TF)));
      tma_load_1d(sL, mc.linv + size_t(tk.out) * TILE, TILE * sizeof(TF), &bars[NSTAGE]);
    }
    const int npairs = tk.pe - tk.pb;
    const int nitems = npairs + (tk.qe - tk.qb);
    int issued = 0, stop = nitems;
    bool aborted = false;
    for (int it = 0; it < nitems; ++it) {
      if (tid == 0) {
        while (issued < nitems && issued < it + NSTAGE) {
          const int* f;
          const TF* gL = nullptr;
          const TF* gY;
          if (issued < npairs) {
            const int ls = mc.pairs[2 * (tk.pb + issued)];
            const int bk = mc.pairs[2 * (tk.pb + issued) + 1];
            f = mc.flags + bk;
            gL = mc.tiles + size_t(ls) * TILE;
            gY = mc.Y + size_t(bk) * blk;
          } else {
            const int s = mc.parts[tk.qb + issued - npairs];
            f = mc.sflags + s;
            gY = mc.scratch + size_t(s) * blk;
          }
          if (issued == it) {
            if (!wait_flag(f, 1, limit, a.ctl)) {
              raise_timeout(a.ctl, t);
              sAbort = 1;
              break;
            }
          } else if (ld_acquire(f) != 1) {
            break;
          }
          fence_proxy_async_global();
          const int st = issued % NSTAGE;
          TF* dst = sStage + st * (TILE + Cfg::BLK);
          mbar_arrive_expect_tx(&bars[st], uint32_t((gL ? TILE * sizeof(TF) : 0) + blk * sizeof(TF)));
          if (gL) tma_load_1d(dst, gL, TILE * sizeof(TF), &bars[st]);
          tma_load_1d(dst + TILE, gY, uint32_t(blk * sizeof(TF)), &bars[st]);
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
      const TF* sT = sStage + st * (TILE + Cfg::BLK);
      const TF* sY = sT + TILE;
      if (it < npairs) {
        if (!BACKWARD) {
          // acc(i, r) -= sum_p L(i, p) y(p, r)
#pragma unroll 4
          for (int p = 0; p < B; ++p) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int r = grp + G * u;
              if (r < nr) {
                const TF yv = sY[r * B + p];
#pragma unroll
                for (int s = 0; s < RP; ++s) acc[s][u] = fma_t(-sT[li + W * s + p * B], yv, acc[s][u]);
              }
            }
          }
        } else {
          // acc(i, r) -= sum_p L(p, i) x(p, r); p rotated per lane to spread banks
#pragma unroll 4
          for (int pp = 0; pp < B; ++pp) {
            const int p = (pp + li) & (B - 1);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int r = grp + G * u;
              if (r < nr) {
                const TF xv = sY[r * B + p];
#pragma unroll
                for (int s = 0; s < RP; ++s) acc[s][u] = fma_t(-sT[p + (li + W * s) * B], xv, acc[s][u]);
              }
            }
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int r = grp + G * u;
          if (r < nr)
#pragma unroll
            for (int s = 0; s < RP; ++s) acc[s][u] += sY[r * B + li + W * s];
        }
      }
      __syncthreads();
    }
    if (aborted) {
      if (tid == 0) {
        for (int j = stop; j < issued; ++j) {
          const int st = j % NSTAGE;
          long long spins = 0;
          while (!mbar_try_wait(&bars[st], (phase >> st) & 1u) && ++spins < kTmaWaitLimit) {
          }
        }
        if (tk.type == SOLVE_FINAL) {
          long long spins = 0;
          while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u) && ++spins < kTmaWaitLimit) {
          }
        }
      }
      break;
    }

    if (tk.type != SOLVE_FINAL) {
      TF* dst = mc.scratch + size_t(tk.out) * blk;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = grp + G * u;
        if (r < nr)
#pragma unroll
          for (int s = 0; s < RP; ++s) dst[r * B + li + W * s] = acc[s][u];
      }
      publish(mc.sflags + tk.out);
      if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
      continue;
    }

    // ---- y = L_kk^{-1} acc (forward) or x = L_kk^{-T} acc (backward), L_kk^{-1} prefetched ----
    {
      long long spins = 0;
      while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u)) {
        if (++spins > kTmaWaitLimit) { aborted = true; break; }
      }
    }
    if (aborted) break;
    phase ^= (1u << NSTAGE);
    TF* sAcc = sLt;  // B x nr block of the accumulated right-hand sides
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = grp + G * u;
      if (r < nr)
#pragma unroll
        for (int s = 0; s < RP; ++s) sAcc[r * B + li + W * s] = acc[s][u];
    }
    __syncthreads();
    const int warp_grp0 = (tid & ~31) / W;  // first column group of this warp (warp-uniform guard)
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (warp_grp0 + G * u >= nr) break;
      const int r = grp + G * u;
      const TF* a = sAcc + (r < nr ? r : 0) * B;
#pragma unroll
      for (int s = 0; s < RP; ++s) {
        const int i = li + W * s;
        TF v = TF(0);
        // the inverse is stored with zeros above its diagonal: full-length sums
#pragma unroll
        for (int p = 0; p < B; ++p) v = fma_t(BACKWARD ? sL[p + i * B] : sL[i + p * B], a[p], v);
        acc[s][u] = v;
      }
    }
    {
      TF* dst = mc.Y + size_t(tk.out) * blk;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = grp + G * u;
        if (r < nr)
#pragma unroll
          for (int s = 0; s < RP; ++s) dst[r * B + li + W * s] = acc[s][u];
      }
    }
    publish(mc.flags + tk.out);
    if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
  }
}

}  // namespace dev
}  // namespace stiles
