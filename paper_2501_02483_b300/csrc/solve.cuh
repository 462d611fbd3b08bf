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
  // newest terms folded into precomputed products: two, or one at B = 64 (shared
  // memory: FP64 would not fit, FP32 would drop to one CTA per SM)
  static constexpr int NFOLD = (B == 64) ? 1 : 2;
  // stages | sL (L_kk^{-1}) | sM, sM2 (the folded terms) | sLt (B x (B + 1)) | B
  static constexpr size_t SMEM_ELEMS =
      size_t(NSTAGE) * (TILE + BLK) + size_t(1 + NFOLD) * TILE + size_t(B) * (B + 1) + B;
  static constexpr size_t SMEM = ((SMEM_ELEMS * sizeof(TF) + 15) / 16) * 16 + (NSTAGE + 1) * sizeof(uint64_t) + 16;
};



// One matrix of a solve launch (a batched launch carries one per matrix).
template <typename TF>
struct SolveCtx {
  const TF* tiles;        // factor sub-tiles (FP64, or FP32 for a mixed-precision factor)
  const TF* invdiag;      // nsb * B
  const TF* linv;         // nsb * B * B: L_kk^{-1} of every diagonal sub-tile
  const TF* mlast;        // nsb * B * B: M1_k of every FINAL task (see MlastDesc), or NULL
  const TF* mlast2;       // nsb * B * B: M2_k
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
  // Ready-queue launch (rq_slots != NULL): tickets index a.tickets (batched) or
  // the task list (one matrix) as before, but they are handed out in the order
  // in which tasks were released, and a task is released once every task whose
  // output it reads has started (rq_cnt counts those not yet started; rq_cptr /
  // rq_cons list each task's readers).  Queue slot i (ctl->ticket hands out i,
  // ctl->ticket2 the next free slot) holds the i-th released task, -1 until then.
  // Deadlock-free: a task waits only for tasks that started before it was
  // released, so the earliest-started unfinished task has all its inputs.
  int* rq_slots;
  int* rq_cnt;
  const int32_t* rq_cptr;
  const int32_t* rq_cons;
};

// The ticket in queue slot s once it has been released: -1 when the launch was
// aborted, -2 when the wait gave up (the caller raises the timeout).
__device__ __forceinline__ int wait_slot(const int* s, long long limit, Ctl* ctl) {
  int v = ld_acquire(s);
  if (v >= 0) return v;
  for (long long it = 0; it < limit; ++it) {
    if (it >= 2048) __nanosleep(128);
    v = ld_acquire(s);
    if (v >= 0) return v;
    if ((it & 255) == 255 && ld_volatile(&ctl->abort)) return -1;
  }
  return -2;
}

// Reset of a ready-queue launch: counters from cnt0, the first nsrc slots from
// src (the tasks that read no other task's output), the rest empty.
__global__ void rq_reset_kernel(int* slots, int* cnt, const int32_t* cnt0, const int32_t* src, int nsrc, int n,
                                Ctl* ctl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    cnt[i] = cnt0[i];
    slots[i] = i < nsrc ? src[i] : -1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->ticket = 0;
    ctl->ticket2 = nsrc;
  }
}

// out(i, r) = [z(i, r) -] sum_p M(i, p) w(p, r) for a B x nr block (128
// threads; M column-major, or its transpose with TRANS; out may be global or
// shared memory, and may be z itself).  S threads share one output when there
// are few (each takes B / S terms in two partial sums, combined with shuffles),
// so the dependent FMA chain is B / (2 S) long and all four warps issue.
template <int B, typename TF, int S, bool TRANS, bool SUB>
__device__ __forceinline__ void bmatvec_s(const TF* sM, const TF* sW, const TF* sZ, TF* out, int nr, int tid) {
  constexpr int LEN = B / S;
  const int O = B * nr;
  for (int o0 = 0; o0 < O; o0 += 128 / S) {
    const int o = o0 + tid / S, h = tid % S;
    TF s0 = TF(0), s1 = TF(0);
    if (o < O) {
      const int i = o % B, r = o / B;
      const TF* w = sW + r * B + h * LEN;
#pragma unroll
      for (int q = 0; q < LEN; q += 2) {
        if (TRANS) {  // M(p, i), p rotated per row to spread the banks
          const int p0 = (q + i) % LEN, p1 = (q + 1 + i) % LEN;
          s0 = fma_t(sM[h * LEN + p0 + i * B], w[p0], s0);
          s1 = fma_t(sM[h * LEN + p1 + i * B], w[p1], s1);
        } else {
          s0 = fma_t(sM[i + (h * LEN + q) * B], w[q], s0);
          s1 = fma_t(sM[i + (h * LEN + q + 1) * B], w[q + 1], s1);
        }
      }
    }
    TF v = s0 + s1;
#pragma unroll
    for (int x = 1; x < S; x <<= 1) v += __shfl_xor_sync(0xffffffffu, v, x);
    if (o < O && h == 0) out[o] = SUB ? sZ[o] - v : v;
  }
}

template <int B, typename TF, bool TRANS, bool SUB>
__device__ __forceinline__ void bmatvec(const TF* sM, const TF* sW, const TF* sZ, TF* out, int nr, int tid) {
  const int O = B * nr;
  if (O <= 16) bmatvec_s<B, TF, 8, TRANS, SUB>(sM, sW, sZ, out, nr, tid);
  else if (O <= 32) bmatvec_s<B, TF, 4, TRANS, SUB>(sM, sW, sZ, out, nr, tid);
  else if (O <= 64) bmatvec_s<B, TF, 2, TRANS, SUB>(sM, sW, sZ, out, nr, tid);
  else bmatvec_s<B, TF, 1, TRANS, SUB>(sM, sW, sZ, out, nr, tid);
}

template <int B, bool BACKWARD, typename TF>
__global__ void __launch_bounds__(128) solve_kernel(SolveArgs<TF> a) {
  using Cfg = SolveCfg<B, TF>;
  constexpr int W = Cfg::W, RP = Cfg::RP, G = Cfg::G, U = Cfg::U, TILE = Cfg::TILE, NSTAGE = Cfg::NSTAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TF* sStage = reinterpret_cast<TF*>(smem_raw);                    // NSTAGE * (TILE + BLK)
  TF* sL = sStage + NSTAGE * (TILE + Cfg::BLK);                     // TILE: L_kk^{-1}
  TF* sM = sL + TILE;                                               // TILE: M1_k
  TF* sM2 = sM + TILE;                                              // TILE: M2_k (if NFOLD == 2)
  TF* sLt = sL + (1 + Cfg::NFOLD) * TILE;                           // B x (B + 1): the accumulated block
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

  const bool rq = a.rq_slots != nullptr;
  int next = 0;
  if (tid == 0 && !rq) next = atomicAdd(&a.ctl->ticket, 1);
  while (true) {
    // generic-proxy writes of the previous task to shared buffers that TMA
    // refills (in-place scaling, reused stage areas) before the next copies
    fence_proxy_async_shared();
    if (tid == 0) {
      int cur = -1;
      if (rq) {
        const int slot = ld_volatile(&a.ctl->abort) == 0 ? atomicAdd(&a.ctl->ticket, 1) : a.ntasks;
        if (slot < a.ntasks) {
          cur = wait_slot(a.rq_slots + slot, limit, a.ctl);
          if (cur == -2) raise_timeout(a.ctl, -2 - slot);
        }
      } else {
        cur = next;
        if (cur < a.ntasks && ld_volatile(&a.ctl->abort) == 0) next = atomicAdd(&a.ctl->ticket, 1);
        else cur = -1;
      }
      sTicket = cur;
      sAbort = 0;
    }
    __syncthreads();
    const int t = sTicket;
    if (t < 0) break;
    if (rq) {  // release the readers for which this was the last producer to start
      for (int c = a.rq_cptr[t] + tid; c < a.rq_cptr[t + 1]; c += blockDim.x) {
        const int v = a.rq_cons[c];
        if (atomicSub(a.rq_cnt + v, 1) == 1) atomicExch(a.rq_slots + atomicAdd(&a.ctl->ticket2, 1), v);
      }
    }
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

    // Two accumulators per output (even and odd p) halve the dependent FMA
    // chain of a pair where registers allow (FP64 latency is ~100 cycles).
    constexpr int NACC = (RP * U <= 4) ? 2 : 1;
    TF acc[RP][U], acc2[RP][U];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int s = 0; s < RP; ++s) acc2[s][u] = TF(0);
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

    // The newest terms (the last pairs, produced last) leave the pipeline when
    // their products with L_kk^{-1} are precomputed: block k is then
    // z_k - M2_k w_j2 - M1_k w_j1, z_k = L_kk^{-1} (everything else), so that a
    // newly published block costs one B x B product on the chain.
    const int npairs = tk.pe - tk.pb;
    const int nfold = (tk.type == SOLVE_FINAL && mc.mlast != nullptr) ? min(npairs, Cfg::NFOLD) : 0;
    const int nmain = npairs - nfold;  // pairs through the pipeline
    // the diagonal block's inverse (and the products) do not depend on this sweep: fetch them first
    if (tk.type == SOLVE_FINAL && tid == 0) {
      mbar_arrive_expect_tx(&bars[NSTAGE], uint32_t((1 + nfold) * TILE * sizeof(TF)));
      tma_load_1d(sL, mc.linv + size_t(tk.out) * TILE, TILE * sizeof(TF), &bars[NSTAGE]);
      if (nfold >= 1) tma_load_1d(sM, mc.mlast + size_t(tk.out) * TILE, TILE * sizeof(TF), &bars[NSTAGE]);
      if (nfold >= 2) tma_load_1d(sM2, mc.mlast2 + size_t(tk.out) * TILE, TILE * sizeof(TF), &bars[NSTAGE]);
    }
    const int nitems = nmain + (tk.qe - tk.qb);
    int issued = 0, lissued = 0, stop = nitems;
    bool aborted = false;
    for (int it = 0; it < nitems; ++it) {
      if (tid == 0) {
        // the factor's tiles need no flag: load them as soon as their stage is free
        while (lissued < nitems && lissued < it + NSTAGE) {
          const int st = lissued % NSTAGE;
          if (lissued < nmain) {
            const int ls = mc.pairs[2 * (tk.pb + lissued)];
            mbar_arrive_expect_tx(&bars[st], uint32_t((TILE + blk) * sizeof(TF)));
            tma_load_1d(sStage + st * (TILE + Cfg::BLK), mc.tiles + size_t(ls) * TILE, TILE * sizeof(TF), &bars[st]);
          } else {
            mbar_arrive_expect_tx(&bars[st], uint32_t(blk * sizeof(TF)));
          }
          ++lissued;
        }
        // the right-hand-side blocks once their producers have published them
        while (issued < lissued) {
          const int* f;
          const TF* gY;
          if (issued < nmain) {
            const int bk = mc.pairs[2 * (tk.pb + issued) + 1];
            f = mc.flags + bk;
            gY = mc.Y + size_t(bk) * blk;
          } else {
            const int s = mc.parts[tk.qb + issued - nmain];
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
          tma_load_1d(sStage + st * (TILE + Cfg::BLK) + TILE, gY, uint32_t(blk * sizeof(TF)), &bars[st]);
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
      if (it < nmain) {
        if (!BACKWARD) {
          // acc(i, r) -= sum_p L(i, p) y(p, r)
#pragma unroll 4
          for (int p = 0; p < B; p += NACC) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int r = grp + G * u;
              if (r < nr) {
                const TF yv = sY[r * B + p];
#pragma unroll
                for (int s = 0; s < RP; ++s) acc[s][u] = fma_t(-sT[li + W * s + p * B], yv, acc[s][u]);
                if (NACC == 2) {
                  const TF yw = sY[r * B + p + 1];
#pragma unroll
                  for (int s = 0; s < RP; ++s) acc2[s][u] = fma_t(-sT[li + W * s + (p + 1) * B], yw, acc2[s][u]);
                }
              }
            }
          }
        } else {
          // acc(i, r) -= sum_p L(p, i) x(p, r); p rotated per lane to spread banks
#pragma unroll 4
          for (int pp = 0; pp < B; pp += NACC) {
            const int p = (pp + li) & (B - 1);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int r = grp + G * u;
              if (r < nr) {
                const TF xv = sY[r * B + p];
#pragma unroll
                for (int s = 0; s < RP; ++s) acc[s][u] = fma_t(-sT[p + (li + W * s) * B], xv, acc[s][u]);
                if (NACC == 2) {
                  const int p1 = (p + 1) & (B - 1);
                  const TF xw = sY[r * B + p1];
#pragma unroll
                  for (int s = 0; s < RP; ++s) acc2[s][u] = fma_t(-sT[p1 + (li + W * s) * B], xw, acc2[s][u]);
                }
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
        // stages holding a tile whose block never came: read the block anyway
        // (a valid address; the contents are discarded) so the stage completes
        for (int j = issued; j < lissued; ++j) {
          const TF* gY = (j < nmain) ? mc.Y + size_t(mc.pairs[2 * (tk.pb + j) + 1]) * blk
                                     : mc.scratch + size_t(mc.parts[tk.qb + j - nmain]) * blk;
          tma_load_1d(sStage + (j % NSTAGE) * (TILE + Cfg::BLK) + TILE, gY, uint32_t(blk * sizeof(TF)),
                      &bars[j % NSTAGE]);
        }
        for (int j = stop; j < lissued; ++j) {
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
    if (NACC == 2) {
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int s = 0; s < RP; ++s) acc[s][u] += acc2[s][u];
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
    // z = L_kk^{-1} acc (forward) or L_kk^{-T} acc (backward): the block itself
    // when nothing is folded, else into a free stage's block area
    TF* gOut = mc.Y + size_t(tk.out) * blk;
    static_assert(NSTAGE >= Cfg::NFOLD + 1, "a free stage for z and one per folded block");
    TF* sZ = sStage + ((nitems + Cfg::NFOLD) % NSTAGE) * (TILE + Cfg::BLK) + TILE;
    bmatvec<B, TF, BACKWARD, false>(sL, sAcc, nullptr, nfold > 0 ? sZ : gOut, nr, tid);
    if (nfold > 0) {
      __syncthreads();  // z complete
      // each folded block as it is published, oldest first
      for (int f = 0; f < nfold; ++f) {
        const int st = (nitems + f) % NSTAGE;  // free: every pipeline item has been consumed
        TF* sW = sStage + st * (TILE + Cfg::BLK) + TILE;
        const bool newest = f == nfold - 1;
        if (tid == 0) {
          const int bk = mc.pairs[2 * (tk.pe - nfold + f) + 1];
          if (!wait_flag(mc.flags + bk, 1, limit, a.ctl)) {
            raise_timeout(a.ctl, t);
            sAbort = 1;
          } else {
            if (trace && newest) t_ready = globaltimer();
            fence_proxy_async_global();
            mbar_arrive_expect_tx(&bars[st], uint32_t(blk * sizeof(TF)));
            tma_load_1d(sW, mc.Y + size_t(bk) * blk, uint32_t(blk * sizeof(TF)), &bars[st]);
          }
        }
        __syncthreads();
        if (sAbort) break;  // no copy was issued
        {
          long long spins = 0;
          while (!mbar_try_wait(&bars[st], (phase >> st) & 1u)) {
            if (++spins > kTmaWaitLimit) { aborted = true; break; }
          }
        }
        if (aborted) break;
        phase ^= (1u << st);
        // M2 (second newest) in place on z; M1 (newest) into the output block
        bmatvec<B, TF, false, true>(newest ? sM : sM2, sW, sZ, newest ? gOut : sZ, nr, tid);
        if (!newest) __syncthreads();
      }
      if (sAbort || aborted) break;
    }
    publish(mc.flags + tk.out);
    if (trace && tid == 0) { trace[1] = (long long)t_ready; trace[2] = (long long)globaltimer(); }
  }
}

// The two newest terms of every FINAL sweep task folded with the diagonal
// block, so that one B x B product per published block stays on the sweep's
// dependency chain:
//   forward  (block k, pair L_kj):  M_k = L_kk^{-1} L_kj,
//   backward (block k, pair L_jk):  M_k = L_kk^{-T} L_jk^T,
// M1 for the newest pair, M2 for the one before, column-major at
// mlast / mlast2 + k B^2, applied as w_k = z_k - M2_k w_j2 - M1_k w_j1.
struct MlastDesc {
  void* mlast;             // M1: [fwd: nsb B^2 | bwd: nsb B^2], TF
  void* mlast2;            // M2: same layout
  const void* linv;        // nsb B^2, TF
  const void* tiles;       // factor sub-tiles, TF
  const SolveTask* ftasks;
  const int32_t* fpairs;
  const SolveTask* btasks;
  const int32_t* bpairs;
  int nf, nb;
  int64_t nsb;
};

template <int B, typename TF>
__device__ __forceinline__ void mlast_task(const MlastDesc& d, int t) {
  constexpr int NF = SolveCfg<B, TF>::NFOLD;
  const int task = t / NF, which = t % NF;  // which: 0 = M1 (newest pair), 1 = M2
  const bool backward = task >= d.nf;
  const SolveTask tk = backward ? d.btasks[task - d.nf] : d.ftasks[task];
  if (tk.type != SOLVE_FINAL || tk.pe - tk.pb <= which) return;
  const int32_t* pairs = backward ? d.bpairs : d.fpairs;
  const TF* Li = static_cast<const TF*>(d.linv) + size_t(tk.out) * B * B;
  const TF* L = static_cast<const TF*>(d.tiles) + size_t(pairs[2 * (tk.pe - 1 - which)]) * B * B;
  TF* M = static_cast<TF*>(which ? d.mlast2 : d.mlast) + (size_t(backward ? d.nsb : 0) + tk.out) * B * B;
  for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
    const int i = e % B, p = e / B;
    TF s = TF(0);
    if (!backward) {
#pragma unroll 8
      for (int q = 0; q <= i; ++q) s = fma_t(__ldg(Li + i + q * B), __ldg(L + q + p * B), s);
    } else {
#pragma unroll 8
      for (int q = i; q < B; ++q) s = fma_t(__ldg(Li + q + i * B), __ldg(L + p + q * B), s);
    }
    M[e] = s;
  }
}

template <int B, typename TF>
__global__ void mlast_kernel(MlastDesc d) {
  constexpr int NF = SolveCfg<B, TF>::NFOLD;
  for (int t = blockIdx.x; t < NF * (d.nf + d.nb); t += gridDim.x) mlast_task<B, TF>(d, t);
}

template <int B, typename TF>
__global__ void bmlast_kernel(const MlastDesc* descs) {
  constexpr int NF = SolveCfg<B, TF>::NFOLD;
  const MlastDesc d = descs[blockIdx.y];
  for (int t = blockIdx.x; t < NF * (d.nf + d.nb); t += gridDim.x) mlast_task<B, TF>(d, t);
}

}  // namespace dev
}  // namespace stiles
