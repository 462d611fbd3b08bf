// Selected inverse: Sigma = (P A P^T)^{-1} on the filled sub-tile map of L,
// from Sigma L = L^{-T} in reverse column order (the recursion and task graph
// are described with build_selinv), and the marginal variances diag(A^{-1}).
#pragma once

#include "device_common.cuh"
#include "factor_f64.cuh"

namespace stiles {
namespace dev {

// U_jk = L_jk L_kk^{-1} for every off-diagonal sub-tile (ulist: sub-tile,
// sub-column), one CTA per sub-tile, stored transposed (V = U^T, column-major),
// so that the products read it along its rows without bank conflicts.
// L_kk^{-1} is lower triangular.
template <int B>
__global__ void selinv_u_kernel(double* __restrict__ V, const double* __restrict__ tiles,
                                const double* __restrict__ linv, const int32_t* __restrict__ ulist, int64_t nu) {
  for (int64_t e = blockIdx.x; e < nu; e += gridDim.x) {
    const int64_t s = ulist[2 * e], k = ulist[2 * e + 1];
    const double* Ls = tiles + s * B * B;
    const double* Li = linv + k * B * B;
    for (int o = threadIdx.x; o < B * B; o += blockDim.x) {
      const int i = o % B, c = o / B;
      double v = 0.0;
      for (int p = c; p < B; ++p) v = fma(__ldg(Ls + i + p * B), __ldg(Li + p + c * B), v);
      V[s * B * B + c + i * B] = v;
    }
  }
}

struct SelinvArgs {
  double* sigma;          // nsub * B * B, same layout as the factor's sub-tiles
  double* sigmaT;         // the same sub-tiles transposed (read where a pair wants Sigma^T)
  const double* V;        // nsub * B * B: U_jk^T at the off-diagonal sub-tiles
  const double* linv;     // nsb * B * B: L_kk^{-1}
  const int32_t* tasks;   // 4 per task (see SelinvGraph)
  const int32_t* pairs;   // 2 per pair
  int ntasks;
  int* flags;             // per Sigma sub-tile: 1 when final
  Ctl* ctl;
  long long spin_limit;
};

template <int B>
struct SelinvCfg {
  static constexpr int NSTAGE = 3;
  static constexpr int TILE = B * B;
  static constexpr size_t SMEM = (size_t(NSTAGE) * 2 + 1) * TILE * sizeof(double) + (NSTAGE + 1) * sizeof(uint64_t) + 16;
};

// Persistent over the tasks in ticket order (every dependency carries a
// smaller ticket).  A task accumulates sum_j S_j U_j over its pairs (S_j a
// Sigma sub-tile, or its transpose -- kept as a second copy -- when bit 30
// says so; U_j from the transposed U array), with the pairs staged by TMA
// once the Sigma sub-tile's flag is set, and stores -sum (off-diagonal) or
// L_kk^{-T} L_kk^{-1} - sum (diagonal), and its transpose.  Thread layout as
// the FP64 factorization (thread (row, q) holds columns q + RPT m), so both
// operands are read along rows of the stored tiles (no bank conflicts).
template <int B>
__global__ void __launch_bounds__(128) selinv_kernel(SelinvArgs a) {
  using Cfg = FactorCfg<B>;
  constexpr int RPT = Cfg::RPT, CPT = Cfg::CPT, TILE = Cfg::TILE;
  constexpr int NSTAGE = SelinvCfg<B>::NSTAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  double* sStage = reinterpret_cast<double*>(smem_raw);  // NSTAGE * 2 * TILE
  double* sLi = sStage + NSTAGE * 2 * TILE;               // TILE: L_kk^{-1} of a diagonal task
  uint64_t* bars = reinterpret_cast<uint64_t*>(sLi + TILE);
  __shared__ int sTicket, sAbort;
  const int tid = threadIdx.x;
  const int row = tid / RPT, q = tid % RPT;
  if (tid == 0) {
    for (int s = 0; s <= NSTAGE; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  const long long limit = a.spin_limit;
  int next = 0;
  if (tid == 0) next = atomicAdd(&a.ctl->ticket, 1);
  while (true) {
    fence_proxy_async_shared();
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
    const int out = a.tasks[4 * t], dcol = a.tasks[4 * t + 1], pb = a.tasks[4 * t + 2], pe = a.tasks[4 * t + 3];
    if (dcol >= 0 && tid == 0) {
      mbar_arrive_expect_tx(&bars[NSTAGE], uint32_t(TILE * sizeof(double)));
      tma_load_1d(sLi, a.linv + size_t(dcol) * TILE, TILE * sizeof(double), &bars[NSTAGE]);
    }
    double acc[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = 0.0;
    const int nitems = pe - pb;
    int issued = 0, stop = nitems;
    bool aborted = false;
    for (int it = 0; it < nitems; ++it) {
      if (tid == 0) {
        while (issued < nitems && issued < it + NSTAGE) {
          const int raw = a.pairs[2 * (pb + issued)];
          const int sg = raw & ((1 << 30) - 1), su = a.pairs[2 * (pb + issued) + 1];
          const int* f = a.flags + sg;
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
          double* dst = sStage + st * 2 * TILE;
          mbar_arrive_expect_tx(&bars[st], uint32_t(2 * TILE * sizeof(double)));
          const double* src = ((raw >> 30) & 1) ? a.sigmaT : a.sigma;
          tma_load_1d(dst, src + size_t(sg) * TILE, TILE * sizeof(double), &bars[st]);
          tma_load_1d(dst + TILE, a.V + size_t(su) * TILE, TILE * sizeof(double), &bars[st]);
          ++issued;
        }
      }
      __syncthreads();
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
      const double* sS = sStage + st * 2 * TILE;
      const double* sV = sS + TILE;
#pragma unroll 4
      for (int p = 0; p < B; ++p) {
        const double sv = sS[row + p * B];
#pragma unroll
        for (int m = 0; m < CPT; ++m) acc[m] = fma(sv, sV[q + RPT * m + p * B], acc[m]);
      }
      __syncthreads();  // stage `st` may be refilled
    }
    if (aborted) {
      if (tid == 0) {
        for (int j = stop; j < issued; ++j) {
          const int st = j % NSTAGE;
          long long spins = 0;
          while (!mbar_try_wait(&bars[st], (phase >> st) & 1u) && ++spins < kTmaWaitLimit) {
          }
        }
        if (dcol >= 0) {
          long long spins = 0;
          while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u) && ++spins < kTmaWaitLimit) {
          }
        }
      }
      break;
    }
    double v[CPT];
    if (dcol >= 0) {
      {
        long long spins = 0;
        while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u)) {
          if (++spins > kTmaWaitLimit) { aborted = true; break; }
        }
      }
      if (aborted) break;
      phase ^= (1u << NSTAGE);
      // L_kk^{-T} L_kk^{-1} (row, c) = sum_p Li(p, row) Li(p, c)
#pragma unroll
      for (int m = 0; m < CPT; ++m) v[m] = -acc[m];
#pragma unroll 4
      for (int p = 0; p < B; ++p) {
        const double lr = sLi[p + row * B];
#pragma unroll
        for (int m = 0; m < CPT; ++m) v[m] = fma(lr, sLi[p + (q + RPT * m) * B], v[m]);
      }
    } else {
#pragma unroll
      for (int m = 0; m < CPT; ++m) v[m] = -acc[m];
    }
    double* dst = a.sigma + size_t(out) * TILE;
    double* dstT = a.sigmaT + size_t(out) * TILE;
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      dst[(q + RPT * m) * B + row] = v[m];
      dstT[row * B + q + RPT * m] = v[m];
    }
    publish(a.flags + out);
  }
}

// out[perm[i]] = Sigma_ii (permuted index i < n): the marginal variances.
template <int B>
__global__ void selinv_diag_kernel(double* __restrict__ out, const double* __restrict__ sigma,
                                   const int32_t* __restrict__ diag_sub, const int64_t* __restrict__ perm, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = i / B, r = i % B;
    out[perm[i]] = sigma[int64_t(diag_sub[k]) * B * B + r * (B + 1)];
  }
}

}  // namespace dev
}  // namespace stiles
