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

// G_k = L_kk^{-T} L_kk^{-1} into Sigma's diagonal sub-tile of every sub-column
// (the first term of Sigma_kk), ahead of the persistent launch.
template <int B>
__global__ void selinv_g_kernel(double* __restrict__ sigma, const double* __restrict__ linv,
                                const int32_t* __restrict__ diag_sub, int64_t nsb) {
  for (int64_t k = blockIdx.x; k < nsb; k += gridDim.x) {
    const double* Li = linv + k * B * B;
    for (int o = threadIdx.x; o < B * B; o += blockDim.x) {
      const int r = o % B, c = o / B;
      double v = 0.0;
      for (int p = (r > c ? r : c); p < B; ++p) v = fma(__ldg(Li + p + r * B), __ldg(Li + p + c * B), v);
      sigma[int64_t(diag_sub[k]) * B * B + o] = v;
    }
  }
}

struct SelinvArgs {
  double* sigma;          // nsub * B * B, same layout as the factor's sub-tiles
  double* sigmaT;         // the same sub-tiles transposed (read where a pair wants Sigma^T)
  const double* V;        // nsub * B * B: U_jk^T at the off-diagonal sub-tiles
  double* W;              // nsub * B * B: Sigma_jk^T U_jk at the off-diagonal sub-tiles
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
// smaller ticket).
//  - Off-diagonal task (m, k): accumulates sum_j S_j U_jk over its pairs (S_j a
//    Sigma sub-tile, or its transpose -- kept as a second copy -- when bit 30
//    says so; U from the transposed U array), staged by TMA once the Sigma
//    sub-tile's flag is set; stores Sigma_mk = -sum and its transpose, and the
//    term Sigma_mk^T U_mk of the diagonal sub-tile Sigma_kk into W, then
//    publishes them together.
//  - Diagonal task k: Sigma_kk = G_k - sum_m W(m, k) over the sub-rows m of
//    the column (G_k stored in place beforehand), so the column's last step on
//    the dependency chain is a sum of finished products, not a run of products.
// Thread layout as the FP64 factorization (thread (row, q) holds columns
// q + RPT m), so both operands are read along rows of the stored tiles (no
// bank conflicts).
template <int B>
__global__ void __launch_bounds__(128) selinv_kernel(SelinvArgs a) {
  using Cfg = FactorCfg<B>;
  constexpr int RPT = Cfg::RPT, CPT = Cfg::CPT, TILE = Cfg::TILE;
  constexpr int NSTAGE = SelinvCfg<B>::NSTAGE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  double* sStage = reinterpret_cast<double*>(smem_raw);  // NSTAGE * 2 * TILE
  double* sU = sStage + NSTAGE * 2 * TILE;                // TILE: U_mk^T of an off-diagonal task
  uint64_t* bars = reinterpret_cast<uint64_t*>(sU + TILE);
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
    double* dst = a.sigma + size_t(out) * TILE;
    double* dstT = a.sigmaT + size_t(out) * TILE;
    double acc[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = 0.0;

    if (dcol >= 0) {
      // ---- diagonal task: the column's W terms, each behind its sub-tile's flag ----
      if (tid == 0) {
        for (int i = pb; i < pe; ++i)
          if (!wait_flag(a.flags + (a.pairs[2 * i] & kIndexMask), 1, limit, a.ctl)) {
            raise_timeout(a.ctl, t);
            sAbort = 1;
            break;
          }
      }
      __syncthreads();
      if (sAbort) break;
      int i = pb;
      for (; i + 4 <= pe; i += 4) {  // four sub-tiles' loads in flight per thread
        const double* w0 = a.W + size_t(a.pairs[2 * i] & kIndexMask) * TILE;
        const double* w1 = a.W + size_t(a.pairs[2 * i + 2] & kIndexMask) * TILE;
        const double* w2 = a.W + size_t(a.pairs[2 * i + 4] & kIndexMask) * TILE;
        const double* w3 = a.W + size_t(a.pairs[2 * i + 6] & kIndexMask) * TILE;
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
          const int o = (q + RPT * m) * B + row;
          acc[m] += (__ldcg(w0 + o) + __ldcg(w1 + o)) + (__ldcg(w2 + o) + __ldcg(w3 + o));
        }
      }
      for (; i < pe; ++i) {
        const double* w0 = a.W + size_t(a.pairs[2 * i] & kIndexMask) * TILE;
#pragma unroll
        for (int m = 0; m < CPT; ++m) acc[m] += __ldcg(w0 + (q + RPT * m) * B + row);
      }
#pragma unroll
      for (int m = 0; m < CPT; ++m) {
        const int o = (q + RPT * m) * B + row;
        const double v = dst[o] - acc[m];  // dst holds G_k
        dst[o] = v;
        dstT[row * B + q + RPT * m] = v;
      }
      publish(a.flags + out);
      continue;
    }

    // ---- off-diagonal task ----
    if (tid == 0) {  // U_mk^T for the W term, into its own buffer
      mbar_arrive_expect_tx(&bars[NSTAGE], uint32_t(TILE * sizeof(double)));
      tma_load_1d(sU, a.V + size_t(out) * TILE, TILE * sizeof(double), &bars[NSTAGE]);
    }
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
          double* d = sStage + st * 2 * TILE;
          mbar_arrive_expect_tx(&bars[st], uint32_t(2 * TILE * sizeof(double)));
          const double* src = ((raw >> 30) & 1) ? a.sigmaT : a.sigma;
          tma_load_1d(d, src + size_t(sg) * TILE, TILE * sizeof(double), &bars[st]);
          tma_load_1d(d + TILE, a.V + size_t(su) * TILE, TILE * sizeof(double), &bars[st]);
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
    if (!aborted) {
      long long spins = 0;
      while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u)) {
        if (++spins > kTmaWaitLimit) { aborted = true; break; }
      }
    }
    if (aborted) {
      if (tid == 0) {
        for (int j = stop; j < issued; ++j) {
          const int st = j % NSTAGE;
          long long spins = 0;
          while (!mbar_try_wait(&bars[st], (phase >> st) & 1u) && ++spins < kTmaWaitLimit) {
          }
        }
        long long spins = 0;
        while (!mbar_try_wait(&bars[NSTAGE], (phase >> NSTAGE) & 1u) && ++spins < kTmaWaitLimit) {
        }
      }
      break;
    }
    phase ^= (1u << NSTAGE);
    // Sigma_mk = -acc; its transpose goes to stage 0 (every stage has been
    // consumed) as the left operand of W = Sigma_mk^T U_mk
    double* sT = sStage;
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const double v = -acc[m];
      dst[(q + RPT * m) * B + row] = v;
      dstT[row * B + q + RPT * m] = v;
      sT[q + RPT * m + row * B] = v;
    }
    __syncthreads();
    double w[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) w[m] = 0.0;
#pragma unroll 4
    for (int p = 0; p < B; ++p) {
      const double sv = sT[row + p * B];
#pragma unroll
      for (int m = 0; m < CPT; ++m) w[m] = fma(sv, sU[q + RPT * m + p * B], w[m]);
    }
    double* dW = a.W + size_t(out) * TILE;
#pragma unroll
    for (int m = 0; m < CPT; ++m) dW[(q + RPT * m) * B + row] = w[m];
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
