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
  double* W;              // nsub * B * B: W(j, k) = Sigma_jk^T U_jk at the off-diagonal sub-tiles
  double* X;              // nsub * B * B: X(m, c) = Sigma_mp^T U_mc, p the parent of sub-column c
  const int32_t* tasks;   // 8 per task (see SelinvGraph)
  const int32_t* pairs;   // 2 per product
  const int32_t* loads;   // 3 per finished term
  const int32_t* posts;   // 1 per X product
  int ntasks;
  int* flags;             // per Sigma sub-tile: 1 when final (with its W and X terms)
  Ctl* ctl;
  long long spin_limit;
  long long* trace;       // NULL, or 4 stamps per task: start, operands ready, done (ns), SM id
};

template <int B>
struct SelinvCfg {
  static constexpr int NSTAGE = 3;
  static constexpr int TILE = B * B;
  static constexpr size_t SMEM = (size_t(NSTAGE) * 2 + 1) * TILE * sizeof(double) + (NSTAGE + 1) * sizeof(uint64_t) + 16;
};

// Persistent over the tasks in ticket order (every dependency carries a
// smaller ticket).  With p the parent of sub-column k (its first sub-row):
//  - Off-diagonal task (m, k), m > p: Sigma_mk = -sum_j S_j U_jk over its
//    product pairs (S_j a Sigma sub-tile, or its transpose -- kept as a second
//    copy -- when bit 30 says so; U from the transposed U array), staged by TMA
//    once the Sigma sub-tile's flag is set.
//  - Parent-row task (p, k): Sigma_pk = -(Sigma_pp U_pk + sum_j X(j, k)); the
//    X terms were formed by the tasks of column p, so only one product waits
//    for that column.
//  - Every off-diagonal task then stores Sigma_mk and its transpose, forms
//    W(m, k) = Sigma_mk^T U_mk for the diagonal sub-tile and X(m, c) =
//    Sigma_mk^T U_mc for each child c of k, and publishes them together.
//  - Diagonal task k: Sigma_kk = G_k - sum_m W(m, k) (G_k stored in place
//    beforehand).
// Thread layout as the FP64 factorization (thread (row, q) holds columns
// q + RPT m), so both operands are read along rows of the stored tiles (no
// bank conflicts).
template <int B>
__global__ void __launch_bounds__(128) selinv_kernel(SelinvArgs a) {
  using Cfg = FactorCfg<B>;
  constexpr int RPT = Cfg::RPT, CPT = Cfg::CPT, TILE = Cfg::TILE;
  constexpr int NSTAGE = SelinvCfg<B>::NSTAGE;
  constexpr int NPOST = 2 * NSTAGE - 1;  // U tiles of X products staged at once (stage tiles 1..)
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
    const int32_t* tk = a.tasks + 8 * size_t(t);
    long long* const trace = a.trace ? a.trace + 4 * size_t(t) : nullptr;
    if (trace && tid == 0) {
      trace[0] = (long long)globaltimer();
      trace[3] = smid();
    }
    const int out = tk[0], dcol = tk[1], pb = tk[2], pe = tk[3], lb = tk[4], le = tk[5], ob = tk[6], oe = tk[7];
    double* dst = a.sigma + size_t(out) * TILE;
    double* dstT = a.sigmaT + size_t(out) * TILE;
    double acc[CPT];
#pragma unroll
    for (int m = 0; m < CPT; ++m) acc[m] = 0.0;

    // ---- finished terms (W for a diagonal task, X for a parent-row task) ----
    if (le > lb) {
      if (tid == 0 && !wait_flags([&](int i) { return a.flags + a.loads[3 * (lb + i)]; },
                                  [&](int i) { return a.loads[3 * (lb + i) + 1]; }, le - lb, limit, a.ctl)) {
        raise_timeout(a.ctl, t);
        sAbort = 1;
      }
      __syncthreads();
      if (sAbort) break;
      auto term = [&](int i) {
        const int x = a.loads[3 * i + 2];
        return ((x >> 30) & 1 ? a.W : a.X) + size_t(x & ((1 << 30) - 1)) * TILE;
      };
      int i = lb;
      for (; i + 4 <= le; i += 4) {  // four sub-tiles' loads in flight per thread
        const double* w0 = term(i);
        const double* w1 = term(i + 1);
        const double* w2 = term(i + 2);
        const double* w3 = term(i + 3);
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
          const int o = (q + RPT * m) * B + row;
          acc[m] += (__ldcg(w0 + o) + __ldcg(w1 + o)) + (__ldcg(w2 + o) + __ldcg(w3 + o));
        }
      }
      for (; i < le; ++i) {
        const double* w0 = term(i);
#pragma unroll
        for (int m = 0; m < CPT; ++m) acc[m] += __ldcg(w0 + (q + RPT * m) * B + row);
      }
    }
    if (dcol >= 0) {
      if (trace && tid == 0) trace[1] = (long long)globaltimer();
#pragma unroll
      for (int m = 0; m < CPT; ++m) {
        const int o = (q + RPT * m) * B + row;
        const double v = dst[o] - acc[m];  // dst holds G_k
        dst[o] = v;
        dstT[row * B + q + RPT * m] = v;
      }
      publish(a.flags + out);
      if (trace && tid == 0) trace[2] = (long long)globaltimer();
      continue;
    }

    // ---- off-diagonal task: products ----
    if (tid == 0) {  // U_mk^T for the W term, into its own buffer
      mbar_arrive_expect_tx(&bars[NSTAGE], uint32_t(TILE * sizeof(double)));
      tma_load_1d(sU, a.V + size_t(out) * TILE, TILE * sizeof(double), &bars[NSTAGE]);
    }
    const int nitems = pe - pb;
    int issued = 0, stop = nitems;
    int known = 0;  // thread 0: items [0, known) have their flags acquired
    auto pflag = [&](int i) { return a.flags + (a.pairs[2 * (pb + i)] & ((1 << 30) - 1)); };
    bool aborted = false;
    for (int it = 0; it < nitems; ++it) {
      if (tid == 0) {
        const int want = min(nitems, it + NSTAGE);
        if (known < want) {  // poll ahead in batches; block only for item `it`
          const int k0 = known;
          known = count_set_flags(pflag, known, min(nitems, want + 16));
          if (known <= it) {
            if (wait_flags([&](int i) { return pflag(it + i); }, 1, limit, a.ctl)) {
              known = it + 1;
            } else {
              raise_timeout(a.ctl, t);
              sAbort = 1;
            }
          } else if (known > k0) {
            fence_acq_rel_gpu();
          }
        }
        while (!sAbort && issued < want && issued < known) {
          const int raw = a.pairs[2 * (pb + issued)];
          const int sg = raw & ((1 << 30) - 1), su = a.pairs[2 * (pb + issued) + 1];
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
    if (trace && tid == 0) trace[1] = (long long)globaltimer();
    // every stage has been consumed: stage tile 0 takes Sigma_mk^T (the left
    // operand of W and X), tiles 1..NPOST the U tiles of the X products, whose
    // first batch is in flight while W is formed
    auto issue_posts = [&](int o0) {
      const int nb = min(NPOST, oe - o0);
      mbar_arrive_expect_tx(&bars[0], uint32_t(nb * TILE * sizeof(double)));
      for (int i = 0; i < nb; ++i)
        tma_load_1d(sStage + (1 + i) * TILE, a.V + size_t(a.posts[o0 + i]) * TILE, TILE * sizeof(double), &bars[0]);
    };
    if (tid == 0 && oe > ob) issue_posts(ob);
    double* sT = sStage;
#pragma unroll
    for (int m = 0; m < CPT; ++m) {
      const double v = -acc[m];
      dst[(q + RPT * m) * B + row] = v;
      dstT[row * B + q + RPT * m] = v;
      sT[q + RPT * m + row * B] = v;
    }
    __syncthreads();
    // T^T U for a U^T tile in shared memory, stored column-major at d
    auto product = [&](const double* sUt, double* d) {
      double w[CPT];
#pragma unroll
      for (int m = 0; m < CPT; ++m) w[m] = 0.0;
#pragma unroll 4
      for (int p = 0; p < B; ++p) {
        const double sv = sT[row + p * B];
#pragma unroll
        for (int m = 0; m < CPT; ++m) w[m] = fma(sv, sUt[q + RPT * m + p * B], w[m]);
      }
#pragma unroll
      for (int m = 0; m < CPT; ++m) d[(q + RPT * m) * B + row] = w[m];
    };
    product(sU, a.W + size_t(out) * TILE);
    for (int o0 = ob; o0 < oe && !aborted; o0 += NPOST) {
      const int nb = min(NPOST, oe - o0);
      {
        long long spins = 0;
        while (!mbar_try_wait(&bars[0], phase & 1u)) {
          if (++spins > kTmaWaitLimit) { aborted = true; break; }
        }
      }
      if (aborted) break;
      phase ^= 1u;
      for (int i = 0; i < nb; ++i) product(sStage + (1 + i) * TILE, a.X + size_t(a.posts[o0 + i]) * TILE);
      if (o0 + NPOST < oe) {
        __syncthreads();  // every thread is done with the staged U tiles
        if (tid == 0) issue_posts(o0 + NPOST);
      }
    }
    if (aborted) {
      if (tid == 0) {
        long long spins = 0;
        while (!mbar_try_wait(&bars[0], phase & 1u) && ++spins < kTmaWaitLimit) {
        }
      }
      break;
    }
    publish(a.flags + out);
    if (trace && tid == 0) trace[2] = (long long)globaltimer();
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
