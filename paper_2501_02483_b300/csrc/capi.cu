// C ABI of libstiles.so: plan/factor lifetime, device uploads and launches.
// Declarations and argument conventions are in include/stiles.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "aux_kernels.cuh"
#include "factor_f64.cuh"
#include "factor_lp.cuh"
#include "factor_oz.cuh"
#include "plan.h"
#include "selinv.cuh"
#include "solve.cuh"

namespace {

thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};  // kernels launched by this library (all threads)

inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

stiles_status fail(stiles_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define CUDA_TRY(expr)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (expr);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,            \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                              \
    }                                                                                               \
  } while (0)

template <class T>
cudaError_t upload(T** dptr, const std::vector<T>& v) {
  *dptr = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dptr), v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min<int64_t>(g, 148 * 32)));
}

}  // namespace

namespace stiles {

struct DevGraph {
  DevTask* tasks = nullptr;
  SolveTask* stasks = nullptr;
  int32_t* pairs = nullptr;
  int32_t* parts = nullptr;
  int32_t* chain = nullptr;  // factor graph: the two queues of a split launch
  int32_t* bulk = nullptr;
  int ntasks = 0;
};

struct DevPlan {
  int device = -1;
  int64_t* scatter = nullptr;
  int64_t* pad = nullptr;
  int64_t* perm = nullptr;
  int32_t* diag_sub = nullptr;
  int64_t* colptr = nullptr;
  int32_t* rowidx = nullptr;
  int64_t* rptr = nullptr;   // CSR index of the strict lower part (residual SpMV)
  int32_t* rcol = nullptr;
  int64_t* rval = nullptr;
  DevGraph fac, fwd, bwd;
  DevGraph fus;          // factorization with the forward sweep folded in (built on first use)
  bool fus_ready = false;
  int grid_factor = 0, grid_solve = 0;
  // selected inverse (uploaded on first use)
  int32_t* sinv_tasks = nullptr;
  int32_t* sinv_pairs = nullptr;
  int32_t* sinv_loads = nullptr;
  int32_t* sinv_posts = nullptr;
  int32_t* sinv_ulist = nullptr;
  int sinv_ntasks = 0;
  int64_t sinv_nu = 0;
  bool sinv_ready = false;
};

}  // namespace stiles

struct stiles_factor {
  const stiles_plan* plan = nullptr;
  int device = -1;
  bool lp = false;            // mixed precision (BF16/FP16 updates, FP32 tiles, FP64 diagonal)
  bool sliced = false;        // FP64 tiles, updates from BF16 digit slices on the tensor cores
  double* values = nullptr;   // FP64 copy of A's values (CSC order) for residuals
  double* tiles = nullptr;    // FP64 path
  double* scratch = nullptr;
  double* invdiag = nullptr;
  double* linv = nullptr;     // L_kk^{-1} of every diagonal sub-tile (nsb * B * B), for the sweeps, then
                              // the sweeps' folded terms M1 (fwd, bwd), M2 (fwd, bwd): nsb * B * B each
  uint16_t* slices = nullptr; // sliced path: 4 BF16 digit slices per sub-tile
  int* rowexp = nullptr;      // sliced path: power-of-two row scales (nsb * B)
  float* tiles32 = nullptr;   // mixed-precision path
  float* linv32 = nullptr;
  uint16_t* tiles16 = nullptr;
  float* scratch32 = nullptr;
  float* invdiag32 = nullptr;
  double* ldiag = nullptr;
  double* irwork = nullptr;   // refinement: correction, residual, CG direction and A p, 4 * n * SOLVE_MAXR
  double* cgs = nullptr;      // CG scalars: dot products and step lengths, 2 * SOLVE_MAXR
  int last_refine_iters = 0;
  int last_cg_iters = 0;      // of those, conjugate-gradient iterations (refinement stalled)
  int* flags = nullptr;       // nsub + nsb (sub-tiles, forward blocks) + scratch
  int* claim = nullptr;       // reserved-SM claims of a split factor launch
  stiles::dev::Ctl* ctl = nullptr;  // [0] factor, [1] forward, [2] backward
  double* logdet_part = nullptr;    // LOGDET_BLOCKS + 1
  // solve workspace (grown on demand)
  double* Y = nullptr;
  double* sscratch = nullptr;
  int* sflags = nullptr;
  int64_t solve_nr = 0;
  double* bstage = nullptr;   // host-input staging (n * nrhs)
  double* xstage = nullptr;
  double* ywork = nullptr;    // residual work n * nr
  double* norms = nullptr;    // 2 * SOLVE_MAXR
  int64_t stage_elems = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // call start, persistent kernel start / end
  long long* trace[4] = {nullptr, nullptr, nullptr, nullptr};  // per-ticket stamps: factor, forward, backward,
                                                              // selected inverse (allocated at its launch)
  bool trace_on = false;
  unsigned long long* info = nullptr;  // first bad pivot column (&ctl[0].info, or a batch slot)
  bool view = false;                   // tiles and values belong to a stiles_batch
  bool pending = false;
  // selected inverse (allocated on first use): Sigma and U sub-tiles, Sigma flags
  double* sigma = nullptr;
  double* sigmaT = nullptr;            // Sigma's sub-tiles transposed
  double* sinv_u = nullptr;            // (L_jk L_kk^{-1})^T
  double* sinv_w = nullptr;            // Sigma_jk^T L_jk L_kk^{-1} (terms of Sigma_kk)
  double* sinv_x = nullptr;            // Sigma_mp^T L_mc L_cc^{-1}, p the parent of c (terms of Sigma_pc)
  int* sinv_flags = nullptr;
  stiles::dev::Ctl* sinv_ctl = nullptr;
  bool sinv_valid = false;             // Sigma belongs to the current factorization
};

namespace {

using namespace stiles;

void free_graph(DevGraph& g) {
  cudaFree(g.chain);
  cudaFree(g.bulk);
  cudaFree(g.tasks);
  cudaFree(g.stasks);
  cudaFree(g.pairs);
  cudaFree(g.parts);
  g = DevGraph{};
}

void free_dev_plan(stiles_plan* p) {
  if (!p->dev) return;
  DevPlan* d = p->dev;
  cudaFree(d->scatter);
  cudaFree(d->pad);
  cudaFree(d->perm);
  cudaFree(d->diag_sub);
  cudaFree(d->colptr);
  cudaFree(d->rowidx);
  cudaFree(d->rptr);
  cudaFree(d->rcol);
  cudaFree(d->rval);
  free_graph(d->fac);
  free_graph(d->fwd);
  free_graph(d->bwd);
  free_graph(d->fus);
  cudaFree(d->sinv_tasks);
  cudaFree(d->sinv_pairs);
  cudaFree(d->sinv_loads);
  cudaFree(d->sinv_posts);
  cudaFree(d->sinv_ulist);
  delete d;
  p->dev = nullptr;
}

template <int B>
cudaError_t factor_occupancy(int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(dev::factor_f64_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(dev::FactorCfg<B>::SMEM));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::factor_f64_kernel<B>, 128, dev::FactorCfg<B>::SMEM);
}

template <int B, typename TF>
cudaError_t solve_occupancy(int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(dev::solve_kernel<B, false, TF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(dev::SolveCfg<B, TF>::SMEM));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(dev::solve_kernel<B, true, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(dev::SolveCfg<B, TF>::SMEM));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::solve_kernel<B, false, TF>, 128,
                                                       dev::SolveCfg<B, TF>::SMEM);
}

std::mutex g_plan_mutex;  // plans are shared between threads (plan caches); uploads happen once

// SMs reserved for the diagonal chain of a one-matrix FP64 factor launch (one
// CTA each, alone on its SM, so its POTRF does not share the SM's FP64 pipe
// with band updates); used when the launch has at least two CTAs per SM.
#ifndef STILES_CHAIN_SMS
#define STILES_CHAIN_SMS 8
#endif
constexpr int kChainSms = STILES_CHAIN_SMS;
// reserved SMs of a sliced-update launch: one chain slot each (at least the two chains of a
// nested dissection, plus slots that prefetch the next chain tasks' operands)
#ifndef STILES_OZ_CHAIN_SMS
#define STILES_OZ_CHAIN_SMS 4
#endif
constexpr int kOzChainSms = STILES_OZ_CHAIN_SMS;
static_assert(kOzChainSms <= kChainSms, "the claim array holds kChainSms entries");

#ifndef STILES_SOLVE_CTAS_PER_MATRIX
#define STILES_SOLVE_CTAS_PER_MATRIX 128
#endif
constexpr int kSolveCtasPerMatrix = STILES_SOLVE_CTAS_PER_MATRIX;  // persistent CTAs per matrix of a solve launch

stiles_status ensure_dev_plan(const stiles_plan* cp) {
  std::lock_guard<std::mutex> lock(g_plan_mutex);
  stiles_plan* p = const_cast<stiles_plan*>(cp);
  int device = 0;
  CUDA_TRY(cudaGetDevice(&device));
  if (p->dev) {
    if (p->dev->device != device) return fail(STILES_ERR_INVALID, "plan was uploaded to another device");
    return STILES_OK;
  }
  if (!p->executable) return fail(STILES_ERR_UNSUPPORTED, "tile size must be a multiple of 16 to factorize");
  DevPlan* d = new (std::nothrow) DevPlan();
  if (!d) return fail(STILES_ERR_NOMEM, "host allocation");
  p->dev = d;
  d->device = device;
  auto chk = [&](cudaError_t e) { return e == cudaSuccess; };
  bool ok = chk(upload(&d->scatter, p->scatter)) && chk(upload(&d->pad, p->pad)) && chk(upload(&d->perm, p->perm)) &&
            chk(upload(&d->diag_sub, p->diag_sub)) && chk(upload(&d->colptr, p->colptr)) &&
            chk(upload(&d->rowidx, p->rowidx)) && chk(upload(&d->rptr, p->rptr)) && chk(upload(&d->rcol, p->rcol)) &&
            chk(upload(&d->rval, p->rval)) && chk(upload(&d->fac.tasks, p->graph.tasks)) &&
            chk(upload(&d->fac.chain, p->chain_order)) && chk(upload(&d->fac.bulk, p->bulk_order)) &&
            chk(upload(&d->fac.pairs, p->graph.pairs)) && chk(upload(&d->fac.parts, p->graph.parts)) &&
            chk(upload(&d->fwd.stasks, p->fwd.tasks)) && chk(upload(&d->fwd.pairs, p->fwd.pairs)) &&
            chk(upload(&d->fwd.parts, p->fwd.parts)) && chk(upload(&d->bwd.stasks, p->bwd.tasks)) &&
            chk(upload(&d->bwd.pairs, p->bwd.pairs)) && chk(upload(&d->bwd.parts, p->bwd.parts));
  if (!ok) {
    cudaError_t e = cudaGetLastError();
    free_dev_plan(p);
    return fail(e == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,
                std::string("plan upload: ") + cudaGetErrorString(e));
  }
  d->fac.ntasks = int(p->graph.tasks.size());
  d->fwd.ntasks = int(p->fwd.tasks.size());
  d->bwd.ntasks = int(p->bwd.tasks.size());
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  int fb = 0, sb = 0;
  cudaError_t e = cudaSuccess;
  if (p->opts.precision == STILES_PREC_SLICED) {
    e = cudaFuncSetAttribute(dev::factor_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(dev::OZ_KERNEL_SMEM));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fb, dev::factor_oz_kernel, dev::OZ_THREADS, dev::OZ_KERNEL_SMEM);
    // each resident CTA holds all 512 TMEM columns of its SM
    fb = std::min(fb, 1);
    if (e == cudaSuccess) e = solve_occupancy<32, float>(&sb);
  } else if (p->opts.precision != STILES_PREC_F64) {
    e = cudaFuncSetAttribute(dev::factor_lp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(dev::LP_KERNEL_SMEM));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fb, dev::factor_lp_kernel, dev::LP_THREADS, dev::LP_KERNEL_SMEM);
    // each resident CTA holds 128 TMEM columns of the SM's 512
    fb = std::min(fb, 4);
    if (e == cudaSuccess) e = solve_occupancy<64, float>(&sb);
  } else switch (p->B) {
    case 16: e = factor_occupancy<16>(&fb); if (e == cudaSuccess) e = solve_occupancy<16, double>(&sb); break;
    case 32: e = factor_occupancy<32>(&fb); if (e == cudaSuccess) e = solve_occupancy<32, double>(&sb); break;
    case 64: e = factor_occupancy<64>(&fb); if (e == cudaSuccess) e = solve_occupancy<64, double>(&sb); break;
    default: return fail(STILES_ERR_UNSUPPORTED, "block size");
  }
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("occupancy: ") + cudaGetErrorString(e));
  if (fb < 1 || sb < 1) return fail(STILES_ERR_UNSUPPORTED, "kernel does not fit on an SM");
  if (p->opts.ctas_per_sm > 0) {
    fb = std::min(fb, int(p->opts.ctas_per_sm));
    sb = std::min(sb, int(p->opts.ctas_per_sm));
  }
  d->grid_factor = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(fb) * sms, d->fac.ntasks)));
  // a sweep is a few dependency chains (two per nested-dissection level plus the
  // arrow tree): a small grid keeps them fed and leaves the other SMs to
  // concurrent launches (a waiting persistent CTA holds its SM slot)
  d->grid_solve = int(std::max<int64_t>(
      1, std::min<int64_t>({int64_t(sb) * sms, int64_t(kSolveCtasPerMatrix), std::max(d->fwd.ntasks, d->bwd.ntasks)})));
  return STILES_OK;
}

void free_factor(stiles_factor* f) {
  if (!f) return;
  if (f->view) {  // the batch owns the factor arrays; only the solve workspace is the view's
    f->values = f->tiles = f->scratch = f->invdiag = f->ldiag = f->linv = nullptr;
    f->tiles32 = f->scratch32 = f->invdiag32 = f->linv32 = nullptr;
    f->tiles16 = nullptr;
    f->slices = nullptr;
    f->rowexp = nullptr;
    f->flags = nullptr;
    f->ctl = nullptr;
    f->logdet_part = f->norms = nullptr;
  }
  cudaFree(f->values);
  cudaFree(f->tiles);
  cudaFree(f->scratch);
  cudaFree(f->invdiag);
  cudaFree(f->linv);
  cudaFree(f->linv32);
  cudaFree(f->slices);
  cudaFree(f->rowexp);
  cudaFree(f->tiles32);
  cudaFree(f->tiles16);
  cudaFree(f->scratch32);
  cudaFree(f->invdiag32);
  cudaFree(f->ldiag);
  cudaFree(f->irwork);
  cudaFree(f->cgs);
  cudaFree(f->flags);
  cudaFree(f->claim);
  cudaFree(f->ctl);
  cudaFree(f->logdet_part);
  cudaFree(f->Y);
  cudaFree(f->sscratch);
  cudaFree(f->sflags);
  cudaFree(f->bstage);
  cudaFree(f->xstage);
  cudaFree(f->ywork);
  cudaFree(f->norms);
  cudaFree(f->sigma);
  cudaFree(f->sigmaT);
  cudaFree(f->sinv_u);
  cudaFree(f->sinv_w);
  cudaFree(f->sinv_x);
  cudaFree(f->sinv_flags);
  cudaFree(f->sinv_ctl);
  if (f->done) cudaEventDestroy(f->done);
  for (cudaEvent_t e : f->ev)
    if (e) cudaEventDestroy(e);
  for (long long* t : f->trace) cudaFree(t);
  delete f;
}

stiles_status alloc_factor(const stiles_plan* p, stiles_factor** out) {
  stiles_factor* f = new (std::nothrow) stiles_factor();
  if (!f) return fail(STILES_ERR_NOMEM, "host allocation");
  f->plan = p;
  cudaGetDevice(&f->device);
  const size_t tile = size_t(p->B) * p->B;
  // scratch and flags also cover the factorization with the forward sweep
  // folded in: nsb more tiles (the right-hand-side blocks) and its partials
  const int64_t nscr = std::max<int64_t>(p->graph.nscratch + p->fwd.nscratch, 1);
  f->sliced = p->opts.precision == STILES_PREC_SLICED;
  f->lp = p->opts.precision != STILES_PREC_F64 && !f->sliced;
  cudaError_t e = cudaMalloc(&f->values, size_t(p->nnz) * sizeof(double));
  if (!f->lp) {
    if (e == cudaSuccess) e = cudaMalloc(&f->tiles, size_t(p->nsub + p->nsb) * tile * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->scratch, size_t(nscr) * tile * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->invdiag, size_t(p->nsb) * p->B * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->linv, 5 * size_t(p->nsb) * tile * sizeof(double));
    if (f->sliced && e == cudaSuccess) e = cudaMalloc(&f->slices, size_t(p->nsub) * dev::OZ_OP_BYTES);
    if (f->sliced && e == cudaSuccess) e = cudaMalloc(&f->rowexp, size_t(p->nsb) * p->B * sizeof(int));
    // sliced factors: FP32 copies for the sweeps (refined in FP64)
    if (f->sliced && e == cudaSuccess) e = cudaMalloc(&f->tiles32, size_t(p->nsub) * tile * sizeof(float));
    if (f->sliced && e == cudaSuccess) e = cudaMalloc(&f->invdiag32, size_t(p->nsb) * p->B * sizeof(float));
    if (f->sliced && e == cudaSuccess) e = cudaMalloc(&f->linv32, size_t(p->nsb) * tile * sizeof(float));
  } else {
    if (e == cudaSuccess) e = cudaMalloc(&f->tiles32, size_t(p->nsub) * tile * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->tiles16, size_t(p->nsub) * tile * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&f->scratch32, size_t(nscr) * tile * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->invdiag32, size_t(p->nsb) * p->B * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->ldiag, size_t(p->nsb) * p->B * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->linv32, size_t(p->nsb) * tile * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&f->flags, size_t(p->nsub + p->nsb + nscr) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&f->ctl, 3 * sizeof(dev::Ctl));
  if (e == cudaSuccess) e = cudaMalloc(&f->claim, kChainSms * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&f->logdet_part, (dev::LOGDET_BLOCKS + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&f->norms, 2 * dev::SOLVE_MAXR * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&f->ev[i]);
  if (e != cudaSuccess) {
    free_factor(f);
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,
                std::string("factor allocation: ") + cudaGetErrorString(e));
  }
  f->info = &f->ctl[0].info;
  *out = f;
  return STILES_OK;
}

dev::MatCtx mat_ctx(const stiles_plan* p, stiles_factor* f, bool fused = false) {
  dev::MatCtx c;
  const DevGraph& g = fused ? p->dev->fus : p->dev->fac;
  c.tiles = f->tiles;
  c.scratch = f->scratch;
  c.invdiag = f->invdiag;
  c.tasks = g.tasks;
  c.pairs = g.pairs;
  c.parts = g.parts;
  c.flags = f->flags;
  c.sflags = f->flags + p->nsub + p->nsb;
  c.info = f->info;
  c.trace = f->trace[0];
  return c;
}

dev::LPMatCtx lp_mat_ctx(const stiles_plan* p, stiles_factor* f) {
  dev::LPMatCtx c;
  c.tiles32 = f->tiles32;
  c.tiles16 = f->tiles16;
  c.scratch = f->scratch32;
  c.invdiag32 = f->invdiag32;
  c.ldiag = f->ldiag;
  c.tasks = p->dev->fac.tasks;
  c.pairs = p->dev->fac.pairs;
  c.parts = p->dev->fac.parts;
  c.flags = f->flags;
  c.sflags = f->flags + p->nsub + p->nsb;
  c.info = f->info;
  c.trace = f->trace[0];
  return c;
}

template <int B>
cudaError_t launch_factor(const stiles_plan* p, stiles_factor* f, cudaStream_t s, bool fused = false) {
  dev::FactorArgs a{};
  const DevGraph& g = fused ? p->dev->fus : p->dev->fac;
  a.single = mat_ctx(p, f, fused);
  if (fused) a.single.trace = nullptr;  // the trace array is sized for the plain factorization
  a.mats = nullptr;
  a.tickets = nullptr;
  a.ntasks = g.ntasks;
  a.ctl = f->ctl;
  a.spin_limit = p->opts.spin_limit;
  a.chain = g.chain;
  a.bulk = g.bulk;
  a.nchain = int(fused ? p->fused_chain.size() : p->chain_order.size());
  a.nbulk = int(fused ? p->fused_bulk.size() : p->bulk_order.size());
  a.sm_claim = f->claim;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
  // split only when every SM hosts several CTAs and both queues have work
  a.chain_sms = (p->split_queues && p->dev->grid_factor >= 2 * sms && sms > kChainSms && a.nchain > 0 && a.nbulk > 0)
                    ? kChainSms : 0;
  if (a.chain_sms) {
    cudaError_t e = cudaMemsetAsync(f->claim, 0, kChainSms * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  dev::factor_f64_kernel<B><<<p->dev->grid_factor, 128, dev::FactorCfg<B>::SMEM, s>>>(a);
  return cudaGetLastError();
}

dev::OZMatCtx oz_mat_ctx(const stiles_plan* p, stiles_factor* f) {
  dev::OZMatCtx c;
  c.tiles = f->tiles;
  c.slices = f->slices;
  c.scratch = f->scratch;
  c.invdiag = f->invdiag;
  c.rowexp = f->rowexp;
  c.tasks = p->dev->fac.tasks;
  c.pairs = p->dev->fac.pairs;
  c.parts = p->dev->fac.parts;
  c.flags = f->flags;
  c.sflags = f->flags + p->nsub + p->nsb;
  c.info = f->info;
  c.trace = f->trace[0];
  return c;
}

// the sliced-update factorization: row scales from the scattered diagonal, then the persistent kernel
cudaError_t launch_factor_oz(const stiles_plan* p, stiles_factor* f, cudaStream_t s) {
  dev::oz_rowexp_kernel<<<grid_for(p->nsb * p->B, 256), 256, 0, s>>>(f->tiles, p->dev->diag_sub, p->nsb, f->rowexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dev::OZArgs a;
  a.single = oz_mat_ctx(p, f);
  a.mats = nullptr;
  a.tickets = nullptr;
  a.ntasks = p->dev->fac.ntasks;
  a.ctl = f->ctl;
  a.spin_limit = p->opts.spin_limit;
  // the diagonal chain on reserved SMs (one chain slot per SM) when the graph has both queues
  a.chain = p->dev->fac.chain;
  a.bulk = p->dev->fac.bulk;
  a.nchain = int(p->chain_order.size());
  a.nbulk = int(p->bulk_order.size());
  a.sm_claim = f->claim;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device);
  a.chain_sms = (p->dev->grid_factor >= sms && sms > 4 * kOzChainSms && a.nchain > 0 && a.nbulk > 0) ? kOzChainSms : 0;
  if (a.chain_sms) {
    e = cudaMemsetAsync(f->claim, 0, kChainSms * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  dev::factor_oz_kernel<<<p->dev->grid_factor, dev::OZ_THREADS, dev::OZ_KERNEL_SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_factor_lp(const stiles_plan* p, stiles_factor* f, cudaStream_t s) {
  dev::LPArgs a;
  a.single = lp_mat_ctx(p, f);
  a.mats = nullptr;
  a.tickets = nullptr;
  a.ntasks = p->dev->fac.ntasks;
  a.ctl = f->ctl;
  a.spin_limit = p->opts.spin_limit;
  a.fp16 = p->opts.precision == STILES_PREC_F16 ? 1 : 0;
  dev::factor_lp_kernel<<<p->dev->grid_factor, dev::LP_THREADS, dev::LP_KERNEL_SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diag_inverse(const stiles_plan* p, stiles_factor* f, cudaStream_t st) {
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>((p->nsb * 32 + 255) / 256, 148 * 16)));
  if (f->lp) {
    dev::diag_inverse_kernel<64, float><<<grid, 256, 0, st>>>(f->linv32, f->tiles32, f->invdiag32,
                                                              p->dev->diag_sub, p->nsb);
  } else {
    switch (p->B) {
      case 16:
        dev::diag_inverse_kernel<16, double><<<grid, 256, 0, st>>>(f->linv, f->tiles, f->invdiag, p->dev->diag_sub,
                                                                   p->nsb);
        break;
      case 32:
        dev::diag_inverse_kernel<32, double><<<grid, 256, 0, st>>>(f->linv, f->tiles, f->invdiag, p->dev->diag_sub,
                                                                   p->nsb);
        break;
      default:
        dev::diag_inverse_kernel<64, double><<<grid, 256, 0, st>>>(f->linv, f->tiles, f->invdiag, p->dev->diag_sub,
                                                                   p->nsb);
        break;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || f->lp) return e;
  if (f->sliced) {
    // the sweeps of a sliced-update factor run in FP32 and are refined in FP64:
    // an FP32 copy of its tiles and the inverses of that copy's diagonal blocks
    // (the FP64 inverses above serve the selected inverse)
    const int64_t ne = p->nsub * int64_t(p->B) * p->B;
    dev::to_f32_kernel<<<grid_for(ne, 256), 256, 0, st>>>(f->tiles32, f->tiles, ne);
    dev::to_f32_kernel<<<grid_for(p->nsb * p->B, 256), 256, 0, st>>>(f->invdiag32, f->invdiag, p->nsb * p->B);
    dev::diag_inverse_kernel<32, float><<<grid, 256, 0, st>>>(f->linv32, f->tiles32, f->invdiag32, p->dev->diag_sub,
                                                              p->nsb);
    return cudaGetLastError();
  }
  // then the folded newest terms of every sweep task (reads the inverses; FP64 factors)
  const size_t nt = size_t(p->nsb) * p->B * p->B;
  dev::MlastDesc md{};
  md.mlast = f->linv + nt;
  md.mlast2 = f->linv + 3 * nt;
  md.linv = f->linv;
  md.tiles = f->tiles;
  md.ftasks = p->dev->fwd.stasks;
  md.fpairs = p->dev->fwd.pairs;
  md.btasks = p->dev->bwd.stasks;
  md.bpairs = p->dev->bwd.pairs;
  md.nf = p->dev->fwd.ntasks;
  md.nb = p->dev->bwd.ntasks;
  md.nsb = p->nsb;
  const int gm = std::max(1, std::min(2 * (md.nf + md.nb), 148 * 8));
  switch (p->B) {
    case 16: dev::mlast_kernel<16, double><<<gm, 128, 0, st>>>(md); break;
    case 32: dev::mlast_kernel<32, double><<<gm, 128, 0, st>>>(md); break;
    default: dev::mlast_kernel<64, double><<<gm, 128, 0, st>>>(md); break;
  }
  return cudaGetLastError();
}

template <typename TF>
dev::SolveCtx<TF> solve_ctx(const stiles_plan* p, stiles_factor* f, bool backward, int nr, const TF* tiles,
                            const TF* invdiag, const TF* linv, TF* Y, TF* scratch, int* flags) {
  const int64_t nf = std::max<int64_t>(p->fwd.nscratch, 1);
  dev::SolveCtx<TF> c;
  c.tiles = tiles;
  c.invdiag = invdiag;
  c.linv = linv;
  // folded sweep terms for FP64 factors only: the FP32 sweeps of a mixed-precision
  // factor have short FMA chains, and their batches would pay the products' cost
  const bool fold = sizeof(TF) == sizeof(double);
  c.mlast = fold ? linv + (backward ? 2 : 1) * size_t(p->nsb) * p->B * p->B : nullptr;
  c.mlast2 = fold ? linv + (backward ? 4 : 3) * size_t(p->nsb) * p->B * p->B : nullptr;
  c.Y = Y;
  c.nr = nr;
  c.pad0 = 0;
  if (!backward) {
    c.scratch = scratch;
    c.tasks = p->dev->fwd.stasks;
    c.pairs = p->dev->fwd.pairs;
    c.parts = p->dev->fwd.parts;
    c.flags = flags;
    c.sflags = flags + p->nsb;
    c.trace = f ? f->trace[1] : nullptr;
  } else {
    c.scratch = scratch + size_t(nf) * p->B * dev::SOLVE_MAXR;
    c.tasks = p->dev->bwd.stasks;
    c.pairs = p->dev->bwd.pairs;
    c.parts = p->dev->bwd.parts;
    c.flags = flags + p->nsb + nf;
    c.sflags = flags + 2 * p->nsb + nf;
    c.trace = f ? f->trace[2] : nullptr;
  }
  return c;
}

template <int B, typename TF>
cudaError_t launch_solve(const stiles_plan* p, stiles_factor* f, cudaStream_t s, int nr, const TF* tiles,
                         const TF* invdiag, const TF* linv) {
  dev::SolveArgs<TF> a{};
  a.mats = nullptr;
  a.tickets = nullptr;
  a.spin_limit = p->opts.spin_limit;
  TF* Y = reinterpret_cast<TF*>(f->Y);  // the double-sized workspaces also hold FP32 sweeps
  TF* scr = reinterpret_cast<TF*>(f->sscratch);
  a.single = solve_ctx<TF>(p, f, false, nr, tiles, invdiag, linv, Y, scr, f->sflags);
  a.ntasks = p->dev->fwd.ntasks;
  a.ctl = f->ctl + 1;
  dev::solve_kernel<B, false, TF><<<p->dev->grid_solve, 128, dev::SolveCfg<B, TF>::SMEM, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  a.single = solve_ctx<TF>(p, f, true, nr, tiles, invdiag, linv, Y, scr, f->sflags);
  a.ntasks = p->dev->bwd.ntasks;
  a.ctl = f->ctl + 2;
  dev::solve_kernel<B, true, TF><<<p->dev->grid_solve, 128, dev::SolveCfg<B, TF>::SMEM, s>>>(a);
  return cudaGetLastError();
}

// The backward sweep alone (the forward one having run inside the factorization).
template <int B>
cudaError_t launch_backward(const stiles_plan* p, stiles_factor* f, cudaStream_t s, int nr) {
  dev::SolveArgs<double> a{};
  a.mats = nullptr;
  a.tickets = nullptr;
  a.spin_limit = p->opts.spin_limit;
  a.single = solve_ctx<double>(p, f, true, nr, f->tiles, f->invdiag, f->linv, f->Y, f->sscratch, f->sflags);
  a.ntasks = p->dev->bwd.ntasks;
  a.ctl = f->ctl + 2;
  dev::solve_kernel<B, true, double><<<p->dev->grid_solve, 128, dev::SolveCfg<B, double>::SMEM, s>>>(a);
  return cudaGetLastError();
}

stiles_status read_ctl(stiles_factor* f, int idx, int64_t* info) {
  dev::Ctl c;
  CUDA_TRY(cudaMemcpy(&c, f->ctl + idx, sizeof(c), cudaMemcpyDeviceToHost));
  if (info) *info = (c.info == ~0ull) ? 0 : int64_t(c.info);
  if (c.status != 0) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "device wait timed out (launch %d, ticket %lld)", idx, c.where);
    return fail(STILES_ERR_TIMEOUT, buf);
  }
  if (c.info != ~0ull) return fail(STILES_ERR_NOT_SPD, "matrix is not positive definite");
  return STILES_OK;
}

}  // namespace

extern "C" {

void stiles_default_opts(stiles_opts* opts) {
  if (opts) stiles::default_opts(opts);
}

const char* stiles_last_error(void) { return g_last_error.c_str(); }

const char* stiles_strerror(stiles_status s) {
  switch (s) {
    case STILES_OK: return "ok";
    case STILES_ERR_INVALID: return "invalid argument or input";
    case STILES_ERR_NOT_SPD: return "matrix is not positive definite";
    case STILES_ERR_NOMEM: return "out of memory";
    case STILES_ERR_CUDA: return "CUDA error";
    case STILES_ERR_TIMEOUT: return "device wait timed out";
    case STILES_ERR_NOT_CONVERGED: return "iterative refinement did not converge";
    case STILES_ERR_UNSUPPORTED: return "unsupported option";
  }
  return "unknown status";
}

stiles_status stiles_analyze(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                             const stiles_opts* opts, stiles_plan** out) {
  if (!out) return fail(STILES_ERR_INVALID, "out is NULL");
  *out = nullptr;
  stiles_opts o;
  if (opts) o = *opts;
  else stiles::default_opts(&o);
  stiles_plan* p = new (std::nothrow) stiles_plan();
  if (!p) return fail(STILES_ERR_NOMEM, "host allocation");
  std::string err;
  stiles_status s;
  try {
    s = stiles::build_plan(n, colptr, rowidx, n_arrow, o, p, &err);
  } catch (const std::bad_alloc&) {
    s = STILES_ERR_NOMEM;
    err = "host allocation during analysis";
  } catch (const std::exception& ex) {
    s = STILES_ERR_INVALID;
    err = ex.what();
  }
  if (s != STILES_OK) {
    delete p;
    return fail(s, err);
  }
  *out = p;
  return STILES_OK;
}

stiles_status stiles_plan_get_info(const stiles_plan* p, stiles_plan_info* info) {
  if (!p || !info) return fail(STILES_ERR_INVALID, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->n = p->n;
  info->n_arrow = p->n_arrow;
  info->nnz = p->nnz;
  info->tile = p->T;
  info->nt = p->nt;
  info->nnzt = p->nnzt;
  info->block = p->executable ? p->B : 0;
  info->nsub = p->nsub;
  info->ntasks = int64_t(p->graph.tasks.size());
  info->npairs = int64_t(p->graph.pairs.size() / 2);
  info->nscratch = p->graph.nscratch;
  info->flops_potrf = p->flops_potrf;
  info->flops_syrk = p->flops_syrk;
  info->flops_gemm = p->flops_gemm;
  info->flops_trsm = p->flops_trsm;
  info->flops_total = p->flops_potrf + p->flops_syrk + p->flops_gemm + p->flops_trsm;
  // FP64 tiles; 16-bit factors hold FP32 tiles plus a 16-bit copy (the same 6 B per entry are
  // counted as 8); sliced factors add four 2-byte digit slices and an FP32 copy per entry
  info->factor_bytes = p->nsub * int64_t(p->B) * p->B *
                       int64_t(p->opts.precision == STILES_PREC_SLICED ? 20 : sizeof(double));
  info->ordering_used = p->ordering_used;
  info->chain_split = (p->split_queues && p->opts.precision == STILES_PREC_F64) ? 1 : 0;
  return STILES_OK;
}

stiles_status stiles_plan_perm(const stiles_plan* p, int64_t* perm) {
  if (!p || !perm) return fail(STILES_ERR_INVALID, "null argument");
  std::memcpy(perm, p->perm.data(), p->perm.size() * sizeof(int64_t));
  return STILES_OK;
}

stiles_status stiles_plan_tilemap(const stiles_plan* p, int64_t* tcolptr, int32_t* trowidx) {
  if (!p) return fail(STILES_ERR_INVALID, "null plan");
  if (tcolptr) std::memcpy(tcolptr, p->tcolptr.data(), p->tcolptr.size() * sizeof(int64_t));
  if (trowidx) std::memcpy(trowidx, p->trowidx.data(), p->trowidx.size() * sizeof(int32_t));
  return STILES_OK;
}

void stiles_plan_destroy(stiles_plan* p) {
  if (!p) return;
  free_dev_plan(p);
  delete p;
}

void stiles_factor_destroy(stiles_factor* f) { free_factor(f); }

stiles_status stiles_factorize_async(const stiles_plan* p, const double* values, void* stream, stiles_factor** inout) {
  if (!p || !values || !inout) return fail(STILES_ERR_INVALID, "null argument");
  stiles_status s = ensure_dev_plan(p);
  if (s != STILES_OK) return s;
  stiles_factor* f = *inout;
  if (f && f->plan != p) return fail(STILES_ERR_INVALID, "factor belongs to another plan");
  if (f && f->view) return fail(STILES_ERR_INVALID, "a factor of a batch is factorized through its batch");
  if (!f) {
    s = alloc_factor(p, &f);
    if (s != STILES_OK) return s;
    *inout = f;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  f->stream = st;
  const size_t tile = size_t(p->B) * p->B;
  const int64_t nscr = std::max<int64_t>(p->graph.nscratch + p->fwd.nscratch, 1);
  CUDA_TRY(cudaEventRecord(f->ev[0], st));
  CUDA_TRY(cudaMemcpyAsync(f->values, values, size_t(p->nnz) * sizeof(double), cudaMemcpyDefault, st));
  if (!f->lp) {
    CUDA_TRY(cudaMemsetAsync(f->tiles, 0, size_t(p->nsub) * tile * sizeof(double), st));
    dev::scatter_kernel<<<grid_for(p->nnz, 256), 256, 0, st>>>(f->tiles, f->values, p->dev->scatter, p->nnz);
    CUDA_TRY(cudaGetLastError());
    if (!p->pad.empty()) {
      dev::set_ones_kernel<double><<<1, 128, 0, st>>>(f->tiles, p->dev->pad, int64_t(p->pad.size()));
      CUDA_TRY(cudaGetLastError());
    }
  } else {
    CUDA_TRY(cudaMemsetAsync(f->tiles32, 0, size_t(p->nsub) * tile * sizeof(float), st));
    dev::scatter_f32_kernel<<<grid_for(p->nnz, 256), 256, 0, st>>>(f->tiles32, f->values, p->dev->scatter, p->nnz);
    CUDA_TRY(cudaGetLastError());
    if (!p->pad.empty()) {
      dev::set_ones_kernel<float><<<1, 128, 0, st>>>(f->tiles32, p->dev->pad, int64_t(p->pad.size()));
      CUDA_TRY(cudaGetLastError());
    }
  }
  CUDA_TRY(cudaMemsetAsync(f->flags, 0, size_t(p->nsub + p->nsb + nscr) * sizeof(int), st));
  dev::init_ctl_kernel<<<1, 32, 0, st>>>(f->ctl, 1);
  CUDA_TRY(cudaGetLastError());
  count_launch(p->pad.empty() ? 2 : 3);
  CUDA_TRY(cudaEventRecord(f->ev[1], st));
  cudaError_t e;
  if (f->lp) e = launch_factor_lp(p, f, st);
  else if (f->sliced) e = launch_factor_oz(p, f, st);
  else switch (p->B) {
    case 16: e = launch_factor<16>(p, f, st); break;
    case 32: e = launch_factor<32>(p, f, st); break;
    default: e = launch_factor<64>(p, f, st); break;
  }
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("factor launch: ") + cudaGetErrorString(e));
  count_launch(f->sliced ? 2 : 1);
  CUDA_TRY(cudaEventRecord(f->ev[2], st));
  // inverses of the diagonal blocks for the sweeps (after the kernel's timing window)
  e = launch_diag_inverse(p, f, st);
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("diagonal inverses: ") + cudaGetErrorString(e));
  count_launch(f->lp ? 1 : (f->sliced ? 4 : 2));
  CUDA_TRY(cudaEventRecord(f->done, st));
  f->pending = true;
  f->sinv_valid = false;
  return STILES_OK;
}

stiles_status stiles_factor_wait(stiles_factor* f, int64_t* info) {
  if (!f) return fail(STILES_ERR_INVALID, "null factor");
  if (f->view) return fail(STILES_ERR_INVALID, "a factor of a batch is waited on through its batch");
  if (info) *info = 0;
  CUDA_TRY(cudaEventSynchronize(f->done));
  f->pending = false;
  return read_ctl(f, 0, info);
}

stiles_status stiles_factorize(const stiles_plan* p, const double* values, void* stream, stiles_factor** inout,
                               int64_t* info) {
  if (info) *info = 0;
  stiles_status s = stiles_factorize_async(p, values, stream, inout);
  if (s != STILES_OK) return s;
  return stiles_factor_wait(*inout, info);
}

stiles_status stiles_factorize_solve(const stiles_plan* p, const double* values, const double* b, double* x,
                                     int32_t nrhs, int64_t ld, void* stream, stiles_factor** inout, int64_t* info) {
  if (info) *info = 0;
  if (!p || !values || !b || !x || !inout) return fail(STILES_ERR_INVALID, "null argument");
  if (p->opts.precision != STILES_PREC_F64)
    return fail(STILES_ERR_UNSUPPORTED, "the forward sweep is folded into FP64 factorizations only");
  if (nrhs < 1 || nrhs > std::min<int64_t>(p->B, dev::SOLVE_MAXR) || ld < p->n)
    return fail(STILES_ERR_INVALID, "nrhs must be 1 .. min(B, 16) and ld >= n");
  if (!is_device_ptr(b) || !is_device_ptr(x)) return fail(STILES_ERR_INVALID, "b and x must be device memory");
  stiles_status s = ensure_dev_plan(p);
  if (s != STILES_OK) return s;
  {
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    stiles_plan* pm = const_cast<stiles_plan*>(p);
    std::string err;
    s = build_fused(pm, &err);
    if (s != STILES_OK) return fail(s, err);
    DevPlan* d = pm->dev;
    if (!d->fus_ready) {
      cudaError_t e = upload(&d->fus.tasks, pm->fused.tasks);
      if (e == cudaSuccess) e = upload(&d->fus.pairs, pm->fused.pairs);
      if (e == cudaSuccess) e = upload(&d->fus.parts, pm->fused.parts);
      if (e == cudaSuccess) e = upload(&d->fus.chain, pm->fused_chain);
      if (e == cudaSuccess) e = upload(&d->fus.bulk, pm->fused_bulk);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,
                    std::string("folded graph upload: ") + cudaGetErrorString(e));
      }
      d->fus.ntasks = int(pm->fused.tasks.size());
      d->fus_ready = true;
    }
  }
  stiles_factor* f = *inout;
  if (f && f->plan != p) return fail(STILES_ERR_INVALID, "factor belongs to another plan");
  if (f && f->view) return fail(STILES_ERR_INVALID, "a factor of a batch is factorized through its batch");
  if (!f) {
    s = alloc_factor(p, &f);
    if (s != STILES_OK) return s;
    *inout = f;
  }
  const int64_t n = p->n, B = p->B;
  const int64_t nf = std::max<int64_t>(p->fwd.nscratch, 1), nb = std::max<int64_t>(p->bwd.nscratch, 1);
  if (f->solve_nr < dev::SOLVE_MAXR) {
    cudaFree(f->Y);
    cudaFree(f->sscratch);
    cudaFree(f->sflags);
    cudaFree(f->ywork);
    f->Y = f->sscratch = f->ywork = nullptr;
    f->sflags = nullptr;
    f->solve_nr = 0;
    CUDA_TRY(cudaMalloc(&f->Y, size_t(p->nsb) * B * dev::SOLVE_MAXR * sizeof(double)));
    CUDA_TRY(cudaMalloc(&f->sscratch, size_t(nf + nb) * B * dev::SOLVE_MAXR * sizeof(double)));
    CUDA_TRY(cudaMalloc(&f->sflags, size_t(2 * p->nsb + nf + nb) * sizeof(int)));
    CUDA_TRY(cudaMalloc(&f->ywork, size_t(n) * dev::SOLVE_MAXR * sizeof(double)));
    f->solve_nr = dev::SOLVE_MAXR;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  f->stream = st;
  const size_t tile = size_t(B) * B;
  const int64_t nscr = std::max<int64_t>(p->graph.nscratch + p->fwd.nscratch, 1);
  CUDA_TRY(cudaEventRecord(f->ev[0], st));
  CUDA_TRY(cudaMemcpyAsync(f->values, values, size_t(p->nnz) * sizeof(double), cudaMemcpyDefault, st));
  CUDA_TRY(cudaMemsetAsync(f->tiles, 0, size_t(p->nsub + p->nsb) * tile * sizeof(double), st));
  dev::scatter_kernel<<<grid_for(p->nnz, 256), 256, 0, st>>>(f->tiles, f->values, p->dev->scatter, p->nnz);
  CUDA_TRY(cudaGetLastError());
  if (!p->pad.empty()) {
    dev::set_ones_kernel<double><<<1, 128, 0, st>>>(f->tiles, p->dev->pad, int64_t(p->pad.size()));
    CUDA_TRY(cudaGetLastError());
  }
  dev::rhs_to_tiles_kernel<<<grid_for(p->nsb * B * nrhs, 256), 256, 0, st>>>(f->tiles, b, p->dev->perm, n, ld, nrhs,
                                                                           int(B), p->nsb, p->nsub);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(f->flags, 0, size_t(p->nsub + p->nsb + nscr) * sizeof(int), st));
  dev::init_ctl_kernel<<<1, 32, 0, st>>>(f->ctl, 3);
  CUDA_TRY(cudaGetLastError());
  count_launch(p->pad.empty() ? 3 : 4);
  CUDA_TRY(cudaEventRecord(f->ev[1], st));
  cudaError_t e;
  switch (B) {
    case 16: e = launch_factor<16>(p, f, st, true); break;
    case 32: e = launch_factor<32>(p, f, st, true); break;
    default: e = launch_factor<64>(p, f, st, true); break;
  }
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("factor launch: ") + cudaGetErrorString(e));
  count_launch();
  CUDA_TRY(cudaEventRecord(f->ev[2], st));
  e = launch_diag_inverse(p, f, st);
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("diagonal inverses: ") + cudaGetErrorString(e));
  count_launch(2);
  CUDA_TRY(cudaEventRecord(f->done, st));
  f->sinv_valid = false;
  // the backward sweep from the forward result tiles
  dev::tiles_to_blocks_kernel<<<grid_for(p->nsb * B * nrhs, 256), 256, 0, st>>>(f->Y, f->tiles, nrhs, int(B), p->nsb,
                                                                              p->nsub);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(f->sflags, 0, size_t(2 * p->nsb + nf + nb) * sizeof(int), st));
  switch (B) {
    case 16: e = launch_backward<16>(p, f, st, nrhs); break;
    case 32: e = launch_backward<32>(p, f, st, nrhs); break;
    default: e = launch_backward<64>(p, f, st, nrhs); break;
  }
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("solve launch: ") + cudaGetErrorString(e));
  dev::permute_out_kernel<double><<<grid_for(n * nrhs, 256), 256, 0, st>>>(x, f->Y, p->dev->perm, n, ld, 0, nrhs,
                                                                          int(B));
  CUDA_TRY(cudaGetLastError());
  count_launch(3);
  CUDA_TRY(cudaStreamSynchronize(st));
  f->pending = false;
  s = read_ctl(f, 0, info);
  if (s != STILES_OK) return s;
  return read_ctl(f, 2, nullptr);
}

stiles_status stiles_logdet(const stiles_factor* cf, double* out) {
  if (!cf || !out) return fail(STILES_ERR_INVALID, "null argument");
  stiles_factor* f = const_cast<stiles_factor*>(cf);
  const stiles_plan* p = f->plan;
  cudaStream_t st = f->stream;
  if (f->lp)
    dev::logdet_vec_pass1<<<dev::LOGDET_BLOCKS, dev::LOGDET_THREADS, 0, st>>>(f->ldiag, p->n, f->logdet_part);
  else
    dev::logdet_pass1<<<dev::LOGDET_BLOCKS, dev::LOGDET_THREADS, 0, st>>>(f->tiles, p->dev->diag_sub, p->n, p->B,
                                                                          f->logdet_part);
  CUDA_TRY(cudaGetLastError());
  dev::logdet_pass2<<<1, 32, 0, st>>>(f->logdet_part, dev::LOGDET_BLOCKS, f->logdet_part + dev::LOGDET_BLOCKS);
  CUDA_TRY(cudaGetLastError());
  count_launch(2);
  CUDA_TRY(cudaMemcpyAsync(out, f->logdet_part + dev::LOGDET_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return STILES_OK;
}

}  // extern "C"

namespace {

// One forward + backward sweep for right-hand-side columns [r0, r0 + nr) of
// `rhs` (leading dimension rld), result into the same columns of `out`.
stiles_status solve_chunk(const stiles_plan* p, stiles_factor* f, cudaStream_t st, const double* rhs, int64_t rld,
                          double* out, int64_t old_, int r0, int nr) {
  const int64_t n = p->n, B = p->B;
  const int64_t nf = std::max<int64_t>(p->fwd.nscratch, 1), nb = std::max<int64_t>(p->bwd.nscratch, 1);
  const bool f32 = f->lp || f->sliced;  // FP32 sweeps (refined in FP64)
  if (f32)
    dev::permute_in_kernel<float><<<grid_for(p->nsb * B * nr, 256), 256, 0, st>>>(
        reinterpret_cast<float*>(f->Y), rhs, p->dev->perm, n, rld, r0, nr, int(B), p->nsb);
  else
    dev::permute_in_kernel<double><<<grid_for(p->nsb * B * nr, 256), 256, 0, st>>>(f->Y, rhs, p->dev->perm, n, rld,
                                                                                r0, nr, int(B), p->nsb);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(f->sflags, 0, size_t(2 * p->nsb + nf + nb) * sizeof(int), st));
  dev::init_ctl_kernel<<<1, 32, 0, st>>>(f->ctl + 1, 2);
  CUDA_TRY(cudaGetLastError());
  cudaError_t e;
  if (f->lp) e = launch_solve<64, float>(p, f, st, nr, f->tiles32, f->invdiag32, f->linv32);
  else if (f->sliced) e = launch_solve<32, float>(p, f, st, nr, f->tiles32, f->invdiag32, f->linv32);
  else switch (p->B) {
    case 16: e = launch_solve<16, double>(p, f, st, nr, f->tiles, f->invdiag, f->linv); break;
    case 32: e = launch_solve<32, double>(p, f, st, nr, f->tiles, f->invdiag, f->linv); break;
    default: e = launch_solve<64, double>(p, f, st, nr, f->tiles, f->invdiag, f->linv); break;
  }
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("solve launch: ") + cudaGetErrorString(e));
  if (f32)
    dev::permute_out_kernel<float><<<grid_for(n * nr, 256), 256, 0, st>>>(out, reinterpret_cast<const float*>(f->Y),
                                                                          p->dev->perm, n, old_, r0, nr, int(B));
  else
    dev::permute_out_kernel<double><<<grid_for(n * nr, 256), 256, 0, st>>>(out, f->Y, p->dev->perm, n, old_, r0, nr,
                                                                           int(B));
  CUDA_TRY(cudaGetLastError());
  count_launch(5);
  CUDA_TRY(cudaStreamSynchronize(st));
  stiles_status s1 = read_ctl(f, 1, nullptr);
  if (s1 == STILES_OK) s1 = read_ctl(f, 2, nullptr);
  return s1;
}

// FP64 residual of columns [r0, r0 + nr): optionally r = b - A x into rout
// (leading dimension n), and the largest ||b - A x|| / ||b|| of the chunk.
stiles_status residual_chunk(const stiles_plan* p, stiles_factor* f, cudaStream_t st, const double* x, int64_t ldx,
                             const double* b, int64_t ldb, int r0, int nr, double* rout, double* worst) {
  const int64_t n = p->n;
  CUDA_TRY(cudaMemsetAsync(f->norms, 0, 2 * dev::SOLVE_MAXR * sizeof(double), st));
  dev::symv_kernel<<<grid_for(n * 32, 256), 256, 0, st>>>(f->ywork, x + r0 * ldx, p->dev->colptr, p->dev->rowidx,
                                                         p->dev->rptr, p->dev->rcol, p->dev->rval, f->values, n,
                                                         ldx, nr);
  CUDA_TRY(cudaGetLastError());
  dev::residual_norms_kernel<<<dim3(64, nr), 256, 0, st>>>(f->ywork, b + r0 * ldb, n, ldb, nr, f->norms);
  CUDA_TRY(cudaGetLastError());
  count_launch(2);
  if (rout) {
    dev::sub_cols_kernel<<<grid_for(n * nr, 256), 256, 0, st>>>(rout, b + r0 * ldb, f->ywork, n, ldb, nr);
    CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  double h[2 * dev::SOLVE_MAXR];
  CUDA_TRY(cudaMemcpyAsync(h, f->norms, 2 * nr * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  double w = 0.0;
  for (int r = 0; r < nr; ++r) {
    const double rel = h[2 * r + 1] > 0 ? std::sqrt(h[2 * r] / h[2 * r + 1]) : std::sqrt(h[2 * r]);
    w = std::max(w, rel);
  }
  *worst = w;
  return STILES_OK;
}

// Conjugate gradients on A x = b preconditioned by the mixed-precision factor
// (z = (L L^T)^{-1} r through the factor's sweeps), started from the current x
// of columns [r0, r0 + nr) and its residual r = b - A x (held in the second
// quarter of irwork); per-column step lengths in FP64.  Used when iterative
// refinement stalls.  Stops when the recomputed true residual meets refine_tol
// or after `budget` iterations; *worst = the largest ||b - A x|| / ||b||.
stiles_status pcg_chunk(const stiles_plan* p, stiles_factor* f, cudaStream_t st, double* dx, int64_t dld,
                        const double* db, int64_t bld, int r0, int nr, int budget, int* used, double* worst) {
  constexpr int R = dev::SOLVE_MAXR;
  const int64_t n = p->n;
  double* z = f->irwork;                   // preconditioned residual
  double* r = f->irwork + size_t(n) * R;   // residual
  double* pv = r + size_t(n) * R;          // search direction
  double* q = pv + size_t(n) * R;          // A p
  double* xc = dx + r0 * dld;
  const double* bc = db + r0 * bld;
  auto dots = [&](const double* a, int64_t lda, const double* c, int64_t ldc, double* h) -> stiles_status {
    CUDA_TRY(cudaMemsetAsync(f->cgs, 0, nr * sizeof(double), st));
    dev::dot_cols_kernel<<<dim3(64, nr), 256, 0, st>>>(a, lda, c, ldc, n, f->cgs);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    CUDA_TRY(cudaMemcpyAsync(h, f->cgs, nr * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return STILES_OK;
  };
  auto set_coef = [&](const double* h) -> stiles_status {
    CUDA_TRY(cudaMemcpyAsync(f->cgs + R, h, nr * sizeof(double), cudaMemcpyHostToDevice, st));
    return STILES_OK;
  };
  double bb[R], rz[R], tmp[R], coef[R];
  stiles_status s = dots(bc, bld, bc, bld, bb);
  if (s != STILES_OK) return s;
  s = solve_chunk(p, f, st, r, n, z, n, 0, nr);
  if (s != STILES_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(pv, z, size_t(n) * nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if ((s = dots(r, n, z, n, rz)) != STILES_OK) return s;
  *worst = std::numeric_limits<double>::infinity();
  for (int k = 0; k < budget; ++k) {
    dev::symv_kernel<<<grid_for(n * 32, 256), 256, 0, st>>>(q, pv, p->dev->colptr, p->dev->rowidx, p->dev->rptr,
                                                           p->dev->rcol, p->dev->rval, f->values, n, n, nr);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    if ((s = dots(pv, n, q, n, tmp)) != STILES_OK) return s;
    for (int c = 0; c < nr; ++c) coef[c] = tmp[c] > 0 ? rz[c] / tmp[c] : 0.0;
    if ((s = set_coef(coef)) != STILES_OK) return s;
    dev::cg_update_kernel<<<grid_for(n * nr, 256), 256, 0, st>>>(xc, dld, r, pv, q, f->cgs + R, n, nr);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    ++*used;
    if ((s = dots(r, n, r, n, tmp)) != STILES_OK) return s;
    double w = 0.0;
    for (int c = 0; c < nr; ++c) w = std::max(w, bb[c] > 0 ? std::sqrt(tmp[c] / bb[c]) : std::sqrt(tmp[c]));
    if (!(w > p->opts.refine_tol)) {
      // the recursive residual says done: confirm with the true one (and continue from it if not)
      if ((s = residual_chunk(p, f, st, dx, dld, db, bld, r0, nr, r, worst)) != STILES_OK) return s;
      if (!(*worst > p->opts.refine_tol)) return STILES_OK;
    }
    *worst = w;
    if ((s = solve_chunk(p, f, st, r, n, z, n, 0, nr)) != STILES_OK) return s;
    if ((s = dots(r, n, z, n, tmp)) != STILES_OK) return s;
    for (int c = 0; c < nr; ++c) {
      coef[c] = rz[c] > 0 ? tmp[c] / rz[c] : 0.0;
      rz[c] = tmp[c];
    }
    if ((s = set_coef(coef)) != STILES_OK) return s;
    dev::cg_direction_kernel<<<grid_for(n * nr, 256), 256, 0, st>>>(pv, z, f->cgs + R, n, nr);
    CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  return residual_chunk(p, f, st, dx, dld, db, bld, r0, nr, r, worst);
}

}  // namespace

extern "C" {

stiles_status stiles_solve(const stiles_factor* cf, const double* b, double* x, int64_t nrhs, int64_t ld, void* stream,
                           double* final_relres) {
  if (!cf || !b || !x) return fail(STILES_ERR_INVALID, "null argument");
  stiles_factor* f = const_cast<stiles_factor*>(cf);
  const stiles_plan* p = f->plan;
  if (nrhs < 1 || ld < p->n) return fail(STILES_ERR_INVALID, "nrhs < 1 or ld < n");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  if (bdev != xdev) return fail(STILES_ERR_INVALID, "b and x must both be host or both be device memory");
  const int64_t n = p->n, B = p->B;
  const int64_t nf = std::max<int64_t>(p->fwd.nscratch, 1), nb = std::max<int64_t>(p->bwd.nscratch, 1);
  if (f->solve_nr < dev::SOLVE_MAXR) {
    cudaFree(f->Y);
    cudaFree(f->sscratch);
    cudaFree(f->sflags);
    cudaFree(f->ywork);
    f->Y = f->sscratch = f->ywork = nullptr;
    f->sflags = nullptr;
    f->solve_nr = 0;
    CUDA_TRY(cudaMalloc(&f->Y, size_t(p->nsb) * B * dev::SOLVE_MAXR * sizeof(double)));
    CUDA_TRY(cudaMalloc(&f->sscratch, size_t(nf + nb) * B * dev::SOLVE_MAXR * sizeof(double)));
    CUDA_TRY(cudaMalloc(&f->sflags, size_t(2 * p->nsb + nf + nb) * sizeof(int)));
    CUDA_TRY(cudaMalloc(&f->ywork, size_t(n) * dev::SOLVE_MAXR * sizeof(double)));
    f->solve_nr = dev::SOLVE_MAXR;
  }
  const bool refine = f->lp || f->sliced;  // factors whose solves are refined in FP64
  if (refine && !f->irwork) {
    CUDA_TRY(cudaMalloc(&f->irwork, 4 * size_t(n) * dev::SOLVE_MAXR * sizeof(double)));
    CUDA_TRY(cudaMalloc(&f->cgs, 2 * dev::SOLVE_MAXR * sizeof(double)));
  }
  const double* db = b;
  double* dx = x;
  int64_t bld = ld, xld = ld;  // leading dimensions of the device-side b and x
  if (bdev && b == x && (refine || final_relres)) {
    // in place on the device: keep b for the residuals
    const int64_t need = n * nrhs;
    if (f->stage_elems < need) {
      cudaFree(f->bstage);
      cudaFree(f->xstage);
      f->bstage = f->xstage = nullptr;
      f->stage_elems = 0;
      CUDA_TRY(cudaMalloc(&f->bstage, size_t(need) * sizeof(double)));
      CUDA_TRY(cudaMalloc(&f->xstage, size_t(need) * sizeof(double)));
      f->stage_elems = need;
    }
    CUDA_TRY(cudaMemcpy2DAsync(f->bstage, n * sizeof(double), b, ld * sizeof(double), n * sizeof(double), nrhs,
                               cudaMemcpyDeviceToDevice, st));
    db = f->bstage;
    bld = n;
  }
  if (!bdev) {
    const int64_t need = n * nrhs;
    if (f->stage_elems < need) {
      cudaFree(f->bstage);
      cudaFree(f->xstage);
      f->bstage = f->xstage = nullptr;
      f->stage_elems = 0;
      CUDA_TRY(cudaMalloc(&f->bstage, size_t(need) * sizeof(double)));
      CUDA_TRY(cudaMalloc(&f->xstage, size_t(need) * sizeof(double)));
      f->stage_elems = need;
    }
    CUDA_TRY(cudaMemcpy2DAsync(f->bstage, n * sizeof(double), b, ld * sizeof(double), n * sizeof(double), nrhs,
                               cudaMemcpyHostToDevice, st));
    db = f->bstage;
    dx = f->xstage;
    bld = xld = n;
  }
  double worst = 0.0;
  bool converged = true;
  f->last_refine_iters = 0;
  f->last_cg_iters = 0;
  for (int64_t r0 = 0; r0 < nrhs; r0 += dev::SOLVE_MAXR) {
    const int nr = int(std::min<int64_t>(dev::SOLVE_MAXR, nrhs - r0));
    if (!refine) {
      stiles_status s1 = solve_chunk(p, f, st, db, bld, dx, xld, int(r0), nr);
      if (s1 != STILES_OK) return s1;
      if (final_relres) {
        double w = 0.0;
        s1 = residual_chunk(p, f, st, dx, xld, db, bld, int(r0), nr, nullptr, &w);
        if (s1 != STILES_OK) return s1;
        worst = std::max(worst, w);
      }
      continue;
    }
    // Mixed-precision or sliced-update factor: iterative refinement with FP64 residuals,
    // x <- x + solve(b - A x), until ||b - A x|| / ||b|| <= refine_tol.  A step
    // that does not at least halve the residual (or a NaN) means the factor is
    // too inaccurate for refinement to converge: the remaining budget goes to
    // conjugate gradients preconditioned by the same factor.
    double* dwork = f->irwork;                  // correction, n x nr
    double* rwork = f->irwork + size_t(n) * dev::SOLVE_MAXR;  // residual, n x nr
    stiles_status s1 = solve_chunk(p, f, st, db, bld, dx, xld, int(r0), nr);
    if (s1 != STILES_OK) return s1;
    double w = 0.0, wprev = std::numeric_limits<double>::infinity();
    int it = 0;
    bool stalled = false;
    for (;;) {
      s1 = residual_chunk(p, f, st, dx, xld, db, bld, int(r0), nr, rwork, &w);
      if (s1 != STILES_OK) return s1;
      if (!(w > p->opts.refine_tol) || it >= p->opts.max_refine) break;
      if (!(w <= 0.5 * wprev)) {
        stalled = true;
        break;
      }
      wprev = w;
      s1 = solve_chunk(p, f, st, rwork, n, dwork, n, 0, nr);
      if (s1 != STILES_OK) return s1;
      dev::axpy_cols_kernel<<<grid_for(n * nr, 256), 256, 0, st>>>(dx + r0 * xld, dwork, n, xld, nr);
      CUDA_TRY(cudaGetLastError());
      count_launch();
      ++it;
    }
    if (stalled) {
      if (w != w) {  // the iterate is lost: restart from x = 0 (r = b)
        CUDA_TRY(cudaMemset2DAsync(dx + r0 * xld, xld * sizeof(double), 0, n * sizeof(double), nr, st));
        s1 = residual_chunk(p, f, st, dx, xld, db, bld, int(r0), nr, rwork, &w);
        if (s1 != STILES_OK) return s1;
      }
      int used = 0;
      s1 = pcg_chunk(p, f, st, dx, xld, db, bld, int(r0), nr, std::max(0, p->opts.max_refine - it), &used, &w);
      if (s1 != STILES_OK) return s1;
      it += used;
      f->last_cg_iters = std::max(f->last_cg_iters, used);
    }
    f->last_refine_iters = std::max(f->last_refine_iters, it);
    if (w > p->opts.refine_tol || w != w) converged = false;
    worst = std::max(worst, w);
  }
  if (!xdev) {
    CUDA_TRY(cudaMemcpy2DAsync(x, ld * sizeof(double), dx, n * sizeof(double), n * sizeof(double), nrhs,
                               cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (final_relres) *final_relres = worst;
  if (!converged) return fail(STILES_ERR_NOT_CONVERGED, "iterative refinement did not reach refine_tol");
  return STILES_OK;
}

int32_t stiles_factor_refine_iters(const stiles_factor* f) { return f ? f->last_refine_iters : -1; }

int32_t stiles_factor_cg_iters(const stiles_factor* f) { return f ? f->last_cg_iters : -1; }

stiles_status stiles_factor_tiles(const stiles_factor* cf, double* out, void* stream) {
  if (!cf || !out) return fail(STILES_ERR_INVALID, "null argument");
  stiles_factor* f = const_cast<stiles_factor*>(cf);
  const stiles_plan* p = f->plan;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t elems = size_t(p->nnzt) * p->T * p->T;
  const bool odev = is_device_ptr(out);
  double* dst = out;
  if (!odev) CUDA_TRY(cudaMalloc(&dst, elems * sizeof(double)));
  if (f->lp)
    dev::export_tiles_kernel<float><<<grid_for(int64_t(elems), 256), 256, 0, st>>>(dst, f->tiles32, p->nnzt, p->T, p->B);
  else
    dev::export_tiles_kernel<double><<<grid_for(int64_t(elems), 256), 256, 0, st>>>(dst, f->tiles, p->nnzt, p->T, p->B);
  cudaError_t e = cudaGetLastError();
  count_launch();
  if (e == cudaSuccess && !odev) e = cudaMemcpyAsync(out, dst, elems * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (!odev) cudaFree(dst);
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("tile export: ") + cudaGetErrorString(e));
  return STILES_OK;
}

}  // extern "C"

namespace {

template <int B>
stiles_status launch_selinv(const stiles_plan* p, stiles_factor* f, cudaStream_t st) {
  const DevPlan* d = p->dev;
  const int64_t nu = d->sinv_nu;
  if (nu > 0) {
    const int gu = int(std::max<int64_t>(1, std::min<int64_t>(nu, 148 * 16)));
    dev::selinv_u_kernel<B><<<gu, 128, 0, st>>>(f->sinv_u, f->tiles, f->linv, d->sinv_ulist, nu);
    CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  {
    const int gg = int(std::max<int64_t>(1, std::min<int64_t>(p->nsb, 148 * 16)));
    dev::selinv_g_kernel<B><<<gg, 128, 0, st>>>(f->sigma, f->linv, d->diag_sub, p->nsb);
    CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  static int per_sm = 0;  // resident CTAs of the persistent kernel (per B instantiation)
  if (per_sm == 0) {
    CUDA_TRY(cudaFuncSetAttribute(dev::selinv_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(dev::SelinvCfg<B>::SMEM)));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dev::selinv_kernel<B>, 128,
                                                           dev::SelinvCfg<B>::SMEM));
    per_sm = std::max(per_sm, 1);
  }
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device));
  dev::SelinvArgs a{};
  a.sigma = f->sigma;
  a.sigmaT = f->sigmaT;
  a.V = f->sinv_u;
  a.W = f->sinv_w;
  a.X = f->sinv_x;
  a.tasks = d->sinv_tasks;
  a.pairs = d->sinv_pairs;
  a.loads = d->sinv_loads;
  a.posts = d->sinv_posts;
  a.ntasks = d->sinv_ntasks;
  a.flags = f->sinv_flags;
  a.ctl = f->sinv_ctl;
  a.spin_limit = p->opts.spin_limit;
  if (f->trace_on && !f->trace[3]) {
    const size_t bytes = size_t(d->sinv_ntasks) * 4 * sizeof(long long);
    CUDA_TRY(cudaMalloc(&f->trace[3], bytes));
    CUDA_TRY(cudaMemsetAsync(f->trace[3], 0, bytes, st));
  }
  a.trace = f->trace_on ? f->trace[3] : nullptr;
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(per_sm) * sms, d->sinv_ntasks)));
  dev::selinv_kernel<B><<<grid, 128, dev::SelinvCfg<B>::SMEM, st>>>(a);
  CUDA_TRY(cudaGetLastError());
  count_launch();
  return STILES_OK;
}

// Sigma on the filled sub-tile map for the factor's current values (FP64 factors).
stiles_status ensure_selinv(stiles_factor* f, cudaStream_t st) {
  const stiles_plan* p = f->plan;
  if (f->lp) return fail(STILES_ERR_UNSUPPORTED, "the selected inverse needs an FP64 factor");
  {
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    stiles_plan* pm = const_cast<stiles_plan*>(p);
    std::string err;
    stiles_status s = build_selinv(pm, &err);
    if (s != STILES_OK) return fail(s, err);
    DevPlan* d = pm->dev;
    if (!d->sinv_ready) {
      cudaError_t e = upload(&d->sinv_tasks, pm->selinv.tasks);
      if (e == cudaSuccess) e = upload(&d->sinv_pairs, pm->selinv.pairs);
      if (e == cudaSuccess) e = upload(&d->sinv_loads, pm->selinv.loads);
      if (e == cudaSuccess) e = upload(&d->sinv_posts, pm->selinv.posts);
      if (e == cudaSuccess) e = upload(&d->sinv_ulist, pm->selinv.ulist);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,
                    std::string("selected-inverse upload: ") + cudaGetErrorString(e));
      }
      d->sinv_ntasks = int(pm->selinv.tasks.size() / 8);
      d->sinv_nu = int64_t(pm->selinv.ulist.size() / 2);
      d->sinv_ready = true;
    }
  }
  if (f->sinv_valid) return STILES_OK;
  const size_t tile = size_t(p->B) * p->B;
  if (!f->sigma) CUDA_TRY(cudaMalloc(&f->sigma, size_t(p->nsub) * tile * sizeof(double)));
  if (!f->sigmaT) CUDA_TRY(cudaMalloc(&f->sigmaT, size_t(p->nsub) * tile * sizeof(double)));
  if (!f->sinv_u) CUDA_TRY(cudaMalloc(&f->sinv_u, size_t(p->nsub) * tile * sizeof(double)));
  if (!f->sinv_w) CUDA_TRY(cudaMalloc(&f->sinv_w, size_t(p->nsub) * tile * sizeof(double)));
  if (!f->sinv_x) CUDA_TRY(cudaMalloc(&f->sinv_x, size_t(p->nsub) * tile * sizeof(double)));
  if (!f->sinv_flags) CUDA_TRY(cudaMalloc(&f->sinv_flags, size_t(p->nsub) * sizeof(int)));
  if (!f->sinv_ctl) CUDA_TRY(cudaMalloc(&f->sinv_ctl, sizeof(dev::Ctl)));
  if (f->done) CUDA_TRY(cudaStreamWaitEvent(st, f->done, 0));  // the factorization has finished
  CUDA_TRY(cudaMemsetAsync(f->sinv_flags, 0, size_t(p->nsub) * sizeof(int), st));
  dev::init_ctl_kernel<<<1, 32, 0, st>>>(f->sinv_ctl, 1);
  CUDA_TRY(cudaGetLastError());
  count_launch();
  stiles_status s;
  switch (p->B) {
    case 16: s = launch_selinv<16>(p, f, st); break;
    case 32: s = launch_selinv<32>(p, f, st); break;
    default: s = launch_selinv<64>(p, f, st); break;
  }
  if (s != STILES_OK) return s;
  dev::Ctl c;
  CUDA_TRY(cudaMemcpyAsync(&c, f->sinv_ctl, sizeof(c), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (c.status != 0) return fail(STILES_ERR_TIMEOUT, "device wait timed out in the selected inverse");
  f->sinv_valid = true;
  return STILES_OK;
}

}  // namespace

namespace {
bool append_release(const stiles::SolveGraph& g, int64_t nsb, int32_t off, std::vector<int32_t>& cptr,
                    std::vector<int32_t>& cons, std::vector<int32_t>& cnt0, std::vector<int32_t>& src);
}  // namespace

extern "C" {

stiles_status stiles_marginal_variances(stiles_factor* f, double* out, void* stream) {
  if (!f || !out) return fail(STILES_ERR_INVALID, "null argument");
  const stiles_plan* p = f->plan;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : f->stream;
  stiles_status s = ensure_selinv(f, st);
  if (s != STILES_OK) return s;
  const bool odev = is_device_ptr(out);
  double* dst = out;
  if (!odev) CUDA_TRY(cudaMalloc(&dst, size_t(p->n) * sizeof(double)));
  const int g = grid_for(p->n, 256);
  switch (p->B) {
    case 16: dev::selinv_diag_kernel<16><<<g, 256, 0, st>>>(dst, f->sigma, p->dev->diag_sub, p->dev->perm, p->n); break;
    case 32: dev::selinv_diag_kernel<32><<<g, 256, 0, st>>>(dst, f->sigma, p->dev->diag_sub, p->dev->perm, p->n); break;
    default: dev::selinv_diag_kernel<64><<<g, 256, 0, st>>>(dst, f->sigma, p->dev->diag_sub, p->dev->perm, p->n); break;
  }
  cudaError_t e = cudaGetLastError();
  count_launch();
  if (e == cudaSuccess && !odev) e = cudaMemcpyAsync(out, dst, size_t(p->n) * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (!odev) cudaFree(dst);
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("marginal variances: ") + cudaGetErrorString(e));
  return STILES_OK;
}

stiles_status stiles_selected_inverse_tiles(stiles_factor* f, double* out, void* stream) {
  if (!f || !out) return fail(STILES_ERR_INVALID, "null argument");
  const stiles_plan* p = f->plan;
  cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : f->stream;
  stiles_status s = ensure_selinv(f, st);
  if (s != STILES_OK) return s;
  const size_t elems = size_t(p->nnzt) * p->T * p->T;
  const bool odev = is_device_ptr(out);
  double* dst = out;
  if (!odev) CUDA_TRY(cudaMalloc(&dst, elems * sizeof(double)));
  dev::export_tiles_kernel<double><<<grid_for(int64_t(elems), 256), 256, 0, st>>>(dst, f->sigma, p->nnzt, p->T, p->B);
  cudaError_t e = cudaGetLastError();
  count_launch();
  if (e == cudaSuccess && !odev) e = cudaMemcpyAsync(out, dst, elems * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (!odev) cudaFree(dst);
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("selected-inverse export: ") + cudaGetErrorString(e));
  return STILES_OK;
}

stiles_status stiles_factor_timing(const stiles_factor* f, double* ms_call, double* ms_kernel) {
  if (!f) return fail(STILES_ERR_INVALID, "null factor");
  if (!f->ev[0]) return fail(STILES_ERR_INVALID, "a factor of a batch has no own timing (stiles_batch_timing)");
  float a = 0.f, b = 0.f;
  CUDA_TRY(cudaEventSynchronize(f->ev[2]));
  CUDA_TRY(cudaEventElapsedTime(&a, f->ev[0], f->ev[2]));
  CUDA_TRY(cudaEventElapsedTime(&b, f->ev[1], f->ev[2]));
  if (ms_call) *ms_call = a;
  if (ms_kernel) *ms_kernel = b;
  return STILES_OK;
}

stiles_status stiles_factor_set_trace(stiles_factor* f, int32_t enable) {
  if (!f) return fail(STILES_ERR_INVALID, "null factor");
  const stiles_plan* p = f->plan;
  const size_t n[4] = {p->graph.tasks.size(), p->fwd.tasks.size(), p->bwd.tasks.size(), 0};
  f->trace_on = enable != 0;
  for (int i = 0; i < 4; ++i) {
    cudaFree(f->trace[i]);
    f->trace[i] = nullptr;
    if (enable && n[i]) {
      CUDA_TRY(cudaMalloc(&f->trace[i], n[i] * 4 * sizeof(long long)));
      CUDA_TRY(cudaMemset(f->trace[i], 0, n[i] * 4 * sizeof(long long)));
    }
  }
  return STILES_OK;
}

stiles_status stiles_factor_get_trace(const stiles_factor* f, int32_t which, int64_t* out, int64_t* ntasks) {
  if (!f || which < 0 || which > 3) return fail(STILES_ERR_INVALID, "bad argument");
  const stiles_plan* p = f->plan;
  const size_t n = which == 0   ? p->graph.tasks.size()
                   : which == 1 ? p->fwd.tasks.size()
                   : which == 2 ? p->bwd.tasks.size()
                                : (p->selinv_built ? p->selinv.tasks.size() / 8 : 0);
  if (ntasks) *ntasks = int64_t(n);
  if (!out) return STILES_OK;
  if (!f->trace[which]) return fail(STILES_ERR_INVALID, "tracing is not enabled");
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(out, f->trace[which], n * 4 * sizeof(long long), cudaMemcpyDeviceToHost));
  return STILES_OK;
}

stiles_status stiles_plan_tasks(const stiles_plan* p, int32_t which, int32_t* out, int64_t* ntasks) {
  if (!p || which < 0 || which > 17) return fail(STILES_ERR_INVALID, "bad argument");
  if (which >= 12) {  // a sweep's ready-queue release lists (12-14 forward, 15-17 backward)
    std::vector<int32_t> cptr{0}, cons, cnt0, src;
    if (!append_release(which < 15 ? p->fwd : p->bwd, p->nsb, 0, cptr, cons, cnt0, src))
      return fail(STILES_ERR_INVALID, "internal: a sweep task reads an output produced after it");
    const int k = (which - 12) % 3;
    const std::vector<int32_t>& v = k == 0 ? cnt0 : k == 1 ? cptr : cons;
    if (ntasks) *ntasks = int64_t(v.size());
    if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
    return STILES_OK;
  }
  if (which >= 8) {  // a sweep's operand pairs (8 forward, 9 backward) or partial lists (10, 11)
    const SolveGraph& g = (which % 2 == 0) ? p->fwd : p->bwd;
    const std::vector<int32_t>& v = which < 10 ? g.pairs : g.parts;
    if (ntasks) *ntasks = int64_t(which < 10 ? v.size() / 2 : v.size());
    if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
    return STILES_OK;
  }
  if (which == 7) {  // the factorization with the forward sweep folded in (host only; built on first use)
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    stiles_plan* pm = const_cast<stiles_plan*>(p);
    std::string err;
    stiles_status s = build_fused(pm, &err);
    if (s != STILES_OK) return fail(s, err);
    if (ntasks) *ntasks = int64_t(pm->fused.tasks.size());
    if (out && !pm->fused.tasks.empty()) std::memcpy(out, pm->fused.tasks.data(), pm->fused.tasks.size() * sizeof(DevTask));
    return STILES_OK;
  }
  if (which >= 3) {  // the selected inverse's graph (host only; built on first use)
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    stiles_plan* pm = const_cast<stiles_plan*>(p);
    std::string err;
    stiles_status s = build_selinv(pm, &err);
    if (s != STILES_OK) return fail(s, err);
    const std::vector<int32_t>& v = which == 3   ? pm->selinv.tasks
                                    : which == 4 ? pm->selinv.pairs
                                    : which == 5 ? pm->selinv.loads
                                                 : pm->selinv.posts;
    const size_t width = which == 3 ? 8 : which == 6 ? 1 : which == 5 ? 3 : 2;
    if (ntasks) *ntasks = int64_t(v.size() / width);
    if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
    return STILES_OK;
  }
  const void* src;
  size_t n;
  if (which == 0) { src = p->graph.tasks.data(); n = p->graph.tasks.size(); }
  else if (which == 1) { src = p->fwd.tasks.data(); n = p->fwd.tasks.size(); }
  else { src = p->bwd.tasks.data(); n = p->bwd.tasks.size(); }
  if (ntasks) *ntasks = int64_t(n);
  const size_t width = which == 0 ? sizeof(DevTask) : sizeof(SolveTask);
  if (out && n) std::memcpy(out, src, n * width);
  return STILES_OK;
}

int64_t stiles_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

stiles_status stiles_probe_fp64_peak(double* tflops) {
  if (!tflops) return fail(STILES_ERR_INVALID, "null argument");
  int device = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&device));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  double* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, 64));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = 4000, blocks = sms * 2, threads = 256;
  dev::fp64_probe_kernel<<<blocks, threads>>>(d, 200, 1.0000001, 1e-9);
  count_launch(2);
  cudaEventRecord(e0);
  dev::fp64_probe_kernel<<<blocks, threads>>>(d, iters, 1.0000001, 1e-9);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, cudaGetErrorString(e));
  *tflops = 2.0 * 8 * double(iters) * threads * blocks / (double(ms) * 1e-3) / 1e12;
  return STILES_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched factorization (many matrices, one persistent launch).  The batch owns
// concatenated device arrays for every matrix (values, tiles, flags, ...), a
// merged ticket list that interleaves the matrices' task lists in proportion
// to their lengths (each matrix keeps its own topological order, so the launch
// stays deadlock-free), and a CUDA graph of the per-call device work (zeroing,
// scatter, the persistent kernel).  Per-matrix factor views borrow the batch's
// arrays for logdet and solves.
// ---------------------------------------------------------------------------
struct stiles_batch {
  std::vector<const stiles_plan*> plans;
  std::vector<stiles_factor*> views;
  bool lp = false;
  bool sliced = false;
  int B = 0;
  int device = -1;
  int fp16 = 0;
  int64_t nnz_total = 0, pad_total = 0, tile_elems = 0, scratch_elems = 0, diag_elems = 0, flag_total = 0;
  std::vector<int64_t> val_off;
  double* values = nullptr;
  void* dscatter = nullptr;  // per-matrix BScatter descriptors (each plan's own device scatter map)
  int64_t max_scatter = 0;   // largest nnz + padding count of one matrix
  int64_t max_nsb = 0;       // largest number of diagonal sub-tiles of one matrix
  double* tiles = nullptr;
  double* scratch = nullptr;
  double* invdiag = nullptr;
  double* linv = nullptr;       // per matrix: L_kk^{-1} and the sweeps' folded terms (5 nsb B^2)
  void* dinv = nullptr;         // per-matrix BInverse descriptors
  void* dinv32 = nullptr;       // sliced updates: the same for the FP32 copies (the sweeps)
  void* dmlast = nullptr;       // per-matrix MlastDesc descriptors (the sweeps' folded newest terms)
  int64_t max_stasks = 0;       // largest 2 x (forward + backward sweep tasks) of one matrix
  float* tiles32 = nullptr;
  uint16_t* tiles16 = nullptr;
  float* scratch32 = nullptr;
  float* invdiag32 = nullptr;
  float* linv32 = nullptr;
  double* ldiag = nullptr;
  uint16_t* slices = nullptr;   // sliced updates: 4 BF16 digit slices per sub-tile
  int* rowexp = nullptr;        // sliced updates: row scales
  void* drowexp = nullptr;      // sliced updates: per-matrix OZRowexpDesc
  int* flags = nullptr;
  unsigned long long* infos = nullptr;
  stiles::dev::Ctl* ctl = nullptr;
  void* dmats = nullptr;
  int2* dtickets = nullptr;
  int ntickets = 0;
  int grid = 0;
  long long spin_limit = 0;
  double* logdet_out = nullptr;
  void* dlog = nullptr;
  stiles::dev::Ctl* vctl = nullptr;  // the views' small arrays, 3 Ctl / logdet partials / norms each
  double* vlog = nullptr;
  double* vnorm = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;  // around the persistent kernel (recorded inside the graph)
  cudaGraphExec_t gexec = nullptr;
  // batched solves (allocated on first use)
  bool solve_ready = false;
  int solve_grid = 0;
  int64_t vec_total = 0;          // sum of n * SOLVE_MAXR
  std::vector<int64_t> vec_off;   // per matrix offset of its n x SOLVE_MAXR vectors
  double* sY = nullptr;
  double* sScr = nullptr;
  int* sFlags = nullptr;
  int64_t sflag_total = 0;
  double* vb = nullptr;  // right-hand sides, solutions, residuals, corrections, A x
  double* vx = nullptr;
  double* vr = nullptr;
  double* vd = nullptr;
  double* vy = nullptr;
  double* vnorms = nullptr;
  stiles::dev::Ctl* sctl = nullptr;
  void* dfwd = nullptr;
  void* dbwd = nullptr;
  void* ddesc = nullptr;
  int2* dspmv = nullptr;            // (matrix, its block) of every block of a batched A x
  int nspmv = 0;
  std::vector<int> spmv_blocks;     // per matrix
  int2* tfwd = nullptr;  // sweep ticket -> (matrix, task): every matrix's list in turn
  int2* tbwd = nullptr;
  int nfwd = 0, nbwd = 0;
  // ready-queue release lists of both sweeps over the batch's tickets (readers
  // CSR, producer counts, tickets without producers) and the launch's working
  // arrays (queue slots, counters; shared by the two launches, reset before each)
  int32_t *rq_cptr_f = nullptr, *rq_cons_f = nullptr, *rq_cnt0_f = nullptr, *rq_src_f = nullptr;
  int32_t *rq_cptr_b = nullptr, *rq_cons_b = nullptr, *rq_cnt0_b = nullptr, *rq_src_b = nullptr;
  int* rq_slots = nullptr;
  int* rq_cnt = nullptr;
  std::vector<int32_t> src_f, src_b;               // host copies of the source tickets
  std::vector<int64_t> src_f_off, src_b_off;       // per matrix: first source ticket (count + 1 entries)
  int32_t* rq_call_f = nullptr;  // sources of a call that solves only some matrices
  int32_t* rq_call_b = nullptr;
  std::vector<int64_t> y_off, scr_off, flag_off;
};

namespace {

// Per-matrix descriptor of the batched diagonal inverses (L_kk^{-1} for the sweeps).
struct BInverse {
  void* linv;
  const void* tiles;
  const void* invdiag;
  const int32_t* diag_sub;
  int64_t nsb;
};

template <int B, typename TF>
__global__ void bdiag_inverse_kernel(const BInverse* desc) {
  const BInverse c = desc[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; k < c.nsb; k += nwarps)
    dev::diag_inverse_tile<B, TF>(static_cast<TF*>(c.linv) + k * B * B,
                                  static_cast<const TF*>(c.tiles) + int64_t(c.diag_sub[k]) * B * B,
                                  static_cast<const TF*>(c.invdiag) + k * B, lane);
}

// Per-matrix descriptor of the batched scatter: the plan's own device scatter
// map and padding list, offset into the batch's concatenated values and tiles.
struct BScatter {
  const int64_t* map;
  const int64_t* pad;
  int64_t nnz, npad, val_off, tile_off;
};

// tiles[tile_off + map[e]] = values[val_off + e] and the padding diagonal ones,
// matrix blockIdx.y (targets are distinct: the tiles are zeroed beforehand).
template <typename T>
__global__ void bscatter_kernel(T* __restrict__ tiles, const double* __restrict__ values, const BScatter* desc) {
  const BScatter c = desc[blockIdx.y];
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < c.nnz; e += stride)
    tiles[c.tile_off + __ldg(c.map + e)] = T(__ldg(values + c.val_off + e));
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < c.npad; e += stride)
    tiles[c.tile_off + __ldg(c.pad + e)] = T(1);
}

// Per-matrix descriptor of the batched helper kernels around the solves.
struct BSolveDesc {
  const int64_t* perm;
  int64_t n, nsb;
  int B, nr;
  int spmv_blocks, pad0;  // blocks of the batched A x that serve this matrix
  void* Y;  // sweep blocks, in the factor's storage type
  double* b;
  double* x;
  double* r;
  double* d;
  double* y;
  const int64_t* colptr;
  const int32_t* rowidx;
  const int64_t* rptr;
  const int32_t* rcol;
  const int64_t* rval;
  const double* values;
  double* norms;  // 2 per right-hand side: ||b - A x||^2, ||b||^2
};

// which = 0: b -> Y / Y -> x;  which = 1: r -> Y / Y -> d
template <typename TY>
__global__ void bpermute_in_kernel(const BSolveDesc* desc, int which) {
  const BSolveDesc c = desc[blockIdx.y];
  const double* src = which ? c.r : c.b;
  TY* Y = static_cast<TY*>(c.Y);
  const int64_t total = c.nsb * c.B * c.nr;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = e / (int64_t(c.B) * c.nr);
    const int64_t rem = e % (int64_t(c.B) * c.nr);
    const int64_t r = rem / c.B, i = rem % c.B;
    const int64_t g = k * c.B + i;
    Y[e] = (g < c.n) ? TY(src[c.perm[g] + r * c.n]) : TY(0);
  }
}

template <typename TY>
__global__ void bpermute_out_kernel(const BSolveDesc* desc, int which) {
  const BSolveDesc c = desc[blockIdx.y];
  double* dst = which ? c.d : c.x;
  const TY* Y = static_cast<const TY*>(c.Y);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < c.n * c.nr; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / c.n, g = e % c.n;
    dst[c.perm[g] + r * c.n] = double(Y[((g / c.B) * c.nr + r) * c.B + (g % c.B)]);
  }
}

// d = x with the right-hand sides interleaved (d[i nr + r] = x[i + r n]): the
// SpMV's gathers of one entry then read one contiguous run instead of nr
// sectors n elements apart.  d is free here (the next correction overwrites it).
__global__ void binterleave_kernel(const BSolveDesc* desc) {
  const BSolveDesc c = desc[blockIdx.y];
  const int64_t total = c.n * c.nr;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / c.nr, r = e % c.nr;
    c.d[e] = c.x[i + r * c.n];
  }
}

// y = A x for matrix blockIdx.y (x read interleaved from d), one warp per index (no atomics)
// Batched A x: block b serves matrix blocks[b].x as its blocks[b].y-th of
// desc.spmv_blocks blocks, whose warps stride over the matrix's indices (the
// dense arrow rows, consecutive indices, land on different warps and SMs).
// Every matrix gets blocks in proportion to its nonzeros, largest first: one
// row of blocks per matrix left the largest matrices' rows on a few SMs (SMs
// active 56% of a 52-matrix product, its FP64 pipe 92% busy while they were).
__global__ void bspmv_kernel(const BSolveDesc* desc, const int2* blocks) {
  const int2 bl = blocks[blockIdx.x];
  const BSolveDesc c = desc[bl.x];
  if (c.nr == 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(c.spmv_blocks) * (blockDim.x >> 5);
  for (int64_t k = int64_t(bl.y) * (blockDim.x >> 5) + (threadIdx.x >> 5); k < c.n; k += warps)
    dev::symv_index_any(k, lane, c.colptr, c.rowidx, c.rptr, c.rcol, c.rval, c.values, c.d, c.nr, 1, c.y, c.n, c.nr);
}

// r = b - y and the squared norms per right-hand side (grid.z = right-hand side)
__global__ void bresidual_kernel(const BSolveDesc* desc) {
  __shared__ double rr[256], bb[256];
  const BSolveDesc c = desc[blockIdx.y];
  const int r = blockIdx.z;
  if (r >= c.nr) return;
  double sr = 0.0, sb = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < c.n; i += int64_t(gridDim.x) * blockDim.x) {
    const double bv = c.b[i + r * c.n];
    const double dv = bv - c.y[i + r * c.n];
    c.r[i + r * c.n] = dv;
    sr = fma(dv, dv, sr);
    sb = fma(bv, bv, sb);
  }
  rr[threadIdx.x] = sr;
  bb[threadIdx.x] = sb;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      bb[threadIdx.x] += bb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(c.norms + 2 * r, rr[0]);
    atomicAdd(c.norms + 2 * r + 1, bb[0]);
  }
}

struct BatchLogCtx {
  const double* tiles;      // FP64 factor tiles (FP64 path)
  const int32_t* diag_sub;  // diagonal sub-tile of each sub-column
  const double* ldiag;      // FP64 diagonal entries (mixed-precision path)
  int64_t n;
  int B;
  int pad0;
};

// One block per matrix, each summing 2 log L_ii over its rows in a fixed order.
__global__ void batch_logdet_kernel(const BatchLogCtx* ctx, double* out) {
  __shared__ double red[256];
  const BatchLogCtx c = ctx[blockIdx.x];
  double s = 0.0;
  for (int64_t g = threadIdx.x; g < c.n; g += blockDim.x) {
    const double l = c.ldiag ? c.ldiag[g]
                             : c.tiles[int64_t(c.diag_sub[g / c.B]) * c.B * c.B + (g % c.B) * c.B + (g % c.B)];
    s += 2.0 * log(l);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Batch arrays come from the device's stream-ordered memory pool, allocated
// and freed on the batch's private stream: creating and destroying batches in a
// serving loop then neither maps fresh device pages each time nor waits for the
// whole device (as a cudaFree may while other streams run).  The pool keeps
// freed memory for reuse (release threshold raised once per device).
void keep_pool_memory(int device) {
  static std::mutex m;
  static std::vector<int> done;
  std::lock_guard<std::mutex> lock(m);
  if (std::find(done.begin(), done.end(), device) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t threshold = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  cudaGetLastError();
  done.push_back(device);
}

template <class T>
cudaError_t batch_alloc(stiles_batch* b, T** p, size_t count) {
  return cudaMallocAsync(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T), b->stream);
}

template <class T>
cudaError_t batch_upload(stiles_batch* b, T** p, const std::vector<T>& v) {
  cudaError_t e = batch_alloc(b, p, v.size());
  if (e == cudaSuccess && !v.empty())
    e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream);
  return e;
}

void free_batch(stiles_batch* b) {
  if (!b) return;
  for (stiles_factor* v : b->views) free_factor(v);
  // batch arrays come from the stream-ordered pool (batch_alloc)
  auto release = [&](void* q) {
    if (q) cudaFreeAsync(q, b->stream);
  };
  release(b->values);
  release(b->dscatter);
  release(b->tiles);
  release(b->scratch);
  release(b->invdiag);
  release(b->linv);
  release(b->linv32);
  release(b->slices);
  release(b->rowexp);
  release(b->drowexp);
  release(b->dinv);
  release(b->dinv32);
  release(b->dspmv);
  release(b->dmlast);
  release(b->tiles32);
  release(b->tiles16);
  release(b->scratch32);
  release(b->invdiag32);
  release(b->ldiag);
  release(b->flags);
  release(b->infos);
  release(b->ctl);
  release(b->dmats);
  release(b->dtickets);
  release(b->logdet_out);
  release(b->dlog);
  release(b->vctl);
  release(b->vlog);
  release(b->vnorm);
  release(b->sY);
  release(b->sScr);
  release(b->sFlags);
  release(b->vb);
  release(b->vx);
  release(b->vr);
  release(b->vd);
  release(b->vy);
  release(b->vnorms);
  release(b->sctl);
  release(b->dfwd);
  release(b->dbwd);
  release(b->ddesc);
  release(b->tfwd);
  release(b->tbwd);
  for (int32_t** q : {&b->rq_cptr_f, &b->rq_cons_f, &b->rq_cnt0_f, &b->rq_src_f, &b->rq_cptr_b, &b->rq_cons_b,
                       &b->rq_cnt0_b, &b->rq_src_b, &b->rq_call_f, &b->rq_call_b})
    release(*q);
  release(b->rq_slots);
  release(b->rq_cnt);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_k0) cudaEventDestroy(b->ev_k0);
  if (b->ev_k1) cudaEventDestroy(b->ev_k1);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Enqueue the per-call device work after the values are in place.
stiles_status batch_enqueue(stiles_batch* b, cudaStream_t st) {
  const size_t tbytes = b->lp ? sizeof(float) : sizeof(double);
  const int count = int(b->plans.size());
  // The per-matrix helper grids below span the largest matrix up to a cap that
  // does not shrink with the batch (blocks past a smaller matrix's end leave at
  // once): a cap of 148 x k / count blocks left the largest matrices' entries
  // and diagonal tiles to a few SMs.
  const dim3 sg(unsigned(std::max<int64_t>(1, std::min<int64_t>((b->max_scatter + 255) / 256,
                                                                  std::max<int64_t>(256, 148 * 32 / count)))),
                unsigned(count));
  const BScatter* sd = static_cast<const BScatter*>(b->dscatter);
  if (b->lp) {
    CUDA_TRY(cudaMemsetAsync(b->tiles32, 0, size_t(b->tile_elems) * tbytes, st));
    bscatter_kernel<float><<<sg, 256, 0, st>>>(b->tiles32, b->values, sd);
  } else {
    CUDA_TRY(cudaMemsetAsync(b->tiles, 0, size_t(b->tile_elems) * tbytes, st));
    bscatter_kernel<double><<<sg, 256, 0, st>>>(b->tiles, b->values, sd);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(b->flags, 0, size_t(b->flag_total) * sizeof(int), st));
  CUDA_TRY(cudaMemsetAsync(b->infos, 0xFF, b->plans.size() * sizeof(unsigned long long), st));
  dev::init_ctl_kernel<<<1, 32, 0, st>>>(b->ctl, 1);
  CUDA_TRY(cudaGetLastError());
  if (b->sliced) {
    const dim3 gr(unsigned(std::max<int64_t>(1, std::min<int64_t>((b->max_nsb * 32 + 255) / 256,
                                                                    std::max<int64_t>(64, 148 * 8 / count)))),
                  unsigned(count));
    dev::oz_browexp_kernel<<<gr, 256, 0, st>>>(static_cast<const dev::OZRowexpDesc*>(b->drowexp));
    CUDA_TRY(cudaGetLastError());
  }
  CUDA_TRY(cudaEventRecordWithFlags(b->ev_k0, st, cudaEventRecordExternal));  // a node of the captured graph
  if (b->sliced) {
    dev::OZArgs a{};
    a.mats = static_cast<const dev::OZMatCtx*>(b->dmats);
    a.tickets = b->dtickets;
    a.ntasks = b->ntickets;
    a.ctl = b->ctl;
    a.spin_limit = b->spin_limit;
    dev::factor_oz_kernel<<<b->grid, dev::OZ_THREADS, dev::OZ_KERNEL_SMEM, st>>>(a);
  } else if (b->lp) {
    dev::LPArgs a{};
    a.mats = static_cast<const dev::LPMatCtx*>(b->dmats);
    a.tickets = b->dtickets;
    a.ntasks = b->ntickets;
    a.ctl = b->ctl;
    a.spin_limit = b->spin_limit;
    a.fp16 = b->fp16;
    dev::factor_lp_kernel<<<b->grid, dev::LP_THREADS, dev::LP_KERNEL_SMEM, st>>>(a);
  } else {
    dev::FactorArgs a{};
    a.mats = static_cast<const dev::MatCtx*>(b->dmats);
    a.tickets = b->dtickets;
    a.ntasks = b->ntickets;
    a.ctl = b->ctl;
    a.spin_limit = b->spin_limit;
    switch (b->B) {
      case 16: dev::factor_f64_kernel<16><<<b->grid, 128, dev::FactorCfg<16>::SMEM, st>>>(a); break;
      case 32: dev::factor_f64_kernel<32><<<b->grid, 128, dev::FactorCfg<32>::SMEM, st>>>(a); break;
      default: dev::factor_f64_kernel<64><<<b->grid, 128, dev::FactorCfg<64>::SMEM, st>>>(a); break;
    }
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecordWithFlags(b->ev_k1, st, cudaEventRecordExternal));
  {
    const int count = int(b->plans.size());
    const dim3 g(unsigned(std::max<int64_t>(1, std::min<int64_t>((b->max_nsb * 32 + 255) / 256,
                                                                   std::max<int64_t>(128, 148 * 16 / count)))),
                 unsigned(count));
    const BInverse* di = static_cast<const BInverse*>(b->dinv);
    if (b->lp) bdiag_inverse_kernel<64, float><<<g, 256, 0, st>>>(di);
    else switch (b->B) {
      case 16: bdiag_inverse_kernel<16, double><<<g, 256, 0, st>>>(di); break;
      case 32: bdiag_inverse_kernel<32, double><<<g, 256, 0, st>>>(di); break;
      default: bdiag_inverse_kernel<64, double><<<g, 256, 0, st>>>(di); break;
    }
    CUDA_TRY(cudaGetLastError());
    if (b->sliced) {  // the FP32 copies that the sweeps read (see launch_diag_inverse)
      dev::to_f32_kernel<<<grid_for(b->tile_elems, 256), 256, 0, st>>>(b->tiles32, b->tiles, b->tile_elems);
      dev::to_f32_kernel<<<grid_for(b->diag_elems, 256), 256, 0, st>>>(b->invdiag32, b->invdiag, b->diag_elems);
      bdiag_inverse_kernel<32, float><<<g, 256, 0, st>>>(static_cast<const BInverse*>(b->dinv32));
      CUDA_TRY(cudaGetLastError());
      return STILES_OK;
    }
    // x spans the largest matrix's products (CTAs past a smaller matrix's end leave at once):
    // x = 148 * 8 / count left the largest matrices' products nearly serial (~11 ms of a
    // 256-matrix batch at B = 16, ~70 ms at B = 32)
    const dim3 gm(unsigned(std::max<int64_t>(1, std::min<int64_t>(b->max_stasks, 148 * 8))), unsigned(count));
    const dev::MlastDesc* dm = static_cast<const dev::MlastDesc*>(b->dmlast);
    if (!b->lp) switch (b->B) {
      case 16: dev::bmlast_kernel<16, double><<<gm, 128, 0, st>>>(dm); break;
      case 32: dev::bmlast_kernel<32, double><<<gm, 128, 0, st>>>(dm); break;
      default: dev::bmlast_kernel<64, double><<<gm, 128, 0, st>>>(dm); break;
    }
    CUDA_TRY(cudaGetLastError());
  }
  return STILES_OK;
}

// Merged ticket order of per-matrix task lists: matrix i's task j sits at
// (j + 0.5) / n_i (ties by matrix), so every matrix keeps its own order.
std::vector<int2> merge_tickets(const std::vector<int64_t>& lens) {
  std::vector<std::pair<double, int2>> keyed;
  for (size_t i = 0; i < lens.size(); ++i)
    for (int64_t j = 0; j < lens[i]; ++j)
      keyed.push_back({(double(j) + 0.5) / double(lens[i]), make_int2(int(i), int(j))});
  std::stable_sort(keyed.begin(), keyed.end(), [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) {
    return x.first < y.first;
  });
  std::vector<int2> tick(keyed.size());
  for (size_t q = 0; q < keyed.size(); ++q) tick[q] = keyed[q].second;
  return tick;
}

// Release lists of one sweep for a ready-queue launch, appended to a batch's
// arrays with ticket offset off: per task the tasks that read its output (CSR,
// each reader once), the number of distinct tasks it reads from, and the tasks
// that read from none.  Producers: block k is written by the FINAL task with
// out = k, scratch block s by the tree task with out = s.
bool append_release(const stiles::SolveGraph& g, int64_t nsb, int32_t off, std::vector<int32_t>& cptr,
                    std::vector<int32_t>& cons, std::vector<int32_t>& cnt0, std::vector<int32_t>& src) {
  const int32_t n = int32_t(g.tasks.size());
  std::vector<int32_t> blk(size_t(nsb), -1), scr(size_t(std::max<int64_t>(g.nscratch, 1)), -1);
  for (int32_t t = 0; t < n; ++t) {
    const stiles::SolveTask& tk = g.tasks[size_t(t)];
    (tk.type == stiles::SOLVE_FINAL ? blk : scr)[size_t(tk.out)] = t;
  }
  std::vector<int32_t> stamp(size_t(n), -1), ep, ec, deg(size_t(n) + 1, 0);
  const size_t c0 = cnt0.size();
  cnt0.resize(c0 + size_t(n), 0);
  auto edge = [&](int32_t pr, int32_t t) {
    if (pr < 0 || pr >= t) return false;  // every producer precedes its reader in the list
    if (stamp[size_t(pr)] != t) {
      stamp[size_t(pr)] = t;
      ep.push_back(pr);
      ec.push_back(t);
      ++deg[size_t(pr) + 1];
      ++cnt0[c0 + size_t(t)];
    }
    return true;
  };
  for (int32_t t = 0; t < n; ++t) {
    const stiles::SolveTask& tk = g.tasks[size_t(t)];
    for (int32_t q = tk.pb; q < tk.pe; ++q)
      if (!edge(blk[size_t(g.pairs[2 * size_t(q) + 1])], t)) return false;
    for (int32_t q = tk.qb; q < tk.qe; ++q)
      if (!edge(scr[size_t(g.parts[size_t(q)])], t)) return false;
  }
  for (int32_t t = 0; t < n; ++t) deg[size_t(t) + 1] += deg[size_t(t)];
  const int32_t base = int32_t(cons.size());
  cons.resize(cons.size() + ep.size());
  std::vector<int32_t> fill(deg.begin(), deg.end() - 1);
  for (size_t e = 0; e < ep.size(); ++e) cons[size_t(base) + size_t(fill[size_t(ep[e])]++)] = off + ec[e];
  for (int32_t t = 0; t < n; ++t) cptr.push_back(base + deg[size_t(t) + 1]);
  for (int32_t t = 0; t < n; ++t)
    if (cnt0[c0 + size_t(t)] == 0) src.push_back(off + t);
  return true;
}

// Device workspace of batched solves, allocated on the first call: per
// matrix room for SOLVE_MAXR right-hand sides in every vector.
stiles_status ensure_batch_solve(stiles_batch* b) {
  if (b->solve_ready) return STILES_OK;
  const int count = int(b->plans.size());
  if (count > 65535) return fail(STILES_ERR_UNSUPPORTED, "batched solves take at most 65535 matrices");
  const int64_t R = dev::SOLVE_MAXR;
  int64_t ytot = 0, stot = 0, ftot = 0, vtot = 0;
  std::vector<int64_t> lf(count), lb(count);
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = b->plans[i];
    const int64_t nf = std::max<int64_t>(p->fwd.nscratch, 1), nb = std::max<int64_t>(p->bwd.nscratch, 1);
    b->y_off.push_back(ytot);
    b->scr_off.push_back(stot);
    b->flag_off.push_back(ftot);
    b->vec_off.push_back(vtot);
    ytot += p->nsb * p->B * R;
    stot += (nf + nb) * p->B * R;
    ftot += 2 * p->nsb + nf + nb;
    vtot += p->n * R;
    lf[i] = int64_t(p->fwd.tasks.size());
    lb[i] = int64_t(p->bwd.tasks.size());
  }
  b->vec_total = vtot;
  b->sflag_total = ftot;
  // tickets: every matrix's list in turn; release lists over those tickets
  std::vector<int2> tf, tb;
  std::vector<int32_t> cpf{0}, cnf, c0f, cpb{0}, cnb, c0b;
  b->src_f.clear();
  b->src_b.clear();
  b->src_f_off.assign(1, 0);
  b->src_b_off.assign(1, 0);
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = b->plans[i];
    if (int64_t(tf.size()) + lf[i] >= (int64_t(1) << 31) || int64_t(tb.size()) + lb[i] >= (int64_t(1) << 31) ||
        int64_t(cnf.size()) + int64_t(p->fwd.pairs.size() / 2 + p->fwd.parts.size()) >= (int64_t(1) << 31) ||
        int64_t(cnb.size()) + int64_t(p->bwd.pairs.size() / 2 + p->bwd.parts.size()) >= (int64_t(1) << 31))
      return fail(STILES_ERR_UNSUPPORTED, "too many solve tasks in one batch");
    if (!append_release(p->fwd, p->nsb, int32_t(tf.size()), cpf, cnf, c0f, b->src_f) ||
        !append_release(p->bwd, p->nsb, int32_t(tb.size()), cpb, cnb, c0b, b->src_b))
      return fail(STILES_ERR_INVALID, "internal: a sweep task reads an output produced after it");
    for (int64_t j = 0; j < lf[i]; ++j) tf.push_back(make_int2(i, int(j)));
    for (int64_t j = 0; j < lb[i]; ++j) tb.push_back(make_int2(i, int(j)));
    b->src_f_off.push_back(int64_t(b->src_f.size()));
    b->src_b_off.push_back(int64_t(b->src_b.size()));
  }
  b->nfwd = int(tf.size());
  b->nbwd = int(tb.size());
  const size_t ctx_bytes = (b->lp || b->sliced) ? sizeof(dev::SolveCtx<float>) : sizeof(dev::SolveCtx<double>);
  cudaError_t e = batch_alloc(b, &b->sY, size_t(ytot));
  if (e == cudaSuccess) e = batch_alloc(b, &b->sScr, size_t(stot));
  if (e == cudaSuccess) e = batch_alloc(b, &b->sFlags, size_t(ftot));
  for (double** v : {&b->vb, &b->vx, &b->vr, &b->vd, &b->vy})
    if (e == cudaSuccess) e = batch_alloc(b, v, size_t(vtot));
  if (e == cudaSuccess) e = batch_alloc(b, &b->vnorms, size_t(count) * 2 * R);
  if (e == cudaSuccess) e = batch_alloc(b, &b->sctl, 2);
  if (e == cudaSuccess) e = batch_alloc(b, reinterpret_cast<unsigned char**>(&b->dfwd), size_t(count) * ctx_bytes);
  if (e == cudaSuccess) e = batch_alloc(b, reinterpret_cast<unsigned char**>(&b->dbwd), size_t(count) * ctx_bytes);
  if (e == cudaSuccess) e = batch_alloc(b, reinterpret_cast<BSolveDesc**>(&b->ddesc), size_t(count));
  if (e == cudaSuccess) e = batch_upload(b, &b->tfwd, tf);
  if (e == cudaSuccess) e = batch_upload(b, &b->tbwd, tb);
  {
    // blocks of the batched A x: 148 x 32 in all, in proportion to each matrix's
    // nonzeros (at least one, at most one warp per index), largest matrix first
    std::vector<int> ord(count);
    std::iota(ord.begin(), ord.end(), 0);
    double wsum = 0.0;
    for (int i = 0; i < count; ++i) wsum += double(b->plans[i]->nnz);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return b->plans[x]->nnz > b->plans[y]->nnz; });
    b->spmv_blocks.assign(count, 1);
    std::vector<int2> sb;
    for (int i : ord) {
      const stiles_plan* p = b->plans[i];
      const int64_t cap = std::max<int64_t>(1, (p->n + 7) / 8);
      const int64_t nb = std::min<int64_t>(cap, std::max<int64_t>(1, int64_t(148.0 * 32.0 * double(p->nnz) / wsum + 0.5)));
      b->spmv_blocks[i] = int(nb);
      for (int64_t j = 0; j < nb; ++j) sb.push_back(make_int2(i, int(j)));
    }
    b->nspmv = int(sb.size());
    if (e == cudaSuccess) e = batch_upload(b, &b->dspmv, sb);
  }
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_cptr_f, cpf);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_cons_f, cnf);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_cnt0_f, c0f);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_src_f, b->src_f);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_cptr_b, cpb);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_cons_b, cnb);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_cnt0_b, c0b);
  if (e == cudaSuccess) e = batch_upload(b, &b->rq_src_b, b->src_b);
  if (e == cudaSuccess) e = batch_alloc(b, &b->rq_slots, std::max(tf.size(), tb.size()));
  if (e == cudaSuccess) e = batch_alloc(b, &b->rq_cnt, std::max(tf.size(), tb.size()));
  if (e == cudaSuccess) e = batch_alloc(b, &b->rq_call_f, std::max<size_t>(b->src_f.size(), 1));
  if (e == cudaSuccess) e = batch_alloc(b, &b->rq_call_b, std::max<size_t>(b->src_b.size(), 1));
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // the arrays are used from the caller's streams
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,
                std::string("batched solve allocation: ") + cudaGetErrorString(e));
  }
  int sms = 0, per_sm = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  cudaError_t oe;
  if (b->lp) oe = solve_occupancy<64, float>(&per_sm);
  else if (b->sliced) oe = solve_occupancy<32, float>(&per_sm);
  else switch (b->B) {
    case 16: oe = solve_occupancy<16, double>(&per_sm); break;
    case 32: oe = solve_occupancy<32, double>(&per_sm); break;
    default: oe = solve_occupancy<64, double>(&per_sm); break;
  }
  if (oe != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("occupancy: ") + cudaGetErrorString(oe));
  if (b->plans[0]->opts.ctas_per_sm > 0) per_sm = std::min(per_sm, int(b->plans[0]->opts.ctas_per_sm));
  b->solve_grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(std::max(per_sm, 1)) * sms,
                                                            std::max(b->nfwd, b->nbwd))));
  b->solve_ready = true;
  return STILES_OK;
}

// Upload the per-call contexts (they carry each matrix's right-hand-side count).
template <typename TF>
stiles_status upload_solve_ctx(stiles_batch* b, const std::vector<int>& nr, cudaStream_t st) {
  const int count = int(b->plans.size());
  std::vector<dev::SolveCtx<TF>> cf(count), cb(count);
  std::vector<BSolveDesc> desc(count);
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = b->plans[i];
    const stiles_factor* v = b->views[i];
    const TF* tiles;
    const TF* inv;
    const TF* linv;
    if constexpr (sizeof(TF) == 4) {
      tiles = v->tiles32;
      inv = v->invdiag32;
      linv = v->linv32;
    } else {
      tiles = v->tiles;
      inv = v->invdiag;
      linv = v->linv;
    }
    TF* Y = reinterpret_cast<TF*>(b->sY) + b->y_off[i];  // double-sized buffers also hold FP32 sweeps
    TF* scr = reinterpret_cast<TF*>(b->sScr) + b->scr_off[i];
    cf[i] = solve_ctx<TF>(p, nullptr, false, nr[i], tiles, inv, linv, Y, scr, b->sFlags + b->flag_off[i]);
    cb[i] = solve_ctx<TF>(p, nullptr, true, nr[i], tiles, inv, linv, Y, scr, b->sFlags + b->flag_off[i]);
    BSolveDesc& d = desc[i];
    d.perm = p->dev->perm;
    d.n = p->n;
    d.nsb = p->nsb;
    d.B = p->B;
    d.nr = nr[i];
    d.spmv_blocks = b->spmv_blocks[i];
    d.Y = Y;
    d.b = b->vb + b->vec_off[i];
    d.x = b->vx + b->vec_off[i];
    d.r = b->vr + b->vec_off[i];
    d.d = b->vd + b->vec_off[i];
    d.y = b->vy + b->vec_off[i];
    d.colptr = p->dev->colptr;
    d.rowidx = p->dev->rowidx;
    d.rptr = p->dev->rptr;
    d.rcol = p->dev->rcol;
    d.rval = p->dev->rval;
    d.values = v->values;
    d.norms = b->vnorms + size_t(i) * 2 * dev::SOLVE_MAXR;
  }
  // synchronous copies: the host vectors go out of scope on return
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaMemcpy(b->dfwd, cf.data(), count * sizeof(cf[0]), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->dbwd, cb.data(), count * sizeof(cb[0]), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->ddesc, desc.data(), count * sizeof(desc[0]), cudaMemcpyHostToDevice));
  return STILES_OK;
}

// One batched solve call: the source tickets of the matrices that take part and
// their task counts (every matrix, or only those with right-hand sides).
struct SweepTickets {
  const int32_t* src_f;
  const int32_t* src_b;
  int nsrc_f, nsrc_b;
  int nfwd, nbwd;  // tasks handed out
  int nmat;        // matrices taking part
};

// Both sweeps of a batched solve as ready-queue launches over the batch's
// tickets: a task enters the queue once every task it reads from has started,
// so the persistent CTAs take tasks in the order the matrices' chains reach
// them rather than in one fixed interleaving of all the lists (256 matrices
// with ND plans: FP64 solves 12% faster, FP32 ones ~10%).  For FP64 sweeps what
// remains is the FP64 pipe: seven CTAs share an SM's 2 FMA a cycle, so a chain
// task next to heavy tree partials runs several times slower than alone.
template <int B, typename TF>
cudaError_t launch_batch_sweeps(stiles_batch* b, const SweepTickets& tk, cudaStream_t st) {
  dev::SolveArgs<TF> a{};
  a.spin_limit = b->spin_limit;
  a.mats = static_cast<const dev::SolveCtx<TF>*>(b->dfwd);
  a.tickets = b->tfwd;
  a.ntasks = tk.nfwd;
  a.ctl = b->sctl;
  a.rq_slots = b->rq_slots;
  a.rq_cnt = b->rq_cnt;
  a.rq_cptr = b->rq_cptr_f;
  a.rq_cons = b->rq_cons_f;
  const int gf = std::max(1, std::min({b->solve_grid, tk.nfwd, kSolveCtasPerMatrix * tk.nmat}));
  const int gb = std::max(1, std::min({b->solve_grid, tk.nbwd, kSolveCtasPerMatrix * tk.nmat}));
  const int gr = int(std::min<int64_t>(1184, (std::max(b->nfwd, b->nbwd) + 255) / 256));
  dev::rq_reset_kernel<<<gr, 256, 0, st>>>(b->rq_slots, b->rq_cnt, b->rq_cnt0_f, tk.src_f, tk.nsrc_f, b->nfwd,
                                           b->sctl);
  dev::solve_kernel<B, false, TF><<<gf, 128, dev::SolveCfg<B, TF>::SMEM, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  a.mats = static_cast<const dev::SolveCtx<TF>*>(b->dbwd);
  a.tickets = b->tbwd;
  a.ntasks = tk.nbwd;
  a.ctl = b->sctl + 1;
  a.rq_cptr = b->rq_cptr_b;
  a.rq_cons = b->rq_cons_b;
  dev::rq_reset_kernel<<<gr, 256, 0, st>>>(b->rq_slots, b->rq_cnt, b->rq_cnt0_b, tk.src_b, tk.nsrc_b, b->nbwd,
                                           b->sctl + 1);
  dev::solve_kernel<B, true, TF><<<gb, 128, dev::SolveCfg<B, TF>::SMEM, st>>>(a);
  return cudaGetLastError();
}

// Grid of the per-matrix helper kernels: x covers the largest matrix, y the matrices.
dim3 batch_grid(const stiles_batch* b, int64_t max_work) {
  const int64_t count = int64_t(b->plans.size());
  const int64_t cap = std::max<int64_t>(1, 148 * 32 / count);
  return dim3(unsigned(std::max<int64_t>(1, std::min<int64_t>((max_work + 255) / 256, cap))), unsigned(count));
}

// One solve of every matrix: which = 0 solves b into x, which = 1 solves r into d.
stiles_status batch_solve_pass(stiles_batch* b, const SweepTickets& tk, cudaStream_t st, int which,
                               int64_t max_rows) {
  const BSolveDesc* desc = static_cast<const BSolveDesc*>(b->ddesc);
  const dim3 g = batch_grid(b, max_rows * dev::SOLVE_MAXR);
  if (b->lp || b->sliced) bpermute_in_kernel<float><<<g, 256, 0, st>>>(desc, which);
  else bpermute_in_kernel<double><<<g, 256, 0, st>>>(desc, which);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(b->sFlags, 0, size_t(b->sflag_total) * sizeof(int), st));
  dev::init_ctl_kernel<<<1, 32, 0, st>>>(b->sctl, 2);
  CUDA_TRY(cudaGetLastError());
  cudaError_t e;
  if (b->lp) e = launch_batch_sweeps<64, float>(b, tk, st);
  else if (b->sliced) e = launch_batch_sweeps<32, float>(b, tk, st);
  else switch (b->B) {
    case 16: e = launch_batch_sweeps<16, double>(b, tk, st); break;
    case 32: e = launch_batch_sweeps<32, double>(b, tk, st); break;
    default: e = launch_batch_sweeps<64, double>(b, tk, st); break;
  }
  if (e != cudaSuccess) return fail(STILES_ERR_CUDA, std::string("batched solve launch: ") + cudaGetErrorString(e));
  if (b->lp || b->sliced) bpermute_out_kernel<float><<<g, 256, 0, st>>>(desc, which);
  else bpermute_out_kernel<double><<<g, 256, 0, st>>>(desc, which);
  CUDA_TRY(cudaGetLastError());
  count_launch(7);
  dev::Ctl c[2];
  CUDA_TRY(cudaMemcpyAsync(c, b->sctl, sizeof(c), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < 2; ++k)
    if (c[k].status != 0) {
      char buf[96];
      std::snprintf(buf, sizeof buf, "device wait timed out in the batched %s sweep (ticket %lld)",
                    k ? "backward" : "forward", c[k].where);
      return fail(STILES_ERR_TIMEOUT, buf);
    }
  return STILES_OK;
}

// r = b - A x for every matrix and ||r|| / ||b|| per matrix (largest over its columns).
stiles_status batch_residual(stiles_batch* b, cudaStream_t st, int64_t max_rows, const std::vector<int>& nr,
                             std::vector<double>* rel) {
  const BSolveDesc* desc = static_cast<const BSolveDesc*>(b->ddesc);
  const int count = int(b->plans.size());
  CUDA_TRY(cudaMemsetAsync(b->vnorms, 0, size_t(count) * 2 * dev::SOLVE_MAXR * sizeof(double), st));
  binterleave_kernel<<<batch_grid(b, max_rows * dev::SOLVE_MAXR), 256, 0, st>>>(desc);
  bspmv_kernel<<<unsigned(b->nspmv), 256, 0, st>>>(desc, b->dspmv);
  CUDA_TRY(cudaGetLastError());
  dim3 g = batch_grid(b, max_rows);
  g.z = dev::SOLVE_MAXR;
  bresidual_kernel<<<g, 256, 0, st>>>(desc);
  CUDA_TRY(cudaGetLastError());
  count_launch(3);
  std::vector<double> h(size_t(count) * 2 * dev::SOLVE_MAXR);
  CUDA_TRY(cudaMemcpyAsync(h.data(), b->vnorms, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  rel->assign(count, 0.0);
  for (int i = 0; i < count; ++i)
    for (int r = 0; r < nr[i]; ++r) {
      const double* q = h.data() + size_t(i) * 2 * dev::SOLVE_MAXR + 2 * r;
      const double w = q[1] > 0 ? std::sqrt(q[0] / q[1]) : std::sqrt(q[0]);
      if (!(w <= (*rel)[i])) (*rel)[i] = w;  // NaN propagates
    }
  return STILES_OK;
}

__global__ void baxpy_active_kernel(const BSolveDesc* desc, const int* active) {
  if (!active[blockIdx.y]) return;
  const BSolveDesc c = desc[blockIdx.y];
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < c.n * c.nr; e += int64_t(gridDim.x) * blockDim.x)
    c.x[e] += c.d[e];
}

}  // namespace

extern "C" {

stiles_status stiles_batch_create(const stiles_plan* const* plans, int32_t count, stiles_batch** out) {
  if (!plans || count < 1 || !out) return fail(STILES_ERR_INVALID, "bad argument");
  *out = nullptr;
  if (count > 65535) return fail(STILES_ERR_UNSUPPORTED, "a batch holds at most 65,535 matrices");
  stiles_batch* b = new (std::nothrow) stiles_batch();
  if (!b) return fail(STILES_ERR_NOMEM, "host allocation");
  auto bail = [&](stiles_status s) {
    free_batch(b);
    return s;
  };
  b->plans.assign(plans, plans + count);
  if (!plans[0]) return bail(fail(STILES_ERR_INVALID, "null plan"));
  b->sliced = plans[0]->opts.precision == STILES_PREC_SLICED;
  b->lp = plans[0]->opts.precision != STILES_PREC_F64 && !b->sliced;
  b->B = plans[0]->B;
  b->fp16 = plans[0]->opts.precision == STILES_PREC_F16 ? 1 : 0;
  b->spin_limit = plans[0]->opts.spin_limit;
  CUDA_TRY(cudaGetDevice(&b->device));
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = plans[i];
    if (!p || p->opts.precision != plans[0]->opts.precision || p->B != b->B)
      return bail(fail(STILES_ERR_INVALID, "batched plans must share precision and block size"));
    stiles_status s = ensure_dev_plan(p);
    if (s != STILES_OK) return bail(s);
    b->spin_limit = std::max<long long>(b->spin_limit, p->opts.spin_limit);
  }
  // offsets of every matrix inside the concatenated arrays
  const int64_t TB = int64_t(b->B) * b->B;
  std::vector<int64_t> t_off(count), s_off(count), d_off(count), f_off(count);
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = plans[i];
    b->val_off.push_back(b->nnz_total);
    t_off[i] = b->tile_elems;
    s_off[i] = b->scratch_elems;
    d_off[i] = b->diag_elems;
    f_off[i] = b->flag_total;
    b->nnz_total += p->nnz;
    b->pad_total += int64_t(p->pad.size());
    b->tile_elems += p->nsub * TB;
    b->scratch_elems += std::max<int64_t>(p->graph.nscratch, 1) * TB;
    b->diag_elems += p->nsb * b->B;
    b->flag_total += p->nsub + p->nsb + std::max<int64_t>(p->graph.nscratch, 1);  // the factor flag layout
  }
  std::vector<BScatter> scat(count);
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = plans[i];
    scat[i] = BScatter{p->dev->scatter, p->dev->pad, p->nnz, int64_t(p->pad.size()), b->val_off[i], t_off[i]};
    b->max_scatter = std::max<int64_t>(b->max_scatter, std::max<int64_t>(p->nnz, int64_t(p->pad.size())));
  }
  keep_pool_memory(b->device);
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = batch_alloc(b, &b->values, size_t(b->nnz_total));
  if (e == cudaSuccess) e = batch_upload(b, reinterpret_cast<BScatter**>(&b->dscatter), scat);
  if (e == cudaSuccess && !b->lp) e = batch_alloc(b, &b->tiles, size_t(b->tile_elems));
  if (e == cudaSuccess && !b->lp) e = batch_alloc(b, &b->scratch, size_t(b->scratch_elems));
  if (e == cudaSuccess && !b->lp) e = batch_alloc(b, &b->invdiag, size_t(b->diag_elems));
  if (e == cudaSuccess && !b->lp) e = batch_alloc(b, &b->linv, 5 * size_t(b->diag_elems) * b->B);
  if (e == cudaSuccess && b->sliced) e = batch_alloc(b, &b->slices, size_t(b->tile_elems) * dev::OZ_NSLICE);
  if (e == cudaSuccess && b->sliced) e = batch_alloc(b, &b->rowexp, size_t(b->diag_elems));
  if (e == cudaSuccess && b->sliced) e = batch_alloc(b, &b->tiles32, size_t(b->tile_elems));
  if (e == cudaSuccess && b->sliced) e = batch_alloc(b, &b->invdiag32, size_t(b->diag_elems));
  if (e == cudaSuccess && b->sliced) e = batch_alloc(b, &b->linv32, size_t(b->diag_elems) * b->B);
  if (e == cudaSuccess && b->lp) e = batch_alloc(b, &b->tiles32, size_t(b->tile_elems));
  if (e == cudaSuccess && b->lp) e = batch_alloc(b, &b->tiles16, size_t(b->tile_elems));
  if (e == cudaSuccess && b->lp) e = batch_alloc(b, &b->scratch32, size_t(b->scratch_elems));
  if (e == cudaSuccess && b->lp) e = batch_alloc(b, &b->invdiag32, size_t(b->diag_elems));
  if (e == cudaSuccess && b->lp) e = batch_alloc(b, &b->ldiag, size_t(b->diag_elems));
  if (e == cudaSuccess && b->lp) e = batch_alloc(b, &b->linv32, size_t(b->diag_elems) * b->B);
  if (e == cudaSuccess) e = batch_alloc(b, &b->flags, size_t(b->flag_total));
  if (e == cudaSuccess) e = batch_alloc(b, &b->infos, size_t(count));
  if (e == cudaSuccess) e = batch_alloc(b, &b->ctl, 1);
  if (e == cudaSuccess) e = batch_alloc(b, &b->logdet_out, size_t(count));
  if (e == cudaSuccess) e = batch_alloc(b, &b->vctl, size_t(count) * 3);
  if (e == cudaSuccess) e = batch_alloc(b, &b->vlog, size_t(count) * (dev::LOGDET_BLOCKS + 1));
  if (e == cudaSuccess) e = batch_alloc(b, &b->vnorm, size_t(count) * 2 * dev::SOLVE_MAXR);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(e == cudaErrorMemoryAllocation ? STILES_ERR_NOMEM : STILES_ERR_CUDA,
                     std::string("batch allocation: ") + cudaGetErrorString(e)));
  }
  // factor views and per-matrix contexts
  std::vector<dev::MatCtx> mats;
  std::vector<dev::LPMatCtx> lmats;
  std::vector<dev::OZMatCtx> omats;
  std::vector<dev::OZRowexpDesc> orow;
  std::vector<BatchLogCtx> logs(count);
  std::vector<BInverse> binv(count), binv32;
  std::vector<dev::MlastDesc> bml(count);
  for (int i = 0; i < count; ++i) {
    const stiles_plan* p = plans[i];
    stiles_factor* v = new (std::nothrow) stiles_factor();
    if (!v) return bail(fail(STILES_ERR_NOMEM, "host allocation"));
    b->views.push_back(v);
    v->plan = p;
    v->device = b->device;
    v->view = true;
    v->lp = b->lp;
    v->sliced = b->sliced;
    v->values = b->values + b->val_off[i];
    v->flags = b->flags + f_off[i];
    v->info = b->infos + i;
    if (b->lp) {
      v->tiles32 = b->tiles32 + t_off[i];
      v->tiles16 = b->tiles16 + t_off[i];
      v->scratch32 = b->scratch32 + s_off[i];
      v->invdiag32 = b->invdiag32 + d_off[i];
      v->linv32 = b->linv32 + d_off[i] * b->B;
      v->ldiag = b->ldiag + d_off[i];
    } else {
      v->tiles = b->tiles + t_off[i];
      v->scratch = b->scratch + s_off[i];
      v->invdiag = b->invdiag + d_off[i];
      v->linv = b->linv + 5 * d_off[i] * b->B;
      if (b->sliced) {
        v->slices = b->slices + t_off[i] * dev::OZ_NSLICE;
        v->rowexp = b->rowexp + d_off[i];
        v->tiles32 = b->tiles32 + t_off[i];
        v->invdiag32 = b->invdiag32 + d_off[i];
        v->linv32 = b->linv32 + d_off[i] * b->B;
        binv32.push_back(BInverse{v->linv32, v->tiles32, v->invdiag32, p->dev->diag_sub, p->nsb});
      }
    }
    // the view's small arrays are slices of batch-wide ones; a view never
    // factorizes, so it has no events
    v->ctl = b->vctl + 3 * size_t(i);
    v->logdet_part = b->vlog + size_t(i) * (dev::LOGDET_BLOCKS + 1);
    v->norms = b->vnorm + size_t(i) * 2 * dev::SOLVE_MAXR;
    if (b->lp) lmats.push_back(lp_mat_ctx(p, v));
    else if (b->sliced) {
      omats.push_back(oz_mat_ctx(p, v));
      omats.back().trace = nullptr;
      orow.push_back(dev::OZRowexpDesc{v->tiles, p->dev->diag_sub, p->nsb, v->rowexp});
    } else mats.push_back(mat_ctx(p, v));
    logs[i] = BatchLogCtx{v->tiles, p->dev->diag_sub, v->ldiag, p->n, b->B, 0};
    binv[i] = BInverse{b->lp ? static_cast<void*>(v->linv32) : static_cast<void*>(v->linv),
                       b->lp ? static_cast<const void*>(v->tiles32) : static_cast<const void*>(v->tiles),
                       b->lp ? static_cast<const void*>(v->invdiag32) : static_cast<const void*>(v->invdiag),
                       p->dev->diag_sub, p->nsb};
    b->max_nsb = std::max<int64_t>(b->max_nsb, p->nsb);
    {
      dev::MlastDesc& md = bml[i];
      const size_t nt = size_t(p->nsb) * b->B * b->B;
      md.mlast = b->lp ? nullptr : static_cast<void*>(v->linv + nt);  // FP64 factors only
      md.mlast2 = b->lp ? nullptr : static_cast<void*>(v->linv + 3 * nt);
      md.linv = binv[i].linv;
      md.tiles = binv[i].tiles;
      md.ftasks = p->dev->fwd.stasks;
      md.fpairs = p->dev->fwd.pairs;
      md.btasks = p->dev->bwd.stasks;
      md.bpairs = p->dev->bwd.pairs;
      md.nf = p->dev->fwd.ntasks;
      md.nb = p->dev->bwd.ntasks;
      md.nsb = p->nsb;
      b->max_stasks = std::max<int64_t>(b->max_stasks, 2 * (int64_t(md.nf) + md.nb));
    }
  }
  if (b->lp) e = batch_upload(b, reinterpret_cast<dev::LPMatCtx**>(&b->dmats), lmats);
  else if (b->sliced) {
    e = batch_upload(b, reinterpret_cast<dev::OZMatCtx**>(&b->dmats), omats);
    if (e == cudaSuccess) e = batch_upload(b, reinterpret_cast<dev::OZRowexpDesc**>(&b->drowexp), orow);
  } else e = batch_upload(b, reinterpret_cast<dev::MatCtx**>(&b->dmats), mats);
  if (e == cudaSuccess) e = batch_upload(b, reinterpret_cast<BatchLogCtx**>(&b->dlog), logs);
  if (e == cudaSuccess) e = batch_upload(b, reinterpret_cast<BInverse**>(&b->dinv), binv);
  if (e == cudaSuccess && b->sliced) e = batch_upload(b, reinterpret_cast<BInverse**>(&b->dinv32), binv32);
  if (e == cudaSuccess) e = batch_upload(b, reinterpret_cast<dev::MlastDesc**>(&b->dmlast), bml);
  if (e != cudaSuccess) return bail(fail(STILES_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e)));
  std::vector<int64_t> lens(count);
  for (int i = 0; i < count; ++i) lens[i] = int64_t(plans[i]->graph.tasks.size());
  std::vector<int2> tick = merge_tickets(lens);
  if (tick.size() >= size_t(1) << 31) return bail(fail(STILES_ERR_UNSUPPORTED, "too many tasks in one batch"));
  b->ntickets = int(tick.size());
  e = batch_upload(b, &b->dtickets, tick);
  if (e != cudaSuccess) return bail(fail(STILES_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e)));
  // persistent grid: as many resident CTAs as fit
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  int per_sm = std::max(1, plans[0]->dev->grid_factor / std::max(1, sms));
  if (b->sliced) {
    per_sm = 1;  // each CTA holds all 512 TMEM columns of its SM
  } else if (b->lp) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dev::factor_lp_kernel, dev::LP_THREADS,
                                                  dev::LP_KERNEL_SMEM);
    per_sm = std::min(per_sm, 4);
  } else {
    switch (b->B) {
      case 16: factor_occupancy<16>(&per_sm); break;
      case 32: factor_occupancy<32>(&per_sm); break;
      default: factor_occupancy<64>(&per_sm); break;
    }
  }
  if (plans[0]->opts.ctas_per_sm > 0) per_sm = std::min(per_sm, int(plans[0]->opts.ctas_per_sm));
  b->grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(std::max(per_sm, 1)) * sms, b->ntickets)));
  // private stream + graph of the per-call work
  CUDA_TRY(cudaStreamSynchronize(b->stream));  // pool arrays in place before other streams use them
  CUDA_TRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreate(&b->ev_k0));
  CUDA_TRY(cudaEventCreate(&b->ev_k1));
  {
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    stiles_status s = batch_enqueue(b, b->stream);
    cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (s != STILES_OK) {
      if (g) cudaGraphDestroy(g);
      return bail(s);
    }
    if (ce != cudaSuccess) return bail(fail(STILES_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce)));
    ce = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return bail(fail(STILES_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce)));
  }
  *out = b;
  return STILES_OK;
}

stiles_status stiles_batch_factorize(stiles_batch* b, const double* const* values, void* stream,
                                     stiles_status* statuses, int64_t* infos) {
  if (!b || !values) return fail(STILES_ERR_INVALID, "null argument");
  const int count = int(b->plans.size());
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaEventRecord(b->ev_in, st));
  CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  for (int i = 0; i < count; ++i) {
    if (!values[i]) return fail(STILES_ERR_INVALID, "null values pointer");
    CUDA_TRY(cudaMemcpyAsync(b->values + b->val_off[i], values[i], size_t(b->plans[i]->nnz) * sizeof(double),
                             cudaMemcpyDefault, b->stream));
  }
  CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
  count_launch(b->lp ? 4 : (b->sliced ? 8 : 5));  // scatter, init, (row scales), persistent kernel, diagonal
                                                  // inverses, folded terms (FP64 tiles)
  CUDA_TRY(cudaEventRecord(b->ev_out, b->stream));
  CUDA_TRY(cudaStreamWaitEvent(st, b->ev_out, 0));
  CUDA_TRY(cudaEventSynchronize(b->ev_out));
  for (stiles_factor* v : b->views) {
    v->stream = st;
    v->sinv_valid = false;
  }
  dev::Ctl c;
  CUDA_TRY(cudaMemcpy(&c, b->ctl, sizeof(c), cudaMemcpyDeviceToHost));
  std::vector<unsigned long long> hinfo(count);
  CUDA_TRY(cudaMemcpy(hinfo.data(), b->infos, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  stiles_status worst = STILES_OK;
  for (int i = 0; i < count; ++i) {
    stiles_status s = STILES_OK;
    if (c.status != 0) s = STILES_ERR_TIMEOUT;
    else if (hinfo[i] != ~0ull) s = STILES_ERR_NOT_SPD;
    if (statuses) statuses[i] = s;
    if (infos) infos[i] = hinfo[i] == ~0ull ? 0 : int64_t(hinfo[i]);
    if (s != STILES_OK && worst == STILES_OK) worst = s;
  }
  if (worst == STILES_ERR_TIMEOUT) return fail(worst, "device wait timed out in the batched launch");
  if (worst == STILES_ERR_NOT_SPD) return fail(worst, "a matrix of the batch is not positive definite");
  return STILES_OK;
}

stiles_status stiles_batch_factor(const stiles_batch* b, int32_t index, stiles_factor** out) {
  if (!b || !out || index < 0 || index >= int32_t(b->views.size())) return fail(STILES_ERR_INVALID, "bad argument");
  *out = b->views[index];
  return STILES_OK;
}

stiles_status stiles_batch_logdet(stiles_batch* b, double* out, void* stream) {
  if (!b || !out) return fail(STILES_ERR_INVALID, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int count = int(b->plans.size());
  batch_logdet_kernel<<<count, 256, 0, st>>>(static_cast<const BatchLogCtx*>(b->dlog), b->logdet_out);
  CUDA_TRY(cudaGetLastError());
  count_launch();
  CUDA_TRY(cudaMemcpyAsync(out, b->logdet_out, count * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return STILES_OK;
}

stiles_status stiles_batch_solve(stiles_batch* b, const double* const* rhs, double* const* x, const int32_t* nrhs,
                                 void* stream, double* relres, int32_t* iters) {
  if (!b || !rhs || !x || !nrhs) return fail(STILES_ERR_INVALID, "null argument");
  const int count = int(b->plans.size());
  std::vector<int> nr(count);
  int64_t max_rows = 0;
  for (int i = 0; i < count; ++i) {
    if (nrhs[i] < 0 || nrhs[i] > dev::SOLVE_MAXR) return fail(STILES_ERR_INVALID, "nrhs must be in [0, 16]");
    if (nrhs[i] > 0 && (!rhs[i] || !x[i])) return fail(STILES_ERR_INVALID, "null right-hand side or solution");
    nr[i] = nrhs[i];
    max_rows = std::max<int64_t>(max_rows, b->plans[i]->nsb * b->plans[i]->B);
  }
  stiles_status s = ensure_batch_solve(b);
  if (s != STILES_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // sources: the batch's full lists, or those of the matrices that take part
  const int nact = int(count - std::count(nr.begin(), nr.end(), 0));
  SweepTickets tk{b->rq_src_f, b->rq_src_b, int(b->src_f.size()), int(b->src_b.size()), b->nfwd, b->nbwd, nact};
  if (nact == 0) {  // nothing to solve
    if (relres) std::fill(relres, relres + count, 0.0);
    if (iters) std::fill(iters, iters + count, 0);
    return STILES_OK;
  }
  if (nact < count) {
    std::vector<int32_t> sf, sb;
    int64_t nf = 0, nb = 0;
    for (int i = 0; i < count; ++i)
      if (nr[i]) {
        sf.insert(sf.end(), b->src_f.begin() + b->src_f_off[i], b->src_f.begin() + b->src_f_off[i + 1]);
        sb.insert(sb.end(), b->src_b.begin() + b->src_b_off[i], b->src_b.begin() + b->src_b_off[i + 1]);
        nf += int64_t(b->plans[i]->fwd.tasks.size());
        nb += int64_t(b->plans[i]->bwd.tasks.size());
      }
    CUDA_TRY(cudaMemcpy(b->rq_call_f, sf.data(), sf.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(b->rq_call_b, sb.data(), sb.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    tk = SweepTickets{b->rq_call_f, b->rq_call_b, int(sf.size()), int(sb.size()), int(nf), int(nb), nact};
  }
  if (b->lp || b->sliced) s = upload_solve_ctx<float>(b, nr, st);
  else s = upload_solve_ctx<double>(b, nr, st);
  if (s != STILES_OK) return s;
  for (int i = 0; i < count; ++i)
    if (nr[i])
      CUDA_TRY(cudaMemcpyAsync(b->vb + b->vec_off[i], rhs[i], size_t(b->plans[i]->n) * nr[i] * sizeof(double),
                               cudaMemcpyDefault, st));
  s = batch_solve_pass(b, tk, st, 0, max_rows);
  if (s != STILES_OK) return s;
  std::vector<double> rel;
  std::vector<int> it(count, 0);
  bool converged = true;
  if (b->lp || b->sliced) {
    // iterative refinement in FP64 per matrix until its residual meets refine_tol
    std::vector<int> active(count);
    int* dactive = nullptr;
    CUDA_TRY(cudaMalloc(&dactive, size_t(count) * sizeof(int)));
    for (;;) {
      s = batch_residual(b, st, max_rows, nr, &rel);
      if (s != STILES_OK) break;
      int any = 0;
      for (int i = 0; i < count; ++i) {
        const stiles_plan* p = b->plans[i];
        active[i] = (rel[i] > p->opts.refine_tol && it[i] < p->opts.max_refine) ? 1 : 0;
        any |= active[i];
      }
      if (!any) break;
      if (cudaMemcpy(dactive, active.data(), size_t(count) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
        s = fail(STILES_ERR_CUDA, "batched refinement upload");
        break;
      }
      s = batch_solve_pass(b, tk, st, 1, max_rows);
      if (s != STILES_OK) break;
      baxpy_active_kernel<<<batch_grid(b, max_rows * dev::SOLVE_MAXR), 256, 0, st>>>(
          static_cast<const BSolveDesc*>(b->ddesc), dactive);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) {
        s = fail(STILES_ERR_CUDA, "batched refinement update");
        break;
      }
      for (int i = 0; i < count; ++i) it[i] += active[i];
    }
    cudaFree(dactive);
    if (s != STILES_OK) return s;
    for (int i = 0; i < count; ++i)
      if (nr[i] && !(rel[i] <= b->plans[i]->opts.refine_tol)) converged = false;
  } else if (relres) {
    s = batch_residual(b, st, max_rows, nr, &rel);
    if (s != STILES_OK) return s;
  }
  for (int i = 0; i < count; ++i)
    if (nr[i])
      CUDA_TRY(cudaMemcpyAsync(x[i], b->vx + b->vec_off[i], size_t(b->plans[i]->n) * nr[i] * sizeof(double),
                               cudaMemcpyDefault, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i) {
    if (relres) relres[i] = rel.empty() ? 0.0 : rel[i];
    if (iters) iters[i] = it[i];
  }
  if (!converged) return fail(STILES_ERR_NOT_CONVERGED, "iterative refinement did not reach refine_tol in the batch");
  return STILES_OK;
}

stiles_status stiles_batch_kernel_window(const stiles_batch* b, void* base_event, double* start_ms, double* end_ms) {
  if (!b || !base_event || !start_ms || !end_ms) return fail(STILES_ERR_INVALID, "null argument");
  float a = 0.f, e = 0.f;
  cudaEvent_t base = static_cast<cudaEvent_t>(base_event);
  CUDA_TRY(cudaEventElapsedTime(&a, base, b->ev_k0));
  CUDA_TRY(cudaEventElapsedTime(&e, base, b->ev_k1));
  *start_ms = a;
  *end_ms = e;
  return STILES_OK;
}

stiles_status stiles_batch_timing(const stiles_batch* b, double* ms_kernel) {
  if (!b || !ms_kernel) return fail(STILES_ERR_INVALID, "null argument");
  float k = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&k, b->ev_k0, b->ev_k1));
  *ms_kernel = k;
  return STILES_OK;
}

void stiles_batch_destroy(stiles_batch* b) { free_batch(b); }

}  // extern "C"

extern "C" {

stiles_status stiles_autotune(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                              const stiles_opts* opts, const int32_t* tiles, int32_t ntiles, const double* values,
                              void* stream, int32_t* best_tile, double* ms) {
  if (!tiles || ntiles < 1 || !values || !best_tile) return fail(STILES_ERR_INVALID, "bad argument");
  stiles_opts o;
  if (opts) o = *opts;
  else stiles::default_opts(&o);
  std::vector<stiles_plan*> plans(ntiles, nullptr);
  std::vector<int64_t> flops(ntiles, -1);
  int64_t fmin = -1;
  for (int i = 0; i < ntiles; ++i) {
    o.tile = tiles[i];
    if (stiles_analyze(n, colptr, rowidx, n_arrow, &o, &plans[i]) != STILES_OK || !plans[i]->executable) continue;
    stiles_plan_info inf;
    stiles_plan_get_info(plans[i], &inf);
    flops[i] = inf.flops_total;
    if (fmin < 0 || flops[i] < fmin) fmin = flops[i];
  }
  double best = -1.0;
  stiles_status result = STILES_ERR_INVALID;
  for (int i = 0; i < ntiles; ++i) {
    if (ms) ms[i] = -1.0;
    // a tile whose padding multiplies the work beyond 4x cannot win on parallelism alone
    if (!plans[i] || flops[i] < 0 || flops[i] > 4 * fmin) continue;
    stiles_factor* f = nullptr;
    stiles_status s = stiles_factorize(plans[i], values, stream, &f, nullptr);
    double t = 1e300;
    for (int rep = 0; rep < 2 && s == STILES_OK; ++rep) {
      s = stiles_factorize(plans[i], values, stream, &f, nullptr);
      double call = 0.0;
      if (s == STILES_OK && stiles_factor_timing(f, &call, nullptr) == STILES_OK) t = std::min(t, call);
    }
    stiles_factor_destroy(f);
    if (s != STILES_OK) {
      result = s;
      continue;
    }
    if (ms) ms[i] = t;
    if (best < 0 || t < best) {
      best = t;
      *best_tile = tiles[i];
      result = STILES_OK;
    }
  }
  for (stiles_plan* p : plans) stiles_plan_destroy(p);
  if (result != STILES_OK) return fail(result, "no candidate tile size could be factorized");
  return STILES_OK;
}

}  // extern "C"
