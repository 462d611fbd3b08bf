// Internal plan and factor structures shared by the host analysis (analyze.cpp)
// and the CUDA side (capi.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/stiles.h"

namespace stiles {

// One unit of device work of the factorization (a ticket of the persistent
// scheduler).  Tickets are issued in a topological order: every tile a task
// waits for is produced by a task with a smaller ticket.
enum TaskType : int32_t {
  TASK_DIAG = 0,     // L_kk = chol(A_kk - sum L_kn L_kn^T - sum partials)           (SYRK + POTRF)
  TASK_OFF = 1,      // L_mk = (A_mk - sum L_mn L_kn^T - sum partials) L_kk^{-T}       (GEMM + TRSM)
  TASK_PARTIAL = 2,  // P = sum over a chunk of L_an L_bn^T   (a tree leaf, Algorithm 3)
  TASK_COMBINE = 3,  // P = sum of partial tiles             (a tree node, GEADD)
  TASK_CHAIN = 4,    // OFF(k, k-1) then DIAG(k) in one CTA: the diagonal chain step
};

// For TASK_CHAIN the first output is the OFF tile (k, k-1) (diag = L_{k-1,k-1},
// col = k-1) and the second the diagonal tile (k, k) (col2 = k); the SYRK term
// with L_{k,k-1} is applied from shared memory.  The terms of both tiles share
// one list, ordered by when their producers run; bit 30 of a pair's first index
// (or of a partial index) marks the terms of the diagonal tile.
struct DevTask {
  int32_t type;
  int32_t out;   // sub-tile index (DIAG/OFF/CHAIN) or scratch tile index (PARTIAL/COMBINE)
  int32_t diag;  // sub-tile index of L_kk (OFF, CHAIN), else -1
  int32_t col;   // sub-column of `out` (slot of the 1/L_jj vector of its diagonal)
  int32_t pb, pe;  // update pairs [pb, pe) into `out`
  int32_t qb, qe;  // partial tiles [qb, qe) (scratch indices) into `out`
  int32_t out2;    // CHAIN: the diagonal sub-tile, else -1
  int32_t col2;    // CHAIN: its sub-column
  int32_t pb2, pe2, qb2, qe2;  // unused (CHAIN terms for `out2` are tagged inside [pb, pe) / [qb, qe))
  int32_t trow, tcol;  // block row and block column of the tile the first accumulator updates
                       // (the output, or a tree partial's owner tile; a CHAIN's second target is (col2, col2))
};
static_assert(sizeof(DevTask) == 64, "DevTask layout");

// Solve task: one B x nrhs block of y (forward) or x (backward).
enum SolveType : int32_t { SOLVE_FINAL = 0, SOLVE_PARTIAL = 2, SOLVE_COMBINE = 3 };
struct SolveTask {
  int32_t type;
  int32_t out;   // block index (FINAL) or scratch block index (PARTIAL/COMBINE)
  int32_t diag;  // sub-tile index of L_kk (FINAL)
  int32_t pad0;
  int32_t pb, pe;  // pairs (L sub-tile, block index)
  int32_t qb, qe;  // scratch blocks
};
static_assert(sizeof(SolveTask) == 32, "SolveTask layout");

struct TaskGraph {
  std::vector<DevTask> tasks;
  std::vector<int32_t> pairs;  // 2 per pair
  std::vector<int32_t> parts;
  int64_t nscratch = 0;
};

struct SolveGraph {
  std::vector<SolveTask> tasks;
  std::vector<int32_t> pairs;
  std::vector<int32_t> parts;
  int64_t nscratch = 0;
};

// Selected inverse (Sigma = (P A P^T)^{-1} on the filled sub-tile map), reverse
// column order: per task 4 int32 (output sub-tile, its sub-column if it is a
// diagonal sub-tile else -1, first pair, end pair); per pair 2 int32 (Sigma
// sub-tile with bit 30 set when it is read transposed, U sub-tile); per
// off-diagonal sub-tile 2 int32 (sub-tile, sub-column) for U = L_jk L_kk^{-1}.
struct SelinvGraph {
  std::vector<int32_t> tasks;  // 8 per task: output, column of a diagonal task or -1, products,
                               // loads, X products (each a [begin, end) range)
  std::vector<int32_t> pairs;  // 2 per product: Sigma sub-tile (bit 30: transposed), U sub-tile
  std::vector<int32_t> loads;  // 3 per finished term: flag sub-tile, value it waits for, term
                               // sub-tile (bit 30: in W, else in X)
  std::vector<int32_t> posts;  // 1 per X product: sub-tile (m, c) of U and of X
  std::vector<int32_t> ulist;  // 2 per U product: sub-tile, sub-column
};

struct DevPlan;  // device copies, defined in capi.cu

}  // namespace stiles

struct stiles_plan {
  stiles_opts opts{};
  int64_t n = 0, n_arrow = 0, nnz = 0;
  int32_t T = 0, B = 0, R = 0;
  int32_t ordering_used = 0;
  std::vector<int64_t> colptr;   // copy of the input pattern (for the residual SpMV)
  std::vector<int32_t> rowidx;
  std::vector<int64_t> rptr;     // CSR index of its strict lower part: row i holds columns j < i
  std::vector<int32_t> rcol;
  std::vector<int64_t> rval;     //   and the CSC position of each entry
  std::vector<int64_t> perm;     // perm[new] = old
  std::vector<int64_t> iperm;    // iperm[old] = new
  // T-level tile map (tile-CSC, diagonal first)
  int64_t nt = 0, nnzt = 0;
  std::vector<int64_t> tcolptr;
  std::vector<int32_t> trowidx;
  int64_t flops_potrf = 0, flops_syrk = 0, flops_gemm = 0, flops_trsm = 0;
  // B-level executor (only when T % B == 0 and B in {16, 32, 64})
  bool executable = false;
  int64_t nsb = 0;               // sub-rows/columns holding rows < n
  int64_t nsub = 0;              // stored sub-tiles = nnzt * R * R
  std::vector<int32_t> diag_sub; // [nsb] sub-tile index of each diagonal sub-tile
  std::vector<int64_t> scatter;  // [nnz] element offset of each input entry in the tile buffer
  std::vector<int64_t> pad;      // element offsets of padding diagonal entries (rows >= n)
  stiles::TaskGraph graph;
  std::vector<int32_t> chain_order;  // factor tasks of the diagonal chain (DIAG, CHAIN), ticket order
  std::vector<int32_t> bulk_order;   // every other factor task, ticket order
  bool split_queues = false;         // thin DAG: run the chain on reserved SMs (little work per chain step)
  stiles::SolveGraph fwd, bwd;
  stiles::SelinvGraph selinv;        // built on first use (stiles_marginal_variances)
  bool selinv_built = false;
  // factorization with the forward sweep folded in (built on first use): the
  // factor tasks plus one OFF-type task per forward block (output nsub + k, the
  // block's right-hand sides transposed as a tile) and the forward tree
  // partials (scratch after the factor's), each right after its inputs' producers
  stiles::TaskGraph fused;
  std::vector<int32_t> fused_chain, fused_bulk;
  bool fused_built = false;
  stiles::DevPlan* dev = nullptr;
};

namespace stiles {
// analyze.cpp
stiles_status build_plan(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t n_arrow,
                         const stiles_opts& opts, stiles_plan* p, std::string* err);
stiles_status build_selinv(stiles_plan* p, std::string* err);
stiles_status build_fused(stiles_plan* p, std::string* err);
void default_opts(stiles_opts* o);
}  // namespace stiles
