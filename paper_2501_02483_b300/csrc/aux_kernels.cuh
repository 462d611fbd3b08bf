// Bandwidth-bound helper kernels around the factorization and the solves:
// CTSF scatter (Section III.B), log-determinant reduction, permutation of
// right-hand sides, FP64 residual SpMV, tile export and the FP64 peak probe.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace stiles {
namespace dev {

// tiles[map[e]] = values[e]  (tiles zeroed beforehand; each target written once)
__global__ void scatter_kernel(double* __restrict__ tiles, const double* __restrict__ values,
                               const int64_t* __restrict__ map, int64_t nnz) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz; e += stride)
    tiles[__ldg(map + e)] = __ldg(values + e);
}

// Mixed-precision factor: the values are rounded to FP32 on the way into the tiles.
__global__ void scatter_f32_kernel(float* __restrict__ tiles, const double* __restrict__ values,
                                   const int64_t* __restrict__ map, int64_t nnz) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz; e += stride)
    tiles[__ldg(map + e)] = float(__ldg(values + e));
}

template <typename T>
__global__ void set_ones_kernel(T* __restrict__ tiles, const int64_t* __restrict__ offs, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) tiles[offs[i]] = T(1);
}

// x += d (n x nr blocks, leading dimensions ldx / n)
__global__ void axpy_cols_kernel(double* __restrict__ x, const double* __restrict__ d, int64_t n, int64_t ldx, int nr) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * nr; e += stride) {
    const int64_t r = e / n, i = e % n;
    x[i + r * ldx] += d[i + r * n];
  }
}

// r = b - y (y: n x nr, ld n; b: ld ldb; r: ld n)
__global__ void sub_cols_kernel(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ y,
                                int64_t n, int64_t ldb, int nr) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n * nr; e += stride) {
    const int64_t c = e / n, i = e % n;
    r[i + c * n] = b[i + c * ldb] - y[i + c * n];
  }
}

__global__ void init_ctl_kernel(Ctl* ctl, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    ctl[i].ticket = 0;
    ctl[i].status = 0;
    ctl[i].abort = 0;
    ctl[i].pad = 0;
    ctl[i].info = ~0ull;
    ctl[i].where = -1;
  }
}

// log det = 2 sum_i log L_ii = sum_i log(L_ii^2).  Pass 1: block b sums a fixed
// contiguous range of rows (fixed order inside the block); pass 2 adds the
// block sums in index order.  The result does not depend on scheduling.
constexpr int LOGDET_BLOCKS = 148;
constexpr int LOGDET_THREADS = 256;

__global__ void logdet_pass1(const double* __restrict__ tiles, const int32_t* __restrict__ diag_sub, int64_t n,
                             int B, double* __restrict__ partial) {
  __shared__ double red[LOGDET_THREADS];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = int64_t(blockIdx.x) * per;
  const int64_t hi = min(n, lo + per);
  double s = 0.0;
  for (int64_t g = lo + threadIdx.x; g < hi; g += blockDim.x) {
    const int64_t k = g / B, j = g % B;
    const double l = tiles[int64_t(diag_sub[k]) * B * B + j * B + j];
    s += 2.0 * log(l);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// The same reduction over a vector of the factor's diagonal entries (mixed-precision factors).
__global__ void logdet_vec_pass1(const double* __restrict__ ldiag, int64_t n, double* __restrict__ partial) {
  __shared__ double red[LOGDET_THREADS];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = int64_t(blockIdx.x) * per;
  const int64_t hi = min(n, lo + per);
  double s = 0.0;
  for (int64_t g = lo + threadIdx.x; g < hi; g += blockDim.x) s += 2.0 * log(ldiag[g]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void logdet_pass2(const double* __restrict__ partial, int np, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += partial[i];
    *out = s;
  }
}

// Y[block k][r][i] = b[perm[k*B+i] + (r0 + r) * ld]   (zero past n; Y in the sweep's type)
template <typename TY>
__global__ void permute_in_kernel(TY* __restrict__ Y, const double* __restrict__ b, const int64_t* __restrict__ perm,
                                  int64_t n, int64_t ld, int r0, int nr, int B, int64_t nsb) {
  const int64_t total = nsb * B * nr;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t k = e / (int64_t(B) * nr);
    const int64_t rem = e % (int64_t(B) * nr);
    const int r = int(rem / B), i = int(rem % B);
    const int64_t g = k * B + i;
    Y[e] = (g < n) ? TY(b[perm[g] + (r0 + r) * ld]) : TY(0);
  }
}

template <typename TY>
__global__ void permute_out_kernel(double* __restrict__ x, const TY* __restrict__ Y, const int64_t* __restrict__ perm,
                                   int64_t n, int64_t ld, int r0, int nr, int B) {
  const int64_t total = n * nr;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int r = int(e / n);
    const int64_t g = e % n;
    const int64_t k = g / B, i = g % B;
    x[perm[g] + (r0 + r) * ld] = double(Y[(k * nr + r) * B + i]);
  }
}

// y = A x for the symmetric A stored as its lower CSC (diagonal included):
// column j contributes a_jj x_j and sum_{i>j} a_ij x_i to y_j (gather) and
// a_ij x_j to y_i (scatter, atomic).  r = b - y, then per column the sums of
// squares of r and b.
__global__ void spmv_lower_kernel(double* __restrict__ y, const double* __restrict__ x, const int64_t* __restrict__ colptr,
                                  const int32_t* __restrict__ rowidx, const double* __restrict__ val, int64_t n,
                                  int64_t ldx, int nr) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < n * nr; w += stride) {
    const int r = int(w / n);
    const int64_t j = w % n;
    const double* xr = x + r * ldx;
    double* yr = y + r * n;
    const double xj = xr[j];
    double s = 0.0;
    for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
      const int64_t i = rowidx[e];
      const double v = val[e];
      s = fma(v, xr[i], s);
      if (i != j) atomicAdd(yr + i, v * xj);
    }
    atomicAdd(yr + j, s);
  }
}

__global__ void residual_norms_kernel(const double* __restrict__ y, const double* __restrict__ b, int64_t n, int64_t ldb,
                                      int nr, double* __restrict__ sums /* 2 per column */) {
  __shared__ double rr[256], bb[256];
  const int r = blockIdx.y;
  double sr = 0.0, sb = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double bv = b[i + r * ldb];
    const double d = bv - y[i + r * n];
    sr = fma(d, d, sr);
    sb = fma(bv, bv, sb);
  }
  rr[threadIdx.x] = sr;
  bb[threadIdx.x] = sb;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      bb[threadIdx.x] += bb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(sums + 2 * r, rr[0]);
    atomicAdd(sums + 2 * r + 1, bb[0]);
  }
}

// Export T x T column-major tiles from the sub-tile layout (R = T / B).
template <typename TF>
__global__ void export_tiles_kernel(double* __restrict__ out, const TF* __restrict__ tiles, int64_t nnzt, int T, int B) {
  const int64_t TT = int64_t(T) * T;
  const int R = T / B;
  const int64_t total = nnzt * TT;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t t = e / TT;
    const int64_t w = e % TT;
    const int c = int(w / T), r = int(w % T);
    const int64_t s = t * R * R + int64_t(c / B) * R + (r / B);
    out[e] = double(tiles[s * B * B + int64_t(c % B) * B + (r % B)]);
  }
}

// FP64 throughput probe: independent FMA chains per thread.
__global__ void fp64_probe_kernel(double* out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  if (s == 1.2345678e300) out[0] = s;
}

}  // namespace dev
}  // namespace stiles
