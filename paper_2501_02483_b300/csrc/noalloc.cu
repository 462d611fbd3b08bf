// Log-determinant from caller-owned factor tiles, without any device allocation.
//
// For callers that cannot allocate device memory themselves or through this
// library: a process that hands its whole HBM budget to its own memory pool or
// arena at start-up, or code that runs where a cudaMalloc would block the
// device or is not allowed.  The caller passes the factor tiles, the tile
// column pointers and the output; the only scratch is the fixed-size array
// below, which lives for as long as the library is loaded.
//
// The computation is the same fixed-order, two-pass reduction as
// stiles_logdet, with the per-tile-column partial sums kept in that array.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/stiles.h"

namespace {

// Upper bound on tile columns (ceil(n / T)) a call may cover: 65,536 partial
// sums, 512 KB per device.
constexpr int64_t kNoallocMaxTileColumns = 65536;

static __device__ __align__(256) double g_logdet_columns[kNoallocMaxTileColumns];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Pass 1: one partial per tile column k, 2 * sum_j log L_jj over the rows of
// its diagonal tile (the first tile of column k in tile-CSC order).
__global__ void noalloc_logdet_columns(double* __restrict__ part, const double* __restrict__ tiles,
                                       const int64_t* __restrict__ tcolptr, int64_t n, int T, int64_t nt) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t TT = int64_t(T) * T;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < nt; k += stride) {
    const double* d = tiles + tcolptr[k] * TT;
    const int64_t rows = (n - k * T) < T ? (n - k * T) : T;
    double s = 0.0;
    for (int64_t j = 0; j < rows; ++j) s += 2.0 * log(d[j * T + j]);
    part[k] = s;
  }
}

// Pass 2: one block adds the partials in a fixed order.
__global__ void noalloc_logdet_sum(const double* __restrict__ part, int64_t nt, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < nt; k += blockDim.x) s += part[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (int(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

extern "C" stiles_status stiles_logdet_tiles_noalloc(const double* tiles, const int64_t* tcolptr, int64_t n,
                                                      int32_t tile, double* out, void* stream) {
  if (!tiles || !tcolptr || !out || n < 1 || tile < 1) return STILES_ERR_INVALID;
  const int64_t nt = (n + tile - 1) / tile;
  if (nt > kNoallocMaxTileColumns) return STILES_ERR_INVALID;  // ceil(n / tile) above 65,536
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return STILES_ERR_CUDA;
  void* scratch = nullptr;
  {
    // First call on each device: look up the device address of the static array
    // with that device current (the host-side symbol is not a device address).
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_logdet_columns) != cudaSuccess || !addr) {
        cudaGetLastError();
        return STILES_ERR_CUDA;
      }
      g_scratch_addr[device] = addr;
    }
    scratch = g_scratch_addr[device];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int threads = 256;
  int blocks = int((nt + threads - 1) / threads);
  if (blocks > 1024) blocks = 1024;
  noalloc_logdet_columns<<<blocks, threads, 0, st>>>(static_cast<double*>(scratch), tiles, tcolptr, n, tile, nt);
  noalloc_logdet_sum<<<1, 256, 0, st>>>(static_cast<const double*>(scratch), nt, out);
  if (cudaGetLastError() != cudaSuccess) return STILES_ERR_CUDA;
  return STILES_OK;
}
