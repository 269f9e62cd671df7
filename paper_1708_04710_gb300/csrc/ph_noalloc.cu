// beta (Definition 4) of one dimension's boundary columns without allocating device memory.
//
// Some callers cannot allocate: code running inside another framework's memory pool or arena
// (where a stray cudaMalloc would bypass its accounting or fragment a nearly full device),
// real-time or embedded callers that forbid allocation after start-up, and callers holding no
// library context at all. For them this entry point keeps its only scratch -- left(i), the
// first column holding each row (Definition 3) -- in a fixed file-scope device array, so the
// caller passes just its input and output buffers.
#include "ph_internal.cuh"

namespace {

constexpr int64_t kStaticRows = int64_t(1) << 22;  // 4,194,304 rows: 16 MiB of int32

// Resident on every GPU that loads the library, until the process exits.
__device__ __align__(256) int32_t g_left_scratch[kStaticRows];
__device__ __align__(256) unsigned long long g_bad_rows;


__global__ void k_fill_left(int32_t* left, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    left[i] = INT32_MAX;
}

__global__ void k_left_static(const int32_t* __restrict__ rows, int64_t n_cols, int k,
                              int64_t n_rows, int32_t* left, int32_t* beta,
                              unsigned long long* bad) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_cols;
       j += (int64_t)gridDim.x * blockDim.x) {
    beta[j] = -1;
    for (int q = 0; q < k; q++) {
      int32_t r = rows[j * k + q];
      if (r < 0 || r >= n_rows) {  // out-of-range rows are skipped and reported
        atomicAdd(bad, 1ull);
        continue;
      }
      atomicMin(&left[r], (int32_t)j);
    }
  }
}

__global__ void k_beta_static(const int32_t* __restrict__ left, int64_t n_rows, int32_t* beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = left[i];
    if (j != INT32_MAX) atomicMax(&beta[j], (int32_t)i);
  }
}

// The device addresses of the two static arrays in the current context, looked up on every
// call (a lookup allocates nothing): an address kept from an earlier call would be stale once
// the module is loaded again, after a device reset or in another context on the device. In host
// code the symbol names are host stand-ins, never device addresses, so kernels get these.
int static_arrays(int* dev_out, int32_t** left, unsigned long long** bad) {
  int dev = -1;
  void* p = nullptr;
  void* q = nullptr;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 ||
      cudaGetSymbolAddress(&p, g_left_scratch) != cudaSuccess ||
      cudaGetSymbolAddress(&q, g_bad_rows) != cudaSuccess || !p || !q) {
    cudaGetLastError();
    return PH_ERR_CUDA;
  }
  *dev_out = dev;
  *left = static_cast<int32_t*>(p);
  *bad = static_cast<unsigned long long*>(q);
  return PH_OK;
}

}  // namespace

extern "C" int ph_beta_static(const int32_t* rows, int64_t n_cols, int32_t rows_per_col,
                              int64_t n_rows, int32_t* beta, void* stream) {
  if (n_cols < 0 || n_rows < 0 || rows_per_col < 1 || rows_per_col > 64) return PH_ERR_INVALID;
  if (n_rows > kStaticRows || n_cols >= INT32_MAX) return PH_ERR_CAPACITY;
  if (n_cols == 0) return PH_OK;
  if (!rows || !beta) return PH_ERR_INVALID;
  int dev = 0;
  int32_t* left = nullptr;
  unsigned long long* bad = nullptr;
  int rc = static_arrays(&dev, &left, &bad);
  if (rc != PH_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256;
  auto grid = [&](int64_t n) {
    int64_t g = (n + threads - 1) / threads, cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
  };
  // the array keeps the previous call's contents: reset what this call reads
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    k_fill_left<<<grid(n_rows), threads, 0, st>>>(left, n_rows);
    k_left_static<<<grid(n_cols), threads, 0, st>>>(rows, n_cols, rows_per_col, n_rows, left,
                                                    beta, bad);
    k_beta_static<<<grid(n_rows), threads, 0, st>>>(left, n_rows, beta);
    e = cudaGetLastError();
  }
  unsigned long long h_bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PH_ERR_CUDA;
  }
  return h_bad ? PH_ERR_INVALID : PH_OK;
}
