// Device scans and the LSD radix sort used to order simplices by squared diameter.
//
// Both are tile based: a tile is kThreads * kItems consecutive elements handled by one block.
// (1) per-tile reduction, (2) one block scans the tile aggregates, (3) per-tile scan with the
// tile's prefix. No kernel waits on another block, so nothing here can spin.
#include "ph_internal.cuh"

namespace ph {

constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

// ---------------------------------------------------------------------------------------------
// exclusive scan of int64
// ---------------------------------------------------------------------------------------------
__global__ void k_tile_sum_i64(const int64_t* __restrict__ in, int64_t n, int64_t* tile_sums) {
  __shared__ int64_t sh[kWarps + 1];
  int64_t base = (int64_t)blockIdx.x * kTile;
  int64_t s = 0;
  for (int it = 0; it < kItems; it++) {
    int64_t i = base + it * kThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int64_t total;
  block_excl_sum<int64_t>(s, sh, total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// single block: exclusive scan of the tile sums in place; writes the grand total
__global__ void k_scan_tiles_i64(int64_t* sums, int64_t ntiles, int64_t* total_out) {
  __shared__ int64_t sh[kWarps + 1];
  int64_t carry = 0;
  for (int64_t base = 0; base < ntiles; base += kThreads) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < ntiles ? sums[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_sum<int64_t>(v, sh, tot);
    if (i < ntiles) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_tile_scan_i64(const int64_t* __restrict__ in, int64_t* out, int64_t n,
                                const int64_t* __restrict__ tile_prefix) {
  __shared__ int64_t sh[kWarps + 1];
  int64_t base = (int64_t)blockIdx.x * kTile;
  int64_t carry = tile_prefix[blockIdx.x];
  for (int it = 0; it < kItems; it++) {
    int64_t i = base + it * kThreads + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_sum<int64_t>(v, sh, tot);
    if (i < n) out[i] = carry + ex;
    carry += tot;
  }
}

void excl_scan_i64(ph_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev) {
  int64_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles == 0) {
    if (total_dev) PH_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int64_t), ctx->stream));
    return;
  }
  int64_t* sums = alloc_n<int64_t>(ctx, ntiles);
  k_tile_sum_i64<<<(unsigned)ntiles, kThreads, 0, ctx->stream>>>(in, n, sums);
  PH_CHECK_LAUNCH();
  k_scan_tiles_i64<<<1, kThreads, 0, ctx->stream>>>(sums, ntiles, total_dev);
  PH_CHECK_LAUNCH();
  k_tile_scan_i64<<<(unsigned)ntiles, kThreads, 0, ctx->stream>>>(in, out, n, sums);
  PH_CHECK_LAUNCH();
  ctx->dfree(sums);
}

// ---------------------------------------------------------------------------------------------
// LSD radix sort of (uint64 key, uint64 value) pairs by key bits [lo_bit, hi_bit), stable.
// 8-bit digits. Histograms are digit-major ([256][ntiles]) so that one exclusive scan over
// them gives every tile's output offset per digit.
// ---------------------------------------------------------------------------------------------
__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                             int64_t ntiles, int64_t* hist) {
  __shared__ unsigned cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int it = 0; it < kItems; it++) {
    int64_t i = base + it * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const uint64_t* __restrict__ vin,
                                uint64_t* __restrict__ kout, uint64_t* __restrict__ vout,
                                int64_t n, int shift, int64_t ntiles,
                                const int64_t* __restrict__ offs) {
  __shared__ int64_t base[256];
  __shared__ unsigned wcnt[kWarps][256];
  __shared__ unsigned tot[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; w++) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kTile;
  for (int it = 0; it < kItems; it++) {
    int64_t i = tile0 + it * kThreads + tid;
    bool valid = i < n;
    uint64_t k = valid ? kin[i] : 0, v = valid ? vin[i] : 0;
    unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; w++) {
      unsigned c = wcnt[w][tid];
      wcnt[w][tid] = run;
      run += c;
    }
    tot[tid] = run;
    __syncthreads();
    if (valid) {
      int64_t pos = base[d] + wcnt[warp][d] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    base[tid] += tot[tid];
#pragma unroll
    for (int w = 0; w < kWarps; w++) wcnt[w][tid] = 0;
    __syncthreads();
  }
}

void radix_sort_u64(ph_ctx* ctx, uint64_t* keys, uint64_t* vals, int64_t n, int lo_bit,
                    int hi_bit, uint64_t* tmp_keys, uint64_t* tmp_vals) {
  if (n <= 1 || hi_bit <= lo_bit) return;
  int64_t ntiles = (n + kTile - 1) / kTile;
  int64_t nh = 256 * ntiles;
  int64_t* hist = alloc_n<int64_t>(ctx, nh);
  int passes = (hi_bit - lo_bit + 7) / 8;
  uint64_t *ka = keys, *va = vals, *kb = tmp_keys, *vb = tmp_vals;
  for (int p = 0; p < passes; p++) {
    int shift = lo_bit + 8 * p;
    k_radix_hist<<<(unsigned)ntiles, kThreads, 0, ctx->stream>>>(ka, n, shift, ntiles, hist);
    PH_CHECK_LAUNCH();
    excl_scan_i64(ctx, hist, hist, nh, nullptr);
    k_radix_scatter<<<(unsigned)ntiles, kThreads, 0, ctx->stream>>>(ka, va, kb, vb, n, shift,
                                                                   ntiles, hist);
    PH_CHECK_LAUNCH();
    uint64_t* t = ka;
    ka = kb;
    kb = t;
    t = va;
    va = vb;
    vb = t;
  }
  if (ka != keys) {
    PH_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                            ctx->stream));
    PH_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  }
  ctx->dfree(hist);
}

}  // namespace ph
