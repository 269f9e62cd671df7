// Internal definitions of the GB300 persistent-homology library (not part of the ABI).
//
// Simplex identifiers ("ids") are dim-major over all clouds: every simplex of dimension d
// lies in [dimoff[d], dimoff[d+1]); inside a dimension, cloud c owns the contiguous segment
// s = d * n_clouds + c, and inside a segment simplices follow the filtration order of the
// cloud. Rows of a column of dimension d are ids of dimension d-1 of the same cloud, so one
// id space carries every table of the reduction (low, beta, owner, left-most table).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ph_gb300.h"

namespace ph {

constexpr int kMaxDim = 8;  // largest simplex dimension of a loaded complex
constexpr int kMaxVrDim = 5;   // largest simplex dimension of a VR build (6 vertices)
constexpr int kVrSlots = kMaxVrDim + 1;
// packed vertex tuples: a 16-bit cloud above 48 bits of vertex slots, 4 x 12 bits when the
// build stops at dimension 3, 6 x 8 bits above (an all-ones slot marks no vertex)
constexpr int kVertBits = 12;
constexpr int kVertBitsHigh = 8;
constexpr int kMaxCloudPoints = 1 << kVertBits;

__host__ __device__ __forceinline__ int vert_bits_for(int max_dim) {
  return max_dim <= 3 ? kVertBits : kVertBitsHigh;
}
__host__ __device__ __forceinline__ int packed_vert_at(uint64_t p, int i, int vbits) {
  return (int)((p >> (48 - vbits * (i + 1))) & ((1u << vbits) - 1u));
}
constexpr int kMaxClouds = 65535;

// column flags
constexpr uint8_t F_PROVEN = 1;  // pivot: low(j) = lowstar(j) > 0 is known
constexpr uint8_t F_FINAL = 2;   // column is zero and positive for good
constexpr uint8_t F_NEWPIV = 4;  // proven in the current pass

// Per-column metadata of the reduction, one 16-byte record per id, so that reading a column
// (its own or a source's) costs one sector rather than one per field.
struct __align__(16) ColMeta {
  int32_t* ptr;     // its rows (ascending): boundary matrix, arena or pivot store
  int32_t len;      // number of rows
  uint8_t flags;    // F_PROVEN | F_FINAL | F_NEWPIV
  uint8_t cleared;  // zeroed by clearing (Lemma 1)
  uint8_t low_seen; // the id was the low of some column at the start of some pass
  uint8_t spare;
};
static_assert(sizeof(ColMeta) == 16, "one 16-byte record per column");

__device__ __forceinline__ ColMeta load_meta(const ColMeta* p) {
  const int4 v = *reinterpret_cast<const int4*>(p);
  ColMeta m;
  m.ptr = reinterpret_cast<int32_t*>((unsigned long long)(unsigned)v.x |
                                     ((unsigned long long)(unsigned)v.y << 32));
  m.len = v.z;
  m.flags = (uint8_t)(v.w & 0xff);
  m.cleared = (uint8_t)((v.w >> 8) & 0xff);
  m.low_seen = (uint8_t)((v.w >> 16) & 0xff);
  m.spare = 0;
  return m;
}

// Membership of id x in the essential estimate E^l of Eq. (essential_iteration): E^0 = [m] and
// E^{l+1} = (E^l \ Paired^l) \ low^l([m]). Paired only grows, so x is in E^l iff it is not
// paired now (proven pivot, beta_x >= 0 by Thm 5, or the low of a proven pivot) and was never
// the low of a column at the start of a pass.
__device__ __forceinline__ bool in_essential_estimate(const ColMeta& mx, int32_t beta_x,
                                                      int32_t owner_x) {
  return !(mx.flags & F_PROVEN) && beta_x < 0 && owner_x < 0 && !mx.low_seen;
}

// Every buffer that holds columns (boundary matrix, arenas, pivot store) is allocated with this
// many words past its capacity: the additions kernel stages a column by 16-byte copies that
// round its start down and its end up to 16 bytes, so they may read up to 4 words past the last
// column, and those words must lie inside the allocation.
constexpr int64_t kColSlack = 8;

struct ColStore {  // a device buffer that holds column storage (int32 rows)
  int32_t* p = nullptr;
  int64_t cap = 0;  // words
};

struct ReduceState {
  int32_t* act = nullptr;      // active list buffers (which one is current: device state)
  int32_t* act2 = nullptr;
  int32_t* alen = nullptr;     // per slot: the column's stored length (both lists)
  int32_t* alen2 = nullptr;
  int64_t act_cap = 0;
  void* meta = nullptr;        // per id: ColMeta (rows, length, flags, clearing mark)
  int32_t** nxt_ptr = nullptr; // per active slot: new location
  int32_t* nxt_len = nullptr;
  int32_t* owner = nullptr;    // per row id: proven pivot with that low, -1
  int32_t* tab = nullptr;      // two tables per row id: left-most column with that low (pass p: p & 1)
  int32_t* first_unp = nullptr;// per segment: first row id not known to be paired
  void* tiles = nullptr;       // scan scratch
  void* look = nullptr;        // look-back states of the survivor scan
  void* dlist = nullptr;       // deferred column updates
  void* src_e = nullptr;       // per active slot: source candidate of Phase II
  uint32_t* unp_bits = nullptr;  // Corollary 10 predictions: unpaired-row bitmap
  int32_t* unp_words = nullptr;  // and its per-word prefix counts
  int32_t* pred = nullptr;       // per id: predicted lowstar, -1
  // Phase II limited to p neighbour sets (phase2_sets > 0), per row of the boundary:
  int32_t* set_n = nullptr;      // targets of the row's set whose addition this pass may do
  int32_t* set_neg = nullptr;    // those of them known to be negative (beta >= 0)
  uint8_t* set_on = nullptr;     // the set is among the p acted on
  uint64_t* set_key = nullptr;   // [4][rows] priority sort keys, rows, and their scratch
  int64_t tiles_bytes = 0;
  void* dstate = nullptr;      // per-pass state in device memory
  void* hstate = nullptr;      // pinned host mirror of it
  int64_t* pass_stats = nullptr;  // device [stats_rows][PH_PS_N]
  int32_t stats_rows = 0;
  ColStore arena[2];           // pass p writes its survivors into arena[p & 1]
  std::vector<ColStore> pivots;  // chunks holding proven columns
  // the pass loop: one pass as the body of a conditional while node, per variant of the
  // additions kernel (+1 bit-packed columns, +2 one chunk per warp, +4 jobs merged by lanes;
  // 8, 9: 8-slot warp chunks with merge pieces, without and with bit-packed columns)
  static constexpr int kAddVariants = 10;
  cudaGraph_t graph[kAddVariants] = {};
  cudaGraphExec_t graph_exec[kAddVariants] = {};
  int32_t passes = 0;
  bool init = false;
  bool done = false;
  int status = PH_OK;
  std::vector<int64_t> h_stats;  // host copy of per-pass counters
  std::vector<cudaEvent_t> ev;   // start/stop pairs around the addition kernel
  int64_t add_launches = 0;
  double ms_add = 0;
  std::vector<float> add_ms;     // per timed launch
};

}  // namespace ph

struct ph_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  ph_opts opts{};
  ph_allocator alloc{};
  bool has_alloc = false;
  std::string err;
  int64_t launches = 0;  // kernels launched by this context

  struct Block {
    void* p;
    size_t bytes;
  };
  std::vector<Block> blocks;  // every device allocation of the context

  // filtration
  bool built = false;
  bool reduced = false;
  bool is_vr = false;  // built from points (vertex tuples known)
  int32_t D = 0;          // coordinates per point of a VR build (0: none)
  int64_t n_points = 0;   // points of a VR build: coordinate arrays hold n_points * D values
  int32_t n_clouds = 0;
  int32_t max_dim = 0;
  int64_t m = 0;
  std::vector<int64_t> pt_off;     // host [n_clouds + 1]
  std::vector<int64_t> seg_start;  // host [nseg + 1], nseg = (max_dim + 1) * n_clouds
  int64_t dimoff[ph::kMaxDim + 2] = {0};
  int64_t* d_seg_start = nullptr;
  int32_t* seg = nullptr;     // per id: segment
  int32_t* low = nullptr;     // per id: low, as an id (-1 none)
  int32_t* beta = nullptr;    // per id: beta, as an id (-1 none)
  int32_t* key = nullptr;     // per id: dense squared-diameter rank (-1: vertex/loaded)
  int64_t* gidx = nullptr;    // per id: filtration index within its cloud
  uint64_t* verts = nullptr;  // per id: packed (cloud, vertex slots of vbits bits)
  int vbits = ph::kVertBits;  // bits per packed vertex of this build
  int64_t* d2tab = nullptr;   // dense rank -> squared diameter
  int64_t n_d2 = 0;
  int32_t* rows0 = nullptr;   // initial column storage (boundary matrix, CSC by id)
  // loaded matrices: per id, the offset of its column in rows0 ([m + 1]); VR builds store
  // d + 1 rows per column at a fixed stride and leave this null
  int64_t* col_off = nullptr;
  int64_t nnz = 0;

  ph::ReduceState rs;

  // extraction cache
  bool extracted = false;
  std::vector<int64_t> pair_off, ess_off;  // per cloud, host
  int64_t n_pairs = 0, n_ess = 0;
  int64_t *p_birth = nullptr, *p_death = nullptr, *p_bd2 = nullptr, *p_dd2 = nullptr;
  int32_t* p_dim = nullptr;
  int64_t *e_idx = nullptr, *e_d2 = nullptr;
  int32_t* e_dim = nullptr;

  void* dalloc(size_t bytes);
  void dfree(void* p);
  void free_all();
};

namespace ph {

// Device-side bounds checks of the debug build (-DPH_DEBUG; the library's stand-in for a memory
// checker): a failed check records its code in *word (the first failure wins) and yields false,
// so that the caller skips the access; the host reports the code as an error. Without
// PH_DEBUG every check is `true` and costs nothing.
#ifdef PH_DEBUG
#define PH_DCHECK(word, cond, code) ((cond) ? true : (atomicCAS((word), 0, (code)), false))
#else
#define PH_DCHECK(word, cond, code) true
#endif

// an NVTX range for the lifetime of the object: a profiler timeline shows every entry point and
// pass (no cost without a profiler attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------------------------------------
// error handling
// ------------------------------------------------------------------------------------------
struct Fail {
  int code;
};

#define PH_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                       \
      throw ::ph::Fail{PH_ERR_CUDA};                                                       \
    }                                                                                      \
  } while (0)

#define PH_CHECK_LAUNCH()      \
  do {                         \
    ctx->launches++;           \
    PH_CUDA(cudaGetLastError()); \
  } while (0)

#define PH_REQUIRE(cond, code, msg) \
  do {                              \
    if (!(cond)) {                  \
      ctx->err = (msg);             \
      throw ::ph::Fail{code};       \
    }                               \
  } while (0)

template <class T>
T* alloc_n(ph_ctx* ctx, int64_t n) {
  return static_cast<T*>(ctx->dalloc(sizeof(T) * (size_t)(n > 0 ? n : 1)));
}

inline int grid_for(ph_ctx* ctx, int64_t n, int threads, int per_sm = 8) {
  int64_t want = (n + threads - 1) / threads;
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// ------------------------------------------------------------------------------------------
// device building blocks (256-thread blocks)
// ------------------------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

// inclusive warp scan of (a, b) sums
template <class T>
__device__ __forceinline__ T warp_incl_sum(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += u;
  }
  return v;
}

// exclusive block scan (sum) of one value per thread; returns the exclusive prefix and the
// block total, for blocks of W warps. `sh` must hold W + 1 elements.
template <class T, int W = kWarps>
__device__ __forceinline__ T block_excl_sum(T v, T* sh, T& total) {
  T inc = warp_incl_sum(v);
  int w = threadIdx.x >> 5;
  if (lane_id() == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    T x = (lane_id() < W) ? sh[lane_id()] : T(0);
    T xi = warp_incl_sum(x);
    if (lane_id() < W) sh[lane_id()] = xi - x;
    if (lane_id() == W - 1) sh[W] = xi;
  }
  __syncthreads();
  T res = inc - v + sh[w];
  total = sh[W];
  __syncthreads();
  return res;
}

// segmented running maximum: elements carry a segment id (non-decreasing along the array);
// combine(a, b) for a before b keeps b's segment and takes the max only inside one segment.
struct SegMax {
  int32_t seg;
  int32_t val;
};

__device__ __forceinline__ SegMax segmax_combine(SegMax a, SegMax b) {
  SegMax r;
  r.seg = b.seg;
  r.val = (a.seg == b.seg) ? (a.val > b.val ? a.val : b.val) : b.val;
  return r;
}

__device__ __forceinline__ SegMax warp_incl_segmax(SegMax v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    SegMax u;
    u.seg = __shfl_up_sync(0xffffffffu, v.seg, o);
    u.val = __shfl_up_sync(0xffffffffu, v.val, o);
    if ((int)lane_id() >= o) v = segmax_combine(u, v);
  }
  return v;
}

}  // namespace ph

// host entry points shared between translation units
namespace ph {
// scale_step > 0: simplices enter at the first scale r_i = i * scale_step (grid units,
// i = 0..n_scales) with diameter <= 2 r_i, and the filtration value is i
void build_vr(ph_ctx* ctx, const int32_t* coords, const int64_t* cloud_offsets, int32_t n_clouds,
              int64_t n_points, int32_t D, int32_t max_dim, int64_t max_diam2,
              int64_t scale_step = 0, int32_t n_scales = 0);
void load_boundary(ph_ctx* ctx, int64_t m, const int32_t* dims, const int64_t* colptr,
                   const int32_t* rows);
void compute_beta(ph_ctx* ctx);
void reduce_init(ph_ctx* ctx);
int reduce_run(ph_ctx* ctx, int32_t max_passes);
void extract_all(ph_ctx* ctx);
void free_reduce_state(ph_ctx* ctx);
// E^l of one cloud, one byte per simplex in filtration order, into host memory (n bytes)
void essential_estimate(ph_ctx* ctx, int32_t cloud, uint8_t* host_out, int64_t n);
// predicted lowstar per simplex of one cloud (filtration indices, -1), into host memory
void predicted_lows(ph_ctx* ctx, int32_t cloud, int32_t* host_out, int64_t n);
void reduced_columns(ph_ctx* ctx, int32_t cloud, int64_t n, int64_t* colptr, int32_t* rows,
                     int64_t capacity, int64_t* nnz_out);
// generic device helpers (ph_scan.cu)
void excl_scan_i64(ph_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev);
void radix_sort_u64(ph_ctx* ctx, uint64_t* keys, uint64_t* vals, int64_t n, int lo_bit,
                    int hi_bit, uint64_t* tmp_keys, uint64_t* tmp_vals);
}  // namespace ph
