// Parallel multi-scale reduction (Algorithm 2, Sec. 3.1) on the device.
//
// One pass = one cycle of the outer loop of Algorithm 2. Every decision of a pass is taken from
// the state at its start, so the result of a pass does not depend on thread scheduling:
//   (table)      tab[low(j)] = min j over the active columns and the pivots: the left-most
//                column with each low, which defines the neighbour sets N(j) (Eq. neighbours).
//                Two tables alternate between passes: the pass before resets one to the proven
//                pivots (owner), and its new pivots (k_phase1) and its survivors with their new
//                lows (k_add, atomicMin) fill it, so no kernel gathers the lows again; k_tab
//                builds the first pass's at set-up. With it, the first row of each (cloud, dim)
//                that is not known to be paired (for Corollary 10).
//   k_phase1     Phase I (Algorithm 5) as a segmented exclusive prefix-max over the active
//                columns of each (cloud, dim), P_j = largest low of an earlier colliding column,
//                in one pass over tiles with a decoupled look-back; then the marks: j is proven
//                if it is left-most for its low and low(j) = beta_j (Thm 5) or low(j) > P_j
//                (Thms 6-7); empty columns become final; the zero case of Corollary 10 zeroes a
//                column whose candidate rows are all paired; each new pivot clears column
//                low(j) (Lemma 1); each active slot's source candidate is stored for Phase II.
//                Also upper bounds of the space Phase II can need: the grid's last block stops
//                the pass after its marks if they exceed what the host provided (the host grows
//                it and continues the pass at Phase II).
//   k_add        Phase II: every colliding column l gets column tab[low(l)] added (XOR of two
//                sorted row lists, or of bitmaps once a column fills in). Sources are
//                left-most, hence never targets, so additions are independent. Survivors take
//                their place in the next active list by a decoupled look-back and their slot in
//                the other arena by one atomic per chunk; new pivots move to the pivot store
//                (their columns never change again). Blocks of 128 threads take 128-slot chunks
//                from a device work queue (64 and 64 once the lanes share merge pieces), or
//                each warp 32 slots once the list is short and its jobs long, and 8 slots in
//                the last, short passes. While jobs are short
//                each lane merges its own job; later the lanes share every job's merge-path
//                pieces. Ten specialisations (row lists / bitmaps x block / 32-slot warp
//                chunks x lane / piece merges, and 8-slot warp chunks with pieces); the loop
//                switches between them at most four times per reduction.
//   (p sets)     With Phase II limited to p neighbour sets (Sec. 3.4), k_set_* rank the sets
//                between k_phase1 and k_add and hold back the other targets.
//   k_commit     publishes the new locations of the columns other jobs may have been reading
//                and prepares the next pass's row state; its last block ends the pass: the
//                next active list, convergence (no collision left, Thm 8), the pass cap and
//                time bound, and inside a CUDA graph the conditional that repeats the pass.
// All per-pass state lives in device memory (DevState), so the same kernel sequence runs either
// from a host loop or as the body of a graph's conditional while node. Each kernel may start
// while its predecessor drains (programmatic dependent launch) and waits for it first.
#include <algorithm>

#include "ph_internal.cuh"

namespace ph {


enum : int32_t { ST_RUN = 0, ST_DONE = 1, ST_CAPPED = 2, ST_HOST = 3, ST_FAULT = 4,
                 ST_TIMEOUT = 5, ST_SWITCH = 6 };
constexpr int kSpinLimit = 1 << 22;  // iterations of a look-back wait before it gives up

struct DevState {
  int32_t* act;   // active ids, ascending
  int32_t* act2;  // next active list
  int32_t* alen;   // per slot of act: its column's stored length (ColMeta::len)
  int32_t* alen2;  // the same for act2
  int64_t n_act;
  int32_t* arena[2];  // pass p writes its survivors into arena[p & 1]
  int32_t* tab[2];    // pass p reads its left-most-column table tab[p & 1], builds tab[(p+1) & 1]
  int64_t arena_cap[2];
  int32_t* piv_base;  // current chunk of the pivot store
  int64_t piv_cap;
  // counters that many blocks update by atomics each sit on their own 128-byte line, so that
  // different L2 slices serve them
  alignas(128) unsigned long long piv_used;
  int64_t* stats;  // [stats_rows][PH_PS_N] or nullptr
  int32_t stats_rows;
  int32_t pass;
  int32_t max_passes;
  int32_t status;
  int32_t passes;
  int32_t host_reason;  // 1 arena, 2 pivot store, 4 counter rows
  unsigned int blocks_done;       // blocks of the current grid that have finished (last-block)
  unsigned long long t_start;     // global timer (ns) when this ph_reduce's loop began
  unsigned long long t_limit;     // ns the loop may run before it stops with ST_TIMEOUT
  alignas(128) unsigned long long totals[2];  // [1]: targets of the current pass ([0] unused)
  unsigned long long bound_words, bound_piv;
  alignas(128) unsigned long long arena_used;  // words taken in the arena of the current pass
  alignas(128) unsigned int queue;             // next chunk for k_add
  alignas(128) unsigned int tile_queue;        // next tile for k_phase1
  alignas(128) int32_t n_deferred;             // entries of dlist
  alignas(128) int32_t fault;                  // a bounded wait ran out
  int32_t debug_fault;  // the first failed bounds check of the debug build (PH_DCHECK), 0 if none
  // bit-packed columns: the passes after the first one that saw a target that may reach its
  // threshold run the additions kernel that handles them (and converts columns); the pass loop
  // stops once there (ST_SWITCH) so that the host continues it with that kernel
  int32_t dense_on;
  int32_t dense_want;
  // Phase II work shape: 128-slot chunks per block while the active list is long or its jobs
  // short, 32-slot chunks per warp (no block barriers, more queue atomics) once it holds fewer
  // than warp_below columns whose survivors reserve warp_words or more arena words on
  // average; this switches once per reduction (ST_SWITCH)
  int32_t warp_on;
  int64_t warp_below;
  int64_t warp_words;  // the mean arena words per survivor the switch needs
  // Phase II merges each job in its own lane while jobs are short (lane_on), and merge pieces
  // spread over the lanes once the mean arena words per survivor reach lane_words; this
  // switches once per reduction (ST_SWITCH)
  int32_t lane_on;
  int64_t lane_words;
  // ... and once merge pieces are on and fewer than narrow_below columns are active, warp
  // chunks of 8 slots, so that the short late passes spread over more warps (ST_SWITCH, once)
  int32_t narrow_on;
  int64_t narrow_below;
  int32_t chunk_slots;  // slots per chunk of this pass's additions kernel (8, 32 or 128)
};

struct RArgs {
  DevState* ds;
  int32_t* low;
  const int32_t* beta;
  ColMeta* meta;      // per id: the column's rows, length, flags and clearing mark
  int32_t** nxt_ptr;
  int32_t* nxt_len;
  int32_t* owner;
  int32_t* first_unp;
  const int32_t* seg;
  int64_t rows_end;
  int nseg;           // (cloud, dim) segments
  int nc;
  int strict;
  int cor10;
  unsigned long long* tile_st;  // per Phase I tile: look-back state of its aggregate / prefix
  unsigned long long* look;  // per Phase II chunk: look-back state of the survivor count
  int32_t* dlist;     // active slots whose column update waits for k_commit
  int32_t* src_e;     // per active slot: the colliding column's left-most column, -1 if none
  // bit-packed columns: a job's result is a bitmap over its row segment when the sum of the two
  // row counts exceeds the threshold, max(the stored bitmap's words, t0) with t0 = dense_mode
  // when > 0, else 32 (dense_mode < 0: never), or when either column is already a bitmap
  int dense_mode;
  int32_t dense_floor;             // no addition of at most this many rows goes bit-packed
  int32_t dense_min[kMaxDim + 1];  // per column dimension: smallest threshold of its segments
  int32_t dim_start[kMaxDim + 1];  // first column id of each dimension (m above the top one)
  const int64_t* seg_start;        // device copy of the segment table
  int predict;        // 1: Corollary 10 non-zero case (pair predictions)
  uint32_t* unp_bits; // per row, bit: not known to be paired at the start of the pass
  int32_t* unp_words; // [nwords + 1] exclusive prefix of unpaired rows per 32-row word
  int32_t* pred;      // per id: predicted lowstar (Corollary 10), -1
  int staged_max;     // merges of more rows than this run from global memory
  int force_km;       // > 0: merge-path positions per lane for every warp
  // Phase II limited to p neighbour sets per pass (Sec. 3.4): per row of the boundary
  int32_t* set_n;     // eligible targets of the row's set
  int32_t* set_neg;   // those known to be negative
  uint8_t* set_on;    // the set is acted on this pass
};

// per-pass values, read once at kernel start (no kernel changes them while others read them)
struct PV {
  int32_t* act;
  int32_t* act2;
  int32_t* alen;
  int32_t* alen2;
  int64_t n_act;
  int do_adds;
  int64_t* stats;
  int32_t* arena_next;
  int32_t* piv_base;
  int dense_on;
  int64_t arena_next_cap;  // words of arena_next and of the pivot store's chunk (bounds checks)
  int64_t piv_cap;
  int32_t* tab;       // per row: the left-most active column with that low (or its pivot)
  int32_t* tab_next;  // the same for the next pass, built during this one
};

__device__ __forceinline__ PV pass_view(const DevState* ds) {
  PV v;
  v.act = ds->act;
  v.act2 = ds->act2;
  v.alen = ds->alen;
  v.alen2 = ds->alen2;
  v.n_act = ds->n_act;
  v.do_adds = ds->pass < ds->max_passes;
  v.stats = ds->stats ? ds->stats + (int64_t)ds->pass * PH_PS_N : nullptr;
  v.arena_next = ds->arena[ds->pass & 1];
  v.piv_base = ds->piv_base;
  v.dense_on = ds->dense_on;
  v.arena_next_cap = ds->arena_cap[ds->pass & 1];
  v.piv_cap = ds->piv_cap;
  v.tab = ds->tab[ds->pass & 1];
  v.tab_next = ds->tab[(ds->pass + 1) & 1];
  return v;
}

__device__ __forceinline__ void stat_add(int64_t* stats, int k, int64_t v) {
  // warp-aggregated counter update
  int64_t s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane_id() == 0 && s != 0) atomicAdd((unsigned long long*)&stats[k], (unsigned long long)s);
}


// Programmatic dependent launch. The kernels of a pass are launched so that each may start
// while the one before it in the stream drains (its blocks fill the SMs that kernel frees): every
// pass kernel first waits here until the previous kernel has completed and its writes are
// visible, before it reads or writes anything. Without such a predecessor the wait returns at
// once. The trigger, given once a kernel's blocks run, lets the next kernel's launch begin.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// True in the one block that finishes the grid last; it then sees every other block's writes.
// Only the first `participants` blocks of the grid may call it (the others have no work and
// may leave at once).
__device__ __forceinline__ bool last_block(unsigned int* done, unsigned int participants) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == participants - 1;
  __syncthreads();
  return s_last;
}

// ------------------------------------------------------------------------------------------
// The row state pass q reads, from the pivots, flags and beta as they stand when the pass before
// it ends (k_commit; at set-up for the first pass): the reset, to the proven pivots (owner), of
// the table that pass q's additions fill for pass q + 1; the first row of each (cloud, dim)
// segment that is not known to be paired (Corollary 10; two copies alternate between passes);
// and the unpaired bitmap (pair predictions). Every block of the grid takes part; the grid's last
// block then finishes it with rows_of_pass_last.
__device__ void rows_of_pass(const RArgs& a, int32_t q) {
  int32_t* tab_reset = a.ds->tab[(q + 1) & 1];
  int32_t* fu = a.first_unp + (int64_t)(q & 1) * a.nseg;
  // warp-uniform loop: each iteration a warp covers 32 consecutive rows, one bitmap word
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); x0 < a.rows_end;
       x0 += stride) {
    const int64_t x = x0 + (threadIdx.x & 31);
    bool unpaired = false;
    if (x < a.rows_end) {
      int32_t o = a.owner[x];
      tab_reset[x] = o < 0 ? INT32_MAX : o;
      unpaired = !((a.meta[x].flags & F_PROVEN) || a.beta[x] >= 0 || o >= 0);
    }
    const unsigned w = __ballot_sync(0xffffffffu, unpaired);
    if (unpaired) {  // one atomic per segment present among the warp's unpaired rows: its first
      const int32_t sg = a.seg[x];
      const unsigned same = __match_any_sync(w, sg);
      if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMin(&fu[sg], (int32_t)x);
    }
    if (a.predict && (threadIdx.x & 31) == 0) a.unp_bits[x0 >> 5] = w;
  }
}

// by the last block: the bitmap's prefix counts per word, and the first-unpaired copy of pass
// q + 1 cleared for the atomics at the end of pass q
__device__ void rows_of_pass_last(const RArgs& a, int32_t q) {
  if (a.predict) {
    __shared__ int64_t sh[kWarps + 1];
    const int64_t nwords = (a.rows_end + 31) / 32;
    int64_t carry = 0;
    for (int64_t base = 0; base < nwords; base += kThreads) {
      const int64_t w = base + threadIdx.x;
      const int64_t c = w < nwords ? __popc(__ldcg(a.unp_bits + w)) : 0;
      int64_t tot;
      const int64_t ex = block_excl_sum<int64_t>(c, sh, tot);
      if (w < nwords) a.unp_words[w] = (int32_t)(carry + ex);
      carry += tot;
    }
    if (threadIdx.x == 0) a.unp_words[nwords] = (int32_t)carry;
  }
  int32_t* fu_next = a.first_unp + (int64_t)((q + 1) & 1) * a.nseg;
  for (int i = threadIdx.x; i < a.nseg; i += blockDim.x) fu_next[i] = INT32_MAX;
}

// set-up: the first pass's row state
__global__ void k_rows_first(RArgs a) {
  const int32_t q = a.ds->pass;
  rows_of_pass(a, q);
  if (last_block(&a.ds->blocks_done, gridDim.x)) {
    rows_of_pass_last(a, q);
    if (threadIdx.x == 0) a.ds->blocks_done = 0;
  }
}

// rows of the start-of-pass unpaired bitmap before row x
__device__ __forceinline__ int32_t unpaired_before(const RArgs& a, int64_t x) {
  const int64_t w = x >> 5;
  const unsigned low_bits = (x & 31) ? (0xffffffffu >> (32 - (x & 31))) : 0u;
  return a.unp_words[w] + ((x & 31) ? __popc(a.unp_bits[w] & low_bits) : 0);
}

// Corollary 10, non-zero case: beta_j >= 0 makes j negative (Thm 5), so its candidate set L_j
// holds the unpaired rows of K_{d-1} in [beta_j, low(j)] only (rows of one cloud's segment are
// contiguous ids). One candidate is lowstar(j) (Lemma 9). Returns it, -1 if there are several,
// -2 if there is none (impossible; counted as a check).
__device__ __forceinline__ int32_t predicted_low(const RArgs& a, int32_t b, int32_t l) {
  const int32_t c0 = unpaired_before(a, b);
  const int32_t n = unpaired_before(a, (int64_t)l + 1) - c0;
  if (n != 1) return n == 0 ? -2 : -1;
  int64_t lo = b >> 5, hi = l >> 5;  // last word whose prefix is <= c0
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (a.unp_words[mid] <= c0) lo = mid; else hi = mid - 1;
  }
  unsigned bits = a.unp_bits[lo];
  for (int32_t k = c0 - a.unp_words[lo]; k > 0; k--) bits &= bits - 1;  // skip k set bits
  return (int32_t)(lo * 32 + __ffs(bits) - 1);
}

// The first pass's left-most-column table (at set-up; every later pass's table is filled by the
// pass before it): tab[low(j)] = min j over the active columns by atomicMin, and every low
// marked as seen for the essential estimate. kTI consecutive slots per thread and iteration,
// their loads issued together.
constexpr int kTabItems = 4;
__global__ void k_tab(RArgs a) {
  pdl_wait();
  pdl_trigger();
  if (a.ds->status != ST_RUN) return;
  const PV v = pass_view(a.ds);
  constexpr int kTI = kTabItems;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kTI;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kTI; i0 < v.n_act;
       i0 += stride) {
    int32_t j[kTI], l[kTI];
#pragma unroll
    for (int k = 0; k < kTI; k++) j[k] = i0 + k < v.n_act ? v.act[i0 + k] : -1;
#pragma unroll
    for (int k = 0; k < kTI; k++) l[k] = j[k] >= 0 ? a.low[j[k]] : -1;
#pragma unroll
    for (int k = 0; k < kTI; k++) {
      if (l[k] >= 0 && PH_DCHECK(&a.ds->debug_fault, l[k] < a.rows_end, 1)) {
        if (v.tab[l[k]] > j[k]) atomicMin(&v.tab[l[k]], j[k]);
        if (!a.meta[l[k]].low_seen) a.meta[l[k]].low_seen = 1;  // for the essential estimate
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// bit-packed columns
// ------------------------------------------------------------------------------------------
// the smallest threshold over the segments of column j's dimension (fixed indices only: a
// kernel parameter array indexed at run time would be copied out)
__device__ __forceinline__ int32_t dense_min_of(const RArgs& a, int32_t j) {
  int32_t t = a.dense_min[0];
#pragma unroll
  for (int k = 1; k <= kMaxDim; k++) t = j >= a.dim_start[k] ? a.dense_min[k] : t;
  return t;
}

// the (cloud, dim) segment of column j, seg[j] = dim * clouds + cloud: with one cloud the
// dimension, found from the dimension starts (no load); else loaded
__device__ __forceinline__ int32_t seg_of(const RArgs& a, int32_t j) {
  if (a.nc != 1) return a.seg[j];
  int32_t d = 0;
#pragma unroll
  for (int k = 1; k <= kMaxDim; k++) d += j >= a.dim_start[k] ? 1 : 0;
  return d;
}

// first column id of column j's dimension
__device__ __forceinline__ int32_t dim_start_of(const RArgs& a, int32_t j) {
  int32_t b = 0;
#pragma unroll
  for (int k = 1; k <= kMaxDim; k++) b = j >= a.dim_start[k] ? a.dim_start[k] : b;
  return b;
}
// the smallest threshold over the dimensions of the columns j0..j1 (none: INT32_MAX)
__device__ __forceinline__ int32_t dense_min_between(const RArgs& a, int32_t j0, int32_t j1) {
  int32_t t = INT32_MAX;
#pragma unroll
  for (int k = 0; k <= kMaxDim; k++) {
    const int32_t end = k < kMaxDim ? a.dim_start[k + 1] : INT32_MAX;
    if (j0 <= j1 && a.dim_start[k] <= j1 && end > j0) t = min(t, a.dense_min[k]);
  }
  return t;
}

// row segment of column j: first row id and bitmap words
__device__ __forceinline__ void row_segment(const RArgs& a, int32_t j, int64_t& base,
                                            int32_t& words) {
  const int rs = a.seg[j] - a.nc;
  base = a.seg_start[rs];
  words = (int32_t)((a.seg_start[rs + 1] - base + 31) / 32);
}

// A bit-packed column is stored as one header word (its row count) followed by the bitmap, bit
// r - base of word (r - base) / 32 for row r of the segment. Its length field holds
// -(stored words) - 1, so a plain length load tells the two forms apart, and the stored words of
// either form are what a move of the column takes: Phase I reserves that much for it.
constexpr int kDenseHead = 1;
__device__ __forceinline__ int32_t stored_words(int32_t len) { return len < 0 ? -len - 1 : len; }
__device__ __forceinline__ int32_t dense_len(int32_t words) { return -words - 1; }

// does an addition of n rows in all (target + source) into column j produce a bitmap? The
// stored bitmap is smaller than n, so it fits the n words Phase I reserved for the result
__device__ __noinline__ bool goes_dense_slow(const RArgs& a, int32_t j, int64_t n) {
  int64_t base;
  int32_t words;
  row_segment(a, j, base, words);
  return n > max(words + kDenseHead, a.dense_mode > 0 ? a.dense_mode : 32);
}
// the cheap part first: no bitmap at or below the floor, nor below every segment of j's dimension
__device__ __forceinline__ bool goes_dense(const RArgs& a, int32_t j, int64_t n) {
  return n > a.dense_floor && n > dense_min_of(a, j) && goes_dense_slow(a, j, n);
}


// ------------------------------------------------------------------------------------------
// Phase I scan
// ------------------------------------------------------------------------------------------
// exclusive block scan with carry-in; returns the exclusive prefix, sets the running total
__device__ __forceinline__ SegMax block_scan_segmax(SegMax v, SegMax carry, SegMax* sh,
                                                    SegMax& total) {
  const int lane = lane_id(), w = threadIdx.x >> 5;
  SegMax inc = warp_incl_segmax(v);
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    SegMax x = lane < kWarps ? sh[lane] : SegMax{INT32_MAX, -1};
    SegMax xi = warp_incl_segmax(x);
    SegMax xe;
    xe.seg = __shfl_up_sync(0xffffffffu, xi.seg, 1);
    xe.val = __shfl_up_sync(0xffffffffu, xi.val, 1);
    xe = lane == 0 ? carry : segmax_combine(carry, xe);
    if (lane < kWarps) sh[lane] = xe;
    if (lane == kWarps - 1) sh[kWarps] = segmax_combine(carry, xi);
  }
  __syncthreads();
  SegMax pre = sh[w];
  SegMax ex;
  ex.seg = __shfl_up_sync(0xffffffffu, inc.seg, 1);
  ex.val = __shfl_up_sync(0xffffffffu, inc.val, 1);
  ex = lane == 0 ? pre : segmax_combine(pre, ex);
  total = sh[kWarps];
  __syncthreads();
  return ex;
}


// the space this pass's Phase II can need (arena, pivot store) against what the host provided;
// no column has changed yet, and the marks made depend only on the pass's starting state, so a
// pass stopped here continues at Phase II once the host has grown the buffers
__device__ __forceinline__ void check_capacity(DevState* ds) {
  int reason = 0;
  if (ds->bound_words > (unsigned long long)ds->arena_cap[ds->pass & 1]) reason |= 1;
  if (ds->bound_piv + ds->piv_used > (unsigned long long)ds->piv_cap) reason |= 2;
  if (reason) {
    ds->host_reason = reason;
    ds->status = ST_HOST;
  }
}

// Phase I and the marks in one kernel, a single-pass scan over tiles of kFTile active slots
// (kFItems consecutive slots per thread), claimed in order from a work queue. A tile loads its
// slots' columns, lows, sources and lengths once; takes its Phase I aggregate and each thread's
// prefix within the tile from one block scan; publishes the aggregate and looks back over the
// tiles before it for its prefix (decoupled look-back, as the additions kernel's survivor
// count); then applies the marks. The space bounds of the pass are summed on the way, and the
// grid's last block checks them against what the host provided: a pass that does not fit stops
// after its marks (which depend only on the state at the pass's start) and the host continues it
// at Phase II once the buffers have grown.
constexpr int kFItems = 4;
constexpr int kFTile = kThreads * kFItems;
// tile state word: pass tag (8 bits) | flags (2) | segment (23) | val + 1 (31). Eight bits of
// tag tell this pass from the previous ones: the active list never grows within a reduction, so
// a tile in use in pass p was in use, and published, in pass p - 1, and set-up clears every state
constexpr unsigned long long kTAgg = 1ull << 54, kTIncl = 2ull << 54, kTFlags = 3ull << 54;
__device__ __forceinline__ unsigned long long tile_word(unsigned long long tag, unsigned long long flag,
                                                       SegMax x) {
  return tag | flag | ((unsigned long long)(x.seg & 0x7fffff) << 31) |
         (unsigned long long)((uint32_t)(x.val + 1) & 0x7fffffffu);
}
__device__ __forceinline__ SegMax tile_value(unsigned long long w) {
  return SegMax{(int32_t)((w >> 31) & 0x7fffff), (int32_t)(w & 0x7fffffffu) - 1};
}

// by warp 0: publishes tile t's aggregate, returns the Phase I value of every tile before it
// (SegMax{-1, -1}, a left identity of segmax_combine, for none) and publishes t's inclusive state
__device__ __forceinline__ SegMax tile_look_back(const RArgs& a, int32_t pass, int64_t t,
                                                 SegMax agg, bool& fault) {
  const int lane = lane_id();
  const unsigned long long tag = (unsigned long long)(pass & 0xff) << 56;
  unsigned long long* st = a.tile_st;
  const SegMax none{-1, -1};
  if (t == 0) {
    if (lane == 0) atomicExch(st, tile_word(tag, kTIncl, agg));
    return none;
  }
  if (lane == 0) atomicExch(st + t, tile_word(tag, kTAgg, agg));
  SegMax acc = none;
  bool have = false;
  for (int64_t p = t - 1;; p -= 32) {
    const int64_t q = p - lane;  // lane 0 the nearest tile
    SegMax x = none;
    bool incl = true;  // before tile 0: an inclusive state of nothing
    if (q >= 0) {
      unsigned long long w = 0;
      for (int it = 0;; it++) {
        w = *(const volatile unsigned long long*)(st + q);
        if ((w >> 56) == (tag >> 56) && (w & kTFlags)) break;
        if (it > kSpinLimit) {
          fault = true;
          w = tag | kTIncl;
          break;
        }
        __nanosleep(32);
      }
      x = tile_value(w);
      incl = (w & kTFlags) == kTIncl;
    }
    const unsigned im = __ballot_sync(0xffffffffu, incl);
    const int stop = im ? __ffs(im) - 1 : 32;
    // the window in order, farthest (highest lane) first; lanes past the stop are left identities
    SegMax val = lane <= stop ? x : none;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      SegMax u;
      u.seg = __shfl_down_sync(0xffffffffu, val.seg, o);
      u.val = __shfl_down_sync(0xffffffffu, val.val, o);
      if (lane + o < 32) val = segmax_combine(u, val);
    }
    SegMax win;
    win.seg = __shfl_sync(0xffffffffu, val.seg, 0);
    win.val = __shfl_sync(0xffffffffu, val.val, 0);
    acc = have ? segmax_combine(win, acc) : win;  // this window comes before the later ones
    have = true;
    if (im) break;
  }
  if (lane == 0) atomicExch(st + t, tile_word(tag, kTIncl, segmax_combine(acc, agg)));
  return acc;
}

__global__ void __launch_bounds__(kThreads, 4) k_phase1(RArgs a) {
  __shared__ SegMax sh[kWarps + 1];
  __shared__ int64_t shs[kWarps + 1];
  __shared__ int64_t s_tile;
  __shared__ SegMax s_pre;
  constexpr int kFI = kFItems;
  pdl_wait();
  pdl_trigger();
  DevState* ds = a.ds;
  if (ds->status != ST_RUN) return;
  const PV v = pass_view(ds);
  const int32_t pass = ds->pass;
  const int32_t* fu = a.first_unp + (int64_t)(pass & 1) * a.nseg;  // this pass's copy
  const int64_t ntiles = (v.n_act + kFTile - 1) / kFTile;
  // no more blocks take part than there are tiles (the others leave at once: a short pass's
  // grid is mostly idle); block 0 always does (the last block checks capacity)
  const unsigned parts = (unsigned)std::max<int64_t>(1, std::min<int64_t>(gridDim.x, ntiles));
  if (blockIdx.x >= parts) return;
  int64_t bw = 0, bp = 0;
  int64_t n_zero = 0, n_piv = 0, n_c10 = 0, n_pred = 0, n_empty = 0;
  bool want = false;  // a target whose addition may reach its dimension's bit-packing threshold
  bool fault = false;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&ds->tile_queue, 1u);
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= ntiles) break;
    const int64_t tile0 = t * kFTile;
    // bit-packing thresholds of the tile's columns (ascending ids, so dimensions too): exact in
    // the top dimension (ids from t_b on), the smallest of the others below it
    int32_t t_b = 0, t_hi = INT32_MAX, t_lo = INT32_MAX;
    if (a.dense_floor != INT32_MAX) {
      const int32_t j0 = v.act[tile0];
      const int32_t j1 = v.act[min(tile0 + kFTile, v.n_act) - 1];
      t_b = dim_start_of(a, j1);
      t_hi = dense_min_of(a, j1);
      t_lo = dense_min_between(a, j0, t_b - 1);
    }
    const int64_t e0 = tile0 + (int64_t)threadIdx.x * kFI;
    int32_t j[kFI], l[kFI], sg[kFI], n[kFI], b[kFI], s[kFI];
#pragma unroll
    for (int i = 0; i < kFI; i++) j[i] = e0 + i < v.n_act ? v.act[e0 + i] : -1;
#pragma unroll
    for (int i = 0; i < kFI; i++) {
      l[i] = j[i] >= 0 ? a.low[j[i]] : -1;
      sg[i] = j[i] >= 0 ? seg_of(a, j[i]) : INT32_MAX;
      n[i] = j[i] >= 0 ? v.alen[e0 + i] : 0;
      b[i] = j[i] >= 0 ? a.beta[j[i]] : -1;
    }
#pragma unroll
    for (int i = 0; i < kFI; i++) {
      if (!PH_DCHECK(&ds->debug_fault, l[i] < a.rows_end, 2)) l[i] = -1, j[i] = -1;
      s[i] = l[i] >= 0 ? v.tab[l[i]] : -1;
    }
    // Phase I values (the low of a colliding column, in its (cloud, dim) segment) and the space
    // bounds: a column's reservation is its stored words (its rows, or its bitmap with the
    // header); a target's source may be added; a left-most column may be proven and move
    SegMax x[kFI];
#pragma unroll
    for (int i = 0; i < kFI; i++) {
      const bool collide = l[i] >= 0 && s[i] != j[i];
      bw += stored_words(n[i]);
      if (collide) {
        const int32_t ns = stored_words(a.meta[s[i]].len);
        bw += ns;
        want |= n[i] + ns > (j[i] >= t_b ? t_hi : t_lo);
      } else if (l[i] >= 0) {
        bp += stored_words(n[i]);
      }
      x[i] = SegMax{sg[i], collide ? l[i] : -1};
    }
    SegMax agg = x[0];
#pragma unroll
    for (int i = 1; i < kFI; i++) agg = segmax_combine(agg, x[i]);
    SegMax tot;
    const SegMax pre_t = block_scan_segmax(agg, SegMax{-1, -1}, sh, tot);  // within the tile
    if (threadIdx.x < 32) {
      const SegMax P = tile_look_back(a, pass, t, tot, fault);
      if (threadIdx.x == 0) s_pre = P;
    }
    // the marks: a new pivot proven by Thm 5 (left-most, low = beta) or by Phase I (left-most,
    // low > P_j); else the zero case of Corollary 10, else a pair prediction. Every active
    // column carries no flag (proven, final and cleared columns leave the active list in the
    // pass that marks them; the new-pivot mark goes with them), so marks are stored without a
    // load. Only a left-most column whose low is not its beta needs P_j: the others are marked
    // while warp 0 looks back, the rest after the tile's prefix is known.
    auto pivot = [&](int i) {
      a.meta[j[i]].flags = F_PROVEN | F_NEWPIV;
      a.owner[l[i]] = j[i];
      atomicMin(&v.tab_next[l[i]], j[i]);  // its row's pivot from the next pass on
      a.meta[l[i]].cleared = 1;  // clearing (Lemma 1): column l is positive and paired with j
      n_piv++;
    };
    auto unproven = [&](int i) {
      if (a.cor10 && b[i] < 0 && l[i] < fu[sg[i] - a.nc]) {
        a.meta[j[i]].flags = F_FINAL;  // Corollary 10, zero case
        n_c10++;
      } else if (a.predict && b[i] >= 0 && a.pred[j[i]] < 0) {
        const int32_t pi = predicted_low(a, b[i], l[i]);
        if (pi >= 0) {
          a.pred[j[i]] = pi;
          n_pred++;
        } else if (pi == -2) {
          n_empty++;
        }
      }
    };
    unsigned waits = 0;  // items whose mark needs P_j
#pragma unroll
    for (int i = 0; i < kFI; i++) {
      if (j[i] < 0) continue;
      a.src_e[e0 + i] = s[i] != j[i] ? s[i] : -1;  // Phase II reads it in list order
      (void)PH_DCHECK(&ds->debug_fault, a.meta[j[i]].flags == 0, 7);
      if (l[i] < 0) {
        a.meta[j[i]].flags = F_FINAL;
        n_zero++;
      } else if (s[i] != j[i]) {
        unproven(i);
      } else if (l[i] == b[i]) {
        pivot(i);
      } else {
        waits |= 1u << i;
      }
    }
    __syncthreads();
    if (waits) {
      SegMax run = threadIdx.x == 0 ? s_pre : segmax_combine(s_pre, pre_t);
#pragma unroll
      for (int i = 0; i < kFI; i++) {
        const SegMax pre = run;
        run = segmax_combine(run, x[i]);
        if (!((waits >> i) & 1u)) continue;
        const int32_t P = (pre.seg == x[i].seg) ? pre.val : -1;
        if (l[i] > P) pivot(i); else unproven(i);
      }
    }
  }
  if (v.stats) {
    stat_add(v.stats, PH_PS_ZERO_FINAL, n_zero);
    stat_add(v.stats, PH_PS_NEW_PIVOTS, n_piv);
    stat_add(v.stats, PH_PS_PREDICTED, n_pred);
    stat_add(v.stats, PH_PS_EMPTY_L, n_empty);
    stat_add(v.stats, PH_PS_COR10, n_c10);
  }
  if (want && !v.dense_on) ds->dense_want = 1;  // bit-packed additions from the next pass
  if (__any_sync(0xffffffffu, fault) && lane_id() == 0) ds->fault = 1;
  int64_t tw, tp;
  block_excl_sum<int64_t>(bw, shs, tw);
  block_excl_sum<int64_t>(bp, shs, tp);
  if (threadIdx.x == 0 && (tw || tp)) {
    atomicAdd(&ds->bound_words, (unsigned long long)tw);
    atomicAdd(&ds->bound_piv, (unsigned long long)tp);
  }
  // the last of the taking-part blocks checks the space this pass's Phase II needs
  if (last_block(&ds->blocks_done, parts)) {
    if (threadIdx.x == 0) {
      ds->blocks_done = 0;
      check_capacity(ds);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Phase II with p processors (Sec. 3.4): the neighbour sets a pass acts on
// ------------------------------------------------------------------------------------------
// every active target whose addition this pass may do is counted in its set (row low(j));
// the tests are those of the additions themselves, applied to the marks of this pass
__global__ void k_set_count(RArgs a) {
  if (a.ds->status != ST_RUN) return;
  const PV v = pass_view(a.ds);
  if (!v.do_adds) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n_act; e += stride) {
    const int32_t s = a.src_e[e];
    if (s < 0) continue;
    const int32_t j = v.act[e];
    const ColMeta mj = load_meta(a.meta + j);
    if ((mj.flags & (F_PROVEN | F_FINAL)) || mj.cleared) continue;
    const ColMeta ms = load_meta(a.meta + s);
    if ((ms.flags & F_FINAL) || ms.cleared || (a.strict && !(ms.flags & F_PROVEN))) continue;
    const int32_t i = a.low[j];
    atomicAdd(a.set_n + i, 1);
    if (a.beta[j] >= 0) atomicAdd(a.set_neg + i, 1);
  }
}

// Ties between sets go to the row that comes first in its cloud's filtration (then to the
// lower id): the rows are first sorted by their filtration index, and the stable sort by
// priority below keeps that order among equal keys.
__global__ void k_set_tiekeys(RArgs a, const int64_t* __restrict__ gidx, uint64_t* key,
                              uint64_t* row) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.rows_end; i += stride) {
    key[i] = (uint64_t)gidx[i];
    row[i] = (uint64_t)i;
    a.set_on[i] = 0;
  }
}

// Sort keys of the sets, in the current order of the rows: ascending key order is the priority
// order (priority 0: larger sets first; 1: more known-negative targets first, then larger
// sets); rows without a set sort last. bits: enough for any count.
__global__ void k_set_keys(RArgs a, int priority, int bits, uint64_t* key,
                           const uint64_t* __restrict__ row) {
  const uint64_t top = (1ull << bits) - 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.rows_end; t += stride) {
    const int64_t i = (int64_t)row[t];
    const uint64_t n = (uint64_t)a.set_n[i], g = (uint64_t)a.set_neg[i];
    key[t] = priority == 1 ? ((top - g) << bits) | (top - n) : top - n;
  }
}

// the first p sets of the sorted order are acted on
__global__ void k_set_select(RArgs a, int64_t p, const uint64_t* __restrict__ row) {
  const int64_t n = p < a.rows_end ? p : a.rows_end;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += stride) {
    const int64_t i = (int64_t)row[t];
    if (a.set_n[i] > 0) a.set_on[i] = 1;
  }
}

// a target outside the chosen sets keeps its collision (it counts as a target) but skips its
// addition this pass: its slot's source becomes -2 - s
__global__ void k_set_apply(RArgs a) {
  if (a.ds->status != ST_RUN) return;
  const PV v = pass_view(a.ds);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < v.n_act; e += stride) {
    const int32_t s = a.src_e[e];
    if (s >= 0 && !a.set_on[a.low[v.act[e]]]) a.src_e[e] = -2 - s;
  }
}

// ------------------------------------------------------------------------------------------
// what happens to an active column in Phase II
// ------------------------------------------------------------------------------------------
// One job by the whole warp on bitmaps: column A (rows, or a bit-packed column if dense_a) plus
// source B (likewise, dense_b) into the bit-packed column T, the job's reserved slot. Writes
// T's header and returns its row count; its largest row goes to low, its stored words to words.
__device__ __noinline__ int32_t dense_job_warp(const RArgs& a, int32_t j, const int32_t* A,
                                              int na, bool dense_a, const int32_t* B, int nb,
                                              bool dense_b, int32_t* T, int32_t& low,
                                              int32_t& words) {
  const int lane = lane_id();
  int64_t base;
  int32_t W;
  row_segment(a, j, base, W);
#ifdef PH_DEBUG
  // the bitmap fits the slot reserved for the job (na + nb stored words)
  if (!PH_DCHECK(&a.ds->debug_fault, W + kDenseHead <= na + nb, 6)) {
    low = -1;
    words = 0;
    return 0;
  }
#endif
  uint32_t* bits = reinterpret_cast<uint32_t*>(T + kDenseHead);
  const uint32_t* Ab = reinterpret_cast<const uint32_t*>(A + kDenseHead);
  const uint32_t* Bb = reinterpret_cast<const uint32_t*>(B + kDenseHead);
  const bool wb = B != nullptr && dense_b;
  for (int w = lane; w < W; w += 32) bits[w] = (dense_a ? Ab[w] : 0u) ^ (wb ? Bb[w] : 0u);
  __syncwarp();
  // the row lists, scattered bit by bit (rows of one list are distinct; the lists may share)
  if (!dense_a)
    for (int q = lane; q < na; q += 32) {
      const int64_t r = A[q] - base;
      atomicXor(bits + (r >> 5), 1u << (r & 31));
    }
  if (B != nullptr && !dense_b)
    for (int q = lane; q < nb; q += 32) {
      const int64_t r = B[q] - base;
      atomicXor(bits + (r >> 5), 1u << (r & 31));
    }
  __syncwarp();
  // rows and the largest row of the result (read from L2, where the atomics landed)
  int cnt = 0, top_w = -1;
  uint32_t top_bits = 0;
  for (int w = lane; w < W; w += 32) {
    const uint32_t x = __ldcg(bits + w);
    cnt += __popc(x);
    if (x) {
      top_w = w;
      top_bits = x;
    }
  }
  const int best = __reduce_max_sync(0xffffffffu, (unsigned)(top_w + 1)) - 1;
  const unsigned who = __ballot_sync(0xffffffffu, top_w == best && best >= 0);
  low = -1;
  if (best >= 0) {
    const uint32_t tb = __shfl_sync(0xffffffffu, top_bits, __ffs(who) - 1);
    low = (int32_t)(base + 32 * (int64_t)best + 31 - __clz(tb));
  }
  const int32_t rows = (int32_t)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
  if (lane == 0) T[0] = rows;
  __syncwarp();
  words = W + kDenseHead;
  return rows;
}

struct Job {
  int32_t j;
  int32_t src;    // source column for an addition, -1 if none
  bool surv;      // stays active
  bool newpiv;    // proven this pass: moves to the pivot store
  bool target;    // collides with an earlier column
  int64_t words;  // arena words reserved (survivors only)
  const int32_t* A;  // the column's rows (new pivots and survivors)
  const int32_t* B;  // the source's rows (additions)
  int na, nb;
  bool dense_a, dense_b;  // A / B is a bit-packed column (na / nb are then its stored words)
};

// kDense: columns may be bit-packed (the length field tells); otherwise every column is a row list
template <bool kDense>
__device__ __forceinline__ Job job_of(const RArgs& a, const PV& v, int64_t e) {
  Job jb{-1, -1, false, false, false, 0, nullptr, nullptr, 0, 0, false, false};
  if (e >= v.n_act) return jb;
  // every load is issued up front: the column and its source candidate are known from the
  // active list and k_phase1's per-slot source, so no load waits on another's result
  const int32_t j = v.act[e];
  const int32_t se = a.src_e[e];  // -1: no collision; <= -2: a target whose set waits
  const int32_t s = se >= 0 ? se : -1;
  const ColMeta mj = load_meta(a.meta + j);  // one 16-byte load per column
  const uint8_t f = mj.flags;
  const uint8_t cj = mj.cleared;
  const int32_t nj = kDense ? stored_words(mj.len) : mj.len;
  const int32_t* pj = mj.ptr;
  uint8_t fs = 0, cs = 0;
  int32_t ns = 0;
  const int32_t* ps = nullptr;
  if (s >= 0) {
    const ColMeta ms = load_meta(a.meta + s);
    fs = ms.flags;
    cs = ms.cleared;
    ns = ms.len;
    ps = ms.ptr;
  }
  jb.j = j;
  jb.newpiv = (f & F_NEWPIV) != 0;
  jb.surv = !(f & (F_PROVEN | F_FINAL)) && !cj;
  if (jb.surv) {
    jb.words = nj;
    jb.target = se != -1;
    if (s >= 0) {
      if (v.do_adds && !(fs & F_FINAL) && !cs && (!a.strict || (fs & F_PROVEN))) {
        jb.src = s;
        jb.dense_b = kDense && ns < 0;
        jb.nb = kDense ? stored_words(ns) : ns;
        jb.words += jb.nb;
        jb.B = ps;
      }
    }
  }
  if (jb.newpiv || jb.surv) {
    jb.A = pj;
    jb.na = nj;
    jb.dense_a = kDense && mj.len < 0;
  }
  return jb;
}

// ------------------------------------------------------------------------------------------
// column arithmetic over F2: symmetric difference of two ascending row lists
// ------------------------------------------------------------------------------------------
// merge-path split on diagonal d with ties taken from A first; an equal pair A[x-1] == B[y]
// is kept on the same side of the split so that cancellations never straddle two lanes
__device__ __forceinline__ void merge_split(const int32_t* __restrict__ A, int na,
                                            const int32_t* __restrict__ B, int nb, int d, int& x,
                                            int& y) {
  int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  x = lo;
  y = d - lo;
  if (x > 0 && y < nb && A[x - 1] == B[y]) y++;
}

// warp-cooperative symmetric difference straight from global memory (used for merges too long
// to stage in shared memory); every lane returns the output length and the last row written
__device__ __forceinline__ int warp_symdiff(const int32_t* __restrict__ A, int na,
                                            const int32_t* __restrict__ B, int nb,
                                            int32_t* __restrict__ dst, int32_t& last) {
  constexpr int K = 4;
  const int lane = lane_id();
  const int N = na + nb;
  int out = 0;
  last = -1;
  for (int base = 0; base < N; base += 32 * K) {
    int d0 = min(base + lane * K, N), d1 = min(base + (lane + 1) * K, N);
    int x0, y0, x1, y1;
    merge_split(A, na, B, nb, d0, x0, y0);
    merge_split(A, na, B, nb, d1, x1, y1);
    int cnt = 0;
    {
      int i = x0, k = y0;
      while (i < x1 || k < y1) {
        if (k >= y1 || (i < x1 && A[i] < B[k])) {
          cnt++;
          i++;
        } else if (i >= x1 || B[k] < A[i]) {
          cnt++;
          k++;
        } else {
          i++;
          k++;
        }
      }
    }
    int incl = warp_incl_sum(cnt);
    int pos = out + incl - cnt;
    int32_t mylast = -1;
    {
      int i = x0, k = y0;
      while (i < x1 || k < y1) {
        if (k >= y1 || (i < x1 && A[i] < B[k])) {
          mylast = A[i++];
          dst[pos++] = mylast;
        } else if (i >= x1 || B[k] < A[i]) {
          mylast = B[k++];
          dst[pos++] = mylast;
        } else {
          i++;
          k++;
        }
      }
    }
    unsigned has = __ballot_sync(0xffffffffu, cnt > 0);
    if (has) last = __shfl_sync(0xffffffffu, mylast, 31 - __clz(has));
    out += __shfl_sync(0xffffffffu, incl, 31);
  }
  return out;
}

// Per-warp shared staging of a batch of the warp's jobs, and per-job bookkeeping (indexed by
// the job's ordinal among the warp's staged jobs). Each staged list (a job's column A, its source
// B) has a span that starts on a 16-byte boundary: its first row lands at the span's start plus
// the list's misalignment in global memory (0-3 words), so whole 16-byte chunks copy it, and the
// word after its last row holds a sentinel (INT32_MAX), so a merge needs no bounds checks. A
// batch fills at most kStage words; kStageSlack more absorb a merge's reads past the last
// sentinel (at most KM + 1 words, KM <= 16).
constexpr int kStage = 1024;
constexpr int kStageSlack = 32;
struct __align__(16) WarpStage {
  int32_t in[kStage + kStageSlack];
  int32_t* jout[32];  // output slot of the job (its reserved words in the next arena)
  int32_t ia[32];     // index in `in` of the job's first row of A (current batch)
  int32_t ib[32];     // index in `in` of the job's first row of B
  int32_t na[32];
  int32_t nb[32];
  int32_t pc[33];     // first merge piece of the job: exclusive prefix of pieces over the jobs
  int32_t jcnt[32];   // output rows of the job so far
  int32_t jlow[32];   // largest output row (new low), -1 if none
};
// Phase II blocks: 128 threads, so a block's barriers wait on 4 warps rather than 8
constexpr int kAddThreads = 128;
constexpr int kAddWarps = kAddThreads / 32;
constexpr size_t kAddSmem = sizeof(WarpStage) * kAddWarps;
// block chunks with shared merge pieces: 64-thread blocks, whose chunk barriers wait on two warps
constexpr int kPieceBlockThreads = 64;
// the default switch to 8-slot warp chunks: fewer active columns than this many per warp of the
// grid. An 8-slot chunk takes about half as long as a 32-slot one, but pays its fixed costs
// (claim, column records, look-back) on a quarter of the columns: it wins once its chunks fit in
// about two waves of the grid's warps, where the 32-slot chunks leave most warps idle
constexpr int kNarrowColsPerWarp = 16;

// merge the staged rows A[x0..x1), B[y0..y1) of one lane's range; equal rows cancel.
// With WRITE, the surviving rows go to dst; returns their count and the last one in *last.
template <bool WRITE>
__device__ __forceinline__ int lane_symdiff(const int32_t* __restrict__ sA, int x0, int x1,
                                            const int32_t* __restrict__ sB, int y0, int y1,
                                            int32_t* __restrict__ dst, int32_t* last) {
  int cnt = 0;
  int32_t va = x0 < x1 ? sA[x0] : INT32_MAX;
  int32_t vb = y0 < y1 ? sB[y0] : INT32_MAX;
  int i = x0, j = y0;
  int32_t v = -1;
  while (i < x1 || j < y1) {
    if (va == vb) {
      ++i;
      ++j;
      va = i < x1 ? sA[i] : INT32_MAX;
      vb = j < y1 ? sB[j] : INT32_MAX;
    } else if (va < vb) {
      v = va;
      if (WRITE) dst[cnt] = v;
      ++cnt;
      ++i;
      va = i < x1 ? sA[i] : INT32_MAX;
    } else {
      v = vb;
      if (WRITE) dst[cnt] = v;
      ++cnt;
      ++j;
      vb = j < y1 ? sB[j] : INT32_MAX;
    }
  }
  if (WRITE) *last = v;
  return cnt;
}

// Symmetric difference of two short sorted columns (na, nb <= S) by one thread: both are loaded
// into registers, padded with INT32_MAX, B reversed so that the 2S values form a bitonic
// sequence, sorted by a bitonic merge network (static indices: no divergence, no local memory);
// equal rows -- one from each column -- end up adjacent and cancel. Returns the output length
// and the last (largest) row written, -1 if none.
template <int S>
__device__ __forceinline__ int reg_symdiff(const int32_t* __restrict__ A, int na,
                                           const int32_t* __restrict__ B, int nb,
                                           int32_t* __restrict__ dst, int32_t& last) {
  int32_t c[2 * S];
#pragma unroll
  for (int i = 0; i < S; i++) c[i] = i < na ? __ldg(A + i) : INT32_MAX;
#pragma unroll
  for (int i = 0; i < S; i++) c[2 * S - 1 - i] = i < nb ? __ldg(B + i) : INT32_MAX;
#pragma unroll
  for (int st = S; st >= 1; st >>= 1) {
#pragma unroll
    for (int i = 0; i < 2 * S; i++) {
      if ((i & st) == 0) {
        const int32_t x = c[i], y = c[i + st];
        c[i] = min(x, y);
        c[i + st] = max(x, y);
      }
    }
  }
  int k = 0;
  last = -1;
#pragma unroll
  for (int i = 0; i < 2 * S; i++) {
    const int32_t v = c[i];
    const bool drop = v == INT32_MAX || (i > 0 && c[i - 1] == v) || (i + 1 < 2 * S && c[i + 1] == v);
    if (!drop) {
      dst[k++] = v;
      last = v;
    }
  }
  return k;
}

constexpr unsigned long long kLookAgg = 1ull << 38, kLookIncl = 2ull << 38;
constexpr unsigned long long kLookFlags = 3ull << 38, kLookVal = (1ull << 38) - 1;

// Decoupled look-back over the chunks before `chunk`: the number of survivors in all earlier
// chunks. A chunk publishes its own count (an aggregate state) as soon as its block scan is
// done and looks back only after its merges, when its predecessors have mostly finished and
// published inclusive prefixes. Each state word holds its value, so no fence is needed; states
// carry the pass number and never need resetting within one reduction. Chunks are claimed in
// order from the work queue, so every predecessor belongs to a running or finished block. A
// wait that runs past its bound records a fault (reported as an error) and counts as zero.
__device__ __forceinline__ unsigned long long look_tag(int32_t pass) {
  return (unsigned long long)(pass & 0xffffff) << 40;
}

__device__ __forceinline__ void look_publish(const RArgs& a, int32_t pass, int64_t chunk,
                                             int64_t agg) {
  atomicExch(a.look + chunk,
             look_tag(pass) | (chunk == 0 ? kLookIncl : kLookAgg) | (unsigned long long)agg);
}

// by one full warp; returns the exclusive prefix of `chunk` and publishes its inclusive one
__device__ __forceinline__ int64_t look_back(const RArgs& a, int32_t pass, int64_t chunk,
                                             int64_t agg) {
  if (chunk == 0) return 0;
  const int lane = lane_id();
  const unsigned long long tag = look_tag(pass);
  const unsigned long long* st = a.look;
  int64_t prefix = 0;
  bool fault = false;
  for (int64_t p = chunk - 1;; p -= 32) {
    const int64_t q = p - lane;
    unsigned long long w = tag | kLookIncl;  // before chunk 0: nothing
    if (q >= 0) {
      for (int it = 0;; it++) {
        w = *(const volatile unsigned long long*)(st + q);
        if ((w >> 40) == (tag >> 40) && (w & kLookFlags)) break;
        if (it > kSpinLimit) {
          fault = true;
          w = tag | kLookIncl;
          break;
        }
        __nanosleep(32);
      }
    }
    const bool incl = (w & kLookFlags) == kLookIncl;
    const unsigned im = __ballot_sync(0xffffffffu, incl);
    const int stop = im ? __ffs(im) - 1 : 32;  // nearest inclusive state
    const int64_t val = lane <= stop ? (int64_t)(w & kLookVal) : 0;
    prefix += __shfl_sync(0xffffffffu, warp_incl_sum(val), 31);
    if (im || p < 32) break;
  }
  if (lane == 0) atomicExch(a.look + chunk, tag | kLookIncl | (unsigned long long)(prefix + agg));
  if (__any_sync(0xffffffffu, fault) && lane == 0) a.ds->fault = 1;
  return prefix;
}

// waits for all of this thread's asynchronous copies (cp_async16)
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned), cached in L2 only
__device__ __forceinline__ void cp_async16(int32_t* smem_dst, const int32_t* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}

// merge-path split of the staged lists A = in[ia..ia+na), B = in[ib..ib+nb) on diagonal d, ties
// taken from A first; an equal pair A[x-1] == B[y] is kept on the same side of the split, so that
// cancellations never straddle two pieces
__device__ __forceinline__ void split_staged(const int32_t* __restrict__ in, int ia, int na,
                                             int ib, int nb, int d, int& x, int& y) {
  int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (in[ia + mid] <= in[ib + d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  x = lo;
  y = d - lo;
  if (x > 0 && y < nb && in[ia + x - 1] == in[ib + y]) y++;
}

// Merge rounds over the pieces [P0, P1) of one batch: a job of N staged rows is cut into
// ceil(N / km) pieces of km merge-path positions, and in each round lane l takes piece h0 + l.
// A piece's job is found from a bitmask of the pieces that start a job (each lane of the batch
// owns one job, with its first piece p_first); its end split comes from a binary search, its
// start split from the previous lane (or the previous round). A piece holds at most km + 1 rows
// (a split moves an equal pair to one side). KM > 0 (km = KM): a branch-free merge into
// registers, one shared load per row, the sentinels ending each list; the two copies of a row
// common to both columns come out adjacent and cancel. KM = 0 (any other km): merged
// sequentially, counted first and then merged again to write. Kept rows go to the job's slot
// after the kept rows of its earlier pieces.
template <int KM>
__device__ __forceinline__ void staged_rounds(WarpStage& S_, int P0, int P1, int o0, bool in_batch,
                                              int p_first, int km) {
  constexpr int S = KM > 0 ? KM + 1 : 0;  // register slots: the most rows a piece holds
  const int lane = lane_id();
  const int32_t* __restrict__ in = S_.in;
  int cx = 0, cy = 0;    // end split of the previous round's last piece
  int kprev = o0 - 1;    // job of the piece before the round
  for (int h0 = P0; h0 < P1; h0 += 32) {
    const unsigned start_bit =
        in_batch && p_first >= h0 && p_first < h0 + 32 ? 1u << (p_first - h0) : 0u;
    const unsigned heads = __reduce_or_sync(0xffffffffu, start_bit);
    const int h = h0 + lane;
    const bool valid = h < P1;
    const unsigned upto = 0xffffffffu >> (31 - lane);  // bits 0..lane
    const int o = kprev + __popc(heads & upto);        // this piece's job
    kprev = __shfl_sync(0xffffffffu, o, 31);
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0, d0 = 0, ia = 0, ib = 0, na = 0, nb = 0;
    if (valid) {
      na = S_.na[o];
      nb = S_.nb[o];
      ia = S_.ia[o];
      ib = S_.ib[o];
      d0 = (h - S_.pc[o]) * km;
      const int n = na + nb;
      const int d1 = d0 + km < n ? d0 + km : n;
      if (d1 == n) {
        x1 = na;
        y1 = nb;
      } else {
        split_staged(in, ia, na, ib, nb, d1, x1, y1);
      }
    }
    const int px = __shfl_up_sync(0xffffffffu, x1, 1);
    const int py = __shfl_up_sync(0xffffffffu, y1, 1);
    if (valid && d0 > 0) {  // not a job's first piece: the previous piece is the same job's
      x0 = lane > 0 ? px : cx;
      y0 = lane > 0 ? py : cy;
    }
    cx = __shfl_sync(0xffffffffu, x1, 31);
    cy = __shfl_sync(0xffffffffu, y1, 31);
    const int cnt = valid ? (x1 - x0) + (y1 - y0) : 0;
    unsigned keep = 0;
    int32_t c[S > 0 ? S : 1];
    int kept = 0;
    if constexpr (S > 0) {
      if (valid) {  // branch-free sequential merge; the sentinels end each list
        int i = ia + x0, j = ib + y0;
        int32_t va = in[i], vb = in[j];
#pragma unroll
        for (int t = 0; t < S; t++) {
          const bool ta = va <= vb;
          c[t] = ta ? va : vb;
          if (t + 1 < S) {
            i += ta ? 1 : 0;
            j += ta ? 0 : 1;
            const int32_t nv = in[ta ? i : j];
            va = ta ? nv : va;
            vb = ta ? vb : nv;
          }
        }
        // bit t of eq: row t equals row t + 1 (an equal pair, which cancels); rows past the
        // piece's cnt are masked off, so a pair never reaches past the piece
        const unsigned in_piece = cnt >= 32 ? 0xffffffffu : (1u << cnt) - 1u;
        unsigned eq = 0;
#pragma unroll
        for (int t = 0; t + 1 < S; t++) eq |= (c[t] == c[t + 1] ? 1u : 0u) << t;
        eq &= in_piece >> 1;
        keep = in_piece & ~(eq | (eq << 1));
        kept = __popc(keep);
      }
    } else {
      if (valid) kept = lane_symdiff<false>(in + ia, x0, x1, in + ib, y0, y1, nullptr, nullptr);
    }
    // this piece's place among the kept rows of its job: a scan over the round, restarted at the
    // pieces that start a job (and at lane 0, which continues the previous round's job)
    const unsigned run_heads = __ballot_sync(0xffffffffu, valid && (d0 == 0 || lane == 0));
    const int incl = warp_incl_sum(kept);
    const int rs = 31 - __clz(run_heads & upto);
    const int run_base = __shfl_sync(0xffffffffu, incl - kept, rs);
    const int jc = valid ? S_.jcnt[o] : 0;
    const bool run_last =
        valid && (lane == 31 || ((run_heads >> (lane + 1)) & 1u) || h + 1 >= P1);
    __syncwarp();  // every lane has read its job's count before the run's last lane moves it
    if (kept) {
      int32_t* dst = S_.jout[o] + jc + (incl - kept - run_base);
      int32_t lastv = -1;
      if constexpr (S > 0) {
        int q = 0;
#pragma unroll
        for (int t = 0; t < S; t++) {
          if (keep & (1u << t)) {
            dst[q++] = c[t];
            lastv = c[t];
          }
        }
      } else {
        lane_symdiff<true>(in + ia, x0, x1, in + ib, y0, y1, dst, &lastv);
      }
      atomicMax(&S_.jlow[o], lastv);
    }
    if (run_last) S_.jcnt[o] = jc + (incl - run_base);
    __syncwarp();
  }
}

// One job merged by its own lane, sequentially from the staged lists (the sentinels end each
// list), straight into its slot: a row equal to the one before it cancels that one, so the two
// copies of a row common to both columns never reach the slot. Returns the output length; the
// last row written (the new low) goes to *last, -1 if none.
__device__ __forceinline__ int lane_merge_job(const int32_t* __restrict__ in, int ia, int ib, int n,
                                              int32_t* __restrict__ dst, int32_t* last) {
  int i = ia, j = ib, q = 0;
  int32_t va = in[i], vb = in[j];
  int32_t p = -1, w = -1;
  bool held = false;  // p is a merged row not written yet (it may still cancel)
  for (int t = 0; t < n; t++) {
    const bool ta = va <= vb;
    const int32_t v = ta ? va : vb;
    i += ta ? 1 : 0;
    j += ta ? 0 : 1;
    const int32_t nv = in[ta ? i : j];
    va = ta ? nv : va;
    vb = ta ? vb : nv;
    if (held && v == p) {
      held = false;
    } else {
      if (held) {
        dst[q++] = p;
        w = p;
      }
      p = v;
      held = true;
    }
  }
  if (held) {
    dst[q++] = p;
    w = p;
  }
  *last = w;
  return q;
}

// A survivor j with low l enters the next pass's left-most-column table (and a new low l is
// marked as seen, for the essential estimate; a low that stays was marked when it appeared): the
// table is built while the pass's additions write the new lows, so no kernel of the next pass
// gathers the lows for it
template <bool kNewLow>
__device__ __forceinline__ void next_tab(const RArgs& a, const PV& v, int32_t l, int32_t j) {
  if (l < 0 || !PH_DCHECK(&a.ds->debug_fault, l < a.rows_end, 1)) return;
  if (v.tab_next[l] > j) atomicMin(&v.tab_next[l], j);
  if (kNewLow && !a.meta[l].low_seen) a.meta[l].low_seen = 1;
}

// Phase II for one chunk of the active list (128 slots of a block, or 32 of a warp). Survivors
// get their place in the next active list from a block (or warp) scan plus the look-back, and
// their rows a slot of the next arena from one atomic per chunk. New pivots are copied to the
// pivot store, one run per warp; survivors (with or without an addition) are merged in
// registers (short columns, one thread per job) or staged in shared memory and merged, each job
// by its own lane (short jobs) or by a merge path over the batch's jobs cut into pieces of km
// positions (8 unless ph_opts.merge_items says otherwise); merges longer than the staging
// bound run from global memory; bit-packed jobs run one at a time by the whole warp. Targets
// and zeroed columns are updated in place (no other job reads them this pass); new pivots and
// left-most survivors, which other jobs may be reading as sources, are updated by k_commit.
enum : int {
  kCntTargets, kCntActive, kCntCleared, kCntAdds, kCntXors, kCntCopied, kCntPacked, kNumCnt
};

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// kSlots > 0: the chunk is kSlots (32 or 8) slots of one warp, lanes kSlots.. without a job
// (warp scan, no block barrier); kSlots = 0: kBT slots of the whole block of kBT threads
template <bool kDense, int kSlots, bool kLane, int kBT>
__device__ __forceinline__ void add_chunk(const RArgs& a, const PV& v, int64_t chunk,
                                          WarpStage& S, int64_t* sh, int64_t* s_prefix,
                                          unsigned long long* s_cnt) {
  constexpr bool kWarp = kSlots > 0;
  const int lane = lane_id();
  const int64_t e = !kWarp         ? chunk * kBT + threadIdx.x
                    : kSlots == 32 ? chunk * 32 + lane
                                   : (lane < kSlots ? chunk * kSlots + lane : v.n_act);
  Job jb = job_of<kDense>(a, v, e);
  const int32_t pass = a.ds->pass;
  int64_t off, n_surv;
  int rank;
  if constexpr (kWarp) {
    // survivor ranks by ballot, arena words by a warp scan
    const unsigned survm = __ballot_sync(0xffffffffu, jb.surv);
    n_surv = __popc(survm);
    rank = __popc(survm & ((1u << lane) - 1));
    const int64_t w = jb.surv ? jb.words : 0;
    const int64_t wincl = warp_incl_sum(w);
    const int64_t wtot = __shfl_sync(0xffffffffu, wincl, 31);
    unsigned long long wbase = 0;
    if (lane == 0) {
      look_publish(a, pass, chunk, n_surv);
      // the chunk's survivors take one contiguous run of the next arena
      if (wtot) wbase = atomicAdd(&a.ds->arena_used, (unsigned long long)wtot);
    }
    off = (int64_t)__shfl_sync(0xffffffffu, wbase, 0) + wincl - w;
  } else {
    // one block scan gives both the survivor rank (high 16 bits) and the arena words (low 48)
    constexpr int kRankShift = 48;
    constexpr int64_t kWordMask = (int64_t(1) << kRankShift) - 1;
    const int64_t packed = jb.surv ? ((int64_t(1) << kRankShift) | jb.words) : 0;
    int64_t tot;
    const int64_t excl = block_excl_sum<int64_t, kBT / 32>(packed, sh, tot);
    n_surv = tot >> kRankShift;
    if (threadIdx.x == 0) {
      look_publish(a, pass, chunk, n_surv);
      // the chunk's survivors take one contiguous run of the next arena
      s_prefix[1] = (tot & kWordMask) ? (int64_t)atomicAdd(&a.ds->arena_used,
                                                           (unsigned long long)(tot & kWordMask))
                                      : 0;
    }
    __syncthreads();
    off = s_prefix[1] + (excl & kWordMask);
    rank = (int)(excl >> kRankShift);
  }

#ifdef PH_DEBUG
  // the job's slot lies in the arena this pass writes (else the job is dropped and reported)
  if (jb.surv && !PH_DCHECK(&a.ds->debug_fault, off >= 0 && off + jb.words <= v.arena_next_cap, 3)) {
    jb.surv = false;
    jb.newpiv = false;
  }
#endif
  const int32_t* A = jb.A;
  const int32_t* B = jb.B;
  const int na = jb.na, nb = jb.nb;
  int32_t* o_ptr = nullptr;  // the column's new place and length
  int o_len = 0;

  // ---- new pivots: their columns never change again; move them to the pivot store (a
  // bit-packed column moves as its stored words)
  unsigned pmask = __ballot_sync(0xffffffffu, jb.newpiv);
  if (pmask) {  // the warp's new pivots take one run of the pivot store
    const int mine = jb.newpiv ? na : 0;
    const int incl = warp_incl_sum(mine);
    const int ptot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long w0 = 0;
    if (lane == 0) w0 = atomicAdd(&a.ds->piv_used, (unsigned long long)ptot);
    w0 = __shfl_sync(0xffffffffu, w0, 0) + (unsigned long long)(incl - mine);
#ifdef PH_DEBUG
    // the warp's run lies in the pivot store's chunk (else the warp's copies are dropped)
    const bool in_store = PH_DCHECK(&a.ds->debug_fault, (int64_t)(w0 + mine) <= v.piv_cap, 4);
    if (!__all_sync(0xffffffffu, in_store)) pmask = 0;
#endif
    if (jb.newpiv) o_ptr = v.piv_base + w0;
  }
  while (pmask) {
    const int src = __ffs(pmask) - 1;
    pmask &= pmask - 1;
    const int32_t* wA = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)A, src);
    const int wna = __shfl_sync(0xffffffffu, na, src);
    int32_t* dst = (int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)o_ptr, src);
    for (int q = lane; q < wna; q += 32) dst[q] = wA[q];
    if (lane == src) {
      o_ptr = dst;
      o_len = kDense && jb.dense_a ? dense_len(wna) : wna;
    }
  }

  // ---- survivors: every job writes into its own reserved slot of the next arena
  int32_t* slot = jb.surv ? v.arena_next + off : nullptr;
  const int N = jb.surv ? na + nb : 0;
  // short merges: one thread per job, in registers
  // (cls 1: register merge, 3: staged or from global memory). The register path pays off when
  // most of the warp takes it; a few short jobs among long ones would keep the rest of the warp
  // waiting, so they join the staged path instead. One network size serves the whole warp.
  const int need = max(na, nb);
  // cls 4: bit-packed (the column is, or the source is, or the sum exceeds the threshold)
  const bool dense_job =
      kDense && jb.surv &&
      (jb.dense_a || (B != nullptr && (jb.dense_b || goes_dense(a, jb.j, N))));
  // the register network for jobs of up to kRegMax rows per column; the piece kernels keep it
  // small (8), their registers go to the merge pieces
  constexpr int kRegMax = kLane ? 16 : 8;
  int cls = !jb.surv ? 0 : (dense_job ? 4 : (need <= kRegMax ? 1 : 3));
  constexpr int kRegMinJobs = kWarp ? 12 * kSlots / 32 : 12;  // of the warp's slots
  if (__popc(__ballot_sync(0xffffffffu, cls == 1)) < kRegMinJobs && cls == 1) cls = 3;
  const unsigned wneed = __reduce_max_sync(0xffffffffu, cls == 1 ? (unsigned)need : 0u);
  if (cls == 1) {
    int32_t last;
    int len;
    if constexpr (kRegMax == 16) {
      len = wneed <= 4   ? reg_symdiff<4>(A, na, B, nb, slot, last)
            : wneed <= 8 ? reg_symdiff<8>(A, na, B, nb, slot, last)
                         : reg_symdiff<16>(A, na, B, nb, slot, last);
    } else {
      len = wneed <= 4 ? reg_symdiff<4>(A, na, B, nb, slot, last)
                       : reg_symdiff<8>(A, na, B, nb, slot, last);
    }
    o_ptr = slot;
    o_len = len;
    if (B) {
      a.low[jb.j] = last;
      next_tab<true>(a, v, last, jb.j);
    }
  }
  const unsigned smask = __ballot_sync(0xffffffffu, cls == 3);
  if (smask) {
    // longer merges: staged in shared memory, merge path over the concatenated jobs. Each list
    // takes a 16-byte aligned span (its misalignment, its rows, a sentinel, rounded up to 4 words)
    const int ra = (int)(((uintptr_t)A >> 2) & 3u);
    const int rb = B ? (int)(((uintptr_t)B >> 2) & 3u) : 0;
    const int span_a = (ra + na + 1 + 3) & ~3;
    const int span_b = (rb + nb + 1 + 3) & ~3;
    const bool staged = cls == 3 && N <= a.staged_max && span_a + span_b <= kStage;
    const bool big = cls == 3 && !staged;
    const unsigned stmask = __ballot_sync(0xffffffffu, staged);
    const int ord = __popc(stmask & ((1u << lane) - 1u));  // ordinal among the staged jobs
    const int words = staged ? span_a + span_b : 0;
    const int w_ex = warp_incl_sum(words) - words;
    const int km = a.force_km > 0 ? a.force_km : 8;
    const int npc = staged ? (N + km - 1) / km : 0;  // merge pieces of the job
    const int p_first = warp_incl_sum(npc) - npc;
    if (staged) {
      S.jout[ord] = slot;
      S.na[ord] = na;
      S.nb[ord] = nb;
      S.pc[ord] = p_first;
      S.jcnt[ord] = 0;
      S.jlow[ord] = -1;
    }
    __syncwarp();
    unsigned rest = stmask;
    while (rest) {
      // batch: the staged jobs from lane c on whose spans fit together
      const int c = __ffs(rest) - 1;
      const int w0 = __shfl_sync(0xffffffffu, w_ex, c);
      const bool mine = staged && lane >= c && w_ex + words - w0 <= kStage;
      const unsigned bmask = __ballot_sync(0xffffffffu, mine);
      rest &= ~bmask;
      const int o0 = __popc(stmask & ((1u << c) - 1u));
      const int base = w_ex - w0;  // this job's spans in `in`
      if (mine) {
        S.ia[ord] = base + ra;
        S.ib[ord] = base + span_a + rb;
      }
      // stage: 16-byte chunks from the lists' aligned starts (the column stores carry slack
      // after their last column for the rounding); jobs of 16+ chunks by the whole warp,
      // shorter ones by their lane; all copies of the batch are in flight together
      const int ch_a = span_a >> 2;
      const int ch_n = ch_a + (B ? span_b >> 2 : 0);
      const int32_t* ga = A - ra;
      const int32_t* gb = B ? B - rb : nullptr;
      unsigned lmask = __ballot_sync(0xffffffffu, mine && ch_n >= 16);
      while (lmask) {
        const int src = __ffs(lmask) - 1;
        lmask &= lmask - 1;
        const int32_t* wa = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)ga, src);
        const int32_t* wb = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)gb, src);
        const int wca = __shfl_sync(0xffffffffu, ch_a, src);
        const int wcn = __shfl_sync(0xffffffffu, ch_n, src);
        int32_t* d = S.in + __shfl_sync(0xffffffffu, base, src);
        for (int q = lane; q < wcn; q += 32)
          cp_async16(d + 4 * q, q < wca ? wa + 4 * q : wb + 4 * (q - wca));
      }
      if (mine && ch_n < 16) {
        int32_t* d = S.in + base;
        for (int q = 0; q < ch_n; q++) cp_async16(d + 4 * q, q < ch_a ? ga + 4 * q : gb + 4 * (q - ch_a));
      }
      cp_async_wait_all();
      __syncwarp();
      if (mine) {  // the sentinels go after the copies, which may have covered their words
        S.in[base + ra + na] = INT32_MAX;
        S.in[base + span_a + rb + nb] = INT32_MAX;
      }
      __syncwarp();
      if constexpr (kLane) {  // each job by its own lane
        if (mine) {
          int32_t lastv;
          const int len = lane_merge_job(S.in, base + ra, base + span_a + rb, N, slot, &lastv);
          S.jcnt[ord] = len;
          S.jlow[ord] = lastv;
        }
      } else {  // pieces of every job spread over the lanes
        const int P0 = __shfl_sync(0xffffffffu, p_first, c);
        const int P1 = P0 + (int)__reduce_add_sync(0xffffffffu, mine ? (unsigned)npc : 0u);
        switch (km) {
          case 8: staged_rounds<8>(S, P0, P1, o0, mine, p_first, km); break;
          default: staged_rounds<0>(S, P0, P1, o0, mine, p_first, km); break;
        }
      }
      __syncwarp();
    }
    if (staged) {
      o_ptr = slot;
      o_len = S.jcnt[ord];
      if (B) {
        a.low[jb.j] = S.jlow[ord];
        next_tab<true>(a, v, S.jlow[ord], jb.j);
      }
    }
    // merges too long to stage: straight from global memory into their slot
    unsigned bmask = __ballot_sync(0xffffffffu, big);
    while (bmask) {
      const int src = __ffs(bmask) - 1;
      bmask &= bmask - 1;
      const int32_t* wA = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)A, src);
      const int32_t* wB = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)B, src);
      const int wna = __shfl_sync(0xffffffffu, na, src);
      const int wnb = __shfl_sync(0xffffffffu, nb, src);
      int32_t* wd = (int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)slot, src);
      int len;
      int32_t last = -1;
      if (wB) {
        len = warp_symdiff(wA, wna, wB, wnb, wd, last);
      } else {
        for (int q = lane; q < wna; q += 32) wd[q] = wA[q];
        len = wna;
      }
      if (lane == src) {
        if (B) {
          a.low[jb.j] = last;
          next_tab<true>(a, v, last, jb.j);
        }
        o_ptr = wd;
        o_len = len;
      }
    }
  }
  // ---- bit-packed columns, one job at a time by the whole warp
  unsigned dnmask = kDense ? __ballot_sync(0xffffffffu, cls == 4) : 0u;
  while (dnmask) {
    const int src = __ffs(dnmask) - 1;
    dnmask &= dnmask - 1;
    const int32_t* wA = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)A, src);
    const int32_t* wB = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)B, src);
    const int wna = __shfl_sync(0xffffffffu, na, src);
    int32_t* wd = (int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)slot, src);
    const bool wdense_a = __shfl_sync(0xffffffffu, (int)jb.dense_a, src) != 0;
    if (wB == nullptr) {  // a bit-packed column with nothing to add moves as it is
      for (int q = lane; q < wna; q += 32) wd[q] = wA[q];
      if (lane == src) {
        o_ptr = wd;
        o_len = dense_len(wna);
      }
      continue;
    }
    int32_t low, words;
    const int32_t rows = dense_job_warp(a, __shfl_sync(0xffffffffu, jb.j, src), wA, wna, wdense_a,
                                        wB, __shfl_sync(0xffffffffu, nb, src),
                                        __shfl_sync(0xffffffffu, (int)jb.dense_b, src) != 0, wd,
                                        low, words);
    if (lane == src) {
      o_ptr = wd;
      o_len = rows ? dense_len(words) : 0;  // a zero column stores nothing
      a.low[jb.j] = low;
      next_tab<true>(a, v, low, jb.j);
    }
  }
  // ---- the survivors' places in the next active list
  if constexpr (kWarp) {
    const int64_t pre = look_back(a, pass, chunk, n_surv);
    if (jb.surv && PH_DCHECK(&a.ds->debug_fault, pre + rank < v.n_act, 5)) {
      v.act2[pre + rank] = jb.j;
      v.alen2[pre + rank] = o_len;
    }
  } else {
    if (threadIdx.x < 32) {
      const int64_t pre = look_back(a, pass, chunk, n_surv);
      if (threadIdx.x == 0) s_prefix[0] = pre;
    }
    __syncthreads();
    if (jb.surv && PH_DCHECK(&a.ds->debug_fault, s_prefix[0] + rank < v.n_act, 5)) {
      v.act2[s_prefix[0] + rank] = jb.j;
      v.alen2[s_prefix[0] + rank] = o_len;
    }
  }
  // ---- publish: in place for targets and zeroed columns, through k_commit for the others
  if (jb.surv && B == nullptr) next_tab<false>(a, v, a.low[jb.j], jb.j);  // its low stays
  if (jb.j >= 0) {
    if (jb.surv && jb.target) {
      a.meta[jb.j].ptr = o_ptr;
      a.meta[jb.j].len = o_len;
    } else if (!jb.surv && !jb.newpiv) {
      a.meta[jb.j].flags |= F_FINAL;
      a.low[jb.j] = -1;
      a.meta[jb.j].len = 0;
    }
  }
  const bool defer = jb.newpiv || (jb.surv && !jb.target);
  if (defer) {
    a.nxt_ptr[e] = o_ptr;
    a.nxt_len[e] = o_len;
  }
  const unsigned dmask = __ballot_sync(0xffffffffu, defer);
  if (dmask) {
    int d0 = 0;
    if (lane == __ffs(dmask) - 1) d0 = atomicAdd(&a.ds->n_deferred, __popc(dmask));
    d0 = __shfl_sync(0xffffffffu, d0, __ffs(dmask) - 1);
    if (defer) a.dlist[d0 + __popc(dmask & ((1u << lane) - 1))] = (int32_t)e;
  }
  // ---- counters, per warp into the block's shared totals
  const int n_tgt = __popc(__ballot_sync(0xffffffffu, jb.target));
  if (lane == 0 && n_tgt) atomicAdd(&s_cnt[kCntTargets], (unsigned long long)n_tgt);
  if (v.stats) {
    const bool add = jb.surv && B != nullptr;
    const bool copy = jb.newpiv || (jb.surv && B == nullptr);
    const int n_act = __popc(__ballot_sync(0xffffffffu, jb.j >= 0));
    const int n_clr = __popc(__ballot_sync(0xffffffffu, jb.j >= 0 && a.meta[jb.j].cleared));
    const int n_add = __popc(__ballot_sync(0xffffffffu, add));
    const int n_pk = kDense ? __popc(__ballot_sync(0xffffffffu, add && cls == 4)) : 0;
    // row counts: a bit-packed column keeps its own in its header
    const int ra = kDense && jb.dense_a ? A[0] : na;
    const int64_t xr = warp_sum64(
        add ? (ra + (kDense && jb.dense_b ? B[0] : nb) + (kDense && o_len < 0 ? o_ptr[0] : o_len)) / 2
            : 0);
    const int64_t cp = warp_sum64(copy ? ra : 0);
    if (lane == 0) {
      atomicAdd(&s_cnt[kCntActive], (unsigned long long)n_act);
      atomicAdd(&s_cnt[kCntCleared], (unsigned long long)n_clr);
      atomicAdd(&s_cnt[kCntAdds], (unsigned long long)n_add);
      atomicAdd(&s_cnt[kCntXors], (unsigned long long)xr);
      atomicAdd(&s_cnt[kCntCopied], (unsigned long long)cp);
      if (n_pk) atomicAdd(&s_cnt[kCntPacked], (unsigned long long)n_pk);
    }
  }
}

// kDense: the pass may meet bit-packed columns or convert some; the row-list variant carries none
// of it. kSlots: chunks of kSlots (32 or 8) slots claimed by single warps, 0: chunks of 128 slots
// claimed by blocks. kLane: each staged job merged by its own lane (short columns), else merge
// pieces spread over the lanes. The host picks the variant from DevState::dense_on, warp_on,
// narrow_on and lane_on (a separate graph for each).
template <bool kDense, int kSlots, bool kLane, int kBT = kAddThreads>
__global__ void __launch_bounds__(kBT, 1024 / kBT) k_add(RArgs a) {
  constexpr bool kWarp = kSlots > 0;
  __shared__ int64_t sh[kBT / 32 + 1];
  __shared__ int64_t s_chunk;
  __shared__ int64_t s_prefix[2];
  __shared__ unsigned long long s_cnt[kNumCnt];
  __shared__ PV s_v;  // per-pass values from shared memory rather than held in registers
  extern __shared__ __align__(16) unsigned char add_smem[];
  pdl_wait();
  pdl_trigger();
  if (a.ds->status != ST_RUN) return;
  if (threadIdx.x == 0) s_v = pass_view(a.ds);
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ds->chunk_slots = kWarp ? kSlots : kBT;
  const PV& v = s_v;
  WarpStage& S = reinterpret_cast<WarpStage*>(add_smem)[threadIdx.x >> 5];
  if (threadIdx.x < kNumCnt) s_cnt[threadIdx.x] = 0;
  if constexpr (kWarp) {
    __syncthreads();  // publishes s_v and the zeroed counters
    const int64_t nchunks = (v.n_act + kSlots - 1) / kSlots;
    for (;;) {  // device work queue of kSlots-slot chunks, claimed in order by whole warps
      unsigned int chunk = 0;
      if (lane_id() == 0) chunk = atomicAdd(&a.ds->queue, 1u);
      chunk = __shfl_sync(0xffffffffu, chunk, 0);
      if ((int64_t)chunk >= nchunks) break;
      add_chunk<kDense, kSlots, kLane, kBT>(a, v, chunk, S, sh, s_prefix, s_cnt);
    }
    __syncthreads();
  } else {
    for (;;) {  // device work queue of 128-slot chunks, claimed in order
      if (threadIdx.x == 0) s_chunk = atomicAdd(&a.ds->queue, 1u);
      __syncthreads();  // also publishes s_v, written by thread 0 before the loop
      const int64_t chunk = s_chunk;
      const int64_t nchunks = (v.n_act + kBT - 1) / kBT;
      __syncthreads();
      if (chunk >= nchunks) break;
      add_chunk<kDense, 0, kLane, kBT>(a, v, chunk, S, sh, s_prefix, s_cnt);
    }
  }
  if (threadIdx.x == 0 && s_cnt[kCntTargets]) atomicAdd(&a.ds->totals[1], s_cnt[kCntTargets]);
  if (v.stats && threadIdx.x == 0) {
    const int idx[kNumCnt] = {PH_PS_TARGETS, PH_PS_ACTIVE, PH_PS_CLEARED,
                              PH_PS_ADDS,    PH_PS_XORS,   PH_PS_COPIED, PH_PS_PACKED};
    for (int i = 0; i < kNumCnt; i++)
      if (s_cnt[i]) atomicAdd((unsigned long long*)&v.stats[idx[i]], s_cnt[i]);
  }
}

// |E^l| after this pass's marks (per-pass counter; only with collect_stats)
__global__ void k_ess_count(RArgs a, int64_t m) {
  __shared__ int64_t sh[kWarps + 1];
  pdl_wait();
  pdl_trigger();
  if (a.ds->status != ST_RUN) return;
  int64_t n = 0;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x)
    n += in_essential_estimate(load_meta(a.meta + x), a.beta[x], a.owner[x]);
  int64_t tot;
  block_excl_sum<int64_t>(n, sh, tot);
  if (threadIdx.x == 0 && tot)
    atomicAdd((unsigned long long*)&a.ds->stats[(int64_t)a.ds->pass * PH_PS_N + PH_PS_ESS_EST],
              (unsigned long long)tot);
}

// E^l of the ids [lo, hi) (one dimension of one cloud), as bytes at their filtration index
__global__ void k_ess_flags(int64_t lo, int64_t hi, const ColMeta* __restrict__ meta,
                            const int32_t* __restrict__ beta, const int32_t* __restrict__ owner,
                            const int64_t* __restrict__ gidx, int64_t n, uint8_t* out,
                            int32_t* bad) {
  for (int64_t x = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < hi;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = gidx[x];
    if (g < 0 || g >= n) {
      *bad = 1;
      continue;
    }
    out[g] = in_essential_estimate(load_meta(meta + x), beta[x], owner[x]) ? 1 : 0;
  }
}

// the deferred column updates: new pivots (now in the pivot store) and left-most survivors
__device__ void end_of_pass(const RArgs& a, cudaGraphConditionalHandle cond, int in_graph);

// the counters a pass accumulates, cleared for the next one
__host__ __device__ inline void reset_counters(DevState* ds) {
  ds->bound_words = 0;
  ds->bound_piv = 0;
  ds->queue = 0;
  ds->tile_queue = 0;
  ds->arena_used = 0;
  ds->n_deferred = 0;
  ds->totals[0] = ds->totals[1] = 0;
}

// the deferred column updates and the next pass's row state, then (last block) the end of the
// pass and the reset of the per-pass counters. A pass stopped for space (ST_HOST) continues at
// Phase II on the row state it had, so neither is touched then (the host resets the counters).
__global__ void k_commit(RArgs a, cudaGraphConditionalHandle cond, int in_graph) {
  pdl_wait();
  DevState* ds = a.ds;
  const bool run = ds->status == ST_RUN;
  const int32_t p = ds->pass;
  const int64_t n = run ? (int64_t)ds->n_deferred : 0;
  if (n > 0) {
    const PV v = pass_view(ds);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      const int32_t e = a.dlist[i];
      const int32_t j = v.act[e];
      a.meta[j].ptr = a.nxt_ptr[e];
      a.meta[j].len = a.nxt_len[e];
      a.meta[j].flags &= (uint8_t)~F_NEWPIV;
    }
  }
  if (run) rows_of_pass(a, p + 1);
  if (last_block(&ds->blocks_done, gridDim.x)) {
    if (run) rows_of_pass_last(a, p + 1);
    if (threadIdx.x == 0) {
      ds->blocks_done = 0;
      end_of_pass(a, cond, in_graph);
      if (run) reset_counters(ds);
    }
  }
}

// the device's global timer, in ns
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_clock_start(DevState* ds) { ds->t_start = global_ns(); }

// end of a pass: the next active list, convergence (no target left), the pass cap, the time
// bound, and the graph's loop condition
__device__ void end_of_pass(const RArgs& a, cudaGraphConditionalHandle cond, int in_graph) {
  DevState* ds = a.ds;
  if (ds->status == ST_RUN && (ds->fault || ds->debug_fault)) ds->status = ST_FAULT;
  const bool to_dense = ds->dense_want && !ds->dense_on;
  if (to_dense) ds->dense_on = 1;
  if (ds->status == ST_RUN) {
    const int32_t p = ds->pass;
    // the survivors of the pass: the inclusive prefix the last chunk published in its look-back
    // (anything but an inclusive state of this pass is an internal error)
    const int64_t nch = (ds->n_act + ds->chunk_slots - 1) / ds->chunk_slots;
    int64_t n_surv = 0;
    if (nch > 0) {
      const unsigned long long w = *(const volatile unsigned long long*)(a.look + nch - 1);
      if ((w >> 40) != (look_tag(p) >> 40) || (w & kLookFlags) != kLookIncl) {
        ds->status = ST_FAULT;
        if (in_graph) cudaGraphSetConditional(cond, 0u);
        return;
      }
      n_surv = (int64_t)(w & kLookVal);
    }
    ds->n_act = n_surv;
    int32_t* t = ds->act;
    ds->act = ds->act2;
    ds->act2 = t;
    t = ds->alen;
    ds->alen = ds->alen2;
    ds->alen2 = t;
    if (ds->totals[1] == 0) {
      ds->status = ST_DONE;
      ds->passes = p;
    } else if (p >= ds->max_passes) {
      ds->status = ST_CAPPED;
      ds->passes = p;
    } else {
      ds->pass = p + 1;
      // ... and only once the jobs are long (mean arena words per survivor), where warps of one
      // block would otherwise wait on each other's merges
      const bool to_warp = !ds->warp_on && ds->n_act < ds->warp_below &&
                           ds->arena_used >= (unsigned long long)ds->warp_words * n_surv;
      if (to_warp) ds->warp_on = 1;
      // merge pieces over the lanes once the jobs are long enough to share them out
      const bool to_pieces =
          ds->lane_on && ds->arena_used >= (unsigned long long)ds->lane_words * n_surv;
      if (to_pieces) ds->lane_on = 0;
      // 8-slot warp chunks once the active list is short
      const bool to_narrow =
          ds->warp_on && !ds->lane_on && !ds->narrow_on && n_surv < ds->narrow_below;
      if (to_narrow) ds->narrow_on = 1;
      // the pass is complete, so a later call can resume from the next one
      if (global_ns() - ds->t_start > ds->t_limit) ds->status = ST_TIMEOUT;
      else if (to_dense || to_warp || to_pieces || to_narrow) ds->status = ST_SWITCH;
      // counter rows for the next pass: its first kernel writes them before any capacity check
      if (ds->status != ST_TIMEOUT && ds->stats && ds->pass >= ds->stats_rows) {
        ds->host_reason = 4;
        ds->status = ST_HOST;
      }
    }
  }
  if (in_graph) cudaGraphSetConditional(cond, ds->status == ST_RUN ? 1u : 0u);
}

// ------------------------------------------------------------------------------------------
// set-up and host orchestration
// ------------------------------------------------------------------------------------------
struct InitLayout {
  int64_t dimoff[kMaxDim + 2];
  int64_t rowbase[kMaxDim + 2];
  int maxd;
};

// the boundary matrix of a simplicial complex: a column of dimension d > 0 has d + 1 rows,
// stored in id order from rowbase[d]
// col_off: the columns of a loaded matrix (any length); null: d + 1 rows at a fixed stride
__global__ void k_reduce_init(int64_t m, InitLayout L, int32_t* rows0,
                              const int64_t* __restrict__ col_off, ColMeta* meta, int32_t* low,
                              int32_t* act, int32_t* alen, int32_t* owner, int32_t* tab0) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    int d = 0;
    while (d < L.maxd && x >= L.dimoff[d + 1]) d++;
    int32_t* c = col_off ? rows0 + col_off[x]
                         : rows0 + L.rowbase[d] + (int64_t)(d > 0 ? d + 1 : 0) * (x - L.dimoff[d]);
    const int32_t n = col_off ? (int32_t)(col_off[x + 1] - col_off[x]) : (d > 0 ? d + 1 : 0);
    ColMeta mx;
    mx.ptr = c;
    mx.len = n;
    mx.flags = 0;
    mx.cleared = 0;
    mx.low_seen = 0;
    mx.spare = 0;
    meta[x] = mx;
    low[x] = n > 0 ? c[n - 1] : -1;  // largest row of the unreduced column
    act[x] = (int32_t)x;
    alen[x] = n;
    owner[x] = -1;
    tab0[x] = INT32_MAX;  // the first pass's table before its atomics: no pivot yet
  }
}

static RArgs make_args(ph_ctx* ctx) {
  ReduceState& rs = ctx->rs;
  RArgs a{};
  a.ds = static_cast<DevState*>(rs.dstate);
  a.low = ctx->low;
  a.beta = ctx->beta;
  a.meta = static_cast<ColMeta*>(rs.meta);
  a.nxt_ptr = rs.nxt_ptr;
  a.nxt_len = rs.nxt_len;
  a.owner = rs.owner;
  a.first_unp = rs.first_unp;
  a.seg = ctx->seg;
  a.rows_end = ctx->dimoff[ctx->max_dim];
  a.nseg = (int)ctx->seg_start.size() - 1;
  a.nc = ctx->n_clouds;
  a.strict = ctx->opts.strict_phase2;
  a.cor10 = ctx->opts.use_cor10;
  a.tile_st = static_cast<unsigned long long*>(rs.tiles);
  a.look = static_cast<unsigned long long*>(rs.look);
  a.dlist = static_cast<int32_t*>(rs.dlist);
  a.src_e = static_cast<int32_t*>(rs.src_e);
  a.predict = ctx->opts.predict_pairs ? 1 : 0;
  a.unp_bits = rs.unp_bits;
  a.unp_words = rs.unp_words;
  a.pred = rs.pred;
  a.staged_max = ctx->opts.staged_merge_max > 0 ? std::min(ctx->opts.staged_merge_max, kStage)
                                                 : kStage;
  a.force_km = std::max(0, std::min(ctx->opts.merge_items, 64));
  a.set_n = rs.set_n;
  a.set_neg = rs.set_neg;
  a.set_on = rs.set_on;
  // bit-packed columns: per column dimension the smallest threshold over its row segments
  a.dense_mode = ctx->opts.dense_threshold;
  a.seg_start = ctx->d_seg_start;
  for (int d = 0; d <= kMaxDim; d++)
    a.dim_start[d] = (int32_t)(d <= ctx->max_dim ? ctx->dimoff[d] : ctx->m);
  const int64_t t0 = a.dense_mode > 0 ? a.dense_mode : 32;
  a.dense_floor = INT32_MAX;
  for (int d = 0; d <= kMaxDim; d++) {
    int64_t mn = INT32_MAX;
    for (int c = 0; a.dense_mode >= 0 && d >= 1 && d <= ctx->max_dim && c < ctx->n_clouds; c++) {
      const int rs = (d - 1) * ctx->n_clouds + c;
      const int64_t n = ctx->seg_start[rs + 1] - ctx->seg_start[rs];
      if (n > 0) mn = std::min<int64_t>(mn, std::max<int64_t>((n + 31) / 32 + kDenseHead, t0));
    }
    a.dense_min[d] = (int32_t)std::min<int64_t>(mn, INT32_MAX);
    a.dense_floor = std::min(a.dense_floor, a.dense_min[d]);
  }
  return a;
}

// the additions kernel a pass runs: 1 = handles bit-packed columns (DevState::dense_on) + 2 = one
// chunk per warp (DevState::warp_on) + 4 = each job merged by its own lane (DevState::lane_on);
// 8 + 1 = bit-packed: 8-slot warp chunks with merge pieces (DevState::narrow_on)
static int add_variant(const DevState& h) {
  if (h.narrow_on) return 8 + (h.dense_on ? 1 : 0);
  return (h.dense_on ? 1 : 0) + (h.warp_on ? 2 : 0) + (h.lane_on ? 4 : 0);
}

// grid of the persistent additions kernel: add_blocks_per_sm units of two 128-thread blocks per
// SM, no more blocks than the largest active list (all m columns) can use
static unsigned add_grid_of(const ph_ctx* ctx) {
  const int64_t m = std::max<int64_t>(ctx->m, 1);
  const int bps = ctx->opts.add_blocks_per_sm > 0 ? std::min(ctx->opts.add_blocks_per_sm, 4) : 4;
  const int64_t full = (int64_t)ctx->num_sms * bps * (kThreads / kAddThreads);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(full, (m + kAddThreads - 1) / kAddThreads));
}

// launches one pass kernel; pdl: the kernel may start while the kernel before it in the stream
// drains (programmatic dependent launch; the kernel waits in pdl_wait)
constexpr bool kUsePdl = true;
template <typename... KArgs, typename... Args>
static void launch_k(ph_ctx* ctx, bool pdl, void (*kern)(KArgs...), unsigned grid, unsigned block,
                     size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl && kUsePdl ? 1 : 0;
  ctx->launches++;
  PH_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

// the kernels of one pass, in order; grids are fixed (persistent blocks loop over the work).
// The pass's first kernel (Phase I and the marks), then the rest: a pass stopped for more space
// after its marks continues with the rest alone (launch_pass_rest)
// variant: the additions kernel (add_variant)
static unsigned pass_blocks(ph_ctx* ctx, int64_t full, int64_t per_block) {
  // the full machine for large complexes, no more blocks than the largest active list (all m
  // columns) can use for small ones, so a small complex's pass costs little
  const int64_t m = std::max<int64_t>(ctx->m, 1);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(full, (m + per_block - 1) / per_block));
}

static void launch_pass_rest(ph_ctx* ctx, const RArgs& a, cudaGraphConditionalHandle cond,
                             bool in_graph, int variant, bool time_add, cudaStream_t st) {
  ReduceState& rs = ctx->rs;
  const int sms = ctx->num_sms;
  auto blocks = [&](int64_t full, int64_t per_block) { return pass_blocks(ctx, full, per_block); };
  if (ctx->opts.collect_stats)
    launch_k(ctx, true, k_ess_count, (unsigned)sms * 4, kThreads, 0, st, a, ctx->m);
  if (ctx->opts.phase2_sets > 0 && a.rows_end > 0) {  // host-driven loop only
    const int64_t rows = a.rows_end;
    int bits = 1;
    while (bits < 31 && (int64_t(1) << bits) <= ctx->m) bits++;
    PH_CUDA(cudaMemsetAsync(rs.set_n, 0, (size_t)rows * sizeof(int32_t), st));
    PH_CUDA(cudaMemsetAsync(rs.set_neg, 0, (size_t)rows * sizeof(int32_t), st));
    k_set_count<<<blocks(sms * 8, kThreads), kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
    uint64_t* key = rs.set_key;
    uint64_t* row = rs.set_key + rows;
    k_set_tiekeys<<<grid_for(ctx, rows, kThreads), kThreads, 0, st>>>(a, ctx->gidx, key, row);
    PH_CHECK_LAUNCH();
    radix_sort_u64(ctx, key, row, rows, 0, bits, rs.set_key + 2 * rows, rs.set_key + 3 * rows);
    k_set_keys<<<grid_for(ctx, rows, kThreads), kThreads, 0, st>>>(
        a, ctx->opts.phase2_priority, bits, key, row);
    PH_CHECK_LAUNCH();
    radix_sort_u64(ctx, key, row, rows, 0, ctx->opts.phase2_priority == 1 ? 2 * bits : bits,
                   rs.set_key + 2 * rows, rs.set_key + 3 * rows);
    const int64_t p = std::min<int64_t>(ctx->opts.phase2_sets, rows);
    k_set_select<<<grid_for(ctx, p, kThreads), kThreads, 0, st>>>(a, p, row);
    PH_CHECK_LAUNCH();
    k_set_apply<<<blocks(sms * 8, kThreads), kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
  }
  if (time_add) {
    cudaEvent_t e0, e1;
    PH_CUDA(cudaEventCreate(&e0));
    PH_CUDA(cudaEventCreate(&e1));
    rs.ev.push_back(e0);
    rs.ev.push_back(e1);
    PH_CUDA(cudaEventRecord(e0, st));
  }
  static void (*const add_kernels[ReduceState::kAddVariants])(RArgs) = {
      k_add<false, 0, false, kPieceBlockThreads>, k_add<true, 0, false, kPieceBlockThreads>,
      k_add<false, 32, false>,
      k_add<true, 32, false>,  k_add<false, 0, true>, k_add<true, 0, true>,
      k_add<false, 32, true>,  k_add<true, 32, true>, k_add<false, 8, false>,
      k_add<true, 8, false>};
  // (an event recorded between two kernels needs the first one complete: no early start then)
  // block chunks with merge pieces (variants 0, 1) in smaller blocks, as many warps per SM
  const int bt = variant <= 1 ? kPieceBlockThreads : kAddThreads;
  launch_k(ctx, !time_add, add_kernels[variant], add_grid_of(ctx) * (kAddThreads / bt), bt,
           sizeof(WarpStage) * (bt / 32), st, a);
  if (time_add) PH_CUDA(cudaEventRecord(rs.ev.back(), st));
  launch_k(ctx, !time_add, k_commit, blocks(sms * 2, kThreads), kThreads, 0, st, a, cond,
           in_graph ? 1 : 0);
}

static void launch_pass(ph_ctx* ctx, const RArgs& a, cudaGraphConditionalHandle cond,
                        bool in_graph, int variant, bool time_add, cudaStream_t st) {
  launch_k(ctx, true, k_phase1, pass_blocks(ctx, ctx->num_sms * 8, kFTile), kThreads, 0, st, a);
  launch_pass_rest(ctx, a, cond, in_graph, variant, time_add, st);
}

// the new buffer is taken before the old one goes, so a failed allocation (PH_ERR_ALLOC)
// leaves the store, and the device state that points into it, as it was: a later call resumes
static void grow_store(ph_ctx* ctx, ColStore& s, int64_t need_words) {
  if (need_words <= s.cap) return;
  const int64_t cap = std::max<int64_t>(2 * need_words, 1 << 20);  // doubling: few regrowth stops
  int32_t* p = alloc_n<int32_t>(ctx, cap + kColSlack);
  if (s.p) ctx->dfree(s.p);
  s.p = p;
  s.cap = cap;
}

void reduce_init(ph_ctx* ctx) {
  free_reduce_state(ctx);  // whatever an earlier, failed initialisation left
  // Phase I's tile states carry a (cloud, dimension) segment in 23 bits
  PH_REQUIRE((int64_t)ctx->seg_start.size() - 1 < (1 << 23), PH_ERR_CAPACITY,
             "at most 8,388,607 (cloud, dimension) segments per reduction");
  ReduceState& rs = ctx->rs;
  cudaStream_t st = ctx->stream;
  const int64_t m = ctx->m;
  rs.act = alloc_n<int32_t>(ctx, m);
  rs.act2 = alloc_n<int32_t>(ctx, m);
  rs.alen = alloc_n<int32_t>(ctx, m);
  rs.alen2 = alloc_n<int32_t>(ctx, m);
  rs.act_cap = m;
  rs.meta = alloc_n<ColMeta>(ctx, m);
  rs.nxt_ptr = alloc_n<int32_t*>(ctx, m);
  rs.nxt_len = alloc_n<int32_t>(ctx, m);
  rs.owner = alloc_n<int32_t>(ctx, m);
  rs.tab = alloc_n<int32_t>(ctx, 2 * std::max<int64_t>(m, 1));  // two alternating tables
  int nseg = (int)ctx->seg_start.size() - 1;
  rs.first_unp = alloc_n<int32_t>(ctx, 2 * nseg);  // two copies, alternating between passes
  PH_CUDA(cudaMemsetAsync(rs.first_unp, 0x7f, 2 * nseg * sizeof(int32_t), st));  // above every id
  const int64_t ntiles = (m + kFTile - 1) / kFTile;
  rs.tiles_bytes = (ntiles + 1) * sizeof(unsigned long long);
  rs.tiles = ctx->dalloc(rs.tiles_bytes);
  PH_CUDA(cudaMemsetAsync(rs.tiles, 0, rs.tiles_bytes, st));  // no state published yet
  const int64_t nchunks = (m + 7) / 8 + 1;  // chunks of any shape (8 slots or more)
  rs.look = alloc_n<unsigned long long>(ctx, nchunks);
  PH_CUDA(cudaMemsetAsync(rs.look, 0, nchunks * sizeof(unsigned long long), st));
  rs.dlist = alloc_n<int32_t>(ctx, m);
  rs.src_e = alloc_n<int32_t>(ctx, m);
  if (ctx->opts.predict_pairs) {
    const int64_t rows = ctx->dimoff[ctx->max_dim];
    const int64_t nwords = (rows + 31) / 32;
    rs.unp_bits = alloc_n<uint32_t>(ctx, nwords + 1);
    rs.unp_words = alloc_n<int32_t>(ctx, nwords + 1);
    rs.pred = alloc_n<int32_t>(ctx, m);
    PH_CUDA(cudaMemsetAsync(rs.pred, 0xff, (size_t)m * sizeof(int32_t), st));
  }
  if (ctx->opts.phase2_sets > 0) {
    const int64_t rows = std::max<int64_t>(ctx->dimoff[ctx->max_dim], 1);
    rs.set_n = alloc_n<int32_t>(ctx, rows);
    rs.set_neg = alloc_n<int32_t>(ctx, rows);
    rs.set_on = alloc_n<uint8_t>(ctx, rows);
    rs.set_key = alloc_n<uint64_t>(ctx, 4 * rows);
  }
  rs.dstate = ctx->dalloc(sizeof(DevState));
  PH_CUDA(cudaMallocHost(&rs.hstate, sizeof(DevState)));
  rs.h_stats.clear();
  InitLayout L{};
  L.maxd = ctx->max_dim;
  for (int d = 0; d <= ctx->max_dim + 1; d++) L.dimoff[d] = ctx->dimoff[d];
  int64_t rb = 0;
  for (int d = 0; d <= ctx->max_dim; d++) {
    L.rowbase[d] = rb;
    rb += (d > 0 ? d + 1 : 0) * (ctx->dimoff[d + 1] - ctx->dimoff[d]);
  }
  k_reduce_init<<<grid_for(ctx, m, kThreads), kThreads, 0, st>>>(
      m, L, ctx->rows0, ctx->col_off, static_cast<ColMeta*>(rs.meta), ctx->low, rs.act,
      rs.alen, rs.owner, rs.tab);
  PH_CHECK_LAUNCH();
  // first arenas: pass 0 needs at most the boundary matrix twice over
  // passes 0 and 1 need about the same; later passes less (they grow on demand otherwise)
  const int64_t arena0 = ctx->opts.arena_words > 0 ? ctx->opts.arena_words : 2 * ctx->nnz + 1;
  grow_store(ctx, rs.arena[0], arena0);
  grow_store(ctx, rs.arena[1], arena0);
  ColStore c{};
  grow_store(ctx, c, ctx->nnz / 4 + 1);
  rs.pivots.push_back(c);
  if (ctx->opts.collect_stats) {
    rs.stats_rows = 256;
    rs.pass_stats = alloc_n<int64_t>(ctx, (int64_t)rs.stats_rows * PH_PS_N);
    PH_CUDA(cudaMemsetAsync(rs.pass_stats, 0, (size_t)rs.stats_rows * PH_PS_N * 8, st));
  }
  DevState& h = *static_cast<DevState*>(rs.hstate);
  h = DevState{};
  h.act = rs.act;
  h.act2 = rs.act2;
  h.alen = rs.alen;
  h.alen2 = rs.alen2;
  h.n_act = m;
  for (int i = 0; i < 2; i++) {
    h.arena[i] = rs.arena[i].p;
    h.arena_cap[i] = rs.arena[i].cap;
    h.tab[i] = rs.tab + i * std::max<int64_t>(m, 1);
  }
  h.piv_base = c.p;
  h.piv_cap = c.cap;
  h.piv_used = 0;
  h.stats = rs.pass_stats;
  h.stats_rows = rs.stats_rows;
  h.pass = 0;
  h.status = ST_RUN;
  h.warp_below = ctx->opts.warp_chunks_below < 0   ? 0
                 : ctx->opts.warp_chunks_below == 0 ? (int64_t)1 << 22
                                                    : ctx->opts.warp_chunks_below;
  h.warp_words = ctx->opts.warp_chunk_words < 0    ? 0
                 : ctx->opts.warp_chunk_words == 0 ? 40
                                                   : ctx->opts.warp_chunk_words;
  // the first passes' jobs are short: block chunks, unless any job length will do
  h.warp_on = h.warp_words == 0 && m < h.warp_below ? 1 : 0;
  h.lane_words = ctx->opts.lane_merge_words == 0 ? 20 : ctx->opts.lane_merge_words;
  h.lane_on = ctx->opts.lane_merge_words < 0 ? 0 : 1;
  h.narrow_below = ctx->opts.narrow_chunks_below < 0 ? 0
                   : ctx->opts.narrow_chunks_below == 0
                       ? (int64_t)add_grid_of(ctx) * kAddWarps * kNarrowColsPerWarp
                       : ctx->opts.narrow_chunks_below;
  h.narrow_on = 0;
  PH_CUDA(cudaMemcpyAsync(rs.dstate, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  // the first pass's row state and table (the later ones come from the pass before)
  {
    const RArgs a0 = make_args(ctx);
    launch_k(ctx, false, k_rows_first, (unsigned)grid_for(ctx, a0.rows_end, kThreads), kThreads,
             0, st, a0);
    launch_k(ctx, false, k_tab, (unsigned)grid_for(ctx, m, kThreads * kTabItems), kThreads, 0, st,
             a0);
  }
  const void* add_kernels[ReduceState::kAddVariants] = {
      (const void*)k_add<false, 0, false, kPieceBlockThreads>,
      (const void*)k_add<true, 0, false, kPieceBlockThreads>,
      (const void*)k_add<false, 32, false>, (const void*)k_add<true, 32, false>,
      (const void*)k_add<false, 0, true>,   (const void*)k_add<true, 0, true>,
      (const void*)k_add<false, 32, true>,  (const void*)k_add<true, 32, true>,
      (const void*)k_add<false, 8, false>,  (const void*)k_add<true, 8, false>};
  for (const void* f : add_kernels)
    PH_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAddSmem));
  rs.passes = 0;
  rs.init = true;
  rs.done = false;
  rs.status = PH_OK;
}

// grows whatever the stopped pass asked for, in the host mirror h
static void serve_host_request(ph_ctx* ctx, DevState& h) {
  ReduceState& rs = ctx->rs;
  cudaStream_t st = ctx->stream;
  if (h.host_reason & 1) {  // the arena this pass writes into; its contents are dead
    ColStore& s = rs.arena[h.pass & 1];
    grow_store(ctx, s, (int64_t)h.bound_words);
    h.arena[h.pass & 1] = s.p;
    h.arena_cap[h.pass & 1] = s.cap;
  }
  if (h.host_reason & 2) {  // a new pivot chunk; the old ones stay (their columns live there)
    ColStore c{};
    grow_store(ctx, c, std::max<int64_t>(2 * (int64_t)h.bound_piv, ctx->nnz / 4 + 1));
    rs.pivots.push_back(c);
    h.piv_base = c.p;
    h.piv_cap = c.cap;
    h.piv_used = 0;
  }
  if (h.host_reason & 4) {
    int32_t rows = std::max(256, rs.stats_rows * 2);
    while (rows <= h.pass) rows *= 2;
    int64_t* ns = alloc_n<int64_t>(ctx, (int64_t)rows * PH_PS_N);
    PH_CUDA(cudaMemsetAsync(ns, 0, (size_t)rows * PH_PS_N * 8, st));
    PH_CUDA(cudaMemcpyAsync(ns, rs.pass_stats, (size_t)rs.stats_rows * PH_PS_N * 8,
                            cudaMemcpyDeviceToDevice, st));
    ctx->dfree(rs.pass_stats);
    rs.pass_stats = ns;
    rs.stats_rows = rows;
    h.stats = ns;
    h.stats_rows = rows;
  }
  h.host_reason = 0;
  h.status = ST_RUN;
}

// the pass loop as one graph: a conditional while node around one pass, with one of the
// additions kernel variants (see launch_pass)
static void build_graph(ph_ctx* ctx, const RArgs& a, int variant) {
  ReduceState& rs = ctx->rs;
  cudaGraph_t g;
  PH_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  PH_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = cond;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  PH_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  // capture on a private stream (the legacy default stream cannot capture); the graph is
  // then launched on the context's stream
  cudaStream_t cs;
  PH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t ce = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    cudaStreamDestroy(cs);
    cudaGraphDestroy(g);
    PH_CUDA(ce);
  }
  const int64_t counted = ctx->launches;  // captured launches run later, counted per pass
  try {
    launch_pass(ctx, a, cond, true, variant, false, cs);
    ctx->launches = counted;
  } catch (...) {
    cudaStreamEndCapture(cs, &body);
    cudaStreamDestroy(cs);
    cudaGraphDestroy(g);
    throw;
  }
  ce = cudaStreamEndCapture(cs, &body);
  cudaStreamDestroy(cs);
  if (ce != cudaSuccess) cudaGraphDestroy(g);
  PH_CUDA(ce);
  cudaGraphExec_t exec;
  PH_CUDA(cudaGraphInstantiate(&exec, g, 0));
  rs.graph[variant] = g;
  rs.graph_exec[variant] = exec;
}

int reduce_run(ph_ctx* ctx, int32_t max_passes) {
  ReduceState& rs = ctx->rs;
  cudaStream_t st = ctx->stream;
  // the budgeted Phase II ranks its sets with host-sized sort launches: host-driven loop
  const bool use_graph = ctx->opts.use_graph != 0 && ctx->opts.phase2_sets <= 0;
  const bool time_add = ctx->opts.time_kernels != 0 && !use_graph;
  DevState& h = *static_cast<DevState*>(rs.hstate);
  // a resumed reduction continues after the pass that hit the previous cap
  PH_CUDA(cudaMemcpyAsync(&h, rs.dstate, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  PH_CUDA(cudaStreamSynchronize(st));
  if (h.status == ST_CAPPED) {
    h.pass = h.passes + 1;
    h.status = ST_RUN;
  } else if (h.status == ST_TIMEOUT) {  // stopped between two passes
    h.status = ST_RUN;
  }
  if (h.stats && h.pass >= h.stats_rows) {  // counter rows for the first pass of this call
    h.host_reason = 4;
    serve_host_request(ctx, h);
  }
  // every pass proves or zeroes at least one column, so m + 1 passes always suffice
  h.max_passes = max_passes < 0 ? (int32_t)std::min<int64_t>(ctx->m + 1, INT32_MAX) : max_passes;
  h.blocks_done = 0;
  const int64_t limit_ms = ctx->opts.timeout_ms > 0 ? ctx->opts.timeout_ms : 60000;
  h.t_limit = (unsigned long long)limit_ms * 1000000ull;
  PH_CUDA(cudaMemcpyAsync(rs.dstate, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
  k_clock_start<<<1, 1, 0, st>>>(static_cast<DevState*>(rs.dstate));
  PH_CHECK_LAUNCH();
  const RArgs a = make_args(ctx);

  bool rest_only = false;  // a pass stopped for space after its marks continues at Phase II
  for (;;) {
    const int32_t first_pass = h.pass;
    NvtxRange nvtx_range_(use_graph ? "pass loop (graph)" : "pass");
    bool ran_graph = false;
    if (rest_only) {
      rest_only = false;
      launch_pass_rest(ctx, a, 0, false, add_variant(h), time_add, st);
      if (time_add) rs.add_launches++;
    } else if (use_graph) {
      ran_graph = true;
      const int variant = add_variant(h);
      if (!rs.graph_exec[variant]) build_graph(ctx, a, variant);
      PH_CUDA(cudaGraphLaunch(rs.graph_exec[variant], st));
    } else {
      launch_pass(ctx, a, 0, false, add_variant(h), time_add, st);
      if (time_add) rs.add_launches++;
    }
    PH_CUDA(cudaMemcpyAsync(&h, rs.dstate, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    PH_CUDA(cudaStreamSynchronize(st));
    if (ran_graph) {  // kernels per executed pass of the graph's loop
      const int32_t last = (h.status == ST_DONE || h.status == ST_CAPPED) ? h.passes : h.pass;
      const int per_pass = 3 + (ctx->opts.collect_stats ? 1 : 0);
      ctx->launches += per_pass * (int64_t)(last - first_pass + 1);
    }
    if (h.status == ST_RUN) continue;
    if (h.status == ST_SWITCH) {  // the next pass on, with the bit-packing additions kernel
      h.status = ST_RUN;
      PH_CUDA(cudaMemcpyAsync(rs.dstate, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
      continue;
    }
    if (h.status == ST_HOST) {
      if (time_add && rs.ev.size() >= 2) {  // the stopped pass's k_add did no work
        cudaEventDestroy(rs.ev.back());
        rs.ev.pop_back();
        cudaEventDestroy(rs.ev.back());
        rs.ev.pop_back();
        rs.add_launches--;
      }
      // space for Phase II (reasons 1, 2): the pass continues there, its marks made; counter
      // rows (reason 4): asked for between two passes, the next pass runs whole
      rest_only = (h.host_reason & 3) != 0;
      serve_host_request(ctx, h);
      if (rest_only) reset_counters(&h);
      PH_CUDA(cudaMemcpyAsync(rs.dstate, &h, sizeof(DevState), cudaMemcpyHostToDevice, st));
      continue;
    }
    break;
  }
  PH_REQUIRE(h.status != ST_FAULT || h.debug_fault == 0, PH_ERR_CUDA,
             "device bounds check " + std::to_string(h.debug_fault) + " failed (debug build)");
  PH_REQUIRE(h.status != ST_FAULT, PH_ERR_CUDA,
             "a bounded wait in the addition kernel ran out (look-back did not complete)");
  PH_REQUIRE(h.status != ST_TIMEOUT, PH_ERR_TIMEOUT,
             "the pass loop ran past the time bound (ph_opts.timeout_ms)");
  rs.passes = h.passes;
  rs.status = h.status == ST_DONE ? PH_OK : PH_NOT_CONVERGED;
  if (ctx->opts.collect_stats) {
    rs.h_stats.assign((size_t)(rs.passes + 1) * PH_PS_N, 0);
    PH_CUDA(cudaMemcpyAsync(rs.h_stats.data(), rs.pass_stats,
                            rs.h_stats.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  }
  PH_CUDA(cudaStreamSynchronize(st));
  for (size_t i = 0; i + 1 < rs.ev.size(); i += 2) {
    float ms = 0;
    PH_CUDA(cudaEventElapsedTime(&ms, rs.ev[i], rs.ev[i + 1]));
    rs.ms_add += ms;
    rs.add_ms.push_back(ms);
    cudaEventDestroy(rs.ev[i]);
    cudaEventDestroy(rs.ev[i + 1]);
  }
  rs.ev.clear();
  rs.done = true;
  return rs.status;
}

void essential_estimate(ph_ctx* ctx, int32_t cloud, uint8_t* host_out, int64_t n) {
  ReduceState& rs = ctx->rs;
  const int nc = ctx->n_clouds;
  uint8_t* d_out = alloc_n<uint8_t>(ctx, n);
  int32_t* d_bad = alloc_n<int32_t>(ctx, 1);
  PH_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), ctx->stream));
  for (int d = 0; d <= ctx->max_dim; d++) {
    const int64_t lo = ctx->seg_start[d * nc + cloud], hi = ctx->seg_start[d * nc + cloud + 1];
    if (hi <= lo) continue;
    k_ess_flags<<<grid_for(ctx, hi - lo, kThreads), kThreads, 0, ctx->stream>>>(
        lo, hi, static_cast<const ColMeta*>(rs.meta), ctx->beta, rs.owner, ctx->gidx, n, d_out,
        d_bad);
    PH_CHECK_LAUNCH();
  }
  int32_t bad = 0;
  PH_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaMemcpyAsync(host_out, d_out, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->dfree(d_out);
  ctx->dfree(d_bad);
  PH_REQUIRE(bad == 0, PH_ERR_INVALID, "internal error: filtration index out of range");
}

__global__ void k_pred_out(int64_t lo, int64_t hi, const int32_t* __restrict__ pred,
                           const int64_t* __restrict__ gidx, int64_t n, int32_t* out,
                           int32_t* bad) {
  for (int64_t x = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < hi;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = gidx[x];
    if (g < 0 || g >= n) {
      *bad = 1;
      continue;
    }
    const int32_t p = pred[x];
    out[g] = p >= 0 ? (int32_t)gidx[p] : -1;
  }
}

void predicted_lows(ph_ctx* ctx, int32_t cloud, int32_t* host_out, int64_t n) {
  ReduceState& rs = ctx->rs;
  const int nc = ctx->n_clouds;
  int32_t* d_out = alloc_n<int32_t>(ctx, std::max<int64_t>(n, 1));
  int32_t* d_bad = alloc_n<int32_t>(ctx, 1);
  PH_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), ctx->stream));
  for (int d = 0; d <= ctx->max_dim; d++) {
    const int64_t lo = ctx->seg_start[d * nc + cloud], hi = ctx->seg_start[d * nc + cloud + 1];
    if (hi <= lo) continue;
    k_pred_out<<<grid_for(ctx, hi - lo, kThreads), kThreads, 0, ctx->stream>>>(
        lo, hi, rs.pred, ctx->gidx, n, d_out, d_bad);
    PH_CHECK_LAUNCH();
  }
  int32_t bad = 0;
  PH_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaMemcpyAsync(host_out, d_out, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->dfree(d_out);
  ctx->dfree(d_bad);
  PH_REQUIRE(bad == 0, PH_ERR_INVALID, "internal error: filtration index out of range");
}

// ------------------------------------------------------------------------------------------
// the reduced matrix R of one cloud, CSC over its filtration indices
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t col_rows(const ColMeta& mx) {
  return mx.len >= 0 ? mx.len : mx.ptr[0];  // a bit-packed column's header holds its rows
}

__global__ void k_col_counts(int64_t lo, int64_t hi, const ColMeta* __restrict__ meta,
                             const int64_t* __restrict__ gidx, int64_t n, int64_t* cnt,
                             int32_t* bad) {
  for (int64_t x = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < hi;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = gidx[x];
    if (f < 0 || f >= n) {
      *bad = 1;
      continue;
    }
    cnt[f] = col_rows(load_meta(meta + x));
  }
}

// rows as filtration indices of the same cloud, ascending (ids of one dimension and cloud are in
// filtration order); a bitmap is read word by word, bit by bit
__global__ void k_col_rows(int64_t lo, int64_t hi, const ColMeta* __restrict__ meta,
                           const int64_t* __restrict__ gidx, const int32_t* __restrict__ seg,
                           const int64_t* __restrict__ seg_start, int nc,
                           const int64_t* __restrict__ off, int64_t n, int64_t nnz, int32_t* out,
                           int32_t* bad) {
  for (int64_t x = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < hi;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = gidx[x];
    if (f < 0 || f >= n) {
      *bad = 1;
      continue;
    }
    const ColMeta mx = load_meta(meta + x);
    int32_t* o = out + off[f];
    const int64_t room = nnz - off[f];
    int64_t k = 0;
    if (mx.len >= 0) {
      for (int32_t q = 0; q < mx.len && k < room; q++) o[k++] = (int32_t)gidx[mx.ptr[q]];
    } else {
      const int rs = seg[x] - nc;
      const int64_t base = seg_start[rs];
      const int64_t words = (seg_start[rs + 1] - base + 31) / 32;
      const uint32_t* bits = reinterpret_cast<const uint32_t*>(mx.ptr + kDenseHead);
      for (int64_t w = 0; w < words; w++)
        for (uint32_t b = bits[w]; b && k < room; b &= b - 1)
          o[k++] = (int32_t)gidx[base + 32 * w + (__ffs(b) - 1)];
    }
    if (k != col_rows(mx)) *bad = 1;
  }
}

void reduced_columns(ph_ctx* ctx, int32_t cloud, int64_t n, int64_t* colptr, int32_t* rows,
                     int64_t capacity, int64_t* nnz_out) {
  ReduceState& rs = ctx->rs;
  const int nc = ctx->n_clouds;
  const ColMeta* meta = static_cast<const ColMeta*>(rs.meta);
  int64_t* d_off = alloc_n<int64_t>(ctx, n + 1);
  int32_t* d_bad = alloc_n<int32_t>(ctx, 1);
  PH_CUDA(cudaMemsetAsync(d_off, 0, (size_t)(n + 1) * sizeof(int64_t), ctx->stream));
  PH_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), ctx->stream));
  for (int d = 0; d <= ctx->max_dim; d++) {
    const int64_t lo = ctx->seg_start[d * nc + cloud], hi = ctx->seg_start[d * nc + cloud + 1];
    if (hi <= lo) continue;
    k_col_counts<<<grid_for(ctx, hi - lo, kThreads), kThreads, 0, ctx->stream>>>(
        lo, hi, meta, ctx->gidx, n, d_off, d_bad);
    PH_CHECK_LAUNCH();
  }
  excl_scan_i64(ctx, d_off, d_off, n + 1, nullptr);
  PH_CUDA(cudaMemcpyAsync(colptr, d_off, (size_t)(n + 1) * sizeof(int64_t),
                          cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  const int64_t nnz = colptr[n];
  if (nnz_out) *nnz_out = nnz;
  int32_t bad = 0;
  if (rows && nnz <= capacity && nnz > 0) {
    int32_t* d_rows = alloc_n<int32_t>(ctx, nnz);
    for (int d = 0; d <= ctx->max_dim; d++) {
      const int64_t lo = ctx->seg_start[d * nc + cloud], hi = ctx->seg_start[d * nc + cloud + 1];
      if (hi <= lo) continue;
      k_col_rows<<<grid_for(ctx, hi - lo, kThreads), kThreads, 0, ctx->stream>>>(
          lo, hi, meta, ctx->gidx, ctx->seg, ctx->d_seg_start, nc, d_off, n, nnz, d_rows, d_bad);
      PH_CHECK_LAUNCH();
    }
    PH_CUDA(cudaMemcpyAsync(rows, d_rows, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            ctx->stream));
    PH_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    PH_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->dfree(d_rows);
  } else {
    PH_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    PH_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  ctx->dfree(d_off);
  ctx->dfree(d_bad);
  PH_REQUIRE(bad == 0, PH_ERR_INVALID, "internal error: column index out of range");
  PH_REQUIRE(!rows || nnz <= capacity, PH_ERR_CAPACITY,
             "rows holds " + std::to_string(capacity) + " entries, the columns need " +
                 std::to_string(nnz));
}

void free_reduce_state(ph_ctx* ctx) {
  ReduceState& rs = ctx->rs;
  for (int d = 0; d < ReduceState::kAddVariants; d++) {
    if (rs.graph_exec[d]) cudaGraphExecDestroy(rs.graph_exec[d]);
    if (rs.graph[d]) cudaGraphDestroy(rs.graph[d]);
  }
  for (void* p : {(void*)rs.act, (void*)rs.act2, (void*)rs.alen, (void*)rs.alen2, rs.meta,
                  (void*)rs.nxt_ptr, (void*)rs.nxt_len, (void*)rs.owner, (void*)rs.tab,
                  (void*)rs.first_unp, rs.tiles, rs.dstate,
                  rs.look, rs.dlist, rs.src_e, (void*)rs.unp_bits, (void*)rs.unp_words,
                  (void*)rs.pred, (void*)rs.set_n, (void*)rs.set_neg, (void*)rs.set_on,
                  (void*)rs.set_key,
                  (void*)rs.pass_stats})
    ctx->dfree(p);
  for (auto& a : rs.arena) ctx->dfree(a.p);
  for (auto& c : rs.pivots) ctx->dfree(c.p);
  if (rs.hstate) cudaFreeHost(rs.hstate);
  for (auto e : rs.ev) cudaEventDestroy(e);
  rs = ReduceState{};
}

}  // namespace ph
