// Parallel multi-scale reduction (Algorithm 2, Sec. 3.1) on the device.
//
// One pass = one cycle of the outer loop of Algorithm 2. Every decision of a pass is taken from
// the state at its start, so the result of a pass does not depend on thread scheduling:
//   k_tab_init   tab[i] <- owner[i] (proven pivot with low i); first row of each (cloud, dim)
//                that is not known to be paired (for Corollary 10).
//   k_tab        tab[low(j)] <- min j over the active columns (atomicMin): the left-most column
//                with each low, which defines the neighbour sets N(j) (Eq. neighbours).
//   k_p1_tiles / k_p1_top / k_mark
//                Phase I (Algorithm 5) as a segmented exclusive prefix-max over the active
//                columns of each (cloud, dim): P_j = largest low of an earlier colliding column.
//                j is proven if it is left-most for its low and low(j) = beta_j (Thm 5) or
//                low(j) > P_j (Thms 6-7). Empty columns become final; the zero case of
//                Corollary 10 zeroes a column whose candidate rows are all paired. Each new
//                pivot clears column low(j) (Lemma 1).
//   k_s2_tiles / k_s2_top
//                sizes of the surviving columns after this pass's additions (upper bounds).
//   k_add        Phase II: every colliding column l gets column tab[low(l)] added (XOR of two
//                sorted row lists). Sources are left-most, hence never targets, so additions
//                are independent. Survivors are written compactly into the other arena, new
//                pivots move to the pivot store (their columns never change again).
//   k_commit     publishes the new column locations and the next active list.
#include <algorithm>

#include "ph_internal.cuh"

namespace ph {

constexpr int kRItems = 8;
constexpr int kRTile = kThreads * kRItems;

struct RArgs {
  int32_t* act;
  int32_t* act2;
  int64_t n_act;
  int32_t* low;
  const int32_t* beta;
  uint8_t* flags;
  uint8_t* cleared;
  int32_t** cptr;
  int32_t* clen;
  int32_t** nxt_ptr;
  int32_t* nxt_len;
  int32_t* owner;
  int32_t* tab;
  int32_t* first_unp;
  const int32_t* seg;
  int nc;
  int strict;
  int cor10;
  int do_adds;
  SegMax* tile_sm;    // [ntiles] Phase I tile aggregates (scanned in place to prefixes)
  SegMax* chunk_sm;   // [ntiles][kRItems] aggregate of each 256-entry chunk alone
  int64_t* tile_cnt;  // [ntiles][2] survivors, words (scanned in place to prefixes)
  int64_t* tile_aux;  // [ntiles][2] pivot words, targets
  int64_t* chunk_cnt; // [ntiles][kRItems][2] survivors, words of each chunk alone
  int64_t* totals;    // [4] survivors, words, pivot words, targets
  int32_t* arena_next;
  int32_t* piv_base;
  unsigned long long* piv_bump;
  int64_t* stats;  // this pass's counters or nullptr
  int staged_max;  // merges of more rows than this run from global memory
  int force_km;    // > 0: merge-path positions per lane for every warp
};

__device__ __forceinline__ void stat_add(int64_t* stats, int k, int64_t v) {
  // warp-aggregated counter update
  int64_t s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane_id() == 0 && s != 0) atomicAdd((unsigned long long*)&stats[k], (unsigned long long)s);
}

// ------------------------------------------------------------------------------------------
__global__ void k_tab_init(int64_t rows_end, const int32_t* __restrict__ owner,
                           const uint8_t* __restrict__ flags, const int32_t* __restrict__ beta,
                           const int32_t* __restrict__ seg, int32_t* tab, int32_t* first_unp) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < rows_end;
       x += (int64_t)gridDim.x * blockDim.x) {
    int32_t o = owner[x];
    tab[x] = o < 0 ? INT32_MAX : o;
    bool paired = (flags[x] & F_PROVEN) || beta[x] >= 0 || o >= 0;
    if (!paired) atomicMin(&first_unp[seg[x]], (int32_t)x);
  }
}

__global__ void k_tab(RArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n_act;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = a.act[i];
    int32_t l = a.low[j];
    if (l >= 0 && a.tab[l] > j) atomicMin(&a.tab[l], j);
  }
}

// ------------------------------------------------------------------------------------------
// Phase I scan
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ SegMax p1_value(const RArgs& a, int64_t e) {
  if (e >= a.n_act) return SegMax{INT32_MAX, -1};
  int32_t j = a.act[e];
  int32_t l = a.low[j];
  SegMax v;
  v.seg = a.seg[j];
  v.val = (l >= 0 && a.tab[l] != j) ? l : -1;  // low of a colliding column
  return v;
}

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

__global__ void k_p1_tiles(RArgs a) {
  __shared__ SegMax sh[kWarps + 1];
  int64_t tile0 = (int64_t)blockIdx.x * kRTile;
  SegMax carry{-1, -1};
  for (int it = 0; it < kRItems; it++) {
    SegMax v = p1_value(a, tile0 + it * kThreads + threadIdx.x);
    SegMax tot;
    block_scan_segmax(v, SegMax{-1, -1}, sh, tot);  // this chunk alone
    if (threadIdx.x == 0) a.chunk_sm[(int64_t)blockIdx.x * kRItems + it] = tot;
    carry = segmax_combine(carry, tot);
  }
  if (threadIdx.x == 0) a.tile_sm[blockIdx.x] = carry;
}

__global__ void k_p1_top(SegMax* tile_sm, int64_t ntiles) {
  __shared__ SegMax sh[kWarps + 1];
  SegMax carry{-1, -1};
  for (int64_t base = 0; base < ntiles; base += kThreads) {
    int64_t i = base + threadIdx.x;
    SegMax v = i < ntiles ? tile_sm[i] : SegMax{INT32_MAX, -1};
    SegMax tot;
    SegMax ex = block_scan_segmax(v, carry, sh, tot);
    if (i < ntiles) tile_sm[i] = ex;
    carry = tot;
  }
}

// one block per 256-entry chunk; its prefix is the tile's prefix combined with the aggregates
// of the earlier chunks of the same tile
__global__ void k_mark(RArgs a) {
  __shared__ SegMax sh[kWarps + 1];
  const int64_t chunk = blockIdx.x, tile = chunk / kRItems;
  SegMax carry = a.tile_sm[tile];
  for (int64_t c = tile * kRItems; c < chunk; c++) carry = segmax_combine(carry, a.chunk_sm[c]);
  int64_t n_zero = 0, n_piv = 0, n_c10 = 0;
  {
    int64_t e = chunk * kThreads + threadIdx.x;
    SegMax v = p1_value(a, e);
    SegMax tot;
    SegMax pre = block_scan_segmax(v, carry, sh, tot);
    if (e < a.n_act) {
      int32_t j = a.act[e];
      int32_t l = a.low[j];
      uint8_t f = a.flags[j];
      if (l < 0) {
        a.flags[j] = f | F_FINAL;
        n_zero++;
      } else {
        int32_t P = (pre.seg == v.seg) ? pre.val : -1;
        bool leftmost = a.tab[l] == j;
        int32_t b = a.beta[j];
        if (leftmost && (l == b || l > P)) {
          a.flags[j] = f | F_PROVEN | F_NEWPIV;
          a.owner[l] = j;
          a.cleared[l] = 1;  // clearing (Lemma 1): column l is positive and paired with j
          n_piv++;
        } else if (a.cor10 && b < 0 && l < a.first_unp[v.seg - a.nc]) {
          a.flags[j] = f | F_FINAL;  // Corollary 10, zero case
          n_c10++;
        }
      }
    }
  }
  if (a.stats) {
    stat_add(a.stats, PH_PS_ZERO_FINAL, n_zero);
    stat_add(a.stats, PH_PS_NEW_PIVOTS, n_piv);
    stat_add(a.stats, PH_PS_COR10, n_c10);
  }
}

// ------------------------------------------------------------------------------------------
// what happens to an active column in Phase II
// ------------------------------------------------------------------------------------------
struct Job {
  int32_t j;
  int32_t src;    // source column for an addition, -1 if none
  bool surv;      // stays active
  bool newpiv;    // proven this pass: moves to the pivot store
  bool target;    // collides with an earlier column
  int64_t words;  // arena words reserved (survivors only)
};

__device__ __forceinline__ Job job_of(const RArgs& a, int64_t e) {
  Job jb{-1, -1, false, false, false, 0};
  if (e >= a.n_act) return jb;
  int32_t j = a.act[e];
  jb.j = j;
  uint8_t f = a.flags[j];
  jb.newpiv = (f & F_NEWPIV) != 0;
  jb.surv = !(f & (F_PROVEN | F_FINAL)) && !a.cleared[j];
  if (jb.surv) {
    int32_t l = a.low[j];
    int32_t s = a.tab[l];
    jb.words = a.clen[j];
    if (s != j) {
      jb.target = true;
      if (a.do_adds) {
        uint8_t fs = a.flags[s];
        bool ok = !(fs & F_FINAL) && !a.cleared[s] && (!a.strict || (fs & F_PROVEN));
        if (ok) {
          jb.src = s;
          jb.words += a.clen[s];
        }
      }
    }
  }
  return jb;
}

__global__ void k_s2_tiles(RArgs a) {
  __shared__ int64_t sh[kWarps + 1];
  int64_t tile0 = (int64_t)blockIdx.x * kRTile;
  int64_t t0 = 0, t1 = 0, pivw = 0, targ = 0;
  for (int it = 0; it < kRItems; it++) {
    Job jb = job_of(a, tile0 + it * kThreads + threadIdx.x);
    int64_t cs, cw;
    block_excl_sum<int64_t>(jb.surv ? 1 : 0, sh, cs);
    block_excl_sum<int64_t>(jb.words, sh, cw);
    if (threadIdx.x == 0) {
      a.chunk_cnt[2 * ((int64_t)blockIdx.x * kRItems + it)] = cs;
      a.chunk_cnt[2 * ((int64_t)blockIdx.x * kRItems + it) + 1] = cw;
    }
    t0 += cs;
    t1 += cw;
    targ += jb.target;
    if (jb.newpiv) pivw += a.clen[jb.j];
  }
  int64_t t2, t3;
  block_excl_sum<int64_t>(pivw, sh, t2);
  block_excl_sum<int64_t>(targ, sh, t3);
  if (threadIdx.x == 0) {
    a.tile_cnt[2 * blockIdx.x] = t0;
    a.tile_cnt[2 * blockIdx.x + 1] = t1;
    a.tile_aux[2 * blockIdx.x] = t2;
    a.tile_aux[2 * blockIdx.x + 1] = t3;
  }
}

__global__ void k_s2_top(RArgs a, int64_t ntiles) {
  __shared__ int64_t sh[kWarps + 1];
  int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  for (int64_t base = 0; base < ntiles; base += kThreads) {
    int64_t i = base + threadIdx.x;
    int64_t v0 = i < ntiles ? a.tile_cnt[2 * i] : 0;
    int64_t v1 = i < ntiles ? a.tile_cnt[2 * i + 1] : 0;
    int64_t v2 = i < ntiles ? a.tile_aux[2 * i] : 0;
    int64_t v3 = i < ntiles ? a.tile_aux[2 * i + 1] : 0;
    int64_t t0, t1, t2, t3;
    int64_t e0 = block_excl_sum<int64_t>(v0, sh, t0);
    int64_t e1 = block_excl_sum<int64_t>(v1, sh, t1);
    block_excl_sum<int64_t>(v2, sh, t2);
    block_excl_sum<int64_t>(v3, sh, t3);
    if (i < ntiles) {
      a.tile_cnt[2 * i] = c0 + e0;
      a.tile_cnt[2 * i + 1] = c1 + e1;
    }
    c0 += t0;
    c1 += t1;
    c2 += t2;
    c3 += t3;
  }
  if (threadIdx.x == 0) {
    a.totals[0] = c0;
    a.totals[1] = c1;
    a.totals[2] = c2;
    a.totals[3] = c3;
    if (a.stats) a.stats[PH_PS_TARGETS] = c3;
  }
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

// Per-warp shared staging: the columns (A then B) of a batch of the warp's jobs, stored back
// to back, and per-job bookkeeping. kStage rows per warp bound a staged merge.
constexpr int kStage = 1024;
struct WarpStage {
  int32_t in[kStage];
  int32_t na[32];
  int32_t nin[32];      // rows staged for the job (na + nb), 0 if not staged
  int32_t in_off[33];   // exclusive prefix of nin over the warp's lanes
  int32_t pad_off[33];  // exclusive prefix of nin rounded up to km
  int32_t jstart[32];   // first output row of the job, relative to the warp's output base
  int32_t jcnt[32];     // output rows of the job
  int32_t jlow[32];     // largest output row (new low), -1 if none
};
constexpr size_t kAddSmem = sizeof(WarpStage) * kWarps;

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

// Phase II for one 256-entry chunk of the active list per block. After one block scan for the
// output offsets, every warp works on its own 32 jobs: new pivots are copied to the pivot store;
// survivors (with or without an addition) are staged in shared memory and merged by a merge
// path over the concatenation of all of the batch's jobs, each job padded to a multiple of km
// positions so that a lane's km positions never span two jobs (km is chosen per warp from the
// mean merge length); outputs are written compactly and in order into the warp's region of the
// next arena. Merges longer than the staging bound run from global memory.
__global__ void __launch_bounds__(kThreads, 4) k_add(RArgs a) {
  __shared__ int64_t sh[kWarps + 1];
  extern __shared__ __align__(16) unsigned char add_smem[];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  WarpStage& S = reinterpret_cast<WarpStage*>(add_smem)[w];
  const int64_t chunk = blockIdx.x, tile = chunk / kRItems;
  int64_t cs = a.tile_cnt[2 * tile], cw = a.tile_cnt[2 * tile + 1];
  for (int64_t c = tile * kRItems; c < chunk; c++) {
    cs += a.chunk_cnt[2 * c];
    cw += a.chunk_cnt[2 * c + 1];
  }
  const int64_t e = chunk * kThreads + threadIdx.x;
  Job jb = job_of(a, e);
  int64_t ts, tw;
  const int64_t pos = cs + block_excl_sum<int64_t>(jb.surv ? 1 : 0, sh, ts);
  const int64_t off = cw + block_excl_sum<int64_t>(jb.words, sh, tw);
  int64_t n_add = 0, n_xor = 0, n_copy = 0;

  const int32_t* A = nullptr;
  const int32_t* B = nullptr;
  int na = 0, nb = 0;
  if (jb.j >= 0 && (jb.newpiv || jb.surv)) {
    A = a.cptr[jb.j];
    na = a.clen[jb.j];
    if (jb.surv && jb.src >= 0) {
      B = a.cptr[jb.src];
      nb = a.clen[jb.src];
    }
  }
  if (jb.j >= 0 && !jb.newpiv && !jb.surv) {
    a.nxt_ptr[e] = nullptr;
    a.nxt_len[e] = 0;
  }
  if (jb.surv) a.act2[pos] = jb.j;

  // ---- new pivots: their columns never change again; move them to the pivot store
  unsigned pmask = __ballot_sync(0xffffffffu, jb.newpiv);
  while (pmask) {
    const int src = __ffs(pmask) - 1;
    pmask &= pmask - 1;
    const int32_t* wA = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)A, src);
    const int wna = __shfl_sync(0xffffffffu, na, src);
    unsigned long long w0 = 0;
    if (lane == src) w0 = atomicAdd(a.piv_bump, (unsigned long long)wna);
    w0 = __shfl_sync(0xffffffffu, w0, src);
    int32_t* dst = a.piv_base + w0;
    for (int q = lane; q < wna; q += 32) dst[q] = wA[q];
    if (lane == src) {
      a.nxt_ptr[e] = dst;
      a.nxt_len[e] = wna;
      n_copy += wna;
    }
  }

  // ---- survivors
  const unsigned smask = __ballot_sync(0xffffffffu, jb.surv);
  if (smask) {
    const int first = __ffs(smask) - 1;
    const int64_t wbase = __shfl_sync(0xffffffffu, off, first);  // warp's output region
    const int N = jb.surv ? na + nb : 0;
    const bool big = N > a.staged_max;
    const int nin = big ? 0 : N;
    const int in_ex = warp_incl_sum(nin) - nin;
    const int small_total = __shfl_sync(0xffffffffu, in_ex + nin, 31);
    const int n_staged = __popc(__ballot_sync(0xffffffffu, nin > 0));
    const int mean = n_staged ? small_total / n_staged : 0;
    // longer chunks amortise the two merge-path splits, shorter ones keep lanes balanced
    const int km = a.force_km > 0 ? a.force_km
                                  : (mean >= 160 ? 32 : (mean >= 80 ? 16 : (mean >= 32 ? 8 : 4)));
    const int npad = (nin + km - 1) / km * km;
    const int pad_ex = warp_incl_sum(npad) - npad;
    const int bigN = big ? N : 0;
    const int big_ex = warp_incl_sum(bigN) - bigN;
    S.na[lane] = na;
    S.nin[lane] = nin;
    S.in_off[lane] = in_ex;
    S.pad_off[lane] = pad_ex;
    S.jstart[lane] = 0;
    S.jcnt[lane] = 0;
    S.jlow[lane] = -1;
    if (lane == 31) {
      S.in_off[32] = in_ex + nin;
      S.pad_off[32] = pad_ex + npad;
    }
    __syncwarp();
    int32_t* out = a.arena_next + wbase;  // compact outputs of the staged jobs
    int ocur = 0;
    int c = 0;
    while (c < 32) {
      // batch: jobs c.. whose staged rows fit together
      const int in_c = S.in_off[c];
      const bool fits = lane >= c && S.in_off[lane] + S.nin[lane] - in_c <= kStage;
      const int c_end = c + __popc(__ballot_sync(0xffffffffu, fits));
      const int nch = (S.pad_off[c_end] - S.pad_off[c]) / km;
      const bool mine = lane >= c && lane < c_end && nin > 0;
      if (__ballot_sync(0xffffffffu, mine)) {
        // stage: columns of 32+ rows by the whole warp (coalesced), shorter ones by their lane
        unsigned lmask = __ballot_sync(0xffffffffu, mine && nin >= 32);
        while (lmask) {
          const int src = __ffs(lmask) - 1;
          lmask &= lmask - 1;
          const int32_t* wA = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)A, src);
          const int32_t* wB = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)B, src);
          const int wna = __shfl_sync(0xffffffffu, na, src);
          const int wn = __shfl_sync(0xffffffffu, nin, src);
          int32_t* d = S.in + (__shfl_sync(0xffffffffu, in_ex, src) - in_c);
          for (int q = lane; q < wn; q += 64) {
            const int q2 = q + 32;
            const int32_t v0 = q < wna ? __ldg(wA + q) : __ldg(wB + (q - wna));
            int32_t v1 = 0;
            if (q2 < wn) v1 = q2 < wna ? __ldg(wA + q2) : __ldg(wB + (q2 - wna));
            d[q] = v0;
            if (q2 < wn) d[q2] = v1;
          }
        }
        if (mine && nin < 32) {
          int32_t* d = S.in + (in_ex - in_c);
          int q = 0;
          for (; q + 4 <= na; q += 4) {
            const int32_t v0 = __ldg(A + q), v1 = __ldg(A + q + 1), v2 = __ldg(A + q + 2),
                          v3 = __ldg(A + q + 3);
            d[q] = v0;
            d[q + 1] = v1;
            d[q + 2] = v2;
            d[q + 3] = v3;
          }
          for (; q < na; q++) d[q] = __ldg(A + q);
          int r = 0;
          for (; r + 4 <= nb; r += 4) {
            const int32_t v0 = __ldg(B + r), v1 = __ldg(B + r + 1), v2 = __ldg(B + r + 2),
                          v3 = __ldg(B + r + 3);
            d[na + r] = v0;
            d[na + r + 1] = v1;
            d[na + r + 2] = v2;
            d[na + r + 3] = v3;
          }
          for (; r < nb; r++) d[na + r] = __ldg(B + r);
        }
        __syncwarp();
        // merge: lane takes one km-position chunk per round
        const int p0 = S.pad_off[c];
        for (int h0 = 0; h0 < nch; h0 += 32) {
          const int h = h0 + lane;
          int cnt = 0, k = -1, x0 = 0, y0 = 0, x1 = 0, y1 = 0;
          const int32_t* sA = S.in;
          const int32_t* sB = S.in;
          if (h < nch) {
            const int gp = p0 + h * km;
            int lo = c, hi = c_end - 1;
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (S.pad_off[mid] <= gp) lo = mid; else hi = mid - 1;
            }
            k = lo;
            const int d = gp - S.pad_off[k];
            const int nk = S.nin[k];
            if (d < nk) {
              sA = S.in + (S.in_off[k] - in_c);
              const int ka = S.na[k], kb = nk - ka;
              sB = sA + ka;
              merge_split(sA, ka, sB, kb, d, x0, y0);
              merge_split(sA, ka, sB, kb, min(d + km, nk), x1, y1);
              cnt = lane_symdiff<false>(sA, x0, x1, sB, y0, y1, nullptr, nullptr);
            }
          }
          const int incl = warp_incl_sum(cnt);
          const int o = ocur + incl - cnt;
          if (k >= 0) {
            if (h * km == S.pad_off[k] - p0) S.jstart[k] = o;
            if (cnt) {
              int32_t last;
              lane_symdiff<true>(sA, x0, x1, sB, y0, y1, out + o, &last);
              atomicAdd(&S.jcnt[k], cnt);
              atomicMax(&S.jlow[k], last);
            }
          }
          ocur += __shfl_sync(0xffffffffu, incl, 31);
        }
      }
      __syncwarp();
      c = c_end;
    }
    __syncwarp();
    if (jb.surv && !big) {
      const int len = S.jcnt[lane];
      a.nxt_ptr[e] = out + S.jstart[lane];
      a.nxt_len[e] = len;
      if (B) {
        a.low[jb.j] = S.jlow[lane];
        n_add++;
        n_xor += (na + nb + len) / 2;
      } else {
        n_copy += na;
      }
    }
    // merges too long to stage: straight from global memory, after the staged outputs
    unsigned bmask = __ballot_sync(0xffffffffu, big);
    while (bmask) {
      const int src = __ffs(bmask) - 1;
      bmask &= bmask - 1;
      const int32_t* wA = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)A, src);
      const int32_t* wB = (const int32_t*)__shfl_sync(0xffffffffu, (unsigned long long)B, src);
      const int wna = __shfl_sync(0xffffffffu, na, src);
      const int wnb = __shfl_sync(0xffffffffu, nb, src);
      int32_t* wd = a.arena_next + wbase + small_total + __shfl_sync(0xffffffffu, big_ex, src);
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
          n_add++;
          n_xor += (na + nb + len) / 2;
        } else {
          n_copy += na;
        }
        a.nxt_ptr[e] = wd;
        a.nxt_len[e] = len;
      }
    }
  }
  if (a.stats) {
    stat_add(a.stats, PH_PS_ADDS, n_add);
    stat_add(a.stats, PH_PS_XORS, n_xor);
    stat_add(a.stats, PH_PS_COPIED, n_copy);
  }
}

__global__ void k_commit(RArgs a) {
  int64_t n_clear = 0, n_act = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.n_act;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = a.act[e];
    uint8_t f = a.flags[j];
    uint8_t c = a.cleared[j];
    n_act++;
    n_clear += c;
    bool surv = !(f & (F_PROVEN | F_FINAL)) && !c;
    if (f & F_NEWPIV) {
      a.cptr[j] = a.nxt_ptr[e];
      a.clen[j] = a.nxt_len[e];
      a.flags[j] = f & (uint8_t)~F_NEWPIV;
    } else if (surv) {
      a.cptr[j] = a.nxt_ptr[e];
      a.clen[j] = a.nxt_len[e];
    } else {
      a.flags[j] = f | F_FINAL;
      a.low[j] = -1;
      a.clen[j] = 0;
    }
  }
  if (a.stats) {
    stat_add(a.stats, PH_PS_ACTIVE, n_act);
    stat_add(a.stats, PH_PS_CLEARED, n_clear);
  }
}

// ------------------------------------------------------------------------------------------
// set-up
// ------------------------------------------------------------------------------------------
struct InitLayout {
  int64_t dimoff[kMaxDim + 2];
  int64_t rowbase[kMaxDim + 2];
  int maxd;
};

// the boundary matrix of a simplicial complex: a column of dimension d > 0 has d + 1 rows,
// stored in id order from rowbase[d]
__global__ void k_reduce_init(int64_t m, InitLayout L, int32_t* rows0, int32_t** cptr,
                              int32_t* clen, int32_t* low, int32_t* act, int32_t* owner,
                              uint8_t* flags, uint8_t* cleared) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    int d = 0;
    while (d < L.maxd && x >= L.dimoff[d + 1]) d++;
    int32_t* c = rows0 + L.rowbase[d] + (int64_t)(d > 0 ? d + 1 : 0) * (x - L.dimoff[d]);
    cptr[x] = c;
    clen[x] = d > 0 ? d + 1 : 0;
    low[x] = d > 0 ? c[d] : -1;  // largest row of the unreduced column
    act[x] = (int32_t)x;
    owner[x] = -1;
    flags[x] = 0;
    cleared[x] = 0;
  }
}

static void grow_store(ph_ctx* ctx, ColStore& s, int64_t need_words) {
  if (need_words <= s.cap) return;
  if (s.p) ctx->dfree(s.p);
  int64_t cap = std::max<int64_t>(need_words + need_words / 4, 1 << 20);
  s.p = alloc_n<int32_t>(ctx, cap);
  s.cap = cap;
}

void reduce_init(ph_ctx* ctx) {
  ReduceState& rs = ctx->rs;
  const int64_t m = ctx->m;
  rs.act = alloc_n<int32_t>(ctx, m);
  rs.act2 = alloc_n<int32_t>(ctx, m);
  rs.act_cap = m;
  rs.cptr = alloc_n<int32_t*>(ctx, m);
  rs.clen = alloc_n<int32_t>(ctx, m);
  rs.nxt_ptr = alloc_n<int32_t*>(ctx, m);
  rs.nxt_len = alloc_n<int32_t>(ctx, m);
  rs.owner = alloc_n<int32_t>(ctx, m);
  rs.tab = alloc_n<int32_t>(ctx, m);
  rs.flags = alloc_n<uint8_t>(ctx, m);
  rs.cleared = alloc_n<uint8_t>(ctx, m);
  int nseg = (int)ctx->seg_start.size() - 1;
  rs.first_unp = alloc_n<int32_t>(ctx, nseg);
  int64_t ntiles = (m + kRTile - 1) / kRTile;
  rs.tiles_bytes = ntiles * ((1 + kRItems) * sizeof(SegMax) + (4 + 2 * kRItems) * sizeof(int64_t));
  rs.tiles = ctx->dalloc(rs.tiles_bytes);
  rs.totals = alloc_n<int64_t>(ctx, 8);
  PH_CUDA(cudaMallocHost(&rs.h_totals, 8 * sizeof(int64_t)));
  rs.stats_rows = 0;
  rs.pass_stats = nullptr;
  rs.h_stats.clear();
  InitLayout L{};
  L.maxd = ctx->max_dim;
  for (int d = 0; d <= ctx->max_dim + 1; d++) L.dimoff[d] = ctx->dimoff[d];
  int64_t rb = 0;
  for (int d = 0; d <= ctx->max_dim; d++) {
    L.rowbase[d] = rb;
    rb += (d > 0 ? d + 1 : 0) * (ctx->dimoff[d + 1] - ctx->dimoff[d]);
  }
  k_reduce_init<<<grid_for(ctx, m, kThreads), kThreads, 0, ctx->stream>>>(
      m, L, ctx->rows0, rs.cptr, rs.clen, ctx->low, rs.act, rs.owner, rs.flags, rs.cleared);
  PH_CHECK_LAUNCH();
  rs.n_act = m;
  rs.cur = 0;
  rs.arena[0].p = ctx->rows0;  // the boundary matrix is the first arena
  rs.arena[0].cap = ctx->nnz;
  rs.arena[1] = ColStore{};
  rs.pivots.clear();
  rs.piv_used = 0;
  rs.piv_bump = alloc_n<int64_t>(ctx, 1);
  PH_CUDA(cudaMemsetAsync(rs.piv_bump, 0, sizeof(int64_t), ctx->stream));
  rs.passes = 0;
  rs.next_pass = 0;
  rs.init = true;
  rs.done = false;
  rs.status = PH_OK;
}

int reduce_run(ph_ctx* ctx, int32_t max_passes) {
  ReduceState& rs = ctx->rs;
  cudaStream_t st = ctx->stream;
  const int64_t m = ctx->m;
  const int64_t rows_end = ctx->dimoff[ctx->max_dim];
  const int nseg = (int)ctx->seg_start.size() - 1;
  const bool stats = ctx->opts.collect_stats != 0;
  if (max_passes < 0) max_passes = INT32_MAX;

  RArgs a{};
  a.low = ctx->low;
  a.beta = ctx->beta;
  a.flags = rs.flags;
  a.cleared = rs.cleared;
  a.cptr = rs.cptr;
  a.clen = rs.clen;
  a.nxt_ptr = rs.nxt_ptr;
  a.nxt_len = rs.nxt_len;
  a.owner = rs.owner;
  a.tab = rs.tab;
  a.first_unp = rs.first_unp;
  a.seg = ctx->seg;
  a.nc = ctx->n_clouds;
  a.strict = ctx->opts.strict_phase2;
  a.cor10 = ctx->opts.use_cor10;
  a.totals = rs.totals;
  a.piv_bump = (unsigned long long*)rs.piv_bump;
  a.staged_max = ctx->opts.staged_merge_max > 0 ? std::min(ctx->opts.staged_merge_max, kStage)
                                                 : kStage;
  a.force_km = std::max(0, std::min(ctx->opts.merge_items, 64));

  for (int pass = rs.next_pass;; pass++) {
    const int64_t n_act = rs.n_act;
    const int64_t ntiles = std::max<int64_t>((n_act + kRTile - 1) / kRTile, 1);
    a.act = rs.act;
    a.act2 = rs.act2;
    a.n_act = n_act;
    const int64_t nchunks = std::max<int64_t>((n_act + kThreads - 1) / kThreads, 1);
    a.tile_sm = (SegMax*)rs.tiles;
    a.chunk_sm = a.tile_sm + ntiles;
    a.tile_cnt = (int64_t*)(a.chunk_sm + ntiles * kRItems);
    a.tile_aux = a.tile_cnt + 2 * ntiles;
    a.chunk_cnt = a.tile_aux + 2 * ntiles;
    a.do_adds = pass < max_passes;
    if (stats) {
      if (pass >= rs.stats_rows) {
        int32_t rows = std::max(64, rs.stats_rows * 2);
        int64_t* ns = alloc_n<int64_t>(ctx, (int64_t)rows * PH_PS_N);
        PH_CUDA(cudaMemsetAsync(ns, 0, (size_t)rows * PH_PS_N * sizeof(int64_t), st));
        if (rs.pass_stats) {
          PH_CUDA(cudaMemcpyAsync(ns, rs.pass_stats,
                                  (size_t)rs.stats_rows * PH_PS_N * sizeof(int64_t),
                                  cudaMemcpyDeviceToDevice, st));
          ctx->dfree(rs.pass_stats);
        }
        rs.pass_stats = ns;
        rs.stats_rows = rows;
      }
      a.stats = rs.pass_stats + (int64_t)pass * PH_PS_N;
    }
    PH_CUDA(cudaMemsetAsync(rs.first_unp, 0x7f, nseg * sizeof(int32_t), st));
    k_tab_init<<<grid_for(ctx, rows_end, kThreads), kThreads, 0, st>>>(
        rows_end, rs.owner, rs.flags, ctx->beta, ctx->seg, rs.tab, rs.first_unp);
    PH_CHECK_LAUNCH();
    k_tab<<<grid_for(ctx, n_act, kThreads), kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
    k_p1_tiles<<<(unsigned)ntiles, kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
    k_p1_top<<<1, kThreads, 0, st>>>(a.tile_sm, ntiles);
    PH_CHECK_LAUNCH();
    k_mark<<<(unsigned)nchunks, kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
    k_s2_tiles<<<(unsigned)ntiles, kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
    k_s2_top<<<1, kThreads, 0, st>>>(a, ntiles);
    PH_CHECK_LAUNCH();
    PH_CUDA(cudaMemcpyAsync(rs.h_totals, rs.totals, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                            st));
    PH_CUDA(cudaStreamSynchronize(st));
    const int64_t surv = rs.h_totals[0], words = rs.h_totals[1], pivw = rs.h_totals[2],
                  targets = rs.h_totals[3];
    // capacity: next arena and pivot store
    ColStore& nxt = rs.arena[1 - rs.cur];
    if (nxt.p == ctx->rows0) {  // never overwrite the boundary matrix in place
      nxt = ColStore{};
    }
    grow_store(ctx, nxt, words);
    if (rs.pivots.empty() || rs.piv_used + pivw > rs.pivots.back().cap) {
      ColStore c{};
      grow_store(ctx, c, std::max<int64_t>(pivw, ctx->nnz / 4 + 1));
      rs.pivots.push_back(c);
      rs.piv_used = 0;
      PH_CUDA(cudaMemsetAsync(rs.piv_bump, 0, sizeof(int64_t), st));
    }
    a.arena_next = nxt.p;
    a.piv_base = rs.pivots.back().p;
    rs.piv_used += pivw;
    if (ctx->opts.time_kernels) {
      cudaEvent_t e0, e1;
      PH_CUDA(cudaEventCreate(&e0));
      PH_CUDA(cudaEventCreate(&e1));
      rs.ev.push_back(e0);
      rs.ev.push_back(e1);
      PH_CUDA(cudaEventRecord(e0, st));
    }
    PH_CUDA(cudaFuncSetAttribute(k_add, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kAddSmem));
    k_add<<<(unsigned)nchunks, kThreads, kAddSmem, st>>>(a);
    PH_CHECK_LAUNCH();
    rs.add_launches++;
    if (ctx->opts.time_kernels) PH_CUDA(cudaEventRecord(rs.ev.back(), st));
    k_commit<<<grid_for(ctx, n_act, kThreads), kThreads, 0, st>>>(a);
    PH_CHECK_LAUNCH();
    std::swap(rs.act, rs.act2);
    rs.n_act = surv;
    // the old arena is dead now unless it is the boundary matrix, which stays for reuse
    rs.cur = 1 - rs.cur;
    if (targets == 0) {
      rs.passes = pass;
      rs.status = PH_OK;
      break;
    }
    if (pass >= max_passes) {
      rs.passes = pass;
      rs.next_pass = pass + 1;
      rs.status = PH_NOT_CONVERGED;
      break;
    }
  }
  if (stats) {
    rs.h_stats.assign((size_t)(rs.passes + 1) * PH_PS_N, 0);
    PH_CUDA(cudaMemcpyAsync(rs.h_stats.data(), rs.pass_stats,
                            rs.h_stats.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  }
  PH_CUDA(cudaStreamSynchronize(st));
  for (size_t i = 0; i + 1 < rs.ev.size(); i += 2) {
    float ms = 0;
    PH_CUDA(cudaEventElapsedTime(&ms, rs.ev[i], rs.ev[i + 1]));
    rs.ms_add += ms;
    cudaEventDestroy(rs.ev[i]);
    cudaEventDestroy(rs.ev[i + 1]);
  }
  rs.ev.clear();
  rs.done = true;
  (void)m;
  return rs.status;
}

void free_reduce_state(ph_ctx* ctx) {
  ReduceState& rs = ctx->rs;
  for (void* p : {(void*)rs.act, (void*)rs.act2, (void*)rs.cptr, (void*)rs.clen,
                  (void*)rs.nxt_ptr, (void*)rs.nxt_len, (void*)rs.owner, (void*)rs.tab,
                  (void*)rs.flags, (void*)rs.cleared, (void*)rs.first_unp, rs.tiles,
                  (void*)rs.totals, (void*)rs.pass_stats, (void*)rs.piv_bump})
    ctx->dfree(p);
  for (auto& a : rs.arena)
    if (a.p && a.p != ctx->rows0) ctx->dfree(a.p);
  for (auto& c : rs.pivots) ctx->dfree(c.p);
  if (rs.h_totals) cudaFreeHost(rs.h_totals);
  for (auto e : rs.ev) cudaEventDestroy(e);
  rs = ReduceState{};
}

}  // namespace ph
