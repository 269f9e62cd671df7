// Filtration and boundary-matrix construction on the device (Sec. 2.2-2.3, Definition 4).
//
// Vietoris-Rips: a simplex enters at its diameter (f_r(sigma) = 1{diam(sigma) <= 2r}); its
// squared diameter is the largest squared edge length among its vertices, an exact int64 on
// the 2^-16 grid. The compatible ordering is (squared diameter, dimension, vertex tuple in
// lexicographic order). Rather than sorting 64-bit diameters for every dimension, edges are
// sorted once by (cloud, diameter, lex) and given the dense rank of their squared diameter; a
// higher simplex's key is the largest rank among its edges, which orders exactly like its
// squared diameter. Candidates are enumerated in (cloud, lex) order, so a stable sort by that
// key yields (cloud, diameter, lex) directly: dense ranks grow with the cloud index.
#include <algorithm>

#include "ph_internal.cuh"

namespace ph {

// cloud in the top 16 bits, then 48 / vbits vertex slots of vbits bits (unused: all ones)
__host__ __device__ __forceinline__ uint64_t pack_simplex(uint32_t cloud, int k, const int* v,
                                                          int vbits) {
  uint64_t p = (uint64_t)cloud << 48;
  const int slots = 48 / vbits;
  const uint64_t none = (1ull << vbits) - 1ull;
  for (int i = 0; i < slots; i++) {
    uint64_t x = i < k ? (uint64_t)v[i] : none;
    p |= x << (48 - vbits * (i + 1));
  }
  return p;
}
__device__ __forceinline__ uint32_t packed_cloud(uint64_t p) { return (uint32_t)(p >> 48); }

// C(n, k) for the small k of a VR build (k <= 6); exact in int64 for n < 2^12. A product of k
// consecutive integers divided by k!, each case a division by a constant (a multiply and a
// shift), so the unranking's binary searches carry no run-time 64-bit division
__host__ __device__ __forceinline__ int64_t binom_small(int64_t n, int k) {
  if (n < k || n < 0 || k < 0) return 0;
  switch (k) {
    case 0: return 1;
    case 1: return n;
    case 2: return n * (n - 1) / 2;
    case 3: return n * (n - 1) * (n - 2) / 6;
    case 4: return n * (n - 1) * (n - 2) * (n - 3) / 24;
    case 5: return n * (n - 1) * (n - 2) * (n - 3) * (n - 4) / 120;
    default: {
      int64_t r = 1;
      for (int i = 0; i < k; i++) r = r * (n - i) / (i + 1);  // each prefix is a binomial
      return r;
    }
  }
}

// k-subset of [n] with lexicographic rank r (0-based). Uses the complement map
// v -> n-1-v, which turns lexicographic order into reversed colexicographic order, where a
// subset's rank is sum_i C(u_i, i+1) and can be peeled off greedily.
__device__ __forceinline__ void lex_unrank(int64_t r, int n, int k, int* v) {
  int64_t R = binom_small(n, k) - 1 - r;
  int u[kVrSlots];
  int hi = n - 1;
  for (int i = k - 1; i >= 0; i--) {
    int lo = i, h = hi;
    while (lo < h) {
      int mid = (lo + h + 1) >> 1;
      if (binom_small(mid, i + 1) <= R) lo = mid; else h = mid - 1;
    }
    u[i] = lo;
    R -= binom_small(lo, i + 1);
    hi = lo - 1;
  }
  for (int i = 0; i < k; i++) v[i] = n - 1 - u[k - 1 - i];
}

__device__ __forceinline__ int64_t lex_rank(const int* v, int n, int k) {
  int64_t R = 0;
  for (int i = 0; i < k; i++) R += binom_small(n - 1 - v[k - 1 - i], i + 1);
  return binom_small(n, k) - 1 - R;
}

__device__ __forceinline__ int find_cloud(const int64_t* __restrict__ off, int nc, int64_t t) {
  int lo = 0, hi = nc - 1;  // last c with off[c] <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct CloudTabs {
  const int64_t* pt_off;  // [nc+1] point offsets
  const int64_t* mo;      // [nc+1] offsets of the n_c x n_c tables
  int nc;
  int vbits;              // bits per packed vertex
};

__device__ __forceinline__ int packed_vert(const CloudTabs& ct, uint64_t p, int i) {
  return packed_vert_at(p, i, ct.vbits);
}

// ------------------------------------------------------------------------------------------
__global__ void k_check_coords(const int32_t* __restrict__ x, int64_t n, int32_t* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = x[i];
    if (v > (1 << 24) || v < -(1 << 24)) *bad = 1;
  }
}

// squared distances of every ordered pair of each cloud; block row y = cloud
__global__ void k_pairwise(const int32_t* __restrict__ x, int D, CloudTabs ct, int64_t* d2,
                           unsigned long long* maxd2) {
  int c = blockIdx.y;
  int64_t p0 = ct.pt_off[c];
  int n = (int)(ct.pt_off[c + 1] - p0);
  int64_t nn = (int64_t)n * n;
  unsigned long long mx = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn;
       t += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(t / n), b = (int)(t % n);
    const int32_t* xa = x + (p0 + a) * D;
    const int32_t* xb = x + (p0 + b) * D;
    int64_t s = 0;
    for (int k = 0; k < D; k++) {
      int64_t dd = (int64_t)xa[k] - (int64_t)xb[k];
      s += dd * dd;
    }
    d2[ct.mo[c] + t] = s;
    mx = s > (int64_t)mx ? (unsigned long long)s : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_down_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(maxd2, mx);
}

// Index of the first scale r_i = i * step with d <= 2 r_i for a squared distance d2 (Sec. 2.2:
// a simplex is in the complex at scale r when its diameter is at most 2r), by exact integer
// comparison: the smallest i >= 0 with d2 <= (2 i step)^2.
__host__ __device__ __forceinline__ int64_t scale_index_of(int64_t d2, int64_t step) {
  if (d2 <= 0) return 0;
  int64_t i = (int64_t)ceil(sqrt((double)d2) / (2.0 * (double)step));
  while (i > 0 && (2 * (i - 1) * step) * (2 * (i - 1) * step) >= d2) i--;
  while ((2 * i * step) * (2 * i * step) < d2) i++;
  return i;
}

__global__ void k_scale_index(int64_t* d2, int64_t n, int64_t step) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    d2[t] = scale_index_of(d2[t], step);
}

// count one kept candidate for cloud c with one atomic per group of lanes sharing c
__device__ __forceinline__ void count_kept(int64_t* count_per_cloud, int c, bool keep) {
  const unsigned peers = __match_any_sync(__activemask(), keep ? c : -1);
  if (keep && (threadIdx.x & 31) == __ffs(peers) - 1)
    atomicAdd((unsigned long long*)&count_per_cloud[c], (unsigned long long)__popc(peers));
}

// edge candidates in (cloud, lex) order; truncated edges get key = sent
__global__ void k_edge_cand(CloudTabs ct, const int64_t* __restrict__ cand, int64_t ncand,
                            const int64_t* __restrict__ d2, int64_t max_d2, uint64_t sent,
                            uint64_t* keys, uint64_t* vals, int64_t* count_per_cloud) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncand;
       t += (int64_t)gridDim.x * blockDim.x) {
    int c = find_cloud(cand, ct.nc, t);
    int n = (int)(ct.pt_off[c + 1] - ct.pt_off[c]);
    int v[2];
    lex_unrank(t - cand[c], n, 2, v);
    int64_t e = d2[ct.mo[c] + (int64_t)v[0] * n + v[1]];
    bool keep = max_d2 < 0 || e <= max_d2;
    keys[t] = keep ? (uint64_t)e : sent;
    vals[t] = pack_simplex((uint32_t)c, 2, v, ct.vbits);
    count_kept(count_per_cloud, c, keep);
  }
}

__global__ void k_rekey_cloud(const uint64_t* __restrict__ vals, uint64_t* keys, int64_t n,
                              uint64_t sent, uint64_t nc) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    keys[t] = keys[t] == sent ? nc : (uint64_t)packed_cloud(vals[t]);
}

// first element of each distinct (cloud, squared diameter) among the sorted edges
__global__ void k_edge_newflag(const uint64_t* __restrict__ vals, int64_t E, CloudTabs ct,
                               const int64_t* __restrict__ d2, int64_t* flag, int64_t* ed2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p = vals[i];
    int c = (int)packed_cloud(p);
    int n = (int)(ct.pt_off[c + 1] - ct.pt_off[c]);
    int64_t e = d2[ct.mo[c] + (int64_t)packed_vert(ct, p, 0) * n + packed_vert(ct, p, 1)];
    ed2[i] = e;
    int64_t f = 1;
    if (i > 0) {
      uint64_t q = vals[i - 1];
      int cq = (int)packed_cloud(q);
      if (cq == c) {
        int64_t eq = d2[ct.mo[c] + (int64_t)packed_vert(ct, q, 0) * n + packed_vert(ct, q, 1)];
        f = (eq != e);
      }
    }
    flag[i] = f;
  }
}

struct IdOut {
  int32_t* seg;
  int32_t* key;
  int32_t* low;
  uint64_t* verts;
  int32_t* rows0;
};

__global__ void k_edge_finish(const uint64_t* __restrict__ vals, int64_t E, CloudTabs ct,
                              const int64_t* __restrict__ flag, const int64_t* __restrict__ excl,
                              const int64_t* __restrict__ ed2, int64_t id0, int32_t* eid,
                              int32_t* erank, int64_t* d2tab, IdOut o, int64_t rowbase) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p = vals[i];
    int c = (int)packed_cloud(p);
    int n = (int)(ct.pt_off[c + 1] - ct.pt_off[c]);
    int a = packed_vert(ct, p, 0), b = packed_vert(ct, p, 1);
    int32_t rank = (int32_t)(excl[i] + flag[i] - 1);
    if (flag[i]) d2tab[rank] = ed2[i];
    int64_t id = id0 + i;
    int64_t mo = ct.mo[c];
    eid[mo + (int64_t)a * n + b] = (int32_t)id;
    eid[mo + (int64_t)b * n + a] = (int32_t)id;
    erank[mo + (int64_t)a * n + b] = rank;
    erank[mo + (int64_t)b * n + a] = rank;
    o.seg[id] = ct.nc + c;
    o.key[id] = rank;
    o.verts[id] = p;
    int32_t r0 = (int32_t)(ct.pt_off[c] + a), r1 = (int32_t)(ct.pt_off[c] + b);
    o.rows0[rowbase + 2 * i] = r0;
    o.rows0[rowbase + 2 * i + 1] = r1;
    o.low[id] = r1;
  }
}

// candidates of dimension k-1 (k vertices, 3 <= k <= 6): key = largest edge rank
__global__ void k_simplex_cand(CloudTabs ct, const int64_t* __restrict__ cand, int64_t ncand,
                               int k, const int32_t* __restrict__ erank, uint64_t sent,
                               uint64_t* keys, uint64_t* vals, int64_t* count_per_cloud) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncand;
       t += (int64_t)gridDim.x * blockDim.x) {
    int c = find_cloud(cand, ct.nc, t);
    int n = (int)(ct.pt_off[c + 1] - ct.pt_off[c]);
    int v[kVrSlots];
    lex_unrank(t - cand[c], n, k, v);
    const int32_t* er = erank + ct.mo[c];
    int32_t mx = -1;
    bool keep = true;
    for (int p = 0; p < k; p++)
      for (int q = p + 1; q < k; q++) {
        int32_t r = er[(int64_t)v[p] * n + v[q]];
        if (r < 0) keep = false;
        mx = r > mx ? r : mx;
      }
    keys[t] = keep ? (uint64_t)mx : sent;
    vals[t] = pack_simplex((uint32_t)c, k, v, ct.vbits);
    count_kept(count_per_cloud, c, keep);
  }
}

__device__ __forceinline__ void sort_small(int32_t* r, int k) {
  for (int i = 1; i < k; i++) {
    int32_t x = r[i];
    int j = i - 1;
    while (j >= 0 && r[j] > x) {
      r[j + 1] = r[j];
      j--;
    }
    r[j + 1] = x;
  }
}

__global__ void k_tri_finish(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                             int64_t T, CloudTabs ct, const int32_t* __restrict__ eid, int64_t id0,
                             IdOut o, int64_t rowbase, int32_t* tid_tab,
                             const int64_t* __restrict__ tri_lex_off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p = vals[i];
    int c = (int)packed_cloud(p);
    int n = (int)(ct.pt_off[c + 1] - ct.pt_off[c]);
    int v[3] = {packed_vert(ct, p, 0), packed_vert(ct, p, 1), packed_vert(ct, p, 2)};
    const int32_t* e = eid + ct.mo[c];
    int32_t r[3] = {e[(int64_t)v[1] * n + v[2]], e[(int64_t)v[0] * n + v[2]],
                    e[(int64_t)v[0] * n + v[1]]};
    sort_small(r, 3);
    int64_t id = id0 + i;
    for (int q = 0; q < 3; q++) o.rows0[rowbase + 3 * i + q] = r[q];
    o.low[id] = r[2];
    o.seg[id] = 2 * ct.nc + c;
    o.key[id] = (int32_t)keys[i];
    o.verts[id] = p;
    if (tid_tab) tid_tab[tri_lex_off[c] + lex_rank(v, n, 3)] = (int32_t)id;
  }
}

// simplices of k >= 4 vertices (dimension >= 3): faces are the (k-1)-subsets, found by their
// lexicographic rank in the table the previous dimension filled; this dimension fills its own
// table when a higher one follows
__global__ void k_high_finish(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                              int64_t Q, int k, CloudTabs ct, const int32_t* __restrict__ face_tab,
                              const int64_t* __restrict__ face_lex_off, int32_t* self_tab,
                              const int64_t* __restrict__ self_lex_off, int64_t id0, IdOut o,
                              int64_t rowbase) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t p = vals[i];
    int c = (int)packed_cloud(p);
    int n = (int)(ct.pt_off[c + 1] - ct.pt_off[c]);
    int v[kVrSlots];
    for (int q = 0; q < k; q++) v[q] = packed_vert(ct, p, q);
    int32_t r[kVrSlots];
    for (int drop = 0; drop < k; drop++) {
      int f[kVrSlots], m = 0;
      for (int q = 0; q < k; q++)
        if (q != drop) f[m++] = v[q];
      r[drop] = face_tab[face_lex_off[c] + lex_rank(f, n, k - 1)];
    }
    sort_small(r, k);
    int64_t id = id0 + i;
    for (int q = 0; q < k; q++) o.rows0[rowbase + (int64_t)k * i + q] = r[q];
    o.low[id] = r[k - 1];
    o.seg[id] = (k - 1) * ct.nc + c;
    o.key[id] = (int32_t)keys[i];
    o.verts[id] = p;
    if (self_tab) self_tab[self_lex_off[c] + lex_rank(v, n, k)] = (int32_t)id;
  }
}

__global__ void k_vertex_init(CloudTabs ct, int64_t N, IdOut o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = find_cloud(ct.pt_off, ct.nc, i);
    int v = (int)(i - ct.pt_off[c]);
    o.seg[i] = c;
    o.key[i] = -1;
    o.low[i] = -1;
    o.verts[i] = pack_simplex((uint32_t)c, 1, &v, ct.vbits);
  }
}

// ------------------------------------------------------------------------------------------
// left(i) (Definition 3) by atomicMin over the columns holding row i, then
// beta_j = max{ i : left(i) = j } (Definition 4) by atomicMax.
// ------------------------------------------------------------------------------------------
struct ColLayout {  // initial column storage: dim d column x at rowbase[d] + (d+1)(x - dimoff[d])
  int64_t dimoff[kMaxDim + 2];
  int64_t rowbase[kMaxDim + 2];
  int maxd;
};

__device__ __forceinline__ int id_dim(const ColLayout& L, int64_t x) {
  int d = 0;
  while (d < L.maxd && x >= L.dimoff[d + 1]) d++;
  return d;
}

// col_off: the columns of a loaded matrix (any length); null: d + 1 rows at a fixed stride
__global__ void k_left(ColLayout L, const int32_t* __restrict__ rows0,
                       const int64_t* __restrict__ col_off, int32_t* left) {
  int64_t n = L.dimoff[L.maxd + 1] - L.dimoff[1];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = L.dimoff[1] + t;
    int d = id_dim(L, j);
    const int32_t* r = col_off ? rows0 + col_off[j]
                               : rows0 + L.rowbase[d] + (int64_t)(d + 1) * (j - L.dimoff[d]);
    const int64_t len = col_off ? col_off[j + 1] - col_off[j] : d + 1;
    for (int64_t q = 0; q < len; q++) atomicMin(&left[r[q]], (int32_t)j);
  }
}

__global__ void k_beta(int64_t nrows, const int32_t* __restrict__ left, int32_t* beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t j = left[i];
    if (j < nrows) atomicMax(&beta[j], (int32_t)i);  // rows without a coface keep the fill
  }
}

// filtration index of every simplex within its cloud: simplices of other dimensions that
// precede it are those of lower dimension with diameter <= its own and of higher dimension with
// diameter < its own (ties are broken by dimension); all vertices (diameter 0) come first.
__global__ void k_gidx(int64_t m, int nc, int maxd, const int32_t* __restrict__ seg,
                       const int32_t* __restrict__ key, const int64_t* __restrict__ seg_start,
                       const int64_t* __restrict__ pt_off, int64_t* gidx) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    int s = seg[x];
    int d = s / nc, c = s % nc;
    int64_t g = x - seg_start[s];
    if (d > 0) {
      int32_t k = key[x];
      g += pt_off[c + 1] - pt_off[c];
      for (int dd = 1; dd <= maxd; dd++) {
        if (dd == d) continue;
        int64_t lo = seg_start[dd * nc + c], hi = seg_start[dd * nc + c + 1];
        int64_t a = lo, b = hi;
        if (dd < d) {  // count key <= k
          while (a < b) {
            int64_t mid = (a + b) >> 1;
            if (key[mid] <= k) a = mid + 1; else b = mid;
          }
        } else {  // count key < k
          while (a < b) {
            int64_t mid = (a + b) >> 1;
            if (key[mid] < k) a = mid + 1; else b = mid;
          }
        }
        g += a - lo;
      }
    }
    gidx[x] = g;
  }
}

static int bitlen(uint64_t v) {
  int b = 0;
  while (v) {
    b++;
    v >>= 1;
  }
  return b;
}

// common tail of build_vr and load_boundary: segment table, per-id arrays already filled
static void finish_layout(ph_ctx* ctx) {
  ctx->d_seg_start = alloc_n<int64_t>(ctx, (int64_t)ctx->seg_start.size());
  PH_CUDA(cudaMemcpyAsync(ctx->d_seg_start, ctx->seg_start.data(),
                          ctx->seg_start.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                          ctx->stream));
}

// beta of every column (Definition 4): left(i) first, then the largest row per left column
void compute_beta(ph_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  ColLayout L{};
  L.maxd = ctx->max_dim;
  for (int d = 0; d <= ctx->max_dim + 1; d++) L.dimoff[d] = ctx->dimoff[d];
  int64_t rb = 0;
  for (int d = 0; d <= ctx->max_dim; d++) {
    L.rowbase[d] = rb;
    rb += (d > 0 ? d + 1 : 0) * (ctx->dimoff[d + 1] - ctx->dimoff[d]);
  }
  int32_t* left = alloc_n<int32_t>(ctx, ctx->m);
  ctx->beta = alloc_n<int32_t>(ctx, ctx->m);
  PH_CUDA(cudaMemsetAsync(left, 0x7f, ctx->m * sizeof(int32_t), st));  // > every id
  PH_CUDA(cudaMemsetAsync(ctx->beta, 0xff, ctx->m * sizeof(int32_t), st));
  k_left<<<grid_for(ctx, ctx->m, kThreads), kThreads, 0, st>>>(L, ctx->rows0, ctx->col_off,
                                                               left);
  PH_CHECK_LAUNCH();
  k_beta<<<grid_for(ctx, ctx->m, kThreads), kThreads, 0, st>>>(ctx->m, left, ctx->beta);
  PH_CHECK_LAUNCH();
  ctx->dfree(left);
}

// An explicit complex given in filtration order: re-index it dim-major (stable inside each
// dimension, which keeps every order the reduction compares) and store its boundary. A column
// may hold any number of rows of the dimension below (a simplicial, cubical or cellular
// boundary over F2, or a partially reduced matrix R = D V), so columns are kept with offsets.
void load_boundary(ph_ctx* ctx, int64_t m, const int32_t* dims, const int64_t* colptr,
                   const int32_t* rows) {
  cudaStream_t st = ctx->stream;
  PH_REQUIRE(m >= 1 && m < 0x7f000000LL, PH_ERR_INVALID, "m out of range");
  PH_REQUIRE(dims && colptr && rows, PH_ERR_INVALID, "NULL argument");
  int maxd = 0;
  std::vector<int64_t> cnt(kMaxDim + 1, 0);
  for (int64_t j = 0; j < m; j++) {
    PH_REQUIRE(dims[j] >= 0 && dims[j] <= kMaxDim, PH_ERR_INVALID, "dimension out of range");
    maxd = std::max(maxd, (int)dims[j]);
    cnt[dims[j]]++;
  }
  std::vector<int64_t> dimoff(maxd + 2, 0);
  for (int d = 0; d <= maxd; d++) dimoff[d + 1] = dimoff[d] + cnt[d];
  std::vector<int32_t> id_of(m);
  std::vector<int64_t> fill(maxd + 1, 0);
  for (int64_t j = 0; j < m; j++) id_of[j] = (int32_t)(dimoff[dims[j]] + fill[dims[j]]++);
  PH_REQUIRE(colptr[0] == 0, PH_ERR_INVALID, "colptr[0] must be 0");
  std::vector<int64_t> h_off(m + 1, 0);  // column offsets in id order
  for (int64_t j = 0; j < m; j++) {
    const int64_t n = colptr[j + 1] - colptr[j];
    PH_REQUIRE(n >= 0 && (dims[j] > 0 || n == 0), PH_ERR_INVALID,
               "column lengths must be >= 0, and 0 in dimension 0");
    h_off[id_of[j] + 1] = n;
  }
  for (int64_t x = 0; x < m; x++) h_off[x + 1] += h_off[x];
  const int64_t nnz = h_off[m];
  std::vector<int32_t> h_rows(std::max<int64_t>(nnz, 1)), h_seg(m), h_key(m, -1), h_low(m, -1);
  std::vector<int64_t> h_gidx(m);
  std::vector<uint64_t> h_verts(m, ~0ull);
  for (int64_t j = 0; j < m; j++) {
    int d = dims[j];
    int64_t x = id_of[j];
    int64_t n = colptr[j + 1] - colptr[j];
    int64_t base = h_off[x];
    int32_t prev = -1;
    for (int64_t p = 0; p < n; p++) {
      int32_t r = rows[colptr[j] + p];
      PH_REQUIRE(r >= 0 && r < j && dims[r] == d - 1, PH_ERR_INVALID,
                 "rows must be earlier simplices of dimension d - 1");
      PH_REQUIRE(r > prev, PH_ERR_INVALID, "rows must be strictly ascending");
      prev = r;
      h_rows[base + p] = id_of[r];
    }
    h_seg[x] = d;
    h_gidx[x] = j;
    h_low[x] = n > 0 ? id_of[rows[colptr[j + 1] - 1]] : -1;
  }
  ctx->n_clouds = 1;
  ctx->max_dim = maxd;
  ctx->m = m;
  ctx->nnz = nnz;
  ctx->pt_off = {0, cnt[0]};
  for (int d = 0; d <= maxd + 1; d++) ctx->dimoff[d] = dimoff[d];
  ctx->seg_start.assign(dimoff.begin(), dimoff.end());
  ctx->seg = alloc_n<int32_t>(ctx, m);
  ctx->key = alloc_n<int32_t>(ctx, m);
  ctx->low = alloc_n<int32_t>(ctx, m);
  ctx->gidx = alloc_n<int64_t>(ctx, m);
  ctx->verts = alloc_n<uint64_t>(ctx, m);
  ctx->rows0 = alloc_n<int32_t>(ctx, std::max<int64_t>(nnz, 1) + kColSlack);
  ctx->col_off = alloc_n<int64_t>(ctx, m + 1);
  ctx->d2tab = alloc_n<int64_t>(ctx, 1);
  ctx->n_d2 = 0;
  PH_CUDA(cudaMemcpyAsync(ctx->seg, h_seg.data(), m * 4, cudaMemcpyHostToDevice, st));
  PH_CUDA(cudaMemcpyAsync(ctx->key, h_key.data(), m * 4, cudaMemcpyHostToDevice, st));
  PH_CUDA(cudaMemcpyAsync(ctx->low, h_low.data(), m * 4, cudaMemcpyHostToDevice, st));
  PH_CUDA(cudaMemcpyAsync(ctx->gidx, h_gidx.data(), m * 8, cudaMemcpyHostToDevice, st));
  PH_CUDA(cudaMemcpyAsync(ctx->verts, h_verts.data(), m * 8, cudaMemcpyHostToDevice, st));
  PH_CUDA(cudaMemcpyAsync(ctx->rows0, h_rows.data(), std::max<int64_t>(nnz, 1) * 4,
                          cudaMemcpyHostToDevice, st));
  PH_CUDA(cudaMemcpyAsync(ctx->col_off, h_off.data(), (m + 1) * 8, cudaMemcpyHostToDevice, st));
  finish_layout(ctx);
  compute_beta(ctx);
  PH_CUDA(cudaStreamSynchronize(st));
}

void build_vr(ph_ctx* ctx, const int32_t* coords, const int64_t* cloud_offsets, int32_t nc,
              int64_t n_points, int32_t D, int32_t max_dim, int64_t max_diam2,
              int64_t scale_step, int32_t n_scales) {
  cudaStream_t st = ctx->stream;
  PH_REQUIRE(coords != nullptr, PH_ERR_INVALID, "coords is NULL");
  PH_REQUIRE(nc >= 1 && nc <= kMaxClouds, PH_ERR_INVALID, "n_clouds out of range");
  PH_REQUIRE(D >= 1 && D <= 16, PH_ERR_INVALID, "D must be in 1..16");
  PH_REQUIRE(max_dim >= 1 && max_dim <= kMaxVrDim, PH_ERR_INVALID, "max_dim must be 1..5");
  const int vbits = vert_bits_for(max_dim);
  std::vector<int64_t> off(nc + 1);
  if (cloud_offsets) {
    for (int c = 0; c <= nc; c++) off[c] = cloud_offsets[c];
  } else {
    PH_REQUIRE(nc == 1, PH_ERR_INVALID, "cloud_offsets required for several clouds");
    off[0] = 0;
    off[1] = n_points;
  }
  PH_REQUIRE(off[0] == 0 && off[nc] == n_points, PH_ERR_INVALID,
             "cloud_offsets must start at 0 and end at n_points");
  // per cloud: n x n table offsets and, for k = 2..max_dim+1 vertices, the candidate offsets
  const int K = max_dim + 1;  // largest vertex count
  std::vector<int64_t> mo(nc + 1, 0);
  std::vector<std::vector<int64_t>> cand(kVrSlots + 1, std::vector<int64_t>(nc + 1, 0));
  int64_t ncand_all = 0;
  for (int c = 0; c < nc; c++) {
    int64_t n = off[c + 1] - off[c];
    PH_REQUIRE(n >= 1 && n < (1 << vbits) - 1, PH_ERR_CAPACITY,
               max_dim <= 3 ? "each cloud needs 1..4094 points"
                            : "each cloud needs 1..254 points above dimension 3");
    mo[c + 1] = mo[c] + n * n;
    for (int k = 2; k <= kVrSlots; k++)
      cand[k][c + 1] = cand[k][c] + (k <= K ? binom_small(n, k) : 0);
  }
  for (int k = 2; k <= K; k++) ncand_all += cand[k][nc];
  PH_REQUIRE(n_points + ncand_all < INT32_MAX, PH_ERR_CAPACITY,
             "more than 2^31 - 1 candidate simplices");
  ctx->n_clouds = nc;
  ctx->max_dim = max_dim;
  ctx->vbits = vbits;
  ctx->pt_off = off;
  ctx->D = D;
  ctx->n_points = n_points;

  // device copies of the small tables: off, mo, cand[2..kVrSlots]
  const int ntab = 2 + (kVrSlots - 1);
  int64_t* d_tabs = alloc_n<int64_t>(ctx, ntab * (nc + 1));
  std::vector<int64_t> h_tabs;
  h_tabs.insert(h_tabs.end(), off.begin(), off.end());
  h_tabs.insert(h_tabs.end(), mo.begin(), mo.end());
  for (int k = 2; k <= kVrSlots; k++) h_tabs.insert(h_tabs.end(), cand[k].begin(), cand[k].end());
  PH_CUDA(cudaMemcpyAsync(d_tabs, h_tabs.data(), h_tabs.size() * sizeof(int64_t),
                          cudaMemcpyHostToDevice, st));
  CloudTabs ct{d_tabs, d_tabs + (nc + 1), nc, vbits};
  auto d_cand = [&](int k) -> const int64_t* { return d_tabs + (int64_t)k * (nc + 1); };

  // scratch: status words [0] bad coords, [1] max d2, then per-cloud counts of every dimension
  int64_t* d_misc = alloc_n<int64_t>(ctx, 2 + (int64_t)kMaxVrDim * nc);
  PH_CUDA(cudaMemsetAsync(d_misc, 0, (2 + (int64_t)kMaxVrDim * nc) * sizeof(int64_t), st));
  auto cnt_dim = [&](int d) { return d_misc + 2 + (int64_t)(d - 1) * nc; };  // d >= 1
  k_check_coords<<<grid_for(ctx, n_points * D, kThreads), kThreads, 0, st>>>(
      coords, n_points * D, (int32_t*)d_misc);
  PH_CHECK_LAUNCH();

  int64_t nn = mo[nc];
  int64_t* d2 = alloc_n<int64_t>(ctx, nn);
  int32_t* eid = alloc_n<int32_t>(ctx, nn);
  int32_t* erank = alloc_n<int32_t>(ctx, nn);
  PH_CUDA(cudaMemsetAsync(eid, 0xff, nn * sizeof(int32_t), st));
  PH_CUDA(cudaMemsetAsync(erank, 0xff, nn * sizeof(int32_t), st));
  int64_t nmax = 0;
  for (int c = 0; c < nc; c++) nmax = std::max(nmax, off[c + 1] - off[c]);
  {
    dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>((nmax * nmax + 255) / 256, 4096)),
           (unsigned)nc);
    k_pairwise<<<g, kThreads, 0, st>>>(coords, D, ct, d2, (unsigned long long*)(d_misc + 1));
    PH_CHECK_LAUNCH();
  }
  int64_t h_misc[2];
  PH_CUDA(cudaMemcpyAsync(h_misc, d_misc, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  PH_CUDA(cudaStreamSynchronize(st));
  PH_REQUIRE(h_misc[0] == 0, PH_ERR_INVALID, "coordinates must lie in [-2^24, 2^24] grid units");
  int64_t maxkey = h_misc[1];
  if (scale_step > 0) {  // filtration values on the grid of scales: d2 -> scale index
    PH_REQUIRE(n_scales >= 1 && scale_step <= (int64_t)1 << 26, PH_ERR_INVALID,
               "the scale grid needs n_scales >= 1 and a step of at most 2^26 grid units");
    k_scale_index<<<grid_for(ctx, nn, kThreads), kThreads, 0, st>>>(d2, nn, scale_step);
    PH_CHECK_LAUNCH();
    maxkey = scale_index_of(h_misc[1], scale_step);
    max_diam2 = n_scales;  // simplices above the largest scale are left out
  }
  const int d2bits = bitlen((uint64_t)maxkey) + 1;  // one extra bit for the sentinel

  // ---------------- edges ----------------
  int64_t ncand_max = 0;
  for (int k = 2; k <= K; k++) ncand_max = std::max(ncand_max, cand[k][nc]);
  uint64_t* kbuf = alloc_n<uint64_t>(ctx, ncand_max);
  uint64_t* vbuf = alloc_n<uint64_t>(ctx, ncand_max);
  uint64_t* ktmp = alloc_n<uint64_t>(ctx, ncand_max);
  uint64_t* vtmp = alloc_n<uint64_t>(ctx, ncand_max);
  const uint64_t sent_e = (1ull << d2bits) - 1ull;
  std::vector<int64_t> cnts(K, 0);  // simplices per dimension
  cnts[0] = n_points;
  std::vector<int64_t> h_cnt((int64_t)kMaxVrDim * nc, 0);  // per (dimension >= 1, cloud)
  if (cand[2][nc] > 0) {
    k_edge_cand<<<grid_for(ctx, cand[2][nc], kThreads), kThreads, 0, st>>>(
        ct, d_cand(2), cand[2][nc], d2, max_diam2, sent_e, kbuf, vbuf, cnt_dim(1));
    PH_CHECK_LAUNCH();
    radix_sort_u64(ctx, kbuf, vbuf, cand[2][nc], 0, d2bits, ktmp, vtmp);
    if (nc > 1) {
      k_rekey_cloud<<<grid_for(ctx, cand[2][nc], kThreads), kThreads, 0, st>>>(
          vbuf, kbuf, cand[2][nc], sent_e, (uint64_t)nc);
      PH_CHECK_LAUNCH();
      radix_sort_u64(ctx, kbuf, vbuf, cand[2][nc], 0, bitlen((uint64_t)nc), ktmp, vtmp);
    }
  }
  PH_CUDA(cudaMemcpyAsync(h_cnt.data(), cnt_dim(1), nc * sizeof(int64_t), cudaMemcpyDeviceToHost,
                          st));
  PH_CUDA(cudaStreamSynchronize(st));
  for (int c = 0; c < nc; c++) cnts[1] += h_cnt[c];
  const int64_t E = cnts[1];

  // sizes known for dims 0, 1; ids and initial storage for those two now, higher dims after
  // their candidate counts are known. Provisional allocation uses candidate counts as bounds.
  const int64_t N = n_points;
  int64_t m_bound = N + E, nnz_bound = 2 * E;
  for (int k = 3; k <= K; k++) {
    m_bound += cand[k][nc];
    nnz_bound += (int64_t)k * cand[k][nc];
  }
  ctx->seg = alloc_n<int32_t>(ctx, m_bound);
  ctx->key = alloc_n<int32_t>(ctx, m_bound);
  ctx->low = alloc_n<int32_t>(ctx, m_bound);
  ctx->verts = alloc_n<uint64_t>(ctx, m_bound);
  ctx->rows0 = alloc_n<int32_t>(ctx, nnz_bound + kColSlack);
  IdOut o{ctx->seg, ctx->key, ctx->low, ctx->verts, ctx->rows0};

  k_vertex_init<<<grid_for(ctx, N, kThreads), kThreads, 0, st>>>(ct, N, o);
  PH_CHECK_LAUNCH();

  ctx->d2tab = alloc_n<int64_t>(ctx, std::max<int64_t>(E, 1));
  int64_t n_d2 = 0;
  if (E > 0) {
    int64_t* flag = alloc_n<int64_t>(ctx, E);
    int64_t* excl = alloc_n<int64_t>(ctx, E);
    int64_t* ed2 = alloc_n<int64_t>(ctx, E);
    int64_t* d_nd2 = alloc_n<int64_t>(ctx, 1);
    k_edge_newflag<<<grid_for(ctx, E, kThreads), kThreads, 0, st>>>(vbuf, E, ct, d2, flag, ed2);
    PH_CHECK_LAUNCH();
    excl_scan_i64(ctx, flag, excl, E, d_nd2);
    k_edge_finish<<<grid_for(ctx, E, kThreads), kThreads, 0, st>>>(
        vbuf, E, ct, flag, excl, ed2, N, eid, erank, ctx->d2tab, o, 0);
    PH_CHECK_LAUNCH();
    PH_CUDA(cudaMemcpyAsync(&n_d2, d_nd2, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PH_CUDA(cudaStreamSynchronize(st));
    ctx->dfree(flag);
    ctx->dfree(excl);
    ctx->dfree(ed2);
    ctx->dfree(d_nd2);
  }
  ctx->n_d2 = n_d2;
  const int rbits = bitlen((uint64_t)n_d2);  // keys 0..n_d2-1, sentinel n_d2

  // ---------------- dimensions 2..max_dim ----------------
  // id of each simplex by the lexicographic rank of its vertex set, for the next dimension's
  // faces (edges use the n x n table eid instead)
  std::vector<int32_t*> lex_tab(kVrSlots + 1, nullptr);
  int64_t id0 = N + E, rowbase = 2 * E;
  for (int k = 3; k <= K; k++) {
    const int d = k - 1;
    if (k < K) {  // the next dimension looks its faces up here
      lex_tab[k] = alloc_n<int32_t>(ctx, std::max<int64_t>(cand[k][nc], 1));
      PH_CUDA(cudaMemsetAsync(lex_tab[k], 0xff,
                              std::max<int64_t>(cand[k][nc], 1) * sizeof(int32_t), st));
    }
    int64_t Q = 0;
    if (cand[k][nc] > 0) {
      k_simplex_cand<<<grid_for(ctx, cand[k][nc], kThreads), kThreads, 0, st>>>(
          ct, d_cand(k), cand[k][nc], k, erank, (uint64_t)n_d2, kbuf, vbuf, cnt_dim(d));
      PH_CHECK_LAUNCH();
      radix_sort_u64(ctx, kbuf, vbuf, cand[k][nc], 0, rbits, ktmp, vtmp);
      PH_CUDA(cudaMemcpyAsync(h_cnt.data() + (int64_t)(d - 1) * nc, cnt_dim(d),
                              nc * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      PH_CUDA(cudaStreamSynchronize(st));
      for (int c = 0; c < nc; c++) Q += h_cnt[(int64_t)(d - 1) * nc + c];
    }
    if (Q > 0) {
      if (k == 3) {
        k_tri_finish<<<grid_for(ctx, Q, kThreads), kThreads, 0, st>>>(
            kbuf, vbuf, Q, ct, eid, id0, o, rowbase, lex_tab[3], d_cand(3));
      } else {
        k_high_finish<<<grid_for(ctx, Q, kThreads), kThreads, 0, st>>>(
            kbuf, vbuf, Q, k, ct, lex_tab[k - 1], d_cand(k - 1), lex_tab[k], d_cand(k), id0, o,
            rowbase);
      }
      PH_CHECK_LAUNCH();
    }
    cnts[d] = Q;
    id0 += Q;
    rowbase += (int64_t)k * Q;
  }

  // ---------------- layout ----------------
  ctx->m = 0;
  ctx->nnz = 0;
  for (int d = 0; d <= max_dim; d++) {
    ctx->m += cnts[d];
    if (d > 0) ctx->nnz += (int64_t)(d + 1) * cnts[d];
  }
  ctx->dimoff[0] = 0;
  for (int d = 0; d <= max_dim; d++) ctx->dimoff[d + 1] = ctx->dimoff[d] + cnts[d];
  ctx->seg_start.assign((max_dim + 1) * nc + 1, 0);
  int64_t pos = 0;
  for (int d = 0; d <= max_dim; d++)
    for (int c = 0; c < nc; c++) {
      ctx->seg_start[d * nc + c] = pos;
      pos += d == 0 ? off[c + 1] - off[c] : h_cnt[(int64_t)(d - 1) * nc + c];
    }
  ctx->seg_start[(max_dim + 1) * nc] = pos;
  finish_layout(ctx);

  compute_beta(ctx);

  ctx->gidx = alloc_n<int64_t>(ctx, ctx->m);
  k_gidx<<<grid_for(ctx, ctx->m, kThreads), kThreads, 0, st>>>(
      ctx->m, nc, max_dim, ctx->seg, ctx->key, ctx->d_seg_start, d_tabs, ctx->gidx);
  PH_CHECK_LAUNCH();
  PH_CUDA(cudaStreamSynchronize(st));

  ctx->dfree(kbuf);
  ctx->dfree(vbuf);
  ctx->dfree(ktmp);
  ctx->dfree(vtmp);
  ctx->dfree(d2);
  ctx->dfree(eid);
  ctx->dfree(erank);
  for (int32_t* t : lex_tab)
    if (t) ctx->dfree(t);
  ctx->dfree(d_misc);
  // d_tabs holds pt_off, needed by extraction: keep it alive as ctx->... (freed with ctx)
}

}  // namespace ph
