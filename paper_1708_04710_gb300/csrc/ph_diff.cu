// Differentiable persistence diagrams: a loss over the finite pairs of one dimension and its
// gradient with respect to the point coordinates.
//
// The pairing (which simplex kills which, Lemma 1) is computed exactly from grid-rounded
// coordinates and is piecewise constant in the coordinates, so it carries no gradient. The
// birth and death values of a pair are Euclidean diameters (Sec. 2.2, VR: f_r(sigma) =
// 1{diam(sigma) <= 2r}); a simplex's diameter is the length of one of its edges, its realising
// edge: an edge realises itself, a higher simplex is realised by the realising edge of its last
// face in the filtration (the largest row of its boundary column), which has the same diameter.
// For a pair with realising edges (p, q) at birth and (r, s) at death,
//   b = |x_p - x_q|, d = |x_r - x_s|, loss = sum over pairs of (d - b)^2,
//   dloss/dx_r = 2 (d - b) (x_r - x_s) / d,  dloss/dx_s = -dloss/dx_r,
//   dloss/dx_p = -2 (d - b) (x_p - x_q) / b, dloss/dx_q = -dloss/dx_p,
// with the term of a zero-length edge left out (its direction is undefined).
#include <cmath>

#include "ph_internal.cuh"

namespace ph {

struct DiagLayout {
  int64_t dimoff[kMaxDim + 2];
  int64_t rowbase[kMaxDim + 2];
  int maxd;
  int nc;
  int vbits;  // bits per packed vertex of the build
};

__global__ void k_to_grid(const float* __restrict__ x, int64_t n, int32_t* g, int32_t* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i] * 65536.0f;  // exact: a power-of-two scaling
    if (!(fabsf(v) <= 16777216.0f)) {  // also catches NaN
      *bad = 1;
      g[i] = 0;
    } else {
      g[i] = __float2int_rn(v);  // round half to even
    }
  }
}

// the realising edge of simplex x (an id of dimension >= 1): follow the last face down to an
// edge; returns the two point indices (global rows of the coordinate array)
__device__ __forceinline__ void realising_edge(const DiagLayout& L, const int32_t* __restrict__ rows0,
                                               const uint64_t* __restrict__ verts,
                                               const int64_t* __restrict__ pt_off, int64_t x,
                                               int64_t& p, int64_t& q) {
  int d = 0;
  while (d < L.maxd && x >= L.dimoff[d + 1]) d++;
  while (d > 1) {
    x = rows0[L.rowbase[d] + (int64_t)(d + 1) * (x - L.dimoff[d]) + d];  // largest row
    d--;
  }
  const uint64_t v = verts[x];
  const int64_t base = pt_off[(int)(v >> 48)];
  p = base + (int64_t)packed_vert_at(v, 0, L.vbits);
  q = base + (int64_t)packed_vert_at(v, 1, L.vbits);
}

__device__ __forceinline__ float edge_len(const float* __restrict__ x, int D, int64_t p,
                                          int64_t q) {
  float s = 0.f;
  for (int k = 0; k < D; k++) {
    const float t = x[p * D + k] - x[q * D + k];
    s += t * t;
  }
  return sqrtf(s);
}

// one block per cloud: the finite pairs whose death simplex has dimension dd = dim + 1 are the
// columns of segment (dd, cloud) with a low; the block sums their terms in a fixed order
__global__ void k_diag_loss(DiagLayout L, int dd, const int64_t* __restrict__ seg_start,
                            const int32_t* __restrict__ low, const int32_t* __restrict__ rows0,
                            const uint64_t* __restrict__ verts, const int64_t* __restrict__ pt_off,
                            const float* __restrict__ x, int D, float* loss,
                            unsigned long long* npairs) {
  __shared__ float sh[kThreads];
  const int c = blockIdx.x;
  const int64_t lo = seg_start[dd * L.nc + c], hi = seg_start[dd * L.nc + c + 1];
  float acc = 0.f;
  unsigned long long cnt = 0;
  for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    const int32_t b = low[j];
    if (b < 0) continue;
    int64_t r, s;
    realising_edge(L, rows0, verts, pt_off, j, r, s);
    const float dlen = edge_len(x, D, r, s);
    float blen = 0.f;
    if (dd >= 2) {
      int64_t p, q;
      realising_edge(L, rows0, verts, pt_off, b, p, q);
      blen = edge_len(x, D, p, q);
    }
    const float t = dlen - blen;
    acc += t * t;
    cnt++;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[c] = sh[0];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(npairs, cnt);
}

__global__ void k_diag_total(const float* __restrict__ loss, int nc, float* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int c = 0; c < nc; c++) s += loss[c];
    *total = s;
  }
}

__global__ void k_diag_bwd(DiagLayout L, int dd, int64_t lo, int64_t hi,
                           const int32_t* __restrict__ seg, const int32_t* __restrict__ low,
                           const int32_t* __restrict__ rows0, const uint64_t* __restrict__ verts,
                           const int64_t* __restrict__ pt_off, const float* __restrict__ x, int D,
                           const float* __restrict__ gloss, float* grad) {
  for (int64_t j = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < hi;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = low[j];
    if (b < 0) continue;
    const int c = seg[j] % L.nc;
    int64_t r, s, p = -1, q = -1;
    realising_edge(L, rows0, verts, pt_off, j, r, s);
    const float dlen = edge_len(x, D, r, s);
    float blen = 0.f;
    if (dd >= 2) {
      realising_edge(L, rows0, verts, pt_off, b, p, q);
      blen = edge_len(x, D, p, q);
    }
    const float g = 2.f * (dlen - blen) * gloss[c];
    if (dlen > 0.f) {
      const float f = g / dlen;
      for (int k = 0; k < D; k++) {
        const float t = f * (x[r * D + k] - x[s * D + k]);
        atomicAdd(&grad[r * D + k], t);
        atomicAdd(&grad[s * D + k], -t);
      }
    }
    if (p >= 0 && blen > 0.f) {
      const float f = g / blen;
      for (int k = 0; k < D; k++) {
        const float t = f * (x[p * D + k] - x[q * D + k]);
        atomicAdd(&grad[p * D + k], -t);
        atomicAdd(&grad[q * D + k], t);
      }
    }
  }
}

static DiagLayout layout_of(ph_ctx* ctx) {
  DiagLayout L{};
  L.maxd = ctx->max_dim;
  L.vbits = ctx->vbits;
  L.nc = ctx->n_clouds;
  int64_t rb = 0;
  for (int d = 0; d <= ctx->max_dim + 1; d++) L.dimoff[d] = ctx->dimoff[d];
  for (int d = 0; d <= ctx->max_dim; d++) {
    L.rowbase[d] = rb;
    rb += (d > 0 ? d + 1 : 0) * (ctx->dimoff[d + 1] - ctx->dimoff[d]);
  }
  return L;
}

}  // namespace ph

#define PH_API_BEGIN \
  if (!ctx) return PH_ERR_INVALID; \
  ctx->err.clear();                \
  try {
#define PH_API_END                                    \
  }                                                   \
  catch (const ph::Fail& f) {                         \
    return f.code;                                    \
  }                                                   \
  catch (...) {                                       \
    ctx->err = "unexpected failure";                  \
    return PH_ERR_INVALID;                            \
  }

extern "C" {

int ph_build_filtration_f32(ph_ctx* ctx, const float* coords, const int64_t* cloud_offsets,
                            int32_t n_clouds, int64_t n_points, int32_t D, int32_t max_dim,
                            int64_t max_diam2, int64_t* m_out) {
  PH_API_BEGIN
  PH_REQUIRE(coords != nullptr && n_points >= 1 && D >= 1 && D <= 16, PH_ERR_INVALID,
             "bad coordinates");
  ctx->free_all();
  const int64_t n = n_points * D;
  // the rounded copy lives with the filtration (freed with it)
  int32_t* g = ph::alloc_n<int32_t>(ctx, n);
  int32_t* bad = ph::alloc_n<int32_t>(ctx, 1);
  PH_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), ctx->stream));
  ph::k_to_grid<<<ph::grid_for(ctx, n, ph::kThreads), ph::kThreads, 0, ctx->stream>>>(coords, n,
                                                                                     g, bad);
  PH_CHECK_LAUNCH();
  int32_t h_bad = 0;
  PH_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  PH_REQUIRE(h_bad == 0, PH_ERR_INVALID, "coordinates must be finite with |x| <= 256");
  ph::build_vr(ctx, g, cloud_offsets, n_clouds, n_points, D, max_dim, max_diam2);
  ctx->built = true;
  ctx->is_vr = true;
  if (m_out) *m_out = ctx->m;
  return PH_OK;
  PH_API_END
}

int ph_diagram_loss(ph_ctx* ctx, const float* coords, int32_t D, int32_t dim, float* loss,
                    int64_t* n_pairs) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(ctx->is_vr, PH_ERR_INVALID, "diagram losses need a filtration built from points");
  PH_REQUIRE(coords && loss, PH_ERR_INVALID, "NULL argument");
  PH_REQUIRE(dim >= 0 && dim + 1 <= ctx->max_dim, PH_ERR_INVALID,
             "dim + 1 must not exceed the filtration's max_dim");
  // the kernels index coords by the build's point rows: any other shape reads out of bounds
  PH_REQUIRE(D == ctx->D, PH_ERR_INVALID,
             "D must equal the D of the build (" + std::to_string(ctx->D) + ")");
  const ph::DiagLayout L = ph::layout_of(ctx);
  unsigned long long* cnt = ph::alloc_n<unsigned long long>(ctx, 1);
  int64_t* d_pt = ph::alloc_n<int64_t>(ctx, ctx->n_clouds + 1);
  PH_CUDA(cudaMemcpyAsync(d_pt, ctx->pt_off.data(), (ctx->n_clouds + 1) * sizeof(int64_t),
                          cudaMemcpyHostToDevice, ctx->stream));
  PH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), ctx->stream));
  ph::k_diag_loss<<<ctx->n_clouds, ph::kThreads, 0, ctx->stream>>>(
      L, dim + 1, ctx->d_seg_start, ctx->low, ctx->rows0, ctx->verts, d_pt, coords, D, loss, cnt);
  PH_CHECK_LAUNCH();
  ph::k_diag_total<<<1, 32, 0, ctx->stream>>>(loss, ctx->n_clouds, loss + ctx->n_clouds);
  PH_CHECK_LAUNCH();
  unsigned long long h = 0;
  PH_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->dfree(cnt);
  ctx->dfree(d_pt);
  if (n_pairs) *n_pairs = (int64_t)h;
  return PH_OK;
  PH_API_END
}

int ph_diagram_backward(ph_ctx* ctx, const float* coords, int32_t D, int32_t dim,
                        const float* grad_loss, float* grad_coords) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(ctx->is_vr, PH_ERR_INVALID, "diagram losses need a filtration built from points");
  PH_REQUIRE(coords && grad_loss && grad_coords, PH_ERR_INVALID, "NULL argument");
  PH_REQUIRE(dim >= 0 && dim + 1 <= ctx->max_dim, PH_ERR_INVALID,
             "dim + 1 must not exceed the filtration's max_dim");
  PH_REQUIRE(D == ctx->D, PH_ERR_INVALID,
             "D must equal the D of the build (" + std::to_string(ctx->D) + ")");
  const ph::DiagLayout L = ph::layout_of(ctx);
  int64_t* d_pt = ph::alloc_n<int64_t>(ctx, ctx->n_clouds + 1);
  PH_CUDA(cudaMemcpyAsync(d_pt, ctx->pt_off.data(), (ctx->n_clouds + 1) * sizeof(int64_t),
                          cudaMemcpyHostToDevice, ctx->stream));
  const int64_t lo = ctx->dimoff[dim + 1], hi = ctx->dimoff[dim + 2];
  ph::k_diag_bwd<<<ph::grid_for(ctx, hi - lo, ph::kThreads), ph::kThreads, 0, ctx->stream>>>(
      L, dim + 1, lo, hi, ctx->seg, ctx->low, ctx->rows0, ctx->verts, d_pt, coords, D, grad_loss,
      grad_coords);
  PH_CHECK_LAUNCH();
  ctx->dfree(d_pt);
  return PH_OK;
  PH_API_END
}

}  // extern "C"
