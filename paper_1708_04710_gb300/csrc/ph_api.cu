// C ABI of the library: context life cycle, device memory, extraction of pairs and essential
// simplices (Lemma 1, Eq. paired), and inspection of the filtration.
#include <algorithm>
#include <cstring>
#include <new>

#include "ph_internal.cuh"

// ---------------------------------------------------------------------------------------------
// device memory of a context
// ---------------------------------------------------------------------------------------------
void* ph_ctx::dalloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (has_alloc) {
    p = alloc.alloc(bytes, alloc.user, (void*)stream);
  } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) {
    err = "device allocation of " + std::to_string(bytes) + " bytes failed";
    throw ph::Fail{PH_ERR_ALLOC};
  }
  if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {  // the kernels copy in 16-byte units
    if (has_alloc) alloc.free(p, bytes, alloc.user, (void*)stream);
    else cudaFreeAsync(p, stream);
    err = "the device allocator returned memory that is not 256-byte aligned";
    throw ph::Fail{PH_ERR_ALLOC};
  }
  blocks.push_back({p, bytes});
  return p;
}

void ph_ctx::dfree(void* p) {
  if (!p) return;
  for (size_t i = 0; i < blocks.size(); i++) {
    if (blocks[i].p == p) {
      if (has_alloc) alloc.free(p, blocks[i].bytes, alloc.user, (void*)stream);
      else cudaFreeAsync(p, stream);
      blocks[i] = blocks.back();
      blocks.pop_back();
      return;
    }
  }
}

void ph_ctx::free_all() {
  ph::free_reduce_state(this);
  for (auto& b : blocks) {
    if (has_alloc) alloc.free(b.p, b.bytes, alloc.user, (void*)stream);
    else cudaFreeAsync(b.p, stream);
  }
  blocks.clear();
  built = reduced = extracted = is_vr = false;
  // every pointer into the freed blocks must go: a stale one handed to dfree later could match
  // a new allocation at the same address and free it while it is in use
  p_birth = p_death = p_bd2 = p_dd2 = e_idx = e_d2 = nullptr;
  p_dim = e_dim = nullptr;
  seg = low = beta = key = rows0 = nullptr;
  col_off = nullptr;
  gidx = nullptr;
  verts = nullptr;
  d2tab = nullptr;
  d_seg_start = nullptr;
  m = nnz = 0;
  D = 0;
  n_points = 0;
}

namespace ph {

// ---------------------------------------------------------------------------------------------
// extraction: pairs (low(j), j) for low(j) >= 0 and essential simplices (low(j) = -1 and j not
// the low of any column), written per cloud, ordered by (dimension, index)
// ---------------------------------------------------------------------------------------------
__global__ void k_mark_image(int64_t m, const int32_t* __restrict__ low, uint8_t* is_low) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    int32_t l = low[x];
    if (l >= 0) is_low[l] = 1;
  }
}

__global__ void k_out_flags(int64_t m, const int32_t* __restrict__ low,
                            const uint8_t* __restrict__ is_low, int64_t* fp, int64_t* fe) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    int32_t l = low[x];
    fp[x] = l >= 0;
    fe[x] = l < 0 && !is_low[x];
  }
}

__global__ void k_gather_seg(int nseg, const int64_t* __restrict__ seg_start,
                             const int64_t* __restrict__ pp, const int64_t* __restrict__ pe,
                             int64_t* out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= nseg; s += gridDim.x * blockDim.x) {
    out[2 * s] = pp[seg_start[s]];
    out[2 * s + 1] = pe[seg_start[s]];
  }
}

__device__ __forceinline__ int64_t diam2_of(const int32_t* key, const int64_t* d2tab, int32_t x) {
  int32_t k = key[x];
  return k >= 0 ? d2tab[k] : 0;
}

__global__ void k_write_out(int64_t m, int nc, const int32_t* __restrict__ seg,
                            const int32_t* __restrict__ low, const uint8_t* __restrict__ is_low,
                            const int64_t* __restrict__ gidx, const int32_t* __restrict__ key,
                            const int64_t* __restrict__ d2tab, const int64_t* __restrict__ pp,
                            const int64_t* __restrict__ pe, const int64_t* __restrict__ segtab,
                            int64_t* p_birth, int64_t* p_death, int32_t* p_dim, int64_t* p_bd2,
                            int64_t* p_dd2, int64_t* e_idx, int32_t* e_dim, int64_t* e_d2,
                            int64_t n_pairs, int64_t n_ess, int32_t* bad) {
  // segtab: per segment [first pair pos, first ess pos, out base pairs, out base ess]
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < m;
       x += (int64_t)gridDim.x * blockDim.x) {
    int s = seg[x];
    int32_t l = low[x];
    const int64_t* t = segtab + 4 * s;
    if (l >= 0) {
      int64_t o = t[2] + pp[x] - t[0];
      if (o < 0 || o >= n_pairs) {
        *bad = 1;
        continue;
      }
      p_birth[o] = gidx[l];
      p_death[o] = gidx[x];
      p_dim[o] = s / nc - 1;
      p_bd2[o] = diam2_of(key, d2tab, l);
      p_dd2[o] = diam2_of(key, d2tab, (int32_t)x);
    } else if (!is_low[x]) {
      int64_t o = t[3] + pe[x] - t[1];
      if (o < 0 || o >= n_ess) {
        *bad = 1;
        continue;
      }
      e_idx[o] = gidx[x];
      e_dim[o] = s / nc;
      e_d2[o] = diam2_of(key, d2tab, (int32_t)x);
    }
  }
}

void extract_all(ph_ctx* ctx) {
  if (ctx->extracted) return;
  for (void* p : {(void*)ctx->p_birth, (void*)ctx->p_death, (void*)ctx->p_dim, (void*)ctx->p_bd2,
                  (void*)ctx->p_dd2, (void*)ctx->e_idx, (void*)ctx->e_dim, (void*)ctx->e_d2})
    ctx->dfree(p);
  cudaStream_t st = ctx->stream;
  const int64_t m = ctx->m;
  const int nc = ctx->n_clouds;
  const int nseg = (int)ctx->seg_start.size() - 1;
  uint8_t* is_low = alloc_n<uint8_t>(ctx, m);
  int64_t* fp = alloc_n<int64_t>(ctx, m + 1);
  int64_t* fe = alloc_n<int64_t>(ctx, m + 1);
  int64_t* pp = alloc_n<int64_t>(ctx, m + 1);
  int64_t* pe = alloc_n<int64_t>(ctx, m + 1);
  PH_CUDA(cudaMemsetAsync(is_low, 0, m, st));
  PH_CUDA(cudaMemsetAsync(fp + m, 0, sizeof(int64_t), st));
  PH_CUDA(cudaMemsetAsync(fe + m, 0, sizeof(int64_t), st));
  k_mark_image<<<grid_for(ctx, m, kThreads), kThreads, 0, st>>>(m, ctx->low, is_low);
  PH_CHECK_LAUNCH();
  k_out_flags<<<grid_for(ctx, m, kThreads), kThreads, 0, st>>>(m, ctx->low, is_low, fp, fe);
  PH_CHECK_LAUNCH();
  excl_scan_i64(ctx, fp, pp, m + 1, nullptr);
  excl_scan_i64(ctx, fe, pe, m + 1, nullptr);
  int64_t* d_sg = alloc_n<int64_t>(ctx, 2 * (nseg + 1));
  k_gather_seg<<<1, kThreads, 0, st>>>(nseg, ctx->d_seg_start, pp, pe, d_sg);
  PH_CHECK_LAUNCH();
  std::vector<int64_t> sg(2 * (nseg + 1));
  PH_CUDA(cudaMemcpyAsync(sg.data(), d_sg, sg.size() * sizeof(int64_t), cudaMemcpyDeviceToHost,
                          st));
  PH_CUDA(cudaStreamSynchronize(st));
  // output bases: clouds in order, inside a cloud dimensions in order
  const int ndim = ctx->max_dim + 1;
  std::vector<int64_t> segtab(4 * nseg);
  ctx->pair_off.assign(nc + 1, 0);
  ctx->ess_off.assign(nc + 1, 0);
  int64_t bp = 0, be = 0;
  for (int c = 0; c < nc; c++) {
    ctx->pair_off[c] = bp;
    ctx->ess_off[c] = be;
    for (int d = 0; d < ndim; d++) {
      int s = d * nc + c;
      segtab[4 * s] = sg[2 * s];
      segtab[4 * s + 1] = sg[2 * s + 1];
      segtab[4 * s + 2] = bp;
      segtab[4 * s + 3] = be;
      bp += sg[2 * (s + 1)] - sg[2 * s];
      be += sg[2 * (s + 1) + 1] - sg[2 * s + 1];
    }
  }
  ctx->pair_off[nc] = bp;
  ctx->ess_off[nc] = be;
  ctx->n_pairs = bp;
  ctx->n_ess = be;
  PH_CUDA(cudaMemsetAsync(d_sg, 0, sizeof(int64_t), st));  // reused as the error flag
  int64_t* d_segtab = alloc_n<int64_t>(ctx, 4 * nseg);
  PH_CUDA(cudaMemcpyAsync(d_segtab, segtab.data(), segtab.size() * sizeof(int64_t),
                          cudaMemcpyHostToDevice, st));
  ctx->p_birth = alloc_n<int64_t>(ctx, bp);
  ctx->p_death = alloc_n<int64_t>(ctx, bp);
  ctx->p_dim = alloc_n<int32_t>(ctx, bp);
  ctx->p_bd2 = alloc_n<int64_t>(ctx, bp);
  ctx->p_dd2 = alloc_n<int64_t>(ctx, bp);
  ctx->e_idx = alloc_n<int64_t>(ctx, be);
  ctx->e_dim = alloc_n<int32_t>(ctx, be);
  ctx->e_d2 = alloc_n<int64_t>(ctx, be);
  k_write_out<<<grid_for(ctx, m, kThreads), kThreads, 0, st>>>(
      m, nc, ctx->seg, ctx->low, is_low, ctx->gidx, ctx->key, ctx->d2tab, pp, pe, d_segtab,
      ctx->p_birth, ctx->p_death, ctx->p_dim, ctx->p_bd2, ctx->p_dd2, ctx->e_idx, ctx->e_dim,
      ctx->e_d2, bp, be, (int32_t*)d_sg);
  PH_CHECK_LAUNCH();
  int32_t bad = 0;
  PH_CUDA(cudaMemcpyAsync(&bad, d_sg, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  PH_CUDA(cudaStreamSynchronize(st));
  PH_REQUIRE(bad == 0, PH_ERR_INVALID, "internal error: extraction index out of range");
  for (void* p : {(void*)is_low, (void*)fp, (void*)fe, (void*)pp, (void*)pe, (void*)d_sg,
                  (void*)d_segtab})
    ctx->dfree(p);
  ctx->extracted = true;
}

__global__ void k_inspect(int64_t lo, int64_t hi, const int32_t* __restrict__ seg, int nc,
                          const int64_t* __restrict__ gidx, const int32_t* __restrict__ key,
                          const int64_t* __restrict__ d2tab, const uint64_t* __restrict__ verts,
                          const int32_t* __restrict__ beta, const int32_t* __restrict__ low,
                          int32_t* o_dim, int64_t* o_d2, int32_t* o_v, int32_t* o_beta,
                          int32_t* o_low, int64_t n, int vbits, int32_t* bad) {
  for (int64_t x = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < hi;
       x += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = gidx[x];
    if (g < 0 || g >= n) {
      *bad = 1;
      continue;
    }
    int d = seg[x] / nc;
    o_dim[g] = d;
    o_d2[g] = diam2_of(key, d2tab, (int32_t)x);
    uint64_t p = verts[x];
    for (int q = 0; q < kVrSlots; q++)
      o_v[kVrSlots * g + q] = (p == ~0ull || q > d) ? -1 : packed_vert_at(p, q, vbits);
    o_beta[g] = beta[x] >= 0 ? (int32_t)gidx[beta[x]] : -1;
    o_low[g] = low[x] >= 0 ? (int32_t)gidx[low[x]] : -1;
  }
}

}  // namespace ph

// ---------------------------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------------------------
#define PH_API_BEGIN                  \
  if (!ctx) return PH_ERR_INVALID;    \
  ctx->err.clear();                   \
  ph::NvtxRange nvtx_range_(__func__); \
  try {
#define PH_API_END                                    \
  }                                                   \
  catch (const ph::Fail& f) {                         \
    return f.code;                                    \
  }                                                   \
  catch (const std::bad_alloc&) {                     \
    ctx->err = "host allocation failed";              \
    return PH_ERR_ALLOC;                              \
  }                                                   \
  catch (...) {                                       \
    ctx->err = "unexpected failure";                  \
    return PH_ERR_INVALID;                            \
  }

extern "C" {

void ph_default_opts(ph_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->strict_phase2 = 0;
  o->use_cor10 = 1;
  o->lane_merge_words = 0;
  o->staged_merge_max = 0;
  o->merge_items = 0;
  o->collect_stats = 0;
  o->use_graph = 1;
  o->time_kernels = 0;
  o->add_blocks_per_sm = 0;
  o->timeout_ms = 0;
  o->predict_pairs = 0;
  o->dense_threshold = 0;
  o->warp_chunks_below = 0;
  o->warp_chunk_words = 0;
  o->narrow_chunks_below = 0;
  o->phase2_sets = 0;
  o->phase2_priority = 0;
  o->arena_words = 0;
}

int ph_create(ph_ctx** out, const ph_opts* opts, const ph_allocator* alloc, void* stream) {
  if (!out) return PH_ERR_INVALID;
  *out = nullptr;
  ph_ctx* ctx = new (std::nothrow) ph_ctx();
  if (!ctx) return PH_ERR_ALLOC;
  if (opts) ctx->opts = *opts;
  else ph_default_opts(&ctx->opts);
  if (ctx->opts.phase2_priority < 0 || ctx->opts.phase2_priority > 1) {
    delete ctx;
    return PH_ERR_INVALID;
  }
  if (alloc && alloc->alloc && alloc->free) {
    ctx->alloc = *alloc;
    ctx->has_alloc = true;
  }
  ctx->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
          cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return PH_ERR_CUDA;
  }
  *out = ctx;
  return PH_OK;
}

void ph_destroy(ph_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ctx->free_all();
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

int ph_build_filtration(ph_ctx* ctx, const int32_t* coords, const int64_t* cloud_offsets,
                        int32_t n_clouds, int64_t n_points, int32_t D, int32_t max_dim,
                        int64_t max_diam2, int64_t* m_out) {
  PH_API_BEGIN
  ctx->free_all();
  ph::build_vr(ctx, coords, cloud_offsets, n_clouds, n_points, D, max_dim, max_diam2);
  ctx->built = true;
  ctx->is_vr = true;
  if (m_out) *m_out = ctx->m;
  return PH_OK;
  PH_API_END
}

int ph_build_filtration_scales(ph_ctx* ctx, const int32_t* coords, const int64_t* cloud_offsets,
                               int32_t n_clouds, int64_t n_points, int32_t D, int32_t max_dim,
                               int64_t scale_step, int32_t n_scales, int64_t* m_out) {
  PH_API_BEGIN
  PH_REQUIRE(scale_step >= 1, PH_ERR_INVALID, "scale_step must be >= 1 grid unit");
  ctx->free_all();
  ph::build_vr(ctx, coords, cloud_offsets, n_clouds, n_points, D, max_dim, -1, scale_step,
               n_scales);
  ctx->built = true;
  ctx->is_vr = true;
  if (m_out) *m_out = ctx->m;
  return PH_OK;
  PH_API_END
}

int ph_load_boundary(ph_ctx* ctx, int64_t m, const int32_t* dims, const int64_t* colptr,
                     const int32_t* rows) {
  PH_API_BEGIN
  ctx->free_all();
  ph::load_boundary(ctx, m, dims, colptr, rows);
  ctx->built = true;
  return PH_OK;
  PH_API_END
}

int ph_reduce(ph_ctx* ctx, int32_t max_passes, ph_stats* out) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->built, PH_ERR_INVALID, "no filtration: call ph_build_filtration first");
  if (!ctx->rs.init) ph::reduce_init(ctx);
  int rc = ctx->rs.status;
  if (!(ctx->rs.done && ctx->rs.status == PH_OK)) rc = ph::reduce_run(ctx, max_passes);
  ctx->extracted = false;
  ctx->reduced = true;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->passes = ctx->rs.passes;
    out->status = rc;
    out->m = ctx->m;
    const auto& hs = ctx->rs.h_stats;
    for (size_t r = 0; r + PH_PS_N <= hs.size(); r += PH_PS_N) {
      out->col_adds += hs[r + PH_PS_ADDS];
      out->xors += hs[r + PH_PS_XORS];
      // algorithmic bytes: per active column per pass 4 (low) + 4 (table atomic) + 4 (table
      // read) + 1 (flags) + 8 (active list) + 8 (scan) = 29; per addition 8 bytes per XOR
      // (4 * (|src| + |tgt| + |out|) = 8 * |src union tgt|)
      out->alg_bytes += 29 * hs[r + PH_PS_ACTIVE] + 8 * hs[r + PH_PS_XORS];
      out->add_bytes += 8 * hs[r + PH_PS_XORS] + 8 * hs[r + PH_PS_COPIED] +
                        40 * hs[r + PH_PS_ACTIVE];
    }
    out->add_launches = ctx->rs.add_launches;
    out->ms_add = ctx->rs.ms_add;
  }
  return rc;
  PH_API_END
}

int ph_reset_reduction(ph_ctx* ctx) {
  PH_API_BEGIN
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  ph::free_reduce_state(ctx);
  for (void* p : {(void*)ctx->p_birth, (void*)ctx->p_death, (void*)ctx->p_dim, (void*)ctx->p_bd2,
                  (void*)ctx->p_dd2, (void*)ctx->e_idx, (void*)ctx->e_dim, (void*)ctx->e_d2})
    ctx->dfree(p);
  ctx->p_birth = ctx->p_death = ctx->p_bd2 = ctx->p_dd2 = ctx->e_idx = ctx->e_d2 = nullptr;
  ctx->p_dim = ctx->e_dim = nullptr;
  ctx->reduced = ctx->extracted = false;
  return PH_OK;
  PH_API_END
}

int ph_get_pass_stats(ph_ctx* ctx, int64_t* out, int32_t max_rows, int32_t* rows_out) {
  PH_API_BEGIN
  const auto& hs = ctx->rs.h_stats;
  int32_t rows = (int32_t)(hs.size() / PH_PS_N);
  if (rows_out) *rows_out = rows;
  if (out) std::memcpy(out, hs.data(), (size_t)std::min(rows, max_rows) * PH_PS_N * 8);
  return PH_OK;
  PH_API_END
}

int ph_get_add_times(ph_ctx* ctx, float* out, int32_t max_n, int32_t* n_out) {
  PH_API_BEGIN
  const auto& v = ctx->rs.add_ms;
  if (n_out) *n_out = (int32_t)v.size();
  if (out) std::memcpy(out, v.data(), sizeof(float) * std::min<size_t>(v.size(), (size_t)max_n));
  return PH_OK;
  PH_API_END
}

static void copy_out(ph_ctx* ctx, void* dst, const void* src, size_t bytes, int on_device) {
  if (!dst || bytes == 0) return;
  PH_CUDA(cudaMemcpyAsync(dst, src, bytes,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          ctx->stream));
}

int ph_get_pairs(ph_ctx* ctx, int32_t cloud, int64_t* birth, int64_t* death, int32_t* dim,
                 int64_t* birth_diam2, int64_t* death_diam2, int64_t capacity, int64_t* count,
                 int32_t on_device) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(cloud >= -1 && cloud < ctx->n_clouds, PH_ERR_INVALID, "cloud out of range");
  ph::extract_all(ctx);
  int64_t a = cloud < 0 ? 0 : ctx->pair_off[cloud];
  int64_t n = (cloud < 0 ? ctx->pair_off[ctx->n_clouds] : ctx->pair_off[cloud + 1]) - a;
  if (count) *count = n;
  if (!birth && !death && !dim && !birth_diam2 && !death_diam2) return PH_OK;
  PH_REQUIRE(capacity >= n, PH_ERR_CAPACITY, "output capacity too small");
  copy_out(ctx, birth, ctx->p_birth + a, n * 8, on_device);
  copy_out(ctx, death, ctx->p_death + a, n * 8, on_device);
  copy_out(ctx, dim, ctx->p_dim + a, n * 4, on_device);
  copy_out(ctx, birth_diam2, ctx->p_bd2 + a, n * 8, on_device);
  copy_out(ctx, death_diam2, ctx->p_dd2 + a, n * 8, on_device);
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  return PH_OK;
  PH_API_END
}

int ph_get_essential(ph_ctx* ctx, int32_t cloud, int64_t* idx, int32_t* dim, int64_t* diam2,
                     int64_t capacity, int64_t* count, int32_t on_device) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(cloud >= -1 && cloud < ctx->n_clouds, PH_ERR_INVALID, "cloud out of range");
  ph::extract_all(ctx);
  int64_t a = cloud < 0 ? 0 : ctx->ess_off[cloud];
  int64_t n = (cloud < 0 ? ctx->ess_off[ctx->n_clouds] : ctx->ess_off[cloud + 1]) - a;
  if (count) *count = n;
  if (!idx && !dim && !diam2) return PH_OK;
  PH_REQUIRE(capacity >= n, PH_ERR_CAPACITY, "output capacity too small");
  copy_out(ctx, idx, ctx->e_idx + a, n * 8, on_device);
  copy_out(ctx, dim, ctx->e_dim + a, n * 4, on_device);
  copy_out(ctx, diam2, ctx->e_d2 + a, n * 8, on_device);
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  return PH_OK;
  PH_API_END
}

int ph_get_essential_estimate(ph_ctx* ctx, int32_t cloud, uint8_t* in_e, int64_t* count) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced && ctx->rs.init, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(cloud >= 0 && cloud < ctx->n_clouds, PH_ERR_INVALID, "cloud out of range");
  const int nc = ctx->n_clouds;
  int64_t n = 0;
  for (int d = 0; d <= ctx->max_dim; d++)
    n += ctx->seg_start[d * nc + cloud + 1] - ctx->seg_start[d * nc + cloud];
  if (count) *count = n;
  if (!in_e) return PH_OK;
  ph::essential_estimate(ctx, cloud, in_e, n);
  return PH_OK;
  PH_API_END
}

int ph_get_columns(ph_ctx* ctx, int32_t cloud, int64_t* colptr, int32_t* rows, int64_t capacity,
                   int64_t* nnz) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced && ctx->rs.init, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(cloud >= 0 && cloud < ctx->n_clouds, PH_ERR_INVALID, "cloud out of range");
  PH_REQUIRE(colptr != nullptr, PH_ERR_INVALID, "colptr is required");
  const int nc = ctx->n_clouds;
  int64_t n = 0;
  for (int d = 0; d <= ctx->max_dim; d++)
    n += ctx->seg_start[d * nc + cloud + 1] - ctx->seg_start[d * nc + cloud];
  ph::reduced_columns(ctx, cloud, n, colptr, rows, capacity, nnz);
  return PH_OK;
  PH_API_END
}

int ph_get_predicted_lows(ph_ctx* ctx, int32_t cloud, int32_t* pred, int64_t* count) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->reduced && ctx->rs.init, PH_ERR_INVALID, "call ph_reduce first");
  PH_REQUIRE(ctx->opts.predict_pairs, PH_ERR_INVALID, "the context was made without predict_pairs");
  PH_REQUIRE(cloud >= 0 && cloud < ctx->n_clouds, PH_ERR_INVALID, "cloud out of range");
  const int nc = ctx->n_clouds;
  int64_t n = 0;
  for (int d = 0; d <= ctx->max_dim; d++)
    n += ctx->seg_start[d * nc + cloud + 1] - ctx->seg_start[d * nc + cloud];
  if (count) *count = n;
  if (!pred) return PH_OK;
  ph::predicted_lows(ctx, cloud, pred, n);
  return PH_OK;
  PH_API_END
}

int ph_get_filtration(ph_ctx* ctx, int32_t cloud, int32_t* dim, int64_t* diam2, int32_t* verts,
                      int32_t* beta, int32_t* low, int64_t* count) {
  PH_API_BEGIN
  PH_REQUIRE(ctx->built, PH_ERR_INVALID, "no filtration");
  PH_REQUIRE(cloud >= 0 && cloud < ctx->n_clouds, PH_ERR_INVALID, "cloud out of range");
  const int nc = ctx->n_clouds;
  int64_t n = 0;
  for (int d = 0; d <= ctx->max_dim; d++)
    n += ctx->seg_start[d * nc + cloud + 1] - ctx->seg_start[d * nc + cloud];
  if (count) *count = n;
  if (!dim) return PH_OK;
  int32_t* o_dim = ph::alloc_n<int32_t>(ctx, n);
  int64_t* o_d2 = ph::alloc_n<int64_t>(ctx, n);
  int32_t* o_v = ph::alloc_n<int32_t>(ctx, ph::kVrSlots * n);
  int32_t* o_beta = ph::alloc_n<int32_t>(ctx, n);
  int32_t* o_low = ph::alloc_n<int32_t>(ctx, n);
  int32_t* d_bad = ph::alloc_n<int32_t>(ctx, 1);
  PH_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), ctx->stream));
  for (int d = 0; d <= ctx->max_dim; d++) {
    int64_t lo = ctx->seg_start[d * nc + cloud], hi = ctx->seg_start[d * nc + cloud + 1];
    if (hi <= lo) continue;
    ph::k_inspect<<<ph::grid_for(ctx, hi - lo, ph::kThreads), ph::kThreads, 0, ctx->stream>>>(
        lo, hi, ctx->seg, nc, ctx->gidx, ctx->key, ctx->d2tab, ctx->verts, ctx->beta, ctx->low,
        o_dim, o_d2, o_v, o_beta, o_low, n, ctx->vbits, d_bad);
    PH_CHECK_LAUNCH();
  }
  int32_t bad = 0;
  PH_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  copy_out(ctx, dim, o_dim, n * 4, 0);
  copy_out(ctx, diam2, o_d2, n * 8, 0);
  copy_out(ctx, verts, o_v, n * 4 * ph::kVrSlots, 0);
  copy_out(ctx, beta, o_beta, n * 4, 0);
  copy_out(ctx, low, o_low, n * 4, 0);
  PH_CUDA(cudaStreamSynchronize(ctx->stream));
  for (void* p : {(void*)o_dim, (void*)o_d2, (void*)o_v, (void*)o_beta, (void*)o_low,
                  (void*)d_bad})
    ctx->dfree(p);
  PH_REQUIRE(bad == 0, PH_ERR_INVALID, "internal error: filtration index out of range");
  return PH_OK;
  PH_API_END
}

int64_t ph_kernel_launches(const ph_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* ph_last_error(const ph_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

}  // extern "C"
