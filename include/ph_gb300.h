/*
 * ph_gb300.h -- C ABI of the GB300 parallel multi-scale reduction library.
 *
 * The library computes persistent homology of Vietoris-Rips filtrations over F2 following
 * Mendoza-Smith & Tanner, "Parallel multi-scale reduction of persistent homology filtrations"
 * (arXiv:1708.04710). Every step runs in the library's own CUDA kernels for sm_103a:
 *   - the filtration (Sec. 2.2) and boundary matrix (Sec. 2.3) are built on the device;
 *   - the boundary matrix is reduced by Algorithm 2 (Sec. 3.1), pass by pass;
 *   - pairs and the essential set (Lemma 1, Eq. paired) are extracted on the device.
 *
 * Conventions
 *   - Indices are 0-based; "none" is -1 (the paper is 1-based with 0 = none).
 *   - A simplex's index is its position in the filtration of its own cloud, ordered by
 *     (squared diameter, dimension, vertex tuple in lexicographic order): a compatible
 *     ordering in the sense of Sec. 2.2.
 *   - Coordinates are int32 grid units (value * 2^16); squared diameters are exact int64.
 *   - `stream` arguments are cudaStream_t values passed as void*. All work of a context runs
 *     on its stream. Calls return after enqueueing, except where a host-visible count or
 *     host buffer is produced (those synchronise the stream).
 *   - Pointers documented as "device" must be device (or managed) memory of the context's
 *     device; "host" pointers are ordinary host memory.
 *   - Every entry point returns an int status (PH_OK = 0, PH_NOT_CONVERGED = 1, negative on
 *     error). No C++ exception crosses the ABI and no kernel traps; the text of the last error
 *     of a context is available from ph_last_error.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef PH_GB300_H
#define PH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PH_OK = 0,
  PH_NOT_CONVERGED = 1, /* max_passes reached; the state is a valid partial reduction */
  PH_ERR_INVALID = -1,  /* bad argument or call order */
  PH_ERR_ALLOC = -2,    /* device allocation failed */
  PH_ERR_CUDA = -3,     /* a CUDA call failed (message in ph_last_error) */
  PH_ERR_CAPACITY = -4, /* a size limit of the library was exceeded */
  PH_ERR_TIMEOUT = -5   /* the pass loop ran past ph_opts.timeout_ms; the reduction state is
                         * left as it was after the last complete pass */
};

typedef struct ph_ctx ph_ctx;

/* Device memory provider. alloc returns device memory of at least `bytes` bytes usable on
 * `stream`, aligned to 256 bytes (as cudaMalloc's is), or NULL on failure; free releases it.
 * Both are called from the thread that calls the library. A misaligned block is given back and
 * the call fails with PH_ERR_ALLOC. With a NULL provider the library uses cudaMallocAsync /
 * cudaFreeAsync. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user, void* stream);
  void (*free)(void* ptr, size_t bytes, void* user, void* stream);
  void* user;
} ph_allocator;

typedef struct {
  /* 1: Phase II adds only proven pivots, the rule printed in Algorithm 2.
   * 0 (default): adds the left-most column with the same low, proven or not; both are
   * left-to-right additions that strictly lower the target's low, so lowstar is the same
   * (Sec. 2.3: lowstar does not depend on the reduction) and only pass counts differ. */
  int32_t strict_phase2;
  /* 1 (default): zero case of Corollary 10 -- a column with beta_j = 0 whose candidate rows
   * (all rows of K_{d-1} up to low(j)) are all known to be paired is set to zero. */
  int32_t use_cor10;
  /* Phase II starts by merging each job in its own lane (sequentially, from shared memory),
   * which suits short columns, and switches once, for the rest of the reduction, to merge
   * pieces spread over the lanes when the mean job (target + source rows reserved per
   * surviving column) reaches this many rows; 0 = library default (20), -1 = pieces from the
   * first pass */
  int32_t lane_merge_words;
  /* Phase II merges of more rows than this (target + source) run from global memory; shorter
   * ones are staged in shared memory first (0 = library default = the largest staged size,
   * 1024) */
  int32_t staged_merge_max;
  /* merge-path positions per lane in Phase II (1..64); 0 = library default (8). With 8 a lane
   * merges its piece into registers; any other value merges it from shared memory twice
   * (count, then write), which is slower and kept for testing the merge path */
  int32_t merge_items;
  /* 1: per-pass counters are collected (column additions, XORs, pivots, ...) */
  int32_t collect_stats;
  /* 1 (default): the pass loop runs inside one CUDA graph whose conditional while node reads
   * a device flag, so no host round trip happens per pass; 0: the host launches each pass and
   * reads the flag. Both run the same kernels on the same device state. */
  int32_t use_graph;
  /* 1: CUDA events time every launch of the Phase II addition kernel (ph_stats.ms_add); only
   * with use_graph = 0 (events cannot sit inside a conditional graph body) */
  int32_t time_kernels;
  /* occupancy of the persistent Phase II addition kernel: 1..4 units of 256 threads per SM
   * (two 128-thread blocks each; 0 = library default, 4) */
  int32_t add_blocks_per_sm;
  /* wall-clock bound of one ph_reduce's pass loop in ms, checked on the device at the end of
   * every pass (0 = library default, 60000); past it the call returns PH_ERR_TIMEOUT */
  int32_t timeout_ms;
  /* 1: every pass also applies the non-zero case of Corollary 10 (Lemma 9): an active column j
   * with beta_j >= 0 whose candidate set L_j (rows of K_{d-1} in [beta_j, low(j)] not known to
   * be paired) holds one row i has lowstar(j) = i, which ph_get_predicted_lows reports before
   * the column is reduced. 0 (default): off. */
  int32_t predict_pairs;
  /* Bit-packed columns: when a column addition (target + source rows) exceeds
   * max(dense_threshold, the bitmap's words), the result is kept as a bitmap over the column's
   * row segment (one bit per (d-1)-simplex of its cloud, after a 1-word header) and later
   * additions into it XOR whole words; a bit-packed source is XORed word by word. Results are
   * identical either way. 0 (default): the threshold is 32 rows, so a column goes bit-packed
   * once the bitmap is its smaller form; < 0: never. */
  int32_t dense_threshold;
  /* Phase II work shape: a block of 4 warps claims 128 columns at a time (one block scan and
   * barrier per chunk) until, at the end of some pass, fewer than this many columns are active
   * and their jobs are long (warp_chunk_words or more arena words reserved per survivor, on
   * average); from then on every warp claims its own 32 columns (no block barriers, 4x the
   * queue atomics). A reduction switches at most once. Results are identical either way.
   * 0 (default): 4,194,304; < 0: block chunks throughout. */
  int32_t warp_chunks_below;
  /* The job length that switch needs, in mean arena words per survivor. 0 (default): 40;
   * < 0: any (then a complex of fewer than warp_chunks_below columns starts with warp chunks). */
  int32_t warp_chunk_words;
  /* Once warp chunks and merge pieces are on, a pass that ends with fewer than this many active
   * columns switches the warps, for the rest of the reduction, to chunks of 8 columns (lanes
   * 8..31 hold no column of their own and take merge pieces), so that the short late passes
   * spread over more warps. Results are identical either way. 0 (default): 16 columns per warp
   * of the addition kernel's grid (77,824 columns on 152 SMs with add_blocks_per_sm = 4);
   * < 0: 32-column chunks throughout. */
  int32_t narrow_chunks_below;
  /* Phase II with p processors (Sec. 3.4.1-3.4.2). phase2_sets = p > 0: each pass the targets
   * fall into neighbour sets, one per low row i, holding the targets whose addition the pass
   * may do; only the targets of the first p sets in priority order receive their addition, the
   * others stay active unchanged (and count as targets). phase2_priority 0: larger sets first
   * (Sec. 3.4.1); 1: sets with more targets known to be negative (beta >= 0, Thm 5) first,
   * then larger sets (Sec. 3.4.2); ties by the row first in the filtration. Any budget reaches
   * the same lowstar (Sec. 2.3); passes and counters differ. The pass loop is then host-driven
   * (use_graph is ignored). 0 (default): every set, as in Algorithm 2. ph_create rejects a
   * priority other than 0 or 1 (PH_ERR_INVALID). */
  int32_t phase2_sets;
  int32_t phase2_priority;
  /* Initial capacity of each of the two survivor arenas, in int32 words (0, default: twice the
   * boundary's nonzeros). A pass whose Phase I bound does not fit stops after its marks,
   * before any column changes; the host grows the arena and the pass continues with its column
   * additions, so a small value trades memory for extra host round trips; results are the
   * same. */
  int64_t arena_words;
} ph_opts;

/* Per-pass counters (rows of ph_get_pass_stats), in this order. */
enum {
  PH_PS_ACTIVE = 0,    /* active columns at the start of the pass */
  PH_PS_NEW_PIVOTS,    /* columns proven reduced in this pass (Thm 5 test or Phase I) */
  PH_PS_ZERO_FINAL,    /* active columns found empty (positive) */
  PH_PS_COR10,         /* columns set to zero by the zero case of Corollary 10 */
  PH_PS_CLEARED,       /* active columns set to zero by clearing (Lemma 1) */
  PH_PS_TARGETS,       /* active columns whose low collides with an earlier column */
  PH_PS_ADDS,          /* column additions done */
  PH_PS_XORS,          /* nontrivial scalar XORs, |target union source| (Sec. 4.1) */
  PH_PS_COPIED,        /* rows moved without an addition (survivors and new pivots) */
  PH_PS_ESS_EST,       /* |E^l| after the pass's marks: the essential estimate of
                        * Eq. (essential_iteration), which contains Ess (Lemma 11) */
  PH_PS_PREDICTED,     /* columns whose pair Corollary 10 (non-zero case) predicts for the first
                        * time (needs predict_pairs) */
  PH_PS_EMPTY_L,       /* columns with an empty candidate set L_j: always 0 (Lemma 9) */
  PH_PS_PACKED,        /* additions computed on bitmaps (see dense_threshold); a property of
                        * the storage, not of Algorithm 2 */
  PH_PS_N
};

typedef struct {
  int32_t passes;      /* passes that found collisions (iterations of Algorithm 2) */
  int32_t status;      /* PH_OK or PH_NOT_CONVERGED */
  int64_t m;           /* simplices in the context */
  int64_t col_adds;    /* column additions, all passes (needs collect_stats) */
  int64_t xors;        /* nontrivial XORs, all passes (needs collect_stats) */
  int64_t alg_bytes;   /* algorithmic bytes of the reduction (needs collect_stats) */
  int64_t add_bytes;   /* algorithmic bytes of the addition kernel (needs collect_stats):
                          8 per XOR + 8 per copied row + 40 per active column per pass */
  int64_t add_launches;/* launches of the addition kernel */
  double ms_add;       /* summed duration of those launches (needs time_kernels) */
} ph_stats;

/* Fills `opts` with the defaults described above. */
void ph_default_opts(ph_opts* opts);

/* Creates a context bound to the current CUDA device and to `stream` (NULL = legacy default
 * stream). `opts` and `alloc` may be NULL (defaults). On success *out owns all library
 * workspace until ph_destroy. */
int ph_create(ph_ctx** out, const ph_opts* opts, const ph_allocator* alloc, void* stream);

/* Releases the context and all of its device memory. NULL is ignored. */
void ph_destroy(ph_ctx* ctx);

/* Builds the Vietoris-Rips filtrations (Sec. 2.2, f_r(sigma) = 1{diam(sigma) <= 2r}) of
 * n_clouds point clouds, and the boundary matrix (Sec. 2.3) and beta (Definition 4,
 * Algorithm 4) of each.
 *   coords        device int32 [N][D], row-major, the clouds stored back to back.
 *   cloud_offsets host int64 [n_clouds + 1]: cloud c owns points [off[c], off[c+1]).
 *                 NULL with n_clouds == 1 means one cloud of N = coords rows given by
 *                 n_points.
 *   n_points      total number of points N (rows of coords).
 *   D             coordinate dimension, 1..16.
 *   max_dim       largest simplex dimension, 1..5 (above 3, at most 254 points per cloud).
 *   max_diam2     simplices with squared diameter above this are left out; < 0 keeps all.
 *   m_out         host, optional: total number of simplices over all clouds.
 * Limits: 1..4094 points per cloud up to dimension 3 (1..254 above); at most 65535 clouds and
 * 2^31 - 1 candidate simplices in total.
 * Replaces any filtration the context held. Synchronises the stream. */
int ph_build_filtration(ph_ctx* ctx, const int32_t* coords, const int64_t* cloud_offsets,
                        int32_t n_clouds, int64_t n_points, int32_t D, int32_t max_dim,
                        int64_t max_diam2, int64_t* m_out);

/* The same VR complex on a grid of scales, the setting of the paper's experiments (Sec. 4:
 * scales r_1 < ... < r_T with uniform spacing h): a simplex enters at the first scale
 * r_i = i * scale_step with diameter <= 2 r_i (Sec. 2.2), i = 0..n_scales, and simplices above
 * r_T = n_scales * scale_step are left out. The order is (scale index, dimension, lexicographic
 * vertex tuple), so simplices of one scale tie and are ordered by dimension and vertices. The
 * squared diameters that ph_get_pairs and ph_get_essential report are then scale indices.
 *   scale_step    grid units (1 = 2^-16), 1..2^26.   n_scales   >= 1.
 * Other arguments and limits as ph_build_filtration. */
int ph_build_filtration_scales(ph_ctx* ctx, const int32_t* coords, const int64_t* cloud_offsets,
                               int32_t n_clouds, int64_t n_points, int32_t D, int32_t max_dim,
                               int64_t scale_step, int32_t n_scales, int64_t* m_out);

/* As ph_build_filtration, from fp32 coordinates (device float [N][D], plain units): each is
 * rounded on the device to the 2^-16 grid, rint(x * 65536) with ties to even, and must be
 * finite with |x| <= 256 (PH_ERR_INVALID otherwise). The pairing is computed from the rounded
 * values; ph_diagram_loss / ph_diagram_backward use the fp32 values. */
int ph_build_filtration_f32(ph_ctx* ctx, const float* coords, const int64_t* cloud_offsets,
                            int32_t n_clouds, int64_t n_points, int32_t D, int32_t max_dim,
                            int64_t max_diam2, int64_t* m_out);

/* Loads an explicit filtration of one complex instead of building a VR one.
 *   m             number of cells, in a compatible order (faces before cofaces).
 *   dims          host int32 [m], dimension of each cell (0..8).
 *   colptr        host int64 [m + 1], CSC column pointers of the boundary matrix over F2.
 *   rows          host int32 [colptr[m]], row indices (earlier positions of dimension
 *                 dims[j] - 1, strictly ascending per column; none in dimension 0).
 * A column may hold any number of rows: a simplicial boundary (d + 1 faces), a cubical or
 * cellular one, or a partially reduced matrix R = D V as ph_get_columns returns it; reducing R
 * gives the pairs of D (lowstar depends only on the spans of the column prefixes, Sec. 2.3),
 * so R is a checkpoint of a reduction. Squared diameters of loaded complexes are reported as
 * 0. Synchronises the stream. */
int ph_load_boundary(ph_ctx* ctx, int64_t m, const int32_t* dims, const int64_t* colptr,
                     const int32_t* rows);

/* Reduces the boundary matrices of the context with Algorithm 2 (Sec. 3.1): each pass builds
 * the table of left-most columns per low with atomicMin, marks pivots (Thm 5, Phase I /
 * Algorithm 5 with Thms 6-7), zero columns and the zero case of Corollary 10, clears the
 * partners of new pivots (Lemma 1), then adds every colliding column's left-most column into
 * it, until no low collides (Thm 8). All clouds are reduced together.
 *   max_passes    cap on passes with additions (< 0: m + 1, which a reduction never needs:
 *                 every pass proves or zeroes at least one column). When it is hit the call
 *                 returns PH_NOT_CONVERGED and the state stays a valid partial reduction.
 *   out           host, optional: summary counters.
 * A later call continues a reduction that stopped at its pass cap (PH_NOT_CONVERGED), at the
 * time bound (PH_ERR_TIMEOUT) or on a failed allocation (PH_ERR_ALLOC, the state left as
 * before the pass that needed the memory); after a complete reduction it returns the result
 * again. The pass loop runs in a CUDA graph (use_graph) or from the host. Synchronises the
 * stream. */
int ph_reduce(ph_ctx* ctx, int32_t max_passes, ph_stats* out);

/* Discards the reduction state (and extracted outputs) of the context; the next ph_reduce
 * starts again from the unreduced boundary matrix. Synchronises the stream. */
int ph_reset_reduction(ph_ctx* ctx);

/* Copies the per-pass counters (PH_PS_N int64 per pass, passes + 1 rows including the final
 * pass that found no collision) to host `out` with room for `max_rows` rows; *rows_out gets
 * the number of rows available. Needs collect_stats. */
int ph_get_pass_stats(ph_ctx* ctx, int64_t* out, int32_t max_rows, int32_t* rows_out);

/* Durations (ms, CUDA events) of the Phase II addition kernel, one per pass of the last
 * ph_reduce with time_kernels = 1 and use_graph = 0; host `out` with room for `max_n`,
 * *n_out gets the number available. */
int ph_get_add_times(ph_ctx* ctx, float* out, int32_t max_n, int32_t* n_out);

/* Persistence pairs (sigma_birth, sigma_death) of cloud `cloud` with lowstar(death) = birth
 * (Lemma 1), ordered by (dimension of death, death index); cloud = -1 gives every cloud's pairs,
 * clouds in order (indices stay per cloud). Two-call protocol: with
 * birth == NULL only *count is written. Output buffers (capacity >= count entries each) are
 * device pointers when on_device != 0, host pointers otherwise; any of them may be NULL.
 *   birth, death        int64 filtration indices within the cloud.
 *   dim                 int32 dimension of the birth simplex.
 *   birth_diam2, death_diam2   int64 squared diameters (grid units^2).
 * Synchronises the stream. */
int ph_get_pairs(ph_ctx* ctx, int32_t cloud, int64_t* birth, int64_t* death, int32_t* dim,
                 int64_t* birth_diam2, int64_t* death_diam2, int64_t capacity, int64_t* count,
                 int32_t on_device);

/* Essential simplices of cloud `cloud`: positive simplices that are never paired (Sec. 2.3,
 * set Ess), ordered by (dimension, index); cloud = -1 gives all clouds in order. Same protocol
 * and buffer rules as ph_get_pairs.
 *   idx    int64 filtration indices; dim int32; diam2 int64. */
int ph_get_essential(ph_ctx* ctx, int32_t cloud, int64_t* idx, int32_t* dim, int64_t* diam2,
                     int64_t capacity, int64_t* count, int32_t on_device);

/* Essential estimate E^l of cloud `cloud` after the passes run so far (Sec. 3.3): E^0 = [m],
 * E^{l+1} = (E^l minus Paired^l) minus {low(j)} (Eq. essential_iteration), so every essential
 * simplex is in E^l (Lemma 11) and, after a partial reduction (ph_reduce with max_passes), E^l
 * is the early-stopping estimate of Ess. Host buffer `in_e` of `count` bytes, one per simplex
 * of the cloud in filtration order: 1 if in E^l. With in_e == NULL only *count is written.
 * Needs ph_reduce first. Synchronises the stream. */
int ph_get_essential_estimate(ph_ctx* ctx, int32_t cloud, uint8_t* in_e, int64_t* count);

/* Pairs predicted by Corollary 10 (non-zero case) so far, for cloud `cloud`: host buffer
 * `pred` of `count` int32, one per simplex in filtration order, holding the predicted
 * lowstar as a filtration index, or -1 where no prediction was made. Every prediction is
 * exact (Lemma 9), also after a partial reduction. With pred == NULL only *count is written.
 * Needs ph_reduce first with predict_pairs = 1. Synchronises the stream. */
int ph_get_predicted_lows(ph_ctx* ctx, int32_t cloud, int32_t* pred, int64_t* count);

/* The reduced matrix R of cloud `cloud` as the last ph_reduce left it (complete or partial),
 * in compressed columns over the cloud's filtration indices: column f holds
 * rows[colptr[f] .. colptr[f + 1] - 1], the filtration indices of its rows, ascending. R comes
 * from D by left-to-right column additions (Sec. 2.3), except for columns set to zero as
 * positive (clearing, Lemma 1; Corollary 10), which are empty. Once the reduction is complete,
 * a negative column j holds a cycle that becomes a boundary at j: a representative of the
 * class born at low(j) and killed by j (Lemma 1).
 *   colptr  host int64 [count + 1], count being the cloud's number of simplices
 *           (ph_get_filtration); always filled.
 *   rows    host int32 [capacity], or NULL to learn *nnz first.
 *   nnz     host, optional: total number of rows.
 * PH_ERR_CAPACITY if rows is too small (colptr and *nnz are filled all the same). Needs
 * ph_reduce first. Synchronises the stream. */
int ph_get_columns(ph_ctx* ctx, int32_t cloud, int64_t* colptr, int32_t* rows, int64_t capacity,
                   int64_t* nnz);

/* Inspection of the filtration of cloud `cloud` in filtration order, for testing the build
 * against an independent implementation. Host buffers of `count` entries (any may be NULL):
 *   dim int32; diam2 int64; verts int32 [count][6] (-1 padded); beta int32 (Definition 4, as
 *   a filtration index, -1 = none); low int32 (current low, filtration index, -1 = zero).
 * *count receives the number of simplices of the cloud; with dim == NULL nothing else is
 * copied. Synchronises the stream. */
int ph_get_filtration(ph_ctx* ctx, int32_t cloud, int32_t* dim, int64_t* diam2, int32_t* verts,
                      int32_t* beta, int32_t* low, int64_t* count);

/* Diagram loss of a reduced VR filtration: over the finite pairs (sigma_b, sigma_d) whose birth
 * simplex has dimension `dim` (Lemma 1), b and d are the fp32 Euclidean lengths of the edges that
 * realise the diameters of sigma_b and sigma_d (Sec. 2.2: the VR value of a simplex is its
 * diameter; a simplex's realising edge is itself for an edge, else the realising edge of its
 * last face in the filtration), and loss = sum (d - b)^2 per cloud. The pairing is exact and
 * piecewise constant, so only b and d carry gradient.
 *   coords   device float [N][D], the coordinates the filtration was built from: N and D of
 *            that build (n_points * D floats). The kernels read coords at the build's point
 *            rows, so a smaller array is read out of bounds; the library cannot see its size.
 *   D        must equal the build's D (PH_ERR_INVALID otherwise, before any launch).
 *   loss     device float [n_clouds + 1]: per-cloud losses, then their sum.
 *   n_pairs  host, optional: number of pairs summed.
 * Needs ph_reduce first and dim + 1 <= max_dim. Synchronises the stream. */
int ph_diagram_loss(ph_ctx* ctx, const float* coords, int32_t D, int32_t dim, float* loss,
                    int64_t* n_pairs);

/* Gradient of the per-cloud losses of ph_diagram_loss with respect to the coordinates:
 * grad_coords (device float [N][D]) += sum over clouds of grad_loss[c] * d loss_c / d coords,
 * scattered to the two points of each realising edge (a zero-length edge contributes nothing).
 *   coords, grad_coords  device float, n_points * D each, N and D of the build (as above).
 *   D          must equal the build's D (PH_ERR_INVALID otherwise, before any launch).
 *   grad_loss  device float [n_clouds]. Asynchronous. */
int ph_diagram_backward(ph_ctx* ctx, const float* coords, int32_t D, int32_t dim,
                        const float* grad_loss, float* grad_coords);

/* Allocation-free beta, for callers that cannot allocate device memory: code running inside
 * another framework's memory pool or arena, programs that forbid allocation after start-up,
 * and callers that hold no library context. The paper has no counterpart of this entry point;
 * it computes beta of Definition 4 like ph_build_filtration does, but keeps its only scratch
 * (left(i) of Definition 3, one int32 per row) in a fixed device array of the library.
 *   rows          device int32 [n_cols][rows_per_col]: boundary rows of n_cols columns of one
 *                 dimension, columns in filtration order; a row is the 0-based filtration
 *                 position of a face among the n_rows simplices one dimension lower.
 *   n_rows        at most 4,194,304; larger values return PH_ERR_CAPACITY. The scratch array
 *                 (16 MiB) stays resident on every GPU that loads the library until exit.
 *   beta          device int32 [n_cols], output: largest row whose first column is j, or -1.
 *   stream        cudaStream_t as void*.
 * Allocates nothing (no cudaMalloc, cudaFree or allocator call). Every call looks up the
 * scratch's device address in the current context with cudaGetSymbolAddress (which allocates
 * nothing), so a device reset or another context on the device leaves no stale address; the
 * first call in a context loads the library's module, so make it before any stream capture in
 * that context. Every call shares the one scratch array, which it resets
 * at its start: calls that overlap on the GPU (other streams or threads) race and give wrong
 * results. Rows outside [0, n_rows) are skipped and make the call return PH_ERR_INVALID.
 * Synchronises `stream`. */
int ph_beta_static(const int32_t* rows, int64_t n_cols, int32_t rows_per_col, int64_t n_rows,
                   int32_t* beta, void* stream);

/* Number of kernels the context has launched since it was created. */
int64_t ph_kernel_launches(const ph_ctx* ctx);

/* Text of the last error of the context (empty when none). Valid until the next call. */
const char* ph_last_error(const ph_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PH_GB300_H */
