/*
 * CPU oracle for the persistent-homology reduction path (arXiv:1708.04710).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this file;
 * only the tests, the package's smoke check and the bench's cpu_baseline / reference leg do.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Everything here is deliberately plain and sequential: nested loops, qsort, bsearch and
 * columns held as sorted int32 arrays. Indices are 0-based global filtration positions and
 * "no value" is -1 (the paper uses 1-based indices with 0 = none, Sec. 2, notation).
 *
 * Contents
 *   orc_vr_build      Vietoris-Rips filtration (Sec. 2.2) with compatible ordering, plus the
 *                     boundary matrix of Sec. 2.3 (Eq. def:boundary_matrix) in CSC form.
 *   orc_beta          beta_j of Definition 4, built as in Algorithm 4 (Thm 5, P.6).
 *   orc_reduce_std    standard reduction, Algorithm 1 (optionally tracking V with R = D V).
 *   orc_reduce_twist  standard reduction with a twist (clearing), Algorithm 3.
 *   orc_reduce_pms    parallel multi-scale reduction, Algorithm 2 (Phase 0, Phase I as in
 *                     Algorithm 5, Phase II), executed pass by pass, with clearing, the zero
 *                     case of Corollary 10, the essential estimate of Eq. essential_iteration
 *                     and, optionally, Phase II limited to p neighbour sets (Sec. 3.4).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_ALLOC (-2)

/* ------------------------------------------------------------------------------------------ */
/* Columns over F2: sorted arrays of row indices.                                             */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int32_t* v;
  int64_t n, cap;
} col_t;

static int col_reserve(col_t* c, int64_t cap) {
  if (cap <= c->cap) return 0;
  int64_t nc = c->cap ? c->cap : 4;
  while (nc < cap) nc *= 2;
  int32_t* p = (int32_t*)realloc(c->v, (size_t)nc * sizeof(int32_t));
  if (!p) return -1;
  c->v = p;
  c->cap = nc;
  return 0;
}

static int32_t col_low(const col_t* c) { return c->n ? c->v[c->n - 1] : -1; }

/* dst <- dst + src over F2: the symmetric difference of two sorted sets. Returns the number of
 * nontrivial scalar XORs (1+1, 1+0, 0+1), i.e. |dst union src| (Sec. 4.1). */
static int64_t col_add(col_t* dst, const col_t* src, col_t* tmp) {
  int64_t i = 0, j = 0, k = 0, ops = 0;
  if (col_reserve(tmp, dst->n + src->n) != 0) return -1;
  while (i < dst->n && j < src->n) {
    if (dst->v[i] < src->v[j]) {
      tmp->v[k++] = dst->v[i++];
    } else if (dst->v[i] > src->v[j]) {
      tmp->v[k++] = src->v[j++];
    } else {
      i++;
      j++;
    }
    ops++;
  }
  while (i < dst->n) { tmp->v[k++] = dst->v[i++]; ops++; }
  while (j < src->n) { tmp->v[k++] = src->v[j++]; ops++; }
  tmp->n = k;
  /* swap storage */
  col_t t = *dst;
  *dst = *tmp;
  *tmp = t;
  return ops;
}

static col_t* cols_from_csc(int64_t m, const int64_t* colptr, const int32_t* rows) {
  col_t* c = (col_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(col_t));
  if (!c) return NULL;
  for (int64_t j = 0; j < m; j++) {
    int64_t n = colptr[j + 1] - colptr[j];
    if (col_reserve(&c[j], n) != 0) return NULL;
    memcpy(c[j].v, rows + colptr[j], (size_t)n * sizeof(int32_t));
    c[j].n = n;
  }
  return c;
}

static void cols_free(col_t* c, int64_t m) {
  if (!c) return;
  for (int64_t j = 0; j < m; j++) free(c[j].v);
  free(c);
}

/* ------------------------------------------------------------------------------------------ */
/* Vietoris-Rips filtration, Sec. 2.2.                                                         */
/*   f_r(sigma) = 1{diam(sigma) <= 2r}; diam is the Euclidean diameter, compared squared in    */
/*   exact integer grid units. The compatible ordering (simplices of an earlier complex first, */
/*   faces before cofaces) is realised by sorting on (diam^2, dim, vertex tuple in lexicographic */
/*   order); a face never has a larger diameter nor a larger dimension than its coface.        */
/* ------------------------------------------------------------------------------------------ */
#define ORC_VR_MAX_DIM 5 /* largest simplex dimension of a VR build (6 vertices) */
#define ORC_VR_NV (ORC_VR_MAX_DIM + 1)

typedef struct {
  int64_t diam2;
  int32_t dim;
  int32_t v[ORC_VR_NV];
} simplex_t;

static int cmp_filtration(const void* a, const void* b) {
  const simplex_t* x = (const simplex_t*)a;
  const simplex_t* y = (const simplex_t*)b;
  if (x->diam2 != y->diam2) return x->diam2 < y->diam2 ? -1 : 1;
  if (x->dim != y->dim) return x->dim < y->dim ? -1 : 1;
  for (int k = 0; k <= x->dim; k++)
    if (x->v[k] != y->v[k]) return x->v[k] < y->v[k] ? -1 : 1;
  return 0;
}

typedef struct {
  int64_t m, nnz;
  int32_t* dim;
  int64_t* diam2;
  int32_t* verts; /* m x ORC_VR_NV, -1 beyond the simplex's dim */
  int64_t* colptr;
  int32_t* rows;
} orc_complex;

/* lexicographic lookup of a vertex tuple among the simplices of one dimension */
static const simplex_t* g_lex_base; /* single-threaded oracle */
static int g_lex_len;
static int cmp_lex_idx(const void* a, const void* b) {
  const simplex_t* x = &g_lex_base[*(const int64_t*)a];
  const simplex_t* y = &g_lex_base[*(const int64_t*)b];
  for (int k = 0; k < g_lex_len; k++)
    if (x->v[k] != y->v[k]) return x->v[k] < y->v[k] ? -1 : 1;
  return 0;
}
static const int32_t* g_key_tuple;
static int cmp_key_idx(const void* key, const void* b) {
  (void)key;
  const simplex_t* y = &g_lex_base[*(const int64_t*)b];
  for (int k = 0; k < g_lex_len; k++)
    if (g_key_tuple[k] != y->v[k]) return g_key_tuple[k] < y->v[k] ? -1 : 1;
  return 0;
}

static int64_t sqdist(const int32_t* coords, int D, int a, int b) {
  int64_t s = 0;
  for (int k = 0; k < D; k++) {
    int64_t d = (int64_t)coords[(int64_t)a * D + k] - (int64_t)coords[(int64_t)b * D + k];
    s += d * d;
  }
  return s;
}

/* Scale index of a squared diameter on the grid r_i = i * step (Sec. 4's grid of scales): the
 * first i >= 0 with diameter <= 2 r_i (Sec. 2.2), found by counting up. */
static int64_t scale_index(int64_t d2, int64_t step) {
  int64_t i = 0;
  while ((2 * i * step) * (2 * i * step) < d2) i++;
  return i;
}

static int vr_build(const int32_t* coords, int32_t n, int32_t D, int32_t max_dim,
                    int64_t max_diam2, int64_t step, int32_t n_scales, orc_complex** out);

/* Build the VR filtration of the n points `coords` (int32 grid units, row-major n x D) up to
 * dimension max_dim (<= 5). Simplices with squared diameter above max_diam2 are dropped when
 * max_diam2 >= 0. Returns a heap object released by orc_complex_free. */
int orc_vr_build(const int32_t* coords, int32_t n, int32_t D, int32_t max_dim, int64_t max_diam2,
                 orc_complex** out) {
  return vr_build(coords, n, D, max_dim, max_diam2, 0, 0, out);
}

/* The same on the grid of scales r_i = i * step, i = 0..n_scales: a simplex's filtration value
 * (stored in place of its squared diameter) is the scale index of its diameter, and simplices
 * above the last scale are dropped. */
int orc_vr_build_scales(const int32_t* coords, int32_t n, int32_t D, int32_t max_dim,
                        int64_t step, int32_t n_scales, orc_complex** out) {
  if (step <= 0 || n_scales < 1) return ORC_ERR_INVALID;
  return vr_build(coords, n, D, max_dim, -1, step, n_scales, out);
}

static int vr_build(const int32_t* coords, int32_t n, int32_t D, int32_t max_dim,
                    int64_t max_diam2, int64_t step, int32_t n_scales, orc_complex** out) {
  if (!coords || n <= 0 || D <= 0 || max_dim < 0 || max_dim > ORC_VR_MAX_DIM || !out)
    return ORC_ERR_INVALID;
  /* count candidates: C(n, d + 1) for d = 0..max_dim */
  int64_t cap = 0, binom = 1;
  for (int d = 0; d <= max_dim; d++) {
    binom = binom * (n - d) / (d + 1);
    if (binom < 0) binom = 0;
    cap += binom;
  }
  simplex_t* S = (simplex_t*)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(simplex_t));
  if (!S) return ORC_ERR_ALLOC;
  int64_t m = 0;
  /* every k-subset of the points in lexicographic order (an odometer over ascending tuples),
   * each with its largest pairwise squared distance (the VR diameter, Sec. 2.2) */
  for (int k = 1; k <= max_dim + 1 && k <= n; k++) {
    int v[ORC_VR_NV];
    for (int i = 0; i < k; i++) v[i] = i;
    for (;;) {
      int64_t d2 = 0;
      for (int p = 0; p < k; p++)
        for (int q = p + 1; q < k; q++) {
          int64_t t = sqdist(coords, D, v[p], v[q]);
          if (t > d2) d2 = t;
        }
      if (step > 0) d2 = scale_index(d2, step);  /* value on the grid of scales */
      int keep = step > 0 ? d2 <= n_scales : (max_diam2 < 0 || d2 <= max_diam2);
      if (k == 1 || keep) {
        simplex_t s;
        s.diam2 = d2;
        s.dim = k - 1;
        for (int i = 0; i < ORC_VR_NV; i++) s.v[i] = i < k ? v[i] : -1;
        S[m++] = s;
      }
      int i = k - 1; /* advance: last position that can still grow */
      while (i >= 0 && v[i] == n - k + i) i--;
      if (i < 0) break;
      v[i]++;
      for (int j = i + 1; j < k; j++) v[j] = v[j - 1] + 1;
    }
  }
  qsort(S, (size_t)m, sizeof(simplex_t), cmp_filtration);

  orc_complex* K = (orc_complex*)calloc(1, sizeof(orc_complex));
  if (!K) return ORC_ERR_ALLOC;
  K->m = m;
  K->dim = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  K->diam2 = (int64_t*)malloc((size_t)m * sizeof(int64_t));
  K->verts = (int32_t*)malloc((size_t)m * ORC_VR_NV * sizeof(int32_t));
  K->colptr = (int64_t*)malloc((size_t)(m + 1) * sizeof(int64_t));
  int64_t nnz = 0;
  for (int64_t j = 0; j < m; j++) nnz += S[j].dim > 0 ? S[j].dim + 1 : 0;
  K->nnz = nnz;
  K->rows = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  if (!K->dim || !K->diam2 || !K->verts || !K->colptr || !K->rows) return ORC_ERR_ALLOC;
  for (int64_t j = 0; j < m; j++) {
    K->dim[j] = S[j].dim;
    K->diam2[j] = S[j].diam2;
    for (int k = 0; k < ORC_VR_NV; k++) K->verts[j * ORC_VR_NV + k] = S[j].v[k];
  }

  /* per dimension: global indices sorted by vertex tuple, for face lookup */
  int64_t* bydim[ORC_VR_NV] = {0};
  int64_t cnt[ORC_VR_NV] = {0};
  for (int64_t j = 0; j < m; j++) cnt[S[j].dim]++;
  for (int d = 0; d <= max_dim; d++) {
    bydim[d] = (int64_t*)malloc((size_t)(cnt[d] > 0 ? cnt[d] : 1) * sizeof(int64_t));
    if (!bydim[d]) return ORC_ERR_ALLOC;
    cnt[d] = 0;
  }
  for (int64_t j = 0; j < m; j++) bydim[S[j].dim][cnt[S[j].dim]++] = j;
  g_lex_base = S;
  for (int d = 0; d <= max_dim; d++) {
    g_lex_len = d + 1;
    qsort(bydim[d], (size_t)cnt[d], sizeof(int64_t), cmp_lex_idx);
  }

  /* boundary matrix: column j holds the global indices of its codimension-1 faces */
  int64_t pos = 0;
  for (int64_t j = 0; j < m; j++) {
    K->colptr[j] = pos;
    int d = S[j].dim;
    if (d == 0) continue;
    int32_t face[ORC_VR_NV];
    int64_t start = pos;
    for (int drop = 0; drop <= d; drop++) {
      int k = 0;
      for (int p = 0; p <= d; p++)
        if (p != drop) face[k++] = S[j].v[p];
      g_lex_len = d;
      g_key_tuple = face;
      int64_t* hit = (int64_t*)bsearch(face, bydim[d - 1], (size_t)cnt[d - 1], sizeof(int64_t),
                                       cmp_key_idx);
      g_key_tuple = NULL;
      if (!hit) return ORC_ERR_INVALID; /* a face is missing: cannot happen for VR */
      K->rows[pos++] = (int32_t)*hit;
    }
    /* ascending row order (insertion sort of d+1 <= 6 entries) */
    for (int64_t a = start + 1; a < pos; a++) {
      int32_t x = K->rows[a];
      int64_t b = a - 1;
      while (b >= start && K->rows[b] > x) {
        K->rows[b + 1] = K->rows[b];
        b--;
      }
      K->rows[b + 1] = x;
    }
  }
  K->colptr[m] = pos;
  for (int d = 0; d <= max_dim; d++) free(bydim[d]);
  free(S);
  *out = K;
  return ORC_OK;
}

int64_t orc_complex_size(const orc_complex* K) { return K ? K->m : -1; }
int64_t orc_complex_nnz(const orc_complex* K) { return K ? K->nnz : -1; }

void orc_complex_export(const orc_complex* K, int32_t* dim, int64_t* diam2, int32_t* verts,
                        int64_t* colptr, int32_t* rows) {
  if (dim) memcpy(dim, K->dim, (size_t)K->m * sizeof(int32_t));
  if (diam2) memcpy(diam2, K->diam2, (size_t)K->m * sizeof(int64_t));
  if (verts) memcpy(verts, K->verts, (size_t)K->m * ORC_VR_NV * sizeof(int32_t));
  if (colptr) memcpy(colptr, K->colptr, (size_t)(K->m + 1) * sizeof(int64_t));
  if (rows) memcpy(rows, K->rows, (size_t)K->nnz * sizeof(int32_t));
}

void orc_complex_free(orc_complex* K) {
  if (!K) return;
  free(K->dim);
  free(K->diam2);
  free(K->verts);
  free(K->colptr);
  free(K->rows);
  free(K);
}

/* ------------------------------------------------------------------------------------------ */
/* beta, Definition 4, built by Algorithm 4: walk the columns in order; a row seen for the     */
/* first time has its left() at the current column, and beta_j is the largest such row.       */
/* ------------------------------------------------------------------------------------------ */
int orc_beta(int64_t m, const int64_t* colptr, const int32_t* rows, int32_t* beta_out) {
  uint8_t* visited = (uint8_t*)calloc((size_t)(m > 0 ? m : 1), 1);
  if (!visited) return ORC_ERR_ALLOC;
  for (int64_t j = 0; j < m; j++) {
    int32_t b = -1;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
      int32_t i = rows[p];
      if (!visited[i]) {
        if (i > b) b = i;
        visited[i] = 1;
      }
    }
    beta_out[j] = b;
  }
  free(visited);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1, standard reduction. Columns are reduced left to right; while an earlier column */
/* has the same low, it is added. Earlier columns are already reduced, so at most one earlier  */
/* column carries a given low and `pivot_of` finds it.                                          */
/* With v_dense != NULL (m <= 4096), V is tracked (R = D V) and returned, together with R, as  */
/* dense m x m uint8 matrices in row-major order.                                              */
/* stats: [0] column additions, [1] nontrivial XORs.                                           */
/* ------------------------------------------------------------------------------------------ */
int orc_reduce_std(int64_t m, const int64_t* colptr, const int32_t* rows, int32_t* low_out,
                   int64_t* stats, uint8_t* r_dense, uint8_t* v_dense) {
  col_t* R = cols_from_csc(m, colptr, rows);
  int32_t* pivot_of = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  col_t tmp = {0, 0, 0};
  col_t* V = NULL;
  if (!R || !pivot_of) return ORC_ERR_ALLOC;
  if (v_dense) {
    if (m > 4096) return ORC_ERR_INVALID;
    V = (col_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(col_t));
    for (int64_t j = 0; j < m; j++) {
      col_reserve(&V[j], 1);
      V[j].v[0] = (int32_t)j;
      V[j].n = 1;
    }
  }
  for (int64_t i = 0; i < m; i++) pivot_of[i] = -1;
  int64_t adds = 0, xors = 0;
  for (int64_t j = 0; j < m; j++) {
    int32_t lo;
    while ((lo = col_low(&R[j])) >= 0 && pivot_of[lo] >= 0) {
      int32_t j0 = pivot_of[lo];
      xors += col_add(&R[j], &R[j0], &tmp);
      if (V) col_add(&V[j], &V[j0], &tmp);
      adds++;
    }
    if (lo >= 0) pivot_of[lo] = (int32_t)j;
    low_out[j] = lo;
  }
  if (stats) {
    stats[0] = adds;
    stats[1] = xors;
  }
  if (v_dense) {
    memset(v_dense, 0, (size_t)(m * m));
    if (r_dense) memset(r_dense, 0, (size_t)(m * m));
    for (int64_t j = 0; j < m; j++) {
      for (int64_t k = 0; k < V[j].n; k++) v_dense[(int64_t)V[j].v[k] * m + j] = 1;
      if (r_dense)
        for (int64_t k = 0; k < R[j].n; k++) r_dense[(int64_t)R[j].v[k] * m + j] = 1;
    }
    cols_free(V, m);
  }
  cols_free(R, m);
  free(pivot_of);
  free(tmp.v);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 3, standard reduction with a twist: dimensions in decreasing order; after column  */
/* j is reduced to a nonzero column, column low(j) is set to zero (clearing, justified by      */
/* Lemma 1). stats: [0] column additions, [1] nontrivial XORs, [2] cleared columns.            */
/* ------------------------------------------------------------------------------------------ */
int orc_reduce_twist(int64_t m, const int64_t* colptr, const int32_t* rows, const int32_t* dim,
                     int32_t* low_out, int64_t* stats) {
  col_t* R = cols_from_csc(m, colptr, rows);
  int32_t* pivot_of = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  col_t tmp = {0, 0, 0};
  if (!R || !pivot_of) return ORC_ERR_ALLOC;
  int32_t maxd = 0;
  for (int64_t j = 0; j < m; j++)
    if (dim[j] > maxd) maxd = dim[j];
  for (int64_t i = 0; i < m; i++) pivot_of[i] = -1;
  int64_t adds = 0, xors = 0, cleared = 0;
  for (int32_t d = maxd; d >= 1; d--) {
    for (int64_t j = 0; j < m; j++) {
      if (dim[j] != d) continue;
      int32_t lo;
      while ((lo = col_low(&R[j])) >= 0 && pivot_of[lo] >= 0) {
        xors += col_add(&R[j], &R[pivot_of[lo]], &tmp);
        adds++;
      }
      if (lo >= 0) {
        pivot_of[lo] = (int32_t)j;
        if (R[lo].n) cleared++;
        R[lo].n = 0; /* clearing */
      }
    }
  }
  for (int64_t j = 0; j < m; j++) low_out[j] = col_low(&R[j]);
  if (stats) {
    stats[0] = adds;
    stats[1] = xors;
    stats[2] = cleared;
  }
  cols_free(R, m);
  free(pivot_of);
  free(tmp.v);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 2, parallel multi-scale reduction, executed as a sequence of passes. A pass is one */
/* cycle of the outermost loop (Sec. 4): every decision in it is taken from the state at the  */
/* start of the pass, so the sequential loops below compute exactly what a data-parallel      */
/* execution of the same pass computes.                                                        */
/*                                                                                              */
/* Pass:                                                                                        */
/*  1. tab[i]   = left-most column j with low(j) = i, over all columns.                        */
/*  2. Paired   = rows known to be negative (beta > 0 by Thm 5 P.3, or proven pivots) plus rows */
/*                that are the low of a proven pivot (Eq. paired, Sec. 3.2).                    */
/*  3. Marks, per dimension d >= 1 over the active columns of K_d in filtration order:          */
/*     - low(j) = 0 (empty)                        -> final, positive;                          */
/*     - low(j) = beta_j  (Thm 5, Phase 0/II test) -> pivot;                                     */
/*     - Phase I (Algorithm 5): j is left-most for its low and low(j) exceeds every low of an   */
/*       earlier colliding column (Thms 6-7)       -> pivot;                                     */
/*     - zero case of Corollary 10: beta_j = 0 and every row of K_{d-1} up to low(j) is in      */
/*       Paired                                    -> lowstar(j) = 0, column set to zero.       */
/*  4. Clearing (Lemma 1): for every new pivot j, column low(j) is set to zero.                 */
/*  5. Phase II: every remaining active column l whose low collides receives the left-most      */
/*     column s = tab[low(l)] (a valid left-to-right addition that lowers low(l)); additions   */
/*     are independent because s is never itself a target. If s was zeroed by this pass the    */
/*     addition waits for the next pass. With strict = 1 only proven pivots are used as s,      */
/*     which is the rule printed in Algorithm 2.                                                */
/* The loop stops at the first pass that finds no collision (low injective on its support,    */
/* Sec. 2.3). Otherwise, after max_passes passes with additions, one more pass applies its     */
/* marks and clearing but no additions, and ORC_NOT_CONVERGED is returned with that valid      */
/* partial state. *passes_out is the number of passes that found collisions.                   */
/*                                                                                              */
/* pass_stats (max_passes+1 rows of ORC_PS_N int64), per pass:                                  */
/*   0 active columns at pass start   1 new pivots       2 empty columns finalised              */
/*   3 Cor-10 zeroings                4 cleared columns that were active                        */
/*   5 colliding columns (targets)    6 additions done   7 nontrivial XORs                      */
/*   8 |E| after the pass (essential estimate, Eq. essential_iteration)                         */
/*   9 columns whose pair is predicted by Corollary 10 (non-zero case) for the first time       */
/*  10 columns with an empty candidate set L_j (impossible by Lemma 9; counted as a check)      */
/*                                                                                              */
/* Phase II with p processors (sets > 0; Sec. 3.4.1-3.4.2): the targets of a pass fall into   */
/* neighbour sets N, one per row i, holding the targets whose addition this pass may do        */
/* (source tab[i], eligible as above). Only the targets of the first p sets in priority order  */
/* receive their addition; the rest stay active unchanged. Order: priority 0 by |N| (larger    */
/* first, Sec. 3.4.1); priority 1 by the number of targets known to be negative (beta >= 0,    */
/* Thm 5), then by |N| (Sec. 3.4.2); ties by the smaller row i.                                */
/*                                                                                              */
/* Corollary 10, non-zero case (pred_out): for an active column j of dimension d >= 1 with      */
/* beta_j >= 0 (hence negative, Thm 5, so 0 is not a candidate) that this pass neither proves   */
/* nor zeroes, L_j is the set of rows of K_{d-1} in [beta_j, low(j)] not in Paired (start of    */
/* the pass). If it holds one row i, lowstar(j) = i (Lemma 9): pred_out[j] = i from then on.    */
/* ------------------------------------------------------------------------------------------ */
#define ORC_PS_N 11
#define ORC_MAX_DIM 16

/* priority order of neighbour sets (rows): key1 descending, then key2 descending, then row */
static const int64_t* g_set_key1;
static const int64_t* g_set_key2;
static int cmp_sets(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  if (g_set_key1[x] != g_set_key1[y]) return g_set_key1[x] > g_set_key1[y] ? -1 : 1;
  if (g_set_key2[x] != g_set_key2[y]) return g_set_key2[x] > g_set_key2[y] ? -1 : 1;
  return x < y ? -1 : (x > y);
}

/* The reduced matrix R at the end (optional, r_colptr != NULL): CSC with m + 1 offsets and,
 * when r_rows is given and holds r_cap entries, the rows; *r_nnz receives their number. */
static int pms_run(int64_t m, const int64_t* colptr, const int32_t* rows, const int32_t* dim,
                   const int32_t* beta, int32_t max_passes, int32_t strict, int32_t use_cor10,
                   int32_t sets, int32_t priority, int32_t* low_out, int64_t* pass_stats,
                   int32_t* passes_out, uint8_t* ess_est_out, uint8_t* proven_out,
                   int32_t* pred_out, int64_t* r_colptr, int32_t* r_rows, int64_t r_cap,
                   int64_t* r_nnz) {
  col_t* R = cols_from_csc(m, colptr, rows);
  int64_t M = m > 0 ? m : 1;
  int32_t* low = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  int32_t* tab = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  int32_t* owner = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  uint8_t* proven = (uint8_t*)calloc((size_t)M, 1);
  uint8_t* final_ = (uint8_t*)calloc((size_t)M, 1);
  uint8_t* newpiv = (uint8_t*)calloc((size_t)M, 1);
  uint8_t* zeroed = (uint8_t*)calloc((size_t)M, 1); /* zeroed during the current pass */
  uint8_t* in_E = (uint8_t*)malloc((size_t)M);
  uint8_t* unpaired = (uint8_t*)malloc((size_t)M); /* start of the pass */
  int32_t* pred = (int32_t*)malloc((size_t)M * sizeof(int32_t));
  int64_t* set_n = (int64_t*)calloc((size_t)M, sizeof(int64_t));   /* |N| per row */
  int64_t* set_neg = (int64_t*)calloc((size_t)M, sizeof(int64_t)); /* targets with beta >= 0 */
  int64_t* set_rows = (int64_t*)malloc((size_t)M * sizeof(int64_t));
  uint8_t* set_on = (uint8_t*)calloc((size_t)M, 1);                /* set acted on this pass */
  col_t tmp = {0, 0, 0};
  if (!R || !low || !tab || !owner || !proven || !final_ || !newpiv || !zeroed || !in_E ||
      !unpaired || !pred || !set_n || !set_neg || !set_rows || !set_on)
    return ORC_ERR_ALLOC;
  int32_t maxd = 0;
  for (int64_t j = 0; j < m; j++)
    if (dim[j] > maxd) maxd = dim[j];
  if (maxd >= ORC_MAX_DIM) return ORC_ERR_INVALID;
  int64_t first_unpaired[ORC_MAX_DIM];
  for (int64_t j = 0; j < m; j++) {
    low[j] = col_low(&R[j]);
    owner[j] = -1;
    in_E[j] = 1; /* E^0 = [m] */
    pred[j] = -1;
  }
  int status = ORC_NOT_CONVERGED;
  int32_t pass = 0;
  for (pass = 0;; pass++) {
    int64_t* ps = pass_stats ? pass_stats + (int64_t)pass * ORC_PS_N : NULL;
    int64_t st[ORC_PS_N] = {0};
    /* 1. left-most column per low */
    for (int64_t i = 0; i < m; i++) tab[i] = -1;
    for (int64_t j = 0; j < m; j++)
      if (low[j] >= 0 && tab[low[j]] < 0) tab[low[j]] = (int32_t)j;
    /* 2. first row of each dimension that is not known to be paired */
    for (int d = 0; d < ORC_MAX_DIM; d++) first_unpaired[d] = m;
    for (int64_t x = m - 1; x >= 0; x--) {
      int paired = proven[x] || beta[x] >= 0 || owner[x] >= 0;
      unpaired[x] = (uint8_t)!paired;
      if (!paired) first_unpaired[dim[x]] = x;
    }
    /* 3. marks from the start-of-pass state */
    memset(newpiv, 0, (size_t)M);
    memset(zeroed, 0, (size_t)M);
    for (int32_t d = 0; d <= maxd; d++) {
      int32_t P = -1; /* running maximum of colliding lows (maxCollision of Algorithm 5) */
      for (int64_t j = 0; j < m; j++) {
        if (dim[j] != d || proven[j] || final_[j]) continue;
        st[0]++;
        if (low[j] < 0) {
          zeroed[j] = 1;
          st[2]++;
          continue;
        }
        int leftmost = tab[low[j]] == j;
        if (leftmost && (low[j] == beta[j] || low[j] > P)) {
          newpiv[j] = 1;
          st[1]++;
        } else if (use_cor10 && d >= 1 && beta[j] < 0 && low[j] < first_unpaired[d - 1]) {
          zeroed[j] = 1;
          st[3]++;
        } else if (d >= 1 && beta[j] >= 0) {
          /* the candidate set L_j: unpaired rows of K_{d-1} in [beta_j, low(j)] */
          int64_t n_cand = 0, last = -1;
          for (int64_t x = beta[j]; x <= low[j]; x++)
            if (dim[x] == d - 1 && unpaired[x]) {
              n_cand++;
              last = x;
            }
          if (n_cand == 0) st[10]++;
          if (n_cand == 1 && pred[j] < 0) {
            pred[j] = (int32_t)last;
            st[9]++;
          }
        }
        if (!leftmost && low[j] > P) P = low[j];
      }
    }
    /* 4. apply: new pivots, clearing, zeroings */
    for (int64_t j = 0; j < m; j++) {
      if (!newpiv[j]) continue;
      int32_t i = low[j];
      proven[j] = 1;
      owner[i] = (int32_t)j;
      if (!proven[i] && !final_[i]) st[4]++;
      zeroed[i] = 1; /* clearing */
    }
    for (int64_t j = 0; j < m; j++) {
      if (zeroed[j] && !final_[j]) {
        final_[j] = 1;
        R[j].n = 0;
        low[j] = -1;
      }
    }
    /* essential estimate: E <- (E \ Paired) \ low([m]), with lows taken before this pass's
     * additions and Paired after its marks */
    for (int64_t x = 0; x < m; x++)
      if (proven[x] || beta[x] >= 0 || owner[x] >= 0) in_E[x] = 0;
    for (int64_t j = 0; j < m; j++)
      if (tab[j] >= 0) in_E[j] = 0; /* j is the low of some column */
    /* 5'. with p processors: the neighbour sets this pass acts on */
    if (sets > 0 && pass < max_passes) {
      memset(set_n, 0, (size_t)M * sizeof(int64_t));
      memset(set_neg, 0, (size_t)M * sizeof(int64_t));
      memset(set_on, 0, (size_t)M);
      for (int64_t l = 0; l < m; l++) {
        if (proven[l] || final_[l]) continue;
        int32_t s = tab[low[l]];
        if (s == l || zeroed[s] || (strict && !proven[s])) continue;
        set_n[low[l]]++;
        if (beta[l] >= 0) set_neg[low[l]]++;
      }
      int64_t nsets = 0;
      for (int64_t i = 0; i < m; i++)
        if (set_n[i] > 0) set_rows[nsets++] = i;
      g_set_key1 = priority == 1 ? set_neg : set_n;
      g_set_key2 = set_n; /* priority 0: the same key again, so rows decide ties */
      qsort(set_rows, (size_t)nsets, sizeof(int64_t), cmp_sets);
      for (int64_t k = 0; k < nsets && k < sets; k++) set_on[set_rows[k]] = 1;
    }
    /* 5. Phase II additions (none once max_passes passes with additions have been done) */
    for (int64_t l = 0; l < m; l++) {
      if (proven[l] || final_[l]) continue;
      int32_t s = tab[low[l]];
      if (s == l) continue;
      st[5]++;
      if (pass >= max_passes) continue;
      if (zeroed[s]) continue; /* source zeroed by this pass */
      if (strict && !proven[s]) continue;
      if (sets > 0 && !set_on[low[l]]) continue; /* its set waits for a later pass */
      int64_t x = col_add(&R[l], &R[s], &tmp);
      if (x < 0) return ORC_ERR_ALLOC;
      st[6]++;
      st[7] += x;
      low[l] = col_low(&R[l]);
    }
    int64_t ecount = 0;
    for (int64_t x = 0; x < m; x++) ecount += in_E[x];
    st[8] = ecount;
    if (ps) memcpy(ps, st, sizeof(st));
    if (st[5] == 0) {
      status = ORC_OK;
      break;
    }
    if (pass >= max_passes) break; /* ORC_NOT_CONVERGED; the state stays a valid partial one */
  }
  if (passes_out) *passes_out = pass;
  for (int64_t j = 0; j < m; j++) low_out[j] = low[j];
  if (ess_est_out) memcpy(ess_est_out, in_E, (size_t)m);
  if (proven_out) memcpy(proven_out, proven, (size_t)m);
  if (pred_out) memcpy(pred_out, pred, (size_t)m * sizeof(int32_t));
  if (r_colptr) {
    r_colptr[0] = 0;
    for (int64_t j = 0; j < m; j++) r_colptr[j + 1] = r_colptr[j] + R[j].n;
    if (r_nnz) *r_nnz = r_colptr[m];
    if (r_rows && r_colptr[m] <= r_cap)
      for (int64_t j = 0; j < m; j++)
        memcpy(r_rows + r_colptr[j], R[j].v, (size_t)R[j].n * sizeof(int32_t));
  }
  cols_free(R, m);
  free(low);
  free(tab);
  free(owner);
  free(proven);
  free(final_);
  free(newpiv);
  free(zeroed);
  free(in_E);
  free(unpaired);
  free(pred);
  free(set_n);
  free(set_neg);
  free(set_rows);
  free(set_on);
  free(tmp.v);
  return status;
}

int orc_reduce_pms(int64_t m, const int64_t* colptr, const int32_t* rows, const int32_t* dim,
                   const int32_t* beta, int32_t max_passes, int32_t strict, int32_t use_cor10,
                   int32_t sets, int32_t priority, int32_t* low_out, int64_t* pass_stats,
                   int32_t* passes_out, uint8_t* ess_est_out, uint8_t* proven_out,
                   int32_t* pred_out) {
  return pms_run(m, colptr, rows, dim, beta, max_passes, strict, use_cor10, sets, priority,
                 low_out, pass_stats, passes_out, ess_est_out, proven_out, pred_out, NULL, NULL,
                 0, NULL);
}

/* orc_reduce_pms that also returns the reduced matrix R (CSC, rows ascending): call with
 * r_rows = NULL for r_colptr and *r_nnz, then with r_rows of r_cap >= *r_nnz entries. */
int orc_reduce_pms_columns(int64_t m, const int64_t* colptr, const int32_t* rows,
                           const int32_t* dim, const int32_t* beta, int32_t max_passes,
                           int32_t strict, int32_t use_cor10, int32_t sets, int32_t priority,
                           int32_t* low_out, int64_t* r_colptr, int32_t* r_rows, int64_t r_cap,
                           int64_t* r_nnz) {
  return pms_run(m, colptr, rows, dim, beta, max_passes, strict, use_cor10, sets, priority,
                 low_out, NULL, NULL, NULL, NULL, NULL, r_colptr, r_rows, r_cap, r_nnz);
}
