/*
 * h2gen: seeded synthetic H^2 covariance matrices, built ab initio the way the
 * paper's experiments build theirs (Sec. 4.6): points -> KD cluster tree ->
 * Chebyshev interpolation bases and transfers -> dual traversal -> coupling
 * blocks (kernel at interpolation points) and dense leaf blocks (kernel at
 * points).
 *
 * This module produces INPUTS only. It holds none of the matrix-vector
 * product's arithmetic (no upsweep, coupling product, downsweep or dense
 * product); both the CPU oracle and the CUDA library consume its arrays.
 *
 * Output layout (the library's input format; every block column-major):
 *   tree      complete binary tree of depth q, nodes in heap order
 *             (root 0, children of h are 2h+1 and 2h+2, level l holds nodes
 *             2^l-1 .. 2^(l+1)-2), leaves = level q.
 *   leaf_offset[2^q+1]   point ranges of the leaves in cluster order.
 *   U        leaf i: size_i x k at U + leaf_offset[i]*k   (V == U, symmetric)
 *   E        node h >= 1: k x k transfer at E + (h-1)*k*k  (F == E)
 *            E_c[mu,nu] = L^{parent}_nu(xi^c_mu)  (Eq. 1: U_p = [U_c1 E_c1; U_c2 E_c2])
 *   S        block-sparse rows over ALL nodes: S_rowptr[N_nodes+1], S_colidx
 *            = heap index of the column node (same level as the row),
 *            S_val + b*k*k: S_ij[nu,mu] = K(xi^i_nu, xi^j_mu).
 *   D        block-sparse rows over the leaves: D_rowptr[2^q+1], D_colidx =
 *            leaf index, D_val + D_valoff[b]: size_i x size_j, D[a,b] = K(x_a,x_b).
 *
 * Readings of points the paper leaves open:
 *   split    longest side of the tight bounding box; left child gets
 *            ceil(s/2) points ordered by (coordinate, original index), so all
 *            leaves sit on level q = ceil(log2(n/m)) with size <= m.
 *   boxes    tight axis-aligned bounding boxes; a side narrower than 1e-10 is
 *            widened symmetrically to 1e-10 for the interpolation nodes.
 *   nodes    first-kind Chebyshev points, tensor index with dimension 0 slowest.
 *   admiss.  eta > 0, dist > 0 and max(diam_i, diam_j) <= eta * dist(box_i, box_j)
 *            (diam = box diagonal, dist = Euclidean gap between boxes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define H2GEN_MAXDIM 3
#define H2GEN_MAXP 16

enum { KER_EXP = 0, KER_MATERN32 = 1, KER_POLY = 2, KER_CONST = 3 };

/* ---------------- counter-free seeded generator: xoshiro256** ---------------- */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return result;
}
static double rng_u01(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
/* Box-Muller, cosine branch only: one normal per two uniforms. */
static double rng_normal(rng_t* r) {
  double u1 = 1.0 - rng_u01(r); /* (0, 1] */
  double u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

void h2gen_uniform(uint64_t seed, int64_t count, double* out) {
  rng_t r; rng_seed(&r, seed);
  for (int64_t i = 0; i < count; i++) out[i] = rng_u01(&r);
}
void h2gen_normal(uint64_t seed, int64_t count, double* out) {
  rng_t r; rng_seed(&r, seed);
  for (int64_t i = 0; i < count; i++) out[i] = rng_normal(&r);
}

/* ---------------- kernels ---------------- */
typedef struct { int kind, dim, p; double ell; } kern_t;

static inline double kernel_eval(const kern_t* K, const double* x, const double* y) {
  if (K->kind == KER_CONST) return 1.0;
  if (K->kind == KER_POLY) { /* degree p-1 in every coordinate of x and of y */
    double v = 1.0;
    for (int d = 0; d < K->dim; d++) {
      double t = 1.0 + x[d] * y[d];
      for (int e = 0; e < K->p - 1; e++) v *= t;
    }
    return v;
  }
  double r2 = 0.0;
  for (int d = 0; d < K->dim; d++) { double t = x[d] - y[d]; r2 += t * t; }
  double r = sqrt(r2);
  if (K->kind == KER_EXP) return exp(-r / K->ell);
  /* Matern 3/2, unit variance */
  double s = 1.7320508075688772 * r / K->ell;
  return (1.0 + s) * exp(-s);
}

/* ---------------- handle ---------------- */
typedef struct {
  int dim, m, p, k, q;
  int64_t n, n_nodes, leaves;
  double eta;
  kern_t K;
  double* pts;      /* n*dim, cluster order */
  int64_t* perm;    /* cluster position -> original index */
  int64_t* lo;      /* n_nodes: first point */
  int64_t* hi;      /* n_nodes: one past last point */
  double* bmin;     /* n_nodes*dim tight box */
  double* bmax;
  double* cheb;     /* n_nodes*dim*p: 1D Chebyshev nodes per node and dimension */
  int64_t nS, capS; int64_t* Srow; int64_t* Scol;  /* heap indices */
  int64_t nD, capD; int64_t* Drow; int64_t* Dcol;  /* leaf indices */
  int32_t* S_rowptr; int32_t* S_colidx;
  int32_t* D_rowptr; int32_t* D_colidx; int64_t* D_valoff;
} h2gen_t;

typedef struct { double key; int64_t orig; int64_t pos; } sortrec_t;
static int cmp_rec(const void* a, const void* b) {
  const sortrec_t* x = (const sortrec_t*)a; const sortrec_t* y = (const sortrec_t*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->orig < y->orig) ? -1 : (x->orig > y->orig);
}

static void node_box(const h2gen_t* g, int64_t lo, int64_t hi, double* bmin, double* bmax) {
  for (int d = 0; d < g->dim; d++) { bmin[d] = INFINITY; bmax[d] = -INFINITY; }
  for (int64_t i = lo; i < hi; i++)
    for (int d = 0; d < g->dim; d++) {
      double v = g->pts[i * g->dim + d];
      if (v < bmin[d]) bmin[d] = v;
      if (v > bmax[d]) bmax[d] = v;
    }
}

/* split the node's point range along the longest box side (ties: lowest dim) */
static void split_node(h2gen_t* g, int64_t lo, int64_t hi, sortrec_t* rec, double* tmp_pts, int64_t* tmp_perm) {
  int dim = g->dim;
  double bmin[H2GEN_MAXDIM], bmax[H2GEN_MAXDIM];
  node_box(g, lo, hi, bmin, bmax);
  int ds = 0; double w = bmax[0] - bmin[0];
  for (int d = 1; d < dim; d++) if (bmax[d] - bmin[d] > w) { w = bmax[d] - bmin[d]; ds = d; }
  int64_t s = hi - lo;
  for (int64_t i = 0; i < s; i++) { rec[i].key = g->pts[(lo + i) * dim + ds]; rec[i].orig = g->perm[lo + i]; rec[i].pos = lo + i; }
  qsort(rec, (size_t)s, sizeof(sortrec_t), cmp_rec);
  for (int64_t i = 0; i < s; i++) {
    for (int d = 0; d < dim; d++) tmp_pts[i * dim + d] = g->pts[rec[i].pos * dim + d];
    tmp_perm[i] = g->perm[rec[i].pos];
  }
  memcpy(g->pts + lo * dim, tmp_pts, (size_t)s * dim * sizeof(double));
  memcpy(g->perm + lo, tmp_perm, (size_t)s * sizeof(int64_t));
}

static double box_diam(const h2gen_t* g, int64_t h) {
  double s = 0;
  for (int d = 0; d < g->dim; d++) { double t = g->bmax[h * g->dim + d] - g->bmin[h * g->dim + d]; s += t * t; }
  return sqrt(s);
}
static double box_dist(const h2gen_t* g, int64_t a, int64_t b) {
  double s = 0;
  for (int d = 0; d < g->dim; d++) {
    double gap = 0, t1 = g->bmin[b * g->dim + d] - g->bmax[a * g->dim + d], t2 = g->bmin[a * g->dim + d] - g->bmax[b * g->dim + d];
    if (t1 > gap) gap = t1;
    if (t2 > gap) gap = t2;
    s += gap * gap;
  }
  return sqrt(s);
}

static int push_pair(int64_t** rows, int64_t** cols, int64_t* cnt, int64_t* cap, int64_t r, int64_t c) {
  if (*cnt == *cap) {
    int64_t nc = *cap ? *cap * 2 : 1024;
    int64_t* nr = (int64_t*)realloc(*rows, (size_t)nc * sizeof(int64_t));
    if (!nr) return -1;
    *rows = nr;
    int64_t* ncl = (int64_t*)realloc(*cols, (size_t)nc * sizeof(int64_t));
    if (!ncl) return -1;
    *cols = ncl;
    *cap = nc;
  }
  (*rows)[*cnt] = r; (*cols)[*cnt] = c; (*cnt)++;
  return 0;
}

/* dual traversal of the (row tree, column tree) pair, both the same cluster tree */
static int dual_traverse(h2gen_t* g, int64_t i, int64_t j, int level) {
  double dist = box_dist(g, i, j);
  double di = box_diam(g, i), dj = box_diam(g, j);
  double dm = di > dj ? di : dj;
  if (g->eta > 0 && dist > 0 && dm <= g->eta * dist)
    return push_pair(&g->Srow, &g->Scol, &g->nS, &g->capS, i, j);
  if (level == g->q) {
    int64_t first = ((int64_t)1 << g->q) - 1;
    return push_pair(&g->Drow, &g->Dcol, &g->nD, &g->capD, i - first, j - first);
  }
  for (int a = 1; a <= 2; a++)
    for (int b = 1; b <= 2; b++)
      if (dual_traverse(g, 2 * i + a, 2 * j + b, level + 1)) return -1;
  return 0;
}

typedef struct { int64_t r, c; } pair_t;
static int cmp_pair(const void* a, const void* b) {
  const pair_t* x = (const pair_t*)a; const pair_t* y = (const pair_t*)b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  return (x->c < y->c) ? -1 : (x->c > y->c);
}
static int to_bsr(int64_t cnt, const int64_t* rows, const int64_t* cols, int64_t nrows, int32_t* rowptr, int32_t* colidx) {
  pair_t* P = (pair_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(pair_t));
  if (!P) return -1;
  for (int64_t i = 0; i < cnt; i++) { P[i].r = rows[i]; P[i].c = cols[i]; }
  qsort(P, (size_t)cnt, sizeof(pair_t), cmp_pair);
  for (int64_t r = 0; r <= nrows; r++) rowptr[r] = 0;
  for (int64_t i = 0; i < cnt; i++) { rowptr[P[i].r + 1]++; colidx[i] = (int32_t)P[i].c; }
  for (int64_t r = 0; r < nrows; r++) rowptr[r + 1] += rowptr[r];
  free(P);
  return 0;
}

void h2gen_free(void* hp) {
  h2gen_t* g = (h2gen_t*)hp;
  if (!g) return;
  free(g->pts); free(g->perm); free(g->lo); free(g->hi); free(g->bmin); free(g->bmax); free(g->cheb);
  free(g->Srow); free(g->Scol); free(g->Drow); free(g->Dcol);
  free(g->S_rowptr); free(g->S_colidx); free(g->D_rowptr); free(g->D_colidx); free(g->D_valoff);
  free(g);
}

/*
 * Build the cluster tree, boxes, Chebyshev nodes and block lists.
 * points_or_null: n*dim points in original order (row-major) or NULL for
 * uniform points in [0,1]^dim drawn from `seed`.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int h2gen_build(int dim, int64_t n, int m, int p, double eta, int kernel, double ell, uint64_t seed,
                const double* points_or_null, void** out) {
  *out = NULL;
  if (dim < 1 || dim > H2GEN_MAXDIM || n < 1 || m < 1 || p < 1 || p > H2GEN_MAXP || kernel < 0 || kernel > 3) return -1;
  h2gen_t* g = (h2gen_t*)calloc(1, sizeof(h2gen_t));
  if (!g) return -2;
  g->dim = dim; g->n = n; g->m = m; g->p = p; g->eta = eta;
  int k = 1; for (int d = 0; d < dim; d++) k *= p;
  g->k = k;
  int q = 0; while (((int64_t)m << q) < n) q++;
  g->q = q;
  g->leaves = (int64_t)1 << q;
  g->n_nodes = ((int64_t)2 << q) - 1;
  g->K.kind = kernel; g->K.dim = dim; g->K.p = p; g->K.ell = ell;
  g->pts = (double*)malloc((size_t)n * dim * sizeof(double));
  g->perm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  g->lo = (int64_t*)malloc((size_t)g->n_nodes * sizeof(int64_t));
  g->hi = (int64_t*)malloc((size_t)g->n_nodes * sizeof(int64_t));
  g->bmin = (double*)malloc((size_t)g->n_nodes * dim * sizeof(double));
  g->bmax = (double*)malloc((size_t)g->n_nodes * dim * sizeof(double));
  g->cheb = (double*)malloc((size_t)g->n_nodes * dim * p * sizeof(double));
  if (!g->pts || !g->perm || !g->lo || !g->hi || !g->bmin || !g->bmax || !g->cheb) { h2gen_free(g); return -2; }
  if (points_or_null) memcpy(g->pts, points_or_null, (size_t)n * dim * sizeof(double));
  else h2gen_uniform(seed, n * dim, g->pts);
  for (int64_t i = 0; i < n; i++) g->perm[i] = i;

  /* KD bisection, level by level */
  g->lo[0] = 0; g->hi[0] = n;
  sortrec_t* rec = (sortrec_t*)malloc((size_t)n * sizeof(sortrec_t));
  double* tmp_pts = (double*)malloc((size_t)n * dim * sizeof(double));
  int64_t* tmp_perm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!rec || !tmp_pts || !tmp_perm) { free(rec); free(tmp_pts); free(tmp_perm); h2gen_free(g); return -2; }
  for (int l = 0; l < q; l++) {
    int64_t first = ((int64_t)1 << l) - 1, cnt = (int64_t)1 << l;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < cnt; t++) {
      int64_t h = first + t, lo = g->lo[h], hi = g->hi[h];
      split_node(g, lo, hi, rec + lo, tmp_pts + lo * dim, tmp_perm + lo);
      int64_t mid = lo + (hi - lo + 1) / 2;
      g->lo[2 * h + 1] = lo; g->hi[2 * h + 1] = mid;
      g->lo[2 * h + 2] = mid; g->hi[2 * h + 2] = hi;
    }
  }
  free(rec); free(tmp_pts); free(tmp_perm);

  /* tight boxes and Chebyshev nodes */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t h = 0; h < g->n_nodes; h++) {
    node_box(g, g->lo[h], g->hi[h], g->bmin + h * dim, g->bmax + h * dim);
    for (int d = 0; d < dim; d++) {
      double a = g->bmin[h * dim + d], b = g->bmax[h * dim + d];
      if (b - a < 1e-10) { double c = 0.5 * (a + b); a = c - 0.5e-10; b = c + 0.5e-10; }
      for (int v = 0; v < p; v++)
        g->cheb[(h * dim + d) * p + v] = 0.5 * (a + b) + 0.5 * (b - a) * cos((2.0 * v + 1.0) * 3.141592653589793 / (2.0 * p));
    }
  }

  if (dual_traverse(g, 0, 0, 0)) { h2gen_free(g); return -2; }
  if (g->nS >= INT32_MAX || g->nD >= INT32_MAX) { h2gen_free(g); return -1; }
  g->S_rowptr = (int32_t*)malloc((size_t)(g->n_nodes + 1) * sizeof(int32_t));
  g->S_colidx = (int32_t*)malloc((size_t)(g->nS > 0 ? g->nS : 1) * sizeof(int32_t));
  g->D_rowptr = (int32_t*)malloc((size_t)(g->leaves + 1) * sizeof(int32_t));
  g->D_colidx = (int32_t*)malloc((size_t)(g->nD > 0 ? g->nD : 1) * sizeof(int32_t));
  g->D_valoff = (int64_t*)malloc((size_t)(g->nD + 1) * sizeof(int64_t));
  if (!g->S_rowptr || !g->S_colidx || !g->D_rowptr || !g->D_colidx || !g->D_valoff) { h2gen_free(g); return -2; }
  if (to_bsr(g->nS, g->Srow, g->Scol, g->n_nodes, g->S_rowptr, g->S_colidx)) { h2gen_free(g); return -2; }
  if (to_bsr(g->nD, g->Drow, g->Dcol, g->leaves, g->D_rowptr, g->D_colidx)) { h2gen_free(g); return -2; }
  int64_t leaf0 = g->leaves - 1;
  g->D_valoff[0] = 0;
  for (int64_t i = 0; i < g->leaves; i++)
    for (int32_t b = g->D_rowptr[i]; b < g->D_rowptr[i + 1]; b++) {
      int64_t si = g->hi[leaf0 + i] - g->lo[leaf0 + i];
      int64_t j = g->D_colidx[b];
      int64_t sj = g->hi[leaf0 + j] - g->lo[leaf0 + j];
      g->D_valoff[b + 1] = g->D_valoff[b] + si * sj;
    }
  *out = g;
  return 0;
}

/* info[0]=q info[1]=k info[2]=nS info[3]=nD info[4]=D value count info[5]=n_nodes info[6]=leaves */
void h2gen_info(void* hp, int64_t* info) {
  h2gen_t* g = (h2gen_t*)hp;
  info[0] = g->q; info[1] = g->k; info[2] = g->nS; info[3] = g->nD;
  info[4] = g->D_valoff[g->nD]; info[5] = g->n_nodes; info[6] = g->leaves;
}

/* the first-kind Chebyshev nodes of every node's box: n_nodes*dim*p, node h
   dimension d at (h*dim + d)*p (the interpolation points are their tensor grid,
   dimension 0 slowest) */
int h2gen_fill_cheb(void* hp, double* cheb) {
  const h2gen_t* g = (const h2gen_t*)hp;
  memcpy(cheb, g->cheb, (size_t)g->n_nodes * g->dim * g->p * sizeof(double));
  return 0;
}

int h2gen_fill_structure(void* hp, double* pts, int64_t* perm, int64_t* leaf_offset, int32_t* S_rowptr, int32_t* S_colidx,
                         int32_t* D_rowptr, int32_t* D_colidx, int64_t* D_valoff) {
  h2gen_t* g = (h2gen_t*)hp;
  memcpy(pts, g->pts, (size_t)g->n * g->dim * sizeof(double));
  memcpy(perm, g->perm, (size_t)g->n * sizeof(int64_t));
  int64_t leaf0 = g->leaves - 1;
  for (int64_t i = 0; i < g->leaves; i++) leaf_offset[i] = g->lo[leaf0 + i];
  leaf_offset[g->leaves] = g->n;
  memcpy(S_rowptr, g->S_rowptr, (size_t)(g->n_nodes + 1) * sizeof(int32_t));
  if (g->nS) memcpy(S_colidx, g->S_colidx, (size_t)g->nS * sizeof(int32_t));
  memcpy(D_rowptr, g->D_rowptr, (size_t)(g->leaves + 1) * sizeof(int32_t));
  if (g->nD) memcpy(D_colidx, g->D_colidx, (size_t)g->nD * sizeof(int32_t));
  memcpy(D_valoff, g->D_valoff, (size_t)(g->nD + 1) * sizeof(int64_t));
  return 0;
}

/* Lagrange basis polynomial number `a` of the 1D node set xi[0..p-1], at t */
static inline double lagrange1(const double* xi, int p, int a, double t) {
  double v = 1.0;
  for (int b = 0; b < p; b++)
    if (b != a) v *= (t - xi[b]) / (xi[a] - xi[b]);
  return v;
}
/* tensor Lagrange basis function nu (dimension 0 slowest) of node h at point x */
static inline double lagrange_tensor(const h2gen_t* g, int64_t h, int nu, const double* x) {
  double v = 1.0;
  int rem = nu;
  for (int d = g->dim - 1; d >= 0; d--) {
    int a = rem % g->p; rem /= g->p;
    v *= lagrange1(g->cheb + (h * g->dim + d) * g->p, g->p, a, x[d]);
  }
  return v;
}
/* tensor Chebyshev point nu of node h */
static inline void cheb_point(const h2gen_t* g, int64_t h, int nu, double* x) {
  int rem = nu;
  for (int d = g->dim - 1; d >= 0; d--) {
    int a = rem % g->p; rem /= g->p;
    x[d] = g->cheb[(h * g->dim + d) * g->p + a];
  }
}

/* Fill U (== V), E (== F), S values and D values. Any pointer may be NULL to skip. */
int h2gen_fill_values(void* hp, double* U, double* E, double* S_val, double* D_val) {
  h2gen_t* g = (h2gen_t*)hp;
  int dim = g->dim, k = g->k;
  int64_t leaf0 = g->leaves - 1;
  if (U) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < g->leaves; i++) {
      int64_t h = leaf0 + i, lo = g->lo[h], s = g->hi[h] - lo;
      double* Ui = U + lo * k;
      for (int nu = 0; nu < k; nu++)
        for (int64_t a = 0; a < s; a++) Ui[a + s * nu] = lagrange_tensor(g, h, nu, g->pts + (lo + a) * dim);
    }
  }
  if (E) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 1; c < g->n_nodes; c++) {
      int64_t par = (c - 1) / 2;
      double* Ec = E + (c - 1) * (int64_t)k * k;
      double xc[H2GEN_MAXDIM];
      for (int mu = 0; mu < k; mu++) {
        cheb_point(g, c, mu, xc);
        for (int nu = 0; nu < k; nu++) Ec[mu + (int64_t)k * nu] = lagrange_tensor(g, par, nu, xc);
      }
    }
  }
  if (S_val) {
#pragma omp parallel
    {
      double xi[H2GEN_MAXDIM], xj[H2GEN_MAXDIM];
#pragma omp for schedule(dynamic, 64)
      for (int64_t r = 0; r < g->n_nodes; r++)
        for (int32_t b = g->S_rowptr[r]; b < g->S_rowptr[r + 1]; b++) {
          int64_t j = g->S_colidx[b];
          double* Sb = S_val + (int64_t)b * k * k;
          for (int mu = 0; mu < k; mu++) {
            cheb_point(g, j, mu, xj);
            for (int nu = 0; nu < k; nu++) {
              cheb_point(g, r, nu, xi);
              Sb[nu + (int64_t)k * mu] = kernel_eval(&g->K, xi, xj);
            }
          }
        }
    }
  }
  if (D_val) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < g->leaves; i++) {
      int64_t li = g->lo[leaf0 + i], si = g->hi[leaf0 + i] - li;
      for (int32_t b = g->D_rowptr[i]; b < g->D_rowptr[i + 1]; b++) {
        int64_t j = g->D_colidx[b], lj = g->lo[leaf0 + j], sj = g->hi[leaf0 + j] - lj;
        double* Db = D_val + g->D_valoff[b];
        for (int64_t c = 0; c < sj; c++)
          for (int64_t a = 0; a < si; a++) Db[a + si * c] = kernel_eval(&g->K, g->pts + (li + a) * dim, g->pts + (lj + c) * dim);
      }
    }
  }
  return 0;
}

/*
 * Exact kernel-matrix product for selected rows (cluster order):
 * out[r + nrows*v] = sum_b K(x_rows[r], x_b) x[b + ldx*v]. This is the dense
 * covariance A the H^2 matrix approximates (for the approximation error of
 * Sec. 4.6), not the H^2 product.
 */
int h2gen_exact_matvec_rows(void* hp, const int64_t* rows, int64_t nrows, int nv, const double* x, int64_t ldx, double* out) {
  h2gen_t* g = (h2gen_t*)hp;
  int dim = g->dim;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t r = 0; r < nrows; r++) {
    const double* xa = g->pts + rows[r] * dim;
    for (int v = 0; v < nv; v++) {
      double s = 0.0;
      for (int64_t b = 0; b < g->n; b++) s += kernel_eval(&g->K, xa, g->pts + b * dim) * x[b + ldx * v];
      out[r + nrows * v] = s;
    }
  }
  return 0;
}

/* Exact kernel matrix block: out[r + nrows*c] = K(x_rows[r], x_cols[c]) (cluster order). */
int h2gen_kernel_matrix(void* hp, const int64_t* rows, int64_t nrows, const int64_t* cols, int64_t ncols, double* out) {
  h2gen_t* g = (h2gen_t*)hp;
  int dim = g->dim;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < ncols; c++)
    for (int64_t r = 0; r < nrows; r++) out[r + nrows * c] = kernel_eval(&g->K, g->pts + rows[r] * dim, g->pts + cols[c] * dim);
  return 0;
}
