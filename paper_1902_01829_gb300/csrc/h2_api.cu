// C ABI of the H^2 matrix-vector product library: validation, device layout,
// launch sequence. See include/h2.h for the contract of each entry point.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "h2.h"
#include "hmv_fp64.cuh"
#include "h2_internal.h"
#include "stream_fp64.cuh"

static_assert(sizeof(h2::StreamItem) == 32, "work items are read as two int4");

namespace {

thread_local std::string g_err;

}  // namespace

h2_status h2_fail(h2_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

void h2_internal_set_error(const char* msg) { g_err = msg; }

using namespace h2i;

namespace {

h2_status (&fail)(h2_status, const char*, ...) = h2_fail;

void free_all(h2_matrix_s* h) {
  profile_free(&h->prof);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->side = nullptr;
  h->ev_fork = h->ev_join = nullptr;
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->hx) cudaFree(h->hx);
  if (h->hy) cudaFree(h->hy);
  h->hx = h->hy = nullptr;
}

int level_of(int64_t node) {
  int l = 0;
  while (((int64_t)2 << l) - 1 <= node) l++;
  return l;
}

// values must be finite; the scaled storage forms (FP32 block scales) also need |v| < 2^126
bool values_ok(const double* v, int64_t count, int64_t* bad, bool fp32_range = true) {
  const double lim = fp32_range ? std::ldexp(1.0, 126) : HUGE_VAL;
  for (int64_t i = 0; i < count; i++)
    if (!(std::fabs(v[i]) < lim)) {
      *bad = i;
      return false;
    }
  return true;
}

// ---- range of the FP64 form (exponent offsets, see df64.cuh)
//
// With every vector scaled so that |x'| < 1, the host bounds each intermediate
// of the product by the infinity norms of the blocks that produce it:
//   xhat_leaf <= ||V_j^T||, xhat_p <= sum_c ||F_c^T|| xhat_c          (Alg. 2, Eq. 2)
//   yhat_i <= sum_b ||S_b|| xhat_col(b) + ||E_i|| yhat_parent(i)       (Eq. 3, Eq. 5)
//   y(i) <= sum_b ||D_b|| + ||U_i|| yhat_i                              (Sec. 2.2, Eq. 4)
// Each node's vector is held scaled by 2^-e (2^e >= its bound), and each block
// enters its product split with the exponent offset that maps its input scale
// to its output scale, so every float of the product stays at most about 1.
// Logarithms (base 2) keep the bounds finite for any finite input.

struct BlockStat {
  double lnorm = -HUGE_VAL;  // log2 of the largest row sum of |a| (-inf for a zero block)
  int emax = 0;              // frexp exponent of the largest |a| (0 for a zero block)
  int emin = 0;              // frexp exponent of the smallest nonzero normal |a|
  bool zero = false;         // some entry is zero or an FP64 subnormal
};

// rows x cols block with element (r, c) at a[r * rs + c * cs]
BlockStat block_stat(const double* a, int64_t rows, int64_t cols, int64_t rs, int64_t cs) {
  BlockStat st;
  double mx = 0.0, mn = HUGE_VAL;
  for (int64_t r = 0; r < rows; r++)
    for (int64_t c = 0; c < cols; c++) {
      const double v = std::fabs(a[r * rs + c * cs]);
      if (!(v >= DBL_MIN)) st.zero = true;
      else mn = std::min(mn, v);
      mx = std::max(mx, v);
    }
  if (!(mx >= DBL_MIN)) {
    st.zero = true;
    return st;
  }
  std::frexp(mx, &st.emax);
  std::frexp(mn, &st.emin);
  double best = 0.0;
  for (int64_t r = 0; r < rows; r++) {
    double sum = 0.0;
    for (int64_t c = 0; c < cols; c++) sum += std::ldexp(std::fabs(a[r * rs + c * cs]), -st.emax);
    best = std::max(best, sum);
  }
  st.lnorm = st.emax + std::log2(best);
  return st;
}

// log2(2^a + 2^b)
double lse2(double a, double b) {
  if (a == -HUGE_VAL) return b;
  if (b == -HUGE_VAL) return a;
  const double m = std::max(a, b);
  return m + std::log2(std::exp2(a - m) + std::exp2(b - m));
}

// exponent e with 2^L <= 2^e (0 when the bound is zero)
int exp_of_bound(double L) { return L == -HUGE_VAL ? 0 : (int)std::ceil(L); }

// offset o for a block: the wanted one, raised so that |a'| = |a| 2^-o stays below 2^100
// (that only acts on blocks whose input is zero by its bound)
int block_offset(int want, const BlockStat& st) { return st.zero && st.lnorm == -HUGE_VAL ? 0 : std::max(want, st.emax - 100); }

// some |a'| of the block is below 2^-103 (or zero): the kernel needs the zero-safe split
bool needs_safe_split(const BlockStat& st, int o) { return st.zero || st.emin - 1 - o < -103; }

struct Fp64Ranges {
  std::vector<int32_t> oV, oF, oE, oS, oD, oU, eY;
  std::vector<char> d_safe;
  bool s_tiny = false;
};

Fp64Ranges fp64_ranges(const h2_desc* d, int64_t leaves, int64_t n_nodes, int64_t nS, int64_t nD,
                       const std::vector<int64_t>& doff) {
  const int q = d->depth, k = d->rank;
  const int64_t kk = (int64_t)k * k, leaf0 = leaves - 1;
  const double* V = d->symmetric ? d->U : d->V;
  const double* F = d->symmetric ? d->E : d->F;
  const int64_t* lo = d->leaf_offset;
  std::vector<BlockStat> sV((size_t)leaves), sU((size_t)leaves), sF((size_t)n_nodes), sE((size_t)n_nodes),
      sS((size_t)nS), sD((size_t)nD);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < leaves; j++) {
    const int64_t s = lo[j + 1] - lo[j];
    sV[j] = block_stat(V + lo[j] * k, k, s, s, 1);  // V_j^T: rows nu
    sU[j] = block_stat(d->U + lo[j] * k, s, k, 1, s);
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t c = 1; c < n_nodes; c++) {
    sF[c] = block_stat(F + (c - 1) * kk, k, k, k, 1);  // F_c^T: rows nu
    sE[c] = block_stat(d->E + (c - 1) * kk, k, k, 1, k);
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t b = 0; b < nS; b++) sS[b] = block_stat(d->S_val + b * kk, k, k, 1, k);
  std::vector<int32_t> drow((size_t)nD);
  for (int64_t r = 0; r < leaves; r++)
    for (int32_t b = d->D_rowptr[r]; b < d->D_rowptr[r + 1]; b++) drow[b] = (int32_t)r;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t b = 0; b < nD; b++) {
    const int64_t si = lo[drow[b] + 1] - lo[drow[b]];
    const int64_t sj = (doff[b + 1] - doff[b]) / si;
    sD[b] = block_stat(d->D_val + doff[b], si, sj, 1, si);
  }
  // bounds (log2) of xhat, yhat and y rows
  std::vector<double> bx((size_t)n_nodes, -HUGE_VAL), by((size_t)n_nodes, -HUGE_VAL), bY((size_t)leaves, -HUGE_VAL);
  for (int64_t j = 0; j < leaves; j++) bx[leaf0 + j] = sV[j].lnorm;
  for (int64_t p = leaf0 - 1; p >= 0; p--)
    bx[p] = lse2(sF[2 * p + 1].lnorm + bx[2 * p + 1], sF[2 * p + 2].lnorm + bx[2 * p + 2]);
  for (int64_t i = 0; i < n_nodes; i++)
    for (int32_t b = d->S_rowptr[i]; b < d->S_rowptr[i + 1]; b++) by[i] = lse2(by[i], sS[b].lnorm + bx[d->S_colidx[b]]);
  for (int64_t c = 1; c < n_nodes; c++) by[c] = lse2(by[c], sE[c].lnorm + by[(c - 1) / 2]);
  for (int64_t j = 0; j < leaves; j++) {
    for (int32_t b = d->D_rowptr[j]; b < d->D_rowptr[j + 1]; b++) bY[j] = lse2(bY[j], sD[b].lnorm);
    bY[j] = lse2(bY[j], sU[j].lnorm + by[leaf0 + j]);
  }
  std::vector<int> ex((size_t)n_nodes), ey((size_t)n_nodes);
  for (int64_t h = 0; h < n_nodes; h++) {
    ex[h] = exp_of_bound(bx[h]);
    ey[h] = exp_of_bound(by[h]);
  }
  Fp64Ranges R;
  R.oV.resize((size_t)leaves);
  R.oU.resize((size_t)leaves);
  R.eY.resize((size_t)leaves);
  R.oF.assign((size_t)n_nodes, 0);
  R.oE.assign((size_t)n_nodes, 0);
  R.oS.resize((size_t)nS);
  R.oD.resize((size_t)nD);
  R.d_safe.resize((size_t)nD);
  for (int64_t j = 0; j < leaves; j++) {
    R.eY[j] = exp_of_bound(bY[j]);
    R.oV[j] = block_offset(ex[leaf0 + j], sV[j]);
    R.oU[j] = block_offset(R.eY[j] - ey[leaf0 + j], sU[j]);
  }
  for (int64_t c = 1; c < n_nodes; c++) {
    const int64_t p = (c - 1) / 2;
    R.oF[c] = block_offset(ex[p] - ex[c], sF[c]);
    R.oE[c] = block_offset(ey[c] - ey[p], sE[c]);
  }
  for (int64_t i = 0; i < n_nodes; i++)
    for (int32_t b = d->S_rowptr[i]; b < d->S_rowptr[i + 1]; b++) {
      R.oS[b] = block_offset(ey[i] - ex[d->S_colidx[b]], sS[b]);
      if (needs_safe_split(sS[b], R.oS[b])) R.s_tiny = true;
    }
  for (int64_t b = 0; b < nD; b++) {
    R.oD[b] = block_offset(R.eY[drow[b]], sD[b]);
    R.d_safe[b] = needs_safe_split(sD[b], R.oD[b]);
  }
  (void)q;
  return R;
}

// every (row leaf, column leaf) pair covered exactly once by a dense block or
// by a coupling block of an ancestor pair
h2_status check_cover(const h2_desc* d, int64_t leaves) {
  const int q = d->depth;
  std::vector<std::pair<int64_t, int64_t>> iv;
  for (int64_t i = 0; i < leaves; i++) {
    iv.clear();
    for (int32_t b = d->D_rowptr[i]; b < d->D_rowptr[i + 1]; b++) iv.push_back({d->D_colidx[b], d->D_colidx[b] + 1});
    int64_t node = leaves - 1 + i;
    for (int l = q;; l--) {
      for (int32_t b = d->S_rowptr[node]; b < d->S_rowptr[node + 1]; b++) {
        const int64_t col = d->S_colidx[b];
        const int64_t first = ((int64_t)1 << l) - 1, span = (int64_t)1 << (q - l);
        const int64_t lo = (col - first) * span;
        iv.push_back({lo, lo + span});
      }
      if (node == 0) break;
      node = (node - 1) / 2;
    }
    std::sort(iv.begin(), iv.end());
    int64_t at = 0;
    for (auto& r : iv) {
      if (r.first != at)
        return fail(H2_ERR_INVALID, "block cover: leaf row %lld, columns from leaf %lld %s", (long long)i,
                    (long long)std::min(at, r.first), r.first > at ? "are not covered" : "are covered twice");
      at = r.second;
    }
    if (at != leaves)
      return fail(H2_ERR_INVALID, "block cover: leaf row %lld, columns from leaf %lld are not covered", (long long)i,
                  (long long)at);
  }
  return H2_OK;
}

// s_values / d_values: the coupling / dense values are part of the description (not evaluated
// from a kernel)
h2_status validate(const h2_desc* d, bool s_values, bool d_values, int64_t* nS, int64_t* nD, int64_t* nDval,
                   int* m_max) {
  if (!d) return fail(H2_ERR_INVALID, "desc is NULL");
  if (d->n < 1) return fail(H2_ERR_INVALID, "n = %lld < 1", (long long)d->n);
  if (d->n >= ((int64_t)1 << 31)) return fail(H2_ERR_UNSUPPORTED, "n = %lld >= 2^31", (long long)d->n);
  if (d->depth < 0 || d->depth > 24) return fail(H2_ERR_INVALID, "depth = %d outside 0..24", d->depth);
  if (d->rank < 1) return fail(H2_ERR_INVALID, "rank = %d < 1", d->rank);
  if (d->rank > kMaxRank) return fail(H2_ERR_UNSUPPORTED, "rank = %d > %d", d->rank, kMaxRank);
  if (d->storage != H2_FP64 && d->storage != H2_FP16_SCALED && d->storage != H2_BF16_SCALED &&
      d->storage != H2_INT16_SCALED)
    return fail(H2_ERR_UNSUPPORTED, "storage %d not supported", d->storage);
  if (!d->leaf_offset || !d->U || !d->E || !d->S_rowptr || !d->D_rowptr) return fail(H2_ERR_INVALID, "NULL array in desc");
  if (!d->symmetric && (!d->V || !d->F)) return fail(H2_ERR_INVALID, "V/F are NULL but symmetric = 0");
  const int q = d->depth, k = d->rank;
  const int64_t leaves = (int64_t)1 << q, n_nodes = ((int64_t)2 << q) - 1;
  if (d->leaf_offset[0] != 0 || d->leaf_offset[leaves] != d->n) return fail(H2_ERR_INVALID, "leaf_offset must run from 0 to n");
  int mm = 0;
  for (int64_t i = 0; i < leaves; i++) {
    const int64_t s = d->leaf_offset[i + 1] - d->leaf_offset[i];
    if (s < 1) return fail(H2_ERR_INVALID, "leaf %lld has size %lld < 1", (long long)i, (long long)s);
    if (s > kMaxLeaf) return fail(H2_ERR_UNSUPPORTED, "leaf %lld has size %lld > %d", (long long)i, (long long)s, kMaxLeaf);
    mm = std::max(mm, (int)s);
  }
  *m_max = mm;
  if (d->S_rowptr[0] != 0) return fail(H2_ERR_INVALID, "S_rowptr[0] != 0");
  for (int64_t r = 0; r < n_nodes; r++)
    if (d->S_rowptr[r + 1] < d->S_rowptr[r]) return fail(H2_ERR_INVALID, "S_rowptr decreases at row %lld", (long long)r);
  *nS = d->S_rowptr[n_nodes];
  if (*nS > 0 && (!d->S_colidx || (s_values && !d->S_val)))
    return fail(H2_ERR_INVALID, "S_colidx/S_val NULL with %lld blocks", (long long)*nS);
  for (int64_t r = 0; r < n_nodes; r++) {
    const int l = level_of(r);
    const int64_t first = ((int64_t)1 << l) - 1, last = ((int64_t)2 << l) - 2;
    for (int32_t b = d->S_rowptr[r]; b < d->S_rowptr[r + 1]; b++)
      if (d->S_colidx[b] < first || d->S_colidx[b] > last)
        return fail(H2_ERR_INVALID, "S_colidx[%d] = %d is not on the level of row %lld", b, d->S_colidx[b], (long long)r);
  }
  if (d->D_rowptr[0] != 0) return fail(H2_ERR_INVALID, "D_rowptr[0] != 0");
  for (int64_t r = 0; r < leaves; r++)
    if (d->D_rowptr[r + 1] < d->D_rowptr[r]) return fail(H2_ERR_INVALID, "D_rowptr decreases at row %lld", (long long)r);
  *nD = d->D_rowptr[leaves];
  if (*nD > 0 && (!d->D_colidx || (d_values && !d->D_val)))
    return fail(H2_ERR_INVALID, "D_colidx/D_val NULL with %lld blocks", (long long)*nD);
  int64_t dv = 0;
  for (int64_t r = 0; r < leaves; r++)
    for (int32_t b = d->D_rowptr[r]; b < d->D_rowptr[r + 1]; b++) {
      const int32_t j = d->D_colidx[b];
      if (j < 0 || j >= leaves) return fail(H2_ERR_INVALID, "D_colidx[%d] = %d out of range", b, j);
      dv += (d->leaf_offset[r + 1] - d->leaf_offset[r]) * (d->leaf_offset[j + 1] - d->leaf_offset[j]);
    }
  *nDval = dv;
  int64_t bad = 0;
  const bool f32 = d->storage != H2_FP64;  // FP64: any finite value; scaled forms: |v| < 2^126
  if (!values_ok(d->U, d->n * k, &bad, f32)) return fail(H2_ERR_INVALID, "U[%lld] is not finite or too large", (long long)bad);
  if (!values_ok(d->E, (n_nodes - 1) * k * k, &bad, f32))
    return fail(H2_ERR_INVALID, "E[%lld] is not finite or too large", (long long)bad);
  if (!d->symmetric) {
    if (!values_ok(d->V, d->n * k, &bad, f32)) return fail(H2_ERR_INVALID, "V[%lld] is not finite or too large", (long long)bad);
    if (!values_ok(d->F, (n_nodes - 1) * k * k, &bad, f32))
      return fail(H2_ERR_INVALID, "F[%lld] is not finite or too large", (long long)bad);
  }
  if (s_values && *nS && !values_ok(d->S_val, *nS * k * k, &bad, f32))
    return fail(H2_ERR_INVALID, "S_val[%lld] is not finite or too large", (long long)bad);
  if (d_values && *nD && !values_ok(d->D_val, dv, &bad, f32))
    return fail(H2_ERR_INVALID, "D_val[%lld] is not finite or too large", (long long)bad);
  if (d->check_cover) return check_cover(d, leaves);
  return H2_OK;
}

int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// transpose a rows x cols column-major block into dst (cols x rows column-major)
void transpose_block(const double* src, double* dst, int64_t rows, int64_t cols) {
  for (int64_t c = 0; c < cols; c++)
    for (int64_t r = 0; r < rows; r++) dst[c + cols * r] = src[r + rows * c];
}

}  // namespace

namespace h2i {

h2_status validate_desc(const h2_desc* d, bool s_values, bool d_values, int64_t* nS, int64_t* nD, int64_t* nDval,
                        int* m_max) {
  return validate(d, s_values, d_values, nS, nD, nDval, m_max);
}

// Split rows (row r weighs row_bytes[r] and starts at item row_item0[r]) into
// `grid` contiguous ranges of about equal weight; returns each range's first item.
std::vector<int> balance(const std::vector<int64_t>& row_bytes, const std::vector<int64_t>& row_item0, int grid) {
  const int64_t rows = (int64_t)row_bytes.size();
  int64_t total = 0;
  for (int64_t b : row_bytes) total += b;
  std::vector<int> begin((size_t)grid + 1, 0);
  int64_t acc = 0, r = 0;
  for (int c = 0; c < grid; c++) {
    begin[c] = (int)row_item0[r];
    const int64_t target = (total * (c + 1)) / grid;
    while (r < rows && acc + row_bytes[r] / 2 < target) acc += row_bytes[r++];
  }
  begin[grid] = (int)row_item0[rows];
  for (int c = 1; c <= grid; c++) begin[c] = std::max(begin[c], begin[c - 1]);
  return begin;
}

}  // namespace h2i

namespace {

// Every copy a streaming kernel will issue must stay inside its source buffer and
// its stage slot and be 16-byte aligned; checked once on the host so that a
// layout bug is an error here, never an out-of-bounds bulk copy on the device.
//   mat_bytes   size of the matrix buffer the items index
//   v0, v1      float2 counts per vector slot of the two vector sources
h2_status audit_items(const std::vector<h2::StreamItem>& items, const std::vector<int>& begin, int64_t mat_bytes,
                      int64_t v0, int64_t v1) {
  for (size_t c = 0; c + 1 < begin.size(); c++)
    if (begin[c] > begin[c + 1]) return fail(H2_ERR_INVALID, "internal: item ranges not monotone");
  if (begin.front() != 0 || begin.back() != (int)items.size()) return fail(H2_ERR_INVALID, "internal: item ranges do not cover the list");
  for (size_t i = 0; i < items.size(); i++) {
    const h2::StreamItem& it = items[i];
    const int64_t R = it.shape & 0xFF, C = (it.shape >> 8) & 0xFF, vs = (it.shape >> 16) & 0xFF, nb = (it.shape >> 24) & 0xFF;
    // vector chunk: nv * vs float2 at v_off * nv, nv <= kPassVectors; stage slot: 512 * NVB bytes >= 64 * nv * 8
    const int64_t lim = (it.flags & h2::kItemFlagSrc1) ? v1 : v0;
    const bool ok = it.m_off >= 0 && it.m_off % 16 == 0 && it.m_bytes >= 16 && it.m_bytes % 16 == 0 &&
                    it.m_bytes <= h2::kStageMat && it.m_off + it.m_bytes <= mat_bytes && R >= 1 && R <= 64 && C >= 1 &&
                    C <= 64 && vs >= C && vs <= 64 && vs % 2 == 0 && nb == 1 && it.v_off >= 0 && it.v_off % 2 == 0 &&
                    it.v_off + vs <= lim && it.m_bytes == (int64_t)(R * C + ((R * C) & 1)) * 8;
    if (!ok) return fail(H2_ERR_INVALID, "internal: work item %lld fails the layout audit", (long long)i);
  }
  return H2_OK;
}

h2_status upload_items(h2_matrix_s* h, ItemList* L, const std::vector<h2::StreamItem>& items, const std::vector<int>& begin) {
  h2_status st = upload(h, &L->items, items.data(), (int64_t)items.size());
  if (st != H2_OK) return st;
  st = upload(h, &L->cta_begin, begin.data(), (int64_t)begin.size());
  L->count = (int64_t)items.size();
  return st;
}

// ------------------------------------------------------------------ launch sequence
}  // namespace

namespace h2i {

// record a phase-boundary event when profiling (events are pooled per handle)
cudaError_t mark(Profiler* p, cudaStream_t st) {
  if (!p->on) return cudaSuccess;
  if (p->used == p->events.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    p->events.push_back(e);
  }
  return cudaEventRecord(p->events[p->used++], st);
}

h2_status profile_read(Profiler* p, double ms[H2_NPHASES], int64_t* launches) {
  for (int i = 0; i < H2_NPHASES; i++) ms[i] = 0.0;
  const size_t per = H2_NPHASES + 1;
  if (p->used) CUDA_TRY(cudaEventSynchronize(p->events[p->used - 1]));
  for (size_t base = 0; base + per <= p->used; base += per)
    for (int i = 0; i < H2_NPHASES; i++) {
      float t = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&t, p->events[base + i], p->events[base + i + 1]));
      ms[i] += t;
    }
  if (launches) *launches = p->launches;
  p->used = 0;
  p->launches = 0;
  return H2_OK;
}

void profile_free(Profiler* p) {
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  p->events.clear();
  p->used = 0;
}

}  // namespace h2i

namespace {

template <int NVB>
cudaError_t set_stream_smem() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaErrorNotReady) {
    constexpr int CW = h2::dense_consumer_warps(NVB);
    done = cudaFuncSetAttribute(h2::k_dense_stream<NVB, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                h2::stream_smem_bytes(NVB, CW));
  }
  return done;
}

template <int RPL_K, int NVB>
h2_status run_pass(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  using namespace h2;
  const int k = h->k, kp = h->kp, LR = h->lr;
  const unsigned wb = (unsigned)kWarps * 32;
  auto grid = [](int64_t items) { return (unsigned)((items + kWarps - 1) / kWarps); };
  cudaError_t e = set_stream_smem<NVB>();
  if (e != cudaSuccess) return fail(H2_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  constexpr int CW = dense_consumer_warps(NVB);
  constexpr int smem = stream_smem_bytes(NVB, CW);
  const int kkp = (int)even((int64_t)k * k);
  TreeParams T{};
  T.Vt = h->Vt;
  T.Ft = h->Ft;
  T.E = h->E;
  T.leaf_off = h->leaf_off;
  T.xp_off = h->xp_off;
  T.x = x;
  T.ldx = ldx;
  T.x2 = h->x2;
  T.xhat = h->xhat;
  T.yhat = h->yhat;
  T.ticket = h->ticket;
  T.oV = h->oV;
  T.oF = h->oF;
  T.oE = h->oE;
  T.vexp = h->vexp;
  T.k = k;
  T.kp = kp;
  T.LR = LR;
  T.q = h->q;
  T.L = h->tree_L;
  T.nv = nv;
  const unsigned tree_grid = 1u << h->tree_L, tree_threads = kTreeWarps * 32;
  cudaError_t me = mark(&h->prof, st);
  k_vec_scale<<<kScaleBlocks, kScaleThreads, 0, st>>>(x, ldx, h->n, nv, h->vpart, h->vticket, h->vexp);
  k_upsweep_tree<RPL_K, NVB><<<tree_grid, tree_threads, 0, st>>>(T);
  if (me == cudaSuccess) me = mark(&h->prof, st);
  if (h->pair_rows) {
    constexpr int CB = NVB <= 2 ? 4 : (NVB <= 4 ? 2 : 1);
    if (h->s_tiny)
      k_coupling<NVB, CB, true><<<grid(h->n_nodes), wb, 0, st>>>(h->smat, kkp, h->Srow, h->Sco, k, kp, h->n_nodes, nv,
                                                                  h->xhat, h->yhat);
    else
      k_coupling<NVB, CB, false><<<grid(h->n_nodes), wb, 0, st>>>(h->smat, kkp, h->Srow, h->Sco, k, kp, h->n_nodes, nv,
                                                                   h->xhat, h->yhat);
  } else {
    k_coupling_generic<RPL_K, NVB><<<grid(h->n_nodes), wb, 0, st>>>(h->smat, kkp, h->Srow, h->Sco, k, kp, LR, h->n_nodes,
                                                                     nv, h->xhat, h->yhat);
  }
  if (me == cudaSuccess) me = mark(&h->prof, st);
  k_downsweep_tree<RPL_K, NVB><<<tree_grid, tree_threads, 0, st>>>(T);
  if (me == cudaSuccess) me = mark(&h->prof, st);
  StreamParams P{};
  P.items = h->dense_items.items;
  P.cta_begin = h->dense_items.cta_begin;
  P.mat = h->dmat;
  P.vsrc0 = h->x2;
  P.vsrc1 = h->yhat;
  P.nv = nv;
  P.y = y;
  P.ldy = ldy;
  P.vexp = h->vexp;
  P.err = h->err;
  P.budget = h->budget;
  P.inject = h->inject;
  k_dense_stream<NVB, CW><<<h->grid, (CW + 1) * 32, smem, st>>>(P);
  if (h->inject >= 0) {  // the test hook applies to one product only
    h->inject = -1;
    h->budget = kWaitBudget;
  }
  if (me == cudaSuccess) me = mark(&h->prof, st);
  h->prof.launches += 5;
  if (me != cudaSuccess) return fail(H2_ERR_CUDA, "profiling event: %s", cudaGetErrorString(me));
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(H2_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return H2_OK;
}

template <int RPL_K>
h2_status run_pass_nv(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  if (nv <= 1) return run_pass<RPL_K, 1>(h, nv, x, ldx, y, ldy, st);
  if (nv <= 2) return run_pass<RPL_K, 2>(h, nv, x, ldx, y, ldy, st);
  if (nv <= 4) return run_pass<RPL_K, 4>(h, nv, x, ldx, y, ldy, st);
  if (nv <= 8) return run_pass<RPL_K, 8>(h, nv, x, ldx, y, ldy, st);
  return run_pass<RPL_K, 16>(h, nv, x, ldx, y, ldy, st);
}

h2_status matvec_device(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  for (int v0 = 0; v0 < nv; v0 += kPassVectors) {
    const int nvp = std::min(kPassVectors, nv - v0);
    const double* xp = x + (int64_t)v0 * ldx;
    double* yp = y + (int64_t)v0 * ldy;
    h2_status s = (h->storage != H2_FP64) ? mixed_pass(h, nvp, xp, ldx, yp, ldy, st)
                  : (h->k > 32)             ? run_pass_nv<2>(h, nvp, xp, ldx, yp, ldy, st)
                                            : run_pass_nv<1>(h, nvp, xp, ldx, yp, ldy, st);
    if (s != H2_OK) return s;
  }
  return H2_OK;
}

// ------------------------------------------------------------------ device layout
h2_status build_device(h2_matrix_s* h, const h2_desc* d) {
  const int k = h->k;
  const int64_t kk = (int64_t)k * k, kkp = even(kk);
  const double* V = d->symmetric ? d->U : d->V;
  const double* F = d->symmetric ? d->E : d->F;
  const int64_t* lo = d->leaf_offset;
  h2_status st;
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&h->grid, cudaDevAttrMultiProcessorCount, dev));

  if ((st = upload(h, &h->leaf_off, lo, h->leaves + 1)) != H2_OK) return st;
  if ((st = upload(h, &h->Srow, d->S_rowptr, h->n_nodes + 1)) != H2_OK) return st;
  if ((st = upload(h, &h->Scol, d->S_colidx, h->nS)) != H2_OK) return st;
  if ((st = dalloc(h, &h->err, 1)) != H2_OK) return st;
  CUDA_TRY(cudaMemset(h->err, 0, sizeof(int)));
  if ((st = dalloc(h, &h->ticket, h->n_nodes)) != H2_OK) return st;
  CUDA_TRY(cudaMemset(h->ticket, 0, (size_t)h->n_nodes * sizeof(int)));
  // subtree roots of the fused tree kernels: at least two CTAs per SM when the tree is deep enough
  int lmax = 0;
  while (((int64_t)1 << lmax) < 2 * (int64_t)h->grid) lmax++;
  h->tree_L = std::min(h->q, lmax);
  if (h->storage != H2_FP64) return mixed_build(h, d);

  // padded leaf offsets of the split x
  std::vector<int64_t> xp((size_t)h->leaves + 1, 0);
  for (int64_t j = 0; j < h->leaves; j++) xp[j + 1] = xp[j] + even(lo[j + 1] - lo[j]);
  if ((st = upload(h, &h->xp_off, xp.data(), h->leaves + 1)) != H2_OK) return st;

  {  // leaf bases V^T (projection), transfers F^T (upsweep), E (downsweep)
    std::vector<double> tmp((size_t)std::max<int64_t>(h->n * k, (h->n_nodes - 1) * kk));
    for (int64_t j = 0; j < h->leaves; j++) transpose_block(V + lo[j] * k, tmp.data() + lo[j] * k, lo[j + 1] - lo[j], k);
    if ((st = upload(h, &h->Vt, (const double*)tmp.data(), h->n * k)) != H2_OK) return st;
    for (int64_t c = 0; c < h->n_nodes - 1; c++) transpose_block(F + c * kk, tmp.data() + c * kk, k, k);
    if ((st = upload(h, &h->Ft, (const double*)tmp.data(), (h->n_nodes - 1) * kk)) != H2_OK) return st;
    if ((st = upload(h, &h->E, d->E, (h->n_nodes - 1) * kk)) != H2_OK) return st;
  }

  Fp64Ranges R;
  {  // dense blocks + U, each padded to an even count of doubles, and their item list
    std::vector<int64_t> doff((size_t)h->nD + 1, 0), dpo((size_t)h->nD + 1, 0), upo((size_t)h->leaves + 1, 0);
    for (int64_t r = 0, b = 0; r < h->leaves; r++)
      for (; b < d->D_rowptr[r + 1]; b++) {
        const int64_t sz = (lo[r + 1] - lo[r]) * (lo[d->D_colidx[b] + 1] - lo[d->D_colidx[b]]);
        doff[b + 1] = doff[b] + sz;
        dpo[b + 1] = dpo[b] + even(sz);
      }
    for (int64_t i = 0; i < h->leaves; i++) upo[i + 1] = upo[i] + even((lo[i + 1] - lo[i]) * k);
    const int64_t dtot = dpo[h->nD], total = dtot + upo[h->leaves];
    R = fp64_ranges(d, h->leaves, h->n_nodes, h->nS, h->nD, doff);
    for (const std::vector<int32_t>* v : {&R.oV, &R.oF, &R.oE, &R.oS, &R.oD, &R.oU, &R.eY})
      for (int32_t e : *v)
        if (e < -h2::kItemExpMax || e > h2::kItemExpMax) return fail(H2_ERR_INVALID, "internal: exponent offset %d out of range", e);
    double* dm = nullptr;
    if ((st = dalloc(h, &dm, total)) != H2_OK) return st;
    h->dmat = (char*)dm;
    // copy through a host staging buffer, inserting the padding
    const int64_t chunk = (int64_t)1 << 24;
    std::vector<double> stage((size_t)chunk);
    int64_t fill = 0, dst0 = 0;
    auto flush = [&]() -> h2_status {
      if (fill) CUDA_TRY(cudaMemcpy(dm + dst0, stage.data(), (size_t)fill * 8, cudaMemcpyHostToDevice));
      dst0 += fill;
      fill = 0;
      return H2_OK;
    };
    auto put = [&](const double* src, int64_t cnt, int64_t padded) -> h2_status {
      if (fill + padded > chunk) {
        h2_status s2 = flush();
        if (s2 != H2_OK) return s2;
      }
      std::memcpy(stage.data() + fill, src, (size_t)cnt * 8);
      if (padded > cnt) stage[fill + cnt] = 0.0;
      fill += padded;
      return H2_OK;
    };
    for (int64_t b = 0; b < h->nD; b++)
      if ((st = put(d->D_val + doff[b], doff[b + 1] - doff[b], dpo[b + 1] - dpo[b])) != H2_OK) return st;
    for (int64_t i = 0; i < h->leaves; i++)
      if ((st = put(d->U + lo[i] * k, (lo[i + 1] - lo[i]) * k, upo[i + 1] - upo[i])) != H2_OK) return st;
    if ((st = flush()) != H2_OK) return st;

    std::vector<h2::StreamItem> items;
    items.reserve((size_t)(h->nD + h->leaves));
    std::vector<int64_t> row_bytes((size_t)h->leaves), row_item0((size_t)h->leaves + 1);
    for (int64_t i = 0; i < h->leaves; i++) {
      row_item0[i] = (int64_t)items.size();
      const int si = (int)(lo[i + 1] - lo[i]);
      int64_t bytes = 0;
      for (int32_t b = d->D_rowptr[i]; b < d->D_rowptr[i + 1]; b++) {
        const int j = d->D_colidx[b];
        const int sj = (int)(lo[j + 1] - lo[j]);
        h2::StreamItem it{};
        it.m_off = dpo[b] * 8;
        it.m_bytes = (int)((dpo[b + 1] - dpo[b]) * 8);
        it.shape = (unsigned)si | ((unsigned)sj << 8) | ((unsigned)even(sj) << 16) | (1u << 24);
        it.v_off = xp[j];
        it.row = (int)lo[i];
        it.flags = (R.d_safe[b] ? h2::kItemFlagSafe : 0) | h2::item_pack_exp(R.oD[b], 0);
        items.push_back(it);
        bytes += it.m_bytes + 8 * sj;
      }
      h2::StreamItem it{};
      it.m_off = (dtot + upo[i]) * 8;
      it.m_bytes = (int)((upo[i + 1] - upo[i]) * 8);
      it.shape = (unsigned)si | ((unsigned)k << 8) | ((unsigned)h->kp << 16) | (1u << 24);
      it.v_off = (h->leaf0 + i) * h->kp;
      it.row = (int)lo[i];
      it.flags = h2::kItemFlagLast | h2::kItemFlagSrc1 | h2::kItemFlagSafe | h2::item_pack_exp(R.oU[i], R.eY[i]);
      items.push_back(it);
      row_bytes[i] = bytes + it.m_bytes + 8 * h->kp + 16 * si;
    }
    row_item0[h->leaves] = (int64_t)items.size();
    const std::vector<int> begin = balance(row_bytes, row_item0, h->grid);
    // vector sources per slot: split x (padded leaf layout) and yhat (n_nodes x kp)
    if ((st = audit_items(items, begin, total * 8, xp[h->leaves], h->n_nodes * h->kp)) != H2_OK) return st;
    if ((st = upload_items(h, &h->dense_items, items, begin)) != H2_OK) return st;
  }

  {  // coupling blocks, each padded to an even count of doubles
    double* sm = nullptr;
    if ((st = dalloc(h, &sm, h->nS * kkp)) != H2_OK) return st;
    h->smat = sm;
    if (h->nS > 0) {
      if (kkp == kk) {
        CUDA_TRY(cudaMemcpy(sm, d->S_val, (size_t)(h->nS * kk) * 8, cudaMemcpyHostToDevice));
      } else {
        CUDA_TRY(cudaMemset(sm, 0, (size_t)(h->nS * kkp) * 8));
        CUDA_TRY(cudaMemcpy2D(sm, (size_t)kkp * 8, d->S_val, (size_t)kk * 8, (size_t)kk * 8, (size_t)h->nS,
                              cudaMemcpyHostToDevice));
      }
    }
    h->pair_rows = k >= 2 && k <= 64 && (k & (k - 1)) == 0;
    h->s_tiny = R.s_tiny;
  }
  if ((st = upload(h, &h->oV, R.oV.data(), h->leaves)) != H2_OK) return st;
  if ((st = upload(h, &h->oF, R.oF.data(), h->n_nodes)) != H2_OK) return st;
  if ((st = upload(h, &h->oE, R.oE.data(), h->n_nodes)) != H2_OK) return st;
  {
    std::vector<int2> sco((size_t)h->nS);
    for (int64_t b = 0; b < h->nS; b++) sco[b] = make_int2(d->S_colidx[b], R.oS[b]);
    if ((st = upload(h, &h->Sco, (const int2*)sco.data(), h->nS)) != H2_OK) return st;
  }
  if ((st = dalloc(h, &h->vexp, h2i::kPassVectors)) != H2_OK) return st;
  if ((st = dalloc(h, &h->vpart, (int64_t)h2::kScaleBlocks * 16)) != H2_OK) return st;
  if ((st = dalloc(h, &h->vticket, 1)) != H2_OK) return st;
  CUDA_TRY(cudaMemset(h->vticket, 0, sizeof(unsigned)));

  if ((st = dalloc(h, &h->x2, xp[h->leaves] * kPassVectors)) != H2_OK) return st;
  if ((st = dalloc(h, &h->xhat, h->n_nodes * kPassVectors * h->kp)) != H2_OK) return st;
  if ((st = dalloc(h, &h->yhat, h->n_nodes * kPassVectors * h->kp)) != H2_OK) return st;
  return H2_OK;
}

}  // namespace

// h2_create, or h2_create_kernel_coupling with kc (already checked): the coupling phase then
// evaluates the blocks from the kernel and stores none; with gen_points (h2_create_generated,
// already checked) the dense blocks are generated on the device from the points
h2_status create_handle(const h2_desc* d, const h2_coupling_kernel* kc, h2_handle* out,
                        const double* gen_points = nullptr) {
  if (!kc) g_err.clear();
  if (!out) return fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int64_t nS = 0, nD = 0, nDval = 0;
  int m_max = 0;
  h2_status st = validate(d, kc == nullptr, gen_points == nullptr, &nS, &nD, &nDval, &m_max);
  if (st != H2_OK) return st;
  h2_matrix_s* h = new (std::nothrow) h2_matrix_s();
  if (!h) return fail(H2_ERR_OOM, "host allocation failed");
  h->n = d->n;
  h->q = d->depth;
  h->k = d->rank;
  h->kp = (int)even(h->k);
  h->leaves = (int64_t)1 << h->q;
  h->n_nodes = ((int64_t)2 << h->q) - 1;
  h->leaf0 = h->leaves - 1;
  h->nS = nS;
  h->nD = nD;
  h->nDval = nDval;
  h->m_max = m_max;
  h->lr = h->k > 32 ? 32 : pow2ceil(h->k);
  h->storage = d->storage;
  h->kc = kc;
  h->gen_points = gen_points;
  h->kf = kc != nullptr;
  if (kc) {
    h->kf_kind = kc->kernel;
    h->kf_inv_ell = (float)(1.0 / kc->ell);
  }
  try {
    st = build_device(h, d);
  } catch (const std::bad_alloc&) {
    st = fail(H2_ERR_OOM, "host allocation failed");
  }
  h->kc = nullptr;  // the caller's description is not kept
  h->gen_points = nullptr;
  if (st != H2_OK) {
    free_all(h);
    delete h;
    return st;
  }
  const int64_t kk = (int64_t)h->k * h->k, sS = h->kf ? 0 : nS;  // coupling blocks stored
  const int64_t entries = 2 * h->n * h->k + 2 * (h->n_nodes - 1) * kk + sS * kk + nDval;
  if (h->storage == H2_FP64)
    h->paper_bytes = 8 * entries;
  else  // 16-bit codes plus one FP32 scale per block of U, V, E, F, S and D
    h->paper_bytes = d->bases_fp32 ? 2 * (sS * kk + nDval) + 4 * (sS + nD) + 4 * (2 * h->n * h->k + 2 * (h->n_nodes - 1) * kk)
                                   : 2 * entries + 4 * (2 * h->leaves + 2 * (h->n_nodes - 1) + sS + nD);
  *out = h;
  return H2_OK;
}

extern "C" {

const char* h2_last_error(void) { return g_err.c_str(); }

h2_status h2_create(const h2_desc* d, h2_handle* out) { return create_handle(d, nullptr, out); }

// checks of h2_create_kernel_coupling's kernel description; H2_OK or the failure
static h2_status check_kernel_desc(const h2_desc* d, const h2_coupling_kernel* kc) {
  if (!d || !kc || !kc->cheb) return fail(H2_ERR_INVALID, "desc, kernel description or cheb is NULL");
  if (kc->kernel != H2_KERNEL_EXP && kc->kernel != H2_KERNEL_MATERN32)
    return fail(H2_ERR_INVALID, "kernel = %d is not an h2_kernel_kind", kc->kernel);
  if (!(kc->ell > 0.0) || !std::isfinite(kc->ell) || (float)(1.0 / kc->ell) > 3.0e38f)
    return fail(H2_ERR_INVALID, "ell = %g is not a finite positive length", kc->ell);
  if (kc->dim < 1 || kc->dim > 3 || kc->p < 1 || kc->p > 16)
    return fail(H2_ERR_INVALID, "dim = %d, p = %d outside 1..3, 1..16", kc->dim, kc->p);
  int64_t kpow = 1;
  for (int e = 0; e < kc->dim; e++) kpow *= kc->p;
  if (kpow != d->rank) return fail(H2_ERR_INVALID, "p^dim = %lld differs from the rank %d", (long long)kpow, d->rank);
  if (d->storage == H2_FP64)
    return fail(H2_ERR_UNSUPPORTED, "coupling blocks from the kernel need a scaled storage form (FP32 arithmetic)");
  if (d->depth < 0 || d->depth > 24) return fail(H2_ERR_INVALID, "depth = %d outside 0..24", d->depth);
  const int64_t n_nodes = ((int64_t)2 << d->depth) - 1;
  int64_t bad = 0;
  if (!values_ok(kc->cheb, n_nodes * kc->dim * kc->p, &bad))
    return fail(H2_ERR_INVALID, "cheb[%lld] is not finite or too large", (long long)bad);
  return H2_OK;
}

h2_status h2_create_kernel_coupling(const h2_desc* d, const h2_coupling_kernel* kc, h2_handle* out) {
  g_err.clear();
  if (!out) return fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  const h2_status st = check_kernel_desc(d, kc);
  if (st != H2_OK) return st;
  return create_handle(d, kc, out);
}

h2_status h2_create_generated(const h2_desc* d, const h2_coupling_kernel* kc, const double* points, h2_handle* out) {
  g_err.clear();
  if (!out) return fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  h2_status st = check_kernel_desc(d, kc);
  if (st != H2_OK) return st;
  int64_t bad = 0;
  if (!points) return fail(H2_ERR_INVALID, "points is NULL");
  if (!values_ok(points, d->n * kc->dim, &bad, false)) return fail(H2_ERR_INVALID, "points[%lld] is not finite", (long long)bad);
  return create_handle(d, kc, out, points);
}

h2_status h2_matvec(h2_handle h, int32_t nv, const double* x, int64_t ldx, double* y, int64_t ldy, void* stream) {
  if (!h || !x || !y) return fail(H2_ERR_INVALID, "NULL handle or vector");
  if (nv < 1) return fail(H2_ERR_INVALID, "nv = %d < 1", nv);
  if (ldx < h->n || ldy < h->n) return fail(H2_ERR_INVALID, "leading dimension below n");
  return matvec_device(h, nv, x, ldx, y, ldy, (cudaStream_t)stream);
}

h2_status h2_matvec_f32(h2_handle h, int32_t nv, const float* x, int64_t ldx, float* y, int64_t ldy, void* stream) {
  if (!h || !x || !y) return fail(H2_ERR_INVALID, "NULL handle or vector");
  if (nv < 1) return fail(H2_ERR_INVALID, "nv = %d < 1", nv);
  if (ldx < h->n || ldy < h->n) return fail(H2_ERR_INVALID, "leading dimension below n");
  if (h->storage == H2_FP64) return fail(H2_ERR_UNSUPPORTED, "FP32 vectors need a scaled storage form");
  cudaStream_t st = (cudaStream_t)stream;
  for (int v0 = 0; v0 < nv; v0 += kPassVectors) {
    const int nvp = std::min(kPassVectors, nv - v0);
    h2_status s = mixed_pass(h, nvp, x + (int64_t)v0 * ldx, ldx, y + (int64_t)v0 * ldy, ldy, st, 1);
    if (s != H2_OK) return s;
  }
  return H2_OK;
}

h2_status h2_matvec_host(h2_handle h, int32_t nv, const double* x, int64_t ldx, double* y, int64_t ldy, void* stream) {
  if (!h || !x || !y) return fail(H2_ERR_INVALID, "NULL handle or vector");
  if (nv < 1) return fail(H2_ERR_INVALID, "nv = %d < 1", nv);
  if (ldx < h->n || ldy < h->n) return fail(H2_ERR_INVALID, "leading dimension below n");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t need = h->n * nv;
  if (need > h->host_cap) {
    CUDA_TRY(cudaStreamSynchronize(st));
    if (h->hx) cudaFree(h->hx);
    if (h->hy) cudaFree(h->hy);
    h->hx = h->hy = nullptr;
    h->host_cap = 0;
    CUDA_TRY(cudaMalloc(&h->hx, (size_t)need * sizeof(double)));
    CUDA_TRY(cudaMalloc(&h->hy, (size_t)need * sizeof(double)));
    h->host_cap = need;
  }
  CUDA_TRY(cudaMemcpy2DAsync(h->hx, (size_t)h->n * 8, x, (size_t)ldx * 8, (size_t)h->n * 8, (size_t)nv,
                             cudaMemcpyHostToDevice, st));
  h2_status s = matvec_device(h, nv, h->hx, h->n, h->hy, h->n, st);
  if (s != H2_OK) return s;
  CUDA_TRY(cudaMemcpy2DAsync(y, (size_t)ldy * 8, h->hy, (size_t)h->n * 8, (size_t)h->n * 8, (size_t)nv,
                             cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return H2_OK;
}

h2_status h2_tune(h2_handle h, int32_t nv, const double* x, int64_t ldx, double* y, int64_t ldy, void* stream,
                  int32_t chosen[3]) {
  if (!h || !x || !y || !chosen) return fail(H2_ERR_INVALID, "NULL handle, vector or output");
  if (nv < 1) return fail(H2_ERR_INVALID, "nv = %d < 1", nv);
  if (ldx < h->n || ldy < h->n) return fail(H2_ERR_INVALID, "leading dimension below n");
  chosen[0] = chosen[1] = chosen[2] = 0;
  if (h->storage == H2_FP64) return H2_OK;  // the plain form has no launch options
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  // 16 dense consumer warps exist for passes of at most 8 vectors
  const int ncw = 2;  // 8 or 16 dense consumer warps
  float best = 3.4e38f;
  int best_opt = kDefaultChunkOpt, best_cw = h->mx.launch.cw, best_tree = 0;
  h2_status s = H2_OK;
  const int ntree = std::min(3, h->tree_L + 1);  // subtree level: default, one or two levels higher
  for (int c = 0; c < ncw && s == H2_OK; c++)
    for (int opt = 0; opt < 3 && s == H2_OK; opt++)
      for (int tr = 0; tr < ntree && s == H2_OK; tr++) {
      const int cw = c ? 2 * kDenseCW : kDenseCW;
      if ((s = mixed_configure(h, opt, cw, tr)) != H2_OK) break;
      if ((s = matvec_device(h, nv, x, ldx, y, ldy, st)) != H2_OK) break;  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && s == H2_OK; r++) s = matvec_device(h, nv, x, ldx, y, ldy, st);
      cudaEventRecord(e1, st);
      cudaError_t ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) {
        s = fail(H2_ERR_CUDA, "timing a launch configuration: %s", cudaGetErrorString(ce));
        break;
      }
      if (ms < best) {
        best = ms;
        best_opt = opt;
        best_cw = cw;
        best_tree = tr;
      }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != H2_OK) return s;
  if ((s = mixed_configure(h, best_opt, best_cw, best_tree)) != H2_OK) return s;
  chosen[0] = best_cw;
  chosen[1] = kChunkOpts[best_opt];
  chosen[2] = 1 << (h->q - std::max(0, h->tree_L - best_tree));  // leaves per tree CTA
  return H2_OK;
}

h2_status h2_check(h2_handle h, void* stream) {
  if (!h) return fail(H2_ERR_INVALID, "NULL handle");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CUDA_TRY(cudaMemset(h->err, 0, sizeof(int)));
    return fail(H2_ERR_TIMEOUT, "a bounded device wait ran out; products since the last check are invalid");
  }
  return H2_OK;
}

h2_status h2_debug_withhold_copy(h2_handle h, int32_t item, int64_t wait_budget_cycles) {
  if (!h) return fail(H2_ERR_INVALID, "NULL handle");
  h->inject = item;
  h->budget = wait_budget_cycles > 0 ? wait_budget_cycles : kWaitBudget;
  return H2_OK;
}

h2_status h2_info(h2_handle h, int64_t info[8]) {
  if (!h || !info) return fail(H2_ERR_INVALID, "NULL handle or info");
  info[0] = h->paper_bytes;
  info[1] = h->device_bytes + 2 * h->host_cap * 8;
  info[2] = h->nS;
  info[3] = h->nD;
  info[4] = h->q;
  info[5] = h->k;
  info[6] = h->m_max;
  info[7] = h->n;
  return H2_OK;
}

h2_status h2_profile(h2_handle h, int32_t enable) {
  if (!h) return fail(H2_ERR_INVALID, "NULL handle");
  h->prof.on = enable != 0;
  h->prof.used = 0;
  h->prof.launches = 0;
  return H2_OK;
}

h2_status h2_profile_read(h2_handle h, double ms[H2_NPHASES], int64_t* launches) {
  if (!h || !ms) return fail(H2_ERR_INVALID, "NULL handle or output");
  return profile_read(&h->prof, ms, launches);
}

h2_status h2_destroy(h2_handle h) {
  if (!h) return H2_OK;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return H2_OK;
}

}  // extern "C"
