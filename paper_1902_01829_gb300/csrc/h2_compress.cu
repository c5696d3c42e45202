// Algebraic compression of an H^2 matrix on the GPU (Sec. 5 of Boukaram,
// Turkiyyah, Keyes): orthogonalization of the basis trees (Sec. 5.2, Alg. 6),
// projection of the coupling blocks (Alg. 7), generation of the R trees
// (Sec. 5.3, Alg. 9) and truncation of the bases by singular value
// decompositions (Sec. 5.4, Alg. 10), then the second projection.
//
// FP64 throughout. One CTA works on one node (QR, SVD) or one block
// (projection) in shared memory; the sweeps go level by level, one launch per
// level, all on the caller's stream. Ranks found by the truncation live in
// device memory, so a whole run is asynchronous; intermediate arrays keep the
// input rank K as their stride and a level's logical rank bounds the loops.
//
// Differences from the paper's design: no marshaling into batched BLAS/LAPACK
// calls; Householder QR and one-sided Jacobi SVD are written here and run in
// shared memory, one node per CTA. A leaf's W = U R^T with an orthonormal U is
// reduced to the K x K matrix R^T before its SVD.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "h2.h"
#include "h2_internal.h"

using namespace h2i;

struct h2_compressor_s {
  int dev = 0;
  int q = 0, K = 0;
  bool sym = true;
  int64_t n = 0, leaves = 0, n_nodes = 0, nS = 0;
  std::vector<void*> allocs;
  // structure
  int64_t* leaf_off = nullptr;
  int32_t* s_row = nullptr;     // row node of every coupling block
  int32_t* s_col = nullptr;     // column node of every coupling block
  int32_t* r_ptr = nullptr;     // blocks by row node (CSR: the input order)
  int32_t* c_ptr = nullptr;     // blocks by column node (CSC)
  int32_t* c_blk = nullptr;
  // inputs (never written)
  double *U0 = nullptr, *V0 = nullptr, *E0 = nullptr, *F0 = nullptr, *S0 = nullptr;
  // orthogonalization
  double *Uo = nullptr, *Vo = nullptr, *Eo = nullptr, *Fo = nullptr, *TUo = nullptr, *TVo = nullptr, *S1 = nullptr;
  // basis generation and truncation
  double *RU = nullptr, *RV = nullptr, *Ut = nullptr, *Vt = nullptr, *Et = nullptr, *Ft = nullptr;
  double *TUt = nullptr, *TVt = nullptr, *sigU = nullptr, *sigV = nullptr, *workY = nullptr, *workZ = nullptr;
  int* ranks = nullptr;         // [2 (q+1) + 1]: row tree ranks, column tree ranks, uniform rank
  int* stats = nullptr;         // [2]: most and total Jacobi sweeps of the last run
  // results at the uniform rank
  double *oU = nullptr, *oV = nullptr, *oE = nullptr, *oF = nullptr, *oS = nullptr;
  int mode = -1;                // -1 nothing run, 0 orthogonalized, 1 compressed
  bool prof = false;
  cudaEvent_t ev[6] = {};
  int64_t launches = 0;
  int64_t dev_bytes = 0;
};

namespace {

constexpr int kThreads = 256;
constexpr int kSvdThreads = 128;
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int node_level(int64_t h) { return 63 - __clzll((unsigned long long)(h + 1)); }

// In-place Householder QR of the rows x cols matrix A (shared memory, column-major,
// leading dimension lda), by the whole CTA. Afterwards the upper triangle holds R (its
// diagonal of either sign), the strict lower part the reflector vectors (unit leading
// entry implied) and tau[j] their scalars: H_j = I - tau_j v_j v_j^T.
__device__ void cta_householder(double* A, int lda, int rows, int cols, double* tau) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nref = min(rows, cols);
  for (int j = 0; j < nref; j++) {
    if (warp == 0) {
      double s = 0.0;
      for (int i = j + 1 + lane; i < rows; i += 32) s = fma(A[i + j * lda], A[i + j * lda], s);
      s = warp_sum(s);
      const double alpha = A[j + j * lda];
      double t = 0.0, beta = alpha, scale = 1.0;
      if (s > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, s)), alpha);
        t = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      for (int i = j + 1 + lane; i < rows; i += 32) A[i + j * lda] *= scale;
      __syncwarp();
      if (lane == 0) {
        A[j + j * lda] = beta;
        tau[j] = t;
      }
    }
    __syncthreads();
    const double t = tau[j];
    if (t != 0.0) {
      for (int c = j + 1 + warp; c < cols; c += (int)(blockDim.x >> 5)) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) w = fma(A[i + j * lda], A[i + c * lda], w);
        w = t * (warp_sum(w) + A[j + c * lda]);
        if (lane == 0) A[j + c * lda] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) A[i + c * lda] = fma(-w, A[i + j * lda], A[i + c * lda]);
      }
    }
    __syncthreads();
  }
}

// Q = H_0 ... H_{r-1} [I; 0], rows x cols (columns >= rows are zero), from the reflectors
// that cta_householder left in A.
__device__ void cta_form_q(const double* A, int lda, int rows, int cols, const double* tau, double* Q, int ldq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
    const int i = idx % rows, c = idx / rows;
    Q[i + c * ldq] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = min(rows, cols) - 1; j >= 0; j--) {
    const double t = tau[j];
    if (t != 0.0) {
      for (int c = j + warp; c < cols; c += (int)(blockDim.x >> 5)) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) w = fma(A[i + j * lda], Q[i + c * ldq], w);
        w = t * (warp_sum(w) + Q[j + c * ldq]);
        if (lane == 0) Q[j + c * ldq] -= w;
        for (int i = j + 1 + lane; i < rows; i += 32) Q[i + c * ldq] = fma(-w, A[i + j * lda], Q[i + c * ldq]);
      }
    }
    __syncthreads();
  }
}

// sgn[j] = -1 where R's diagonal entry j is negative, else 1 (j < min(rows, cols))
__device__ void cta_diag_signs(const double* A, int lda, int rows, int cols, double* sgn) {
  for (int j = threadIdx.x; j < cols; j += blockDim.x) sgn[j] = (j < rows && A[j + j * lda] < 0.0) ? -1.0 : 1.0;
  __syncthreads();
}

// R (cols x cols, non-negative diagonal, zero rows beyond min(rows, cols)) to global memory
// (column-major, leading dimension ldr)
__device__ void cta_store_r(const double* A, int lda, int rows, int cols, const double* sgn, double* R, int ldr) {
  for (int idx = threadIdx.x; idx < cols * cols; idx += blockDim.x) {
    const int j = idx % cols, c = idx / cols;
    R[j + (int64_t)c * ldr] = (j <= c && j < rows) ? sgn[j] * A[j + c * lda] : 0.0;
  }
}

// ---------------------------------------------------------------------------------------------
// Orthogonalization (Sec. 5.2, Alg. 6)

// Leaf QR: U_i = Q_i T_i. One CTA per leaf; the basis is read from and written to the
// input layout (leaf i at leaf_off[i] * K, column-major size_i x K).
__global__ void __launch_bounds__(kThreads) k_ortho_leaf(const double* __restrict__ U, double* __restrict__ Q,
                                                         double* __restrict__ T, const int64_t* __restrict__ leaf_off,
                                                         int K, int64_t leaf0) {
  extern __shared__ double sm[];
  const int64_t i = blockIdx.x;
  const int64_t off = leaf_off[i];
  const int m = (int)(leaf_off[i + 1] - off);
  double* A = sm;            // m x K
  double* Qs = A + 64 * K;   // m x K
  double* tau = Qs + 64 * K;
  double* sgn = tau + 64;
  for (int idx = threadIdx.x; idx < m * K; idx += blockDim.x) A[idx] = U[off * K + idx];
  __syncthreads();
  cta_householder(A, m, m, K, tau);
  cta_form_q(A, m, m, K, tau, Qs, m);
  cta_diag_signs(A, m, m, K, sgn);
  for (int idx = threadIdx.x; idx < m * K; idx += blockDim.x) Q[off * K + idx] = sgn[idx / m] * Qs[idx];
  cta_store_r(A, m, m, K, sgn, T + (leaf0 + i) * K * K, K);
}

// Inner node p (one CTA each, level l - 1): Z = [T_c1 E_c1; T_c2 E_c2] = Q_Z T_p; the two
// halves of Q_Z are the children's new transfers.
__global__ void __launch_bounds__(kThreads) k_ortho_inner(const double* __restrict__ E, double* __restrict__ Eout,
                                                          double* __restrict__ T, int K, int64_t first) {
  extern __shared__ double sm[];
  const int64_t p = first + blockIdx.x;
  const int rows = 2 * K;
  double* Z = sm;                 // 2K x K
  double* Qs = Z + 2 * K * K;     // 2K x K
  double* tau = Qs + 2 * K * K;
  double* sgn = tau + 64;
  for (int idx = threadIdx.x; idx < rows * K; idx += blockDim.x) {
    const int r = idx % rows, c = idx / rows;
    const int half = r / K, a = r % K;
    const int64_t ch = 2 * p + 1 + half;
    const double* Tc = T + ch * K * K;        // K x K upper triangular
    const double* Ec = E + (ch - 1) * K * K;  // K x K
    double s = 0.0;
    for (int t = a; t < K; t++) s = fma(Tc[a + t * K], Ec[t + c * K], s);
    Z[idx] = s;
  }
  __syncthreads();
  cta_householder(Z, rows, rows, K, tau);
  cta_form_q(Z, rows, rows, K, tau, Qs, rows);
  cta_diag_signs(Z, rows, rows, K, sgn);
  for (int idx = threadIdx.x; idx < rows * K; idx += blockDim.x) {
    const int r = idx % rows, c = idx / rows;
    const int half = r / K, a = r % K;
    Eout[(2 * p + half) * K * K + a + c * K] = sgn[c] * Qs[idx];   // child 2p+1+half at (2p+half) K^2
  }
  cta_store_r(Z, rows, rows, K, sgn, T + p * K * K, K);
}

// ---------------------------------------------------------------------------------------------
// Projection (Alg. 7): S_out = T^U_i S T^V_j^T. T^U_i has ru rows, T^V_j rv rows (the ranks of
// the block's level in the two trees, or K); S_out is ru x rv with leading dimension ldo, at
// block * ldo * ldo (zero-padded to ldo x ldo). tri: both T are upper triangular (the
// orthogonalization's), so each product skips the zero half. One CTA per block, grid-stride.
// X = S T_j^T is kept row-major and the result tile goes through shared memory, so every
// shared-memory access is a broadcast or unit-stride and the global store is coalesced.
__global__ void __launch_bounds__(kThreads) k_project(const double* __restrict__ S, double* __restrict__ Sout,
                                                      const double* __restrict__ TU, const double* __restrict__ TV,
                                                      const int32_t* __restrict__ s_row, const int32_t* __restrict__ s_col,
                                                      int64_t nS, int K, const int* __restrict__ ranks_u,
                                                      const int* __restrict__ ranks_v, const int* __restrict__ ld_out,
                                                      int tri) {
  extern __shared__ double sm[];
  const int K1 = K + 1;
  double* Sb = sm;           // K x K (column-major), then T^U_i
  double* Tj = Sb + K * K;   // K x K (column-major), then the result tile (ld K + 1)
  double* Xt = Tj + K * K1;  // X = S T_j^T, row-major: X[a][c] at c + a (K + 1)
  const int ldo = ld_out ? *ld_out : K;
  for (int64_t b = blockIdx.x; b < nS; b += gridDim.x) {
    const int64_t i = s_row[b], j = s_col[b];
    const int l = node_level(i);
    const int ru = ranks_u ? ranks_u[l] : K, rv = ranks_v ? ranks_v[l] : K;
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
      Sb[idx] = S[b * K * K + idx];
      Tj[idx] = TV[j * K * K + idx];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < K * rv; idx += blockDim.x) {
      const int a = idx % K, c = idx / K;
      double s = 0.0;
      for (int t = tri ? c : 0; t < K; t++) s = fma(Sb[a + t * K], Tj[c + t * K], s);
      Xt[c + a * K1] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Sb[idx] = TU[i * K * K + idx];
    __syncthreads();
    if (rv > 0)
      for (int idx = threadIdx.x; idx < ru * rv; idx += blockDim.x) {
        const int c = idx % rv, a = idx / rv;
        double s = 0.0;
        for (int t = tri ? a : 0; t < K; t++) s = fma(Sb[a + t * K], Xt[c + t * K1], s);
        Tj[a + c * K1] = s;
      }
    __syncthreads();
    double* out = Sout + b * ldo * ldo;
    for (int idx = threadIdx.x; idx < ldo * ldo; idx += blockDim.x) {
      const int a = idx % ldo, c = idx / ldo;
      out[idx] = (a < ru && c < rv) ? Tj[a + c * K1] : 0.0;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Basis generation (Sec. 5.3, Alg. 9): R_i = triangular factor of
// [R_parent E_i^T; S_ij1^T; ...] (row tree, blocks of row i) or [R_parent F_j^T; S_i1j; ...]
// (column tree, blocks of column j). One CTA per node of level l. The stack is reduced a few
// blocks at a time (up to 128 rows): QR of [R; B] with R upper triangular, where the reflector
// of column j touches row j of R and all of B. The warp that updates column j + 1 also forms
// the next reflector, so each column costs one CTA barrier.
__device__ void warp_stack_reflector(double* Rs, int K, double* B, int ldb, int rows, int j, double* tau, int lane) {
  double s = 0.0;
  for (int r = lane; r < rows; r += 32) s = fma(B[r + j * ldb], B[r + j * ldb], s);
  s = warp_sum(s);
  const double alpha = Rs[j + j * K];
  double t = 0.0, beta = alpha, scale = 1.0;
  if (s > 0.0) {
    beta = -copysign(sqrt(fma(alpha, alpha, s)), alpha);
    t = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
  }
  for (int r = lane; r < rows; r += 32) B[r + j * ldb] *= scale;
  __syncwarp();
  if (lane == 0) {
    Rs[j + j * K] = beta;
    tau[j] = t;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kThreads) k_basis_gen(const double* __restrict__ E, const double* __restrict__ S,
                                                        double* __restrict__ R, const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ blk, int columns, int K,
                                                        int64_t first) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t i = first + blockIdx.x;
  const int nb_max = max(1, 128 / K), ldb = nb_max * K;
  double* Rs = sm;            // K x K
  double* B = Rs + K * K;     // up to nb_max stacked K x K blocks (ld ldb)
  double* tau = B + ldb * K;  // K
  double* sgn = tau + 64;
  // M = R_parent E_i^T, then its QR
  const double* Rp = R + ((i - 1) / 2) * K * K;
  const double* Ei = E + (i - 1) * K * K;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int a = idx % K, c = idx / K;
    double s = 0.0;
    for (int t = a; t < K; t++) s = fma(Rp[a + t * K], Ei[c + t * K], s);   // (E_i^T)[t][c] = E_i[c][t]
    Rs[idx] = s;
  }
  __syncthreads();
  cta_householder(Rs, K, K, K, tau);
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int a = idx % K, c = idx / K;
    if (a > c) Rs[idx] = 0.0;
  }
  __syncthreads();
  const int32_t e0 = ptr[i], e1 = ptr[i + 1];
  for (int32_t e = e0; e < e1; e += nb_max) {
    const int nb = min(nb_max, (int)(e1 - e)), rows = nb * K;
    for (int idx = threadIdx.x; idx < rows * K; idx += blockDim.x) {
      const int r = idx % rows, c = idx / rows;
      const int q = r / K, a = r % K;
      const int64_t b = blk ? blk[e + q] : e + q;
      const double* Sb = S + b * K * K;
      B[r + c * ldb] = columns ? Sb[a + c * K] : Sb[c + a * K];   // S_ij or S_ij^T
    }
    __syncthreads();
    if (warp == 0) warp_stack_reflector(Rs, K, B, ldb, rows, 0, tau, lane);
    __syncthreads();
    for (int j = 0; j < K; j++) {
      const double t = tau[j];
      for (int c = j + 1 + warp; c < K; c += nw) {
        if (t != 0.0) {
          double w = 0.0;
          for (int r = lane; r < rows; r += 32) w = fma(B[r + j * ldb], B[r + c * ldb], w);
          w = t * (warp_sum(w) + Rs[j + c * K]);
          __syncwarp();
          if (lane == 0) Rs[j + c * K] -= w;
          for (int r = lane; r < rows; r += 32) B[r + c * ldb] = fma(-w, B[r + j * ldb], B[r + c * ldb]);
        }
        if (c == j + 1) {
          __syncwarp();
          warp_stack_reflector(Rs, K, B, ldb, rows, j + 1, tau, lane);
        }
      }
      __syncthreads();
    }
  }
  cta_diag_signs(Rs, K, K, K, sgn);
  cta_store_r(Rs, K, K, K, sgn, R + i * K * K, K);
}

// ---------------------------------------------------------------------------------------------
// Truncation (Sec. 5.4, Alg. 10)

// One-sided Jacobi (Hestenes) on X (rows x cols, shared memory, column-major, leading
// dimension ld): rotates pairs of columns, in the round-robin order that makes each step's
// pairs disjoint, until every pair is orthogonal to working precision. Afterwards the column
// norms are the singular values of X and the normalized columns its left singular vectors.
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the FP64 work per pair is
// kept to the dot products and the rotation itself: each pair belongs to a group of g lanes
// that split its rows (no CTA-wide reductions), and only the group computes its rotation.
// Returns the number of sweeps.
__device__ int cta_jacobi(double* X, int ld, int rows, int cols, int* flag) {
  const int P = cols + (cols & 1), npairs = P / 2;
  int g = 1;
  while (g < 8 && npairs * g * 2 <= (int)blockDim.x) g <<= 1;
  const int tid = threadIdx.x, grp = tid / g, sub = tid % g, lane = tid & 31;
  const unsigned gmask = (g == 32 ? 0xffffffffu : ((1u << g) - 1u)) << (lane & ~(g - 1));
  const double tol = DBL_EPSILON * (double)max(rows, 8), tol2 = tol * tol;
  int sweeps = 0;
  for (int sweep = 0; sweep < kMaxSweeps; sweep++) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int s = 0; s < P - 1; s++) {
      int a = cols, b = cols;
      if (grp < npairs) {
        if (grp == 0) {
          a = s;
          b = P - 1;
        } else {
          a = (s + grp) % (P - 1);
          b = (s - grp + P - 1) % (P - 1);
        }
      }
      if (a < cols && b < cols) {   // the same for every lane of the group
        double* xa = X + a * ld;
        double* xb = X + b * ld;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = sub; r < rows; r += g) {
          const double u = xa[r], v = xb[r];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        for (int o = 1; o < g; o <<= 1) {
          al += __shfl_xor_sync(gmask, al, o);
          be += __shfl_xor_sync(gmask, be, o);
          ga += __shfl_xor_sync(gmask, ga, o);
        }
        if (ga * ga > tol2 * al * be) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
          const double c = rsqrt(fma(t, t, 1.0)), sn = c * t;
          for (int r = sub; r < rows; r += g) {
            const double u = xa[r], v = xb[r];
            xa[r] = fma(c, u, -sn * v);
            xb[r] = fma(sn, u, c * v);
          }
          if (sub == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    sweeps++;
    if (*flag == 0) break;
    __syncthreads();
  }
  return sweeps;
}

// After cta_jacobi: singular values (descending) to sig[0..cols), the left singular vectors
// in that order, normalized, to Y (rows x cols, leading dimension ldy; zero for a zero
// singular value), and the node's rank (how many of its nsv = min(rows, cols) singular
// values are >= eps times the largest) folded into *rank with atomicMax.
__device__ void cta_sorted_vectors(const double* X, int ld, int rows, int cols, int nsv, double eps, double* nrm,
                                   int* order, double* sig, double* Y, int ldy, int* rank) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < cols; c += (int)(blockDim.x >> 5)) {
    double s = 0.0;
    for (int r = lane; r < rows; r += 32) s = fma(X[r + c * ld], X[r + c * ld], s);
    s = warp_sum(s);
    if (lane == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    int pos = 0;
    for (int d = 0; d < cols; d++) pos += (nrm[d] > nrm[c]) || (nrm[d] == nrm[c] && d < c);
    order[pos] = c;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < cols; t += blockDim.x) sig[t] = nrm[order[t]];
  for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
    const int r = idx % rows, t = idx / rows;
    const int c = order[t];
    const double s = nrm[c];
    Y[r + t * ldy] = s > 0.0 ? X[r + c * ld] / s : 0.0;
  }
  if (threadIdx.x == 0) {
    const double top = nrm[order[0]];
    int cnt = 0;
    if (top > 0.0)
      for (int t = 0; t < nsv; t++) cnt += nrm[order[t]] >= eps * top;
    atomicMax(rank, cnt);
  }
}

// Leaves: W_i = U_i R_i^T with U_i orthonormal (zero columns beyond the leaf size), so the SVD
// of W_i is U_i times that of M = R_i^T with the rows beyond the leaf size cleared. The left
// singular vectors of M go to Y (K x K per leaf).
__global__ void __launch_bounds__(kSvdThreads) k_svd_leaf(const double* __restrict__ R, const int64_t* __restrict__ leaf_off,
                                                          double* __restrict__ sig, double* __restrict__ Y, int* rank,
                                                          int* stats, double eps, int K, int64_t leaf0) {
  extern __shared__ double sm[];
  const int64_t i = blockIdx.x, h = leaf0 + i;
  const int m = (int)(leaf_off[i + 1] - leaf_off[i]);
  double* X = sm;             // K x K
  double* nrm = X + K * K;    // K
  int* order = (int*)(nrm + 64);
  __shared__ int flag;
  const double* Rh = R + h * K * K;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int a = idx % K, c = idx / K;
    X[idx] = a < m ? Rh[c + a * K] : 0.0;   // (R^T)[a][c] = R[c][a]
  }
  __syncthreads();
  const int sw = cta_jacobi(X, K, K, K, &flag);
  if (threadIdx.x == 0) {
    atomicMax(stats, sw);
    atomicAdd(stats + 1, sw);
  }
  cta_sorted_vectors(X, K, K, K, min(m, K), eps, nrm, order, sig + h * K, Y + i * K * K, K, rank);
}

// Inner node p (level l - 1): Z_p = [T_c1 E_c1; T_c2 E_c2] (2 r x K, r the children's new
// rank, E the orthogonal transfers) and W_p = Z_p R_p^T. Z_p goes to global memory (for T_p);
// a warp forms one row of Z_p at a time and from it the same row of W_p, so only W_p needs
// shared memory.
__global__ void __launch_bounds__(kSvdThreads) k_svd_inner(const double* __restrict__ R, const double* __restrict__ E,
                                                           const double* __restrict__ T, double* __restrict__ sig,
                                                           double* __restrict__ Y, double* __restrict__ Zw,
                                                           const int* __restrict__ rank_child, int* rank, int* stats,
                                                           double eps, int K, int64_t first) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t p = first + blockIdx.x;
  const int r = *rank_child, rows = 2 * r;
  const int ld = 2 * K;
  double* X = sm;                  // 2r x K (ld 2K)
  double* nrm = X + 2 * K * K;     // 64
  double* zrow = nrm + 64;         // one row of Z per warp (K each)
  int* order = (int*)(zrow + nw * 64);
  __shared__ int flag;
  const double* Rp = R + p * K * K;
  double* Zp = Zw + blockIdx.x * 2 * K * K;
  for (int a2 = warp; a2 < rows; a2 += nw) {
    const int half = a2 / r, a = a2 % r;
    const int64_t ch = 2 * p + 1 + half;
    const double* Tc = T + ch * K * K;
    const double* Ec = E + (ch - 1) * K * K;
    for (int c = lane; c < K; c += 32) {
      double z = 0.0;
      for (int t = 0; t < K; t++) z = fma(Tc[a + t * K], Ec[t + c * K], z);
      zrow[warp * 64 + c] = z;
      Zp[a2 + c * ld] = z;
    }
    __syncwarp();
    for (int c = lane; c < K; c += 32) {
      double x = 0.0;
      for (int t = c; t < K; t++) x = fma(zrow[warp * 64 + t], Rp[c + t * K], x);   // (R^T)[t][c] = R[c][t], R upper
      X[a2 + c * ld] = x;
    }
    __syncwarp();
  }
  __syncthreads();
  if (rows > 0) {
    const int sw = cta_jacobi(X, ld, rows, K, &flag);
    if (threadIdx.x == 0) {
      atomicMax(stats, sw);
      atomicAdd(stats + 1, sw);
    }
    cta_sorted_vectors(X, ld, rows, K, min(rows, K), eps, nrm, order, sig + p * K, Y + blockIdx.x * 2 * K * K, ld,
                       rank);
  } else {
    for (int t = threadIdx.x; t < K; t += blockDim.x) sig[p * K + t] = 0.0;
  }
}

// Leaves, once the level rank r is known: Q_i = U_i Y[:, :r] (new basis, size_i x r in a
// size_i x K slot) and T_i = Q_i^T U_i (r x K).
__global__ void __launch_bounds__(kThreads) k_trunc_leaf(const double* __restrict__ U, const double* __restrict__ Y,
                                                         double* __restrict__ Ut, double* __restrict__ T,
                                                         const int64_t* __restrict__ leaf_off, const int* __restrict__ rank,
                                                         int K, int64_t leaf0) {
  extern __shared__ double sm[];
  const int64_t i = blockIdx.x;
  const int64_t off = leaf_off[i];
  const int m = (int)(leaf_off[i + 1] - off), r = *rank;
  double* Ui = sm;           // m x K
  double* Q = Ui + 64 * K;   // m x K
  const double* Yi = Y + i * K * K;
  for (int idx = threadIdx.x; idx < m * K; idx += blockDim.x) Ui[idx] = U[off * K + idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * K; idx += blockDim.x) {
    const int a = idx % m, c = idx / m;
    double s = 0.0;
    if (c < r)
      for (int t = 0; t < K; t++) s = fma(Ui[a + t * m], Yi[t + c * K], s);
    Q[idx] = s;
    Ut[off * K + idx] = s;
  }
  __syncthreads();
  double* Th = T + (leaf0 + i) * K * K;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int a = idx % K, c = idx / K;
    double s = 0.0;
    if (a < r)
      for (int t = 0; t < m; t++) s = fma(Q[t + a * m], Ui[t + c * m], s);
    Th[idx] = s;
  }
}

// Inner node p, once the parent level's rank rp is known: Q_p = Y[:, :rp] (2 rc x rp); its
// halves are the children's new transfers (rc x rp in K x K slots) and T_p = Q_p^T Z_p.
__global__ void __launch_bounds__(kThreads) k_trunc_inner(const double* __restrict__ Y, const double* __restrict__ Zw,
                                                          double* __restrict__ Et, double* __restrict__ T,
                                                          const int* __restrict__ rank_child, const int* __restrict__ rank,
                                                          int K, int64_t first) {
  const int64_t p = first + blockIdx.x;
  const int rc = *rank_child, rp = *rank, ld = 2 * K;
  const double* Yp = Y + blockIdx.x * 2 * K * K;
  const double* Zp = Zw + blockIdx.x * 2 * K * K;
  for (int idx = threadIdx.x; idx < 2 * K * K; idx += blockDim.x) {
    const int half = idx / (K * K), w = idx % (K * K);
    const int a = w % K, c = w / K;
    const int64_t ch = 2 * p + 1 + half;
    Et[(ch - 1) * K * K + w] = (a < rc && c < rp) ? Yp[half * rc + a + c * ld] : 0.0;
  }
  double* Tp = T + p * K * K;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
    const int a = idx % K, c = idx / K;
    double s = 0.0;
    if (a < rp)
      for (int t = 0; t < 2 * rc; t++) s = fma(Yp[t + a * ld], Zp[t + c * ld], s);
    Tp[idx] = s;
  }
}

// uniform rank = the largest level rank of either tree (at least 1)
__global__ void k_uniform_rank(int* ranks, int q) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int m = 1;
    for (int l = 0; l < 2 * (q + 1); l++) m = max(m, ranks[l]);
    ranks[2 * (q + 1)] = m;
  }
}

// Repack the truncated bases and transfers (stride K) at the uniform rank Kt.
__global__ void k_pack_bases(const double* __restrict__ Ut, double* __restrict__ oU, const int64_t* __restrict__ leaf_off,
                             int64_t leaves, int K, const int* __restrict__ kt) {
  const int Kt = *kt;
  for (int64_t i = blockIdx.x; i < leaves; i += gridDim.x) {
    const int64_t off = leaf_off[i];
    const int m = (int)(leaf_off[i + 1] - off);
    for (int idx = threadIdx.x; idx < m * Kt; idx += blockDim.x) oU[off * Kt + idx] = Ut[off * K + idx];
  }
}

__global__ void k_pack_transfers(const double* __restrict__ Et, double* __restrict__ oE, int64_t count, int K,
                                 const int* __restrict__ kt) {
  const int Kt = *kt;
  for (int64_t h = blockIdx.x; h < count; h += gridDim.x)
    for (int idx = threadIdx.x; idx < Kt * Kt; idx += blockDim.x) {
      const int a = idx % Kt, c = idx / Kt;
      oE[h * Kt * Kt + idx] = Et[h * K * K + a + c * K];
    }
}

// ---------------------------------------------------------------------------------------------
// host side

h2_status (&fail)(h2_status, const char*, ...) = h2_fail;

template <typename T>
h2_status calloc_dev(h2_compressor_s* c, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) return H2_OK;
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, "cudaMalloc of %lld bytes: %s",
                (long long)(count * (int64_t)sizeof(T)), cudaGetErrorString(e));
  }
  c->allocs.push_back(v);
  c->dev_bytes += count * (int64_t)sizeof(T);
  CUDA_TRY(cudaMemset(v, 0, (size_t)count * sizeof(T)));
  *p = (T*)v;
  return H2_OK;
}

template <typename T>
h2_status upload_dev(h2_compressor_s* c, T** p, const T* src, int64_t count) {
  h2_status st = calloc_dev(c, p, count);
  if (st != H2_OK || count <= 0) return st;
  CUDA_TRY(cudaMemcpy(*p, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice));
  return H2_OK;
}

void release(h2_compressor_s* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  for (cudaEvent_t& e : c->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
}

size_t smem_qr_leaf(int K) { return (size_t)(2 * 64 * K + 128) * sizeof(double); }
size_t smem_qr_inner(int K) { return (size_t)(4 * K * K + 128) * sizeof(double); }
size_t smem_project(int K) { return (size_t)(K * K + 2 * K * (K + 1)) * sizeof(double); }
size_t smem_basis(int K) { return (size_t)(K * K + std::max(1, 128 / K) * K * K + 128) * sizeof(double); }
size_t smem_svd_leaf(int K) { return (size_t)(K * K + 64) * sizeof(double) + 64 * sizeof(int); }
size_t smem_svd_inner(int K) {
  return (size_t)(2 * K * K + 64 + (kSvdThreads / 32) * 64) * sizeof(double) + 64 * sizeof(int);
}
size_t smem_trunc_leaf(int K) { return (size_t)(2 * 64 * K) * sizeof(double); }

h2_status set_smem() {
  const size_t big = smem_qr_inner(64);
  CUDA_TRY(cudaFuncSetAttribute(k_ortho_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_qr_leaf(64)));
  CUDA_TRY(cudaFuncSetAttribute(k_ortho_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big));
  CUDA_TRY(cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_project(64)));
  CUDA_TRY(cudaFuncSetAttribute(k_basis_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_basis(64)));
  CUDA_TRY(cudaFuncSetAttribute(k_svd_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_svd_leaf(64)));
  CUDA_TRY(cudaFuncSetAttribute(k_svd_inner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_svd_inner(64)));
  CUDA_TRY(cudaFuncSetAttribute(k_trunc_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_trunc_leaf(64)));
  return H2_OK;
}

int proj_grid(int64_t nS) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>(nS, (int64_t)sms * 16));
}

// orthogonalize one basis tree: leaves, then the inner levels bottom up
h2_status ortho_tree(h2_compressor_s* c, const double* U, const double* E, double* Uo, double* Eo, double* T,
                     cudaStream_t st) {
  const int K = c->K, q = c->q;
  k_ortho_leaf<<<(unsigned)c->leaves, kThreads, smem_qr_leaf(K), st>>>(U, Uo, T, c->leaf_off, K, c->leaves - 1);
  c->launches++;
  for (int l = q; l >= 1; l--) {
    const int64_t first = ((int64_t)1 << (l - 1)) - 1, cnt = (int64_t)1 << (l - 1);
    k_ortho_inner<<<(unsigned)cnt, kThreads, smem_qr_inner(K), st>>>(E, Eo, T, K, first);
    c->launches++;
  }
  CUDA_TRY(cudaGetLastError());
  return H2_OK;
}

h2_status basis_tree(h2_compressor_s* c, const double* Eo, double* R, bool columns, cudaStream_t st) {
  const int K = c->K;
  CUDA_TRY(cudaMemsetAsync(R, 0, (size_t)K * K * sizeof(double), st));   // R^0 = 0
  for (int l = 1; l <= c->q; l++) {
    const int64_t first = ((int64_t)1 << l) - 1, cnt = (int64_t)1 << l;
    k_basis_gen<<<(unsigned)cnt, kThreads, smem_basis(K), st>>>(Eo, c->S1, R, columns ? c->c_ptr : c->r_ptr,
                                                                columns ? c->c_blk : nullptr, columns ? 1 : 0, K, first);
    c->launches++;
  }
  CUDA_TRY(cudaGetLastError());
  return H2_OK;
}

h2_status trunc_tree(h2_compressor_s* c, const double* Uo, const double* Eo, const double* R, double* Ut, double* Et,
                     double* T, double* sig, int* ranks, double eps, cudaStream_t st) {
  const int K = c->K, q = c->q;
  k_svd_leaf<<<(unsigned)c->leaves, kSvdThreads, smem_svd_leaf(K), st>>>(R, c->leaf_off, sig, c->workY, ranks + q,
                                                                         c->stats, eps, K, c->leaves - 1);
  k_trunc_leaf<<<(unsigned)c->leaves, kThreads, smem_trunc_leaf(K), st>>>(Uo, c->workY, Ut, T, c->leaf_off, ranks + q,
                                                                          K, c->leaves - 1);
  c->launches += 2;
  for (int l = q; l >= 1; l--) {
    const int64_t first = ((int64_t)1 << (l - 1)) - 1, cnt = (int64_t)1 << (l - 1);
    k_svd_inner<<<(unsigned)cnt, kSvdThreads, smem_svd_inner(K), st>>>(R, Eo, T, sig, c->workY, c->workZ, ranks + l,
                                                                       ranks + l - 1, c->stats, eps, K, first);
    k_trunc_inner<<<(unsigned)cnt, kThreads, 0, st>>>(c->workY, c->workZ, Et, T, ranks + l, ranks + l - 1, K, first);
    c->launches += 2;
  }
  CUDA_TRY(cudaGetLastError());
  return H2_OK;
}

void mark(h2_compressor_s* c, int e, cudaStream_t st) {
  if (c->prof) cudaEventRecord(c->ev[e], st);
}

}  // namespace

extern "C" {

h2_status h2_compress_create(const h2_desc* d, h2_compressor* out) {
  if (!out) return fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int64_t nS = 0, nD = 0, nDval = 0;
  int m_max = 0;
  h2_status st = validate_desc(d, true, false, &nS, &nD, &nDval, &m_max);
  if (st != H2_OK) return st;
  if (d->storage != H2_FP64) return fail(H2_ERR_UNSUPPORTED, "compression takes the FP64 storage form");
  if (nS >= ((int64_t)1 << 31)) return fail(H2_ERR_UNSUPPORTED, "%lld coupling blocks >= 2^31", (long long)nS);
  h2_compressor_s* c = new (std::nothrow) h2_compressor_s();
  if (!c) return fail(H2_ERR_OOM, "host allocation failed");
  cudaGetDevice(&c->dev);
  c->q = d->depth;
  c->K = d->rank;
  c->sym = d->symmetric != 0;
  c->n = d->n;
  c->leaves = (int64_t)1 << c->q;
  c->n_nodes = ((int64_t)2 << c->q) - 1;
  c->nS = nS;
  const int K = c->K;
  const int64_t KK = (int64_t)K * K, nodes = c->n_nodes;
  // structure: row and column node of every block, blocks by column node
  std::vector<int32_t> srow((size_t)nS), cptr((size_t)nodes + 1, 0), cblk((size_t)nS);
  for (int64_t r = 0; r < nodes; r++)
    for (int32_t b = d->S_rowptr[r]; b < d->S_rowptr[r + 1]; b++) {
      srow[b] = (int32_t)r;
      cptr[d->S_colidx[b] + 1]++;
    }
  for (int64_t h = 0; h < nodes; h++) cptr[h + 1] += cptr[h];
  {
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t b = 0; b < nS; b++) cblk[fill[d->S_colidx[b]]++] = (int32_t)b;
  }
  st = set_smem();
  const int64_t inner_max = std::max<int64_t>(c->leaves / 2, 1);
  auto run = [&]() -> h2_status {
    h2_status s;
    if ((s = upload_dev(c, &c->leaf_off, d->leaf_offset, c->leaves + 1)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->s_row, srow.data(), nS)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->s_col, d->S_colidx, nS)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->r_ptr, d->S_rowptr, nodes + 1)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->c_ptr, cptr.data(), nodes + 1)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->c_blk, cblk.data(), nS)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->U0, d->U, c->n * K)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->E0, d->E, (nodes - 1) * KK)) != H2_OK) return s;
    if ((s = upload_dev(c, &c->S0, d->S_val, nS * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->Uo, c->n * K)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->Eo, (nodes - 1) * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->TUo, nodes * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->S1, nS * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->RU, nodes * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->Ut, c->n * K)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->Et, (nodes - 1) * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->TUt, nodes * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->sigU, nodes * K)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->workY, std::max(c->leaves * KK, inner_max * 2 * KK))) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->workZ, inner_max * 2 * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->ranks, 2 * (c->q + 1) + 1)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->stats, 2)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->oU, c->n * K)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->oE, (nodes - 1) * KK)) != H2_OK) return s;
    if ((s = calloc_dev(c, &c->oS, nS * KK)) != H2_OK) return s;
    if (!c->sym) {
      if ((s = upload_dev(c, &c->V0, d->V, c->n * K)) != H2_OK) return s;
      if ((s = upload_dev(c, &c->F0, d->F, (nodes - 1) * KK)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->Vo, c->n * K)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->Fo, (nodes - 1) * KK)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->TVo, nodes * KK)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->RV, nodes * KK)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->Vt, c->n * K)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->Ft, (nodes - 1) * KK)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->TVt, nodes * KK)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->sigV, nodes * K)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->oV, c->n * K)) != H2_OK) return s;
      if ((s = calloc_dev(c, &c->oF, (nodes - 1) * KK)) != H2_OK) return s;
    }
    for (cudaEvent_t& e : c->ev) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaDeviceSynchronize());
    return H2_OK;
  };
  if (st == H2_OK) st = run();
  if (st != H2_OK) {
    release(c);
    delete c;
    return st;
  }
  *out = c;
  return H2_OK;
}

h2_status h2_compress_run(h2_compressor c, double eps, void* stream) {
  if (!c) return fail(H2_ERR_INVALID, "compressor is NULL");
  if (!(eps < 1.0) || std::isnan(eps)) return fail(H2_ERR_INVALID, "eps = %g: use eps < 0 (orthogonalize only) or 0 <= eps < 1", eps);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != c->dev) return fail(H2_ERR_INVALID, "compressor lives on device %d, current device is %d", c->dev, dev);
  cudaStream_t st = (cudaStream_t)stream;
  const int K = c->K, q = c->q;
  const bool sym = c->sym;
  h2_status s;
  c->launches = 0;
  mark(c, 0, st);
  // Sec. 5.2, Alg. 6: orthogonal bases and projection trees
  if ((s = ortho_tree(c, c->U0, c->E0, c->Uo, c->Eo, c->TUo, st)) != H2_OK) return s;
  if (!sym && (s = ortho_tree(c, c->V0, c->F0, c->Vo, c->Fo, c->TVo, st)) != H2_OK) return s;
  mark(c, 1, st);
  // Alg. 7: coupling blocks in the orthogonal bases
  k_project<<<proj_grid(c->nS), kThreads, smem_project(K), st>>>(c->S0, c->S1, c->TUo, sym ? c->TUo : c->TVo, c->s_row,
                                                                  c->s_col, c->nS, K, nullptr, nullptr, nullptr, 1);
  c->launches++;
  CUDA_TRY(cudaGetLastError());
  mark(c, 2, st);
  if (eps < 0.0) {
    mark(c, 3, st);
    mark(c, 4, st);
    mark(c, 5, st);
    c->mode = 0;
    return H2_OK;
  }
  // Sec. 5.3, Alg. 9: R trees
  if ((s = basis_tree(c, c->Eo, c->RU, false, st)) != H2_OK) return s;
  if (!sym && (s = basis_tree(c, c->Fo, c->RV, true, st)) != H2_OK) return s;
  mark(c, 3, st);
  // Sec. 5.4, Alg. 10: truncated bases, one rank per level
  CUDA_TRY(cudaMemsetAsync(c->ranks, 0, (size_t)(2 * (q + 1) + 1) * sizeof(int), st));
  CUDA_TRY(cudaMemsetAsync(c->stats, 0, 2 * sizeof(int), st));
  if ((s = trunc_tree(c, c->Uo, c->Eo, c->RU, c->Ut, c->Et, c->TUt, c->sigU, c->ranks, eps, st)) != H2_OK) return s;
  if (sym) {
    CUDA_TRY(cudaMemcpyAsync(c->ranks + q + 1, c->ranks, (size_t)(q + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st));
  } else if ((s = trunc_tree(c, c->Vo, c->Fo, c->RV, c->Vt, c->Ft, c->TVt, c->sigV, c->ranks + q + 1, eps, st)) != H2_OK) {
    return s;
  }
  k_uniform_rank<<<1, 32, 0, st>>>(c->ranks, q);
  c->launches++;
  mark(c, 4, st);
  // second projection, written at the uniform rank; bases and transfers repacked to it
  const int* kt = c->ranks + 2 * (q + 1);
  k_project<<<proj_grid(c->nS), kThreads, smem_project(K), st>>>(c->S1, c->oS, c->TUt, sym ? c->TUt : c->TVt, c->s_row,
                                                                  c->s_col, c->nS, K, c->ranks, c->ranks + q + 1, kt, 0);
  k_pack_bases<<<1024, 128, 0, st>>>(c->Ut, c->oU, c->leaf_off, c->leaves, K, kt);
  k_pack_transfers<<<1024, 128, 0, st>>>(c->Et, c->oE, c->n_nodes - 1, K, kt);
  c->launches += 3;
  if (!sym) {
    k_pack_bases<<<1024, 128, 0, st>>>(c->Vt, c->oV, c->leaf_off, c->leaves, K, kt);
    k_pack_transfers<<<1024, 128, 0, st>>>(c->Ft, c->oF, c->n_nodes - 1, K, kt);
    c->launches += 2;
  }
  CUDA_TRY(cudaGetLastError());
  mark(c, 5, st);
  c->mode = 1;
  return H2_OK;
}

h2_status h2_compress_result(h2_compressor c, int32_t* k_out, int32_t* ranks_u, int32_t* ranks_v, void* stream) {
  if (!c) return fail(H2_ERR_INVALID, "compressor is NULL");
  if (c->mode < 0) return fail(H2_ERR_INVALID, "h2_compress_run has not been called");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  const int q = c->q;
  std::vector<int> r((size_t)(2 * (q + 1) + 1), c->K);
  if (c->mode == 1) CUDA_TRY(cudaMemcpy(r.data(), c->ranks, r.size() * sizeof(int), cudaMemcpyDeviceToHost));
  if (k_out) *k_out = r[2 * (q + 1)];
  for (int l = 0; l <= q; l++) {
    if (ranks_u) ranks_u[l] = r[l];
    if (ranks_v) ranks_v[l] = r[q + 1 + l];
  }
  return H2_OK;
}

h2_status h2_compress_read(h2_compressor c, int32_t what, double* dst, int64_t count, void* stream) {
  if (!c) return fail(H2_ERR_INVALID, "compressor is NULL");
  if (!dst && count > 0) return fail(H2_ERR_INVALID, "dst is NULL");
  if (c->mode < 0) return fail(H2_ERR_INVALID, "h2_compress_run has not been called");
  int32_t kt = c->K;
  h2_status s = h2_compress_result(c, &kt, nullptr, nullptr, stream);
  if (s != H2_OK) return s;
  const int64_t K = c->K, KK = K * K, Kt = kt;
  const bool orth = c->mode == 0;
  const double* src = nullptr;
  int64_t need = 0;
  switch (what) {
    case H2C_U: src = orth ? c->Uo : c->oU; need = c->n * Kt; break;
    case H2C_V: src = c->sym ? (orth ? c->Uo : c->oU) : (orth ? c->Vo : c->oV); need = c->n * Kt; break;
    case H2C_E: src = orth ? c->Eo : c->oE; need = (c->n_nodes - 1) * Kt * Kt; break;
    case H2C_F: src = c->sym ? (orth ? c->Eo : c->oE) : (orth ? c->Fo : c->oF); need = (c->n_nodes - 1) * Kt * Kt; break;
    case H2C_S: src = orth ? c->S1 : c->oS; need = c->nS * Kt * Kt; break;
    case H2C_T_ORTHO_U: src = c->TUo; need = c->n_nodes * KK; break;
    case H2C_T_ORTHO_V: src = c->sym ? c->TUo : c->TVo; need = c->n_nodes * KK; break;
    case H2C_R_U:
    case H2C_R_V:
    case H2C_SIGMA_U:
    case H2C_SIGMA_V:
      if (orth) return fail(H2_ERR_INVALID, "array %d exists only after a compression (eps >= 0)", what);
      if (what == H2C_R_U || what == H2C_R_V) {
        src = (what == H2C_R_U || c->sym) ? c->RU : c->RV;
        need = c->n_nodes * KK;
      } else {
        src = (what == H2C_SIGMA_U || c->sym) ? c->sigU : c->sigV;
        need = c->n_nodes * K;
      }
      break;
    default: return fail(H2_ERR_INVALID, "unknown array %d", what);
  }
  if (count != need) return fail(H2_ERR_INVALID, "array %d holds %lld values, count is %lld", what, (long long)need, (long long)count);
  if (need > 0) CUDA_TRY(cudaMemcpy(dst, src, (size_t)need * sizeof(double), cudaMemcpyDeviceToHost));
  return H2_OK;
}

h2_status h2_compress_profile(h2_compressor c, int32_t enable) {
  if (!c) return fail(H2_ERR_INVALID, "compressor is NULL");
  c->prof = enable != 0;
  return H2_OK;
}

h2_status h2_compress_profile_read(h2_compressor c, double ms[H2C_NPHASES], int64_t* launches) {
  if (!c) return fail(H2_ERR_INVALID, "compressor is NULL");
  if (!c->prof) return fail(H2_ERR_INVALID, "profiling is off");
  CUDA_TRY(cudaEventSynchronize(c->ev[5]));
  for (int p = 0; p < H2C_NPHASES; p++) {
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, c->ev[p], c->ev[p + 1]));
    ms[p] = t;
  }
  if (launches) *launches = c->launches;
  return H2_OK;
}

h2_status h2_compress_info(h2_compressor c, int64_t info[6]) {
  if (!c || !info) return fail(H2_ERR_INVALID, "NULL argument");
  int st[2] = {0, 0};
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(st, c->stats, sizeof st, cudaMemcpyDeviceToHost));
  info[0] = st[0];
  info[1] = st[1];
  info[2] = c->dev_bytes;
  info[3] = c->nS;
  info[4] = c->q;
  info[5] = c->K;
  return H2_OK;
}

h2_status h2_compress_destroy(h2_compressor c) {
  if (!c) return H2_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != c->dev) cudaSetDevice(c->dev);
  release(c);
  if (cur != c->dev) cudaSetDevice(cur);
  delete c;
  return H2_OK;
}

}  // extern "C"
