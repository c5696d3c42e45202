// Construction of an H^2 covariance matrix on the GPU (Sec. 4.6 of Boukaram,
// Turkiyyah, Keyes): the cluster tree by KD bisection, tight boxes and
// Chebyshev interpolation nodes, the dual traversal that yields the coupling
// and dense block structures, and optionally the values of the leaf bases,
// transfers, coupling blocks and dense blocks, all in FP64 device memory.
//
// KD bisection without a sort per node: every dimension d keeps a list L_d of
// the points ordered by (coordinate d, original index), built once with a
// bitonic sort. A node owns the same position range in every list, so its
// tight box is read off the ends of its ranges, and its split (the first
// ceil(s/2) points along the longest side) becomes, in every list, a stable
// partition by a left/right flag: an exclusive scan of the flags gives every
// entry its new position, and each child's ranges stay ordered. The cluster
// order of a leaf is its parent's split list, which is the order the
// definition gives (points ordered by the parent's split coordinate).
//
// The dual traversal runs level by level over a frontier of node pairs; pairs
// are classified, counted and written out with atomics in any order, then the
// blocks are sorted by (row, column) into block-sparse rows. Boxes, diameters,
// distances and Chebyshev nodes use the same operations in the same order as
// their definition (no contraction into FMAs), so the structure is exact.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <new>
#include <vector>

#include "h2.h"
#include "h2_internal.h"

using namespace h2i;

struct h2_built_s {
  int dev = 0;
  int dim = 0, m = 0, p = 0, k = 0, q = 0, kernel = 0, values = 0;
  double eta = 0.0, ell = 0.0;
  int64_t n = 0, leaves = 0, n_nodes = 0, nS = 0, nD = 0, nDval = 0;
  std::vector<void*> allocs;
  int64_t dev_bytes = 0;
  double* X = nullptr;        // n x dim, original order
  double* Xc = nullptr;       // n x dim, cluster order
  int64_t* perm = nullptr;    // cluster position -> original index
  int64_t* leaf_off = nullptr;
  double *bmin = nullptr, *bmax = nullptr;   // n_nodes x dim
  double* cheb = nullptr;     // n_nodes x dim x p
  int32_t *S_rowptr = nullptr, *S_colidx = nullptr, *D_rowptr = nullptr, *D_colidx = nullptr;
  int64_t* D_valoff = nullptr;
  uint64_t* S_keys = nullptr;   // sorted (row << 32 | column) of every coupling block
  uint64_t* D_keys = nullptr;
  double *U = nullptr, *E = nullptr, *S_val = nullptr, *D_val = nullptr;
  double ms[3] = {0, 0, 0};     // tree and boxes, dual traversal and block rows, values
};

namespace {

constexpr int kTile = 2048;   // elements of a shared-memory bitonic tile (1024 threads)

h2_status (&fail)(h2_status, const char*, ...) = h2_fail;

struct DKey {
  double k;     // coordinate
  int32_t i;    // original index
};
__device__ __forceinline__ bool key_less(const DKey& a, const DKey& b) { return a.k < b.k || (a.k == b.k && a.i < b.i); }
__device__ __forceinline__ bool key_less(uint64_t a, uint64_t b) { return a < b; }

// one compare-exchange stage (k, j) of a bitonic sort over N elements (j >= kTile)
template <class T>
__global__ void k_bitonic_global(T* a, int64_t N, int64_t j, int64_t k) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N / 2) return;
  const int64_t lo = (t / j) * 2 * j + (t % j), hi = lo + j;
  const bool asc = (lo & k) == 0;
  const T x = a[lo], y = a[hi];
  if (key_less(y, x) == asc) {
    a[lo] = y;
    a[hi] = x;
  }
}

// the stages j = jstart ... 1 of the merges k0 ... k1 (doubling) inside tiles of kTile elements
template <class T>
__global__ void __launch_bounds__(1024) k_bitonic_tile(T* a, int64_t k0, int64_t k1, int64_t jstart) {
  __shared__ T s[kTile];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) s[i] = a[base + i];
  __syncthreads();
  for (int64_t k = k0; k <= k1; k <<= 1) {
    for (int64_t j = (k == k0 ? jstart : k / 2); j >= 1; j >>= 1) {
      const int t = threadIdx.x;
      const int lo = (int)((t / j) * 2 * j + (t % j)), hi = lo + (int)j;
      const bool asc = ((base + lo) & k) == 0;
      const T x = s[lo], y = s[hi];
      if (key_less(y, x) == asc) {
        s[lo] = y;
        s[hi] = x;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) a[base + i] = s[i];
}

// ascending sort of N (a power of two, >= kTile) elements
template <class T>
void bitonic_sort(T* a, int64_t N, cudaStream_t st) {
  k_bitonic_tile<T><<<(unsigned)(N / kTile), 1024, 0, st>>>(a, 2, kTile, 1);
  for (int64_t k = 2 * (int64_t)kTile; k <= N; k <<= 1) {
    for (int64_t j = k / 2; j >= kTile; j >>= 1)
      k_bitonic_global<T><<<(unsigned)((N / 2 + 255) / 256), 256, 0, st>>>(a, N, j, k);
    k_bitonic_tile<T><<<(unsigned)(N / kTile), 1024, 0, st>>>(a, k, k, kTile / 2);
  }
}

int64_t sort_size(int64_t n) {
  int64_t N = kTile;
  while (N < n) N <<= 1;
  return N;
}

// exclusive scan of 1024-element blocks; block totals to sums
template <class T>
__global__ void __launch_bounds__(1024) k_scan_block(const T* in, T* out, T* sums, int64_t n) {
  __shared__ T wsum[32];
  const int64_t i = blockIdx.x * 1024LL + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T v = i < n ? in[i] : (T)0;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const T excl = x - v + (warp > 0 ? wsum[warp - 1] : (T)0);
  if (i < n) out[i] = excl;
  if (threadIdx.x == 1023) sums[blockIdx.x] = excl + v;
}

template <class T>
__global__ void k_scan_add(T* out, const T* offs, int64_t n) {
  const int64_t i = blockIdx.x * 1024LL + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

// exclusive scan of n values (in may equal out); ws holds at least scan_ws(n) elements
int64_t scan_ws(int64_t n) {
  int64_t total = 0;
  while (n > 1) {
    n = (n + 1023) / 1024;
    total += n + 1;
  }
  return total + 2;
}

template <class T>
void exclusive_scan(const T* in, T* out, int64_t n, T* ws, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t nb = (n + 1023) / 1024;
  T* sums = ws;
  k_scan_block<T><<<(unsigned)nb, 1024, 0, st>>>(in, out, sums, n);
  if (nb > 1) {
    exclusive_scan<T>(sums, sums, nb, ws + nb + 1, st);
    k_scan_add<T><<<(unsigned)nb, 1024, 0, st>>>(out, sums, n);
  }
}

struct Lists {
  int32_t* L[3];
};

__global__ void k_sort_init(const double* X, int dim, int d, int64_t n, int64_t N, DKey* keys) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  keys[i] = i < n ? DKey{X[i * dim + d], (int32_t)i} : DKey{INFINITY, INT32_MAX};
}

__global__ void k_sort_take(const DKey* keys, int64_t n, int32_t* L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) L[i] = keys[i].i;
}

// node of level `first` (cnt nodes) that owns cluster position pos
__device__ __forceinline__ int64_t find_node(const int64_t* nlo, int64_t first, int64_t cnt, int64_t pos) {
  int64_t a = 0, b = cnt - 1;
  while (a < b) {
    const int64_t mid = (a + b + 1) / 2;
    if (nlo[first + mid] <= pos) a = mid;
    else b = mid - 1;
  }
  return first + a;
}

// split dimension of every node of a level: the longest side of its tight box (read off the
// ends of its ordered ranges), the lowest dimension on a tie
__global__ void k_split_dim(const double* X, int dim, Lists Ls, const int64_t* nlo, const int64_t* nhi, int64_t first,
                            int64_t cnt, int8_t* ds) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t h = first + t, lo = nlo[h], hi = nhi[h];
  int best = 0;
  double w = 0.0;
  for (int d = 0; d < dim; d++) {
    const double wd = __dsub_rn(X[(int64_t)Ls.L[d][hi - 1] * dim + d], X[(int64_t)Ls.L[d][lo] * dim + d]);
    if (d == 0 || wd > w) {
      w = wd;
      best = d;
    }
  }
  ds[h] = (int8_t)best;
}

// left (1) / right (0) flag of every point: the first ceil(s/2) of its node's split list
__global__ void k_flags(Lists Ls, const int8_t* ds, const int64_t* nlo, const int64_t* nhi, int64_t first, int64_t cnt,
                        int64_t n, uint8_t* flag) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= n) return;
  const int64_t h = find_node(nlo, first, cnt, pos);
  const int64_t lo = nlo[h], s = nhi[h] - lo;
  flag[Ls.L[ds[h]][pos]] = (pos - lo) < (s + 1) / 2 ? 1 : 0;
}

__global__ void k_gather_flags(const int32_t* L, const uint8_t* flag, int32_t* f, int64_t n) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos < n) f[pos] = flag[L[pos]];
}

// stable partition of every node's range of L by the flags (sc = exclusive scan of f)
__global__ void k_partition(const int32_t* L, const int32_t* f, const int32_t* sc, const int64_t* nlo,
                            const int64_t* nhi, int64_t first, int64_t cnt, int64_t n, int32_t* Lout) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= n) return;
  const int64_t h = find_node(nlo, first, cnt, pos);
  const int64_t lo = nlo[h], hi = nhi[h], mid = lo + (hi - lo + 1) / 2;
  const int64_t left_before = sc[pos] - sc[lo];
  const int64_t np = f[pos] ? lo + left_before : mid + (pos - lo - left_before);
  Lout[np] = L[pos];
}

// cluster order: a leaf's points in its parent's split list (identity for a single leaf)
__global__ void k_perm(const double* X, int dim, Lists Ls, const int8_t* ds, const int64_t* nlo, int64_t first,
                       int64_t cnt, int q, int64_t n, int64_t* perm, double* Xc) {
  const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pos >= n) return;
  int64_t o = pos;
  if (q > 0) {
    const int64_t h = find_node(nlo, first, cnt, pos);
    o = Ls.L[ds[(h - 1) / 2]][pos];
  }
  perm[pos] = o;
  for (int d = 0; d < dim; d++) Xc[pos * dim + d] = X[o * dim + d];
}

// tight boxes: leaves from the ends of their ordered ranges, inner nodes from their children
__global__ void k_leaf_boxes(const double* X, int dim, Lists Ls, const int64_t* nlo, const int64_t* nhi, int64_t first,
                             int64_t cnt, double* bmin, double* bmax) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t h = first + t, lo = nlo[h], hi = nhi[h];
  for (int d = 0; d < dim; d++) {
    bmin[h * dim + d] = X[(int64_t)Ls.L[d][lo] * dim + d];
    bmax[h * dim + d] = X[(int64_t)Ls.L[d][hi - 1] * dim + d];
  }
}

__global__ void k_inner_boxes(int dim, int64_t first, int64_t cnt, double* bmin, double* bmax) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t h = first + t, a = 2 * h + 1, b = 2 * h + 2;
  for (int d = 0; d < dim; d++) {
    bmin[h * dim + d] = fmin(bmin[a * dim + d], bmin[b * dim + d]);
    bmax[h * dim + d] = fmax(bmax[a * dim + d], bmax[b * dim + d]);
  }
}

// first-kind Chebyshev nodes on each box side (cosines from the host); a side shorter than
// 1e-10 is widened to 1e-10 about its centre
__global__ void k_cheb(const double* bmin, const double* bmax, int dim, int p, const double* cosv, int64_t n_nodes,
                       double* cheb) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_nodes * dim * p) return;
  const int v = (int)(idx % p);
  const int64_t hd = idx / p;
  double a = bmin[hd], b = bmax[hd];
  if (__dsub_rn(b, a) < 1e-10) {
    const double c = __dmul_rn(0.5, __dadd_rn(a, b));
    a = __dsub_rn(c, 0.5e-10);
    b = __dadd_rn(c, 0.5e-10);
  }
  cheb[idx] = __dadd_rn(__dmul_rn(0.5, __dadd_rn(a, b)), __dmul_rn(__dmul_rn(0.5, __dsub_rn(b, a)), cosv[v]));
}

__global__ void k_diam(const double* bmin, const double* bmax, int dim, int64_t n_nodes, double* diam) {
  const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (h >= n_nodes) return;
  double s = 0.0;
  for (int d = 0; d < dim; d++) {
    const double t = __dsub_rn(bmax[h * dim + d], bmin[h * dim + d]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  diam[h] = sqrt(s);
}

__device__ __forceinline__ bool admissible(const double* bmin, const double* bmax, const double* diam, int dim,
                                           double eta, int64_t a, int64_t b) {
  double s = 0.0;
  for (int d = 0; d < dim; d++) {
    double gap = 0.0;
    const double t1 = __dsub_rn(bmin[b * dim + d], bmax[a * dim + d]);
    const double t2 = __dsub_rn(bmin[a * dim + d], bmax[b * dim + d]);
    if (t1 > gap) gap = t1;
    if (t2 > gap) gap = t2;
    s = __dadd_rn(s, __dmul_rn(gap, gap));
  }
  const double dist = sqrt(s);
  const double dm = diam[a] > diam[b] ? diam[a] : diam[b];
  return eta > 0.0 && dist > 0.0 && dm <= __dmul_rn(eta, dist);
}

// one level of the dual traversal: count (emit = 0) or write (emit = 1) the coupling blocks,
// dense blocks and child pairs of the frontier
__global__ void k_traverse(const int2* F, int64_t cnt, int level, int q, const double* bmin, const double* bmax,
                           const double* diam, int dim, double eta, unsigned long long* ctr, int emit, uint64_t* S_out,
                           uint64_t* D_out, int2* F_out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int2 pr = F[t];
  const int64_t i = pr.x, j = pr.y;
  int cls;
  if (admissible(bmin, bmax, diam, dim, eta, i, j)) cls = 0;
  else if (level == q) cls = 1;
  else cls = 2;
  const unsigned long long slot = atomicAdd(ctr + cls, 1ULL);
  if (!emit) return;
  if (cls == 0) {
    S_out[slot] = ((uint64_t)i << 32) | (uint64_t)j;
  } else if (cls == 1) {
    const int64_t first = ((int64_t)1 << q) - 1;
    D_out[slot] = ((uint64_t)(i - first) << 32) | (uint64_t)(j - first);
  } else {
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) F_out[4 * slot + 2 * a + b] = make_int2((int)(2 * i + 1 + a), (int)(2 * j + 1 + b));
  }
}

__global__ void k_fill_u64(uint64_t* a, int64_t from, int64_t to, uint64_t v) {
  const int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < to) a[i] = v;
}

// block-sparse rows from sorted (row << 32 | column) keys
__global__ void k_rowptr(const uint64_t* keys, int64_t cnt, int64_t rows, int32_t* rowptr) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r > rows) return;
  const uint64_t target = (uint64_t)r << 32;
  int64_t a = 0, b = cnt;
  while (a < b) {
    const int64_t mid = (a + b) / 2;
    if (keys[mid] < target) a = mid + 1;
    else b = mid;
  }
  rowptr[r] = (int32_t)a;
}

__global__ void k_colidx(const uint64_t* keys, int64_t cnt, int32_t* colidx) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < cnt) colidx[e] = (int32_t)(keys[e] & 0xffffffffu);
}

__global__ void k_dense_sizes(const uint64_t* keys, int64_t cnt, const int64_t* leaf_off, int64_t* sz) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= cnt) return;
  const int64_t i = (int64_t)(keys[e] >> 32), j = (int64_t)(keys[e] & 0xffffffffu);
  sz[e] = (leaf_off[i + 1] - leaf_off[i]) * (leaf_off[j + 1] - leaf_off[j]);
}

// ------------------------------------------------------------------------------------ values

// Lagrange polynomial a of the 1D node set xi (p nodes) at t
__device__ __forceinline__ double lagrange1(const double* xi, int p, int a, double t) {
  double v = 1.0;
  for (int b = 0; b < p; b++)
    if (b != a) v = __dmul_rn(v, __ddiv_rn(__dsub_rn(t, xi[b]), __dsub_rn(xi[a], xi[b])));
  return v;
}

// tensor Lagrange polynomial nu (dimension 0 slowest) of node h at x
__device__ __forceinline__ double lagrange_tensor(const double* cheb, int dim, int p, int64_t h, int nu, const double* x) {
  double v = 1.0;
  int rem = nu;
  for (int d = dim - 1; d >= 0; d--) {
    const int a = rem % p;
    rem /= p;
    v = __dmul_rn(v, lagrange1(cheb + (h * dim + d) * p, p, a, x[d]));
  }
  return v;
}

__device__ __forceinline__ void cheb_point(const double* cheb, int dim, int p, int64_t h, int nu, double* x) {
  int rem = nu;
  for (int d = dim - 1; d >= 0; d--) {
    const int a = rem % p;
    rem /= p;
    x[d] = cheb[(h * dim + d) * p + a];
  }
}

__device__ __forceinline__ double kernel_eval(int kind, double ell, int dim, const double* x, const double* y) {
  double r2 = 0.0;
  for (int d = 0; d < dim; d++) {
    const double t = __dsub_rn(x[d], y[d]);
    r2 = __dadd_rn(r2, __dmul_rn(t, t));
  }
  const double r = sqrt(r2);
  if (kind == H2_KERNEL_EXP) return exp(-__ddiv_rn(r, ell));
  const double s = __ddiv_rn(__dmul_rn(1.7320508075688772, r), ell);
  return __dmul_rn(__dadd_rn(1.0, s), exp(-s));
}

// leaf bases: U_i[a + s nu] = L^i_nu(x_a) (one thread per point and nu)
__global__ void k_values_u(const double* Xc, const double* cheb, const int64_t* leaf_off, int64_t leaves, int dim, int p,
                           int k, int64_t n, double* U) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * k) return;
  const int64_t pos = idx / k;
  const int nu = (int)(idx % k);
  int64_t a = 0, b = leaves - 1;
  while (a < b) {
    const int64_t mid = (a + b + 1) / 2;
    if (leaf_off[mid] <= pos) a = mid;
    else b = mid - 1;
  }
  const int64_t lo = leaf_off[a], s = leaf_off[a + 1] - lo;
  double x[3];
  for (int d = 0; d < dim; d++) x[d] = Xc[pos * dim + d];
  U[lo * k + (pos - lo) + s * nu] = lagrange_tensor(cheb, dim, p, leaves - 1 + a, nu, x);
}

// transfers: E_c[mu + k nu] = L^{parent}_nu(xi^c_mu)
__global__ void k_values_e(const double* cheb, int dim, int p, int k, int64_t n_nodes, double* E) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t kk = (int64_t)k * k;
  if (idx >= (n_nodes - 1) * kk) return;
  const int64_t c = 1 + idx / kk;
  const int w = (int)(idx % kk), mu = w % k, nu = w / k;
  double x[3];
  cheb_point(cheb, dim, p, c, mu, x);
  E[idx] = lagrange_tensor(cheb, dim, p, (c - 1) / 2, nu, x);
}

// coupling blocks: S_b[nu + k mu] = K(xi_row^nu, xi_col^mu)
__global__ void k_values_s(const uint64_t* keys, int64_t nS, const double* cheb, int dim, int p, int k, int kind,
                           double ell, double* S) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t kk = (int64_t)k * k;
  if (idx >= nS * kk) return;
  const int64_t b = idx / kk;
  const int w = (int)(idx % kk), nu = w % k, mu = w / k;
  const int64_t r = (int64_t)(keys[b] >> 32), c = (int64_t)(keys[b] & 0xffffffffu);
  double xi[3], xj[3];
  cheb_point(cheb, dim, p, r, nu, xi);
  cheb_point(cheb, dim, p, c, mu, xj);
  S[idx] = kernel_eval(kind, ell, dim, xi, xj);
}

// dense blocks: D_b[a + si c] = K(x_a, x_c), one CTA per block
__global__ void k_values_d(const uint64_t* keys, const int64_t* valoff, const int64_t* leaf_off, const double* Xc, int dim,
                           int kind, double ell, int64_t nD, double* D) {
  for (int64_t b = blockIdx.x; b < nD; b += gridDim.x) {
    const int64_t i = (int64_t)(keys[b] >> 32), j = (int64_t)(keys[b] & 0xffffffffu);
    const int64_t li = leaf_off[i], si = leaf_off[i + 1] - li, lj = leaf_off[j], sj = leaf_off[j + 1] - lj;
    double* Db = D + valoff[b];
    for (int64_t e = threadIdx.x; e < si * sj; e += blockDim.x) {
      const int64_t a = e % si, c = e / si;
      Db[e] = kernel_eval(kind, ell, dim, Xc + (li + a) * dim, Xc + (lj + c) * dim);
    }
  }
}

// ------------------------------------------------------------------------------------ host

template <typename T>
h2_status dalloc_b(h2_built_s* b, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, "cudaMalloc of %lld bytes: %s",
                (long long)(count * (int64_t)sizeof(T)), cudaGetErrorString(e));
  }
  b->allocs.push_back(v);
  b->dev_bytes += count * (int64_t)sizeof(T);
  *p = (T*)v;
  return H2_OK;
}

// scratch freed at the end of h2_build
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  h2_status get(T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, "cudaMalloc of %lld bytes: %s",
                  (long long)(count * (int64_t)sizeof(T)), cudaGetErrorString(e));
    }
    ptrs.push_back(v);
    *p = (T*)v;
    return H2_OK;
  }
  void drop(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFree(q);
        q = nullptr;
      }
  }
};

unsigned grid_of(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

void release_b(h2_built_s* b) {
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
}

h2_status build_tree(h2_built_s* B, Scratch& S, const std::vector<int64_t>& lo, const std::vector<int64_t>& hi,
                     int64_t* nlo, int64_t* nhi, cudaStream_t st) {
  const int dim = B->dim, q = B->q;
  const int64_t n = B->n, N = sort_size(n);
  h2_status s;
  DKey* keys = nullptr;
  if ((s = S.get(&keys, N)) != H2_OK) return s;
  Lists Ls{}, Lt{};
  for (int d = 0; d < dim; d++) {
    if ((s = S.get(&Ls.L[d], n)) != H2_OK) return s;
    if ((s = S.get(&Lt.L[d], n)) != H2_OK) return s;
    k_sort_init<<<grid_of(N), 256, 0, st>>>(B->X, dim, d, n, N, keys);
    bitonic_sort<DKey>(keys, N, st);
    k_sort_take<<<grid_of(n), 256, 0, st>>>(keys, n, Ls.L[d]);
  }
  S.drop(keys);
  int8_t* ds = nullptr;
  uint8_t* flag = nullptr;
  int32_t *f = nullptr, *sc = nullptr, *ws = nullptr;
  if ((s = S.get(&ds, B->n_nodes)) != H2_OK) return s;
  if ((s = S.get(&flag, n)) != H2_OK) return s;
  if ((s = S.get(&f, n)) != H2_OK) return s;
  if ((s = S.get(&sc, n)) != H2_OK) return s;
  if ((s = S.get(&ws, scan_ws(n))) != H2_OK) return s;
  CUDA_TRY(cudaMemsetAsync(ds, 0, (size_t)B->n_nodes, st));
  for (int l = 0; l < q; l++) {
    const int64_t first = ((int64_t)1 << l) - 1, cnt = (int64_t)1 << l;
    k_split_dim<<<grid_of(cnt), 256, 0, st>>>(B->X, dim, Ls, nlo, nhi, first, cnt, ds);
    k_flags<<<grid_of(n), 256, 0, st>>>(Ls, ds, nlo, nhi, first, cnt, n, flag);
    for (int d = 0; d < dim; d++) {
      k_gather_flags<<<grid_of(n), 256, 0, st>>>(Ls.L[d], flag, f, n);
      exclusive_scan<int32_t>(f, sc, n, ws, st);
      k_partition<<<grid_of(n), 256, 0, st>>>(Ls.L[d], f, sc, nlo, nhi, first, cnt, n, Lt.L[d]);
      std::swap(Ls.L[d], Lt.L[d]);
    }
  }
  const int64_t leaf0 = B->leaves - 1;
  k_perm<<<grid_of(n), 256, 0, st>>>(B->X, dim, Ls, ds, nlo, leaf0, B->leaves, q, n, B->perm, B->Xc);
  k_leaf_boxes<<<grid_of(B->leaves), 256, 0, st>>>(B->X, dim, Ls, nlo, nhi, leaf0, B->leaves, B->bmin, B->bmax);
  for (int l = q - 1; l >= 0; l--) {
    const int64_t first = ((int64_t)1 << l) - 1, cnt = (int64_t)1 << l;
    k_inner_boxes<<<grid_of(cnt), 256, 0, st>>>(dim, first, cnt, B->bmin, B->bmax);
  }
  std::vector<double> cosv((size_t)B->p);
  for (int v = 0; v < B->p; v++) cosv[v] = cos((2.0 * v + 1.0) * 3.141592653589793 / (2.0 * B->p));
  double* cos_d = nullptr;
  if ((s = S.get(&cos_d, B->p)) != H2_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(cos_d, cosv.data(), (size_t)B->p * sizeof(double), cudaMemcpyHostToDevice, st));
  k_cheb<<<grid_of(B->n_nodes * dim * B->p), 256, 0, st>>>(B->bmin, B->bmax, dim, B->p, cos_d, B->n_nodes, B->cheb);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(st));
  (void)lo;
  (void)hi;
  return H2_OK;
}

// sort keys (count of them) into a power-of-two buffer, padding with the largest key
h2_status sort_keys(Scratch& S, uint64_t* keys, int64_t cnt, uint64_t** sorted, cudaStream_t st) {
  const int64_t N = sort_size(cnt);
  h2_status s = S.get(sorted, N);
  if (s != H2_OK) return s;
  if (cnt > 0) CUDA_TRY(cudaMemcpyAsync(*sorted, keys, (size_t)cnt * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
  k_fill_u64<<<grid_of(N - cnt), 256, 0, st>>>(*sorted, cnt, N, ~0ULL);
  bitonic_sort<uint64_t>(*sorted, N, st);
  return H2_OK;
}

h2_status build_blocks(h2_built_s* B, Scratch& S, cudaStream_t st) {
  const int dim = B->dim, q = B->q;
  h2_status s;
  double* diam = nullptr;
  if ((s = S.get(&diam, B->n_nodes)) != H2_OK) return s;
  k_diam<<<grid_of(B->n_nodes), 256, 0, st>>>(B->bmin, B->bmax, dim, B->n_nodes, diam);
  unsigned long long* ctr = nullptr;
  if ((s = S.get(&ctr, 3)) != H2_OK) return s;
  std::vector<uint64_t*> s_parts, d_parts;
  std::vector<int64_t> s_cnt, d_cnt;
  int2* F = nullptr;
  if ((s = S.get(&F, 1)) != H2_OK) return s;
  const int2 root = make_int2(0, 0);
  CUDA_TRY(cudaMemcpyAsync(F, &root, sizeof(int2), cudaMemcpyHostToDevice, st));
  int64_t fcnt = 1;
  for (int l = 0; l <= q && fcnt > 0; l++) {
    unsigned long long c[3] = {0, 0, 0};
    CUDA_TRY(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), st));
    k_traverse<<<grid_of(fcnt), 256, 0, st>>>(F, fcnt, l, q, B->bmin, B->bmax, diam, dim, B->eta, ctr, 0, nullptr,
                                              nullptr, nullptr);
    CUDA_TRY(cudaMemcpyAsync(c, ctr, sizeof c, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    uint64_t *so = nullptr, *dout = nullptr;
    int2* Fn = nullptr;
    if ((s = S.get(&so, (int64_t)c[0])) != H2_OK) return s;
    if ((s = S.get(&dout, (int64_t)c[1])) != H2_OK) return s;
    if ((s = S.get(&Fn, 4 * (int64_t)c[2])) != H2_OK) return s;
    CUDA_TRY(cudaMemsetAsync(ctr, 0, 3 * sizeof(unsigned long long), st));
    k_traverse<<<grid_of(fcnt), 256, 0, st>>>(F, fcnt, l, q, B->bmin, B->bmax, diam, dim, B->eta, ctr, 1, so, dout, Fn);
    CUDA_TRY(cudaGetLastError());
    s_parts.push_back(so);
    s_cnt.push_back((int64_t)c[0]);
    d_parts.push_back(dout);
    d_cnt.push_back((int64_t)c[1]);
    S.drop(F);
    F = Fn;
    fcnt = 4 * (int64_t)c[2];
  }
  int64_t nS = 0, nD = 0;
  for (int64_t v : s_cnt) nS += v;
  for (int64_t v : d_cnt) nD += v;
  if (nS >= INT32_MAX || nD >= INT32_MAX) return fail(H2_ERR_UNSUPPORTED, "%lld coupling / %lld dense blocks: 2^31 or more", (long long)nS, (long long)nD);
  B->nS = nS;
  B->nD = nD;
  uint64_t *sall = nullptr, *dall = nullptr;
  if ((s = S.get(&sall, nS)) != H2_OK) return s;
  if ((s = S.get(&dall, nD)) != H2_OK) return s;
  int64_t o = 0;
  for (size_t t = 0; t < s_parts.size(); t++) {
    if (s_cnt[t]) CUDA_TRY(cudaMemcpyAsync(sall + o, s_parts[t], (size_t)s_cnt[t] * 8, cudaMemcpyDeviceToDevice, st));
    o += s_cnt[t];
  }
  o = 0;
  for (size_t t = 0; t < d_parts.size(); t++) {
    if (d_cnt[t]) CUDA_TRY(cudaMemcpyAsync(dall + o, d_parts[t], (size_t)d_cnt[t] * 8, cudaMemcpyDeviceToDevice, st));
    o += d_cnt[t];
  }
  uint64_t *ss = nullptr, *dsrt = nullptr;
  if ((s = sort_keys(S, sall, nS, &ss, st)) != H2_OK) return s;
  if ((s = sort_keys(S, dall, nD, &dsrt, st)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->S_keys, nS)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->D_keys, nD)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->S_rowptr, B->n_nodes + 1)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->S_colidx, nS)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->D_rowptr, B->leaves + 1)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->D_colidx, nD)) != H2_OK) return s;
  if ((s = dalloc_b(B, &B->D_valoff, nD + 1)) != H2_OK) return s;
  if (nS) CUDA_TRY(cudaMemcpyAsync(B->S_keys, ss, (size_t)nS * 8, cudaMemcpyDeviceToDevice, st));
  if (nD) CUDA_TRY(cudaMemcpyAsync(B->D_keys, dsrt, (size_t)nD * 8, cudaMemcpyDeviceToDevice, st));
  k_rowptr<<<grid_of(B->n_nodes + 1), 256, 0, st>>>(B->S_keys, nS, B->n_nodes, B->S_rowptr);
  k_colidx<<<grid_of(nS), 256, 0, st>>>(B->S_keys, nS, B->S_colidx);
  k_rowptr<<<grid_of(B->leaves + 1), 256, 0, st>>>(B->D_keys, nD, B->leaves, B->D_rowptr);
  k_colidx<<<grid_of(nD), 256, 0, st>>>(B->D_keys, nD, B->D_colidx);
  int64_t *sz = nullptr, *ws = nullptr;
  if ((s = S.get(&sz, nD + 1)) != H2_OK) return s;
  if ((s = S.get(&ws, scan_ws(nD + 1))) != H2_OK) return s;
  CUDA_TRY(cudaMemsetAsync(sz, 0, (size_t)(nD + 1) * sizeof(int64_t), st));
  k_dense_sizes<<<grid_of(nD), 256, 0, st>>>(B->D_keys, nD, B->leaf_off, sz);
  exclusive_scan<int64_t>(sz, B->D_valoff, nD + 1, ws, st);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(&B->nDval, B->D_valoff + nD, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return H2_OK;
}

h2_status build_values(h2_built_s* B, cudaStream_t st) {
  const int dim = B->dim, p = B->p, k = B->k;
  const int64_t kk = (int64_t)k * k;
  h2_status s;
  if (B->values & H2B_VALUES_U) {
    if ((s = dalloc_b(B, &B->U, B->n * k)) != H2_OK) return s;
    k_values_u<<<grid_of(B->n * k), 256, 0, st>>>(B->Xc, B->cheb, B->leaf_off, B->leaves, dim, p, k, B->n, B->U);
  }
  if (B->values & H2B_VALUES_E) {
    if ((s = dalloc_b(B, &B->E, (B->n_nodes - 1) * kk)) != H2_OK) return s;
    k_values_e<<<grid_of((B->n_nodes - 1) * kk), 256, 0, st>>>(B->cheb, dim, p, k, B->n_nodes, B->E);
  }
  if (B->values & H2B_VALUES_S) {
    if ((s = dalloc_b(B, &B->S_val, B->nS * kk)) != H2_OK) return s;
    k_values_s<<<grid_of(B->nS * kk), 256, 0, st>>>(B->S_keys, B->nS, B->cheb, dim, p, k, B->kernel, B->ell, B->S_val);
  }
  if (B->values & H2B_VALUES_D) {
    if ((s = dalloc_b(B, &B->D_val, B->nDval)) != H2_OK) return s;
    k_values_d<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(B->nD, 152 * 64)), 256, 0, st>>>(
        B->D_keys, B->D_valoff, B->leaf_off, B->Xc, dim, B->kernel, B->ell, B->nD, B->D_val);
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(st));
  return H2_OK;
}

}  // namespace

extern "C" {

h2_status h2_build(const h2_build_desc* bd, const double* points, h2_built* out) {
  if (!out) return fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!bd || !points) return fail(H2_ERR_INVALID, "desc or points is NULL");
  if (bd->dim < 1 || bd->dim > 3) return fail(H2_ERR_INVALID, "dim = %d outside 1..3", bd->dim);
  if (bd->m < 2 || bd->m > kMaxLeaf) return fail(H2_ERR_INVALID, "m = %d outside 2..%d", bd->m, kMaxLeaf);
  if (bd->p < 1 || bd->p > 16) return fail(H2_ERR_INVALID, "p = %d outside 1..16", bd->p);
  int k = 1;
  for (int d = 0; d < bd->dim; d++) k *= bd->p;
  if (k > kMaxRank) return fail(H2_ERR_UNSUPPORTED, "rank p^dim = %d > %d", k, kMaxRank);
  if (bd->n < 1 || bd->n >= ((int64_t)1 << 31)) return fail(H2_ERR_INVALID, "n = %lld outside 1 .. 2^31 - 1", (long long)bd->n);
  if (bd->kernel != H2_KERNEL_EXP && bd->kernel != H2_KERNEL_MATERN32) return fail(H2_ERR_INVALID, "kernel %d", bd->kernel);
  if (!(bd->ell > 0.0) || !std::isfinite(bd->ell)) return fail(H2_ERR_INVALID, "ell = %g", bd->ell);
  if (!(bd->eta >= 0.0) || !std::isfinite(bd->eta)) return fail(H2_ERR_INVALID, "eta = %g", bd->eta);
  if (bd->values & ~0xF) return fail(H2_ERR_INVALID, "values = %d: a mask of H2B_VALUES_*", bd->values);
  for (int64_t i = 0; i < bd->n * bd->dim; i++)
    if (!std::isfinite(points[i])) return fail(H2_ERR_INVALID, "points[%lld] is not finite", (long long)i);
  h2_built_s* B = new (std::nothrow) h2_built_s();
  if (!B) return fail(H2_ERR_OOM, "host allocation failed");
  cudaGetDevice(&B->dev);
  B->dim = bd->dim;
  B->m = bd->m;
  B->p = bd->p;
  B->k = k;
  B->kernel = bd->kernel;
  B->values = bd->values;
  B->eta = bd->eta;
  B->ell = bd->ell;
  B->n = bd->n;
  int q = 0;
  while (((int64_t)bd->m << q) < bd->n) q++;
  B->q = q;
  B->leaves = (int64_t)1 << q;
  B->n_nodes = ((int64_t)2 << q) - 1;
  // node ranges follow from n alone: the left child of a node of s points gets ceil(s/2)
  std::vector<int64_t> lo((size_t)B->n_nodes), hi((size_t)B->n_nodes), leaf_off((size_t)B->leaves + 1);
  lo[0] = 0;
  hi[0] = B->n;
  for (int64_t h = 0; h < B->leaves - 1; h++) {
    const int64_t mid = lo[h] + (hi[h] - lo[h] + 1) / 2;
    lo[2 * h + 1] = lo[h];
    hi[2 * h + 1] = mid;
    lo[2 * h + 2] = mid;
    hi[2 * h + 2] = hi[h];
  }
  for (int64_t i = 0; i < B->leaves; i++) leaf_off[i] = lo[B->leaves - 1 + i];
  leaf_off[B->leaves] = B->n;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[4] = {};
  auto run = [&]() -> h2_status {
    h2_status s;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ev) CUDA_TRY(cudaEventCreate(&e));
    Scratch S;
    int64_t *nlo = nullptr, *nhi = nullptr;
    if ((s = S.get(&nlo, B->n_nodes)) != H2_OK) return s;
    if ((s = S.get(&nhi, B->n_nodes)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->X, B->n * B->dim)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->Xc, B->n * B->dim)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->perm, B->n)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->leaf_off, B->leaves + 1)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->bmin, B->n_nodes * B->dim)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->bmax, B->n_nodes * B->dim)) != H2_OK) return s;
    if ((s = dalloc_b(B, &B->cheb, B->n_nodes * B->dim * B->p)) != H2_OK) return s;
    CUDA_TRY(cudaMemcpyAsync(nlo, lo.data(), (size_t)B->n_nodes * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(nhi, hi.data(), (size_t)B->n_nodes * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(B->leaf_off, leaf_off.data(), (size_t)(B->leaves + 1) * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(B->X, points, (size_t)(B->n * B->dim) * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaEventRecord(ev[0], st));
    if ((s = build_tree(B, S, lo, hi, nlo, nhi, st)) != H2_OK) return s;
    CUDA_TRY(cudaEventRecord(ev[1], st));
    if ((s = build_blocks(B, S, st)) != H2_OK) return s;
    CUDA_TRY(cudaEventRecord(ev[2], st));
    if ((s = build_values(B, st)) != H2_OK) return s;
    CUDA_TRY(cudaEventRecord(ev[3], st));
    CUDA_TRY(cudaEventSynchronize(ev[3]));
    for (int t = 0; t < 3; t++) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, ev[t], ev[t + 1]));
      B->ms[t] = ms;
    }
    return H2_OK;
  };
  h2_status s = run();
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  if (st) cudaStreamDestroy(st);
  if (s != H2_OK) {
    release_b(B);
    delete B;
    return s;
  }
  *out = B;
  return H2_OK;
}

h2_status h2_built_info(h2_built b, int64_t info[8]) {
  if (!b || !info) return fail(H2_ERR_INVALID, "NULL argument");
  info[0] = b->q;
  info[1] = b->k;
  info[2] = b->nS;
  info[3] = b->nD;
  info[4] = b->nDval;
  info[5] = b->n_nodes;
  info[6] = b->leaves;
  info[7] = b->dev_bytes;
  return H2_OK;
}

h2_status h2_built_times(h2_built b, double ms[3]) {
  if (!b || !ms) return fail(H2_ERR_INVALID, "NULL argument");
  for (int t = 0; t < 3; t++) ms[t] = b->ms[t];
  return H2_OK;
}

h2_status h2_built_read(h2_built b, int32_t what, void* dst, int64_t count) {
  if (!b) return fail(H2_ERR_INVALID, "built matrix is NULL");
  if (!dst && count > 0) return fail(H2_ERR_INVALID, "dst is NULL");
  const int64_t kk = (int64_t)b->k * b->k;
  const void* src = nullptr;
  int64_t need = 0, size = 8;
  switch (what) {
    case H2B_PERM: src = b->perm; need = b->n; break;
    case H2B_LEAF_OFFSET: src = b->leaf_off; need = b->leaves + 1; break;
    case H2B_POINTS: src = b->Xc; need = b->n * b->dim; break;
    case H2B_CHEB: src = b->cheb; need = b->n_nodes * b->dim * b->p; break;
    case H2B_S_ROWPTR: src = b->S_rowptr; need = b->n_nodes + 1; size = 4; break;
    case H2B_S_COLIDX: src = b->S_colidx; need = b->nS; size = 4; break;
    case H2B_D_ROWPTR: src = b->D_rowptr; need = b->leaves + 1; size = 4; break;
    case H2B_D_COLIDX: src = b->D_colidx; need = b->nD; size = 4; break;
    case H2B_D_VALOFF: src = b->D_valoff; need = b->nD + 1; break;
    case H2B_U: src = b->U; need = b->n * b->k; break;
    case H2B_E: src = b->E; need = (b->n_nodes - 1) * kk; break;
    case H2B_S: src = b->S_val; need = b->nS * kk; break;
    case H2B_D: src = b->D_val; need = b->nDval; break;
    default: return fail(H2_ERR_INVALID, "unknown array %d", what);
  }
  if (what >= H2B_U && !src) return fail(H2_ERR_INVALID, "array %d was not built (see h2_build_desc.values)", what);
  if (count != need) return fail(H2_ERR_INVALID, "array %d holds %lld values, count is %lld", what, (long long)need, (long long)count);
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->dev) return fail(H2_ERR_INVALID, "built matrix lives on device %d, current device is %d", b->dev, cur);
  if (need > 0) CUDA_TRY(cudaMemcpy(dst, src, (size_t)(need * size), cudaMemcpyDeviceToHost));
  return H2_OK;
}

h2_status h2_create_built(h2_built b, int32_t storage, int32_t bases_fp32, int32_t flags, h2_handle* out) {
  if (!out) return fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!b) return fail(H2_ERR_INVALID, "built matrix is NULL");
  if (flags & ~(H2B_CREATE_KERNEL_COUPLING | H2B_CREATE_GENERATED_DENSE)) return fail(H2_ERR_INVALID, "flags = %d", flags);
  const bool kc_mode = (flags & H2B_CREATE_KERNEL_COUPLING) != 0, gen = (flags & H2B_CREATE_GENERATED_DENSE) != 0;
  if (gen && !kc_mode) return fail(H2_ERR_INVALID, "generated dense blocks need kernel-evaluated coupling blocks");
  if (!b->U || !b->E) return fail(H2_ERR_INVALID, "the built matrix has no U or E values (H2B_VALUES_U | H2B_VALUES_E)");
  if (!kc_mode && !b->S_val) return fail(H2_ERR_INVALID, "stored coupling blocks need H2B_VALUES_S");
  if (!gen && !b->D_val) return fail(H2_ERR_INVALID, "stored dense blocks need H2B_VALUES_D");
  const int64_t kk = (int64_t)b->k * b->k;
  // the description in host memory (the library's create path validates and lays it out)
  std::vector<int64_t> leaf_off((size_t)b->leaves + 1);
  std::vector<int32_t> srp((size_t)b->n_nodes + 1), sci((size_t)std::max<int64_t>(b->nS, 1)), drp((size_t)b->leaves + 1),
      dci((size_t)std::max<int64_t>(b->nD, 1));
  std::vector<double> U((size_t)(b->n * b->k)), E((size_t)std::max<int64_t>((b->n_nodes - 1) * kk, 1)), S, D, pts, cheb;
  h2_status s;
  if ((s = h2_built_read(b, H2B_LEAF_OFFSET, leaf_off.data(), b->leaves + 1)) != H2_OK) return s;
  if ((s = h2_built_read(b, H2B_S_ROWPTR, srp.data(), b->n_nodes + 1)) != H2_OK) return s;
  if ((s = h2_built_read(b, H2B_S_COLIDX, sci.data(), b->nS)) != H2_OK) return s;
  if ((s = h2_built_read(b, H2B_D_ROWPTR, drp.data(), b->leaves + 1)) != H2_OK) return s;
  if ((s = h2_built_read(b, H2B_D_COLIDX, dci.data(), b->nD)) != H2_OK) return s;
  if ((s = h2_built_read(b, H2B_U, U.data(), b->n * b->k)) != H2_OK) return s;
  if ((s = h2_built_read(b, H2B_E, E.data(), (b->n_nodes - 1) * kk)) != H2_OK) return s;
  if (!kc_mode) {
    S.resize((size_t)std::max<int64_t>(b->nS * kk, 1));
    if ((s = h2_built_read(b, H2B_S, S.data(), b->nS * kk)) != H2_OK) return s;
  }
  if (!gen) {
    D.resize((size_t)std::max<int64_t>(b->nDval, 1));
    if ((s = h2_built_read(b, H2B_D, D.data(), b->nDval)) != H2_OK) return s;
  } else {
    pts.resize((size_t)(b->n * b->dim));
    if ((s = h2_built_read(b, H2B_POINTS, pts.data(), b->n * b->dim)) != H2_OK) return s;
  }
  if (kc_mode) {
    cheb.resize((size_t)(b->n_nodes * b->dim * b->p));
    if ((s = h2_built_read(b, H2B_CHEB, cheb.data(), b->n_nodes * b->dim * b->p)) != H2_OK) return s;
  }
  h2_desc d{};
  d.n = b->n;
  d.depth = b->q;
  d.rank = b->k;
  d.symmetric = 1;
  d.storage = storage;
  d.leaf_offset = leaf_off.data();
  d.U = U.data();
  d.E = E.data();
  d.S_rowptr = srp.data();
  d.S_colidx = sci.data();
  d.S_val = kc_mode ? nullptr : S.data();
  d.D_rowptr = drp.data();
  d.D_colidx = dci.data();
  d.D_val = gen ? nullptr : D.data();
  d.bases_fp32 = bases_fp32;
  if (!kc_mode) return h2_create(&d, out);
  h2_coupling_kernel kc{};
  kc.kernel = b->kernel;
  kc.dim = b->dim;
  kc.p = b->p;
  kc.ell = b->ell;
  kc.cheb = cheb.data();
  return gen ? h2_create_generated(&d, &kc, pts.data(), out) : h2_create_kernel_coupling(&d, &kc, out);
}

h2_status h2_built_destroy(h2_built b) {
  if (!b) return H2_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->dev) cudaSetDevice(b->dev);
  release_b(b);
  if (cur != b->dev) cudaSetDevice(cur);
  delete b;
  return H2_OK;
}

}  // extern "C"
