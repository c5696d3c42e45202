// h2_matvec_static: the H^2 product without any allocation.
//
// Some callers cannot allocate device memory: code running inside a host
// framework that owns all device memory through its own allocator (and
// forbids cudaMalloc behind its back), or code on a latency-critical path
// where cudaMalloc / cudaFree may synchronize the device. This entry point
// serves them. The caller passes the matrix, x and y in its own device memory;
// the only working memory is the file-scope array below, which every GPU that
// loads the library holds until the process exits.
//
// It is one kernel launched as a single CTA: the product's phases run in
// order inside it, separated by __syncthreads, in native FP64 arithmetic
// (any finite FP64 values). It is written for correctness and small
// matrices, not speed. Before it touches the scratch it checks the structure
// arrays it indexes with (leaf offsets, block row pointers, column indices,
// the dense block count); a malformed description sets a sticky error word
// in the scratch, leaves y untouched, and h2_matvec_static_check reports it.
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "h2.h"

// shared with h2_last_error (defined in h2_api.cu)
void h2_internal_set_error(const char* msg);

namespace {

// 16 MiB of scratch: a control block, the xhat and yhat vector trees and the dense-block offsets.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
constexpr size_t kControlBytes = 256;                     // [0]: error word (sticky until checked)
constexpr int64_t kStaticMaxDenseBlocks = (int64_t)1 << 20;
constexpr int kStaticMaxRank = 64, kStaticMaxLeaf = 64;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kStaticWarps = 32;
constexpr int kMaxDevices = 64;

std::atomic<void*> g_scratch_ptr[kMaxDevices];  // device address of g_static_scratch, per device (null until looked up)

h2_status fail_static(h2_status st, const char* msg) {
  h2_internal_set_error(msg);
  return st;
}

// warp-wide sum; every lane gets the total
__device__ __forceinline__ double warp_sum(double s) {
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
  return s;
}

struct StaticArgs {
  int64_t n, n_dense_blocks;
  int q, k, nv, symmetric;
  const int64_t* leaf_offset;
  const double *U, *V, *E, *F;
  const int32_t *S_rowptr, *S_colidx;
  const double* S_val;
  const int32_t *D_rowptr, *D_colidx;
  const double* D_val;
  const double* x;
  int64_t ldx;
  double* y;
  int64_t ldy;
  int* err;       // scratch: sticky error word
  double* xhat;   // scratch: [node][v][k]
  double* yhat;   // scratch: [node][v][k]
  int64_t* doff;  // scratch: dense block offsets [n_dense_blocks + 1]
};

// level of heap node h
__device__ __forceinline__ int node_level(int64_t h) { return 63 - __clzll(h + 1); }

// The structure arrays the kernel indexes with must describe a tree of depth q
// over n points, leaf sizes 1..64, block rows with non-decreasing pointers
// that start at 0, coupling columns on the row's level, dense columns among
// the leaves and exactly n_dense_blocks dense blocks.
__device__ bool structure_ok(const StaticArgs& a, int* bad) {
  const int64_t leaves = (int64_t)1 << a.q, n_nodes = ((int64_t)2 << a.q) - 1;
  if (threadIdx.x == 0) {
    if (a.leaf_offset[0] != 0 || a.leaf_offset[leaves] != a.n || a.D_rowptr[0] != 0 ||
        a.D_rowptr[leaves] != a.n_dense_blocks || a.S_rowptr[0] != 0)
      *bad = 1;
  }
  for (int64_t i = threadIdx.x; i < leaves; i += blockDim.x) {
    const int64_t s = a.leaf_offset[i + 1] - a.leaf_offset[i];
    if (s < 1 || s > kStaticMaxLeaf || a.D_rowptr[i + 1] < a.D_rowptr[i]) *bad = 1;
  }
  for (int64_t r = threadIdx.x; r < n_nodes; r += blockDim.x)
    if (a.S_rowptr[r + 1] < a.S_rowptr[r]) *bad = 1;
  __syncthreads();
  if (*bad) return false;
  for (int64_t r = threadIdx.x; r < n_nodes; r += blockDim.x) {
    const int l = node_level(r);
    const int64_t first = ((int64_t)1 << l) - 1, last = ((int64_t)2 << l) - 2;
    for (int32_t b = a.S_rowptr[r]; b < a.S_rowptr[r + 1]; b++)
      if (a.S_colidx[b] < first || a.S_colidx[b] > last) *bad = 1;
  }
  for (int64_t b = threadIdx.x; b < a.n_dense_blocks; b += blockDim.x)
    if (a.D_colidx[b] < 0 || a.D_colidx[b] >= leaves) *bad = 1;
  __syncthreads();
  return *bad == 0;
}

// One CTA computes y = A^H x: leaf projection and upsweep (Eq. 2), coupling
// (Eq. 3), downsweep (Eq. 5), leaf expansion (Eq. 4) and the dense blocks.
// Every dot product is spread over a warp's lanes and reduced with shuffles.
__global__ void __launch_bounds__(kStaticWarps * 32) k_matvec_static(StaticArgs a) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (!structure_ok(a, &bad)) {
    if (threadIdx.x == 0) atomicExch(a.err, 1);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = a.k, nv = a.nv;
  const int64_t leaves = (int64_t)1 << a.q, n_nodes = ((int64_t)2 << a.q) - 1, leaf0 = leaves - 1;
  const double* V = a.symmetric ? a.U : a.V;
  const double* F = a.symmetric ? a.E : a.F;

  // dense block offsets (serial prefix sum by thread 0; n_dense_blocks = D_rowptr[2^q] was checked)
  if (threadIdx.x == 0) {
    int64_t off = 0;
    for (int64_t i = 0; i < leaves; i++)
      for (int32_t b = a.D_rowptr[i]; b < a.D_rowptr[i + 1]; b++) {
        a.doff[b] = off;
        const int32_t j = a.D_colidx[b];
        off += (a.leaf_offset[i + 1] - a.leaf_offset[i]) * (a.leaf_offset[j + 1] - a.leaf_offset[j]);
      }
  }
  // leaf projection: xhat_j[nu] = sum_a V_j[a, nu] x(j)[a]
  for (int64_t j = warp; j < leaves; j += kStaticWarps) {
    const int64_t off = a.leaf_offset[j], sj = a.leaf_offset[j + 1] - off;
    for (int v = 0; v < nv; v++)
      for (int nu = 0; nu < k; nu++) {
        double s = 0.0;
        for (int64_t r = lane; r < sj; r += 32) s = fma(V[off * k + r + sj * nu], a.x[v * a.ldx + off + r], s);
        s = warp_sum(s);
        if (lane == 0) a.xhat[((leaf0 + j) * nv + v) * k + nu] = s;
      }
  }
  __syncthreads();
  // upsweep: xhat_p[nu] = sum_c sum_mu F_c[mu, nu] xhat_c[mu]
  for (int l = a.q; l >= 1; l--) {
    const int64_t pfirst = ((int64_t)1 << (l - 1)) - 1, pcount = (int64_t)1 << (l - 1);
    for (int64_t t = warp; t < pcount; t += kStaticWarps) {
      const int64_t p = pfirst + t;
      for (int v = 0; v < nv; v++)
        for (int nu = 0; nu < k; nu++) {
          double s = 0.0;
          for (int ci = 1; ci <= 2; ci++) {
            const int64_t ch = 2 * p + ci;
            for (int mu = lane; mu < k; mu += 32)
              s = fma(F[(ch - 1) * k * k + mu + (int64_t)k * nu], a.xhat[(ch * nv + v) * k + mu], s);
          }
          s = warp_sum(s);
          if (lane == 0) a.xhat[(p * nv + v) * k + nu] = s;
        }
    }
    __syncthreads();
  }
  // coupling: yhat_i[nu] = sum_b sum_mu S_b[nu, mu] xhat_col(b)[mu]  (every node row is written)
  for (int64_t i = warp; i < n_nodes; i += kStaticWarps)
    for (int v = 0; v < nv; v++)
      for (int nu = 0; nu < k; nu++) {
        double s = 0.0;
        for (int32_t b = a.S_rowptr[i]; b < a.S_rowptr[i + 1]; b++) {
          const int64_t col = a.S_colidx[b];
          for (int mu = lane; mu < k; mu += 32)
            s = fma(a.S_val[(int64_t)b * k * k + nu + (int64_t)k * mu], a.xhat[(col * nv + v) * k + mu], s);
        }
        s = warp_sum(s);
        if (lane == 0) a.yhat[(i * nv + v) * k + nu] = s;
      }
  __syncthreads();
  // downsweep: yhat_c[mu] += sum_nu E_c[mu, nu] yhat_parent[nu]
  for (int l = 1; l <= a.q; l++) {
    const int64_t cfirst = ((int64_t)1 << l) - 1, ccount = (int64_t)1 << l;
    for (int64_t t = warp; t < ccount; t += kStaticWarps) {
      const int64_t ch = cfirst + t, par = (ch - 1) / 2;
      for (int v = 0; v < nv; v++)
        for (int mu = 0; mu < k; mu++) {
          double s = 0.0;
          for (int nu = lane; nu < k; nu += 32)
            s = fma(a.E[(ch - 1) * k * k + mu + (int64_t)k * nu], a.yhat[(par * nv + v) * k + nu], s);
          s = warp_sum(s);
          if (lane == 0) a.yhat[(ch * nv + v) * k + mu] += s;
        }
    }
    __syncthreads();
  }
  // leaf expansion and dense blocks: y(i)[r] = sum_nu U_i[r, nu] yhat_i[nu] + sum_b sum_c D_b[r, c] x(j)[c]
  for (int64_t i = warp; i < leaves; i += kStaticWarps) {
    const int64_t off = a.leaf_offset[i], si = a.leaf_offset[i + 1] - off;
    for (int v = 0; v < nv; v++)
      for (int64_t r = 0; r < si; r++) {
        double s = 0.0;
        for (int nu = lane; nu < k; nu += 32) s = fma(a.U[off * k + r + si * nu], a.yhat[((leaf0 + i) * nv + v) * k + nu], s);
        for (int32_t b = a.D_rowptr[i]; b < a.D_rowptr[i + 1]; b++) {
          const int32_t j = a.D_colidx[b];
          const int64_t offj = a.leaf_offset[j], sj = a.leaf_offset[j + 1] - offj;
          for (int64_t cc = lane; cc < sj; cc += 32) s = fma(a.D_val[a.doff[b] + r + si * cc], a.x[v * a.ldx + offj + cc], s);
        }
        s = warp_sum(s);
        if (lane == 0) a.y[v * a.ldy + off + r] = s;
      }
  }
}

// device address of the scratch on the current device (looked up once per device)
h2_status scratch_base(unsigned char** base) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_static(H2_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) {
    char msg[128];
    snprintf(msg, sizeof msg, "device %d: the allocation-free entry points support devices 0..%d", dev, kMaxDevices - 1);
    return fail_static(H2_ERR_UNSUPPORTED, msg);
  }
  void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!p) {  // once per device, with that device current; concurrent first calls store the same address
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail_static(H2_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    }
    g_scratch_ptr[dev].store(p, std::memory_order_release);
  }
  *base = (unsigned char*)p;
  return H2_OK;
}

}  // namespace

extern "C" {

h2_status h2_matvec_static(const h2_desc* d, int64_t n_dense_blocks, int32_t nv, const double* x, int64_t ldx, double* y,
                           int64_t ldy, void* stream) {
  h2_internal_set_error("");
  if (!d || !x || !y) return fail_static(H2_ERR_INVALID, "NULL desc or vector");
  if (nv < 1 || d->n < 1 || d->rank < 1 || d->depth < 0 || d->depth > 24 || n_dense_blocks < 0)
    return fail_static(H2_ERR_INVALID, "invalid size (nv, n, rank, depth or dense block count)");
  if (d->rank > kStaticMaxRank) return fail_static(H2_ERR_UNSUPPORTED, "rank above 64");
  if (n_dense_blocks > kStaticMaxDenseBlocks) return fail_static(H2_ERR_UNSUPPORTED, "more than 2^20 dense blocks");
  if (ldx < d->n || ldy < d->n) return fail_static(H2_ERR_INVALID, "leading dimension below n");
  if (d->storage != H2_FP64) return fail_static(H2_ERR_UNSUPPORTED, "only FP64 storage");
  if (!d->leaf_offset || !d->U || !d->E || !d->S_rowptr || !d->D_rowptr || (!d->symmetric && (!d->V || !d->F)) ||
      (n_dense_blocks > 0 && (!d->D_colidx || !d->D_val)))
    return fail_static(H2_ERR_INVALID, "NULL array in desc");
  // scratch need, one factor at a time so nothing overflows: control + 2 trees + offsets
  const int64_t n_nodes = ((int64_t)2 << d->depth) - 1;
  const int64_t per_vector = n_nodes * d->rank * (int64_t)sizeof(double);  // <= 2^25 * 64 * 8
  const int64_t room = (int64_t)kStaticScratchBytes - (int64_t)kControlBytes - (n_dense_blocks + 1) * (int64_t)sizeof(int64_t);
  if (room < 0 || (int64_t)nv > room / (2 * per_vector))
    return fail_static(H2_ERR_UNSUPPORTED,
                       "the product needs more scratch than the static 16 MiB: "
                       "256 + 2 * (2^(q+1) - 1) * nv * k * 8 + (dense blocks + 1) * 8 bytes must fit");
  const int64_t tree = per_vector * nv;
  unsigned char* base = nullptr;
  h2_status st = scratch_base(&base);
  if (st != H2_OK) return st;
  StaticArgs a;
  std::memset(&a, 0, sizeof a);
  a.n = d->n;
  a.n_dense_blocks = n_dense_blocks;
  a.q = d->depth;
  a.k = d->rank;
  a.nv = nv;
  a.symmetric = d->symmetric;
  a.leaf_offset = d->leaf_offset;
  a.U = d->U;
  a.V = d->V;
  a.E = d->E;
  a.F = d->F;
  a.S_rowptr = d->S_rowptr;
  a.S_colidx = d->S_colidx;
  a.S_val = d->S_val;
  a.D_rowptr = d->D_rowptr;
  a.D_colidx = d->D_colidx;
  a.D_val = d->D_val;
  a.x = x;
  a.ldx = ldx;
  a.y = y;
  a.ldy = ldy;
  a.err = (int*)base;
  a.xhat = (double*)(base + kControlBytes);
  a.yhat = (double*)(base + kControlBytes + tree);
  a.doff = (int64_t*)(base + kControlBytes + 2 * tree);
  k_matvec_static<<<1, kStaticWarps * 32, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_static(H2_ERR_CUDA, "kernel launch failed");
  return H2_OK;
}

h2_status h2_matvec_static_check(void* stream) {
  h2_internal_set_error("");
  unsigned char* base = nullptr;
  h2_status st = scratch_base(&base);
  if (st != H2_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  if (cudaMemcpyAsync(&err, base, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return fail_static(H2_ERR_CUDA, "reading the error word of the static product failed");
  }
  if (err) {
    if (cudaMemsetAsync(base, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return fail_static(H2_ERR_CUDA, "clearing the error word of the static product failed");
    }
    return fail_static(H2_ERR_INVALID,
                       "a static product since the last check found a malformed description (leaf offsets, block "
                       "row pointers, column indices or the dense block count); its y was left untouched");
  }
  return H2_OK;
}

}  // extern "C"
