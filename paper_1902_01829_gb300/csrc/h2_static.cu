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
// order inside it, separated by __syncthreads. It is written for correctness
// and small matrices, not speed.
#include <cstdint>
#include <cstring>

#include "df64.cuh"
#include "h2.h"

// shared with h2_last_error (defined in h2_api.cu)
void h2_internal_set_error(const char* msg);

namespace {

// 16 MiB of scratch: the xhat and yhat vector trees and the dense-block offsets.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kStaticWarps = 32;
constexpr int kMaxDevices = 64;

void* g_scratch_ptr[kMaxDevices] = {nullptr};  // device address of g_static_scratch, per device

h2_status fail_static(h2_status st, const char* msg) {
  h2_internal_set_error(msg);
  return st;
}

// (s, c) += a * x for a double-float x (xh, xl) and an FP64 matrix entry a
__device__ __forceinline__ void acc(float& s, float& c, double a, float2 x) {
  float ah, al;
  h2::split_f64(a, ah, al);
  h2::df_fma(s, c, ah, al, x.x, x.y);
}

// warp-wide sum of a double-float value; every lane gets the total
__device__ __forceinline__ void warp_sum(float& s, float& c) {
  for (int off = 16; off > 0; off >>= 1) {
    const float s2 = __shfl_xor_sync(0xFFFFFFFFu, s, off);
    const float c2 = __shfl_xor_sync(0xFFFFFFFFu, c, off);
    h2::df_add(s, c, s2, c2);
  }
}

struct StaticArgs {
  int64_t n;
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
  float2* xhat;  // scratch: [node][v][k]
  float2* yhat;  // scratch: [node][v][k]
  int64_t* doff; // scratch: dense block offsets
};

// One CTA computes y = A^H x: leaf projection and upsweep (Eq. 2), coupling
// (Eq. 3), downsweep (Eq. 5), leaf expansion (Eq. 4) and the dense blocks.
// Every dot product is spread over a warp's lanes and reduced with shuffles.
__global__ void __launch_bounds__(kStaticWarps * 32) k_matvec_static(StaticArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = a.k, nv = a.nv;
  const int64_t leaves = (int64_t)1 << a.q, n_nodes = ((int64_t)2 << a.q) - 1, leaf0 = leaves - 1;
  const double* V = a.symmetric ? a.U : a.V;
  const double* F = a.symmetric ? a.E : a.F;

  // dense block offsets (serial prefix sum by thread 0; the sizes are small by construction)
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
        float s = 0.f, c = 0.f;
        for (int64_t r = lane; r < sj; r += 32) acc(s, c, V[off * k + r + sj * nu], h2::f64_to_df(a.x[v * a.ldx + off + r]));
        warp_sum(s, c);
        if (lane == 0) a.xhat[((leaf0 + j) * nv + v) * k + nu] = h2::df_norm(s, c);
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
          float s = 0.f, c = 0.f;
          for (int ci = 1; ci <= 2; ci++) {
            const int64_t ch = 2 * p + ci;
            for (int mu = lane; mu < k; mu += 32)
              acc(s, c, F[(ch - 1) * k * k + mu + (int64_t)k * nu], a.xhat[(ch * nv + v) * k + mu]);
          }
          warp_sum(s, c);
          if (lane == 0) a.xhat[(p * nv + v) * k + nu] = h2::df_norm(s, c);
        }
    }
    __syncthreads();
  }
  // coupling: yhat_i[nu] = sum_b sum_mu S_b[nu, mu] xhat_col(b)[mu]  (every node row is written)
  for (int64_t i = warp; i < n_nodes; i += kStaticWarps)
    for (int v = 0; v < nv; v++)
      for (int nu = 0; nu < k; nu++) {
        float s = 0.f, c = 0.f;
        for (int32_t b = a.S_rowptr[i]; b < a.S_rowptr[i + 1]; b++) {
          const int64_t col = a.S_colidx[b];
          for (int mu = lane; mu < k; mu += 32)
            acc(s, c, a.S_val[(int64_t)b * k * k + nu + (int64_t)k * mu], a.xhat[(col * nv + v) * k + mu]);
        }
        warp_sum(s, c);
        if (lane == 0) a.yhat[(i * nv + v) * k + nu] = h2::df_norm(s, c);
      }
  __syncthreads();
  // downsweep: yhat_c[mu] += sum_nu E_c[mu, nu] yhat_parent[nu]
  for (int l = 1; l <= a.q; l++) {
    const int64_t cfirst = ((int64_t)1 << l) - 1, ccount = (int64_t)1 << l;
    for (int64_t t = warp; t < ccount; t += kStaticWarps) {
      const int64_t ch = cfirst + t, par = (ch - 1) / 2;
      for (int v = 0; v < nv; v++)
        for (int mu = 0; mu < k; mu++) {
          float s = 0.f, c = 0.f;
          for (int nu = lane; nu < k; nu += 32)
            acc(s, c, a.E[(ch - 1) * k * k + mu + (int64_t)k * nu], a.yhat[(par * nv + v) * k + nu]);
          warp_sum(s, c);
          if (lane == 0) {
            const float2 old = a.yhat[(ch * nv + v) * k + mu];
            h2::df_add(s, c, old.x, old.y);
            a.yhat[(ch * nv + v) * k + mu] = h2::df_norm(s, c);
          }
        }
    }
    __syncthreads();
  }
  // leaf expansion and dense blocks: y(i)[r] = sum_nu U_i[r, nu] yhat_i[nu] + sum_b sum_c D_b[r, c] x(j)[c]
  for (int64_t i = warp; i < leaves; i += kStaticWarps) {
    const int64_t off = a.leaf_offset[i], si = a.leaf_offset[i + 1] - off;
    for (int v = 0; v < nv; v++)
      for (int64_t r = 0; r < si; r++) {
        float s = 0.f, c = 0.f;
        for (int nu = lane; nu < k; nu += 32)
          acc(s, c, a.U[off * k + r + si * nu], a.yhat[((leaf0 + i) * nv + v) * k + nu]);
        for (int32_t b = a.D_rowptr[i]; b < a.D_rowptr[i + 1]; b++) {
          const int32_t j = a.D_colidx[b];
          const int64_t offj = a.leaf_offset[j], sj = a.leaf_offset[j + 1] - offj;
          for (int64_t cc = lane; cc < sj; cc += 32)
            acc(s, c, a.D_val[a.doff[b] + r + si * cc], h2::f64_to_df(a.x[v * a.ldx + offj + cc]));
        }
        warp_sum(s, c);
        if (lane == 0) a.y[v * a.ldy + off + r] = h2::df_to_f64(s, c);
      }
  }
}

}  // namespace

extern "C" {

h2_status h2_matvec_static(const h2_desc* d, int64_t n_dense_blocks, int32_t nv, const double* x, int64_t ldx, double* y,
                           int64_t ldy, void* stream) {
  h2_internal_set_error("");
  if (!d || !x || !y) return fail_static(H2_ERR_INVALID, "NULL desc or vector");
  if (nv < 1 || d->n < 1 || d->rank < 1 || d->depth < 0 || d->depth > 24 || n_dense_blocks < 0)
    return fail_static(H2_ERR_INVALID, "invalid size (nv, n, rank, depth or dense block count)");
  if (ldx < d->n || ldy < d->n) return fail_static(H2_ERR_INVALID, "leading dimension below n");
  if (d->storage != H2_FP64) return fail_static(H2_ERR_UNSUPPORTED, "only FP64 storage");
  if (!d->leaf_offset || !d->U || !d->E || !d->S_rowptr || !d->D_rowptr || (!d->symmetric && (!d->V || !d->F)))
    return fail_static(H2_ERR_INVALID, "NULL array in desc");
  const int64_t n_nodes = ((int64_t)2 << d->depth) - 1;
  const int64_t tree = n_nodes * nv * d->rank * (int64_t)sizeof(float2);
  const int64_t need = 2 * tree + (n_dense_blocks + 1) * (int64_t)sizeof(int64_t);
  if (need > (int64_t)kStaticScratchBytes)
    return fail_static(H2_ERR_UNSUPPORTED,
                       "the product needs more scratch than the static 16 MiB: "
                       "2 * (2^(q+1) - 1) * nv * k * 8 + (dense blocks + 1) * 8 bytes must fit");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail_static(H2_ERR_CUDA, "cudaGetDevice failed");
  if (!g_scratch_ptr[dev]) {  // once per device, with that device current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail_static(H2_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    }
    g_scratch_ptr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_scratch_ptr[dev];
  StaticArgs a;
  std::memset(&a, 0, sizeof a);
  a.n = d->n;
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
  a.xhat = (float2*)base;
  a.yhat = (float2*)(base + tree);
  a.doff = (int64_t*)(base + 2 * tree);
  k_matvec_static<<<1, kStaticWarps * 32, 0, (cudaStream_t)stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_static(H2_ERR_CUDA, "kernel launch failed");
  return H2_OK;
}

}  // extern "C"
