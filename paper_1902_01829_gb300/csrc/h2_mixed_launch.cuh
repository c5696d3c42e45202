// Launch sequence of one precision-form product pass (up to kPassVectors
// vectors) for storage format F. Each h2_mixed_<format>.cu instantiates it
// once, so the three formats compile in parallel.
#pragma once
#include "h2_internal.h"
#include "mixed.cuh"

namespace h2i {

template <int F, int NVB>
cudaError_t set_mixed_smem() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaErrorNotReady)
    done = cudaFuncSetAttribute(h2::k_dense_stream_m<F, NVB, h2::kMixedCW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                h2::mixed_smem_bytes(NVB, h2::kMixedCW));
  return done;
}

template <int F, int FB, int RPL, int NVB>
h2_status mixed_pass_t(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  using namespace h2;
  MixedData& M = h->mx;
  cudaError_t e = set_mixed_smem<F, NVB>();
  if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  TreeParamsM T{};
  T.Vt = M.Vt;
  T.vscale = M.vscale;
  T.vt_off = M.vt_off;
  T.Ft = M.Ft;
  T.fscale = M.fscale;
  T.E = M.E;
  T.escale = M.escale;
  T.leaf_off = h->leaf_off;
  T.xp4_off = M.xp4_off;
  T.x = x;
  T.ldx = ldx;
  T.x4 = M.x4;
  T.xhat = M.xhat;
  T.yhat = M.yhat;
  T.ticket = h->ticket;
  T.kk8 = M.kk8;
  T.k = h->k;
  T.kp = M.kp4;
  T.LR = h->lr;
  T.q = h->q;
  T.L = h->tree_L;
  T.nv = nv;
  const unsigned tree_grid = 1u << h->tree_L, tree_threads = kTreeWarpsM * 32;
  const unsigned cgrid = (unsigned)((h->n_nodes + 3) / 4);
  const int k = h->k;
  cudaError_t me = mark(h, st);
  k_upsweep_tree_m<FB, RPL, NVB><<<tree_grid, tree_threads, 0, st>>>(T);
  if (me == cudaSuccess) me = mark(h, st);
  if (k >= 4 && k <= 64 && (k & (k - 1)) == 0) {
    constexpr int CB = NVB <= 2 ? 8 : (NVB <= 4 ? 4 : 2);
    k_coupling_m<F, NVB, CB><<<cgrid, 128, 0, st>>>(M.smat, M.sscale, M.kk8, h->Srow, h->Scol, k, M.kp4, h->n_nodes, nv,
                                                     M.xhat, M.yhat);
  } else {
    k_coupling_m_generic<F, RPL, NVB><<<cgrid, 128, 0, st>>>(M.smat, M.sscale, M.kk8, h->Srow, h->Scol, k, M.kp4, h->lr,
                                                              h->n_nodes, nv, M.xhat, M.yhat);
  }
  if (me == cudaSuccess) me = mark(h, st);
  k_downsweep_tree_m<FB, RPL, NVB><<<tree_grid, tree_threads, 0, st>>>(T);
  if (me == cudaSuccess) me = mark(h, st);
  MixedStreamParams P{};
  P.items = M.dense_items.items;
  P.cta_begin = M.dense_items.cta_begin;
  P.mat = reinterpret_cast<const char*>(M.dmat);
  P.blk = reinterpret_cast<const MixedBlock*>(M.dblk);
  P.vsrc0 = M.x4;
  P.vsrc1 = M.yhat;
  P.nv = nv;
  P.y = y;
  P.ldy = ldy;
  P.err = h->err;
  P.budget = h->budget;
  k_dense_stream_m<F, NVB, kMixedCW><<<h->grid, (kMixedCW + 1) * 32, mixed_smem_bytes(NVB, kMixedCW), st>>>(P);
  if (me == cudaSuccess) me = mark(h, st);
  h->launches += 4;
  if (me != cudaSuccess) return h2_fail(H2_ERR_CUDA, "profiling event: %s", cudaGetErrorString(me));
  e = cudaGetLastError();
  if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return H2_OK;
}

template <int F, int FB, int RPL>
h2_status mixed_pass_nv(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  if (nv <= 1) return mixed_pass_t<F, FB, RPL, 1>(h, nv, x, ldx, y, ldy, st);
  if (nv <= 2) return mixed_pass_t<F, FB, RPL, 2>(h, nv, x, ldx, y, ldy, st);
  if (nv <= 4) return mixed_pass_t<F, FB, RPL, 4>(h, nv, x, ldx, y, ldy, st);
  if (nv <= 8) return mixed_pass_t<F, FB, RPL, 8>(h, nv, x, ldx, y, ldy, st);
  return mixed_pass_t<F, FB, RPL, 16>(h, nv, x, ldx, y, ldy, st);
}

// FB: format of the bases and transfers (the storage format, or FP32 entries)
template <int F, int FB>
h2_status mixed_pass_fb(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  return h->k > 32 ? mixed_pass_nv<F, FB, 2>(h, nv, x, ldx, y, ldy, st) : mixed_pass_nv<F, FB, 1>(h, nv, x, ldx, y, ldy, st);
}

template <int F>
h2_status mixed_pass_form(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  return h->mx.bases_fp32 ? mixed_pass_fb<F, h2::kFormF32>(h, nv, x, ldx, y, ldy, st)
                          : mixed_pass_fb<F, F>(h, nv, x, ldx, y, ldy, st);
}

}  // namespace h2i
