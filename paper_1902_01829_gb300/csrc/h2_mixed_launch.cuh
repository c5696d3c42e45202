// Launch sequence of one precision-form product pass (up to kPassVectors
// vectors per matrix) for storage format F, over a table of matrices: one
// handle, or a batch. Each h2_mixed_<format>.cu instantiates it once, so the
// three formats compile in parallel.
#pragma once
#include <algorithm>
#include "h2_internal.h"
#include "mixed.cuh"
#include "tc_dense.cuh"

namespace h2i {

template <int F, int NVB, int CW>
cudaError_t set_mixed_smem() {
  static cudaError_t done = cudaErrorNotReady;
  if (done == cudaErrorNotReady)
    done = cudaFuncSetAttribute(h2::k_dense_stream_m<F, NVB, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                h2::mixed_smem_bytes(NVB, CW));
  return done;
}

// Kernels that run beside the dense stream prefer its L1 / shared memory split (the largest shared
// part): an SM holds CTAs of one configuration at a time.
template <class K>
void prefer_max_shared(K kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// the tree and coupling launches of one vector-count bucket (phase 0: upsweep, 1: coupling, 2: downsweep)
// convert: the upsweep's leaf projection writes the FP32 copy of x (no split kernel ran);
// expand: the downsweep ends with the leaf expansion: 0 none (the tensor-core pass fuses it),
// 1 added to y (zeroed; the dense phase adds beside it), 2 assigned (the dense phase adds after)
template <int F, int FB, int RPL, int NVB>
void bucket_phase(const MixedLaunch& L, int phase, int nvlo, cudaStream_t st, bool convert, int expand) {
  using namespace h2;
  static const bool carveout = [] {
    constexpr int NVW = NVB < 4 ? NVB : 4, VG = NVB / NVW;
    prefer_max_shared(k_upsweep_tree_m<FB, RPL, NVB>);
    prefer_max_shared(k_downsweep_tree_m<FB, RPL, NVB>);
    prefer_max_shared(k_coupling_kf<RPL, NVB, 0>);
    prefer_max_shared(k_coupling_kf<RPL, NVB, 1>);
    prefer_max_shared(k_coupling_m<F, 16, NVW, (NVW <= 2 ? 4 : 2), VG>);
    prefer_max_shared(k_coupling_m<F, 32, NVW, (NVW <= 1 ? 2 : 1), VG>);
    prefer_max_shared(k_coupling_m<F, 64, NVW, (NVW <= 1 ? 2 : 1), VG>);
    prefer_max_shared(k_coupling_m_generic<F, RPL, NVB>);
    return true;
  }();
  (void)carveout;
  const MatDesc* mats = static_cast<const MatDesc*>(L.mats);
  const unsigned tree_threads = kTreeWarpsM * 32;
  if (phase == 0 && L.njobs > 0) {
    k_upsweep_tree_m<FB, RPL, NVB><<<(unsigned)L.njobs, tree_threads, 0, st>>>(mats, L.jobs, nvlo, NVB, convert ? 1 : 0);
  } else if (phase == 1 && L.nchunks > 0) {
    const unsigned cgrid = (unsigned)((L.nchunks + 3) / 4);
    const int k = L.k;
    if (L.kf) {  // coupling blocks evaluated from the kernel
      if (L.kf_kind == 1) k_coupling_kf<RPL, NVB, 1><<<cgrid, 128, 0, st>>>(mats, L.chunks, L.nchunks, nvlo, NVB);
      else k_coupling_kf<RPL, NVB, 0><<<cgrid, 128, 0, st>>>(mats, L.chunks, L.nchunks, nvlo, NVB);
    } else if (k == 16 || k == 32 || k == 64) {
      // up to four vectors per warp; 8 and 16 vectors take two and four warps per chunk
      constexpr int NVW = NVB < 4 ? NVB : 4, VG = NVB / NVW;
      const unsigned grid = (unsigned)((L.nchunks * VG + 3) / 4);
      if (k == 16) {
        constexpr int CB = NVW <= 2 ? 4 : 2;
        k_coupling_m<F, 16, NVW, CB, VG><<<grid, 128, 0, st>>>(mats, L.chunks, L.nchunks, nvlo, NVB);
      } else if (k == 32) {
        constexpr int CB = NVW <= 1 ? 2 : 1;
        k_coupling_m<F, 32, NVW, CB, VG><<<grid, 128, 0, st>>>(mats, L.chunks, L.nchunks, nvlo, NVB);
      } else {
        constexpr int CB = NVW <= 1 ? 2 : 1;
        k_coupling_m<F, 64, NVW, CB, VG><<<grid, 128, 0, st>>>(mats, L.chunks, L.nchunks, nvlo, NVB);
      }
    } else {
      k_coupling_m_generic<F, RPL, NVB><<<cgrid, 128, 0, st>>>(mats, L.chunks, L.nchunks, nvlo, NVB);
    }
  } else if (phase == 2 && L.njobs > 0) {
    k_downsweep_tree_m<FB, RPL, NVB><<<(unsigned)L.njobs, tree_threads, 0, st>>>(mats, L.jobs, nvlo, NVB, expand);
  }
}

template <int F, int FB, int RPL>
void bucket_dispatch(const MixedLaunch& L, int phase, int b, cudaStream_t st, bool convert, int expand) {
  switch (b) {
    case 0: return bucket_phase<F, FB, RPL, 1>(L, phase, kBucketLo[0], st, convert, expand);
    case 1: return bucket_phase<F, FB, RPL, 2>(L, phase, kBucketLo[1], st, convert, expand);
    case 2: return bucket_phase<F, FB, RPL, 4>(L, phase, kBucketLo[2], st, convert, expand);
    case 3: return bucket_phase<F, FB, RPL, 8>(L, phase, kBucketLo[3], st, convert, expand);
    default: return bucket_phase<F, FB, RPL, 16>(L, phase, kBucketLo[4], st, convert, expand);
  }
}

template <int F, int NVB, int CW>
h2_status dense_launch_cw(const MixedLaunch& L, cudaStream_t st) {
  using namespace h2;
  cudaError_t e = set_mixed_smem<F, NVB, CW>();
  if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  MixedStreamParams P{};
  P.items = L.items;
  P.cta_begin = L.cta_begin;
  P.blk = static_cast<const MixedBlock*>(L.blk);
  P.mats = static_cast<const MatDesc*>(L.mats);
  P.err = L.err;
  P.budget = L.budget;
  k_dense_stream_m<F, NVB, CW><<<L.grid, (CW + 1) * 32, mixed_smem_bytes(NVB, CW), st>>>(P);
  return H2_OK;
}

// consumer warps of the dense stream: rows of at most 32 points give each warp little
// arithmetic per item, and twice the warps hide more latency (measured: 163 -> 134 us on a
// 2^17-point matrix with 32-point leaves); 64-point rows run faster with 8. With 16 vectors
// per pass the 16-warp variant fits 96 registers a thread (a few spilled).
template <int F, int NVB>
h2_status dense_launch(const MixedLaunch& L, cudaStream_t st) {
  if (L.cw == 2 * h2::kMixedCW) return dense_launch_cw<F, NVB, 2 * h2::kMixedCW>(L, st);
  return dense_launch_cw<F, NVB, h2::kMixedCW>(L, st);
}

// a phase on the tensor cores (the dense phase, or the coupling phase): per-vector scales, then the
// persistent tcgen05 kernel
template <int F>
h2_status tc_launch(const TcCall& T, cudaStream_t st) {
  using namespace h2;
  if constexpr (F == kFormInt16) {
    return h2_fail(H2_ERR_UNSUPPORTED, "internal: tensor-core path for int16 codes");
  } else {
    static cudaError_t attr = cudaErrorNotReady;
    if (attr == cudaErrorNotReady)
      attr = cudaFuncSetAttribute(k_dense_tc<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (attr != cudaSuccess) return h2_fail(H2_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(attr));
    if (!T.items || !T.cta_begin || !T.brec || !T.dmat || !T.vmax || !T.vscale || !T.y || T.nv < 1 || T.nv > kTcVec ||
        (T.coupling ? !T.xhat : (!T.x4 || !T.yhat || !T.xp4_off)))
      return h2_fail(H2_ERR_INVALID, "internal: tensor-core phase without its buffers");
    const bool fp16 = F == kFormFp16;
    if (fp16) {
      cudaError_t e = cudaMemsetAsync(T.vmax, 0, kTcVec * sizeof(unsigned), st);
      if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
      // 32 warps per SM (152 SMs), each over a stride of leaves (nodes) for one vector
      const long long units = T.coupling ? T.nodes : T.leaves;
      const long long warps = (long long)T.nv * std::max<long long>(1, std::min<long long>(units, 152 * 32 / T.nv));
      if (T.coupling)
        k_tc_vmax_nodes<F><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(T.xhat, T.nodes, T.nv, T.kp, T.k,
                                                                             T.smax, warps, T.vmax);
      else
        k_tc_vmax<F><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
            T.x4, T.yhat, reinterpret_cast<const long long*>(T.xp4_off), T.leaves, T.leaf0, T.nv, T.kp, T.k, T.dmax,
            T.umax, warps, T.vmax);
    }
    k_tc_vscale<F><<<1, 32, 0, st>>>(T.vmax, T.vscale, fp16 ? 1 : 0);
    if (T.coupling) {  // rows without coupling blocks hold zeros; the others are assigned
      cudaError_t e = cudaMemsetAsync(T.y, 0, (size_t)(T.nodes * T.nv * T.kp) * sizeof(float), st);
      if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    TcParams P{};
    P.items = T.items;
    P.cta_begin = T.cta_begin;
    P.blk = static_cast<const MixedBlock*>(T.blk);
    P.dmat = static_cast<const char*>(T.dmat);
    P.x4 = T.x4;
    P.yhat = T.coupling ? T.xhat : T.yhat;  // the builders' second vector source
    P.vscale = T.vscale;
    P.brec = T.brec;
    P.y = T.y;
    P.ldy = T.ldy;
    P.rowmul = T.coupling ? (long long)T.nv * T.kp : 1;
    P.nv = T.nv;
    P.y32 = T.y32;
    P.kp = T.kp;
    P.ppad = T.coupling ? 0 : kPanelPad;
    P.err = T.err;
    P.budget = T.budget;
    k_dense_tc<F><<<T.grid, kTcThreads, kTcSmem, st>>>(P);
    return H2_OK;
  }
}

// The phase launches; the caller has written the product's fields into the matrix table and
// recorded the first profiling mark. On the CUDA cores the dense phase streams the D blocks only
// and adds its row sums into y; the downsweep ends with the leaf expansion U_i yhat_i. Passes of
// up to four vectors (not profiled) run the dense phase on the caller's stream while the tree
// phases (upsweep, coupling, downsweep) run on L.side: k_split_x4 first copies x to FP32 and
// zeroes y, and both sides add into y. Other passes run the phases in order: the leaf projection
// copies x itself, the expansion assigns y and the dense phase adds after it. The tensor-core
// pass fuses the expansion into its dense phase.
template <int F, int FB, int RPL>
h2_status mixed_pass_t(const MixedLaunch& L, unsigned buckets, cudaStream_t st, const TcPass* tp) {
  const TcCall* tc = tp ? tp->dense : nullptr;      // dense phase and expansion on the tensor cores
  const TcCall* tcs = tp ? tp->coupling : nullptr;  // coupling phase on the tensor cores
  cudaError_t me = cudaSuccess;
  auto mk = [&]() {
    if (L.prof && me == cudaSuccess) me = mark(L.prof, st);
  };
  const int top = 31 - __builtin_clz(buckets | 1u);
  auto dense = [&](cudaStream_t ds) -> h2_status {
    return tc         ? tc_launch<F>(*tc, ds)
           : top == 0 ? dense_launch<F, 1>(L, ds)
           : top == 1 ? dense_launch<F, 2>(L, ds)
           : top == 2 ? dense_launch<F, 4>(L, ds)
           : top == 3 ? dense_launch<F, 8>(L, ds)
                      : dense_launch<F, 16>(L, ds);
  };
  // passes of more than four vectors keep the phases in order: their tree kernels' shared memory does
  // not fit beside the dense stream's, and the dense phase is bound by arithmetic there (measured)
  const bool overlap = !tc && !tcs && top <= 2 && !(L.prof && L.prof->on) && L.side && L.ev_fork && L.ev_join;
  h2_status s = H2_OK;
  if (overlap) {
    const long long swarps = std::min<long long>(L.nrjobs, (long long)L.grid * 64);
    h2::k_split_x4<F><<<(unsigned)((swarps + 7) / 8), 256, 0, st>>>(static_cast<const h2::MatDesc*>(L.mats),
                                                                static_cast<const h2::RowJob*>(L.rjobs), L.nrjobs, 1);
    cudaError_t e = cudaEventRecord(L.ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.side, L.ev_fork, 0);
    if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "fork to the side stream: %s", cudaGetErrorString(e));
    if ((s = dense(st)) != H2_OK) return s;
    for (int phase = 0; phase < 3; phase++)
      for (int b = 0; b < kBuckets; b++)
        if ((buckets >> b) & 1u) bucket_dispatch<F, FB, RPL>(L, phase, b, L.side, false, 1);
    e = cudaEventRecord(L.ev_join, L.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, L.ev_join, 0);
    if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "join from the side stream: %s", cudaGetErrorString(e));
  } else {
    for (int phase = 0; phase < 3; phase++) {
      if (phase == 1 && tcs) {
        if ((s = tc_launch<F>(*tcs, st)) != H2_OK) return s;
      } else {
        for (int b = 0; b < kBuckets; b++)
          if ((buckets >> b) & 1u) bucket_dispatch<F, FB, RPL>(L, phase, b, st, true, tc ? 0 : 2);
      }
      mk();
    }
    if ((s = dense(st)) != H2_OK) return s;
  }
  mk();
  if (me != cudaSuccess) return h2_fail(H2_ERR_CUDA, "profiling event: %s", cudaGetErrorString(me));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h2_fail(H2_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return H2_OK;
}

// FB: format of the bases and transfers (the storage format, or FP32 entries)
template <int F>
h2_status mixed_pass_form(const MixedLaunch& L, unsigned buckets, cudaStream_t st, const TcPass* tc) {
  if (L.bases_fp32)
    return L.k > 32 ? mixed_pass_t<F, h2::kFormF32, 2>(L, buckets, st, tc)
                    : mixed_pass_t<F, h2::kFormF32, 1>(L, buckets, st, tc);
  return L.k > 32 ? mixed_pass_t<F, F, 2>(L, buckets, st, tc) : mixed_pass_t<F, F, 1>(L, buckets, st, tc);
}

}  // namespace h2i
