// Precision form of the H^2 matrix-vector product: every block of U, V, E, F,
// S and D is stored as 16-bit codes with one FP32 scale per block, and all
// products accumulate in FP32 (a block's partial sum is multiplied by its
// scale once). Codes convert to FP32 exactly:
//   fp16   IEEE binary16 bits
//   bf16   bfloat16 bits (the top half of an FP32)
//   int16  offset binary: code = q + 32768, q in [-32767, 32767]
// The phases are those of the FP64 form (hmv_fp64.cuh, stream_fp64.cuh):
// fused leaf projection + upsweep (Eq. 2), coupling over all levels (Eq. 3),
// fused downsweep (Eq. 5), and the TMA-streamed dense blocks fused with the
// leaf expansion (Sec. 2.2, Eq. 4). Vectors x, xhat, yhat are FP32 with
// strides rounded up to multiples of 4 (16-byte chunks for the bulk copies).
#pragma once
#include <type_traits>
#include <cuda_fp16.h>

#include "stream_fp64.cuh"
#include "tma.cuh"

namespace h2 {

// kFormF32: plain FP32 entries (the bases and transfers when they are kept in FP32)
enum { kFormFp16 = 0, kFormBf16 = 1, kFormInt16 = 2, kFormF32 = 3 };

template <int F>
struct CodeT {
  using T = uint16_t;
};
template <>
struct CodeT<kFormF32> {
  using T = float;
};

template <int F>
__device__ __forceinline__ float code_to_f(typename CodeT<F>::T c) {
  if constexpr (F == kFormF32) {
    return c;
  } else {
    const uint32_t u = c;
    if (F == kFormFp16) return __half2float(__ushort_as_half((unsigned short)u));
    if (F == kFormBf16) return __uint_as_float(u << 16);
    return __uint_as_float(0x4B000000u | u) - 8421376.0f;  // 2^23 + 32768
  }
}

// two codes packed in a word (low half first)
template <int F>
__device__ __forceinline__ float2 codes_to_f2(uint32_t w) {
  if (F == kFormFp16) {
    __half2 h = *reinterpret_cast<const __half2*>(&w);
    return __half22float2(h);
  }
  if (F == kFormBf16) return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
  // offset-binary int16 c: the float with bits 0x4B00 : c is 2^23 + c; one byte permute each
  return make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7410)) - 8421376.0f,
                     __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7432)) - 8421376.0f);
}

// Per leaf row of a matrix: where U_i is and its block record (the leaf
// expansion at the end of the downsweep and the split of x use them)
struct __align__(16) RowJob {
  long long uoff;  // byte offset of U_i in the matrix's dmat
  int mat;         // matrix index in the table
  int leaf;        // leaf index j (heap node 2^q - 1 + j)
  int ublk;        // block record of U_i (scale, layout)
  int has_dense;   // the dense phase adds a part of this row (it has dense blocks)
  int pad[2];
};
struct __align__(16) MixedBlock {
  long long voff;       // vector chunk offset, in floats per vector slot
  float scale;
  unsigned short cols;  // C
  unsigned char vs;     // vector stride (>= C, multiple of 4)
  unsigned char src;    // bit 0: vector from the second source (yhat); bit 1: FP32 entries (not codes);
                        // bit 2: panel layout (below)
};

// Panel layout of a block of codes (64 rows, C columns): eight panels of 8 rows,
// panel p holding column c's rows 8p .. 8p + 7 as 16 contiguous bytes at c * 16,
// the panels kPanelPad bytes apart beyond their 16 * Cp bytes (Cp = C rounded up
// to 16, padding columns zero). It is the MN-major operand layout of tcgen05.mma
// (8 x 8 core matrices: K stride 128 bytes, M stride the panel stride), and the
// pad staggers the panels over the shared-memory banks for the CUDA-core reader.
constexpr int kPanelPad = 16;
__host__ __device__ constexpr int panel_cols(int C) { return (C + 15) & ~15; }
__host__ __device__ constexpr int panel_stride(int C) { return 16 * panel_cols(C) + kPanelPad; }  // bytes
__host__ __device__ constexpr int panel_block_bytes(int C) { return 8 * panel_stride(C); }

// ---------------------------------------------------------------- per-matrix descriptor
// One entry per matrix of a batch (a single product is a batch of one); the
// kernels of every phase find their matrix through it. The last group of
// fields changes with every product.
struct MatDesc {
  const char* dmat;      // dense stream: per leaf row its blocks then U_i
  const uint16_t* smat;  // coupling blocks (kk8 codes each)
  const float* sscale;
  const int32_t* Srow;
  const int32_t* Scol;
  const void* Vt;        // bases and transfers (codes, or FP32 entries)
  const float* vscale;
  const int64_t* vt_off;
  const void* Ft;
  const float* fscale;
  const void* E;
  const float* escale;
  const int64_t* leaf_off;
  const int64_t* xp4_off;
  float* x4;             // workspace: FP32 x, xhat, yhat
  float* xhat;
  float* yhat;
  int* ticket;
  long long kk8, n_nodes;
  int k, kp, LR, q, L;
  int spanel;            // k = 64: coupling codes in the panel layout (8 panels of 8 rows, 1024 bytes apart)
  // coupling blocks from the kernel (k_coupling_kf): node centres as FP32 high and low parts,
  // the interpolation points' offsets from the centre, 1 / ell and the kernel kind
  const float4* kf_chi;
  const float4* kf_clo;
  const float4* kf_off;
  float kf_inv_ell;
  int kf_kind;
  // the leaf expansion done by the downsweep: the matrix's row jobs and the block records they index
  const RowJob* rjobs;
  const MixedBlock* blk;
  // per product
  const double* x;
  long long ldx;
  double* y;
  long long ldy;
  int nv, xy32;   // xy32: x and y are FP32 (else FP64)
};

// x and y are FP64 or, for products that ask for it, FP32 (MatDesc::xy32)
__device__ __forceinline__ float x_load(const double* x, bool x32, long long idx) {
  return x32 ? __ldg(reinterpret_cast<const float*>(x) + idx) : __double2float_rn(__ldg(x + idx));
}
__device__ __forceinline__ void y_store(void* y, bool y32, long long idx, float v, bool assign) {
  if (y32) {
    float* p = reinterpret_cast<float*>(y) + idx;
    if (assign) *p = v;
    else atomicAdd(p, v);
  } else {
    double* p = reinterpret_cast<double*>(y) + idx;
    if (assign) *p = (double)v;
    else atomicAdd(p, (double)v);
  }
}

// ---------------------------------------------------------------- generic warp routine
// rows += scale * (A * x_cols) for a column-major R x C block of codes; lane
// = g * LR + rl owns rows rl + 32 r, column groups g take columns g, g + G, ...
template <int F, int RPL, int NVB>
__device__ __forceinline__ void warp_mv_m(const typename CodeT<F>::T* __restrict__ A, float scale, int R, int C, int LR,
                                          const float* xin, int64_t xstride, int nv, float (&acc)[RPL][NVB], int lane) {
  constexpr int UB = (NVB <= 2) ? 8 : (NVB <= 4 ? 4 : 2);
  const int G = 32 / LR;
  const int g = lane / LR, rl = lane - g * LR;
  float p[RPL][NVB];
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) p[r][v] = 0.f;
  for (int col0 = g; col0 < C; col0 += UB * G) {
    float a[UB][RPL], xv[UB][NVB];
#pragma unroll
    for (int u = 0; u < UB; u++) {
      const int col = col0 + u * G;
#pragma unroll
      for (int r = 0; r < RPL; r++) {
        const int row = rl + 32 * r;
        a[u][r] = (col < C && row < R) ? code_to_f<F>(__ldg(A + row + (int64_t)R * col)) : 0.f;
      }
#pragma unroll
      for (int v = 0; v < NVB; v++) xv[u][v] = (col < C && v < nv) ? xin[v * xstride + col] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < UB; u++)
#pragma unroll
      for (int r = 0; r < RPL; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) p[r][v] = fmaf(a[u][r], xv[u][v], p[r][v]);
  }
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = fmaf(scale, p[r][v], acc[r][v]);
}

template <int RPL, int NVB>
__device__ __forceinline__ void group_reduce_m(float (&acc)[RPL][NVB], int LR) {
  for (int off = LR; off < 32; off <<= 1)
#pragma unroll
    for (int r = 0; r < RPL; r++)
#pragma unroll
      for (int v = 0; v < NVB; v++) acc[r][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[r][v], off);
}

template <int RPL, int NVB, bool ACCUM>
__device__ __forceinline__ void store_node_m(float* dst, int k, int kp, int LR, int nv, float (&acc)[RPL][NVB], int lane) {
  if (lane >= LR) return;
#pragma unroll
  for (int r = 0; r < RPL; r++) {
    const int row = lane + 32 * r;
    if (row >= k) continue;
#pragma unroll
    for (int v = 0; v < NVB; v++) {
      if (v >= nv) continue;
      dst[v * kp + row] = ACCUM ? dst[v * kp + row] + acc[r][v] : acc[r][v];
    }
  }
}

// ---------------------------------------------------------------- tree phases
// Vt, Ft, E hold codes of the bases' format FB (16-bit codes, or FP32 entries)
struct TreeParamsM {
  const void* Vt;         // leaf j: k x size_j entries at vt_off[j]
  const float* vscale;
  const int64_t* vt_off;
  const void* Ft;         // node h >= 1 at (h - 1) * kk8
  const float* fscale;
  const void* E;
  const float* escale;
  const int64_t* leaf_off;
  const int64_t* xp4_off;
  const double* x;
  int64_t ldx;
  float* x4;
  float* xhat;
  float* yhat;
  int* ticket;
  int64_t kk8;
  int k, kp, LR, q, L, nv, xy32;
};

constexpr int kTreeWarpsM = 8;

__device__ __forceinline__ TreeParamsM tree_params(const MatDesc& D) {
  TreeParamsM P;
  P.Vt = D.Vt;
  P.vscale = D.vscale;
  P.vt_off = D.vt_off;
  P.Ft = D.Ft;
  P.fscale = D.fscale;
  P.E = D.E;
  P.escale = D.escale;
  P.leaf_off = D.leaf_off;
  P.xp4_off = D.xp4_off;
  P.x = D.x;
  P.ldx = D.ldx;
  P.x4 = D.x4;
  P.xhat = D.xhat;
  P.yhat = D.yhat;
  P.ticket = D.ticket;
  P.kk8 = D.kk8;
  P.k = D.k;
  P.kp = D.kp;
  P.LR = D.LR;
  P.q = D.q;
  P.L = D.L;
  P.nv = D.nv;
  P.xy32 = D.xy32;
  return P;
}

// copy n floats (n a multiple of 4, both ends 16-byte aligned) into the warp's staging buffer;
// CG: read through L2 (the data was written by another CTA)
template <bool CG>
__device__ __forceinline__ void stage_vectors(float* __restrict__ dst, const float* __restrict__ src, int n, int lane) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int i = lane; i < n / 4; i += 32) d4[i] = CG ? __ldcg(s4 + i) : s4[i];
  __syncwarp();
}

// Each warp stages the vector block it multiplies (a leaf's x chunk, a child's xhat, a
// parent's yhat: nv x up to 64 floats) in its own shared-memory buffer wbuf, so that
// warp_mv_m's many reads of it are shared-memory reads.
// convert: x(j) is read in FP64 and its FP32 copy written to x4 here (products whose phases run
// in order); else k_split_x4 wrote x4 before the launch
template <int F, int RPL, int NVB>
__device__ __forceinline__ void project_leaf_m(const TreeParamsM& P, int64_t j, int lane, float* wbuf, bool convert) {
  const int64_t leaf0 = ((int64_t)1 << P.q) - 1;
  const int64_t off = P.leaf_off[j];
  const int sj = (int)(P.leaf_off[j + 1] - off);
  const int spad = (sj + 3) & ~3;
  float* xj = P.x4 + P.xp4_off[j] * P.nv;
  if (convert) {
    // every load of the chunk is issued before any store (the stores could alias x for the compiler)
    float xr[NVB][2];
#pragma unroll
    for (int v = 0; v < NVB; v++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int a = lane + 32 * h;
        xr[v][h] = (v < P.nv && a < sj) ? x_load(P.x, P.xy32, off + v * P.ldx + a) : 0.f;  // padding is zero
      }
#pragma unroll
    for (int v = 0; v < NVB; v++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int a = lane + 32 * h;
        if (v < P.nv && a < spad) {
          xj[v * spad + a] = xr[v][h];
          wbuf[v * spad + a] = xr[v][h];
        }
      }
    __syncwarp();
  } else {
    stage_vectors<false>(wbuf, xj, P.nv * spad, lane);  // the FP32 copy of x(j), padding zero
  }
  float acc[RPL][NVB];
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.Vt) + P.vt_off[j], P.vscale[j], P.k, sj, P.LR, wbuf,
                         spad, P.nv, acc, lane);
  __syncwarp();
  group_reduce_m(acc, P.LR);
  store_node_m<RPL, NVB, false>(P.xhat + (leaf0 + j) * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, acc, lane);
}

// parent p of the upsweep for vectors v0 .. v0 + nw - 1 (nw <= NVB)
template <int F, int RPL, int NVB, bool CG>
__device__ __forceinline__ void up_node_m(const TreeParamsM& P, int64_t p, int lane, float* wbuf, int v0, int nw) {
  float acc[RPL][NVB];
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  for (int ci = 1; ci <= 2; ci++) {
    const int64_t ch = 2 * p + ci;
    // CG: the sibling subtree was written by another CTA
    stage_vectors<CG>(wbuf, P.xhat + (ch * P.nv + v0) * P.kp, nw * P.kp, lane);
    warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.Ft) + (ch - 1) * P.kk8, P.fscale[ch - 1], P.k, P.k,
                           P.LR, wbuf, P.kp, nw, acc, lane);
    __syncwarp();
  }
  group_reduce_m(acc, P.LR);
  store_node_m<RPL, NVB, false>(P.xhat + (p * P.nv + v0) * P.kp, P.k, P.kp, P.LR, nw, acc, lane);
}

// vectors per warp where the warps of a CTA split one node's vectors between them
template <int NVB>
__host__ __device__ constexpr int slice_vectors() { return NVB >= kTreeWarpsM ? NVB / kTreeWarpsM : 1; }

// leaf projection + the whole upsweep in one launch (see k_upsweep_tree)
// CTA b works on subtree jobs[b].y of matrix jobs[b].x
template <int F, int RPL, int NVB>
// (the matrices whose vector count lies outside [nvlo, nvhi] are left to another launch: all their CTAs return)
__global__ void __launch_bounds__(kTreeWarpsM * 32) k_upsweep_tree_m(const MatDesc* __restrict__ mats,
                                                                    const int2* __restrict__ jobs, int nvlo, int nvhi,
                                                                    int convert) {
  __shared__ __align__(16) float wstage[kTreeWarpsM][NVB * 64];
  const int2 job = jobs[blockIdx.x];
  const TreeParamsM P = tree_params(mats[job.x]);
  if (P.nv < nvlo || P.nv > nvhi) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* wbuf = wstage[warp];
  const int T = P.q - P.L;
  const int64_t sub = job.y;
  for (int64_t t = warp; t < ((int64_t)1 << T); t += kTreeWarpsM)
    project_leaf_m<F, RPL, NVB>(P, (sub << T) + t, lane, wbuf, convert != 0);
  __syncthreads();
  constexpr int NVW = slice_vectors<NVB>();
  for (int lvl = P.q - 1; lvl >= P.L; lvl--) {
    const int64_t node0 = ((int64_t)1 << lvl) - 1 + (sub << (lvl - P.L));
    const int nn = 1 << (lvl - P.L);
    if (nn >= kTreeWarpsM || P.nv <= NVW) {  // a warp per node, all vectors
      for (int t = warp; t < nn; t += kTreeWarpsM) up_node_m<F, RPL, NVB, false>(P, node0 + t, lane, wbuf, 0, P.nv);
    } else {  // fewer nodes than warps: a warp per (node, slice of NVW vectors)
      const int ns = (P.nv + NVW - 1) / NVW;
      for (int u = warp; u < nn * ns; u += kTreeWarpsM) {
        const int t = u % nn, v0 = (u / nn) * NVW;
        up_node_m<F, RPL, NVW, false>(P, node0 + t, lane, wbuf, v0, min(NVW, P.nv - v0));
      }
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  // climb while this CTA arrives second at the parent; every warp takes a slice of the vectors
  __shared__ int second;
  const int v0 = warp * NVW, nw = min(NVW, P.nv - v0);
  int64_t node = ((int64_t)1 << P.L) - 1 + sub;
  while (node > 0) {
    const int64_t par = (node - 1) / 2;
    if (threadIdx.x == 0) {
      const int s2 = atomicAdd(P.ticket + par, 1) == 1;
      if (s2) P.ticket[par] = 0;
      second = s2;
    }
    __syncthreads();
    if (!second) break;
    __threadfence();
    if (nw > 0) up_node_m<F, RPL, NVW, true>(P, par, lane, wbuf, v0, nw);
    __threadfence();
    __syncthreads();
    node = par;
  }
}

// the whole downsweep in one launch (see k_downsweep_tree)
// Leaf expansion of leaf j (Eq. 4): y(j) = scale * U_j yhat_j (assign: the dense phase runs
// afterwards and adds its part), or y(j) += scale * U_j yhat_j with FP64 atomic adds (the dense
// phase adds its part the same way at the same time, both into a y zeroed before the product).
// U_j is size_j x k, FP32 entries or 16-bit codes of format FB (column-major or panel layout);
// its place and scale come from the matrix's row job and block record.
template <int FB, int NVB>
__device__ __forceinline__ void expand_leaf_m(const MatDesc& D, int64_t j, int lane, float* wbuf, bool assign) {
  const RowJob J = D.rjobs[j];
  const MixedBlock mb = D.blk[J.ublk];
  const int nv = D.nv, k = D.k, kp = D.kp;
  const int64_t off = D.leaf_off[j];
  const int R = (int)(D.leaf_off[j + 1] - off);
  stage_vectors<false>(wbuf, D.yhat + ((((int64_t)1 << D.q) - 1 + j) * nv) * kp, nv * kp, lane);
  const bool f32 = (mb.src & 2) != 0, panel = (mb.src & 4) != 0;
  const unsigned char* U = reinterpret_cast<const unsigned char*>(D.dmat) + J.uoff;
  const int ps2 = panel_stride(k) / 2;
  float acc[2][NVB];
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  for (int nu0 = 0; nu0 < k; nu0 += 8) {  // eight columns' loads before their use
    float u[8][2];
#pragma unroll
    for (int c = 0; c < 8; c++)
#pragma unroll
      for (int r = 0; r < 2; r++) {
        const int row = lane + 32 * r, nu = nu0 + c;
        u[c][r] = 0.f;
        if (row < R && nu < k) {
          if (f32) u[c][r] = __ldg(reinterpret_cast<const float*>(U) + row + R * nu);
          else
            u[c][r] = code_to_f<FB>(__ldg(reinterpret_cast<const uint16_t*>(U) +
                                          (panel ? (row >> 3) * ps2 + 8 * nu + (row & 7) : row + R * nu)));
        }
      }
#pragma unroll
    for (int c = 0; c < 8; c++) {
      if (nu0 + c >= k) break;
#pragma unroll
      for (int v = 0; v < NVB; v++) {
        const float yv = v < nv ? wbuf[v * kp + nu0 + c] : 0.f;
        acc[0][v] = fmaf(u[c][0], yv, acc[0][v]);
        acc[1][v] = fmaf(u[c][1], yv, acc[1][v]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 2; r++) {
    const int row = lane + 32 * r;
    if (row >= R) continue;
#pragma unroll
    for (int v = 0; v < NVB; v++)
      if (v < nv) {
        y_store(D.y, D.xy32, v * D.ldy + off + row, mb.scale * acc[r][v], assign);
      }
  }
  __syncwarp();  // wbuf is reused by the warp's next leaf
}

template <int F, int RPL, int NVB>
__global__ void __launch_bounds__(kTreeWarpsM * 32) k_downsweep_tree_m(const MatDesc* __restrict__ mats,
                                                                      const int2* __restrict__ jobs, int nvlo,
                                                                      int nvhi, int expand) {  // 0 none, 1 add, 2 assign
  __shared__ float path[2][NVB][64];
  __shared__ __align__(16) float wstage[kTreeWarpsM][NVB * 64];
  const int2 job = jobs[blockIdx.x];
  const TreeParamsM P = tree_params(mats[job.x]);
  if (P.nv < nvlo || P.nv > nvhi) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* wbuf = wstage[warp];
  const int64_t sub = job.y;
  const int64_t root = ((int64_t)1 << P.L) - 1 + sub;
  // the path from the root to the subtree root, recomputed by every CTA; every warp takes a
  // slice of the vectors (the slices are independent)
  constexpr int NVW = slice_vectors<NVB>();
  const int v0 = warp * NVW, nw = min(NVW, P.nv - v0);
  if (P.L > 0 && nw > 0) {
    int cur = 0;
    for (int v = v0; v < v0 + nw; v++)
      for (int r = lane; r < P.k; r += 32) path[cur][v][r] = P.yhat[(int64_t)v * P.kp + r];
    __syncwarp();
    for (int l = 1; l <= P.L; l++) {
      const int64_t a = ((root + 1) >> (P.L - l)) - 1;
      float acc[RPL][NVW];
#pragma unroll
      for (int r = 0; r < RPL; r++)
#pragma unroll
        for (int v = 0; v < NVW; v++) acc[r][v] = 0.f;
      warp_mv_m<F, RPL, NVW>(static_cast<const typename CodeT<F>::T*>(P.E) + (a - 1) * P.kk8, P.escale[a - 1], P.k, P.k,
                             P.LR, &path[cur][v0][0], 64, nw, acc, lane);
      group_reduce_m(acc, P.LR);
      if (lane < P.LR) {
#pragma unroll
        for (int rr = 0; rr < RPL; rr++) {
          const int row = lane + 32 * rr;
          if (row >= P.k) continue;
#pragma unroll
          for (int v = 0; v < NVW; v++) {
            if (v >= nw) continue;
            const int64_t at = (a * P.nv + v0 + v) * P.kp + row;
            const float val = acc[rr][v] + P.yhat[at];
            if (l == P.L) P.yhat[at] = val;
            else path[cur ^ 1][v0 + v][row] = val;
          }
        }
      }
      __syncwarp();
      cur ^= 1;
    }
  }
  __syncthreads();
  for (int lvl = P.L + 1; lvl <= P.q; lvl++) {
    const int64_t node0 = ((int64_t)1 << lvl) - 1 + (sub << (lvl - P.L));
    const int nn = 1 << (lvl - P.L);
    if (nn >= kTreeWarpsM || P.nv <= NVW) {  // a warp per node, all vectors
      for (int t = warp; t < nn; t += kTreeWarpsM) {
        const int64_t ch = node0 + t;
        float acc[RPL][NVB];
#pragma unroll
        for (int r = 0; r < RPL; r++)
#pragma unroll
          for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
        stage_vectors<false>(wbuf, P.yhat + ((ch - 1) / 2) * P.nv * P.kp, P.nv * P.kp, lane);
        warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.E) + (ch - 1) * P.kk8, P.escale[ch - 1], P.k,
                               P.k, P.LR, wbuf, P.kp, P.nv, acc, lane);
        __syncwarp();
        group_reduce_m(acc, P.LR);
        store_node_m<RPL, NVB, true>(P.yhat + ch * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, acc, lane);
      }
    } else {  // fewer nodes than warps: a warp per (node, slice of NVW vectors)
      const int ns = (P.nv + NVW - 1) / NVW;
      for (int u = warp; u < nn * ns; u += kTreeWarpsM) {
        const int64_t ch = node0 + u % nn;
        const int s0 = (u / nn) * NVW, sw = min(NVW, P.nv - s0);
        float acc[RPL][NVW];
#pragma unroll
        for (int r = 0; r < RPL; r++)
#pragma unroll
          for (int v = 0; v < NVW; v++) acc[r][v] = 0.f;
        stage_vectors<false>(wbuf, P.yhat + (((ch - 1) / 2) * P.nv + s0) * P.kp, sw * P.kp, lane);
        warp_mv_m<F, RPL, NVW>(static_cast<const typename CodeT<F>::T*>(P.E) + (ch - 1) * P.kk8, P.escale[ch - 1], P.k,
                               P.k, P.LR, wbuf, P.kp, sw, acc, lane);
        __syncwarp();
        group_reduce_m(acc, P.LR);
        store_node_m<RPL, NVW, true>(P.yhat + (ch * P.nv + s0) * P.kp, P.k, P.kp, P.LR, sw, acc, lane);
      }
    }
    __syncthreads();
  }
  // leaf expansion (Eq. 4) of the subtree's leaves: their yhat is final (written by this CTA
  // above, or by the coupling phase when the subtree root is the root and a leaf)
  if (expand) {
    const MatDesc& D = mats[job.x];
    const int T = P.q - P.L;
    for (int64_t t = warp; t < ((int64_t)1 << T); t += kTreeWarpsM)
      expand_leaf_m<F, NVB>(D, (sub << T) + t, lane, wbuf, expand == 2);
  }
}

// ---------------------------------------------------------------- coupling, all levels
// The coupling rows of all levels (Eq. 3) are cut into chunks of consecutive
// rows of one matrix: int4 {matrix, first row, rows (1 .. 31), 0}, about the
// same number of blocks each. One warp per chunk; a launch serves the
// matrices whose vector count lies in [nvlo, nvhi] (the others' chunks return
// at once), so a batch with mixed vector counts runs each count's variant.
constexpr int kChunkRows = 31;

// chunk state shared by both kernels: row pointers of the chunk in lanes 0 .. rows
struct ChunkRows {
  int32_t sr;         // Srow[row0 + lane] (lanes 0 .. rows)
  unsigned nonempty;  // bit j: row row0 + j has coupling blocks
};

// rows without coupling blocks get yhat = 0 (vectors vbase .. vbase + vcount - 1);
// returns the chunk's row pointers
__device__ __forceinline__ ChunkRows chunk_rows(const int32_t* __restrict__ Srow, float* __restrict__ yhat, int row0,
                                                int rows, int nv, int kp, int lane, int vbase, int vcount) {
  ChunkRows c;
  c.sr = (lane <= rows) ? __ldg(Srow + row0 + lane) : 0;
  const int32_t next = __shfl_down_sync(0xFFFFFFFFu, c.sr, 1);
  const bool has = lane < rows && next > c.sr;
  c.nonempty = __ballot_sync(0xFFFFFFFFu, has);
  for (int j = 0; j < rows; j++)
    if (!((c.nonempty >> j) & 1u)) {
      float* dst = yhat + ((int64_t)(row0 + j) * nv + vbase) * kp;
      for (int t = lane; t < vcount * kp; t += 32) dst[t] = 0.f;
    }
  return c;
}

// k = 16, 32 or 64. Lane l reads 16 bytes, 8 consecutive codes (rows 8m ..
// 8m + 7, m = l % RG, RG = k / 8) of a column c = l / RG + (32 / RG) t (16
// contiguous bytes both column-major and in the panel layout), so a
// 16 x 16 block is one 512-byte load of the warp; a slot is OPS such octets
// per lane (a quarter of a 64 x 64 block, a whole block for k <= 32). The
// block scale multiplies the vector entry (S_ij x_j = Q (sigma x_j)). The warp
// walks the slots of its chunk's non-empty rows CB at a time with two batches
// in flight; after a row's last batch its sums are reduced over the lanes of
// the same row group and stored. VG warps of a CTA share a chunk, warp w taking
// vectors (w % VG) * NVW .. + NVW - 1 (the later ones read the blocks from L1).
template <int F, int K, int NVW, int CB, int VG>
__global__ void __launch_bounds__(128) k_coupling_m(const MatDesc* __restrict__ mats, const int4* __restrict__ chunks,
                                                   int64_t nchunks, int nvlo, int nvhi) {
  static_assert(K == 16 || K == 32 || K == 64, "octet layout");
  static_assert(VG == 1 || VG == 2 || VG == 4, "vector groups per chunk");
  constexpr int RG = K / 8, CS = 32 / RG;   // row groups per column; column stride between a lane's octets
  constexpr int OPL = K * K / 256;          // octets per lane per block
  constexpr int OPS = OPL < 4 ? OPL : 4;    // octets per lane per slot
  constexpr int SPB = OPL / OPS;            // slots per block
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cidx = (int64_t)blockIdx.x * (4 / VG) + warp / VG;
  const int vbase = (warp % VG) * NVW;
  if (cidx >= nchunks) return;
  const int4 ch = __ldg(chunks + cidx);
  const MatDesc& D = mats[ch.x];
  const int nv = D.nv;
  if (nv < nvlo || nv > nvhi || vbase >= nv) return;
  const uint16_t* __restrict__ S = D.smat;
  const float* __restrict__ sscale = D.sscale;
  const int64_t kk8 = D.kk8;
  const int32_t* __restrict__ Scol = D.Scol;
  const int kp = D.kp;
  const float* __restrict__ xhat = D.xhat;
  float* __restrict__ yhat = D.yhat;
  const int row0 = ch.y, rows = min(ch.z, kChunkRows);
  const ChunkRows cr = chunk_rows(D.Srow, yhat, row0, rows, nv, kp, lane, vbase, min(NVW, nv - vbase));
  if (!cr.nonempty) return;
  const int m = lane % RG, cl = lane / RG;
  // octet (m, c) of a block: 8 m + K c codes (column-major), or 512 m + 8 c (panel layout, K = 64)
  const bool spanel = K == 64 && D.spanel != 0;
  const int om = spanel ? 512 * m : 8 * m, oc = spanel ? 8 : K;
  float acc[8][NVW];
#pragma unroll
  for (int r = 0; r < 8; r++)
#pragma unroll
    for (int v = 0; v < NVW; v++) acc[r][v] = 0.f;
  uint4 a0[CB][OPS], a1[CB][OPS];
  float x0[CB][OPS][NVW], x1[CB][OPS][NVW], s0[CB], s1[CB];
  int32_t cA[CB], cB[CB];   // column nodes of a batch, fetched one batch before its codes and vectors
  float sA[CB], sB[CB];
  // the column nodes and scales of a batch: loaded one batch ahead, so that the vector loads
  // that depend on them never wait inside `load`
  auto fetch = [&](int32_t b0, int nslot, int bt, int32_t(&col)[CB], float(&scl)[CB]) {
#pragma unroll
    for (int u = 0; u < CB; u++) {
      const int slot = bt * CB + u;
      col[u] = 0;
      scl[u] = 0.f;
      if (slot < nslot) {  // warp-uniform
        const int32_t gb = b0 + slot / SPB;
        col[u] = __ldg(Scol + gb);
        scl[u] = __ldg(sscale + gb);
      }
    }
  };
  // loads only: nothing here consumes a loaded value, so a batch's loads stay in flight
  // while the previous batch is computed
  auto load = [&](int32_t b0, int nslot, int bt, const int32_t(&col)[CB], const float(&scl)[CB],
                  uint4(&a)[CB][OPS], float(&xv)[CB][OPS][NVW], float(&sc)[CB]) {
#pragma unroll
    for (int u = 0; u < CB; u++) {
      const int slot = bt * CB + u;
      sc[u] = scl[u];
#pragma unroll
      for (int o = 0; o < OPS; o++) {
        a[u][o] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int v = 0; v < NVW; v++) xv[u][o][v] = 0.f;
      }
      if (slot < nslot) {  // warp-uniform
        const int32_t gb = b0 + slot / SPB;
        const int tq = slot % SPB;
        const float* X = xhat + ((int64_t)col[u] * nv + vbase) * kp;
        const uint16_t* blk = S + (int64_t)gb * kk8 + om;
#pragma unroll
        for (int o = 0; o < OPS; o++) {
          const int c = cl + CS * (tq * OPS + o);
          a[u][o] = __ldg(reinterpret_cast<const uint4*>(blk + oc * c));
#pragma unroll
          for (int v = 0; v < NVW; v++) xv[u][o][v] = (vbase + v < nv) ? __ldg(X + v * kp + c) : 0.f;
        }
      }
    }
  };
  auto compute = [&](const uint4(&a)[CB][OPS], const float(&xv)[CB][OPS][NVW], const float(&sc)[CB]) {
#pragma unroll
    for (int u = 0; u < CB; u++)
#pragma unroll
      for (int o = 0; o < OPS; o++) {
        const float2 q0 = codes_to_f2<F>(a[u][o].x), q1 = codes_to_f2<F>(a[u][o].y);
        const float2 q2 = codes_to_f2<F>(a[u][o].z), q3 = codes_to_f2<F>(a[u][o].w);
#pragma unroll
        for (int v = 0; v < NVW; v++) {
          const float xs = sc[u] * xv[u][o][v];
          acc[0][v] = fmaf(q0.x, xs, acc[0][v]);
          acc[1][v] = fmaf(q0.y, xs, acc[1][v]);
          acc[2][v] = fmaf(q1.x, xs, acc[2][v]);
          acc[3][v] = fmaf(q1.y, xs, acc[3][v]);
          acc[4][v] = fmaf(q2.x, xs, acc[4][v]);
          acc[5][v] = fmaf(q2.y, xs, acc[5][v]);
          acc[6][v] = fmaf(q3.x, xs, acc[6][v]);
          acc[7][v] = fmaf(q3.y, xs, acc[7][v]);
        }
      }
  };
  auto flush = [&](int r) {  // row row0 + r is complete
#pragma unroll
    for (int off = RG; off < 32; off <<= 1)
#pragma unroll
      for (int rr = 0; rr < 8; rr++)
#pragma unroll
        for (int v = 0; v < NVW; v++) acc[rr][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[rr][v], off);
    if (cl == 0) {
      float* dst = yhat + ((int64_t)(row0 + r) * nv + vbase) * kp + 8 * m;
#pragma unroll
      for (int v = 0; v < NVW; v++)
        if (vbase + v < nv) {
          *reinterpret_cast<float4*>(dst + v * kp) = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
          *reinterpret_cast<float4*>(dst + v * kp + 4) = make_float4(acc[4][v], acc[5][v], acc[6][v], acc[7][v]);
        }
    }
#pragma unroll
    for (int rr = 0; rr < 8; rr++)
#pragma unroll
      for (int v = 0; v < NVW; v++) acc[rr][v] = 0.f;
  };
  // a cursor over the batches of the chunk's non-empty rows, in order
  struct Cursor {
    unsigned mask;  // rows not yet finished; r is its lowest bit
    int r, bt, nslot;
    int32_t b0;
  };
  auto begin = [&](Cursor& c) {
    c.mask = cr.nonempty;
    c.r = __ffs(c.mask) - 1;
    c.bt = 0;
    c.b0 = __shfl_sync(0xFFFFFFFFu, cr.sr, c.r);
    c.nslot = (__shfl_sync(0xFFFFFFFFu, cr.sr, c.r + 1) - c.b0) * SPB;
  };
  auto advance = [&](Cursor& c) -> bool {
    if ((c.bt + 1) * CB < c.nslot) {
      c.bt++;
      return true;
    }
    c.mask &= c.mask - 1u;
    if (!c.mask) return false;
    c.r = __ffs(c.mask) - 1;
    c.bt = 0;
    c.b0 = __shfl_sync(0xFFFFFFFFu, cr.sr, c.r);
    c.nslot = (__shfl_sync(0xFFFFFFFFu, cr.sr, c.r + 1) - c.b0) * SPB;
    return true;
  };
  Cursor ic, lc, cc;   // index fetches run one batch ahead of the loads, the loads one ahead of the compute
  begin(ic);
  begin(lc);
  begin(cc);
  fetch(ic.b0, ic.nslot, ic.bt, cA, sA);
  bool more_i = advance(ic);
  if (more_i) {
    fetch(ic.b0, ic.nslot, ic.bt, cB, sB);
    more_i = advance(ic);
  }
  load(lc.b0, lc.nslot, lc.bt, cA, sA, a0, x0, s0);
  bool more = advance(lc);
  if (more_i) {
    fetch(ic.b0, ic.nslot, ic.bt, cA, sA);
    more_i = advance(ic);
  }
  while (true) {
    if (more) {
      load(lc.b0, lc.nslot, lc.bt, cB, sB, a1, x1, s1);
      more = advance(lc);
      if (more_i) {
        fetch(ic.b0, ic.nslot, ic.bt, cB, sB);
        more_i = advance(ic);
      }
    }
    compute(a0, x0, s0);
    if ((cc.bt + 1) * CB >= cc.nslot) flush(cc.r);
    if (!advance(cc)) break;
    if (more) {
      load(lc.b0, lc.nslot, lc.bt, cA, sA, a0, x0, s0);
      more = advance(lc);
      if (more_i) {
        fetch(ic.b0, ic.nslot, ic.bt, cA, sA);
        more_i = advance(ic);
      }
    }
    compute(a1, x1, s1);
    if ((cc.bt + 1) * CB >= cc.nslot) flush(cc.r);
    if (!advance(cc)) break;
  }
}

// any other k: the chunk's rows one after another, one block at a time
template <int F, int RPL, int NVB>
__global__ void __launch_bounds__(128) k_coupling_m_generic(const MatDesc* __restrict__ mats,
                                                           const int4* __restrict__ chunks, int64_t nchunks, int nvlo,
                                                           int nvhi) {
  __shared__ __align__(16) float wstage[4][NVB * 64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* wbuf = wstage[warp];
  const int64_t cidx = (int64_t)blockIdx.x * 4 + warp;
  if (cidx >= nchunks) return;
  const int4 ch = __ldg(chunks + cidx);
  const MatDesc& D = mats[ch.x];
  const int nv = D.nv;
  if (nv < nvlo || nv > nvhi) return;
  const uint16_t* __restrict__ S = D.smat;
  const float* __restrict__ sscale = D.sscale;
  const int64_t kk8 = D.kk8;
  const int32_t* __restrict__ Scol = D.Scol;
  const int k = D.k, kp = D.kp, LR = D.LR;
  const float* __restrict__ xhat = D.xhat;
  float* __restrict__ yhat = D.yhat;
  const int row0 = ch.y, rows = min(ch.z, kChunkRows);
  const ChunkRows cr = chunk_rows(D.Srow, yhat, row0, rows, nv, kp, lane, 0, nv);
  for (unsigned m = cr.nonempty; m; m &= m - 1u) {
    const int r = __ffs(m) - 1;
    const int32_t b0 = __shfl_sync(0xFFFFFFFFu, cr.sr, r), b1 = __shfl_sync(0xFFFFFFFFu, cr.sr, r + 1);
    float acc[RPL][NVB];
#pragma unroll
    for (int rr = 0; rr < RPL; rr++)
#pragma unroll
      for (int v = 0; v < NVB; v++) acc[rr][v] = 0.f;
    for (int32_t b = b0; b < b1; b++) {  // the column node's vectors staged in shared memory
      stage_vectors<false>(wbuf, xhat + (int64_t)Scol[b] * nv * kp, nv * kp, lane);
      warp_mv_m<F, RPL, NVB>(S + (int64_t)b * kk8, sscale[b], k, k, LR, wbuf, kp, nv, acc, lane);
      __syncwarp();
    }
    group_reduce_m(acc, LR);
    store_node_m<RPL, NVB, false>(yhat + (int64_t)(row0 + r) * nv * kp, k, kp, LR, nv, acc, lane);
  }
}

// ---------------------------------------------------------------- coupling from the kernel
// The coupling blocks evaluated instead of read (the paper's matrices take every block as the
// kernel at the interpolation points of its two clusters, Sec. 4.6): yhat_i = sum_j S_ij xhat_j,
// S_ij[nu][mu] = K(|xi_i^nu - xi_j^mu|), K(r) = exp(-r / ell) or, for the Matern-3/2 kernel,
// (1 + s) exp(-s) with s = sqrt(3) r / ell. A point is its node's centre c (FP32 pair hi + lo)
// plus an FP32 offset o; a coordinate difference is ((hi_i - hi_j) + (lo_i - lo_j)) + (o_i - o_j),
// which keeps FP32 relative precision of the distance at any separation. Rows as warp_mv_m: lane
// g * LR + rl owns rows rl + 32 r. The G = 32 / LR lane groups take different blocks of the row
// (group g the blocks b0 + g, b0 + g + G, ...; GB <= G groups, so that their staged data fit),
// each lane all k columns of its group's block in runs of four, so a vector's four entries are one
// float4 read. A row's sums are reduced over the groups once, after its last block. Each group
// stages its block's column points and vectors in the warp's shared memory; r = r2 * rsqrt(r2)
// and exp(-t) = __expf(-t) (CUDA's fast intrinsics: relative errors of a few 1e-6 here, below the
// form's FP32 accumulation bound).
// 2^x by the special-function unit (PTX ex2.approx: relative error a few 2^-23)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// KIND: H2_KERNEL_EXP (0) or H2_KERNEL_MATERN32 (1); the descriptor's kf_kind selects the instance
template <int RPL, int NVB, int KIND>
__global__ void __launch_bounds__(128, RPL == 1 ? 6 : 4) k_coupling_kf(const MatDesc* __restrict__ mats,
                                                                     const int4* __restrict__ chunks, int64_t nchunks,
                                                                     int nvlo, int nvhi) {
  __shared__ __align__(16) float wstage[4][NVB * 64];
  __shared__ float4 ostage[4][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cidx = (int64_t)blockIdx.x * 4 + warp;
  if (cidx >= nchunks) return;
  const int4 ch = __ldg(chunks + cidx);
  const MatDesc& D = mats[ch.x];
  const int nv = D.nv;
  if (nv < nvlo || nv > nvhi) return;
  const int k = min(D.k, 64), kp = D.kp, LR = D.LR, G = 32 / LR, g = lane / LR, rl = lane - g * LR;
  const int GB = max(1, min(G, 64 / kp));  // groups with a block: GB * kp <= 64 staged columns
  const bool active = g < GB;
  float* wbuf = wstage[warp] + g * nv * kp;  // this group's block: vectors (nv x kp) and points (k)
  float4* obuf = ostage[warp] + g * kp;
  const float4* __restrict__ chi = D.kf_chi;
  const float4* __restrict__ clo = D.kf_clo;
  const float4* __restrict__ off = D.kf_off;
  const float inv_ell = D.kf_inv_ell;
  // exp: K = 2^(-r c), c = log2(e) / ell; Matern-3/2: t = r sqrt(3) / ell, K = (1 + t) 2^(-t log2(e))
  const float tscale = KIND == 1 ? 1.7320508f * inv_ell : 1.4426950f * inv_ell;
  const int32_t* __restrict__ Scol = D.Scol;
  const float* __restrict__ xhat = D.xhat;
  float* __restrict__ yhat = D.yhat;
  const int row0 = ch.y, rows = min(ch.z, kChunkRows);
  const ChunkRows cr = chunk_rows(D.Srow, yhat, row0, rows, nv, kp, lane, 0, nv);
  for (unsigned m = cr.nonempty; m; m &= m - 1u) {
    const int r = __ffs(m) - 1;
    const int64_t i = row0 + r;
    const int32_t b0 = __shfl_sync(0xFFFFFFFFu, cr.sr, r), b1 = __shfl_sync(0xFFFFFFFFu, cr.sr, r + 1);
    float4 oi[RPL];
#pragma unroll
    for (int rr = 0; rr < RPL; rr++) {
      const int nu = rl + 32 * rr;
      oi[rr] = nu < k ? __ldg(off + i * k + nu) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 hi_i = __ldg(chi + i), lo_i = __ldg(clo + i);
    float acc[RPL][NVB];
#pragma unroll
    for (int rr = 0; rr < RPL; rr++)
#pragma unroll
      for (int v = 0; v < NVB; v++) acc[rr][v] = 0.f;
    for (int32_t bb = b0; bb < b1; bb += GB) {  // GB blocks at a time, one per group
      const int32_t b = bb + g;
      const bool mine = active && b < b1;
      const int64_t j = mine ? (int64_t)Scol[b] : 0;
      if (mine) {  // the group's lanes stage its block's column points and vectors
        for (int t = rl; t < k; t += LR) obuf[t] = __ldg(off + j * k + t);
        const float4* src = reinterpret_cast<const float4*>(xhat + j * nv * kp);
        for (int t = rl; t < nv * kp / 4; t += LR) reinterpret_cast<float4*>(wbuf)[t] = src[t];
      }
      __syncwarp();
      if (mine) {
        const float4 hi_j = __ldg(chi + j), lo_j = __ldg(clo + j);
        const float cx = (hi_i.x - hi_j.x) + (lo_i.x - lo_j.x), cy = (hi_i.y - hi_j.y) + (lo_i.y - lo_j.y),
                    cz = (hi_i.z - hi_j.z) + (lo_i.z - lo_j.z);
        // row point minus the column centre, once per block: a coordinate difference is then one
        // subtraction. The clusters of a coupling block are separated (their boxes' distance is
        // positive and at least their diameter / eta), so the difference does not cancel and
        // keeps FP32 relative precision, and r^2 > 0.
        float ax[RPL], ay[RPL], az[RPL];
#pragma unroll
        for (int rr = 0; rr < RPL; rr++) {
          ax[rr] = cx + oi[rr].x;
          ay[rr] = cy + oi[rr].y;
          az[rr] = cz + oi[rr].z;
        }
        // one run of four columns; FULL: all four below k (no clamping or masking)
        auto run = [&](int mu0, auto full_tag) {
          constexpr bool FULL = decltype(full_tag)::value;
          float sv[RPL][4];
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const float4 oj = obuf[FULL ? mu0 + e : min(mu0 + e, k - 1)];
#pragma unroll
            for (int rr = 0; rr < RPL; rr++) {
              const float dx = ax[rr] - oj.x, dy = ay[rr] - oj.y, dz = az[rr] - oj.z;
              const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
              const float t = (r2 * rsqrtf(r2)) * tscale;
              float val;
              if constexpr (KIND == 1) {
                const float ex = ex2_approx(-1.4426950f * t);
                val = fmaf(t, ex, ex);
              } else {
                val = ex2_approx(-t);
              }
              sv[rr][e] = (FULL || mu0 + e < k) ? val : 0.f;
            }
          }
#pragma unroll
          for (int v = 0; v < NVB; v++) {
            if (v >= nv) break;
            float4 xv = *reinterpret_cast<const float4*>(wbuf + v * kp + mu0);
            if (!FULL) {  // entries past k (the vectors' padding) take no part
              if (mu0 + 3 >= k) xv.w = 0.f;
              if (mu0 + 2 >= k) xv.z = 0.f;
              if (mu0 + 1 >= k) xv.y = 0.f;
            }
#pragma unroll
            for (int rr = 0; rr < RPL; rr++)
              acc[rr][v] = fmaf(sv[rr][3], xv.w, fmaf(sv[rr][2], xv.z, fmaf(sv[rr][1], xv.y, fmaf(sv[rr][0], xv.x, acc[rr][v]))));
          }
        };
        int mu0 = 0;
        for (; mu0 + 3 < k; mu0 += 4) run(mu0, std::true_type{});  // columns mu0 .. mu0 + 3
        if (mu0 < k) run(mu0, std::false_type{});                   // the last, partial run (mu0 + 3 < kp)
      }
      __syncwarp();
    }
    // the groups' partial sums: lanes rl, rl + LR, ... hold the same rows
    group_reduce_m(acc, LR);
    store_node_m<RPL, NVB, false>(yhat + i * nv * kp, k, kp, LR, nv, acc, lane);
  }
}

// ---------------------------------------------------------------- dense near field + expansion (TMA stream)
// Per-block side information of the dense stream, 16 bytes.




constexpr int kMixedMaxBlocks = 8;   // blocks of one row per work item
constexpr int kMixedVecCols = 256;   // vector columns of one work item (sum of its blocks' vs)
constexpr int kMixedHeader = 256;
__host__ __device__ constexpr int mixed_vec_area(int nvb) { return kMixedVecCols * nvb * 4; }
__host__ __device__ constexpr int mixed_stage_bytes(int nvb) { return kMixedHeader + kStageMat + mixed_vec_area(nvb); }
// row partials [warp][vector][64 rows]; passes of at most four vectors double-buffer them by row
// parity (rows end without a CTA-wide barrier, see k_dense_stream_m)
__host__ __device__ constexpr int mixed_red_bytes(int nvb, int cw) { return (nvb <= 4 ? 2 : 1) * cw * nvb * 64 * 4; }
// block records of one producer batch of 32 items: their blocks, plus one record per row between
// them (U_i, not streamed) -- at most 32 (kMixedMaxBlocks + 1) records
constexpr int kMixedBatchBlocks = 32 * (kMixedMaxBlocks + 1);
constexpr int kMixedBlkBuf = kMixedBatchBlocks * 16;
__host__ __device__ constexpr int mixed_stages(int nvb, int cw) {
  return (kSmemLimit - 256 - kMixedBlkBuf - mixed_red_bytes(nvb, cw)) / mixed_stage_bytes(nvb) < 6
             ? (kSmemLimit - 256 - kMixedBlkBuf - mixed_red_bytes(nvb, cw)) / mixed_stage_bytes(nvb)
             : 6;
}
__host__ __device__ constexpr int mixed_smem_bytes(int nvb, int cw) {
  return mixed_stages(nvb, cw) * mixed_stage_bytes(nvb) + 256 + mixed_red_bytes(nvb, cw) + kMixedBlkBuf;
}
constexpr int kMixedCW = 8;

// items: m_off (in the matrix's dmat), m_bytes, shape = R | nb << 8, v_off = first block (batch-wide
// index into blk), row = y offset, flags = last-of-row | matrix index << 8
struct MixedStreamParams {
  const StreamItem* items;
  const int* cta_begin;
  const MixedBlock* blk;
  const MatDesc* mats;
  int* err;
  long long budget;
};

// Stage header (ints): [0] R, [1] nb, [2] row, [3] flags, [4] uniform (1: every block a full 64 x 64
// column-major block of 16-bit codes with 64 vector columns, 2: the same in the panel layout; the
// blocks' codes and vector chunks then follow each other at fixed strides); block t at 8 + 4 t:
// cols | FP32-entries flag << 16, vs, matrix offset in bytes, scale (bits);
// [40 + t] block t's vector offset in bytes; [48] nv; [50..51] y; [52..53] ldy.
constexpr int kHdVoff = 40, kHdNv = 48, kHdXy32 = 49, kHdY = 50, kHdLdy = 52;
template <int NST, int SB, int VAREA>
__device__ __forceinline__ void mixed_produce(const MixedStreamParams& P, const StreamShared& S, int ib, int ie,
                                              MixedBlock* blkbuf) {
  const int lane = threadIdx.x & 31;
  const uint64_t pol = policy_evict_first();
  int issued = 0;
  bool ok = true;
  // the waits below use the FP64 stream's bounded-wait helper through a shim
  StreamParams W{};
  W.err = P.err;
  W.budget = P.budget;
  for (int base = ib; base < ie && ok; base += 32) {
    int4 d0 = make_int4(0, 0, 0, 0), d1 = make_int4(0, 0, 0, 0);
    if (base + lane < ie) {
      const int4* src = reinterpret_cast<const int4*>(P.items + base + lane);
      d0 = __ldg(src);
      d1 = __ldg(src + 1);
    }
    const int cnt = min(32, ie - base);
    // the batch's items cover a contiguous range of blocks: stage their records in shared memory
    const long long bfirst = (long long)(((unsigned long long)(unsigned)__shfl_sync(0xFFFFFFFFu, d1.y, 0) << 32) |
                                         (unsigned)__shfl_sync(0xFFFFFFFFu, d1.x, 0));
    const unsigned lshape = (unsigned)__shfl_sync(0xFFFFFFFFu, d0.w, cnt - 1);
    const long long blast = (long long)(((unsigned long long)(unsigned)__shfl_sync(0xFFFFFFFFu, d1.y, cnt - 1) << 32) |
                                        (unsigned)__shfl_sync(0xFFFFFFFFu, d1.x, cnt - 1)) +
                            min((int)((lshape >> 8) & 0xFF), kMixedMaxBlocks);
    const int nbatch = (int)min(blast - bfirst, (long long)kMixedBatchBlocks);
    for (int u = lane; u < nbatch; u += 32) blkbuf[u] = P.blk[bfirst + u];
    // each lane fetches the matrix fields of its own item
    const char* l_dmat = nullptr;
    const float* l_x4 = nullptr;
    const float* l_yhat = nullptr;
    double* l_y = nullptr;
    long long l_ldy = 0;
    int l_nv = 0, l_xy32 = 0;
    if (base + lane < ie) {
      const MatDesc& D = P.mats[d1.w >> 8];
      l_dmat = D.dmat;
      l_x4 = D.x4;
      l_yhat = D.yhat;
      l_y = D.y;
      l_ldy = D.ldy;
      l_nv = D.nv;
      l_xy32 = D.xy32;
    }
    __syncwarp();
    for (int t = 0; t < cnt; t++) {
      const int it = base + t - ib;
      const int s = it % NST, use = it / NST;
      if (use > 0 && !warp_wait(S.empty + s, (use - 1) & 1, W, S.abort_flag)) {
        ok = false;
        break;
      }
      if (__any_sync(0xFFFFFFFFu, *S.abort_flag != 0)) {
        ok = false;
        break;
      }
      const unsigned m_lo = (unsigned)__shfl_sync(0xFFFFFFFFu, d0.x, t);
      const unsigned m_hi = (unsigned)__shfl_sync(0xFFFFFFFFu, d0.y, t);
      const int m_bytes = __shfl_sync(0xFFFFFFFFu, d0.z, t);
      const unsigned shape = (unsigned)__shfl_sync(0xFFFFFFFFu, d0.w, t);
      const unsigned b_lo = (unsigned)__shfl_sync(0xFFFFFFFFu, d1.x, t);
      const unsigned b_hi = (unsigned)__shfl_sync(0xFFFFFFFFu, d1.y, t);
      const int row = __shfl_sync(0xFFFFFFFFu, d1.z, t);
      const int flags = __shfl_sync(0xFFFFFFFFu, d1.w, t);
      const int R = (int)(shape & 0xFF), nb = min((int)((shape >> 8) & 0xFF), kMixedMaxBlocks);
      const long long b0 = (long long)(((unsigned long long)b_hi << 32) | b_lo);
      const char* dmat = reinterpret_cast<const char*>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)l_dmat, t));
      const float* x4 = reinterpret_cast<const float*>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)l_x4, t));
      const float* yh = reinterpret_cast<const float*>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)l_yhat, t));
      const unsigned long long ydst = __shfl_sync(0xFFFFFFFFu, (unsigned long long)l_y, t);
      const long long ldy = (long long)__shfl_sync(0xFFFFFFFFu, (unsigned long long)l_ldy, t);
      const int nv = __shfl_sync(0xFFFFFFFFu, l_nv, t);
      const int xy32 = __shfl_sync(0xFFFFFFFFu, l_xy32, t);
      unsigned char* stage = S.stage0 + s * SB;
      int* hd = reinterpret_cast<int*>(stage);
      // per-block side information, one lane per block
      MixedBlock mb{};
      const long long bi = b0 - bfirst + lane;
      if (lane < nb && bi >= 0 && bi < nbatch) mb = blkbuf[bi];
      const int esize = (mb.src & 2) ? 4 : 2;
      const int codes = (mb.src & 4) ? panel_block_bytes(mb.cols)                   // padded bytes of this block
                                     : (R * (int)mb.cols * esize + 15) & ~15;
      int moff = codes;  // inclusive prefix of the blocks' padded byte counts
#pragma unroll
      for (int d = 1; d < kMixedMaxBlocks; d <<= 1) {
        const int o = __shfl_up_sync(0xFFFFFFFFu, moff, d);
        if (lane >= d) moff += o;
      }
      moff -= codes;
      const unsigned vbytes = (lane < nb) ? (unsigned)(nv * (int)mb.vs * 4) : 0u;
      unsigned voff = vbytes;  // inclusive prefix of the blocks' vector bytes
#pragma unroll
      for (int d = 1; d < kMixedMaxBlocks; d <<= 1) {
        const unsigned o = __shfl_up_sync(0xFFFFFFFFu, voff, d);
        if (lane >= d) voff += o;
      }
      const unsigned vtot = __shfl_sync(0xFFFFFFFFu, voff, kMixedMaxBlocks - 1);
      voff -= vbytes;
      // uniform item: every block full 64 x 64 16-bit codes in one layout, 64 vector columns each
      const int panel0 = __shfl_sync(0xFFFFFFFFu, (int)((mb.src >> 2) & 1), 0);
      const bool full = lane >= nb || (!(mb.src & 2) && mb.cols == 64 && mb.vs == 64 && (int)((mb.src >> 2) & 1) == panel0);
      const int uniform = (__all_sync(0xFFFFFFFFu, full) && R == 64) ? 1 + panel0 : 0;
      if (lane < nb) {
        hd[8 + 4 * lane] = mb.cols | ((mb.src & 2) << 15) | ((mb.src & 4) << 15);
        hd[9 + 4 * lane] = mb.vs;
        hd[10 + 4 * lane] = moff;
        hd[11 + 4 * lane] = __float_as_int(mb.scale);
        hd[kHdVoff + lane] = (int)voff;
      }
      if (lane == 0) {
        hd[0] = R;
        hd[1] = nb;
        hd[2] = row;
        hd[3] = flags;
        hd[4] = uniform;
        hd[kHdNv] = nv;
        hd[kHdXy32] = xy32;
        *reinterpret_cast<unsigned long long*>(hd + kHdY) = ydst;
        *reinterpret_cast<long long*>(hd + kHdLdy) = ldy;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_expect_tx(S.full + s, (unsigned)m_bytes + vtot);
        bulk_g2s_stream(stage + kMixedHeader, dmat + (((unsigned long long)m_hi << 32) | m_lo), (unsigned)m_bytes,
                        S.full + s, pol);
      }
      __syncwarp();
      if (lane < nb && vbytes > 0) {  // a matrix multiplies no vectors in this product: matrix bytes only
        const float* src = (mb.src & 1) ? yh : x4;
        bulk_g2s(stage + kMixedHeader + kStageMat + voff, src + mb.voff * nv, vbytes, S.full + s);
      }
      __syncwarp();
      issued = it + 1;
    }
  }
  if (lane == 0)
    for (int it = max(0, issued - NST); it < issued; it++) {
      const int s = it % NST, use = it / NST;
      if (!mbar_try_wait(S.full + s, use & 1)) {
        const long long t0 = clock64();
        while (!mbar_try_wait(S.full + s, use & 1) && clock64() - t0 < P.budget) {
        }
      }
    }
}

// One work item of the dense stream for up to NV2 vectors (NV2 <= NVB): every
// block's products are added, scaled by the block's scale, into acc (lane:
// rows r0, r0 + 1 of the item's row, summed over the warps at the row end).
// Rows of more than 32: warp w takes columns C w / CW .. C (w + 1) / CW of each
// block (full 64 x 64 blocks of codes on a branch-free path). Rows of at most
// 32: lanes l and l + 16 own rows 2 (l & 15), +1, and the 16 half-warps take
// the item's 4-column units (block, columns 4u .. 4u + 3) in turn, reading the
// four vector entries of a unit as one 16-byte load.
template <int F, int NV2, int NVB, int CW>
__device__ __forceinline__ void consume_item(const unsigned char* stage, const int* hd, int nb, int R, int warp, int lane,
                                             float (&acc)[2][NVB]) {
  constexpr int VAREA = mixed_vec_area(NVB);
  constexpr int SETS = NV2 == 1 ? 4 : (NV2 == 2 ? 2 : 1);
  constexpr bool kScaleCodes = NV2 >= 4;  // scale the codes once instead of per-vector partial sums
  if (R <= 32) {
    constexpr int HW = 2 * CW;  // half-warps
    const int r0 = 2 * (lane & 15), hw = warp * 2 + (lane >> 4);
    const bool even = (R & 1) == 0;
    int base = 0;
    for (int t = 0; t < nb; t++) {
      const int cw = hd[8 + 4 * t];
      const bool f32 = (cw >> 16) & 1;
      const int C = min(cw & 0xFFFF, 64), vs = min(hd[9 + 4 * t], 64);
      const int moff = min(hd[10 + 4 * t], kStageMat - 16) & ~15;
      const float scale = __int_as_float(hd[11 + 4 * t]);
      const int voff = min(hd[kHdVoff + t], VAREA - 16) & ~15;
      const uint16_t* A = reinterpret_cast<const uint16_t*>(stage + kMixedHeader + moff);
      const float* A32 = reinterpret_cast<const float*>(stage + kMixedHeader + moff);
      const float* X = reinterpret_cast<const float*>(stage + kMixedHeader + kStageMat + voff);
      const int G = (C + 3) >> 2;
      int first = hw - (base % HW);
      if (first < 0) first += HW;
      base += G;
      if (r0 >= R) continue;
      for (int grp = first; grp < G; grp += HW) {
        const int c = 4 * grp;
        float2 a[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int col = c + j;
          if (col >= C) {
            a[j] = make_float2(0.f, 0.f);
          } else if (f32) {
            a[j].x = A32[r0 + R * col];
            a[j].y = (r0 + 1 < R) ? A32[r0 + 1 + R * col] : 0.f;
          } else if (even) {
            a[j] = codes_to_f2<F>(*reinterpret_cast<const uint32_t*>(A + r0 + R * col));
          } else {
            a[j].x = code_to_f<F>(A[r0 + R * col]);
            a[j].y = (r0 + 1 < R) ? code_to_f<F>(A[r0 + 1 + R * col]) : 0.f;
          }
          if (kScaleCodes) {
            a[j].x *= scale;
            a[j].y *= scale;
          }
        }
        float p[2][NV2];
#pragma unroll
        for (int v = 0; v < NV2; v++) p[0][v] = p[1][v] = 0.f;
#pragma unroll
        for (int v = 0; v < NV2; v++) {
          const float4 x4 = *reinterpret_cast<const float4*>(X + v * vs + c);
          float* tgt0 = kScaleCodes ? &acc[0][v] : &p[0][v];
          float* tgt1 = kScaleCodes ? &acc[1][v] : &p[1][v];
          *tgt0 = fmaf(a[0].x, x4.x, *tgt0);
          *tgt1 = fmaf(a[0].y, x4.x, *tgt1);
          *tgt0 = fmaf(a[1].x, x4.y, *tgt0);
          *tgt1 = fmaf(a[1].y, x4.y, *tgt1);
          *tgt0 = fmaf(a[2].x, x4.z, *tgt0);
          *tgt1 = fmaf(a[2].y, x4.z, *tgt1);
          *tgt0 = fmaf(a[3].x, x4.w, *tgt0);
          *tgt1 = fmaf(a[3].y, x4.w, *tgt1);
        }
        if (!kScaleCodes)
#pragma unroll
          for (int v = 0; v < NV2; v++) {
            acc[0][v] = fmaf(scale, p[0][v], acc[0][v]);
            acc[1][v] = fmaf(scale, p[1][v], acc[1][v]);
          }
      }
    }
    return;
  }
  const int r0 = 2 * lane;
  for (int t = 0; t < nb; t++) {
    const int cw = hd[8 + 4 * t];
    const bool f32 = (cw >> 16) & 1, panel = (cw >> 17) & 1;
    const int C = min(cw & 0xFFFF, 64), vs = min(hd[9 + 4 * t], 64);
    // codes of rows r0, r0 + 1 in column c: lbase + cstr * c (16-bit units)
    const int lbase = panel ? (r0 >> 3) * (panel_stride(C) / 2) + (r0 & 7) : r0;
    const int cstr = panel ? 8 : R;
    const int moff = min(hd[10 + 4 * t], kStageMat - 16) & ~15;
    const float scale = __int_as_float(hd[11 + 4 * t]);
    const int voff = min(hd[kHdVoff + t], VAREA - 16) & ~15;
    const uint16_t* A = reinterpret_cast<const uint16_t*>(stage + kMixedHeader + moff);
    const float* A32 = reinterpret_cast<const float*>(stage + kMixedHeader + moff);
    const float* X = reinterpret_cast<const float*>(stage + kMixedHeader + kStageMat + voff);
    const int c0 = (C * warp) / CW, c1 = (C * (warp + 1)) / CW;
    float p[SETS][2][NV2];
#pragma unroll
    for (int u = 0; u < SETS; u++)
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int v = 0; v < NV2; v++) p[u][r][v] = 0.f;
    if (!f32 && R == 64 && C == 64 && vs == 64) {
      // full 64 x 64 block of codes: fixed strides, every column loaded up front
      constexpr int CPW = 64 / CW;
      const uint32_t* Aw = reinterpret_cast<const uint32_t*>(A + lbase + cstr * c0);
      uint32_t w[CPW];
#pragma unroll
      for (int u = 0; u < CPW; u++) w[u] = Aw[(cstr >> 1) * u];
#pragma unroll
      for (int v = 0; v < NV2; v++) {
        float xv[CPW];
#pragma unroll
        for (int u = 0; u < CPW; u += 4) {
          const float4 t4 = *reinterpret_cast<const float4*>(X + v * 64 + c0 + u);
          xv[u] = t4.x;
          xv[u + 1] = t4.y;
          xv[u + 2] = t4.z;
          xv[u + 3] = t4.w;
        }
#pragma unroll
        for (int u = 0; u < CPW; u++) {
          const float2 a = codes_to_f2<F>(w[u]);
          p[u % SETS][0][v] = fmaf(a.x, xv[u], p[u % SETS][0][v]);
          p[u % SETS][1][v] = fmaf(a.y, xv[u], p[u % SETS][1][v]);
        }
      }
    } else if (r0 < R) {
      const bool pair = panel || (R & 1) == 0;  // rows r0, r0 + 1 adjacent: one 4-byte load
      for (int col = c0; col < c1; col++) {
        float2 a;
        if (f32) {
          a.x = A32[r0 + R * col];
          a.y = (r0 + 1 < R) ? A32[r0 + 1 + R * col] : 0.f;
        } else if (pair) {
          a = codes_to_f2<F>(*reinterpret_cast<const uint32_t*>(A + lbase + cstr * col));
        } else {
          a.x = code_to_f<F>(A[r0 + R * col]);
          a.y = (r0 + 1 < R) ? code_to_f<F>(A[r0 + 1 + R * col]) : 0.f;
        }
#pragma unroll
        for (int v = 0; v < NV2; v++) {
          const float xv = X[v * vs + col];
          p[0][0][v] = fmaf(a.x, xv, p[0][0][v]);
          p[0][1][v] = fmaf(a.y, xv, p[0][1][v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV2; v++)
#pragma unroll
      for (int r = 0; r < 2; r++) {
        float sum = p[0][r][v];
#pragma unroll
        for (int u = 1; u < SETS; u++) sum += p[u][r][v];
        acc[r][v] = fmaf(scale, sum, acc[r][v]);
      }
  }
}

// Rows of more than 32 points with at most four vectors per product (the
// byte-bound case): lane (g, j) = (lane % 8, lane / 8) owns the eight rows
// 8g .. 8g + 7 and takes columns j, j + 4, ... of its warp's range, so that a
// full 64 x 64 block of codes costs a lane one 16-byte load per column
// (rows 8g .. 8g + 7 of a column are 16 contiguous bytes in both layouts),
// the block scale multiplies the lane's vector entries, and the codes feed
// the accumulators directly. Lanes sharing g meet at the row's end.
template <int F, int NV2, int NVB, int CW>
__device__ __forceinline__ void consume_item8(const unsigned char* stage, const int* hd, int nb, int R, int warp, int lane,
                                              float (&acc)[8][NVB]) {
  constexpr int VAREA = mixed_vec_area(NVB);
  constexpr int CPW = 64 / CW, CPL = CPW / 4;  // columns per warp and per lane of a full block
  static_assert(CPW % 4 == 0, "full blocks need a multiple of four columns per warp");
  const int g = lane & 7, j = lane >> 3;
  for (int t = 0; t < nb; t++) {
    const int4 bh = *reinterpret_cast<const int4*>(hd + 8 + 4 * t);  // cols | flags, vs, matrix offset, scale
    const bool f32 = (bh.x >> 16) & 1, panel = (bh.x >> 17) & 1;
    const int C = min(bh.x & 0xFFFF, 64), vs = min(bh.y, 64);
    const int moff = min(bh.z, kStageMat - 16) & ~15;
    const float scale = __int_as_float(bh.w);
    const int voff = min(hd[kHdVoff + t], VAREA - 16) & ~15;
    const unsigned char* A = stage + kMixedHeader + moff;
    const float* X = reinterpret_cast<const float*>(stage + kMixedHeader + kStageMat + voff);
    if (!f32 && R == 64 && C == 64 && vs == 64) {
      const int gb = panel ? g * panel_stride(64) : 16 * g;  // bytes: rows 8g .. 8g + 7
      const int cb = panel ? 16 : 128;                        // bytes per column
#pragma unroll
      for (int u = 0; u < CPL; u++) {
        const int c = CPW * warp + CPL * j + u;
        const uint4 w = *reinterpret_cast<const uint4*>(A + gb + cb * c);
        const float2 q0 = codes_to_f2<F>(w.x), q1 = codes_to_f2<F>(w.y), q2 = codes_to_f2<F>(w.z),
                     q3 = codes_to_f2<F>(w.w);
#pragma unroll
        for (int v = 0; v < NV2; v++) {
          const float xs = scale * X[v * 64 + c];
          acc[0][v] = fmaf(q0.x, xs, acc[0][v]);
          acc[1][v] = fmaf(q0.y, xs, acc[1][v]);
          acc[2][v] = fmaf(q1.x, xs, acc[2][v]);
          acc[3][v] = fmaf(q1.y, xs, acc[3][v]);
          acc[4][v] = fmaf(q2.x, xs, acc[4][v]);
          acc[5][v] = fmaf(q2.y, xs, acc[5][v]);
          acc[6][v] = fmaf(q3.x, xs, acc[6][v]);
          acc[7][v] = fmaf(q3.y, xs, acc[7][v]);
        }
      }
    } else {
      // any other block: element (row, col) at 16-bit unit row + R col (column-major) or
      // (row / 8) (panel stride / 2) + 8 col + row % 8 (panel layout); FP32 entries column-major
      const uint16_t* A16 = reinterpret_cast<const uint16_t*>(A);
      const float* A32 = reinterpret_cast<const float*>(A);
      const int c0 = (C * warp) / CW, c1 = (C * (warp + 1)) / CW;
      const int ps2 = panel_stride(C) / 2;
      for (int col = c0 + j; col < c1; col += 4) {
        float q[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int row = 8 * g + i;
          q[i] = 0.f;
          if (row < R)
            q[i] = f32 ? A32[row + R * col] : code_to_f<F>(A16[panel ? g * ps2 + 8 * col + i : row + R * col]);
        }
#pragma unroll
        for (int v = 0; v < NV2; v++) {
          const float xs = scale * X[v * vs + col];
#pragma unroll
          for (int i = 0; i < 8; i++) acc[i][v] = fmaf(q[i], xs, acc[i][v]);
        }
      }
    }
  }
}

// A uniform item (header word 4) in the eight-rows-per-lane layout: block t's
// codes at t * block bytes, its vector chunk at t * 64 nv floats, so a block
// costs a lane its 16-byte code loads (issued one block ahead), one scale and
// its vector entries.
template <int F, int NV2, int NVB, int CW>
__device__ __forceinline__ void consume_uniform8(const unsigned char* stage, const int* hd, int nb, int nv, bool panel,
                                                 int warp, int lane, float (&acc)[8][NVB]) {
  constexpr int CPW = 64 / CW, CPL = CPW / 4;
  const int g = lane & 7, j = lane >> 3, c0 = CPW * warp + CPL * j;
  const int bbytes = panel ? panel_block_bytes(64) : 64 * 64 * 2;
  const unsigned char* A = stage + kMixedHeader + (panel ? g * panel_stride(64) + 16 * c0 : 16 * g + 128 * c0);
  const int cb = panel ? 16 : 128;  // bytes per column
  const float* X = reinterpret_cast<const float*>(stage + kMixedHeader + kStageMat) + c0;
  uint4 w[CPL];
#pragma unroll
  for (int u = 0; u < CPL; u++) w[u] = *reinterpret_cast<const uint4*>(A + cb * u);
  for (int t = 0; t < nb; t++) {
    uint4 wn[CPL];
    const int tn = t + 1 < nb ? t + 1 : t;
#pragma unroll
    for (int u = 0; u < CPL; u++) wn[u] = *reinterpret_cast<const uint4*>(A + bbytes * tn + cb * u);
    const float scale = __int_as_float(hd[11 + 4 * t]);
    const float* Xt = X + t * 64 * nv;
#pragma unroll
    for (int u = 0; u < CPL; u++) {
      const float2 q0 = codes_to_f2<F>(w[u].x), q1 = codes_to_f2<F>(w[u].y), q2 = codes_to_f2<F>(w[u].z),
                   q3 = codes_to_f2<F>(w[u].w);
#pragma unroll
      for (int v = 0; v < NV2; v++) {
        const float xs = scale * Xt[v * 64 + u];
        acc[0][v] = fmaf(q0.x, xs, acc[0][v]);
        acc[1][v] = fmaf(q0.y, xs, acc[1][v]);
        acc[2][v] = fmaf(q1.x, xs, acc[2][v]);
        acc[3][v] = fmaf(q1.y, xs, acc[3][v]);
        acc[4][v] = fmaf(q2.x, xs, acc[4][v]);
        acc[5][v] = fmaf(q2.y, xs, acc[5][v]);
        acc[6][v] = fmaf(q3.x, xs, acc[6][v]);
        acc[7][v] = fmaf(q3.y, xs, acc[7][v]);
      }
    }
#pragma unroll
    for (int u = 0; u < CPL; u++) w[u] = wn[u];
  }
}

template <int F, int NVB, int CW>
__global__ void __launch_bounds__((CW + 1) * 32, 1) k_dense_stream_m(MixedStreamParams P) {
  constexpr int NST = mixed_stages(NVB, CW);
  constexpr int SB = mixed_stage_bytes(NVB);
  constexpr int VAREA = mixed_vec_area(NVB);
  static_assert(NST >= 2, "at least two stages");
  extern __shared__ __align__(1024) unsigned char smem[];
  const StreamShared S = stream_shared<NST, SB>(smem);
  // kAsyncRows (passes of at most four vectors): rows end without a CTA-wide barrier. Every warp
  // writes its partial sums into the row's half of the double-buffered red area and counts
  // itself in (cnt[row parity]); the warp that completes the count sums the partials, writes y,
  // resets the count and arrives on rowfree2[parity] (count 1), which a warp waits for before
  // it writes that half again. Wider passes share the row's sum among all warps between the
  // rowfull and rowfree barriers (count CW each).
  constexpr bool kAsyncRows = NVB <= 4;
  uint64_t* rowfree2 = S.rowfull;  // kAsyncRows: rowfree2[0], rowfree2[1] (the stream's two row barriers)
  int* cnt = const_cast<int*>(S.abort_flag) + 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; s++) {
      mbar_init(S.full + s, 1);
      mbar_init(S.empty + s, CW);
    }
    mbar_init(S.rowfull, kAsyncRows ? 1 : CW);
    mbar_init(S.rowfree, kAsyncRows ? 1 : CW);
    *S.abort_flag = 0;
    cnt[0] = cnt[1] = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const int ib = P.cta_begin[blockIdx.x], ie = P.cta_begin[blockIdx.x + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == CW) {
    // producer-private block records: smem after the row reduction buffer
    MixedBlock* blkbuf = reinterpret_cast<MixedBlock*>(smem + NST * SB + 256 + mixed_red_bytes(NVB, CW));
    mixed_produce<NST, SB, VAREA>(P, S, ib, ie, blkbuf);
    return;
  }
  StreamParams W{};
  W.err = P.err;
  W.budget = P.budget;
  float* red = reinterpret_cast<float*>(S.red);
  // kEight: rows of more than 32 points use the eight-rows-per-lane layout (consume_item8); the
  // other layouts keep their sums in the first two rows of acc
  constexpr bool kEight = NVB <= 4;
  constexpr int AR = kEight ? 8 : 2;
  float acc[AR][NVB];
#pragma unroll
  for (int r = 0; r < AR; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  float(&acc2)[2][NVB] = *reinterpret_cast<float(*)[2][NVB]>(&acc[0][0]);
  int rows_done = 0;
  for (int it = 0; it < ie - ib; it++) {
    const int st = it % NST, use = it / NST;
    if (!warp_wait(S.full + st, use & 1, W, S.abort_flag)) break;
    const unsigned char* stage = S.stage0 + st * SB;
    const int* hd = reinterpret_cast<const int*>(stage);
    const int R = min(hd[0], 64), nb = min(hd[1], kMixedMaxBlocks), row = hd[2], flags = hd[3];
    const int nv = min(hd[kHdNv], NVB);
    void* const ydst = reinterpret_cast<void*>(*reinterpret_cast<const unsigned long long*>(hd + kHdY));
    const bool y32 = hd[kHdXy32] != 0;
    const long long ldy = *reinterpret_cast<const long long*>(hd + kHdLdy);
    // the variant for the item's vector count (a matrix of a batch may take fewer than NVB)
    const bool eight = kEight && R > 32;
    if constexpr (kEight) {
      const int uni = hd[4];
      if (eight && (uni == 1 || uni == 2) && nb * 64 * nv <= kMixedVecCols * NVB) {
        const bool pnl = uni == 2;
        if (NVB >= 4 && nv > 2) consume_uniform8<F, (NVB >= 4 ? 4 : 1), NVB, CW>(stage, hd, nb, nv, pnl, warp, lane, acc);
        else if (NVB >= 2 && nv > 1) consume_uniform8<F, (NVB >= 2 ? 2 : 1), NVB, CW>(stage, hd, nb, nv, pnl, warp, lane, acc);
        else consume_uniform8<F, 1, NVB, CW>(stage, hd, nb, nv, pnl, warp, lane, acc);
      } else if (eight) {
        if (NVB >= 4 && nv > 2) consume_item8<F, (NVB >= 4 ? 4 : 1), NVB, CW>(stage, hd, nb, R, warp, lane, acc);
        else if (NVB >= 2 && nv > 1) consume_item8<F, (NVB >= 2 ? 2 : 1), NVB, CW>(stage, hd, nb, R, warp, lane, acc);
        else consume_item8<F, 1, NVB, CW>(stage, hd, nb, R, warp, lane, acc);
      }
    }
    if (!eight) {
      if (NVB >= 16 && nv > 8) consume_item<F, (NVB >= 16 ? 16 : 1), NVB, CW>(stage, hd, nb, R, warp, lane, acc2);
      else if (NVB >= 8 && nv > 4) consume_item<F, (NVB >= 8 ? 8 : 1), NVB, CW>(stage, hd, nb, R, warp, lane, acc2);
      else if (NVB >= 4 && nv > 2) consume_item<F, (NVB >= 4 ? 4 : 1), NVB, CW>(stage, hd, nb, R, warp, lane, acc2);
      else if (NVB >= 2 && nv > 1) consume_item<F, (NVB >= 2 ? 2 : 1), NVB, CW>(stage, hd, nb, R, warp, lane, acc2);
      else consume_item<F, 1, NVB, CW>(stage, hd, nb, R, warp, lane, acc2);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(S.empty + st);
    if (flags & kItemFlagLast) {
      const bool half = R <= 32;
      const int r0 = half ? 2 * (lane & 15) : 2 * lane;
      if (eight) {  // add the columns of the lanes that share the rows (lanes g, g + 8, g + 16, g + 24)
#pragma unroll
        for (int r = 0; r < AR; r++)
#pragma unroll
          for (int v = 0; v < NVB; v++) {
            acc[r][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[r][v], 8);
            acc[r][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[r][v], 16);
          }
      } else if (half) {  // add the other half-warp's columns
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
          for (int v = 0; v < NVB; v++) acc[r][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[r][v], 16);
      }
      const int par = kAsyncRows ? rows_done & 1 : 0;
      if (kAsyncRows) {
        // the half of red this row uses was last summed for row rows_done - 2
        if (rows_done >= 2 && !warp_wait(rowfree2 + par, ((rows_done >> 1) - 1) & 1, W, S.abort_flag)) break;
      } else if (rows_done > 0 && !warp_wait(S.rowfree, (rows_done - 1) & 1, W, S.abort_flag)) {
        break;
      }
      float* redp = red + par * (CW * NVB * 64);
      if (eight) {
        if (lane < 8)
#pragma unroll
          for (int v = 0; v < NVB; v++)
            if (v < nv) {
              float4* dst = reinterpret_cast<float4*>(redp + (warp * NVB + v) * 64 + 8 * lane);
              dst[0] = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
              dst[1] = make_float4(acc[4][v], acc[5][v], acc[6][v], acc[7][v]);
            }
      } else if (!half || lane < 16) {
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
          for (int v = 0; v < NVB; v++)
            if (v < nv) redp[(warp * NVB + v) * 64 + r0 + r] = acc[r][v];
      }
#pragma unroll
      for (int r = 0; r < AR; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
      __syncwarp();
      if (!kAsyncRows) {
        if (lane == 0) mbar_arrive(S.rowfull);
        if (!warp_wait(S.rowfull, rows_done & 1, W, S.abort_flag)) break;
        for (int idx = threadIdx.x; idx < R * nv; idx += CW * 32) {
          const int r = idx % R, v = idx / R;
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < CW; w++) sum += red[(w * NVB + v) * 64 + r];
          y_store(ydst, y32, v * ldy + row + r, sum, false);  // y was zeroed or assigned; the other part adds too
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(S.rowfree);
        rows_done++;
        continue;
      }
      int last = 0;
      if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(cnt + par, 1) == CW - 1;
      }
      last = __shfl_sync(0xFFFFFFFFu, last, 0);
      if (last) {  // every warp's partials of this row are in: sum them and write y
        __threadfence_block();
        for (int idx = lane; idx < R * nv; idx += 32) {
          const int r = idx % R, v = idx / R;
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < CW; w++) sum += redp[(w * NVB + v) * 64 + r];
          y_store(ydst, y32, v * ldy + row + r, sum, false);  // y was zeroed or assigned; the other part adds too
        }
        __syncwarp();
        if (lane == 0) {
          cnt[par] = 0;
          mbar_arrive(rowfree2 + par);
        }
      }
      rows_done++;
    }
  }
}

// ---------------------------------------------------------------- split x and leaf expansion
// Per leaf row of every matrix of the launch: its matrix, leaf, the block
// record of U_i and where U_i's codes are, and whether the dense phase writes
// the row. The two kernels below run over this list; a product then runs its
// tree phases (which need x4 first) concurrently with the dense phase (which
// needs x4 too, and no tree result), and adds U_i yhat_i (Eq. 4) at the end.


// x4(j) = FP32 copy of x(j), padded with zeros to a multiple of 4 per vector, and (zero_y) y(j) = 0
// for the products whose dense phase and leaf expansion add their parts into y; one warp per row
// job (one instance per storage format: each format's launch unit has its own)
template <int F>
__global__ void __launch_bounds__(256) k_split_x4(const MatDesc* __restrict__ mats, const RowJob* __restrict__ jobs,
                                                  int64_t njobs, int zero_y) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < njobs; w += nw) {
    const RowJob J = jobs[w];
    const MatDesc& D = mats[J.mat];
    const int nv = D.nv;
    if (nv <= 0) continue;
    const int64_t off = D.leaf_off[J.leaf];
    const int sj = (int)(D.leaf_off[J.leaf + 1] - off), spad = (sj + 3) & ~3;
    float* xj = D.x4 + D.xp4_off[J.leaf] * nv;
    const bool xy32 = D.xy32 != 0;
#pragma unroll 4
    for (int v = 0; v < nv; v++) {
      // leaf sizes <= 64: two entries per lane
      const float x0 = lane < sj ? x_load(D.x, xy32, off + v * D.ldx + lane) : 0.f;
      const float x1 = lane + 32 < sj ? x_load(D.x, xy32, off + v * D.ldx + lane + 32) : 0.f;
      if (lane < spad) xj[v * spad + lane] = x0;
      if (lane + 32 < spad) xj[v * spad + lane + 32] = x1;
      if (zero_y) {
        if (lane < sj) y_store(D.y, xy32, off + v * D.ldy + lane, 0.f, true);
        if (lane + 32 < sj) y_store(D.y, xy32, off + v * D.ldy + lane + 32, 0.f, true);
      }
    }
  }
}

}  // namespace h2
