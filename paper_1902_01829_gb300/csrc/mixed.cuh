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
  return make_float2(__uint_as_float(0x4B000000u | (w & 0xFFFFu)) - 8421376.0f,
                     __uint_as_float(0x4B000000u | (w >> 16)) - 8421376.0f);
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
  int k, kp, LR, q, L, nv;
};

constexpr int kTreeWarpsM = 8;

template <int F, int RPL, int NVB>
__device__ __forceinline__ void project_leaf_m(const TreeParamsM& P, int64_t j, int lane) {
  const int64_t leaf0 = ((int64_t)1 << P.q) - 1;
  const int64_t off = P.leaf_off[j];
  const int sj = (int)(P.leaf_off[j + 1] - off);
  const int spad = (sj + 3) & ~3;
  float* xj = P.x4 + P.xp4_off[j] * P.nv;
  for (int v = 0; v < P.nv; v++)
    for (int a = lane; a < sj; a += 32) xj[v * spad + a] = __double2float_rn(P.x[v * P.ldx + off + a]);
  __syncwarp();
  float acc[RPL][NVB];
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.Vt) + P.vt_off[j], P.vscale[j], P.k, sj, P.LR, xj,
                         spad, P.nv, acc, lane);
  group_reduce_m(acc, P.LR);
  store_node_m<RPL, NVB, false>(P.xhat + (leaf0 + j) * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, acc, lane);
}

template <int F, int RPL, int NVB, bool CG>
__device__ __forceinline__ void up_node_m(const TreeParamsM& P, int64_t p, int lane) {
  float acc[RPL][NVB];
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  for (int ci = 1; ci <= 2; ci++) {
    const int64_t ch = 2 * p + ci;
    const float* xc = P.xhat + ch * P.nv * P.kp;
    if (CG) {  // the sibling subtree was written by another CTA: read it through L2
      __shared__ float tmp[kTreeWarpsM][16 * 64];
      float* t = tmp[threadIdx.x >> 5];
      for (int i = lane; i < P.nv * P.kp; i += 32) t[i] = __ldcg(xc + i);
      __syncwarp();
      warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.Ft) + (ch - 1) * P.kk8, P.fscale[ch - 1], P.k,
                             P.k, P.LR, t, P.kp, P.nv, acc, lane);
      __syncwarp();
    } else {
      warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.Ft) + (ch - 1) * P.kk8, P.fscale[ch - 1], P.k,
                             P.k, P.LR, xc, P.kp, P.nv, acc, lane);
    }
  }
  group_reduce_m(acc, P.LR);
  store_node_m<RPL, NVB, false>(P.xhat + p * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, acc, lane);
}

// leaf projection + the whole upsweep in one launch (see k_upsweep_tree)
template <int F, int RPL, int NVB>
__global__ void __launch_bounds__(kTreeWarpsM * 32) k_upsweep_tree_m(TreeParamsM P) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = P.q - P.L;
  const int64_t sub = blockIdx.x;
  for (int64_t t = warp; t < ((int64_t)1 << T); t += kTreeWarpsM) project_leaf_m<F, RPL, NVB>(P, (sub << T) + t, lane);
  __syncthreads();
  for (int lvl = P.q - 1; lvl >= P.L; lvl--) {
    const int64_t node0 = ((int64_t)1 << lvl) - 1 + (sub << (lvl - P.L));
    for (int64_t t = warp; t < ((int64_t)1 << (lvl - P.L)); t += kTreeWarpsM)
      up_node_m<F, RPL, NVB, false>(P, node0 + t, lane);
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (warp != 0) return;
  int64_t node = ((int64_t)1 << P.L) - 1 + sub;
  while (node > 0) {
    const int64_t par = (node - 1) / 2;
    int second = 0;
    if (lane == 0) {
      second = atomicAdd(P.ticket + par, 1) == 1;
      if (second) P.ticket[par] = 0;
    }
    second = __shfl_sync(0xFFFFFFFFu, second, 0);
    if (!second) break;
    __threadfence();
    up_node_m<F, RPL, NVB, true>(P, par, lane);
    __threadfence();
    __syncwarp();
    node = par;
  }
}

// the whole downsweep in one launch (see k_downsweep_tree)
template <int F, int RPL, int NVB>
__global__ void __launch_bounds__(kTreeWarpsM * 32) k_downsweep_tree_m(TreeParamsM P) {
  __shared__ float path[2][NVB][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t sub = blockIdx.x;
  const int64_t root = ((int64_t)1 << P.L) - 1 + sub;
  if (warp == 0 && P.L > 0) {
    int cur = 0;
    for (int v = 0; v < P.nv; v++)
      for (int r = lane; r < P.k; r += 32) path[cur][v][r] = P.yhat[(int64_t)v * P.kp + r];
    __syncwarp();
    for (int l = 1; l <= P.L; l++) {
      const int64_t a = ((root + 1) >> (P.L - l)) - 1;
      float acc[RPL][NVB];
#pragma unroll
      for (int r = 0; r < RPL; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
      warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.E) + (a - 1) * P.kk8, P.escale[a - 1], P.k, P.k,
                             P.LR, &path[cur][0][0], 64, P.nv, acc, lane);
      group_reduce_m(acc, P.LR);
      if (lane < P.LR) {
#pragma unroll
        for (int rr = 0; rr < RPL; rr++) {
          const int row = lane + 32 * rr;
          if (row >= P.k) continue;
#pragma unroll
          for (int v = 0; v < NVB; v++) {
            if (v >= P.nv) continue;
            const float val = acc[rr][v] + P.yhat[(a * P.nv + v) * P.kp + row];
            if (l == P.L) P.yhat[(a * P.nv + v) * P.kp + row] = val;
            else path[cur ^ 1][v][row] = val;
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
    for (int64_t t = warp; t < ((int64_t)1 << (lvl - P.L)); t += kTreeWarpsM) {
      const int64_t ch = node0 + t;
      float acc[RPL][NVB];
#pragma unroll
      for (int r = 0; r < RPL; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
      warp_mv_m<F, RPL, NVB>(static_cast<const typename CodeT<F>::T*>(P.E) + (ch - 1) * P.kk8, P.escale[ch - 1], P.k,
                             P.k, P.LR, P.yhat + ((ch - 1) / 2) * P.nv * P.kp, P.kp, P.nv, acc, lane);
      group_reduce_m(acc, P.LR);
      store_node_m<RPL, NVB, true>(P.yhat + ch * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, acc, lane);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- coupling, all levels
// One warp per node row. k = 4 * H with H a power of two (k = 4 .. 64): lane
// = g * H + h owns rows 4h .. 4h + 3, read as one 8-byte load per column;
// column groups g = 0 .. G-1 (G = 32 / H) take columns g, g + G, ... The
// row's (block, column) slots are walked CB at a time, two batches in
// flight; a block's partial sum is scaled once, after its last column.
// Blocks are padded to kk8 codes.
template <int F, int NVB, int CB>
__global__ void __launch_bounds__(128) k_coupling_m(const uint16_t* __restrict__ S, const float* __restrict__ sscale,
                                                   int64_t kk8, const int32_t* __restrict__ Srow,
                                                   const int32_t* __restrict__ Scol, int k, int kp, int64_t n_nodes,
                                                   int nv, const float* __restrict__ xhat, float* __restrict__ yhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 4 + warp;
  if (i >= n_nodes) return;
  const int H = k >> 2, G = 32 / H;
  const int g = lane / H, h = lane - g * H;
  const int cpl = max(1, k / G);  // columns per lane per block, a power of two (lanes with col >= k idle)
  const int lcpl = __ffs(cpl) - 1;
  const int32_t b0 = Srow[i];
  const int nslot = (Srow[i + 1] - b0) * cpl;
  float acc[4][NVB], p[4][NVB];
#pragma unroll
  for (int r = 0; r < 4; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = p[r][v] = 0.f;
  uint2 a0[CB], a1[CB];
  float x0[CB][NVB], x1[CB][NVB], s0[CB], s1[CB];
  auto load = [&](int bt, uint2(&a)[CB], float(&xv)[CB][NVB], float(&sc)[CB]) {
#pragma unroll
    for (int u = 0; u < CB; u++) {
      const int slot = bt * CB + u;
      const int b = slot >> lcpl, c = slot & (cpl - 1);
      const int col = g + G * c;
      const bool ok = slot < nslot && col < k;
      sc[u] = 0.f;
      a[u] = make_uint2(0u, 0u);
#pragma unroll
      for (int v = 0; v < NVB; v++) xv[u][v] = 0.f;
      if (slot < nslot) {
        sc[u] = __ldg(sscale + b0 + b);
        if (ok) {
          a[u] = __ldg(reinterpret_cast<const uint2*>(S + (int64_t)(b0 + b) * kk8 + 4 * h + k * col));
          const float* X = xhat + (int64_t)__ldg(Scol + b0 + b) * nv * kp;
#pragma unroll
          for (int v = 0; v < NVB; v++) xv[u][v] = (v < nv) ? __ldg(X + v * kp + col) : 0.f;
        }
      }
    }
  };
  auto compute = [&](int bt, const uint2(&a)[CB], const float(&xv)[CB][NVB], const float(&sc)[CB]) {
#pragma unroll
    for (int u = 0; u < CB; u++) {
      const int slot = bt * CB + u;
      const float2 lo = codes_to_f2<F>(a[u].x), hi = codes_to_f2<F>(a[u].y);
#pragma unroll
      for (int v = 0; v < NVB; v++) {
        p[0][v] = fmaf(lo.x, xv[u][v], p[0][v]);
        p[1][v] = fmaf(lo.y, xv[u][v], p[1][v]);
        p[2][v] = fmaf(hi.x, xv[u][v], p[2][v]);
        p[3][v] = fmaf(hi.y, xv[u][v], p[3][v]);
      }
      if (slot < nslot && (slot & (cpl - 1)) == cpl - 1) {  // last column of a block: scale its partial sum
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
          for (int v = 0; v < NVB; v++) {
            acc[r][v] = fmaf(sc[u], p[r][v], acc[r][v]);
            p[r][v] = 0.f;
          }
      }
    }
  };
  const int nbatch = (nslot + CB - 1) / CB;
  if (nbatch > 0) load(0, a0, x0, s0);
  for (int bt = 0; bt < nbatch; bt += 2) {
    if (bt + 1 < nbatch) load(bt + 1, a1, x1, s1);
    compute(bt, a0, x0, s0);
    if (bt + 2 < nbatch) load(bt + 2, a0, x0, s0);
    if (bt + 1 < nbatch) compute(bt + 1, a1, x1, s1);
  }
  for (int off = H; off < 32; off <<= 1)
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
      for (int v = 0; v < NVB; v++) acc[r][v] += __shfl_xor_sync(0xFFFFFFFFu, acc[r][v], off);
  if (g == 0) {
    float* dst = yhat + i * nv * kp;
#pragma unroll
    for (int v = 0; v < NVB; v++)
      if (v < nv)
#pragma unroll
        for (int r = 0; r < 4; r++) dst[v * kp + 4 * h + r] = acc[r][v];
  }
}

// any other k: generic row mapping, one block at a time
template <int F, int RPL, int NVB>
__global__ void __launch_bounds__(128) k_coupling_m_generic(const uint16_t* __restrict__ S,
                                                           const float* __restrict__ sscale, int64_t kk8,
                                                           const int32_t* __restrict__ Srow,
                                                           const int32_t* __restrict__ Scol, int k, int kp, int LR,
                                                           int64_t n_nodes, int nv, const float* __restrict__ xhat,
                                                           float* __restrict__ yhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 4 + warp;
  if (i >= n_nodes) return;
  float acc[RPL][NVB];
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  for (int32_t b = Srow[i]; b < Srow[i + 1]; b++)
    warp_mv_m<F, RPL, NVB>(S + (int64_t)b * kk8, sscale[b], k, k, LR, xhat + (int64_t)Scol[b] * nv * kp, kp, nv, acc,
                           lane);
  group_reduce_m(acc, LR);
  store_node_m<RPL, NVB, false>(yhat + i * nv * kp, k, kp, LR, nv, acc, lane);
}

// ---------------------------------------------------------------- dense near field + expansion (TMA stream)
// Per-block side information of the dense stream, 16 bytes.
struct __align__(16) MixedBlock {
  long long voff;       // vector chunk offset, in floats per vector slot
  float scale;
  unsigned short cols;  // C
  unsigned char vs;     // vector stride (>= C, multiple of 4)
  unsigned char src;    // bit 0: vector from the second source (yhat); bit 1: FP32 entries (not codes)
};

constexpr int kMixedMaxBlocks = 4;   // blocks of one row per work item
constexpr int kMixedHeader = 256;
__host__ __device__ constexpr int mixed_vec_slot(int nvb) { return 64 * nvb * 4; }
__host__ __device__ constexpr int mixed_stage_bytes(int nvb) {
  return kMixedHeader + kStageMat + kMixedMaxBlocks * mixed_vec_slot(nvb);
}
__host__ __device__ constexpr int mixed_red_bytes(int nvb, int cw) { return cw * nvb * 64 * 4; }
constexpr int kMixedBlkBuf = 32 * 4 * 16;  // block records of one producer batch (32 items x 4 blocks)
__host__ __device__ constexpr int mixed_stages(int nvb, int cw) {
  return (kSmemLimit - 256 - kMixedBlkBuf - mixed_red_bytes(nvb, cw)) / mixed_stage_bytes(nvb) < 6
             ? (kSmemLimit - 256 - kMixedBlkBuf - mixed_red_bytes(nvb, cw)) / mixed_stage_bytes(nvb)
             : 6;
}
__host__ __device__ constexpr int mixed_smem_bytes(int nvb, int cw) {
  return mixed_stages(nvb, cw) * mixed_stage_bytes(nvb) + 256 + mixed_red_bytes(nvb, cw) + kMixedBlkBuf;
}
constexpr int kMixedCW = 8;

struct MixedStreamParams {
  const StreamItem* items;  // m_off, m_bytes, shape = R | nb << 8, v_off = first block, row = y offset, flags
  const int* cta_begin;
  const char* mat;
  const MixedBlock* blk;
  const float* vsrc0;       // FP32 x (padded leaf layout)
  const float* vsrc1;       // yhat
  int nv;
  double* y;
  long long ldy;
  int* err;
  long long budget;
};

// Stage header: [0] R, [1] nb, [2] row, [3] flags; block t at int index 8 + 4 t:
// cols | FP32-entries flag << 16, vs, matrix offset in bytes, scale (bits).
template <int NST, int SB, int VSLOT>
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
    const int nbatch = (int)min(blast - bfirst, (long long)(32 * kMixedMaxBlocks));
    for (int u = lane; u < nbatch; u += 32) blkbuf[u] = P.blk[bfirst + u];
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
      unsigned char* stage = S.stage0 + s * SB;
      int* hd = reinterpret_cast<int*>(stage);
      // per-block side information, one lane per block
      MixedBlock mb{};
      const long long bi = b0 - bfirst + lane;
      if (lane < nb && bi >= 0 && bi < nbatch) mb = blkbuf[bi];
      const int esize = (mb.src & 2) ? 4 : 2;
      const int codes = (R * (int)mb.cols * esize + 15) & ~15;  // padded bytes of this block
      int moff = codes;  // inclusive prefix of the blocks' padded byte counts
#pragma unroll
      for (int d = 1; d < kMixedMaxBlocks; d <<= 1) {
        const int o = __shfl_up_sync(0xFFFFFFFFu, moff, d);
        if (lane >= d) moff += o;
      }
      moff -= codes;
      unsigned vbytes = (lane < nb) ? (unsigned)(P.nv * (int)mb.vs * 4) : 0u;
      unsigned vtot = vbytes;
#pragma unroll
      for (int d = 1; d < kMixedMaxBlocks; d <<= 1) vtot += __shfl_xor_sync(0xFFFFFFFFu, vtot, d);
      if (lane < nb) {
        hd[8 + 4 * lane] = mb.cols | ((mb.src & 2) << 15);
        hd[9 + 4 * lane] = mb.vs;
        hd[10 + 4 * lane] = moff;
        hd[11 + 4 * lane] = __float_as_int(mb.scale);
      }
      if (lane == 0) {
        hd[0] = R;
        hd[1] = nb;
        hd[2] = row;
        hd[3] = flags;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_expect_tx(S.full + s, (unsigned)m_bytes + vtot);
        bulk_g2s_stream(stage + kMixedHeader, P.mat + (((unsigned long long)m_hi << 32) | m_lo), (unsigned)m_bytes,
                        S.full + s, pol);
      }
      __syncwarp();
      if (lane < nb) {
        const float* src = mb.src ? P.vsrc1 : P.vsrc0;
        bulk_g2s(stage + kMixedHeader + kStageMat + lane * VSLOT, src + mb.voff * P.nv, vbytes, S.full + s);
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

template <int F, int NVB, int CW>
__global__ void __launch_bounds__((CW + 1) * 32, 1) k_dense_stream_m(MixedStreamParams P) {
  constexpr int NST = mixed_stages(NVB, CW);
  constexpr int SB = mixed_stage_bytes(NVB);
  constexpr int VSLOT = mixed_vec_slot(NVB);
  constexpr int SETS = NVB == 1 ? 4 : (NVB == 2 ? 2 : 1);
  static_assert(NST >= 2, "at least two stages");
  extern __shared__ __align__(1024) unsigned char smem[];
  const StreamShared S = stream_shared<NST, SB>(smem);
  stream_init<NST, CW>(S);
  const int ib = P.cta_begin[blockIdx.x], ie = P.cta_begin[blockIdx.x + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == CW) {
    // producer-private block records: smem after the row reduction buffer
    MixedBlock* blkbuf = reinterpret_cast<MixedBlock*>(smem + NST * SB + 256 + mixed_red_bytes(NVB, CW));
    mixed_produce<NST, SB, VSLOT>(P, S, ib, ie, blkbuf);
    return;
  }
  StreamParams W{};
  W.err = P.err;
  W.budget = P.budget;
  float* red = reinterpret_cast<float*>(S.red);
  const int nv = P.nv;
  float acc[2][NVB];
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) acc[r][v] = 0.f;
  const int r0 = 2 * lane;
  int rows_done = 0;
  for (int it = 0; it < ie - ib; it++) {
    const int st = it % NST, use = it / NST;
    if (!warp_wait(S.full + st, use & 1, W, S.abort_flag)) break;
    const unsigned char* stage = S.stage0 + st * SB;
    const int* hd = reinterpret_cast<const int*>(stage);
    const int R = min(hd[0], 64), nb = min(hd[1], kMixedMaxBlocks), row = hd[2], flags = hd[3];
    for (int t = 0; t < nb; t++) {
      const int cw = hd[8 + 4 * t];
      const bool f32 = (cw >> 16) & 1;
      const int C = min(cw & 0xFFFF, 64), vs = min(hd[9 + 4 * t], 64);
      const int moff = min(hd[10 + 4 * t], kStageMat - 16) & ~15;
      const float scale = __int_as_float(hd[11 + 4 * t]);
      const uint16_t* A = reinterpret_cast<const uint16_t*>(stage + kMixedHeader + moff);
      const float* A32 = reinterpret_cast<const float*>(stage + kMixedHeader + moff);
      const float* X = reinterpret_cast<const float*>(stage + kMixedHeader + kStageMat + t * VSLOT);
      const int c0 = (C * warp) / CW, c1 = (C * (warp + 1)) / CW;
      float p[SETS][2][NVB];
#pragma unroll
      for (int u = 0; u < SETS; u++)
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
          for (int v = 0; v < NVB; v++) p[u][r][v] = 0.f;
      if (!f32 && R == 64 && C == 64 && vs == 64) {
        // full 64 x 64 block of codes: fixed strides, every column loaded up front
        constexpr int CPW = 64 / CW;
        const uint32_t* Aw = reinterpret_cast<const uint32_t*>(A + r0 + 64 * c0);
        uint32_t w[CPW];
#pragma unroll
        for (int u = 0; u < CPW; u++) w[u] = Aw[32 * u];
#pragma unroll
        for (int v = 0; v < NVB; v++) {
          if (v >= nv) continue;
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
        const bool even = (R & 1) == 0;
        for (int col = c0; col < c1; col++) {
          float2 a;
          if (f32) {
            a.x = A32[r0 + R * col];
            a.y = (r0 + 1 < R) ? A32[r0 + 1 + R * col] : 0.f;
          } else if (even) {
            a = codes_to_f2<F>(*reinterpret_cast<const uint32_t*>(A + r0 + R * col));
          } else {
            a.x = code_to_f<F>(A[r0 + R * col]);
            a.y = (r0 + 1 < R) ? code_to_f<F>(A[r0 + 1 + R * col]) : 0.f;
          }
#pragma unroll
          for (int v = 0; v < NVB; v++) {
            const float xv = (v < nv) ? X[v * vs + col] : 0.f;
            p[0][0][v] = fmaf(a.x, xv, p[0][0][v]);
            p[0][1][v] = fmaf(a.y, xv, p[0][1][v]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) {
          float sum = p[0][r][v];
#pragma unroll
          for (int u = 1; u < SETS; u++) sum += p[u][r][v];
          acc[r][v] = fmaf(scale, sum, acc[r][v]);
        }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(S.empty + st);
    if (flags & kItemFlagLast) {
      if (rows_done > 0 && !warp_wait(S.rowfree, (rows_done - 1) & 1, W, S.abort_flag)) break;
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) {
          red[(warp * NVB + v) * 64 + r0 + r] = acc[r][v];
          acc[r][v] = 0.f;
        }
      __syncwarp();
      if (lane == 0) mbar_arrive(S.rowfull);
      if (!warp_wait(S.rowfull, rows_done & 1, W, S.abort_flag)) break;
      for (int idx = threadIdx.x; idx < R * nv; idx += CW * 32) {
        const int r = idx % R, v = idx / R;
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < CW; w++) sum += red[(w * NVB + v) * 64 + r];
        P.y[v * P.ldy + row + r] = (double)sum;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(S.rowfree);
      rows_done++;
    }
  }
}

}  // namespace h2
