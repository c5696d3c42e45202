// FP64 plain-form kernels of the H^2 matrix-vector product (Sec. 4), one per phase.
//
// Every phase is a sum of column-major block products "rows += A_block * x_cols":
//   leaf projection  xhat_j  = V_j^T x(j)            A = V_j^T (stored transposed)
//   upsweep          xhat_p  = sum_c F_c^T xhat_c    A = F_c^T (stored transposed)   Eq. 2
//   coupling         yhat_i  = sum_j S_ij xhat_j     A = S_ij                        Eq. 3
//   downsweep        yhat_c += E_c yhat_p            A = E_c                         Eq. 5
//   dense + expand   y(i)    = U_i yhat_i + sum_j D_ij x(j)                          Eq. 4, Sec. 2.2
// so one warp routine serves all of them: a lane owns output rows, consecutive
// lanes read consecutive rows of a column (coalesced), the input vector entry
// of the column is a broadcast, and products accumulate in double-float.
//
// Workspace layouts (float2 = double-float hi, lo):
//   x2    [v * ld2 + point]              the pass's x, split once
//   xhat  [(node * nv + v) * k + row]    vector trees of Sec. 4.2 - 4.4
//   yhat  same as xhat
#pragma once
#include "df64.cuh"

namespace h2 {

constexpr int kWarps = 4;  // warps per CTA for the per-node kernels

// Row mapping of a warp over an R-row block: lane = g * LR + rl owns rows
// rl + 32 r (r < RPL) and columns col = g, g + G, ... with G = 32 / LR groups.
// RPL = 2 requires LR = 32 (R <= 64); RPL = 1 allows LR = 1 .. 32 (R <= LR).
template <int RPL, int NVB>
__device__ __forceinline__ void warp_mv(const double* __restrict__ A, int R, int C, int LR,
                                        const float2* xin, int64_t xstride, int nv,
                                        float (&s)[RPL][NVB], float (&c)[RPL][NVB], int lane) {
  const int G = 32 / LR;
  const int g = lane / LR, rl = lane - g * LR;
  for (int col = g; col < C; col += G) {
    float xh[NVB], xl[NVB];
#pragma unroll
    for (int v = 0; v < NVB; v++) {
      const float2 t = (v < nv) ? xin[v * xstride + col] : make_float2(0.f, 0.f);
      xh[v] = t.x;
      xl[v] = t.y;
    }
#pragma unroll
    for (int r = 0; r < RPL; r++) {
      const int row = rl + 32 * r;
      if (row < R) {
        float ah, al;
        split_f64(__ldg(A + row + (int64_t)R * col), ah, al);
#pragma unroll
        for (int v = 0; v < NVB; v++) df_fma(s[r][v], c[r][v], ah, al, xh[v], xl[v]);
      }
    }
  }
}

template <int RPL, int NVB>
__device__ __forceinline__ void acc_zero(float (&s)[RPL][NVB], float (&c)[RPL][NVB]) {
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) s[r][v] = c[r][v] = 0.f;
}

// sum the partial results of the G column groups (lanes rl, rl + LR, ...)
template <int RPL, int NVB>
__device__ __forceinline__ void group_reduce(float (&s)[RPL][NVB], float (&c)[RPL][NVB], int LR) {
  for (int off = LR; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < RPL; r++)
#pragma unroll
      for (int v = 0; v < NVB; v++) {
        const float s2 = __shfl_xor_sync(0xFFFFFFFFu, s[r][v], off);
        const float c2 = __shfl_xor_sync(0xFFFFFFFFu, c[r][v], off);
        df_add(s[r][v], c[r][v], s2, c2);
      }
  }
}

// write rows of a node vector (k x nv) from lanes of group 0; optionally add the old value
template <int RPL, int NVB, bool ACCUM>
__device__ __forceinline__ void store_node(float2* __restrict__ dst, int k, int LR, int nv,
                                           float (&s)[RPL][NVB], float (&c)[RPL][NVB], int lane) {
  if (lane >= LR) return;
#pragma unroll
  for (int r = 0; r < RPL; r++) {
    const int row = lane + 32 * r;
    if (row >= k) continue;
#pragma unroll
    for (int v = 0; v < NVB; v++) {
      if (v >= nv) continue;
      float ss = s[r][v], cc = c[r][v];
      if (ACCUM) {
        const float2 old = dst[v * k + row];
        df_add(ss, cc, old.x, old.y);
      }
      dst[v * k + row] = df_norm(ss, cc);
    }
  }
}

// ---------------------------------------------------------------- leaf projection
// one warp per leaf: x2(j) = split(x(j)); xhat_j = V_j^T x(j)   (Alg. 2, first step)
template <int RPL, int NVB>
__global__ void __launch_bounds__(kWarps * 32) k_project(const double* __restrict__ Vt, const int64_t* __restrict__ leaf_off,
                                                       int k, int LR, int64_t leaves, int64_t leaf0,
                                                       const double* __restrict__ x, int64_t ldx, int nv,
                                                       float2* __restrict__ x2, int64_t ld2, float2* __restrict__ xhat) {
  __shared__ float2 xs[kWarps][NVB][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kWarps + warp;
  if (j >= leaves) return;
  const int64_t off = leaf_off[j];
  const int sj = (int)(leaf_off[j + 1] - off);
  for (int v = 0; v < nv; v++)
    for (int a = lane; a < sj; a += 32) {
      const float2 t = f64_to_df(x[v * ldx + off + a]);
      xs[warp][v][a] = t;
      x2[v * ld2 + off + a] = t;
    }
  __syncwarp();
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  warp_mv<RPL, NVB>(Vt + off * k, k, sj, LR, &xs[warp][0][0], 64, nv, s, c, lane);
  group_reduce(s, c, LR);
  store_node<RPL, NVB, false>(xhat + (leaf0 + j) * nv * k, k, LR, nv, s, c, lane);
}

// ---------------------------------------------------------------- upsweep, one level
// one warp per parent p on level l-1: xhat_p = F_c1^T xhat_c1 + F_c2^T xhat_c2   (Eq. 2)
template <int RPL, int NVB>
__global__ void __launch_bounds__(kWarps * 32) k_upsweep(const double* __restrict__ Ft, int k, int LR, int64_t pfirst,
                                                       int64_t pcount, int nv, float2* __restrict__ xhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * kWarps + warp;
  if (t >= pcount) return;
  const int64_t p = pfirst + t;
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  for (int ci = 1; ci <= 2; ci++) {
    const int64_t ch = 2 * p + ci;
    warp_mv<RPL, NVB>(Ft + (ch - 1) * k * k, k, k, LR, xhat + ch * nv * k, k, nv, s, c, lane);
  }
  group_reduce(s, c, LR);
  store_node<RPL, NVB, false>(xhat + p * nv * k, k, LR, nv, s, c, lane);
}

// ---------------------------------------------------------------- coupling, all levels
// one warp per node row i: yhat_i = sum_{b in row i} S_b xhat_{col(b)}   (Eq. 3, Alg. 3)
template <int RPL, int NVB>
__global__ void __launch_bounds__(kWarps * 32) k_coupling(const double* __restrict__ S, const int32_t* __restrict__ Srow,
                                                        const int32_t* __restrict__ Scol, int k, int LR, int64_t n_nodes,
                                                        int nv, const float2* __restrict__ xhat, float2* __restrict__ yhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  if (i >= n_nodes) return;
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  const int32_t b0 = Srow[i], b1 = Srow[i + 1];
  for (int32_t b = b0; b < b1; b++)
    warp_mv<RPL, NVB>(S + (int64_t)b * k * k, k, k, LR, xhat + (int64_t)Scol[b] * nv * k, k, nv, s, c, lane);
  group_reduce(s, c, LR);
  store_node<RPL, NVB, false>(yhat + i * nv * k, k, LR, nv, s, c, lane);
}

// ---------------------------------------------------------------- downsweep, one level
// one warp per node c on level l: yhat_c += E_c yhat_parent   (Eq. 5, Alg. 4)
template <int RPL, int NVB>
__global__ void __launch_bounds__(kWarps * 32) k_downsweep(const double* __restrict__ E, int k, int LR, int64_t cfirst,
                                                         int64_t ccount, int nv, float2* __restrict__ yhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * kWarps + warp;
  if (t >= ccount) return;
  const int64_t ch = cfirst + t, par = (ch - 1) / 2;
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  warp_mv<RPL, NVB>(E + (ch - 1) * k * k, k, k, LR, yhat + par * nv * k, k, nv, s, c, lane);
  group_reduce(s, c, LR);
  store_node<RPL, NVB, true>(yhat + ch * nv * k, k, LR, nv, s, c, lane);
}

// ---------------------------------------------------------------- dense near field + leaf expansion
// one CTA per leaf row i: y(i) = U_i yhat_i + sum_j D_ij x(j)   (Eq. 4, Sec. 2.2)
// Warps take the row's dense blocks round-robin and a quarter of U_i's columns
// each; partial rows meet in shared memory. RPL rows per lane cover leaf sizes <= 32 * RPL.
template <int RPL, int NVB>
__global__ void __launch_bounds__(kWarps * 32) k_dense_expand(const double* __restrict__ Dval, const int64_t* __restrict__ Doff,
                                                            const int32_t* __restrict__ Drow, const int32_t* __restrict__ Dcol,
                                                            const int64_t* __restrict__ leaf_off, const double* __restrict__ U,
                                                            int k, int64_t leaf0, const float2* __restrict__ x2, int64_t ld2,
                                                            const float2* __restrict__ yhat, int nv, double* __restrict__ y,
                                                            int64_t ldy) {
  __shared__ float2 red[kWarps][NVB][32 * RPL];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = blockIdx.x;
  const int64_t off = leaf_off[i];
  const int si = (int)(leaf_off[i + 1] - off);
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  const int32_t b0 = Drow[i], b1 = Drow[i + 1];
  for (int32_t b = b0 + warp; b < b1; b += kWarps) {
    const int32_t j = Dcol[b];
    const int64_t offj = leaf_off[j];
    const int sj = (int)(leaf_off[j + 1] - offj);
    warp_mv<RPL, NVB>(Dval + Doff[b], si, sj, 32, x2 + offj, ld2, nv, s, c, lane);
  }
  const int nu0 = (k * warp) / kWarps, nu1 = (k * (warp + 1)) / kWarps;
  if (nu1 > nu0)
    warp_mv<RPL, NVB>(U + off * k + (int64_t)si * nu0, si, nu1 - nu0, 32, yhat + (leaf0 + i) * nv * k + nu0, k, nv, s, c,
                      lane);
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) red[warp][v][lane + 32 * r] = make_float2(s[r][v], c[r][v]);
  __syncthreads();
  for (int t = threadIdx.x; t < si * nv; t += blockDim.x) {
    const int row = t % si, v = t / si;
    float ss = 0.f, cc = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; w++) df_add(ss, cc, red[w][v][row].x, red[w][v][row].y);
    y[v * ldy + off + row] = df_to_f64(ss, cc);
  }
}

}  // namespace h2
