// FP64 plain-form kernels for the tree phases of the H^2 matrix-vector
// product (Sec. 4.2 and 4.4): leaf projection, upsweep and downsweep.
//
// Each phase is a sum of column-major block products "rows += A_block * x_cols":
//   leaf projection  xhat_j  = V_j^T x(j)            A = V_j^T (stored transposed)
//   upsweep          xhat_p  = sum_c F_c^T xhat_c    A = F_c^T (stored transposed)   Eq. 2
//   downsweep        yhat_c += E_c yhat_p            A = E_c                         Eq. 5
// One warp owns one output node: a lane owns output rows, consecutive lanes read
// consecutive rows of a column (coalesced), the column's input entry is a
// broadcast, and products accumulate in double-float. Loads of several columns
// are issued before any of them is used, so a warp keeps many in flight.
//
// Range: every block is split with its exponent offset o (a' = a * 2^-o, see
// df64.cuh) and x is scaled per vector by 2^-vexp[v], so that x, xhat and yhat
// hold values of magnitude at most about 1 (bounds computed by h2_create).
//
// Workspace layouts (float2 = double-float hi, lo; kp = k rounded up to even):
//   x2    leaf j's chunk at xp_off[j] * nv: [v][spad_j] (spad = leaf size rounded up to even)
//   xhat  [(node * nv + v) * kp + row]   vector trees of Sec. 4.2 - 4.4
//   yhat  same as xhat
#pragma once
#include "df64.cuh"

namespace h2 {

constexpr int kWarps = 4;  // warps per CTA for the per-node kernels

// Row mapping of a warp over an R-row block: lane = g * LR + rl owns rows
// rl + 32 r (r < RPL) and columns col = g, g + G, ... with G = 32 / LR groups.
// RPL = 2 requires LR = 32 (R <= 64); RPL = 1 allows LR = 1 .. 32 (R <= LR).
template <int RPL, int NVB, bool CG = false>
__device__ __forceinline__ void warp_mv_impl(const double* __restrict__ A, int o, int R, int C, int LR, const float2* xin,
                                             int64_t xstride, int nv, float (&s)[RPL][NVB], float (&c)[RPL][NVB], int lane) {
  constexpr int UB = (NVB <= 2) ? 8 : (NVB <= 4 ? 4 : 2);  // columns whose loads are issued together
  const int G = 32 / LR;
  const int g = lane / LR, rl = lane - g * LR;
  for (int col0 = g; col0 < C; col0 += UB * G) {
    double a[UB][RPL];
    float2 xv[UB][NVB];
#pragma unroll
    for (int u = 0; u < UB; u++) {
      const int col = col0 + u * G;
#pragma unroll
      for (int r = 0; r < RPL; r++) {
        const int row = rl + 32 * r;
        a[u][r] = (col < C && row < R) ? __ldg(A + row + (int64_t)R * col) : 0.0;
      }
#pragma unroll
      for (int v = 0; v < NVB; v++)
        xv[u][v] = (col < C && v < nv) ? (CG ? __ldcg(xin + v * xstride + col) : xin[v * xstride + col])
                                       : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < UB; u++) {
#pragma unroll
      for (int r = 0; r < RPL; r++) {
        float ah, al;
        split_f64(a[u][r], o, ah, al);
#pragma unroll
        for (int v = 0; v < NVB; v++) df_fma(s[r][v], c[r][v], ah, al, xv[u][v].x, xv[u][v].y);
      }
    }
  }
}

// xin is read with plain loads: it may have been written earlier in the same kernel by this CTA
template <int RPL, int NVB>
__device__ __forceinline__ void warp_mv(const double* __restrict__ A, int o, int R, int C, int LR, const float2* xin,
                                        int64_t xstride, int nv, float (&s)[RPL][NVB], float (&c)[RPL][NVB], int lane) {
  warp_mv_impl<RPL, NVB, false>(A, o, R, C, LR, xin, xstride, nv, s, c, lane);
}

// (S, C) += (s, c) elementwise, (s, c) = 0
template <int RPL, int NVB>
__device__ __forceinline__ void acc_fold(float (&S)[RPL][NVB], float (&C)[RPL][NVB], float (&s)[RPL][NVB],
                                         float (&c)[RPL][NVB]) {
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) df_fold(S[r][v], C[r][v], s[r][v], c[r][v]);
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

// write a node's k x nv vector (stride kp per vector) from lanes of group 0; optionally add the old value
template <int RPL, int NVB, bool ACCUM>
__device__ __forceinline__ void store_node(float2* __restrict__ dst, int k, int kp, int LR, int nv, float (&s)[RPL][NVB],
                                           float (&c)[RPL][NVB], int lane) {
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
        const float2 old = dst[v * kp + row];
        df_add(ss, cc, old.x, old.y);
      }
      dst[v * kp + row] = df_norm(ss, cc);
    }
  }
}

// ---------------------------------------------------------------- tree phases, one launch each
// CTA b owns the subtree rooted at node 2^L - 1 + b on level L (its T = q - L
// levels below hold leaves [b 2^T, (b + 1) 2^T)). One warp computes one node.
constexpr int kTreeWarps = 8;

struct TreeParams {
  const double* Vt;        // leaf j: k x size_j (V_j^T)
  const double* Ft;        // node h >= 1: F_h^T
  const double* E;         // node h >= 1: E_h
  const int64_t* leaf_off;
  const int64_t* xp_off;
  const double* x;         // pass input, ldx
  int64_t ldx;
  float2* x2;              // split x (padded leaf layout)
  float2* xhat;
  float2* yhat;
  int* ticket;             // one counter per node above level L, zero between products
  const int* oV;           // leaf j: exponent offset of V_j (projection)
  const int* oF;           // node h >= 1: exponent offset of F_h (upsweep into the parent)
  const int* oE;           // node h >= 1: exponent offset of E_h (downsweep from the parent)
  const int* vexp;         // per vector of the pass: x enters scaled by 2^-vexp[v]
  int k, kp, LR, q, L, nv;
};

// leaf projection of leaf j: x2(j) = split(x(j)); xhat_j = V_j^T x(j)   (Alg. 2, first step)
template <int RPL, int NVB>
__device__ __forceinline__ void project_leaf(const TreeParams& P, int64_t j, int lane) {
  const int64_t leaf0 = ((int64_t)1 << P.q) - 1;
  const int64_t off = P.leaf_off[j];
  const int sj = (int)(P.leaf_off[j + 1] - off);
  const int spad = sj + (sj & 1);
  float2* x2j = P.x2 + P.xp_off[j] * P.nv;
  for (int v = 0; v < P.nv; v++) {
    const int sv = P.vexp[v];
    for (int a = lane; a < sj; a += 32) x2j[v * spad + a] = f64_to_df(scale2(P.x[v * P.ldx + off + a], -sv));
  }
  __syncwarp();
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  warp_mv<RPL, NVB>(P.Vt + off * P.k, P.oV[j], P.k, sj, P.LR, x2j, spad, P.nv, s, c, lane);
  group_reduce(s, c, P.LR);
  store_node<RPL, NVB, false>(P.xhat + (leaf0 + j) * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, s, c, lane);
}

// Eq. 2 at parent p: xhat_p = F_c1^T xhat_c1 + F_c2^T xhat_c2 (CG: read the children through L2)
template <int RPL, int NVB, bool CG>
__device__ __forceinline__ void up_node(const TreeParams& P, int64_t p, int lane) {
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  for (int ci = 1; ci <= 2; ci++) {
    const int64_t ch = 2 * p + ci;
    warp_mv_impl<RPL, NVB, CG>(P.Ft + (ch - 1) * P.k * P.k, P.oF[ch], P.k, P.k, P.LR, P.xhat + ch * P.nv * P.kp, P.kp,
                               P.nv, s, c, lane);
  }
  group_reduce(s, c, P.LR);
  store_node<RPL, NVB, false>(P.xhat + p * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, s, c, lane);
}

// Leaf projection and the whole upsweep (Alg. 2, Eq. 2) in one launch. Inside
// a subtree the levels are separated by __syncthreads. Above level L, the
// second CTA of a sibling pair to finish (atomic ticket) computes the parent,
// so the climb needs no waiting: a CTA that arrives first simply stops.
template <int RPL, int NVB>
__global__ void __launch_bounds__(kTreeWarps * 32) k_upsweep_tree(TreeParams P) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = P.q - P.L;
  const int64_t sub = blockIdx.x;
  for (int64_t t = warp; t < ((int64_t)1 << T); t += kTreeWarps) project_leaf<RPL, NVB>(P, (sub << T) + t, lane);
  __syncthreads();
  for (int lvl = P.q - 1; lvl >= P.L; lvl--) {
    const int64_t node0 = ((int64_t)1 << lvl) - 1 + (sub << (lvl - P.L));
    for (int64_t t = warp; t < ((int64_t)1 << (lvl - P.L)); t += kTreeWarps) up_node<RPL, NVB, false>(P, node0 + t, lane);
    __syncthreads();
  }
  __threadfence();  // every writer orders its xhat stores before the ticket below
  __syncthreads();
  if (warp != 0) return;
  int64_t node = ((int64_t)1 << P.L) - 1 + sub;
  while (node > 0) {
    const int64_t par = (node - 1) / 2;
    int second = 0;
    if (lane == 0) {
      second = atomicAdd(P.ticket + par, 1) == 1;
      if (second) P.ticket[par] = 0;  // both arrivals are in: reset for the next product
    }
    second = __shfl_sync(0xFFFFFFFFu, second, 0);
    if (!second) break;
    __threadfence();  // order the sibling's xhat (published before its ticket) before our reads
    up_node<RPL, NVB, true>(P, par, lane);
    __threadfence();
    __syncwarp();
    node = par;
  }
}

// Eq. 5 at node c: yhat_c += E_c yhat_parent (parent given explicitly)
template <int RPL, int NVB>
__device__ __forceinline__ void down_node(const TreeParams& P, int64_t ch, const float2* ypar, int lane) {
  float s[RPL][NVB], c[RPL][NVB];
  acc_zero(s, c);
  warp_mv<RPL, NVB>(P.E + (ch - 1) * P.k * P.k, P.oE[ch], P.k, P.k, P.LR, ypar, P.kp, P.nv, s, c, lane);
  group_reduce(s, c, P.LR);
  store_node<RPL, NVB, true>(P.yhat + ch * P.nv * P.kp, P.k, P.kp, P.LR, P.nv, s, c, lane);
}

// The whole downsweep (Alg. 4, Eq. 5) in one launch. Warp 0 first carries the
// parents' sums from the root down the path to this CTA's subtree root (the
// path's nodes are shared with other CTAs, so their partial sums live only in
// this CTA's shared memory; only the subtree root is written back). Then the
// subtree is swept top-down, levels separated by __syncthreads.
template <int RPL, int NVB>
__global__ void __launch_bounds__(kTreeWarps * 32) k_downsweep_tree(TreeParams P) {
  __shared__ float2 path[2][NVB][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t sub = blockIdx.x;
  const int64_t root = ((int64_t)1 << P.L) - 1 + sub;
  if (warp == 0 && P.L > 0) {
    // path nodes a_0 = 0, ..., a_L = root: a_l = (root + 1) >> (L - l) minus 1
    int cur = 0;
    for (int v = 0; v < P.nv; v++)
      for (int r = lane; r < P.k; r += 32) path[cur][v][r] = P.yhat[(int64_t)v * P.kp + r];  // node 0
    __syncwarp();
    for (int l = 1; l <= P.L; l++) {
      const int64_t a = ((root + 1) >> (P.L - l)) - 1;
      float s[RPL][NVB], c[RPL][NVB];
      acc_zero(s, c);
      warp_mv<RPL, NVB>(P.E + (a - 1) * P.k * P.k, P.oE[a], P.k, P.k, P.LR, &path[cur][0][0], 64, P.nv, s, c, lane);
      group_reduce(s, c, P.LR);
      if (lane < P.LR) {
#pragma unroll
        for (int rr = 0; rr < RPL; rr++) {
          const int row = lane + 32 * rr;
          if (row >= P.k) continue;
#pragma unroll
          for (int v = 0; v < NVB; v++) {
            if (v >= P.nv) continue;
            float ss = s[rr][v], cc = c[rr][v];
            const float2 own = P.yhat[(a * P.nv + v) * P.kp + row];
            df_add(ss, cc, own.x, own.y);
            const float2 val = df_norm(ss, cc);
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
    for (int64_t t = warp; t < ((int64_t)1 << (lvl - P.L)); t += kTreeWarps) {
      const int64_t ch = node0 + t;
      down_node<RPL, NVB>(P, ch, P.yhat + ((ch - 1) / 2) * P.nv * P.kp, lane);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- coupling, all levels
// One warp per node row i: yhat_i = sum_{b in row i} S_b xhat_{col(b)}   (Eq. 3, Alg. 3)
// k = 2H with H a power of two: lane = g * H + h owns rows 2h, 2h + 1 of every block,
// read as one 16-byte load per column; column groups g = 0 .. G-1 (G = 32 / H)
// take columns g, g + G, ... The row's blocks are walked in batches of CB
// columns per lane, two batches in flight: the next batch's matrix and xhat
// loads are issued before the current batch is multiplied. Blocks are padded
// to kkp doubles; Sco[b] = (column node, exponent offset) of block b. Every node row
// is written (zero when it has no blocks). A lane's products form chains of
// at most 64 (kFoldProducts) that are folded into a long-term pair, so the
// FP32 sum of the small parts never runs over a whole row.
// SAFE: some coupling entry is zero or below 2^-103 after its offset (zero-safe split).
constexpr int kFoldProducts = 64;
template <int NVB, int CB, bool SAFE>
__global__ void __launch_bounds__(kWarps * 32) k_coupling(const double* __restrict__ S, int kkp,
                                                        const int32_t* __restrict__ Srow, const int2* __restrict__ Sco,
                                                        int k, int kp, int64_t n_nodes, int nv,
                                                        const float2* __restrict__ xhat, float2* __restrict__ yhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  if (i >= n_nodes) return;
  const int H = k >> 1, G = 32 / H;
  const int g = lane / H, h = lane - g * H;
  const bool active = g < G;            // lanes beyond G * H idle
  const int cpl = (k + G - 1) / G;      // columns per lane per block
  const int ncb = (cpl + CB - 1) / CB;  // batches per block
  const int32_t b0 = Srow[i];
  const int nbatch = (Srow[i + 1] - b0) * ncb;
  constexpr int FB = kFoldProducts / CB;  // batches per chain
  float s[2][NVB], c[2][NVB], S2[2][NVB], C2[2][NVB];
  acc_zero(s, c);
  acc_zero(S2, C2);

  double2 a0[CB], a1[CB];
  float2 x0[CB][NVB], x1[CB][NVB];
  int o0 = 0, o1 = 0;
  auto load = [&](int bt, double2(&a)[CB], float2(&xv)[CB][NVB], int& o) {
    const int b = bt / ncb, cb = bt - b * ncb;
    const double* A = S + (int64_t)(b0 + b) * kkp;
    const int2 co = __ldg(Sco + b0 + b);
    const float2* X = xhat + (int64_t)co.x * nv * kp;
    o = co.y;
#pragma unroll
    for (int u = 0; u < CB; u++) {
      const int col = g + G * (cb * CB + u);
      const bool ok = active && col < k;
      a[u] = ok ? __ldg(reinterpret_cast<const double2*>(A + 2 * h + k * col)) : make_double2(0.0, 0.0);
#pragma unroll
      for (int v = 0; v < NVB; v++) xv[u][v] = (ok && v < nv) ? __ldg(X + v * kp + col) : make_float2(0.f, 0.f);
    }
  };
  auto compute = [&](const double2(&a)[CB], const float2(&xv)[CB][NVB], int o) {
#pragma unroll
    for (int u = 0; u < CB; u++) {
      float h0, l0, h1, l1;
      if (SAFE) {
        split_f64(a[u].x, o, h0, l0);
        split_f64(a[u].y, o, h1, l1);
      } else {
        split_f64_fast(a[u].x, o, h0, l0);
        split_f64_fast(a[u].y, o, h1, l1);
      }
#pragma unroll
      for (int v = 0; v < NVB; v++) {
        df_fma(s[0][v], c[0][v], h0, l0, xv[u][v].x, xv[u][v].y);
        df_fma(s[1][v], c[1][v], h1, l1, xv[u][v].x, xv[u][v].y);
      }
    }
  };
  if (nbatch > 0) load(0, a0, x0, o0);
  for (int bt = 0; bt < nbatch; bt += 2) {
    if (bt + 1 < nbatch) load(bt + 1, a1, x1, o1);
    compute(a0, x0, o0);
    if (bt + 2 < nbatch) load(bt + 2, a0, x0, o0);
    if (bt + 1 < nbatch) compute(a1, x1, o1);
    if ((bt + 2) % FB == 0) acc_fold(S2, C2, s, c);
  }
  acc_fold(S2, C2, s, c);
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) {
      s[r][v] = S2[r][v];
      c[r][v] = C2[r][v];
    }
  // sum the column groups (lanes h, h + H, ...)
  for (int off = H; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
      for (int v = 0; v < NVB; v++) {
        const float s2 = __shfl_xor_sync(0xFFFFFFFFu, s[r][v], off);
        const float c2 = __shfl_xor_sync(0xFFFFFFFFu, c[r][v], off);
        df_add(s[r][v], c[r][v], s2, c2);
      }
  }
  if (g == 0) {
    float2* dst = yhat + i * nv * kp;
#pragma unroll
    for (int v = 0; v < NVB; v++)
      if (v < nv) {
        if (2 * h < k) dst[v * kp + 2 * h] = df_norm(s[0][v], c[0][v]);
        if (2 * h + 1 < k) dst[v * kp + 2 * h + 1] = df_norm(s[1][v], c[1][v]);
      }
  }
}

// Any other k: the generic row mapping of warp_mv, one block at a time (each
// block's chain folded into the row's long-term pair).
template <int RPL, int NVB>
__global__ void __launch_bounds__(kWarps * 32) k_coupling_generic(const double* __restrict__ S, int kkp,
                                                            const int32_t* __restrict__ Srow,
                                                            const int2* __restrict__ Sco, int k, int kp, int LR,
                                                            int64_t n_nodes, int nv, const float2* __restrict__ xhat,
                                                            float2* __restrict__ yhat) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  if (i >= n_nodes) return;
  float s[RPL][NVB], c[RPL][NVB], S2[RPL][NVB], C2[RPL][NVB];
  acc_zero(s, c);
  acc_zero(S2, C2);
  for (int32_t b = Srow[i]; b < Srow[i + 1]; b++) {
    const int2 co = Sco[b];
    warp_mv<RPL, NVB>(S + (int64_t)b * kkp, co.y, k, k, LR, xhat + (int64_t)co.x * nv * kp, kp, nv, s, c, lane);
    acc_fold(S2, C2, s, c);
  }
  group_reduce(S2, C2, LR);
#pragma unroll
  for (int r = 0; r < RPL; r++)
#pragma unroll
    for (int v = 0; v < NVB; v++) {
      s[r][v] = S2[r][v];
      c[r][v] = C2[r][v];
    }
  store_node<RPL, NVB, false>(yhat + i * nv * kp, k, kp, LR, nv, s, c, lane);
}

// ---------------------------------------------------------------- per-vector scale
// vexp[v] = s with max_i |x[i, v]| * 2^-s < 1 (frexp exponent; 0 for a zero or
// non-finite maximum), so that the pass works on x * 2^-s. Each block writes
// its maxima to partial[block][v]; the last block to finish (atomic ticket)
// reduces them and resets the ticket for the next launch. A thread keeps
// eight loads in flight; one round covers n = 2^20 on 152 blocks.
constexpr int kScaleBlocks = 152, kScaleThreads = 1024, kScaleUnroll = 8;
__device__ __forceinline__ unsigned long long abs_bits(double a) { return (unsigned long long)__double_as_longlong(fabs(a)); }
__global__ void __launch_bounds__(kScaleThreads) k_vec_scale(const double* __restrict__ x, int64_t ldx, int64_t n, int nv,
                                                            unsigned long long* partial, unsigned* ticket, int* vexp) {
  __shared__ unsigned long long wmax[kScaleThreads / 32][16];
  __shared__ int last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * kScaleThreads;
  for (int v = 0; v < nv; v++) {
    const double* xv = x + v * ldx;
    unsigned long long m = 0;
    int64_t i = (int64_t)blockIdx.x * kScaleThreads + threadIdx.x;
    for (; i + (kScaleUnroll - 1) * stride < n; i += kScaleUnroll * stride) {
      double a[kScaleUnroll];
#pragma unroll
      for (int u = 0; u < kScaleUnroll; u++) a[u] = __ldcs(xv + i + u * stride);
#pragma unroll
      for (int u = 0; u < kScaleUnroll; u++) m = max(m, abs_bits(a[u]));
    }
    for (; i < n; i += stride) m = max(m, abs_bits(__ldcs(xv + i)));
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    if (lane == 0) wmax[warp][v] = m;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    unsigned long long m = 0;
    for (int w = 0; w < kScaleThreads / 32; w++) m = max(m, wmax[w][threadIdx.x]);
    partial[blockIdx.x * 16 + threadIdx.x] = m;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int v = warp; v < nv; v += kScaleThreads / 32) {
    unsigned long long m = 0;
#pragma unroll 4
    for (int b = lane; b < (int)gridDim.x; b += 32) m = max(m, __ldcg(partial + b * 16 + v));
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    if (lane == 0) vexp[v] = vec_exponent(m);
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace h2
