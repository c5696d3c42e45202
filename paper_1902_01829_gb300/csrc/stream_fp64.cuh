// Persistent TMA-streaming kernel for the byte-heavy phase of the FP64 plain
// form: the dense near-field blocks fused with the leaf expansion,
//   y(i) = sum_j D_ij x(j) + U_i yhat_i        (Sec. 2.2, Eq. 4, Sec. 4.1)
//
// One CTA per SM owns a contiguous range of leaf rows, and hence one
// contiguous byte range of the repacked dense blocks. Its producer warp walks
// a host-built list of "items" (one column-major block of the row plus the
// vector chunk it multiplies: D_ij with the split x(j), or U_i with yhat_i as
// the row's last item) and copies each into a ring of shared-memory stages
// with cp.async.bulk. CW consumer warps split each stage's columns, multiply
// in double-float with several independent accumulator sets per lane, and
// hand the stage back. A row's partial sums meet in shared memory at the
// row's last item.
//
// Synchronisation uses mbarriers only (stage full/empty, row partials
// ready/consumed) and every wait is bounded (see tma.cuh): a fault in the
// item stream ends the kernel with the device error word set.
#pragma once
#include "df64.cuh"
#include "tma.cuh"

namespace h2 {

// Host-built work item, 32 bytes.
struct __align__(16) StreamItem {
  long long m_off;  // byte offset of the matrix block in the matrix buffer
  int m_bytes;      // bytes of the matrix block (multiple of 16)
  unsigned shape;   // R | C << 8 | vstride << 16 | nb << 24   (nb = 1)
  long long v_off;  // vector chunk offset, in float2 per vector slot
  int row;          // first point of the row leaf (y offset)
  int flags;        // bit 0: last item of its row; bit 1: vector chunk from the second source (yhat);
                    // bit 2: the block holds zeros or magnitudes below 2^-103 (zero-safe split needed)
};

constexpr int kStageHeader = 128;
constexpr int kStageMat = 32768;
constexpr int kSmemLimit = 232448;  // opt-in shared memory per CTA on sm_103a
constexpr int kItemFlagLast = 1, kItemFlagSrc1 = 2, kItemFlagSafe = 4;

// a stage holds one item: header, matrix block (<= 64 x 64 doubles), vector chunk (<= 64 x NVB float2)
__host__ __device__ constexpr int stage_vec_bytes(int nvb) { return 512 * nvb; }
__host__ __device__ constexpr int stage_bytes(int nvb) { return kStageHeader + kStageMat + stage_vec_bytes(nvb); }
__host__ __device__ constexpr int red_bytes(int nvb, int cw) { return cw * nvb * 64 * 8; }
__host__ __device__ constexpr int stream_stages(int nvb, int cw) {
  return (kSmemLimit - 256 - red_bytes(nvb, cw)) / stage_bytes(nvb) < 6
             ? (kSmemLimit - 256 - red_bytes(nvb, cw)) / stage_bytes(nvb)
             : 6;
}
__host__ __device__ constexpr int stream_smem_bytes(int nvb, int cw) {
  return stream_stages(nvb, cw) * stage_bytes(nvb) + 256 + red_bytes(nvb, cw);
}
// consumer warps per CTA for a vector-slot count (more warps hide more latency;
// wide vector slots need the registers of fewer warps)
__host__ __device__ constexpr int dense_consumer_warps(int nvb) { return 8; }

struct StreamParams {
  const StreamItem* items;
  const int* cta_begin;  // [grid + 1] item ranges
  const char* mat;       // matrix buffer
  const float2* vsrc0;   // split x, padded leaf layout
  const float2* vsrc1;   // yhat (expansion items)
  int nv;                // vectors of this pass (<= NVB)
  double* y;             // output
  long long ldy;
  int* err;              // device error word
  long long budget;      // clock64 cycles a single wait may take
  int inject;            // >= 0: CTA 0 withholds the copy of this local item (bounded-wait test)
};

// every lane polls (so every lane acquires the barrier's phase); the warp
// proceeds only if all lanes saw it complete
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, const StreamParams& P, volatile int* abort_flag) {
  const bool ok = mbar_wait(bar, parity, abort_flag, P.err, P.budget);
  return __all_sync(0xFFFFFFFFu, ok) != 0;
}

struct StreamShared {
  unsigned char* stage0;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* rowfull;
  uint64_t* rowfree;
  volatile int* abort_flag;
  float2* red;
};

template <int NST, int SB>
__device__ __forceinline__ StreamShared stream_shared(unsigned char* smem) {
  StreamShared S;
  S.stage0 = smem;
  S.full = reinterpret_cast<uint64_t*>(smem + NST * SB);
  S.empty = S.full + NST;
  S.rowfull = S.empty + NST;
  S.rowfree = S.rowfull + 1;
  S.abort_flag = reinterpret_cast<volatile int*>(S.rowfree + 1);
  S.red = reinterpret_cast<float2*>(smem + NST * SB + 256);
  return S;
}

template <int NST, int CW>
__device__ __forceinline__ void stream_init(const StreamShared& S) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; s++) {
      mbar_init(S.full + s, 1);
      mbar_init(S.empty + s, CW);
    }
    mbar_init(S.rowfull, CW);
    mbar_init(S.rowfree, CW);
    *S.abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Producer warp: copy items [ib, ie) into the stage ring. Stage header words:
// R, C, vstride, nb, row, flags.
template <int NST, int SB>
__device__ __forceinline__ void stream_produce(const StreamParams& P, const StreamShared& S, int ib, int ie) {
  const int lane = threadIdx.x & 31;
  const uint64_t pol = policy_evict_first();
  int issued = 0;
  bool ok = true;
  for (int base = ib; base < ie && ok; base += 32) {
    int4 d0 = make_int4(0, 0, 0, 0), d1 = make_int4(0, 0, 0, 0);
    if (base + lane < ie) {
      const int4* src = reinterpret_cast<const int4*>(P.items + base + lane);
      d0 = __ldg(src);
      d1 = __ldg(src + 1);
    }
    const int cnt = min(32, ie - base);
    for (int t = 0; t < cnt; t++) {
      const int it = base + t - ib;
      const int s = it % NST, use = it / NST;
      if (use > 0 && !warp_wait(S.empty + s, (use - 1) & 1, P, S.abort_flag)) {
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
      const unsigned v_lo = (unsigned)__shfl_sync(0xFFFFFFFFu, d1.x, t);
      const unsigned v_hi = (unsigned)__shfl_sync(0xFFFFFFFFu, d1.y, t);
      const int row = __shfl_sync(0xFFFFFFFFu, d1.z, t);
      const int flags = __shfl_sync(0xFFFFFFFFu, d1.w, t);
      if (lane == 0) {
        const long long m_off = (long long)(((unsigned long long)m_hi << 32) | m_lo);
        const long long v_off = (long long)(((unsigned long long)v_hi << 32) | v_lo);
        const int vs = (shape >> 16) & 0xFF;
        const unsigned vbytes = (unsigned)(P.nv * vs * 8);
        unsigned char* stage = S.stage0 + s * SB;
        int* h = reinterpret_cast<int*>(stage);
        h[0] = (int)(shape & 0xFF);
        h[1] = (int)((shape >> 8) & 0xFF);
        h[2] = vs;
        h[3] = 1;
        h[4] = row;
        h[5] = flags;
        if (!((P.inject == it) && (blockIdx.x == 0))) {
          mbar_arrive_expect_tx(S.full + s, (unsigned)m_bytes + vbytes);
          bulk_g2s_stream(stage + kStageHeader, P.mat + m_off, (unsigned)m_bytes, S.full + s, pol);
          const float2* src = (flags & kItemFlagSrc1) ? P.vsrc1 : P.vsrc0;
          bulk_g2s(stage + kStageHeader + kStageMat, src + v_off * P.nv, vbytes, S.full + s);
        }
      }
      __syncwarp();
      issued = it + 1;
    }
  }
  // no copy may still be in flight when the warp exits
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

// ---------------------------------------------------------------- dense near field + expansion
template <int NVB, int CW>
__global__ void __launch_bounds__((CW + 1) * 32, 1) k_dense_stream(StreamParams P) {
  constexpr int NST = stream_stages(NVB, CW);
  constexpr int SB = stage_bytes(NVB);
  constexpr int SETS = NVB == 1 ? 4 : (NVB == 2 ? 2 : 1);  // independent accumulator sets per lane
  static_assert(NST >= 2, "at least two stages");
  extern __shared__ __align__(1024) unsigned char smem[];
  const StreamShared S = stream_shared<NST, SB>(smem);
  stream_init<NST, CW>(S);
  const int ib = P.cta_begin[blockIdx.x], ie = P.cta_begin[blockIdx.x + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == CW) {
    stream_produce<NST, SB>(P, S, ib, ie);
    return;
  }
  const int nv = P.nv;
  // lane owns rows 2 lane and 2 lane + 1 of every block; set u takes columns c0 + u, c0 + u + SETS, ...
  float s[SETS][2][NVB], c[SETS][2][NVB];
#pragma unroll
  for (int u = 0; u < SETS; u++)
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
      for (int v = 0; v < NVB; v++) s[u][r][v] = c[u][r][v] = 0.f;
  const int r0 = 2 * lane;
  int rows_done = 0;
  for (int it = 0; it < ie - ib; it++) {
    const int st = it % NST, use = it / NST;
    if (!warp_wait(S.full + st, use & 1, P, S.abort_flag)) break;
    const unsigned char* stage = S.stage0 + st * SB;
    const int* h = reinterpret_cast<const int*>(stage);
    const int R = min(h[0], 64), C = min(h[1], 64), vs = min(h[2], 64), row = h[4], flags = h[5];
    const double* A = reinterpret_cast<const double*>(stage + kStageHeader);
    const float2* X = reinterpret_cast<const float2*>(stage + kStageHeader + kStageMat);
    const int c0 = (C * warp) / CW, c1 = (C * (warp + 1)) / CW;
    if (R == 64 && C == 64 && !(flags & kItemFlagSafe)) {
      // full block without tiny entries: fixed strides, fast split
      constexpr int CPW = 64 / CW;
      constexpr int UNR = NVB >= 4 ? 2 : CPW;  // wide vector slots: keep the loop body small
      const double* Ab = A + r0 + 64 * c0;
      const float2* Xb = X + c0;
#pragma unroll UNR
      for (int u = 0; u < CPW; u++) {
        const double2 a = *reinterpret_cast<const double2*>(Ab + 64 * u);
        float h0, l0, h1, l1;
        split_f64_fast(a.x, h0, l0);
        split_f64_fast(a.y, h1, l1);
#pragma unroll
        for (int v = 0; v < NVB; v++) {
          const float2 xv = (v < nv) ? Xb[v * 64 + u] : make_float2(0.f, 0.f);
          df_fma(s[u % SETS][0][v], c[u % SETS][0][v], h0, l0, xv.x, xv.y);
          df_fma(s[u % SETS][1][v], c[u % SETS][1][v], h1, l1, xv.x, xv.y);
        }
      }
    } else if (r0 < R) {
      const bool even = (R & 1) == 0;
      for (int col0 = c0; col0 < c1; col0 += SETS) {
#pragma unroll
        for (int u = 0; u < SETS; u++) {
          const int col = col0 + u;
          if (col < c1) {
            double a0, a1 = 0.0;
            if (even) {
              const double2 a = *reinterpret_cast<const double2*>(A + r0 + R * col);
              a0 = a.x;
              a1 = a.y;
            } else {
              a0 = A[r0 + R * col];
              if (r0 + 1 < R) a1 = A[r0 + 1 + R * col];
            }
            float h0, l0, h1, l1;
            split_f64(a0, h0, l0);
            split_f64(a1, h1, l1);
#pragma unroll
            for (int v = 0; v < NVB; v++) {
              const float2 xv = (v < nv) ? X[v * vs + col] : make_float2(0.f, 0.f);
              df_fma(s[u][0][v], c[u][0][v], h0, l0, xv.x, xv.y);
              df_fma(s[u][1][v], c[u][1][v], h1, l1, xv.x, xv.y);
            }
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(S.empty + st);
    if (flags & kItemFlagLast) {
      // row end: the R = leaf-size rows of y at point offset `row`
      if (rows_done > 0 && !warp_wait(S.rowfree, (rows_done - 1) & 1, P, S.abort_flag)) break;
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int v = 0; v < NVB; v++) {
#pragma unroll
          for (int u = 1; u < SETS; u++) df_add(s[0][r][v], c[0][r][v], s[u][r][v], c[u][r][v]);
          S.red[(warp * NVB + v) * 64 + r0 + r] = make_float2(s[0][r][v], c[0][r][v]);
#pragma unroll
          for (int u = 0; u < SETS; u++) s[u][r][v] = c[u][r][v] = 0.f;
        }
      __syncwarp();
      if (lane == 0) mbar_arrive(S.rowfull);
      if (!warp_wait(S.rowfull, rows_done & 1, P, S.abort_flag)) break;
      for (int idx = threadIdx.x; idx < R * nv; idx += CW * 32) {
        const int r = idx % R, v = idx / R;
        float ss = 0.f, cc = 0.f;
#pragma unroll
        for (int w = 0; w < CW; w++) {
          const float2 p = S.red[(w * NVB + v) * 64 + r];
          df_add(ss, cc, p.x, p.y);
        }
        P.y[v * P.ldy + row + r] = df_to_f64(ss, cc);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(S.rowfree);
      rows_done++;
    }
  }
}

}  // namespace h2
