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
                    // bit 2: the block holds zeros or magnitudes below 2^-103 after its offset (zero-safe split);
                    // FP64 form: bits 4-17 the block's exponent offset, bits 18-31 (last item) the row's
                    // output exponent (both signed 14-bit)
};

constexpr int kStageHeader = 128;
constexpr int kStageMat = 32768;
constexpr int kSmemLimit = 232448;  // opt-in shared memory per CTA on sm_103a
constexpr int kItemFlagLast = 1, kItemFlagSrc1 = 2, kItemFlagSafe = 4;
constexpr int kItemOffsetShift = 4, kItemRowExpShift = 18, kItemExpMax = 8191;  // 14-bit signed fields
__host__ __device__ constexpr int item_offset(int flags) { return (int)((unsigned)flags << 14) >> 18; }
__host__ __device__ constexpr int item_row_exp(int flags) { return flags >> kItemRowExpShift; }
__host__ __device__ constexpr int item_pack_exp(int offset, int row_exp) {
  return (int)(((unsigned)offset & 0x3FFFu) << kItemOffsetShift) | (int)((unsigned)row_exp << kItemRowExpShift);
}

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
  const int* vexp;       // per vector: the pass's x was scaled by 2^-vexp[v]
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
// Each block is split with its item's exponent offset; the row's sum is
// scaled by 2^(row exponent + vexp[v]) when it is written. A lane's
// accumulator sets are folded every FI items (chains of about 64 products)
// into its long-term pairs, which live in its own slots of the row-partial
// area (red) rather than in registers. A fold inside a row happens only once
// the previous row's partials have been consumed (tested without waiting, so
// warps keep a row of slack); the fold at the row's end waits for that.
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
  int* vexp_s = reinterpret_cast<int*>(const_cast<int*>(S.abort_flag)) + 1;  // [NVB], in the barrier area
  if (threadIdx.x < NVB) vexp_s[threadIdx.x] = threadIdx.x < nv ? P.vexp[threadIdx.x] : 0;
  asm volatile("bar.sync 1, %0;" ::"r"(CW * 32) : "memory");  // consumer warps only
  // lane owns rows 2 lane and 2 lane + 1 of every block; set u takes columns c0 + u, c0 + u + SETS, ...
  float s[SETS][2][NVB], c[SETS][2][NVB];
#pragma unroll
  for (int u = 0; u < SETS; u++)
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
      for (int v = 0; v < NVB; v++) s[u][r][v] = c[u][r][v] = 0.f;
  constexpr int FI = 8 * SETS;  // items per chain: (64 / CW) / SETS products per item
  const int r0 = 2 * lane;
  int rows_done = 0, chain = 0;
  bool red_mine = false;  // this warp's red slots hold the current row's long-term pairs
  // red slot of (v, rows r0 and r0 + 1): one float4 (s, c of row r0, then of row r0 + 1)
  // fold; inside a row (row_end false) only if the slots are free already: returns false when it did not fold
  auto fold = [&](bool row_end) -> bool {
    if (!red_mine && rows_done > 0) {
      if (!row_end) {
        if (!__all_sync(0xFFFFFFFFu, mbar_test_wait(S.rowfree, (rows_done - 1) & 1))) return false;
      } else if (!warp_wait(S.rowfree, (rows_done - 1) & 1, P, S.abort_flag)) {
        return false;
      }
    }
#pragma unroll
    for (int v = 0; v < NVB; v++) {
      float4* slot = reinterpret_cast<float4*>(S.red + (warp * NVB + v) * 64 + r0);
      float4 p = red_mine ? *slot : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < SETS; u++) {
        df_fold(p.x, p.y, s[u][0][v], c[u][0][v]);
        df_fold(p.z, p.w, s[u][1][v], c[u][1][v]);
      }
      *slot = p;
    }
    red_mine = true;
    return true;
  };
  for (int it = 0; it < ie - ib; it++) {
    const int st = it % NST, use = it / NST;
    if (!warp_wait(S.full + st, use & 1, P, S.abort_flag)) break;
    const unsigned char* stage = S.stage0 + st * SB;
    const int* h = reinterpret_cast<const int*>(stage);
    const int R = min(h[0], 64), C = min(h[1], 64), vs = min(h[2], 64), row = h[4], flags = h[5];
    const int o = item_offset(flags);
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
        split_f64_fast(a.x, o, h0, l0);
        split_f64_fast(a.y, o, h1, l1);
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
            split_f64(a0, o, h0, l0);
            split_f64(a1, o, h1, l1);
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
    if (++chain >= FI && !(flags & kItemFlagLast) && fold(false)) chain = 0;
    if (flags & kItemFlagLast) {
      // row end: the R = leaf-size rows of y at point offset `row`
      if (!fold(true)) break;
      chain = 0;
      __syncwarp();
      if (lane == 0) mbar_arrive(S.rowfull);
      if (!warp_wait(S.rowfull, rows_done & 1, P, S.abort_flag)) break;
      const int ey = item_row_exp(flags);
      for (int idx = threadIdx.x; idx < R * nv; idx += CW * 32) {
        const int r = idx % R, v = idx / R;
        float ss = 0.f, cc = 0.f;
#pragma unroll
        for (int w = 0; w < CW; w++) {
          const float2 p = S.red[(w * NVB + v) * 64 + r];
          df_add(ss, cc, p.x, p.y);
        }
        P.y[v * P.ldy + row + r] = scale2(df_to_f64(ss, cc), ey + vexp_s[v]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(S.rowfree);
      rows_done++;
      red_mine = false;
    }
  }
}

}  // namespace h2
