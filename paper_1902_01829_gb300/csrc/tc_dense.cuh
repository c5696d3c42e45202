// Dense near field and leaf expansion of the precision form on the 5th-generation
// tensor cores (tcgen05.mma, FP32 accumulators in tensor memory) for a pass of up
// to 16 vectors:   y(i) = sum_j D_ij x(j) + U_i yhat_i   (Sec. 2.2 dense blocks,
// Eq. 4 leaf expansion), with every block stored as 16-bit codes q and one FP32
// scale sigma (a = sigma q).
//
// One tcgen05.mma costs about the same time for every shape up to M = 128, N = 256
// (K = 16), so the kernel issues as few as it can: two consecutive blocks of a row
// with the same width form one M = 128 operand (the second block's panels follow the
// first's at the same stride), and their B tiles sit side by side in N:
//  A  the two blocks' fp16 / bf16 codes, copied by TMA as stored (the panel layout of
//     mixed.cuh is the MN-major canonical layout: 8 x 8 core matrices, K stride
//     128 bytes, M stride the panel stride);
//  B  built in shared memory per block by four builder warps from the FP32 copy
//     of the vectors (x(j), or yhat_i for U_i): z = sigma * s_v * x_v in FP32,
//     split z = hi + lo into two codes of the block type (rows 2v and 2v + 1 of
//     the K-major tile), so the products keep about FP32 accuracy and sigma enters
//     exactly; s_v is a power of two per vector keeping fp16 parts in range (1 for
//     bf16). The second block's rows are N rows 32 .. 63.
// The 128 x 64 product holds the first block's result in rows 0 .. 63, columns
// 0 .. 31 and the second's in rows 64 .. 127, columns 32 .. 63; the rest is unused.
// A block without a partner is issued the same way with zero B rows 32 .. 63, so
// whatever finite codes follow it in shared memory add exact zeros (the stages are
// zeroed at start). Each row accumulates into one 128 x 64 accumulator (two
// alternate between rows); four epilogue warps read them back (tcgen05.ld), add the
// two halves and the two parts of each vector, divide by s_v and write y in FP64.
//
// The coupling phase (Eq. 3) at k = 64 runs the same kernel: a work item is up to four
// coupling blocks S_ij of one row i (any level; their codes in the panel layout without
// the pad, P.ppad = 0), the builders read xhat_j ([node][v][kp]) through the second vector
// source, and the epilogue assigns the row's yhat_i at row i * P.rowmul (P.rowmul = nv kp,
// FP32); the leaf expansion has no part in it.
//
// Warp roles (320 threads, one CTA per SM, persistent over byte-balanced work items
// of their own, up to four 64 x 64 blocks and U): 0 producer (TMA of the codes and a
// header for the MMA thread), 1 MMA issuer (one thread), 2-5 B-tile builders (reading
// the items themselves, ahead of the stage ring), 6-9 epilogue (TMEM lane quadrants 2,
// 3, 0, 1). Every wait is bounded; on a timeout the kernel sets the error word, the other
// roles stop at their next wait, the MMA thread waits for its issued MMAs, and the
// tensor memory is freed before the kernel returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mixed.cuh"

namespace h2 {

constexpr int kTcVec = 16;                 // vectors per pass
constexpr int kTcN = 2 * kTcVec;           // B rows of one block (high and low part of each vector)
constexpr int kTcMaxBlocks = 5;            // blocks per work item (64 x 64 panels: at most 4 + U)
constexpr int kTcStageMat = 35840;         // codes of one item: four 64 x 64 panel blocks and a 64 x 16 one
constexpr int kTcStageB = 18432;           // B tiles of one item (tc_layout)
constexpr int kTcHeader = 256;
constexpr int kTcSlotA = kTcHeader + kTcStageMat;  // a codes slot: header for the MMA thread, then the codes
constexpr int kTcStages = 5;               // codes slots (copies in flight)
constexpr int kTcStagesB = 2;              // B-tile slots (built shortly before their MMAs)
constexpr int kTcRingB = kTcStages * kTcSlotA;     // offset of the B slots
constexpr int kTcBars = kTcRingB + kTcStagesB * kTcStageB;
constexpr int kTcXBuf = 2 * 64 * (kTcVec + 1) * 4;   // epilogue exchange of the second halves, two rows
constexpr int kTcSmem = kTcBars + 256 + kTcXBuf;
constexpr int kTcThreads = 320;
constexpr int kTcPairShift = 8;            // item flags: bit 8 + t marks a pair starting at block t
// builder record of an item (16 ints): [0] blocks | pair starts << 8; block t at 1 + 3 t:
// vector offset (floats per vector slot), K | (vector from yhat) << 16, scale bits
constexpr int kTcRecInts = 16;
static_assert(1 + 3 * kTcMaxBlocks <= kTcRecInts, "builder record");
constexpr int kTcCols = 2 * 2 * kTcN;      // tensor-memory columns: a 128 x 64 accumulator per row, two rows
static_assert(kTcSmem <= 232448, "tensor-core stages exceed the shared memory of a CTA");
static_assert(kTcStageMat % 16 == 0 && kTcStageB % 16 == 0 && kTcSlotA % 16 == 0, "slot alignment");

// B tiles of a stage. The item's blocks (padded widths kp[0 .. nb-1]) form MMA units:
// two consecutive blocks of equal width a pair, any other block a single. A unit's tile
// holds 2 kTcN K-major rows: the first block's kTcN rows, then the second block's (a
// pair) or zeros (a single); units follow each other. boff[t] is block t's first row;
// bit t of *pairs marks a pair starting at block t, bit t of *singles a single. Returns
// the stage's B bytes. The host stores the pair starts in the item's flags.
__host__ __device__ inline int tc_layout(int nb, const int* kp, int* boff, int* pairs, int* singles) {
  int cur = 0, pm = 0, sm = 0;
  for (int t = 0; t < nb;) {
    const int w = kTcN * kp[t] * 2;  // bytes of one block's rows
    boff[t] = cur;
    if (t + 1 < nb && kp[t + 1] == kp[t]) {
      boff[t + 1] = cur + w;
      pm |= 1 << t;
      t += 2;
    } else {
      sm |= 1 << t;
      t += 1;
    }
    cur += 2 * w;
  }
  *pairs = pm;
  *singles = sm;
  return cur;
}

struct TcParams {
  const StreamItem* items;
  const int* cta_begin;
  const MixedBlock* blk;
  const char* dmat;
  const float* x4;      // FP32 vectors, leaf j at xp4_off[j] * nv (64 entries per vector)
  const float* yhat;    // [node][v][kp]
  const float* vscale;  // [16] per-vector power-of-two scale s_v
  const int4* brec;     // builder records, kTcRecInts / 4 per item
  double* y;            // FP32 when y32
  long long ldy;
  long long rowmul;     // output row r of an item starts at row * rowmul (1: y; nv kp: the coupling's yhat)
  int nv, kp, y32;
  int ppad;             // bytes between a block's panels beyond 16 K (kPanelPad; 0 for coupling blocks)
  int* err;
  long long budget;
};

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);  // no swizzle
}

// kind::f16 instruction descriptor: FP32 accumulator, A and B of the code type,
// A MN-major, B K-major, N = 2 kTcN, M = 128
template <int F>
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | ((F == kFormBf16 ? 1u : 0u) << 7) | ((F == kFormBf16 ? 1u : 0u) << 10) | (1u << 15) |
         ((uint32_t)((2 * kTcN) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int F>
__device__ __forceinline__ uint32_t tc_pack(float a, float b) {  // two codes, a in the low half
  if (F == kFormBf16) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&t);
  }
  const __half2 t = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&t);
}
template <int F>
__device__ __forceinline__ float tc_round(float z) {  // z rounded to the code type
  if (F == kFormBf16) return __bfloat162float(__float2bfloat16_rn(z));
  return __half2float(__float2half_rn(z));
}

// bounded wait of one warp on an mbarrier phase (all lanes poll; false on timeout or abort)
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                        long long budget) {
  const bool ok = mbar_wait(bar, parity, abort_flag, err, budget);
  return __all_sync(0xFFFFFFFFu, ok) != 0;
}

// slot header (ints, for the MMA thread): [0] blocks, [1] item flags; block t at 4 + 3 t:
// A offset (bytes), K, panel stride (bytes)
template <int F>
__global__ void __launch_bounds__(kTcThreads, 1) k_dense_tc(TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* slot0 = smem;               // codes slots
  unsigned char* bslot0 = smem + kTcRingB;    // B-tile slots
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kTcBars);  // codes slot landed
  uint64_t* empty = full + kTcStages;         // codes slot read by its MMAs
  uint64_t* bready = empty + kTcStages;       // B slot written
  uint64_t* bempty = bready + kTcStagesB;     // B slot read by its MMAs
  uint64_t* accfull = bempty + kTcStagesB;
  uint64_t* accempty = accfull + 2;
  uint64_t* xfull = accempty + 2;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(xfull + 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(xfull + 2) + 1;
  float* xbuf = reinterpret_cast<float*>(smem + kTcBars + 256);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ib = P.cta_begin[blockIdx.x], ie = P.cta_begin[blockIdx.x + 1];
  const int n_items = ie - ib;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; s++) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int s = 0; s < kTcStagesB; s++) {
      mbar_init(bready + s, 4);
      mbar_init(bempty + s, 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(accfull + b, 1);
      mbar_init(accempty + b, 4);
      mbar_init(xfull + b, 2);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // zeroed slots: the operand rows a single block leaves unused read finite codes
  for (int i = threadIdx.x; i < kTcBars / 16; i += kTcThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // 32 items at a time: lane l loads item base + l; per item, lanes 0 .. 15 load its builder
    // record (the blocks' widths give their offsets); lane 0 writes the header and issues the copy
    const uint64_t pol = policy_evict_first();
    int issued = 0;
    bool ok = true;
    for (int base = 0; base < n_items && ok; base += 32) {
      const int cnt = min(32, n_items - base);
      StreamItem mine{};
      if (lane < cnt) mine = P.items[ib + base + lane];
      for (int t = 0; t < cnt; t++) {
        const int it = base + t;
        const int s = it % kTcStages, use = it / kTcStages;
        const int* rec = reinterpret_cast<const int*>(P.brec + (long long)(ib + it) * (kTcRecInts / 4));
        const int rv = lane < kTcRecInts ? __ldg(rec + lane) : 0;
        if (use > 0 && !tc_wait(empty + s, (use - 1) & 1, abort_flag, P.err, P.budget)) {
          ok = false;
          break;
        }
        const long long m_off = __shfl_sync(0xFFFFFFFFu, mine.m_off, t);
        const int m_bytes = __shfl_sync(0xFFFFFFFFu, mine.m_bytes, t);
        const int flags = __shfl_sync(0xFFFFFFFFu, mine.flags, t);
        const int nb = min(__shfl_sync(0xFFFFFFFFu, rv, 0) & 0xFF, kTcMaxBlocks);
        int kp[kTcMaxBlocks];
#pragma unroll
        for (int b = 0; b < kTcMaxBlocks; b++) kp[b] = min(__shfl_sync(0xFFFFFFFFu, rv, 2 + 3 * b) & 0xFFFF, 64);
        int* hd = reinterpret_cast<int*>(slot0 + s * kTcSlotA);
        if (lane == 0) {
          int aoff = 0;
#pragma unroll
          for (int b = 0; b < kTcMaxBlocks; b++) {
            if (b < nb) {
              hd[4 + 3 * b] = aoff;
              hd[5 + 3 * b] = kp[b];
              hd[6 + 3 * b] = 16 * kp[b] + P.ppad;  // panel stride
              aoff += 8 * (16 * kp[b] + P.ppad);
            }
          }
          hd[0] = nb;
          hd[1] = flags;
          // the copy's completion also publishes the header (written before it)
          const unsigned bytes = (unsigned)min(m_bytes, kTcStageMat);
          mbar_arrive_expect_tx(full + s, bytes);
          bulk_g2s_stream(slot0 + s * kTcSlotA + kTcHeader, P.dmat + m_off, bytes, full + s, pol);
        }
        __syncwarp();
        issued = it + 1;
      }
    }
    if (lane == 0)
      for (int it = max(0, issued - kTcStages); it < issued; it++) {  // copies in flight land before exit
        const int s = it % kTcStages, use = it / kTcStages;
        const long long t0 = clock64();
        while (!mbar_try_wait(full + s, use & 1) && clock64() - t0 < P.budget) {
        }
      }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc<F>();
      int rows = 0, issued_it = -1;
      bool row_open = false, first = false, ok = true;
      uint32_t acc_col = 0;
      for (int it = 0; it < n_items && ok; it++) {
        const int s = it % kTcStages, use = it / kTcStages;
        const int sb = it % kTcStagesB, useb = it / kTcStagesB;
        if (!mbar_wait(full + s, use & 1, abort_flag, P.err, P.budget) ||
            !mbar_wait(bready + sb, useb & 1, abort_flag, P.err, P.budget)) {
          ok = false;
          break;
        }
        const unsigned char* st = slot0 + s * kTcSlotA;
        const int* hd = reinterpret_cast<const int*>(st);
        const int nb = min(hd[0], kTcMaxBlocks), flags = hd[1], pm = flags >> kTcPairShift;
        if (!row_open) {  // a new row: its accumulator must have been read out
          const int b = rows & 1;
          if (rows >= 2 && !mbar_wait(accempty + b, ((rows >> 1) - 1) & 1, abort_flag, P.err, P.budget)) {
            ok = false;
            break;
          }
          acc_col = (uint32_t)(b * 2 * kTcN);
          row_open = true;
          first = true;
        }
        tc_fence_after();
        const uint32_t a0 = smem_addr(st + kTcHeader), b0 = smem_addr(bslot0 + sb * kTcStageB);
        int bcur = 0;               // B tiles: units follow each other (tc_layout)
        for (int t = 0; t < nb;) {  // one MMA unit (a pair, or a single) per pass
          const int K = max(min(hd[5 + 3 * t], 64), 16), ps = min(hd[6 + 3 * t], panel_stride(64));
          const bool pair = (pm >> t) & 1;
          // a single after the item's first block takes the upper half of the operand (its partner
          // rows are the codes before it); the 16 panels read stay inside the slot's codes
          int aoff = hd[4 + 3 * t] - (!pair && t > 0 ? 8 * ps : 0);
          aoff = max(min(aoff, kTcStageMat - 16 * ps), 0);
          const int boff = max(min(bcur, kTcStageB - 4 * kTcN * K), 0);
          bcur += 4 * kTcN * K;
          // a K-step advances both start addresses by 256 bytes: 16 in the descriptors' address field
          // (the addresses stay below 256 KB, so the field does not carry)
          uint64_t da = tc_desc(a0 + aoff, 128, ps), db = tc_desc(b0 + boff, 128, K * 16);
          for (int ks = 0; ks < K / 16; ks++, da += 16, db += 16) {
            tc_mma(tmem + acc_col, da, db, idesc, first ? 0u : 1u);  // a row's first MMA starts its sum
            first = false;
          }
          t += pair ? 2 : 1;
        }
        tc_commit(empty + s);  // the slots are free once these MMAs complete
        tc_commit(bempty + sb);
        issued_it = it;
        if (flags & kItemFlagLast) {
          tc_commit(accfull + (rows & 1));
          rows++;
          row_open = false;
        }
      }
      if (issued_it >= 0) {  // issued MMAs complete before the tensor memory is freed
        const int s = issued_it % kTcStages, use = issued_it / kTcStages;
        const long long t0 = clock64();
        while (!mbar_try_wait(empty + s, use & 1) && clock64() - t0 < P.budget) {
        }
      }
    }
  } else if (warp < 6) {
    // ---------------------------------------------------------------- B-tile builders
    // thread: vector v (0 .. 15) and K group g (8 entries); it writes the 16-byte high and
    // low rows of its vector for that K group. Lane l of builder warp w takes v = 4 w + (l & 3),
    // g = l >> 2, and threads with odd g store the low row first: each quarter-warp's two
    // stores then cover all eight 16-byte bank groups (rows 0 .. 7 of a core matrix), free of
    // bank conflicts. The builders read their own records of the items (brec) and load the
    // vector entries an item ahead; only the conversion and the stores of item it wait for
    // its B slot to be free.
    const int tid = threadIdx.x - 64, v = 4 * (tid >> 5) + (tid & 3), g = (tid >> 2) & 7;
    const float sv = P.vscale[v];
    const bool vok = v < P.nv;
    struct Rec {
      int4 q[kTcRecInts / 4];
    };
    auto rf = [](const Rec& R, int i) -> int {  // field i (a constant once the loops are unrolled)
      const int4& u = R.q[i >> 2];
      return (i & 3) == 0 ? u.x : (i & 3) == 1 ? u.y : (i & 3) == 2 ? u.z : u.w;
    };
    auto load_rec = [&](int it, Rec& R) {
#pragma unroll
      for (int u = 0; u < kTcRecInts / 4; u++)
        R.q[u] = it < n_items ? __ldg(P.brec + (long long)(ib + it) * (kTcRecInts / 4) + u) : make_int4(0, 0, 0, 0);
    };
    auto load_x = [&](const Rec& R, float4(&ra)[kTcMaxBlocks], float4(&rb)[kTcMaxBlocks]) {
      const int nb = min(rf(R, 0) & 0xFF, kTcMaxBlocks);
#pragma unroll
      for (int t = 0; t < kTcMaxBlocks; t++) {
        ra[t] = rb[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int kw = rf(R, 2 + 3 * t);
        if (t < nb && vok && 8 * g < min(kw & 0xFFFF, 64)) {
          const long long voff = rf(R, 1 + 3 * t);
          const float* src = ((kw >> 16) & 1) ? P.yhat + voff * P.nv + (long long)v * P.kp + 8 * g
                                              : P.x4 + voff * P.nv + (long long)v * 64 + 8 * g;
          ra[t] = __ldg(reinterpret_cast<const float4*>(src));
          rb[t] = __ldg(reinterpret_cast<const float4*>(src + 4));
        }
      }
    };
    // item it's B tiles from its records and entries (tc_layout's units, from the pair starts;
    // a single after the first block has its rows in the upper half of its unit, as its codes)
    auto convert_store = [&](int it, const Rec& R, const float4(&ra)[kTcMaxBlocks], const float4(&rb)[kTcMaxBlocks]) {
      unsigned char* bt = bslot0 + (it % kTcStagesB) * kTcStageB;
      const int nb = min(rf(R, 0) & 0xFF, kTcMaxBlocks), pm = rf(R, 0) >> 8;
      int cur = 0, prev = 0;
      bool second = false;
#pragma unroll
      for (int t = 0; t < kTcMaxBlocks; t++) {
        if (t < nb) {
          const int K = min(rf(R, 2 + 3 * t) & 0xFFFF, 64), w = 2 * kTcN * K;  // one block's rows
          int boff, zoff = -1;  // this block's rows, and the zero partner rows of a single
          if (second) {
            boff = prev + w;
            second = false;
          } else {
            prev = cur;
            cur += 2 * w;
            second = (pm >> t) & 1;
            boff = (second || t == 0) ? prev : prev + w;
            if (!second) zoff = t == 0 ? prev + w : prev;
          }
          boff = max(min(boff, kTcStageB - w), 0);
          zoff = zoff < 0 ? -1 : max(min(zoff, kTcStageB - w), 0);
          if (8 * g < K) {
            const float sc = __int_as_float(rf(R, 3 + 3 * t)) * sv;
            const float z[8] = {ra[t].x * sc, ra[t].y * sc, ra[t].z * sc, ra[t].w * sc,
                                rb[t].x * sc, rb[t].y * sc, rb[t].z * sc, rb[t].w * sc};
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const float h0 = tc_round<F>(z[2 * e]), h1 = tc_round<F>(z[2 * e + 1]);
              hi[e] = tc_pack<F>(h0, h1);
              lo[e] = tc_pack<F>(z[2 * e] - h0, z[2 * e + 1] - h1);
            }
            // K-major tile: row n = 2v (+1), core (n / 8, g) at (n / 8) * K * 16 + g * 128, row n % 8 at 16 bytes
            const int inner = ((2 * v) >> 3) * K * 16 + g * 128 + ((2 * v) & 7) * 16;
            unsigned char* dst = bt + boff + inner;
            const uint4 wh = make_uint4(hi[0], hi[1], hi[2], hi[3]), wl = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            const bool low_first = g & 1;
            *reinterpret_cast<uint4*>(dst + (low_first ? 16 : 0)) = low_first ? wl : wh;
            *reinterpret_cast<uint4*>(dst + (low_first ? 0 : 16)) = low_first ? wh : wl;
            if (zoff >= 0) {  // the partner rows of a single are zeros
              const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
              *reinterpret_cast<uint4*>(bt + zoff + inner) = zero;
              *reinterpret_cast<uint4*>(bt + zoff + inner + 16) = zero;
            }
          }
        }
      }
    };
    // the step of item it converts entries loaded in the step before, then loads the entries of
    // item it + 1 (records loaded in the step before) and the records of item it + 2
    Rec rc, rn;
    float4 xa[kTcMaxBlocks], xb[kTcMaxBlocks];
    load_rec(0, rc);
    load_rec(1, rn);
    load_x(rc, xa, xb);
    for (int it = 0; it < n_items; it++) {
      const int sb = it % kTcStagesB, useb = it / kTcStagesB;
      if (useb > 0 && !tc_wait(bempty + sb, (useb - 1) & 1, abort_flag, P.err, P.budget)) break;
      convert_store(it, rc, xa, xb);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(bready + sb);
      rc = rn;
      load_x(rc, xa, xb);
      load_rec(it + 2, rn);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // warp w reads TMEM lanes 32 (w % 4) ..: row 32 (w % 2) + lane of the row block, from the
    // first blocks of the units (w % 4 < 2, columns 0 .. kTcN - 1) or the second (w % 4 >= 2,
    // columns kTcN .. 2 kTcN - 1). The second-half warps pass their sums through shared memory
    // (a buffer per accumulator; xfull marks it written); the first-half warps add them and
    // write the rows. A buffer is rewritten only after its accumulator was released again,
    // which the first-half warps do after reading it.
    const int q = warp & 3;
    const bool second = q >= 2;
    float inv[kTcVec];
#pragma unroll
    for (int v = 0; v < kTcVec; v++) inv[v] = 1.0f / P.vscale[v];
    int r = 0;
    bool ok = true;
    for (int base = 0; base < n_items && ok; base += 32) {
      // 32 items at a time: the rows that end in them, in order
      int my_flags = 0, my_row = 0;
      if (base + lane < n_items) {
        const StreamItem& I = P.items[ib + base + lane];
        my_flags = I.flags;
        my_row = I.row;
      }
      unsigned ends = __ballot_sync(0xFFFFFFFFu, (my_flags & kItemFlagLast) != 0);
      for (; ends; ends &= ends - 1u) {
        const int row_off = __shfl_sync(0xFFFFFFFFu, my_row, __ffs(ends) - 1);
        const int b = r & 1;
        if (!tc_wait(accfull + b, (r >> 1) & 1, abort_flag, P.err, P.budget)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t c[kTcN];
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 2 * kTcN + (second ? kTcN : 0));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]),
              "=r"(c[8]), "=r"(c[9]), "=r"(c[10]), "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]), "=r"(c[15]),
              "=r"(c[16]), "=r"(c[17]), "=r"(c[18]), "=r"(c[19]), "=r"(c[20]), "=r"(c[21]), "=r"(c[22]),
              "=r"(c[23]), "=r"(c[24]), "=r"(c[25]), "=r"(c[26]), "=r"(c[27]), "=r"(c[28]), "=r"(c[29]),
              "=r"(c[30]), "=r"(c[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float sum[kTcVec];
#pragma unroll
        for (int v = 0; v < kTcVec; v++) sum[v] = __uint_as_float(c[2 * v]) + __uint_as_float(c[2 * v + 1]);
        float* xr = xbuf + (b * 64 + 32 * (q & 1) + lane) * (kTcVec + 1);  // stride 17: no bank conflicts
        tc_fence_before();
        if (second) {
#pragma unroll
          for (int v = 0; v < kTcVec; v++) xr[v] = sum[v];
          __syncwarp();
          if (lane == 0) {
            mbar_arrive(xfull + b);  // release: the sums are visible to the waiting warps
            mbar_arrive(accempty + b);
          }
        } else {
          if (!tc_wait(xfull + b, (r >> 1) & 1, abort_flag, P.err, P.budget)) {
            ok = false;
            break;
          }
#pragma unroll
          for (int v = 0; v < kTcVec; v++) sum[v] += xr[v];
          __syncwarp();
          if (lane == 0) mbar_arrive(accempty + b);
          const long long yo = (long long)row_off * P.rowmul + 32 * q + lane;
#pragma unroll
          for (int v = 0; v < kTcVec; v++)
            if (v < P.nv) {
              if (P.y32) reinterpret_cast<float*>(P.y)[yo + v * P.ldy] = sum[v] * inv[v];
              else P.y[yo + v * P.ldy] = (double)(sum[v] * inv[v]);
            }
        }
        r++;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

// Per-vector power-of-two scales of a pass (fp16 codes): s_v = 2^(14 - e) with 2^e above
// every |sigma x_v| and |sigma_U yhat_v| the builders form, so their parts stay below 2^14.
// vmax holds float bits of the maxima (zeroed before the pass). `warps` (a multiple of nv)
// warps run: warp w takes vector w % nv and leaves w / nv, w / nv + warps / nv, ..., and
// adds its maximum with one atomic.
template <int F>
__global__ void k_tc_vmax(const float* __restrict__ x4, const float* __restrict__ yhat, const long long* __restrict__ xp4_off,
                          long long leaves, long long leaf0, int nv, int kp, int k, float dmax, float umax,
                          long long warps, unsigned* __restrict__ vmax) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= warps || nv < 1) return;
  const int v = (int)(w % nv);
  const long long step = warps / nv;
  float m = 0.f;
  for (long long j = w / nv; j < leaves; j += step) {
    const float* xs = x4 + xp4_off[j] * nv + (long long)v * 64;
    const float* ys = yhat + ((leaf0 + j) * nv + v) * (long long)kp;
    m = fmaxf(m, fmaxf(fabsf(xs[lane]), fabsf(xs[lane + 32])) * dmax);
    for (int r = lane; r < k; r += 32) m = fmaxf(m, fabsf(ys[r]) * umax);
  }
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
  if (lane == 0) atomicMax(vmax + v, __float_as_uint(m));  // non-negative floats order as their bits
}

// The same maxima for the coupling phase: smax |xhat_v| over the first k entries of every node's
// xhat ([node][v][kp]); warp w takes vector w % nv and nodes w / nv, w / nv + warps / nv, ...
template <int F>
__global__ void k_tc_vmax_nodes(const float* __restrict__ xhat, long long nodes, int nv, int kp, int k, float smax,
                                long long warps, unsigned* __restrict__ vmax) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= warps || nv < 1) return;
  const int v = (int)(w % nv);
  const long long step = warps / nv;
  float m = 0.f;
  for (long long j = w / nv; j < nodes; j += step) {
    const float* xs = xhat + (j * nv + v) * (long long)kp;
    for (int r = lane; r < k; r += 32) m = fmaxf(m, fabsf(xs[r]) * smax);
  }
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
  if (lane == 0) atomicMax(vmax + v, __float_as_uint(m));
}

template <int F>
__global__ void k_tc_vscale(const unsigned* __restrict__ vmax, float* __restrict__ vscale, int fp16) {
  const int v = threadIdx.x;
  if (v >= kTcVec) return;
  const float m = __uint_as_float(vmax[v]);
  int e = 0;
  if (fp16 && m > 0.f && m < 3.0e38f) frexpf(m, &e);  // m < 2^e
  vscale[v] = fp16 ? ldexpf(1.0f, 14 - e) : 1.0f;
}

}  // namespace h2
