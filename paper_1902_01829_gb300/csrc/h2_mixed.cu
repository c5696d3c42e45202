// Precision form, host side: per-block quantization of the FP64 input into
// 16-bit codes with one FP32 scale per block, the device layout, the dense
// stream's work items, and the dispatch of a product pass to the storage
// format's kernels (h2_mixed_fp16.cu, h2_mixed_bf16.cu, h2_mixed_int16.cu).
//
// Quantization rule (per block of U, V, E, F, S or D; m = max |a| in FP64):
//   fp16, bf16:  sigma = fl32(m),          code = RNE16(a / sigma)
//   int16:       sigma = fl32(m / 32767),  q = clamp(rint(a / sigma), +-32767), code = q + 32768
// with a / sigma in FP64 and rounding to nearest, ties to even; sigma = 0
// gives the zero code. The block then stands for sigma * q.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "h2_internal.h"
#include "mixed.cuh"
#include "tc_dense.cuh"

namespace h2i {

template <int F>
h2_status mixed_pass_form(const MixedLaunch& L, unsigned buckets, cudaStream_t st, const TcPass* tc);

}  // namespace h2i

using namespace h2i;

namespace {

// Round a finite double to nearest (ties to even) in a binary format with MB
// explicit mantissa bits, minimum normal exponent EMIN and exponent bias EB;
// returns its 16-bit pattern. Magnitudes must stay below the format's maximum.
uint16_t round16(double r, int MB, int EMIN, int EB) {
  uint64_t u;
  std::memcpy(&u, &r, 8);
  const uint16_t sign = (u >> 63) ? 0x8000u : 0u;
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0) return sign;  // zero or an FP64 subnormal: rounds to zero
  const uint64_t mant = (u & ((1ull << 52) - 1)) | (1ull << 52);  // value = mant * 2^(e - 1075)
  const int ue = e - 1023;
  int te = std::max(ue, EMIN);              // exponent of the result's leading bit
  const int shift = (te - MB) - (ue - 52);  // low bits of mant below the result's ulp
  if (shift >= 64) return sign;
  uint64_t q = mant >> shift;
  const uint64_t rem = mant & ((1ull << shift) - 1), half = 1ull << (shift - 1);
  if (rem > half || (rem == half && (q & 1))) q++;
  if (q >> (MB + 1)) {  // carried into the next binade
    q >>= 1;
    te++;
  }
  if (q < (1ull << MB)) return (uint16_t)(sign | q);  // subnormal
  return (uint16_t)(sign | (((uint64_t)(te + EB) << MB) | (q - (1ull << MB))));
}

int form_of(int storage) {
  return storage == H2_FP16_SCALED ? h2::kFormFp16 : storage == H2_BF16_SCALED ? h2::kFormBf16 : h2::kFormInt16;
}

// quantize cnt FP64 values into codes; returns the block's scale
float quantize(const double* a, int64_t cnt, int form, uint16_t* codes) {
  double m = 0.0;
  for (int64_t i = 0; i < cnt; i++) m = std::max(m, std::fabs(a[i]));
  const float sigma = (form == h2::kFormInt16) ? (float)(m / 32767.0) : (float)m;
  const uint16_t zero = (form == h2::kFormInt16) ? 32768u : 0u;
  if (sigma == 0.0f) {
    for (int64_t i = 0; i < cnt; i++) codes[i] = zero;
    return 0.0f;
  }
  const double s = (double)sigma;
  for (int64_t i = 0; i < cnt; i++) {
    const double r = a[i] / s;
    if (form == h2::kFormFp16) {
      codes[i] = round16(r, 10, -14, 15);
    } else if (form == h2::kFormBf16) {
      codes[i] = round16(r, 7, -126, 127);
    } else {
      const double q = std::min(32767.0, std::max(-32767.0, std::nearbyint(r)));
      codes[i] = (uint16_t)((int)q + 32768);
    }
  }
  return sigma;
}

// quantize then transpose a rows x cols column-major block into cols x rows codes
float quantize_transposed(const double* a, int64_t rows, int64_t cols, int form, uint16_t* codes,
                          std::vector<uint16_t>& tmp) {
  tmp.resize((size_t)(rows * cols));
  const float s = quantize(a, rows * cols, form, tmp.data());
  for (int64_t c = 0; c < cols; c++)
    for (int64_t r = 0; r < rows; r++) codes[c + cols * r] = tmp[r + rows * c];
  return s;
}

// the product's fields (vectors, leading dimensions, vector counts) of up to
// kCallChunk matrices, passed by value so that a captured graph replays them
constexpr int kCallChunk = 256;
struct CallChunk {
  int first, count;
  const double* x[kCallChunk];
  double* y[kCallChunk];
  long long ldx[kCallChunk];
  long long ldy[kCallChunk];
  int nv[kCallChunk];
  int xy32;
};
static_assert(sizeof(CallChunk) < 32000, "kernel parameter space");

__global__ void k_set_calls(h2::MatDesc* mats, CallChunk c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < c.count) {
    h2::MatDesc& D = mats[c.first + i];
    D.x = c.x[i];
    D.ldx = c.ldx[i];
    D.y = c.y[i];
    D.ldy = c.ldy[i];
    D.nv = c.nv[i];
    D.xy32 = c.xy32;
  }
}

// static fields of a handle's matrix descriptor; row0 = its first row in the coupling row space
h2::MatDesc fill_desc(const h2_matrix_s* h, int tree_L) {
  const MixedData& M = h->mx;
  h2::MatDesc D{};
  D.dmat = static_cast<const char*>(M.dmat);
  D.smat = M.smat;
  D.sscale = M.sscale;
  D.Srow = h->Srow;
  D.Scol = h->Scol;
  D.Vt = M.Vt;
  D.vscale = M.vscale;
  D.vt_off = M.vt_off;
  D.Ft = M.Ft;
  D.fscale = M.fscale;
  D.E = M.E;
  D.escale = M.escale;
  D.leaf_off = h->leaf_off;
  D.xp4_off = M.xp4_off;
  D.x4 = M.x4;
  D.xhat = M.xhat;
  D.yhat = M.yhat;
  D.ticket = h->ticket;
  D.kk8 = M.kk8;
  D.n_nodes = h->n_nodes;
  D.k = h->k;
  D.kp = M.kp4;
  D.LR = h->lr;
  D.q = h->q;
  D.L = tree_L;
  D.kf_chi = M.kf_chi;
  D.kf_clo = M.kf_clo;
  D.kf_off = M.kf_off;
  D.kf_inv_ell = h->kf_inv_ell;
  D.kf_kind = h->kf_kind;
  D.spanel = M.spanel ? 1 : 0;
  D.rjobs = static_cast<const h2::RowJob*>(M.rjobs);
  D.blk = static_cast<const h2::MixedBlock*>(M.dblk);
  return D;
}

// write the fields of one product pass into a matrix table (entries [0, count))
h2_status set_calls(h2::MatDesc* mats, int64_t count, const int* nv, const double* const* x, const int64_t* ldx,
                    double* const* y, const int64_t* ldy, cudaStream_t st, int xy32 = 0) {
  for (int64_t c0 = 0; c0 < count; c0 += kCallChunk) {
    CallChunk c{};
    c.first = (int)c0;
    c.xy32 = xy32;
    c.count = (int)std::min<int64_t>(kCallChunk, count - c0);
    for (int i = 0; i < c.count; i++) {
      c.x[i] = x[c0 + i];
      c.y[i] = y[c0 + i];
      c.ldx[i] = ldx[c0 + i];
      c.ldy[i] = ldy[c0 + i];
      c.nv[i] = nv[c0 + i];
    }
    k_set_calls<<<(c.count + 127) / 128, 128, 0, st>>>(mats, c);
  }
  return H2_OK;
}

}  // namespace

// ---------------------------------------------------------------- dense blocks generated on the device
// D_ij[a][b] = K(x_a, x_b) for the points of leaves i and j (Sec. 2.2, Sec. 4.6), evaluated in FP64
// exactly as the host generator evaluates it, then quantized with the host quantizer's rule
// (quantize() above): sigma = fl32(max |a|) (int16: fl32(max |a| / 32767)), codes of a / sigma
// rounded to nearest even (int16: rint, clamped to +-32767, offset by 32768). One CTA per block.
struct GenDense {
  const double* pts;        // n x dim, cluster order
  const int64_t* leaf_off;  // [leaves + 1]
  const int32_t* brow;      // per dense block: row leaf, column leaf
  const int32_t* bcol;
  const int64_t* bbyte;     // byte offset of the block's codes in dmat
  const int64_t* bglob;     // index of the block's record
  int64_t nblocks;
  unsigned char* dmat;
  h2::MixedBlock* blk;
  double ell;
  int dim, kind, panel;
};

template <int F>
__device__ __forceinline__ uint16_t gen_code(double v, float sigma) {
  if (sigma == 0.0f) return F == h2::kFormInt16 ? 32768u : 0u;
  const double r = v / (double)sigma;
  if constexpr (F == h2::kFormFp16) return __half_as_ushort(__double2half(r));
  else if constexpr (F == h2::kFormBf16) return __bfloat16_as_ushort(__double2bfloat16(r));
  else return (uint16_t)((int)fmin(32767.0, fmax(-32767.0, rint(r))) + 32768);
}

template <int F>
__global__ void __launch_bounds__(256) k_gen_dense(GenDense a) {
  __shared__ double xs[2][64 * 3];
  __shared__ double wmax[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < a.nblocks; t += gridDim.x) {
    const int i = a.brow[t], j = a.bcol[t];
    const int64_t oi = a.leaf_off[i], oj = a.leaf_off[j];
    const int si = (int)(a.leaf_off[i + 1] - oi < 64 ? a.leaf_off[i + 1] - oi : 64);
    const int sj = (int)(a.leaf_off[j + 1] - oj < 64 ? a.leaf_off[j + 1] - oj : 64);
    for (int e = threadIdx.x; e < si * a.dim; e += 256) xs[0][e] = a.pts[oi * a.dim + e];
    for (int e = threadIdx.x; e < sj * a.dim; e += 256) xs[1][e] = a.pts[oj * a.dim + e];
    __syncthreads();
    double v[16];
    double m = 0.0;
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int e = threadIdx.x + 256 * u;
      v[u] = 0.0;
      if (e < si * sj) {
        const int r = e % si, c = e / si;
        double r2 = 0.0;
        for (int d = 0; d < a.dim; d++) {
          const double df = xs[0][r * a.dim + d] - xs[1][c * a.dim + d];
          r2 += df * df;
        }
        const double rr = sqrt(r2);
        double kv;
        if (a.kind == H2_KERNEL_EXP) {
          kv = exp(-rr / a.ell);
        } else {
          const double s = 1.7320508075688772 * rr / a.ell;
          kv = (1.0 + s) * exp(-s);
        }
        v[u] = kv;
        m = fmax(m, fabs(kv));
      }
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    m = wmax[0];
#pragma unroll
    for (int w = 1; w < 8; w++) m = fmax(m, wmax[w]);
    const float sigma = F == h2::kFormInt16 ? (float)(m / 32767.0) : (float)m;
    uint16_t* dst = reinterpret_cast<uint16_t*>(a.dmat + a.bbyte[t]);
    const int ps2 = h2::panel_stride(sj) / 2;
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int e = threadIdx.x + 256 * u;
      if (e < si * sj) {
        const int r = e % si, c = e / si;
        dst[a.panel ? (r >> 3) * ps2 + 8 * c + (r & 7) : r + si * c] = gen_code<F>(v[u], sigma);
      }
    }
    if (threadIdx.x == 0) a.blk[a.bglob[t]].scale = sigma;
    __syncthreads();  // xs and wmax are reused by the next block
  }
}

// copy blocks of whole 16-byte words: block t from src + soff[t] to dst + doff[t] (bytes[t] bytes)
__global__ void k_scatter_blocks(const unsigned char* __restrict__ src, const int64_t* __restrict__ soff,
                                 unsigned char* __restrict__ dst, const int64_t* __restrict__ doff,
                                 const int64_t* __restrict__ bytes, int64_t nblocks) {
  for (int64_t t = blockIdx.x; t < nblocks; t += gridDim.x) {
    const int4* s = reinterpret_cast<const int4*>(src + soff[t]);
    int4* d = reinterpret_cast<int4*>(dst + doff[t]);
    for (int64_t w = threadIdx.x; w < bytes[t] / 16; w += blockDim.x) d[w] = s[w];
  }
}

// device buffer freed when it goes out of scope (temporaries of a handle's creation)
template <class T>
struct DevTemp {
  T* p = nullptr;
  ~DevTemp() {
    if (p) cudaFree(p);
  }
  h2_status put(const T* src, int64_t count) {
    cudaError_t e = cudaMalloc(&p, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess && count > 0) e = cudaMemcpy(p, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return h2_fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, "temporary device buffer: %s",
                     cudaGetErrorString(e));
    }
    return H2_OK;
  }
};

static_assert(h2i::kDenseCW == h2::kMixedCW, "dense-stream consumer warps");

// The dense stream's producer stages the block records of 32 consecutive items of a CTA at a
// time; their block range must fit its buffer (kMixedBatchBlocks records).
h2_status audit_producer_batches(const std::vector<h2::StreamItem>& items, const std::vector<int>& begin) {
  for (size_t c = 0; c + 1 < begin.size(); c++)
    for (int base = begin[c]; base < begin[c + 1]; base += 32) {
      const h2::StreamItem& a = items[(size_t)base];
      const h2::StreamItem& z = items[(size_t)std::min(base + 31, begin[c + 1] - 1)];
      const long long span = z.v_off + ((z.shape >> 8) & 0xFF) - a.v_off;
      if (span < 0 || span > h2::kMixedBatchBlocks)
        return h2_fail(H2_ERR_INVALID, "internal: 32 work items span %lld block records", span);
    }
  return H2_OK;
}


namespace h2i {

// coupling row chunks of one matrix: consecutive rows, at most kChunkRows rows
// and (unless one row alone has more) about `target` coupling blocks each
std::vector<int4> coupling_chunks(const int32_t* Srow, int64_t n_nodes, int64_t target) {
  std::vector<int4> out;
  for (int64_t r = 0; r < n_nodes;) {
    const int64_t r0 = r;
    int64_t blocks = 0;
    while (r < n_nodes && r - r0 < h2::kChunkRows && (r == r0 || blocks + (Srow[r + 1] - Srow[r]) <= target)) {
      blocks += Srow[r + 1] - Srow[r];
      r++;
    }
    out.push_back(make_int4(0, (int)r0, (int)(r - r0), 0));
  }
  return out;
}

h2_status mixed_configure(h2_matrix_s* h, int chunk_opt, int cw, int tree_opt) {
  MixedData& M = h->mx;
  if (chunk_opt < 0 || chunk_opt > 2 || tree_opt < 0 || tree_opt > 2 ||
      (cw != h2::kMixedCW && cw != 2 * h2::kMixedCW))
    return h2_fail(H2_ERR_INVALID, "internal: launch configuration out of range");
  if (tree_opt != M.tree_opt) {  // subtree level of the tree jobs (in the descriptor and the job list)
    const int L = std::max(0, h->tree_L - tree_opt);
    if (!M.jobs_dev[tree_opt]) {
      std::vector<int2> jobs((size_t)1 << L);
      for (size_t t = 0; t < jobs.size(); t++) jobs[t] = make_int2(0, (int)t);
      h2_status st = upload(h, &M.jobs_dev[tree_opt], jobs.data(), (int64_t)jobs.size());
      if (st != H2_OK) return st;
    }
    const h2::MatDesc D = fill_desc(h, L);
    if (!M.launch.mats) {
      h2::MatDesc* md = nullptr;
      h2_status st = upload(h, &md, &D, 1);
      if (st != H2_OK) return st;
      M.launch.mats = md;
    } else {
      CUDA_TRY(cudaMemcpy(M.launch.mats, &D, sizeof(D), cudaMemcpyHostToDevice));
    }
    M.launch.jobs = M.jobs_dev[tree_opt];
    M.launch.njobs = (int64_t)1 << L;
    M.tree_opt = tree_opt;
  }
  if (!M.chunk_dev[chunk_opt]) {
    const std::vector<int4> c = coupling_chunks(M.srow_host.data(), h->n_nodes, kChunkOpts[chunk_opt]);
    h2_status st = upload(h, &M.chunk_dev[chunk_opt], c.data(), (int64_t)c.size());
    if (st != H2_OK) return st;
    M.chunk_n[chunk_opt] = (int64_t)c.size();
  }
  M.chunks_host = coupling_chunks(M.srow_host.data(), h->n_nodes, kChunkOpts[chunk_opt]);
  M.launch.chunks = M.chunk_dev[chunk_opt];
  M.launch.nchunks = M.chunk_n[chunk_opt];
  M.launch.cw = cw;
  return H2_OK;
}

// The coupling phase's tensor-core items (k = 64, codes in the unpadded panel layout): the blocks of
// each coupling row, up to four per item (two M = 128 pairs), in row order; the builders' records
// name each block's column node (xhat offset j kp, second vector source), K = 64 and its scale.
// Rows are weighed by bytes and MMAs, as the dense phase's.
h2_status build_coupling_items(h2_matrix_s* h, const h2_desc* d, const std::vector<float>& sc) {
  MixedData& M = h->mx;
  const int64_t nodes = h->n_nodes, bbytes = 64 * 64 * 2;
  const int32_t* Srow = d->S_rowptr;
  const int32_t* Scol = d->S_colidx;
  std::vector<h2::StreamItem> items;
  std::vector<int32_t> brec;
  std::vector<int64_t> row_bytes((size_t)nodes, 0), row_item0((size_t)nodes + 1, 0);
  constexpr int kBlocks = 4;
  int kp[h2::kTcMaxBlocks], bo[h2::kTcMaxBlocks], pm = 0, sm = 0;
  for (int u = 0; u < h2::kTcMaxBlocks; u++) kp[u] = 64;
  for (int64_t i = 0; i < nodes; i++) {
    row_item0[(size_t)i] = (int64_t)items.size();
    const int64_t g0 = Srow[i], g1 = Srow[i + 1];
    for (int64_t g = g0; g < g1; g += kBlocks) {
      const int nb = (int)std::min<int64_t>(kBlocks, g1 - g);
      if (h2::tc_layout(nb, kp, bo, &pm, &sm) > h2::kTcStageB || nb * bbytes > h2::kTcStageMat)
        return h2_fail(H2_ERR_INVALID, "internal: coupling item exceeds a tensor-core stage");
      h2::StreamItem it{};
      it.m_off = g * bbytes;
      it.m_bytes = (int)(nb * bbytes);
      it.shape = 64u | ((unsigned)nb << 8);
      it.v_off = g;
      it.row = (int)i;
      it.flags = (g + nb == g1 ? h2::kItemFlagLast : 0) | (pm << h2::kTcPairShift);
      items.push_back(it);
      int32_t r[h2::kTcRecInts] = {0};
      r[0] = nb | (pm << 8);
      for (int u = 0; u < nb; u++) {
        const int64_t j = Scol[g + u];
        if (j < 0 || j >= nodes || j * 64 > INT32_MAX)
          return h2_fail(H2_ERR_UNSUPPORTED, "coupling column %lld exceeds the tensor-core records", (long long)j);
        r[1 + 3 * u] = (int32_t)(j * 64);
        r[2 + 3 * u] = 64 | (1 << 16);
        std::memcpy(&r[3 + 3 * u], &sc[(size_t)(g + u)], sizeof(float));
      }
      brec.insert(brec.end(), r, r + h2::kTcRecInts);
      int64_t mmas = 0;
      for (int u = 0; u < nb; u++)
        if (((pm | sm) >> u) & 1) mmas += 4;
      row_bytes[(size_t)i] += nb * bbytes + 4096 * mmas + 512;
    }
  }
  row_item0[(size_t)nodes] = (int64_t)items.size();
  if (items.empty()) return h2_fail(H2_ERR_INVALID, "internal: coupling blocks without coupling items");
  if (items.size() > (size_t)INT32_MAX) return h2_fail(H2_ERR_UNSUPPORTED, "too many coupling items");
  const std::vector<int> begin = balance(row_bytes, row_item0, h->grid);
  for (size_t c = 0; c + 1 < begin.size(); c++)
    if (begin[c] > begin[c + 1]) return h2_fail(H2_ERR_INVALID, "internal: item ranges not monotone");
  for (const h2::StreamItem& it : items) {  // audit, as the kernel reads the items
    const int nb = (int)((it.shape >> 8) & 0xFF);
    const bool ok = nb >= 1 && nb <= kBlocks && it.m_off % 16 == 0 && it.m_bytes == nb * bbytes &&
                    it.m_off + it.m_bytes <= h->nS * bbytes && it.row >= 0 && it.row < nodes;
    if (!ok) return h2_fail(H2_ERR_INVALID, "internal: coupling tensor-core item fails the layout audit");
  }
  h2_status st;
  if ((st = upload(h, &M.tc_sbrec, reinterpret_cast<const int4*>(brec.data()), (int64_t)items.size() * (h2::kTcRecInts / 4))) != H2_OK)
    return st;
  if ((st = upload(h, &M.tc_sitems.items, items.data(), (int64_t)items.size())) != H2_OK) return st;
  if ((st = upload(h, &M.tc_sitems.cta_begin, begin.data(), (int64_t)begin.size())) != H2_OK) return st;
  M.tc_sitems.count = (int64_t)items.size();
  return H2_OK;
}

h2_status mixed_build(h2_matrix_s* h, const h2_desc* d) {
  MixedData& M = h->mx;
  const int form = form_of(h->storage);
  const int k = h->k;
  const int64_t kk = (int64_t)k * k, kk8 = round_up(kk, 8), leaves = h->leaves, nodes = h->n_nodes;
  M.kk8 = kk8;
  M.kp4 = (int)round_up(k, 4);
  const int64_t* lo = d->leaf_offset;
  const double* V = d->symmetric ? d->U : d->V;
  const double* F = d->symmetric ? d->E : d->F;
  h2_status st;

  // FP32 x layout: leaf chunks padded to multiples of 4
  std::vector<int64_t> xp4((size_t)leaves + 1, 0), vto((size_t)leaves + 1, 0);
  for (int64_t j = 0; j < leaves; j++) {
    xp4[j + 1] = xp4[j] + round_up(lo[j + 1] - lo[j], 4);
    vto[j + 1] = vto[j] + round_up((lo[j + 1] - lo[j]) * k, 8);
  }
  if ((st = upload(h, &M.xp4_off, xp4.data(), leaves + 1)) != H2_OK) return st;
  if ((st = upload(h, &M.vt_off, vto.data(), leaves + 1)) != H2_OK) return st;

  M.bases_fp32 = d->bases_fp32 != 0;
  {  // leaf bases V^T, transfers F^T and E: 16-bit codes, or FP32 entries with scale 1
    const int64_t nb_ent = std::max<int64_t>(vto[leaves], (nodes - 1) * kk8);
    std::vector<float> sc((size_t)std::max<int64_t>(leaves, nodes - 1), 1.f);
    if (M.bases_fp32) {
      std::vector<float> ent((size_t)nb_ent, 0.f);
      for (int64_t j = 0; j < leaves; j++)
        for (int64_t c = 0; c < k; c++)
          for (int64_t r = 0; r < lo[j + 1] - lo[j]; r++)
            ent[vto[j] + c + k * r] = (float)V[lo[j] * k + r + (lo[j + 1] - lo[j]) * c];
      float* p = nullptr;
      if ((st = upload(h, &p, ent.data(), vto[leaves])) != H2_OK) return st;
      M.Vt = p;
      if ((st = upload(h, &M.vscale, sc.data(), leaves)) != H2_OK) return st;
      for (int64_t c = 0; c < nodes - 1; c++)
        for (int64_t i = 0; i < k; i++)
          for (int64_t j = 0; j < k; j++) ent[c * kk8 + j + k * i] = (float)F[c * kk + i + k * j];
      if ((st = upload(h, &p, ent.data(), (nodes - 1) * kk8)) != H2_OK) return st;
      M.Ft = p;
      for (int64_t c = 0; c < nodes - 1; c++)
        for (int64_t i = 0; i < kk; i++) ent[c * kk8 + i] = (float)d->E[c * kk + i];
      if ((st = upload(h, &p, ent.data(), (nodes - 1) * kk8)) != H2_OK) return st;
      M.E = p;
      if ((st = upload(h, &M.fscale, sc.data(), nodes - 1)) != H2_OK) return st;
      if ((st = upload(h, &M.escale, sc.data(), nodes - 1)) != H2_OK) return st;
    } else {
      std::vector<uint16_t> codes((size_t)nb_ent, 0);
#pragma omp parallel
      {
        std::vector<uint16_t> tmp;
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < leaves; j++)
          sc[j] = quantize_transposed(V + lo[j] * k, lo[j + 1] - lo[j], k, form, codes.data() + vto[j], tmp);
      }
      uint16_t* p = nullptr;
      if ((st = upload(h, &p, codes.data(), vto[leaves])) != H2_OK) return st;
      M.Vt = p;
      if ((st = upload(h, &M.vscale, sc.data(), leaves)) != H2_OK) return st;
#pragma omp parallel
      {
        std::vector<uint16_t> tmp;
#pragma omp for schedule(dynamic, 256)
        for (int64_t c = 0; c < nodes - 1; c++)
          sc[c] = quantize_transposed(F + c * kk, k, k, form, codes.data() + c * kk8, tmp);
      }
      if ((st = upload(h, &p, codes.data(), (nodes - 1) * kk8)) != H2_OK) return st;
      M.Ft = p;
      if ((st = upload(h, &M.fscale, sc.data(), nodes - 1)) != H2_OK) return st;
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t c = 0; c < nodes - 1; c++) sc[c] = quantize(d->E + c * kk, kk, form, codes.data() + c * kk8);
      if ((st = upload(h, &p, codes.data(), (nodes - 1) * kk8)) != H2_OK) return st;
      M.E = p;
      if ((st = upload(h, &M.escale, sc.data(), nodes - 1)) != H2_OK) return st;
    }
  }
  if (h->kc) {
    // coupling blocks evaluated in the product from the kernel at the interpolation points
    // (Sec. 4.6): per node its centre c (midpoint of its Chebyshev nodes per dimension) as an
    // FP32 pair hi + lo, and its k points as FP32 offsets from c (tensor index, dimension 0
    // slowest); unused dimensions are 0
    const h2_coupling_kernel* kc = h->kc;
    const int dim = kc->dim, p = kc->p;
    std::vector<float4> chi((size_t)nodes), clo((size_t)nodes), off((size_t)(nodes * k));
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < nodes; n++) {
      double c[3] = {0.0, 0.0, 0.0};
      float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
      for (int e = 0; e < dim; e++) {
        const double* cd = kc->cheb + (n * dim + e) * p;
        double a = cd[0], b = cd[0];
        for (int t = 1; t < p; t++) {
          a = std::min(a, cd[t]);
          b = std::max(b, cd[t]);
        }
        c[e] = 0.5 * (a + b);
        hi[e] = (float)c[e];
        lo[e] = (float)(c[e] - (double)hi[e]);
      }
      chi[(size_t)n] = make_float4(hi[0], hi[1], hi[2], 0.f);
      clo[(size_t)n] = make_float4(lo[0], lo[1], lo[2], 0.f);
      for (int nu = 0; nu < k; nu++) {
        float o[3] = {0.f, 0.f, 0.f};
        int rem = nu;
        for (int e = dim - 1; e >= 0; e--) {
          const int a = rem % p;
          rem /= p;
          o[e] = (float)(kc->cheb[(n * dim + e) * p + a] - c[e]);
        }
        off[(size_t)(n * k + nu)] = make_float4(o[0], o[1], o[2], 0.f);
      }
    }
    if ((st = upload(h, &M.kf_chi, chi.data(), nodes)) != H2_OK) return st;
    if ((st = upload(h, &M.kf_clo, clo.data(), nodes)) != H2_OK) return st;
    if ((st = upload(h, &M.kf_off, off.data(), nodes * k)) != H2_OK) return st;
  } else {  // coupling blocks S (always 16-bit codes)
    std::vector<uint16_t> codes((size_t)std::max<int64_t>(1, h->nS * kk8), 0);
    std::vector<float> sc((size_t)std::max<int64_t>(1, h->nS), 0.f);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t b = 0; b < h->nS; b++) sc[b] = quantize(d->S_val + b * kk, kk, form, codes.data() + b * kk8);
    // fp16 / bf16 at k = 64: the codes in the panel layout without the pad (the tensor cores' MN-major
    // operand layout: rows 8m .. 8m + 7 of column c at codes 512 m + 8 c), so that passes of 8 or
    // more vectors run the coupling phase on the tensor cores
    M.spanel = form != h2::kFormInt16 && k == 64 && h->nS > 0;
    if (M.spanel) {
#pragma omp parallel
      {
        uint16_t tmp[4096];
#pragma omp for schedule(static)
        for (int64_t b = 0; b < h->nS; b++) {
          uint16_t* blk = codes.data() + b * kk8;
          for (int c = 0; c < 64; c++)
            for (int m = 0; m < 8; m++)
              for (int i = 0; i < 8; i++) tmp[512 * m + 8 * c + i] = blk[64 * c + 8 * m + i];
          std::memcpy(blk, tmp, sizeof(tmp));
        }
      }
      for (int64_t b = 0; b < h->nS; b++) M.smax = std::max(M.smax, sc[b]);
      if ((st = build_coupling_items(h, d, sc)) != H2_OK) return st;
    }
    if ((st = upload(h, &M.smat, codes.data(), h->nS * kk8)) != H2_OK) return st;
    if ((st = upload(h, &M.sscale, sc.data(), h->nS)) != H2_OK) return st;
  }

  {  // dense stream: row i holds its dense blocks then U_i, contiguous, each padded to 16 bytes
    const int64_t ubytes = M.bases_fp32 ? 4 : 2;
    std::vector<int64_t> doff((size_t)h->nD + 1, 0);  // FP64 input offsets
    // panel layout (the tensor-core operand layout) when every leaf has 64 points and the
    // blocks are 16-bit floating-point codes with a rank that is a multiple of 16
    bool panel = form != h2::kFormInt16 && !M.bases_fp32 && k % 16 == 0 && k <= 64;
    for (int64_t i = 0; panel && i < leaves; i++) panel = lo[i + 1] - lo[i] == 64;
    M.panel = panel;
    std::vector<int64_t> row_blk0((size_t)leaves + 1, 0), boff((size_t)(h->nD + leaves) + 1, 0);
    for (int64_t i = 0, b = 0; i < leaves; i++) {
      row_blk0[i] = b + i;  // global block index of the row's first block (dense blocks + one U per row)
      const int64_t si = lo[i + 1] - lo[i];
      for (; b < d->D_rowptr[i + 1]; b++) {
        const int64_t sj = lo[d->D_colidx[b] + 1] - lo[d->D_colidx[b]], sz = si * sj;
        doff[b + 1] = doff[b] + sz;
        boff[b + i + 1] = boff[b + i] + (panel ? h2::panel_block_bytes((int)sj) : round_up(sz * 2, 16));
      }
      boff[b + i + 1] = boff[b + i] + (panel ? h2::panel_block_bytes(k) : round_up(si * k * ubytes, 16));  // U_i
    }
    row_blk0[leaves] = h->nD + leaves;
    const int64_t nblk = h->nD + leaves, total = boff[nblk];  // bytes
    // dense blocks generated on the device: the host assembles only the U blocks, compactly
    const bool gen = h->gen_points != nullptr;
    std::vector<int64_t> uoffc(gen ? (size_t)leaves + 1 : 0, 0);
    for (int64_t i = 0; gen && i < leaves; i++) {
      const int64_t g1 = row_blk0[i + 1] - 1;
      uoffc[i + 1] = uoffc[i] + (boff[g1 + 1] - boff[g1]);
    }
    std::vector<unsigned char> bytes_host((size_t)(gen ? uoffc[leaves] : total), 0);
    unsigned char* base = bytes_host.data();
    std::vector<h2::MixedBlock> blk((size_t)nblk);
#pragma omp parallel
    {
      std::vector<uint16_t> tmp;
      // codes of a 64-row column-major block into the panel layout at dst
      auto to_panels = [&](int64_t C, uint16_t* dst) {
        const int64_t ps = h2::panel_stride((int)C) / 2;
        for (int64_t c = 0; c < C; c++)
          for (int64_t r = 0; r < 64; r++) dst[(r >> 3) * ps + c * 8 + (r & 7)] = tmp[r + 64 * c];
      };
#pragma omp for schedule(dynamic, 16)
      for (int64_t i = 0; i < leaves; i++) {
        const int64_t si = lo[i + 1] - lo[i];
        int64_t g = row_blk0[i];
        for (int32_t b = d->D_rowptr[i]; b < d->D_rowptr[i + 1]; b++, g++) {
          const int32_t j = d->D_colidx[b];
          const int64_t sj = lo[j + 1] - lo[j];
          h2::MixedBlock& m = blk[g];
          if (gen) {
            m.scale = 0.f;  // the device writes the codes and the scale
          } else if (panel) {
            tmp.resize((size_t)(si * sj));
            m.scale = quantize(d->D_val + doff[b], si * sj, form, tmp.data());
            to_panels(sj, reinterpret_cast<uint16_t*>(base + boff[g]));
          } else {
            m.scale = quantize(d->D_val + doff[b], si * sj, form, reinterpret_cast<uint16_t*>(base + boff[g]));
          }
          m.voff = xp4[j];
          m.cols = (unsigned short)sj;
          m.vs = (unsigned char)round_up(sj, 4);
          m.src = panel ? 4 : 0;
        }
        h2::MixedBlock& m = blk[g];  // U_i, multiplied with yhat of leaf i
        unsigned char* ub = gen ? base + uoffc[i] : base + boff[g];
        if (M.bases_fp32) {
          float* u = reinterpret_cast<float*>(ub);
          for (int64_t e = 0; e < si * k; e++) u[e] = (float)d->U[lo[i] * k + e];
          m.scale = 1.0f;
          m.src = 1 | 2;
        } else if (panel) {
          tmp.resize((size_t)(si * k));
          m.scale = quantize(d->U + lo[i] * k, si * k, form, tmp.data());
          to_panels(k, reinterpret_cast<uint16_t*>(ub));
          m.src = 1 | 4;
        } else {
          m.scale = quantize(d->U + lo[i] * k, si * k, form, reinterpret_cast<uint16_t*>(ub));
          m.src = 1;
        }
        m.voff = (h->leaf0 + i) * M.kp4;
        m.cols = (unsigned short)k;
        m.vs = (unsigned char)M.kp4;
      }
    }
    unsigned char* dm = nullptr;
    h2::MixedBlock* dblk = nullptr;
    if (!gen) {
      if ((st = upload(h, &dm, base, total)) != H2_OK) return st;
      if ((st = upload(h, &dblk, blk.data(), nblk)) != H2_OK) return st;
    } else {
      // the U blocks go to their places; every dense block is evaluated and quantized on the device
      if ((st = dalloc(h, &dm, total)) != H2_OK) return st;
      CUDA_TRY(cudaMemset(dm, 0, (size_t)total));
      if ((st = upload(h, &dblk, blk.data(), nblk)) != H2_OK) return st;
      {
        std::vector<int64_t> soff((size_t)leaves), doffu((size_t)leaves), ubytes((size_t)leaves);
        for (int64_t i = 0; i < leaves; i++) {
          const int64_t g1 = row_blk0[i + 1] - 1;
          soff[i] = uoffc[i];
          doffu[i] = boff[g1];
          ubytes[i] = boff[g1 + 1] - boff[g1];
        }
        DevTemp<unsigned char> tu;
        DevTemp<int64_t> ts, td, tb;
        if ((st = tu.put(base, uoffc[leaves])) != H2_OK || (st = ts.put(soff.data(), leaves)) != H2_OK ||
            (st = td.put(doffu.data(), leaves)) != H2_OK || (st = tb.put(ubytes.data(), leaves)) != H2_OK)
          return st;
        k_scatter_blocks<<<(unsigned)std::min<int64_t>(leaves, 8 * h->grid), 128>>>(tu.p, ts.p, dm, td.p, tb.p, leaves);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaDeviceSynchronize());
      }
      {
        std::vector<int32_t> brow((size_t)h->nD), bcol((size_t)h->nD);
        std::vector<int64_t> bbyte((size_t)h->nD), bglob((size_t)h->nD);
        for (int64_t i = 0; i < leaves; i++) {
          int64_t g = row_blk0[i];
          for (int32_t b = d->D_rowptr[i]; b < d->D_rowptr[i + 1]; b++, g++) {
            brow[b] = (int32_t)i;
            bcol[b] = d->D_colidx[b];
            bbyte[b] = boff[g];
            bglob[b] = g;
          }
        }
        const int dim = h->kc->dim;
        DevTemp<double> tp;
        DevTemp<int32_t> tr, tc;
        DevTemp<int64_t> tby, tgl;
        if ((st = tp.put(h->gen_points, h->n * dim)) != H2_OK || (st = tr.put(brow.data(), h->nD)) != H2_OK ||
            (st = tc.put(bcol.data(), h->nD)) != H2_OK || (st = tby.put(bbyte.data(), h->nD)) != H2_OK ||
            (st = tgl.put(bglob.data(), h->nD)) != H2_OK)
          return st;
        GenDense ga{};
        ga.pts = tp.p;
        ga.leaf_off = h->leaf_off;
        ga.brow = tr.p;
        ga.bcol = tc.p;
        ga.bbyte = tby.p;
        ga.bglob = tgl.p;
        ga.nblocks = h->nD;
        ga.dmat = dm;
        ga.blk = dblk;
        ga.ell = h->kc->ell;
        ga.dim = dim;
        ga.kind = h->kc->kernel;
        ga.panel = panel ? 1 : 0;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(h->nD, 16 * h->grid));
        if (form == h2::kFormFp16) k_gen_dense<h2::kFormFp16><<<grid, 256>>>(ga);
        else if (form == h2::kFormBf16) k_gen_dense<h2::kFormBf16><<<grid, 256>>>(ga);
        else k_gen_dense<h2::kFormInt16><<<grid, 256>>>(ga);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaDeviceSynchronize());
      }
      CUDA_TRY(cudaMemcpy(blk.data(), dblk, (size_t)nblk * sizeof(h2::MixedBlock), cudaMemcpyDeviceToHost));
    }
    M.dmat = dm;
    M.dblk = dblk;
    for (int64_t g = 0; g < nblk; g++) {
      float& mx = (blk[g].src & 1) ? M.umax : M.dmax;
      mx = std::max(mx, blk[g].scale);
    }

    // work items: consecutive dense blocks of one row, at most kMixedMaxBlocks blocks, 32 KB of
    // entries and kMixedVecCols vector columns per item. U_i (the row's last block) is not
    // streamed: the leaf expansion at the end of the downsweep multiplies it, so that the dense
    // phase does not wait for the tree phases.
    std::vector<h2::StreamItem> items;
    std::vector<int64_t> row_bytes((size_t)leaves), row_item0((size_t)leaves + 1);
    std::vector<h2::RowJob> rj((size_t)leaves);
    for (int64_t i = 0; i < leaves; i++) {
      row_item0[i] = (int64_t)items.size();
      const int64_t g0 = row_blk0[i], g1 = row_blk0[i + 1] - 1;  // [g0, g1) dense blocks, g1 = U_i
      rj[i] = h2::RowJob{boff[g1], 0, (int)i, (int)g1, g1 > g0 ? 1 : 0, {0, 0}};
      int64_t bytes = 0;
      for (int64_t g = g0; g < g1;) {
        int64_t e = g, mb = 0, vc = 0;
        while (e < g1 && e - g < h2::kMixedMaxBlocks && mb + (boff[e + 1] - boff[e]) <= h2::kStageMat &&
               vc + blk[e].vs <= h2::kMixedVecCols) {
          mb += boff[e + 1] - boff[e];
          vc += blk[e].vs;
          e++;
        }
        h2::StreamItem it{};
        it.m_off = boff[g];
        it.m_bytes = (int)mb;
        it.shape = (unsigned)(lo[i + 1] - lo[i]) | ((unsigned)(e - g) << 8);
        it.v_off = g;
        it.row = (int)lo[i];
        it.flags = (e == g1) ? h2::kItemFlagLast : 0;
        items.push_back(it);
        bytes += mb + 4 * vc + 512;  // entries, one vector's columns, and a fixed cost per item
        g = e;
      }
      row_bytes[i] = bytes;
    }
    row_item0[leaves] = (int64_t)items.size();
    const std::vector<int> begin = balance(row_bytes, row_item0, h->grid);
    if ((st = audit_producer_batches(items, begin)) != H2_OK) return st;
    // audit: every copy in bounds, 16-byte aligned, and within its stage slot
    for (size_t c = 0; c + 1 < begin.size(); c++)
      if (begin[c] > begin[c + 1]) return h2_fail(H2_ERR_INVALID, "internal: item ranges not monotone");
    for (size_t t = 0; t < items.size(); t++) {
      const h2::StreamItem& it = items[t];
      const int nb = (int)((it.shape >> 8) & 0xFF);
      bool ok = it.m_off % 16 == 0 && it.m_bytes % 16 == 0 && it.m_bytes > 0 && it.m_bytes <= h2::kStageMat &&
                it.m_off + it.m_bytes <= total && nb >= 1 && nb <= h2::kMixedMaxBlocks && it.v_off + nb <= nblk;
      int64_t vc = 0;
      for (int u = 0; ok && u < nb; u++) {
        const h2::MixedBlock& m = blk[it.v_off + u];
        const int64_t lim = (m.src & 1) ? nodes * M.kp4 : xp4[leaves];
        ok = m.vs % 4 == 0 && m.vs >= m.cols && m.vs <= 64 && m.voff % 4 == 0 && m.voff + m.vs <= lim;
        vc += m.vs;
      }
      ok = ok && vc <= h2::kMixedVecCols;
      if (!ok) return h2_fail(H2_ERR_INVALID, "internal: precision-form work item %lld fails the layout audit", (long long)t);
    }
    if (M.panel) {
      // the tensor-core phase's own items: consecutive blocks of one row, at most kTcMaxBlocks
      // blocks, kTcStageMat bytes of codes and kTcStageB bytes of B tiles (tc_layout); weighed
      // by bytes and by MMAs (one per unit and K-step), the phase's two limits
      std::vector<h2::StreamItem> titems;
      std::vector<int64_t> trow_bytes((size_t)leaves), trow_item0((size_t)leaves + 1);
      int kp[h2::kTcMaxBlocks], bo[h2::kTcMaxBlocks], pm = 0, sm = 0;
      for (int64_t i = 0; i < leaves; i++) {
        trow_item0[i] = (int64_t)titems.size();
        const int64_t g0 = row_blk0[i], g1 = row_blk0[i + 1];
        int64_t bytes = 0;
        for (int64_t g = g0; g < g1;) {
          int64_t e = g, mb = 0;
          while (e < g1 && e - g < h2::kTcMaxBlocks && mb + (boff[e + 1] - boff[e]) <= h2::kTcStageMat) {
            kp[e - g] = h2::panel_cols(blk[e].cols);
            if (h2::tc_layout((int)(e - g + 1), kp, bo, &pm, &sm) > h2::kTcStageB) break;
            mb += boff[e + 1] - boff[e];
            e++;
          }
          if (e == g) return h2_fail(H2_ERR_INVALID, "internal: block %lld exceeds a tensor-core stage", (long long)g);
          h2::StreamItem it{};
          it.m_off = boff[g];
          it.m_bytes = (int)mb;
          it.shape = (unsigned)(lo[i + 1] - lo[i]) | ((unsigned)(e - g) << 8);
          it.v_off = g;
          it.row = (int)lo[i];
          h2::tc_layout((int)(e - g), kp, bo, &pm, &sm);
          it.flags = ((e == g1) ? h2::kItemFlagLast : 0) | (pm << h2::kTcPairShift);
          titems.push_back(it);
          int64_t mmas = 0;
          for (int u = 0; u < (int)(e - g); u++)
            if (((pm | sm) >> u) & 1) mmas += kp[u] / 16;
          bytes += mb + 4096 * mmas + 512;
          g = e;
        }
        trow_bytes[i] = bytes;
      }
      trow_item0[leaves] = (int64_t)titems.size();
      const std::vector<int> tbegin = balance(trow_bytes, trow_item0, h->grid);
      for (size_t t = 0; t < titems.size(); t++) {  // audit, as the kernel reads the items
        const h2::StreamItem& it = titems[t];
        const int nb = (int)((it.shape >> 8) & 0xFF);
        bool ok = (it.shape & 0xFF) == 64 && nb >= 1 && nb <= h2::kTcMaxBlocks && it.v_off + nb <= nblk &&
                  it.m_off % 16 == 0 && it.m_bytes % 16 == 0 && it.m_bytes <= h2::kTcStageMat &&
                  it.m_off + it.m_bytes <= total && it.m_bytes == boff[it.v_off + nb] - boff[it.v_off];
        for (int u = 0; ok && u < nb; u++) {
          const h2::MixedBlock& m = blk[it.v_off + u];
          kp[u] = h2::panel_cols(m.cols);
          ok = (m.src & 4) && m.cols >= 1 && m.cols <= 64 &&
               boff[it.v_off + u + 1] - boff[it.v_off + u] == h2::panel_block_bytes(m.cols);
        }
        ok = ok && h2::tc_layout(nb, kp, bo, &pm, &sm) <= h2::kTcStageB && (it.flags >> h2::kTcPairShift) == pm;
        if (!ok) return h2_fail(H2_ERR_INVALID, "internal: tensor-core work item %lld fails the layout audit", (long long)t);
      }
      for (size_t c = 0; c + 1 < tbegin.size(); c++)
        if (tbegin[c] > tbegin[c + 1]) return h2_fail(H2_ERR_INVALID, "internal: item ranges not monotone");
      // the builders' records (kTcRecInts ints per item): block count and pair starts, then per
      // block its vector offset, K | (vector from yhat) << 16 and scale
      std::vector<int32_t> brec(titems.size() * h2::kTcRecInts, 0);
      for (size_t t = 0; t < titems.size(); t++) {
        const h2::StreamItem& it = titems[t];
        const int nb = (int)((it.shape >> 8) & 0xFF);
        int32_t* r = brec.data() + t * h2::kTcRecInts;
        r[0] = nb | ((it.flags >> h2::kTcPairShift) << 8);
        for (int u = 0; u < nb; u++) {
          const h2::MixedBlock& m = blk[it.v_off + u];
          if (m.voff < 0 || m.voff > INT32_MAX)
            return h2_fail(H2_ERR_UNSUPPORTED, "vector offset %lld exceeds the tensor-core records", (long long)m.voff);
          r[1 + 3 * u] = (int32_t)m.voff;
          r[2 + 3 * u] = h2::panel_cols(m.cols) | ((m.src & 1) << 16);
          std::memcpy(&r[3 + 3 * u], &m.scale, sizeof(float));
        }
      }
      if ((st = upload(h, &M.tc_brec, reinterpret_cast<const int4*>(brec.data()), (int64_t)titems.size() * (h2::kTcRecInts / 4))) != H2_OK)
        return st;
      if ((st = upload(h, &M.tc_items.items, titems.data(), (int64_t)titems.size())) != H2_OK) return st;
      if ((st = upload(h, &M.tc_items.cta_begin, tbegin.data(), (int64_t)tbegin.size())) != H2_OK) return st;
      M.tc_items.count = (int64_t)titems.size();
    }
    if ((st = upload(h, &M.dense_items.items, items.data(), (int64_t)items.size())) != H2_OK) return st;
    if ((st = upload(h, &M.dense_items.cta_begin, begin.data(), (int64_t)begin.size())) != H2_OK) return st;
    M.dense_items.count = (int64_t)items.size();
    M.nblk = nblk;
    M.items_host = std::move(items);
    h2::RowJob* drj = nullptr;
    if ((st = upload(h, &drj, rj.data(), leaves)) != H2_OK) return st;
    M.rjobs = drj;
    M.rjobs_host.assign(reinterpret_cast<const unsigned char*>(rj.data()),
                        reinterpret_cast<const unsigned char*>(rj.data() + leaves));
    M.row_bytes = std::move(row_bytes);
    M.row_item0 = std::move(row_item0);
  }
  if ((st = dalloc(h, &M.x4, xp4[leaves] * kPassVectors)) != H2_OK) return st;
  if ((st = dalloc(h, &M.xhat, nodes * kPassVectors * M.kp4)) != H2_OK) return st;
  if ((st = dalloc(h, &M.yhat, nodes * kPassVectors * M.kp4)) != H2_OK) return st;
  // entries k .. kp4 - 1 of every node vector are padding that no kernel writes except with
  // zeros; the dense stream multiplies them by zero codes, so they must be finite
  CUDA_TRY(cudaMemset(M.xhat, 0, (size_t)(nodes * kPassVectors * M.kp4) * sizeof(float)));
  CUDA_TRY(cudaMemset(M.yhat, 0, (size_t)(nodes * kPassVectors * M.kp4) * sizeof(float)));

  if (M.panel || M.spanel) {  // the per-vector scales of the tensor-core phases
    if ((st = dalloc(h, &M.tc_vmax, 16)) != H2_OK) return st;
    if ((st = dalloc(h, &M.tc_vscale, 16)) != H2_OK) return st;
  }

  // tables of the table-driven kernels: this matrix alone
  MixedLaunch& L = M.launch;
  M.srow_host.assign(d->S_rowptr, d->S_rowptr + nodes + 1);
  L.items = M.dense_items.items;
  L.cta_begin = M.dense_items.cta_begin;
  L.blk = M.dblk;
  L.grid = h->grid;
  L.err = h->err;
  L.k = k;
  L.bases_fp32 = M.bases_fp32;
  L.kf = h->kf;
  L.kf_kind = h->kf_kind;
  L.rjobs = M.rjobs;
  L.nrjobs = leaves;
  CUDA_TRY(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  L.side = h->side;
  L.ev_fork = h->ev_fork;
  L.ev_join = h->ev_join;
  // defaults (h2_tune may choose others): 16 dense consumer warps for leaves of at most 32 points
  // (little arithmetic per item, more warps hide more latency), 128 coupling blocks per chunk
  return mixed_configure(h, kDefaultChunkOpt, h->m_max <= 32 ? 2 * h2::kMixedCW : h2::kMixedCW, 0);
}

h2_status mixed_launch(int storage, const MixedLaunch& L, unsigned buckets, cudaStream_t st, const TcPass* tc) {
  switch (form_of(storage)) {
    case h2::kFormFp16: return mixed_pass_form<h2::kFormFp16>(L, buckets, st, tc);
    case h2::kFormBf16: return mixed_pass_form<h2::kFormBf16>(L, buckets, st, tc);
    default: return mixed_pass_form<h2::kFormInt16>(L, buckets, st, nullptr);
  }
}

h2_status mixed_pass(h2_matrix_s* h, int nv, const void* xv, int64_t ldx, void* yv, int64_t ldy, cudaStream_t st,
                     int xy32) {
  // the kernels take the vectors' element type from the descriptor (xy32)
  const double* x = static_cast<const double*>(xv);
  double* y = static_cast<double*>(yv);
  MixedLaunch L = h->mx.launch;
  L.budget = h->budget;
  L.prof = &h->prof;
  cudaError_t me = mark(&h->prof, st);
  if (me != cudaSuccess) return h2_fail(H2_ERR_CUDA, "profiling event: %s", cudaGetErrorString(me));
  h2_status s = set_calls(static_cast<h2::MatDesc*>(L.mats), 1, &nv, &x, &ldx, &y, &ldy, st, xy32);
  if (s != H2_OK) return s;
  const MixedData& M = h->mx;
  const bool fp16 = h->storage == H2_FP16_SCALED;
  const bool tc_ok = nv >= kTcMinVectors && h->storage != H2_INT16_SCALED;
  TcCall T, TS;
  TcPass P;
  // set_calls, upsweep, coupling, downsweep (+ expansion), dense; the split of x when the dense phase
  // runs beside the tree phases (passes of up to four vectors, not profiled)
  int launches = 5;
  if (M.panel && tc_ok) {  // dense phase on the tensor cores
    T.items = M.tc_items.items;
    T.cta_begin = M.tc_items.cta_begin;
    T.brec = M.tc_brec;
    T.blk = M.dblk;
    T.dmat = M.dmat;
    T.x4 = M.x4;
    T.yhat = M.yhat;
    T.xp4_off = M.xp4_off;
    T.vmax = M.tc_vmax;
    T.vscale = M.tc_vscale;
    T.leaves = h->leaves;
    T.leaf0 = h->leaf0;
    T.k = h->k;
    T.kp = M.kp4;
    T.grid = h->grid;
    T.dmax = M.dmax;
    T.umax = M.umax;
    T.y = y;
    T.ldy = ldy;
    T.y32 = xy32;
    T.nv = nv;
    T.err = h->err;
    T.budget = h->budget;
    P.dense = &T;
    launches += fp16 ? 2 : 1;  // (vmax,) vscale before the tensor-core kernel
  }
  if (M.spanel && tc_ok) {  // coupling phase on the tensor cores
    TS.items = M.tc_sitems.items;
    TS.cta_begin = M.tc_sitems.cta_begin;
    TS.brec = M.tc_sbrec;
    TS.dmat = M.smat;
    TS.vmax = M.tc_vmax;
    TS.vscale = M.tc_vscale;
    TS.k = h->k;
    TS.kp = M.kp4;
    TS.grid = h->grid;
    TS.y = reinterpret_cast<double*>(M.yhat);
    TS.ldy = M.kp4;
    TS.y32 = 1;
    TS.nv = nv;
    TS.err = h->err;
    TS.budget = h->budget;
    TS.coupling = 1;
    TS.xhat = M.xhat;
    TS.nodes = h->n_nodes;
    TS.smax = M.smax;
    P.coupling = &TS;
    launches += fp16 ? 2 : 1;
  }
  if (P.dense || P.coupling) {
    h->prof.launches += launches;
    return mixed_launch(h->storage, L, 1u << bucket_of(nv), st, &P);
  }
  h->prof.launches += launches + (bucket_of(nv) <= 2 && !h->prof.on ? 1 : 0);
  return mixed_launch(h->storage, L, 1u << bucket_of(nv), st);
}

}  // namespace h2i

// ------------------------------------------------------------------ batches
namespace {

template <class T>
h2_status balloc(h2_batch_s* b, T** p, int64_t count, const T* src = nullptr) {
  *p = nullptr;
  if (count <= 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return h2_fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, "cudaMalloc of %lld bytes failed: %s",
                   (long long)(count * sizeof(T)), cudaGetErrorString(e));
  }
  b->allocs.push_back(q);
  b->device_bytes += count * (int64_t)sizeof(T);
  *p = (T*)q;
  if (src) CUDA_TRY(cudaMemcpy(q, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice));
  return H2_OK;
}

void batch_free(h2_batch_s* b) {
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  b->side = nullptr;
  b->ev_fork = b->ev_join = nullptr;
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  profile_free(&b->prof);
}

// the batch's coupling chunks, tree jobs and member descriptors for launch options
// (chunk target kChunkOpts[chunk_opt], 2^kTreeOpts[tree_opt] leaves per tree CTA)
h2_status batch_configure(h2_batch_s* b, int chunk_opt, int tree_opt, int cw) {
  const int64_t count = (int64_t)b->hs.size();
  MixedLaunch& L = b->launch;
  h2_status st;
  if (chunk_opt < 0 || chunk_opt > 2 || tree_opt < 0 || tree_opt > 2 ||
      (cw != h2::kMixedCW && cw != 2 * h2::kMixedCW))
    return h2_fail(H2_ERR_INVALID, "internal: launch configuration out of range");
  if (!b->chunk_dev[chunk_opt]) {
    std::vector<int4> chunks;
    for (int64_t i = 0; i < count; i++) {
      const h2_matrix_s* h = b->hs[(size_t)i];
      for (int4 c : coupling_chunks(h->mx.srow_host.data(), h->n_nodes, kChunkOpts[chunk_opt])) {
        c.x = (int)i;
        chunks.push_back(c);
      }
    }
    if ((st = balloc(b, &b->chunk_dev[chunk_opt], (int64_t)chunks.size(), chunks.data())) != H2_OK) return st;
    b->chunk_n[chunk_opt] = (int64_t)chunks.size();
  }
  const int T = kTreeOpts[tree_opt];
  if (!b->jobs_dev[tree_opt]) {
    std::vector<int2> jobs;
    for (int64_t i = 0; i < count; i++) {
      const int Li = std::max(0, b->hs[(size_t)i]->q - T);
      for (int64_t t = 0; t < ((int64_t)1 << Li); t++) jobs.push_back(make_int2((int)i, (int)t));
    }
    if ((int64_t)jobs.size() >= INT32_MAX) return h2_fail(H2_ERR_UNSUPPORTED, "batch too large: %lld tree jobs", (long long)jobs.size());
    if ((st = balloc(b, &b->jobs_dev[tree_opt], (int64_t)jobs.size(), jobs.data())) != H2_OK) return st;
    b->jobs_n[tree_opt] = (int64_t)jobs.size();
  }
  if (!L.mats || tree_opt != b->tree_opt) {  // the descriptors carry each member's subtree level
    std::vector<h2::MatDesc> descs((size_t)count);
    for (int64_t i = 0, r0 = 0; i < count; r0 += b->hs[(size_t)i]->leaves, i++) {
      descs[(size_t)i] = fill_desc(b->hs[(size_t)i], std::max(0, b->hs[(size_t)i]->q - T));
      descs[(size_t)i].rjobs = static_cast<const h2::RowJob*>(L.rjobs) + r0;  // the batch's row jobs and records
      descs[(size_t)i].blk = static_cast<const h2::MixedBlock*>(L.blk);
    }
    if (!L.mats) {
      h2::MatDesc* md = nullptr;
      if ((st = balloc(b, &md, count, descs.data())) != H2_OK) return st;
      L.mats = md;
    } else {
      CUDA_TRY(cudaMemcpy(L.mats, descs.data(), (size_t)count * sizeof(h2::MatDesc), cudaMemcpyHostToDevice));
    }
  }
  L.chunks = b->chunk_dev[chunk_opt];
  L.nchunks = b->chunk_n[chunk_opt];
  L.jobs = b->jobs_dev[tree_opt];
  L.njobs = b->jobs_n[tree_opt];
  L.cw = cw;
  b->chunk_opt = chunk_opt;
  b->tree_opt = tree_opt;
  return H2_OK;
}

h2_status batch_build(h2_batch_s* b) {
  const int64_t count = (int64_t)b->hs.size();
  const h2_matrix_s* h0 = b->hs[0];
  MixedLaunch& L = b->launch;
  h2_status st;
  std::vector<h2::StreamItem> items;
  std::vector<int64_t> row_bytes, row_item0;
  std::vector<h2::RowJob> rjobs;
  int64_t blk0 = 0;
  for (int64_t i = 0; i < count; i++) {
    const h2_matrix_s* h = b->hs[(size_t)i];
    const MixedData& M = h->mx;
    const int64_t item0 = (int64_t)items.size();
    for (h2::StreamItem it : M.items_host) {
      it.v_off += blk0;
      it.flags = (it.flags & 0xFF) | (int)(i << 8);
      items.push_back(it);
    }
    const h2::RowJob* mr = reinterpret_cast<const h2::RowJob*>(M.rjobs_host.data());
    for (size_t r = 0; r < M.rjobs_host.size() / sizeof(h2::RowJob); r++) {
      h2::RowJob J = mr[r];
      J.mat = (int)i;
      if (blk0 + J.ublk >= INT32_MAX) return h2_fail(H2_ERR_UNSUPPORTED, "batch too large: block records");
      J.ublk += (int)blk0;
      rjobs.push_back(J);
    }
    for (size_t r = 0; r + 1 < M.row_item0.size(); r++) {
      row_item0.push_back(item0 + M.row_item0[r]);
      row_bytes.push_back(M.row_bytes[r]);
      b->row_mat.push_back((int32_t)i);
    }
    blk0 += M.nblk;
  }
  row_item0.push_back((int64_t)items.size());
  if ((int64_t)items.size() >= INT32_MAX)
    return h2_fail(H2_ERR_UNSUPPORTED, "batch too large: %lld dense items", (long long)items.size());
  const std::vector<int> begin = balance(row_bytes, row_item0, h0->grid);
  if ((st = audit_producer_batches(items, begin)) != H2_OK) return st;
  for (size_t c = 0; c + 1 < begin.size(); c++)
    if (begin[c] > begin[c + 1]) return h2_fail(H2_ERR_INVALID, "internal: item ranges not monotone");
  for (const h2::StreamItem& it : items)  // the member audits hold; only the block index moved
    if (it.v_off < 0 || it.v_off + ((it.shape >> 8) & 0xFF) > blk0)
      return h2_fail(H2_ERR_INVALID, "internal: batched work item outside the block records");

  h2::StreamItem* di = nullptr;
  if ((st = balloc(b, &di, (int64_t)items.size(), items.data())) != H2_OK) return st;
  int* db = nullptr;
  if ((st = balloc(b, &db, (int64_t)begin.size(), begin.data())) != H2_OK) return st;
  b->cta_begin_dev = db;
  b->row_bytes = row_bytes;
  b->row_item0 = row_item0;
  b->items_host = items;
  h2::MixedBlock* blk = nullptr;
  if ((st = balloc(b, &blk, blk0)) != H2_OK) return st;
  for (int64_t i = 0, o = 0; i < count; o += b->hs[(size_t)i]->mx.nblk, i++)
    CUDA_TRY(cudaMemcpy(blk + o, b->hs[(size_t)i]->mx.dblk, (size_t)b->hs[(size_t)i]->mx.nblk * sizeof(h2::MixedBlock),
                        cudaMemcpyDeviceToDevice));
  int* err = nullptr;
  if ((st = balloc(b, &err, 1)) != H2_OK) return st;
  CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
  h2::RowJob* drj = nullptr;
  if ((st = balloc(b, &drj, (int64_t)rjobs.size(), rjobs.data())) != H2_OK) return st;
  L.rjobs = drj;
  L.nrjobs = (int64_t)rjobs.size();
  CUDA_TRY(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  L.side = b->side;
  L.ev_fork = b->ev_fork;
  L.ev_join = b->ev_join;
  L.items = di;
  L.cta_begin = db;
  L.blk = blk;
  L.grid = h0->grid;
  L.err = err;
  L.k = h0->k;
  L.bases_fp32 = h0->mx.bases_fp32;
  L.prof = nullptr;
  b->n_items = (int64_t)items.size();
  // defaults (h2_batch_tune may choose others): at most 64 leaves per tree CTA, fewer while the
  // batch has under four tree CTAs per SM; 128 coupling blocks per chunk; 16 dense consumer warps
  // when every member's leaves hold at most 32 points
  int tree_opt = kDefaultTreeOpt;
  auto jobs_for = [&](int T) {
    int64_t n = 0;
    for (const h2_matrix_s* h : b->hs) n += (int64_t)1 << std::max(0, h->q - T);
    return n;
  };
  while (tree_opt > 0 && jobs_for(kTreeOpts[tree_opt]) < 4 * (int64_t)h0->grid) tree_opt--;
  bool small = true;
  for (const h2_matrix_s* h : b->hs) small = small && h->m_max <= 32;
  b->tree_opt = -1;
  return batch_configure(b, kDefaultChunkOpt, tree_opt, small ? 2 * h2::kMixedCW : h2::kMixedCW);
}

}  // namespace

extern "C" {

h2_status h2_batch_create(const h2_handle* hs, int32_t count, h2_batch* out) {
  h2_internal_set_error("");
  if (!out) return h2_fail(H2_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!hs) return h2_fail(H2_ERR_INVALID, "handle array is NULL");
  if (count < 1 || count > (1 << 23)) return h2_fail(H2_ERR_INVALID, "count = %d outside 1 .. 2^23", count);
  std::vector<h2_matrix_s*> v((size_t)count);
  for (int32_t i = 0; i < count; i++) {
    if (!hs[i]) return h2_fail(H2_ERR_INVALID, "handle %d is NULL", i);
    v[(size_t)i] = hs[i];
  }
  if (v[0]->storage == H2_FP64)
    return h2_fail(H2_ERR_UNSUPPORTED, "batches take the scaled storage forms only (handle 0 is H2_FP64)");
  for (int32_t i = 0; i < count; i++)
    if (v[(size_t)i]->kf)
      return h2_fail(H2_ERR_UNSUPPORTED, "handle %d evaluates its coupling blocks from the kernel (not batched)", i);
  for (int32_t i = 1; i < count; i++) {
    const h2_matrix_s* h = v[(size_t)i];
    if (h->storage != v[0]->storage || h->mx.bases_fp32 != v[0]->mx.bases_fp32 || h->k != v[0]->k)
      return h2_fail(H2_ERR_INVALID, "handle %d differs from handle 0 in storage, bases_fp32 or rank", i);
  }
  {
    std::vector<h2_matrix_s*> sorted = v;
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return h2_fail(H2_ERR_INVALID, "a handle appears twice in the batch");
  }
  h2_batch_s* b = new (std::nothrow) h2_batch_s();
  if (!b) return h2_fail(H2_ERR_OOM, "host allocation failed");
  b->hs = std::move(v);
  b->storage = b->hs[0]->storage;
  h2_status st;
  try {
    st = batch_build(b);
  } catch (const std::bad_alloc&) {
    st = h2_fail(H2_ERR_OOM, "host allocation failed");
  }
  if (st != H2_OK) {
    batch_free(b);
    delete b;
    return st;
  }
  *out = b;
  return H2_OK;
}

namespace {

// The dense items' split over the CTAs for the vector counts nv (nullptr: bytes alone): row r of
// member i weighs bytes_r (1 + beta nv_i / 16), since a row's arithmetic grows with its vectors
// while its bytes do not; the split is uploaded after `stream` has drained (no product reads it).
h2_status batch_rebalance(h2_batch b, const int32_t* nv, float beta, cudaStream_t stream) {
  std::vector<int64_t> w(b->row_bytes.size());
  for (size_t r = 0; r < w.size(); r++) {
    const int v = nv ? std::max(0, std::min(nv[b->row_mat[r]], kPassVectors)) : 0;
    w[r] = (int64_t)((double)b->row_bytes[r] * (1.0 + beta * v / kPassVectors));
  }
  const std::vector<int> begin = balance(w, b->row_item0, b->launch.grid);
  h2_status st = audit_producer_batches(b->items_host, begin);
  if (st != H2_OK) return st;
  for (size_t c = 0; c + 1 < begin.size(); c++)
    if (begin[c] > begin[c + 1]) return h2_fail(H2_ERR_INVALID, "internal: item ranges not monotone");
  CUDA_TRY(cudaStreamSynchronize(stream));
  CUDA_TRY(cudaMemcpy(b->cta_begin_dev, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice));
  return H2_OK;
}

}  // namespace

h2_status h2_batch_matvec(h2_batch b, const int32_t* nv, const double* const* x, const int64_t* ldx, double* const* y,
                          const int64_t* ldy, void* stream) {
  if (!b) return h2_fail(H2_ERR_INVALID, "NULL batch");
  if (!nv || !x || !ldx || !y || !ldy) return h2_fail(H2_ERR_INVALID, "NULL argument array");
  const int64_t count = (int64_t)b->hs.size();
  int nvmax = 0;
  for (int64_t i = 0; i < count; i++) {
    if (nv[i] < 0) return h2_fail(H2_ERR_INVALID, "nv[%lld] = %d < 0", (long long)i, nv[i]);
    if (nv[i] == 0) continue;
    if (!x[i] || !y[i]) return h2_fail(H2_ERR_INVALID, "x[%lld] or y[%lld] is NULL", (long long)i, (long long)i);
    if (ldx[i] < b->hs[(size_t)i]->n || ldy[i] < b->hs[(size_t)i]->n)
      return h2_fail(H2_ERR_INVALID, "leading dimension of matrix %lld below its n", (long long)i);
    nvmax = std::max(nvmax, nv[i]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  MixedLaunch L = b->launch;
  L.prof = &b->prof;
  std::vector<int> pnv((size_t)count);
  std::vector<const double*> px((size_t)count);
  std::vector<double*> py((size_t)count);
  std::vector<int64_t> pldx(ldx, ldx + count), pldy(ldy, ldy + count);
  for (int v0 = 0; v0 < nvmax; v0 += kPassVectors) {
    unsigned buckets = 0;
    for (int64_t i = 0; i < count; i++) {
      const int c = std::max(0, std::min(kPassVectors, nv[i] - v0));
      pnv[(size_t)i] = c;
      px[(size_t)i] = c ? x[i] + (int64_t)v0 * ldx[i] : nullptr;
      py[(size_t)i] = c ? y[i] + (int64_t)v0 * ldy[i] : nullptr;
      if (c) buckets |= 1u << bucket_of(c);
    }
    cudaError_t me = mark(&b->prof, st);
    if (me != cudaSuccess) return h2_fail(H2_ERR_CUDA, "profiling event: %s", cudaGetErrorString(me));
    h2_status s = set_calls(static_cast<h2::MatDesc*>(L.mats), count, pnv.data(), px.data(), pldx.data(), py.data(),
                            pldy.data(), st);
    if (s != H2_OK) return s;
    b->prof.launches += (count + kCallChunk - 1) / kCallChunk + 3 * bucket_count(buckets) + 1 +
                        (31 - __builtin_clz(buckets | 1u) <= 2 && !b->prof.on ? 1 : 0);
    s = mixed_launch(b->storage, L, buckets, st);
    if (s != H2_OK) return s;
  }
  return H2_OK;
}

h2_status h2_batch_tune(h2_batch b, const int32_t* nv, const double* const* x, const int64_t* ldx, double* const* y,
                        const int64_t* ldy, void* stream, int32_t chosen[3]) {
  if (!b || !chosen) return h2_fail(H2_ERR_INVALID, "NULL batch or output");
  chosen[0] = chosen[1] = chosen[2] = 0;
  const int64_t count = (int64_t)b->hs.size();
  int nvmax = 0;
  for (int64_t i = 0; nv && i < count; i++) nvmax = std::max(nvmax, nv[i]);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const int ncw = 2;  // 8 or 16 dense consumer warps
  float best = 3.4e38f;
  int best_c = b->chunk_opt, best_t = b->tree_opt, best_cw = b->launch.cw;
  h2_status s = H2_OK;
  for (int c = 0; c < ncw && s == H2_OK; c++)
    for (int co = 0; co < 3 && s == H2_OK; co++)
      for (int to = 0; to < 3 && s == H2_OK; to++) {
        const int cw = c ? 2 * h2::kMixedCW : h2::kMixedCW;
        if ((s = batch_configure(b, co, to, cw)) != H2_OK) break;
        if ((s = h2_batch_matvec(b, nv, x, ldx, y, ldy, stream)) != H2_OK) break;  // warm-up (validates)
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2 && s == H2_OK; r++) s = h2_batch_matvec(b, nv, x, ldx, y, ldy, stream);
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
          s = h2_fail(H2_ERR_CUDA, "timing a launch configuration: %s", cudaGetErrorString(ce));
          break;
        }
        if (ms < best) {
          best = ms;
          best_c = co;
          best_t = to;
          best_cw = cw;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != H2_OK) return s;
  if ((s = batch_configure(b, best_c, best_t, best_cw)) != H2_OK) return s;
  // then the dense items' split over the CTAs: rows weighed by bytes, or also by their vector counts
  if (nv) {
    const float betas[4] = {0.f, 1.f, 2.f, 4.f};
    float best_b = 0.f;
    best = 3.4e38f;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    for (int i = 0; i < 4 && s == H2_OK; i++) {
      if ((s = batch_rebalance(b, nv, betas[i], st)) != H2_OK) break;
      if ((s = h2_batch_matvec(b, nv, x, ldx, y, ldy, stream)) != H2_OK) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && s == H2_OK; r++) s = h2_batch_matvec(b, nv, x, ldx, y, ldy, stream);
      cudaEventRecord(e1, st);
      cudaError_t ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) s = h2_fail(H2_ERR_CUDA, "timing a work split: %s", cudaGetErrorString(ce));
      else if (ms < best) {
        best = ms;
        best_b = betas[i];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != H2_OK) return s;
    if ((s = batch_rebalance(b, nv, best_b, st)) != H2_OK) return s;
  }
  chosen[0] = best_cw;
  chosen[1] = kChunkOpts[best_c];
  chosen[2] = 1 << kTreeOpts[best_t];
  return H2_OK;
}

h2_status h2_batch_check(h2_batch b, void* stream) {
  if (!b) return h2_fail(H2_ERR_INVALID, "NULL batch");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, b->launch.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CUDA_TRY(cudaMemset(b->launch.err, 0, sizeof(int)));
    return h2_fail(H2_ERR_TIMEOUT, "a bounded device wait ran out; batched products since the last check are invalid");
  }
  return H2_OK;
}

h2_status h2_batch_info(h2_batch b, int64_t info[6]) {
  if (!b || !info) return h2_fail(H2_ERR_INVALID, "NULL batch or info");
  const int64_t count = (int64_t)b->hs.size();
  info[0] = count;
  int64_t rows = 0;
  for (const h2_matrix_s* h : b->hs) rows += h->n_nodes;
  info[1] = rows;
  info[2] = b->launch.njobs;
  info[3] = b->n_items;
  info[4] = b->device_bytes;
  info[5] = (count + kCallChunk - 1) / kCallChunk + 4;
  return H2_OK;
}

h2_status h2_batch_profile(h2_batch b, int32_t enable) {
  if (!b) return h2_fail(H2_ERR_INVALID, "NULL batch");
  b->prof.on = enable != 0;
  b->prof.used = 0;
  b->prof.launches = 0;
  return H2_OK;
}

h2_status h2_batch_profile_read(h2_batch b, double ms[H2_NPHASES], int64_t* launches) {
  if (!b || !ms) return h2_fail(H2_ERR_INVALID, "NULL batch or output");
  return profile_read(&b->prof, ms, launches);
}

h2_status h2_batch_destroy(h2_batch b) {
  if (!b) return H2_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  delete b;
  return H2_OK;
}

}  // extern "C"
