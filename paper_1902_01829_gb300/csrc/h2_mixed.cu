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

namespace h2i {

template <int F>
h2_status mixed_pass_form(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st);

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

}  // namespace

namespace h2i {

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
  {  // coupling blocks S (always 16-bit codes)
    std::vector<uint16_t> codes((size_t)std::max<int64_t>(1, h->nS * kk8), 0);
    std::vector<float> sc((size_t)std::max<int64_t>(1, h->nS), 0.f);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t b = 0; b < h->nS; b++) sc[b] = quantize(d->S_val + b * kk, kk, form, codes.data() + b * kk8);
    if ((st = upload(h, &M.smat, codes.data(), h->nS * kk8)) != H2_OK) return st;
    if ((st = upload(h, &M.sscale, sc.data(), h->nS)) != H2_OK) return st;
  }

  {  // dense stream: row i holds its dense blocks then U_i, contiguous, each padded to 16 bytes
    const int64_t ubytes = M.bases_fp32 ? 4 : 2;
    std::vector<int64_t> doff((size_t)h->nD + 1, 0);  // FP64 input offsets
    std::vector<int64_t> row_blk0((size_t)leaves + 1, 0), boff((size_t)(h->nD + leaves) + 1, 0);
    for (int64_t i = 0, b = 0; i < leaves; i++) {
      row_blk0[i] = b + i;  // global block index of the row's first block (dense blocks + one U per row)
      const int64_t si = lo[i + 1] - lo[i];
      for (; b < d->D_rowptr[i + 1]; b++) {
        const int64_t sz = si * (lo[d->D_colidx[b] + 1] - lo[d->D_colidx[b]]);
        doff[b + 1] = doff[b] + sz;
        boff[b + i + 1] = boff[b + i] + round_up(sz * 2, 16);
      }
      boff[b + i + 1] = boff[b + i] + round_up(si * k * ubytes, 16);  // U_i
    }
    row_blk0[leaves] = h->nD + leaves;
    const int64_t nblk = h->nD + leaves, total = boff[nblk];  // bytes
    std::vector<unsigned char> bytes_host((size_t)total, 0);
    unsigned char* base = bytes_host.data();
    std::vector<h2::MixedBlock> blk((size_t)nblk);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < leaves; i++) {
      const int64_t si = lo[i + 1] - lo[i];
      int64_t g = row_blk0[i];
      for (int32_t b = d->D_rowptr[i]; b < d->D_rowptr[i + 1]; b++, g++) {
        const int32_t j = d->D_colidx[b];
        h2::MixedBlock& m = blk[g];
        m.scale = quantize(d->D_val + doff[b], doff[b + 1] - doff[b], form, reinterpret_cast<uint16_t*>(base + boff[g]));
        m.voff = xp4[j];
        m.cols = (unsigned short)(lo[j + 1] - lo[j]);
        m.vs = (unsigned char)round_up(lo[j + 1] - lo[j], 4);
        m.src = 0;
      }
      h2::MixedBlock& m = blk[g];  // U_i, multiplied with yhat of leaf i
      if (M.bases_fp32) {
        float* u = reinterpret_cast<float*>(base + boff[g]);
        for (int64_t e = 0; e < si * k; e++) u[e] = (float)d->U[lo[i] * k + e];
        m.scale = 1.0f;
        m.src = 1 | 2;
      } else {
        m.scale = quantize(d->U + lo[i] * k, si * k, form, reinterpret_cast<uint16_t*>(base + boff[g]));
        m.src = 1;
      }
      m.voff = (h->leaf0 + i) * M.kp4;
      m.cols = (unsigned short)k;
      m.vs = (unsigned char)M.kp4;
    }
    unsigned char* dm = nullptr;
    if ((st = upload(h, &dm, base, total)) != H2_OK) return st;
    M.dmat = dm;
    h2::MixedBlock* dblk = nullptr;
    if ((st = upload(h, &dblk, blk.data(), nblk)) != H2_OK) return st;
    M.dblk = dblk;

    // work items: consecutive blocks of one row, at most 4 and 32 KB per item
    std::vector<h2::StreamItem> items;
    std::vector<int64_t> row_bytes((size_t)leaves), row_item0((size_t)leaves + 1);
    for (int64_t i = 0; i < leaves; i++) {
      row_item0[i] = (int64_t)items.size();
      const int64_t g0 = row_blk0[i], g1 = row_blk0[i + 1];
      int64_t bytes = 0;
      for (int64_t g = g0; g < g1;) {
        int64_t e = g, mb = 0;
        while (e < g1 && e - g < h2::kMixedMaxBlocks && mb + (boff[e + 1] - boff[e]) <= h2::kStageMat) {
          mb += boff[e + 1] - boff[e];
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
        for (int64_t u = g; u < e; u++) bytes += mb / (e - g) + 4 * blk[u].vs;
        g = e;
      }
      row_bytes[i] = bytes;
    }
    row_item0[leaves] = (int64_t)items.size();
    const std::vector<int> begin = balance(row_bytes, row_item0, h->grid);
    // audit: every copy in bounds, 16-byte aligned, and within its stage slot
    for (size_t c = 0; c + 1 < begin.size(); c++)
      if (begin[c] > begin[c + 1]) return h2_fail(H2_ERR_INVALID, "internal: item ranges not monotone");
    for (size_t t = 0; t < items.size(); t++) {
      const h2::StreamItem& it = items[t];
      const int nb = (int)((it.shape >> 8) & 0xFF);
      bool ok = it.m_off % 16 == 0 && it.m_bytes % 16 == 0 && it.m_bytes > 0 && it.m_bytes <= h2::kStageMat &&
                it.m_off + it.m_bytes <= total && nb >= 1 && nb <= h2::kMixedMaxBlocks && it.v_off + nb <= nblk;
      for (int u = 0; ok && u < nb; u++) {
        const h2::MixedBlock& m = blk[it.v_off + u];
        const int64_t lim = m.src ? nodes * M.kp4 : xp4[leaves];
        ok = m.vs % 4 == 0 && m.vs >= m.cols && m.vs <= 64 && m.voff % 4 == 0 && m.voff + m.vs <= lim;
      }
      if (!ok) return h2_fail(H2_ERR_INVALID, "internal: precision-form work item %lld fails the layout audit", (long long)t);
    }
    if ((st = upload(h, &M.dense_items.items, items.data(), (int64_t)items.size())) != H2_OK) return st;
    if ((st = upload(h, &M.dense_items.cta_begin, begin.data(), (int64_t)begin.size())) != H2_OK) return st;
    M.dense_items.count = (int64_t)items.size();
  }
  if ((st = dalloc(h, &M.x4, xp4[leaves] * kPassVectors)) != H2_OK) return st;
  if ((st = dalloc(h, &M.xhat, nodes * kPassVectors * M.kp4)) != H2_OK) return st;
  if ((st = dalloc(h, &M.yhat, nodes * kPassVectors * M.kp4)) != H2_OK) return st;
  return H2_OK;
}

h2_status mixed_pass(h2_matrix_s* h, int nv, const double* x, int64_t ldx, double* y, int64_t ldy, cudaStream_t st) {
  switch (form_of(h->storage)) {
    case h2::kFormFp16: return mixed_pass_form<h2::kFormFp16>(h, nv, x, ldx, y, ldy, st);
    case h2::kFormBf16: return mixed_pass_form<h2::kFormBf16>(h, nv, x, ldx, y, ldy, st);
    default: return mixed_pass_form<h2::kFormInt16>(h, nv, x, ldx, y, ldy, st);
  }
}

}  // namespace h2i
