// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cstdint>
#include <vector>

#include "h2.h"
#include "stream_fp64.cuh"

// error message of the calling thread's last failed call (h2_last_error)
h2_status h2_fail(h2_status st, const char* fmt, ...);
void h2_internal_set_error(const char* msg);

#define CUDA_TRY(call)                                                                                        \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess) {                                                                                  \
      if (e_ == cudaErrorMemoryAllocation) return h2_fail(H2_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_)); \
      return h2_fail(H2_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                                   \
    }                                                                                                         \
  } while (0)

struct h2_matrix_s;

namespace h2i {

constexpr int kMaxLeaf = 64;
constexpr int kMaxRank = 64;
constexpr int kPassVectors = 16;                 // right-hand sides per pass over the matrix
constexpr long long kWaitBudget = 4000000000LL;  // clock64 cycles (about 2 s) a device wait may take

inline int64_t even(int64_t v) { return v + (v & 1); }
inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

struct ItemList {
  h2::StreamItem* items = nullptr;  // device
  int* cta_begin = nullptr;         // device [grid + 1]
  int64_t count = 0;
};

// per-phase profiling: CUDA events recorded at phase boundaries while enabled
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> events;  // pooled
  size_t used = 0;
  int64_t launches = 0;
};

// what one precision-form product launches over: a table of matrices (one
// matrix, or a batch), the tree jobs, the coupling row map and the dense items
struct MixedLaunch {
  void* mats = nullptr;              // device h2::MatDesc table
  const int2* jobs = nullptr;        // (matrix, subtree) per tree CTA
  int64_t njobs = 0;
  const int4* chunks = nullptr;      // coupling row chunks {matrix, first row, rows, 0}
  int64_t nchunks = 0;
  const h2::StreamItem* items = nullptr;
  const int* cta_begin = nullptr;    // [grid + 1]
  const void* blk = nullptr;         // h2::MixedBlock records
  int grid = 0;
  int* err = nullptr;
  long long budget = kWaitBudget;
  int k = 0;
  bool bases_fp32 = false;
  int cw = 8;                        // consumer warps of the dense stream (8, or 16 for passes of <= 8 vectors)
  bool kf = false;                   // coupling blocks evaluated from the kernel (no stored S)
  int kf_kind = 0;                   // its kernel: H2_KERNEL_EXP or H2_KERNEL_MATERN32
  Profiler* prof = nullptr;          // profiler whose events mark the phases (or none)
  const void* rjobs = nullptr;       // h2::RowJob per leaf row of every matrix (split x, leaf expansion)
  int64_t nrjobs = 0;
  // the tree phases run on `side` beside the dense phase (CUDA-core passes, not profiling)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// a tensor-core phase of one pass (one matrix, panel layout, fp16 / bf16 codes): the dense phase with
// the leaf expansion, or (coupling) the coupling blocks of every level, yhat_i = sum_j S_ij xhat_j
struct TcCall {
  const h2::StreamItem* items = nullptr;
  const int* cta_begin = nullptr;
  const int4* brec = nullptr;   // builder records of the items
  const void* blk = nullptr;
  const void* dmat = nullptr;
  const float* x4 = nullptr;
  const float* yhat = nullptr;
  const int64_t* xp4_off = nullptr;
  unsigned* vmax = nullptr;   // [16]
  float* vscale = nullptr;    // [16]
  int64_t leaves = 0, leaf0 = 0;
  int k = 0, kp = 0, grid = 0;
  float dmax = 0.f, umax = 0.f;  // largest block scale of the dense blocks and of the leaf bases
  double* y = nullptr;   // FP32 when y32
  int64_t ldy = 0;
  int y32 = 0;
  int nv = 0;
  int* err = nullptr;
  long long budget = kWaitBudget;
  // coupling: y is the FP32 yhat ([node][v][kp], zeroed first), the vectors come from xhat, the
  // per-vector scales cover smax |xhat| over `nodes` nodes, and the blocks have unpadded panels
  int coupling = 0;
  const float* xhat = nullptr;
  int64_t nodes = 0;
  float smax = 0.f;
};

// the tensor-core phases of one pass (either may be absent)
struct TcPass {
  const TcCall* dense = nullptr;
  const TcCall* coupling = nullptr;
};

// device copy of the precision form (per-block scaled 16-bit storage, FP32 arithmetic)
struct MixedData {
  void* dmat = nullptr;       // per leaf row: its dense blocks then U_i, each padded to 16 bytes
  void* dblk = nullptr;       // per dense-stream block: h2::MixedBlock
  ItemList dense_items;
  uint16_t* smat = nullptr;   // coupling blocks, k*k padded to a multiple of 8 codes each
  float* sscale = nullptr;
  bool bases_fp32 = false;   // U, V, E, F kept as FP32 entries (scale 1) instead of codes
  void* Vt = nullptr;         // leaf j: V_j^T (k x size_j), at vt_off[j] entries
  float* vscale = nullptr;
  int64_t* vt_off = nullptr;
  void* Ft = nullptr;         // node h >= 1: F_h^T at (h-1) * kk8 entries
  float* fscale = nullptr;
  void* E = nullptr;          // node h >= 1: E_h at (h-1) * kk8 entries
  float* escale = nullptr;
  int64_t* xp4_off = nullptr; // leaf offsets of the FP32 x copy, padded to multiples of 4
  float* x4 = nullptr;        // FP32 copy of the pass's x (padded leaf layout)
  float* xhat = nullptr;      // [node][v][kp4]
  float* yhat = nullptr;
  int kp4 = 0;                // k rounded up to a multiple of 4
  int64_t kk8 = 0;            // k*k rounded up to a multiple of 8
  int64_t nblk = 0;           // dense-stream blocks (dense blocks + one U per leaf row)
  bool panel = false;         // blocks in the panel layout (every leaf 64 points, fp16/bf16 codes)
  float dmax = 0.f, umax = 0.f;  // largest scale of the dense blocks and of the U blocks
  unsigned* tc_vmax = nullptr;   // tensor-core passes: per-vector maxima and scales
  float* tc_vscale = nullptr;
  ItemList tc_items;             // tensor-core passes: their own work items (panel layout only)
  float4* kf_chi = nullptr;      // coupling from the kernel: node centres (FP32 high parts, x y z 0)
  float4* kf_clo = nullptr;      // and their low parts
  float4* kf_off = nullptr;      // [node][k] offsets of the interpolation points from the centre
  int4* tc_brec = nullptr;       // and the builders' records of those items
  bool spanel = false;           // coupling codes in the panel layout, unpadded (fp16 / bf16, k = 64)
  float smax = 0.f;              // largest coupling block scale
  ItemList tc_sitems;            // the coupling phase's tensor-core items (spanel) and their records
  int4* tc_sbrec = nullptr;
  void* rjobs = nullptr;         // h2::RowJob per leaf row (matrix index 0)
  std::vector<unsigned char> rjobs_host;  // the same, kept for batches
  // the table-driven kernels' tables for this matrix alone (a batch of one)
  MixedLaunch launch;
  std::vector<h2::StreamItem> items_host;  // the dense items (matrix index 0), kept for batches
  std::vector<int64_t> row_bytes;          // bytes each leaf row streams (load balance)
  std::vector<int64_t> row_item0;          // first item of each leaf row, [leaves + 1]
  std::vector<int4> chunks_host;           // coupling row chunks (matrix index 0), current target
  std::vector<int32_t> srow_host;          // S_rowptr (to cut chunks for another target)
  int4* chunk_dev[3] = {nullptr, nullptr, nullptr};  // device chunk lists per target option
  int64_t chunk_n[3] = {0, 0, 0};
  int2* jobs_dev[3] = {nullptr, nullptr, nullptr};    // tree jobs per subtree-level option
  int tree_opt = -1;                                  // subtree level L = default - tree_opt
};

// launch parameters the tuner chooses between (h2_tune, h2_batch_tune)
constexpr int kChunkOpts[3] = {64, 128, 256};  // coupling blocks per warp chunk (target)
constexpr int kTreeOpts[3] = {4, 5, 6};       // log2 of the leaves per tree CTA (batches)
constexpr int kDefaultChunkOpt = 1, kDefaultTreeOpt = 2;
constexpr int kDenseCW = 8;                   // dense-stream consumer warps (or twice as many)
std::vector<int4> coupling_chunks(const int32_t* Srow, int64_t n_nodes, int64_t target);

// vector-count buckets of the precision-form kernels: bucket b runs the
// variant for up to kBucketNV[b] vectors and takes counts kBucketLo[b] ..
constexpr int kBuckets = 5;
constexpr int kBucketNV[kBuckets] = {1, 2, 4, 8, 16};
constexpr int kBucketLo[kBuckets] = {1, 2, 3, 5, 9};
inline int bucket_of(int nv) { return nv <= 1 ? 0 : nv <= 2 ? 1 : nv <= 4 ? 2 : nv <= 8 ? 3 : 4; }
inline int bucket_count(unsigned mask) { return __builtin_popcount(mask); }


}  // namespace h2i

struct h2_matrix_s {
  int64_t n = 0, leaves = 0, n_nodes = 0, leaf0 = 0, nS = 0, nD = 0, nDval = 0;
  int q = 0, k = 0, kp = 0, m_max = 0, lr = 32, grid = 0;
  int storage = H2_FP64;
  const h2_coupling_kernel* kc = nullptr;  // while h2_create_kernel_coupling builds the handle
  const double* gen_points = nullptr;      // while h2_create_generated builds the handle (host, n x dim)
  bool kf = false;                         // coupling blocks evaluated from the kernel
  int kf_kind = 0;
  float kf_inv_ell = 0.f;
  int64_t paper_bytes = 0, device_bytes = 0;
  std::vector<void*> allocs;
  int64_t* leaf_off = nullptr;
  int64_t* xp_off = nullptr;  // padded leaf offsets of the split x (float2 per vector)
  double* Vt = nullptr;       // leaf j: k x size_j col-major (= V_j^T, projection)
  double* E = nullptr;        // node h >= 1: k x k col-major (downsweep)
  double* Ft = nullptr;       // node h >= 1: F_h^T, k x k col-major (upsweep)
  char* dmat = nullptr;       // dense blocks then leaf bases U, each padded to an even count of doubles
  double* smat = nullptr;     // coupling blocks, each padded to an even count of doubles
  int32_t* Srow = nullptr;
  int32_t* Scol = nullptr;
  // FP64 form: exponent offsets (a' = a * 2^-o) of the blocks of V (per leaf), F, E (per node), and
  // per coupling block its column node with its offset
  int32_t* oV = nullptr;
  int32_t* oF = nullptr;
  int32_t* oE = nullptr;
  int2* Sco = nullptr;
  int* vexp = nullptr;                // per vector of the current pass: x scaled by 2^-vexp[v]
  unsigned long long* vpart = nullptr;  // per-block maxima of the scale pass
  unsigned* vticket = nullptr;        // last-block ticket of the scale pass, zero between products
  h2i::ItemList dense_items;
  h2i::MixedData mx;          // precision form (storage != H2_FP64)
  bool pair_rows = false;     // k = 2^j (j >= 1): the coupling kernel reads row pairs
  bool s_tiny = true;         // some coupling entry is zero or below 2^-103 after its block's offset
  int* err = nullptr;         // device error word (bounded waits)
  int* ticket = nullptr;      // upsweep climb counters, one per node
  int tree_L = 0;             // subtree root level of the fused tree kernels
  float2* x2 = nullptr;       // split x, padded leaf layout, kPassVectors slots
  float2* xhat = nullptr;     // n_nodes x kPassVectors x kp
  float2* yhat = nullptr;
  long long budget = h2i::kWaitBudget;
  int inject = -1;
  h2i::Profiler prof;
  // precision form: the tree phases run on `side` beside the dense phase
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // host-buffer staging (h2_matvec_host)
  double* hx = nullptr;
  double* hy = nullptr;
  int64_t host_cap = 0;
};

namespace h2i {

template <class T>
h2_status dalloc(h2_matrix_s* h, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return h2_fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, "cudaMalloc of %lld bytes failed: %s",
                   (long long)(count * sizeof(T)), cudaGetErrorString(e));
  }
  h->allocs.push_back(q);
  h->device_bytes += count * (int64_t)sizeof(T);
  *p = (T*)q;
  return H2_OK;
}

template <class T>
h2_status upload(h2_matrix_s* h, T** p, const T* src, int64_t count) {
  h2_status st = dalloc(h, p, count);
  if (st != H2_OK) return st;
  if (count > 0) CUDA_TRY(cudaMemcpy(*p, src, (size_t)count * sizeof(T), cudaMemcpyHostToDevice));
  return H2_OK;
}

// rows weighed by bytes -> first item of each of `grid` contiguous, about equal ranges
std::vector<int> balance(const std::vector<int64_t>& row_bytes, const std::vector<int64_t>& row_item0, int grid);
// record a phase-boundary event when profiling
cudaError_t mark(Profiler* p, cudaStream_t st);
// summed milliseconds per phase since the last read (groups of H2_NPHASES + 1 events), then reset
h2_status profile_read(Profiler* p, double ms[H2_NPHASES], int64_t* launches);
void profile_free(Profiler* p);
// precision form: device layout (h2_create) and one product pass of up to kPassVectors vectors
h2_status mixed_build(h2_matrix_s* h, const h2_desc* d);
// structural and value checks of a description (h2_create's); s_values / d_values: the
// coupling / dense values are part of it
h2_status validate_desc(const h2_desc* d, bool s_values, bool d_values, int64_t* nS, int64_t* nD, int64_t* nDval,
                        int* m_max);
// one product pass; buckets: bit b set when some matrix has a vector count in bucket b
h2_status mixed_launch(int storage, const MixedLaunch& L, unsigned buckets, cudaStream_t st, const TcPass* tc = nullptr);
// precision form: use coupling chunk target option `chunk_opt`, `cw` dense consumer warps and
// tree subtrees at level (default level - tree_opt)
h2_status mixed_configure(h2_matrix_s* h, int chunk_opt, int cw, int tree_opt);
// passes of at least this many vectors use the tensor-core dense phase (panel-layout handles)
constexpr int kTcMinVectors = 8;
// one pass of up to 16 vectors; xy32: x and y are FP32 (else FP64)
h2_status mixed_pass(h2_matrix_s* h, int nv, const void* x, int64_t ldx, void* y, int64_t ldy, cudaStream_t st,
                     int xy32 = 0);

}  // namespace h2i

// A batch of precision-form matrices multiplied by one launch per phase.
struct h2_batch_s {
  std::vector<h2_matrix_s*> hs;  // the member handles (not owned)
  int storage = 0;
  h2i::MixedLaunch launch;       // over the concatenated tables
  int chunk_opt = h2i::kDefaultChunkOpt, tree_opt = h2i::kDefaultTreeOpt;
  int4* chunk_dev[3] = {nullptr, nullptr, nullptr};
  int64_t chunk_n[3] = {0, 0, 0};
  int2* jobs_dev[3] = {nullptr, nullptr, nullptr};
  int64_t jobs_n[3] = {0, 0, 0};
  h2i::Profiler prof;
  int64_t n_items = 0, device_bytes = 0;
  std::vector<void*> allocs;
  cudaStream_t side = nullptr;  // the tree phases beside the dense phase
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the dense items' split over the CTAs (h2_batch_tune weighs each row by its member's vector count)
  std::vector<h2::StreamItem> items_host;
  std::vector<int64_t> row_bytes, row_item0;
  std::vector<int32_t> row_mat;
  int* cta_begin_dev = nullptr;
};
