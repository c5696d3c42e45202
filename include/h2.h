/*
 * h2.h -- C ABI of the GB300 H^2 matrix-vector product library (libh2gb300.so).
 *
 * The library computes y = A^H x for an H^2 matrix A^H (Boukaram, Turkiyyah,
 * Keyes, "Hierarchical Matrix Operations on GPUs", Sec. 2.2 and Sec. 4):
 *
 *   A^H = A_D + A_LR, y = A_D x + A_LR x                               (Sec. 4.1)
 *   leaf projection  xhat^q_j = V_j^T x(j)                              (Sec. 4.2, Alg. 2)
 *   upsweep          xhat^{l-1}_p = sum_{c child of p} F_c^T xhat^l_c   (Eq. 2)
 *   coupling         yhat^l_i = sum_{j in b_i} S^l_ij xhat^l_j          (Eq. 3, Alg. 3)
 *   downsweep        yhat^l_c += E_c yhat^{l-1}_p                       (Eq. 5, Alg. 4)
 *   leaf expansion   y(i) = U_i yhat^q_i                                (Eq. 4, Alg. 4)
 *   dense blocks     y(i) += sum_j D_ij x(j)                            (Sec. 2.2)
 *
 * Conventions shared by every entry point
 *   - All integer sizes are int64_t or int32_t as declared; all matrices are
 *     column-major; every block is stored contiguously.
 *   - Vectors are in cluster (tree) order: x(j) is the contiguous range
 *     [leaf_offset[j], leaf_offset[j+1]) of x. Permuting from the caller's
 *     point order is the caller's job.
 *   - The basis trees are one complete binary tree of depth q in heap order:
 *     root 0, children of node h are 2h+1 and 2h+2, level l holds nodes
 *     2^l-1 .. 2^(l+1)-2, the leaves are level q (the paper's flattened tree,
 *     Sec. 3.1, with head/next/parent implied by the numbering).
 *   - Errors: every call returns an h2_status; nothing is thrown across the
 *     ABI. h2_last_error() gives a message for the calling thread's last
 *     failed call.
 */
#ifndef H2GB300_H
#define H2GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  H2_OK = 0,
  H2_ERR_INVALID = 1,      /* bad argument or malformed tree / block structure */
  H2_ERR_OOM = 2,          /* device or host allocation failed */
  H2_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  H2_ERR_UNSUPPORTED = 4,  /* valid input outside what the kernels implement */
  H2_ERR_TIMEOUT = 5       /* a bounded device-side wait ran out */
} h2_status;

/*
 * How h2_create stores the matrix on the device.
 * The scaled forms store every block (each U_i, V_j, E_c, F_c, S_ij, D_ij)
 * as 16-bit values q with one FP32 scale sigma per block, a' = sigma * q;
 * products accumulate in FP32. With m = max |a| over the block:
 *   fp16, bf16: sigma = fl32(m),         q = round-to-nearest-even(a / sigma)
 *   int16:      sigma = fl32(m / 32767), q = clamp(rint(a / sigma), -32767, 32767)
 * (a / sigma evaluated in FP64).
 */
typedef enum {
  H2_FP64 = 0,          /* plain form: FP64 storage; products in double-float
                           (pairs of FP32 with error-free transformations, 46+ bits).
                           Any finite FP64 values: every block and every vector
                           enters the float pairs scaled by a power of two chosen
                           from bounds of the product's intermediates, so no
                           float overflows; entries below 2^-103 times their
                           output's bound (and FP64 subnormals) count as zero */
  H2_FP16_SCALED = 2,   /* IEEE binary16 codes + per-block FP32 scale, FP32 arithmetic */
  H2_BF16_SCALED = 3,   /* bfloat16 codes + per-block FP32 scale, FP32 arithmetic */
  H2_INT16_SCALED = 4   /* int16 codes + per-block FP32 scale, FP32 arithmetic */
} h2_storage;

typedef struct h2_matrix_s* h2_handle;

/*
 * Description of an H^2 matrix (host memory, read-only, owned by the caller;
 * h2_create deep-copies everything, so the caller may free it on return).
 *
 *   n            matrix order (>= 1)
 *   depth        q, leaf level of the cluster tree (0 <= q <= 24)
 *   rank         k, the uniform rank of every basis node (1 <= k <= 64)
 *   symmetric    nonzero: the column tree equals the row tree (V = U, F = E;
 *                V and F are then ignored and may be NULL)
 *   storage      an h2_storage value
 *   leaf_offset  [2^q + 1] int64; leaf_offset[0] = 0, leaf_offset[2^q] = n,
 *                leaf sizes 1 .. 64
 *   U, V         leaf bases: leaf i is a size_i x k block at +leaf_offset[i]*k
 *                (Table 1: U, V)
 *   E, F         transfer matrices: node h >= 1 has a k x k block at
 *                +(h-1)*k*k; E_c relates child c to its parent by Eq. 1
 *   S_rowptr     [2^(q+1)] int32 block-row pointers over ALL nodes (heap order)
 *   S_colidx     [S_rowptr[last]] heap index of each block's column node; it
 *                must lie on the same level as the row node (Sec. 2.2, Fig. 4)
 *   S_val        k x k coupling block b at +b*k*k
 *   D_rowptr     [2^q + 1] int32 block-row pointers over the leaves
 *   D_colidx     [D_rowptr[2^q]] leaf index of each dense block's column
 *   D_val        dense blocks in block order, block (i, j) is size_i x size_j,
 *                each one following the previous one without gaps
 *   check_cover  nonzero: also verify that the coupling and dense blocks
 *                together cover every (row leaf, column leaf) pair exactly
 *                once (O(leaves * (q * row length)) host work)
 *   bases_fp32   scaled forms only: keep U, V, E and F as FP32 entries (S and
 *                D stay 16-bit). The bases and transfers are about 1% of the
 *                entries but their rounding errors compound along the tree's
 *                transfer chains, so this cuts the storage error several-fold.
 */
typedef struct {
  int64_t n;
  int32_t depth;
  int32_t rank;
  int32_t symmetric;
  int32_t storage;
  const int64_t* leaf_offset;
  const double* U;
  const double* V;
  const double* E;
  const double* F;
  const int32_t* S_rowptr;
  const int32_t* S_colidx;
  const double* S_val;
  const int32_t* D_rowptr;
  const int32_t* D_colidx;
  const double* D_val;
  int32_t check_cover;
  int32_t bases_fp32;
} h2_desc;

/*
 * Validate d, copy the matrix to the current CUDA device in the layout the
 * kernels stream, and allocate the per-handle workspace (the xhat / yhat
 * vector trees, Sec. 4.5). Synchronous. On success *out owns all device
 * memory until h2_destroy.
 * Errors: H2_ERR_INVALID (NULL pointers, sizes, non-monotone row pointers,
 * column indices off the row's level or out of range, leaf sizes, non-finite
 * values, |value| >= 2^126 in a scaled storage form, cover violation),
 * H2_ERR_UNSUPPORTED (k > 64, leaf size > 64), H2_ERR_OOM, H2_ERR_CUDA.
 */
h2_status h2_create(const h2_desc* d, h2_handle* out);

/*
 * Coupling blocks evaluated during the product instead of stored. The paper's
 * matrices take every coupling block to be the covariance kernel at the
 * interpolation points of its two clusters (Sec. 4.6):
 *   S_ij[nu][mu] = K(xi_i^nu, xi_j^mu),
 * xi_h^nu the point nu of the tensor grid of node h's first-kind Chebyshev
 * nodes (dimension 0 slowest).
 *   kernel   H2_KERNEL_EXP: K(r) = exp(-r / ell);
 *            H2_KERNEL_MATERN32: K(r) = (1 + s) exp(-s), s = sqrt(3) r / ell
 *   dim, p   1 <= dim <= 3, 1 <= p <= 16, p^dim equal to the descriptor's rank
 *   ell      correlation length, finite and > 0
 *   cheb     host FP64, n_nodes * dim * p finite values: the Chebyshev nodes of
 *            node h (heap order) in dimension d at cheb + (h * dim + d) * p.
 *            Copied; the caller keeps ownership.
 */
typedef enum { H2_KERNEL_EXP = 0, H2_KERNEL_MATERN32 = 1 } h2_kernel_kind;
typedef struct {
  int32_t kernel;
  int32_t dim;
  int32_t p;
  int32_t reserved;  /* 0 */
  double ell;
  const double* cheb;
} h2_coupling_kernel;

/*
 * As h2_create, but the coupling phase evaluates every S_ij from *kc in each
 * product, and no coupling values are stored: d->S_val is ignored (it may be
 * NULL); d->S_rowptr and d->S_colidx give the block structure. Scaled storage
 * forms only (the dense blocks, bases and transfers are stored as h2_create
 * stores them). Kernel values and products are FP32; each point is held as its
 * node's centre (an FP32 pair, high and low part) plus an FP32 offset, and a
 * distance is formed from the centres' difference and the offsets' difference,
 * so it keeps FP32 relative precision at any separation. info[0] of h2_info
 * then counts no coupling bytes. Such a handle cannot join a batch.
 * Errors: those of h2_create; H2_ERR_INVALID (kc or kc->cheb NULL, kernel not an
 * h2_kernel_kind, ell, dim or p out of range, p^dim != rank, non-finite cheb);
 * H2_ERR_UNSUPPORTED (storage H2_FP64).
 */
h2_status h2_create_kernel_coupling(const h2_desc* d, const h2_coupling_kernel* kc, h2_handle* out);

/*
 * As h2_create_kernel_coupling, and the dense blocks are generated on the
 * device instead of copied from the host: D_ij[a][b] = K(x_a, x_b) for the
 * points x of the two leaves (Sec. 2.2, Sec. 4.6), evaluated in FP64 and
 * quantized block by block with the rule of the storage form (h2_storage), so
 * that no host array of dense values is needed. d->D_val is ignored (it may
 * be NULL); d->D_rowptr and d->D_colidx give the block structure; U and E
 * come from d as in h2_create.
 *   kc       the kernel and the Chebyshev nodes, as for h2_create_kernel_coupling
 *   points   host FP64, n * kc->dim finite values: point a of the cluster order
 *            at points + a * dim. Copied; the caller keeps ownership.
 * Kernel values on the device may differ from a host evaluation in the last
 * bit, so a code may differ by one unit where a value lies at a rounding
 * boundary. Errors: those of h2_create_kernel_coupling; H2_ERR_INVALID
 * (points NULL or not finite).
 */
h2_status h2_create_generated(const h2_desc* d, const h2_coupling_kernel* kc, const double* points, h2_handle* out);

/*
 * y = A^H x for nv right-hand sides (Sec. 4, all phases), asynchronously on
 * `stream` (a cudaStream_t; NULL = legacy default stream).
 *   x   device FP64, n x nv, column-major, leading dimension ldx >= n
 *   y   device FP64, n x nv, column-major, leading dimension ldy >= n;
 *       overwritten (never accumulated into); must not overlap x
 * The handle's workspace is reused: calls on one handle must be ordered (same
 * stream or externally synchronized). No host synchronization happens inside.
 * The product runs in passes of up to 16 vectors. In the scaled forms with
 * fp16 or bf16 codes, 16-bit bases, k a multiple of 16 (at most 64) and every
 * leaf of 64 points, a pass of 8 or more vectors runs the dense blocks on the
 * tensor cores (vector operands split into two 16-bit parts, so the result
 * keeps the FP32 accumulation accuracy of the other path). With fp16 or bf16
 * codes and k = 64, such a pass also runs the coupling blocks (Eq. 3) on the
 * tensor cores, whatever the leaves and bases.
 * Errors: H2_ERR_INVALID (NULL, nv < 1, ld < n), H2_ERR_CUDA (launch failed).
 */
h2_status h2_matvec(h2_handle h, int32_t nv, const double* x, int64_t ldx, double* y, int64_t ldy, void* stream);

/*
 * As h2_matvec with FP32 vectors (x read and y written as float), for the
 * scaled storage forms, whose arithmetic is FP32 anyway: half the vector
 * traffic of the FP64 call. H2_ERR_UNSUPPORTED for the FP64 form.
 */
h2_status h2_matvec_f32(h2_handle h, int32_t nv, const float* x, int64_t ldx, float* y, int64_t ldy, void* stream);

/*
 * Same product with HOST buffers: x is copied host->device, the product runs,
 * y is copied device->host, and the call returns after `stream` has drained.
 * Pinned host memory gives full-speed copies; pageable memory works too.
 * Device staging buffers are allocated on the first call and grown when a
 * larger n x nv is requested.
 */
h2_status h2_matvec_host(h2_handle h, int32_t nv, const double* x, int64_t ldx, double* y, int64_t ldy, void* stream);

/*
 * Wait for `stream` to drain and report device-side failures of the products
 * issued since the last check: H2_ERR_TIMEOUT if a bounded wait inside a
 * kernel ran out (the kernel then stopped early and its results are invalid;
 * the CUDA context stays usable). Clears the device error word.
 */
h2_status h2_check(h2_handle h, void* stream);

/*
 * Test hook for the bounded-wait path: in the next product, the streaming
 * dense kernel's first CTA withholds the copy (and its arrival) of its local
 * work item `item`, so the consumers' wait for that item runs out after
 * `wait_budget_cycles` SM clock cycles (0 = the default of about 2 s).
 * h2_check then returns H2_ERR_TIMEOUT. No fault, trap or endless loop is
 * involved; later products run normally.
 */
h2_status h2_debug_withhold_copy(h2_handle h, int32_t item, int64_t wait_budget_cycles);

/*
 * Sizes of the stored representation.
 *   info[0]  paper_bytes: bytes of U, V, E, F, S and D as streamed by one
 *            single-vector product (V and F counted even when aliased to U and
 *            E, since each is read in its own phase; Sec. 4.6 metric); for the
 *            scaled forms 2 bytes per entry plus 4 per block scale
 *   info[1]  total device bytes held by the handle (matrix + workspace)
 *   info[2]  number of coupling blocks     info[3] number of dense blocks
 *   info[4]  q                             info[5] k
 *   info[6]  largest leaf size             info[7] n
 */
h2_status h2_info(h2_handle h, int64_t info[8]);

/*
 * Per-phase timing, for profiling (Sec. 4.6 reports a per-phase breakdown).
 * While enabled, every product records CUDA events on its stream between its
 * phases; h2_profile_read waits for the last recorded event, returns the
 * summed milliseconds of each phase since profiling was enabled (or last
 * read), the number of kernel launches, and starts a new sum.
 * Phases: 0 leaf projection + upsweep, 1 coupling, 2 downsweep,
 * 3 dense blocks + leaf expansion. Disabled by default; enabling costs one
 * event record per phase boundary.
 */
#define H2_NPHASES 4
h2_status h2_profile(h2_handle h, int32_t enable);
h2_status h2_profile_read(h2_handle h, double ms[H2_NPHASES], int64_t* launches);

/*
 * y = A^H x without allocating anything. (The paper has no counterpart: this
 * serves callers that may not allocate device memory, e.g. code inside a
 * host framework that owns all device memory through its own allocator, or
 * code on a latency-critical path where cudaMalloc / cudaFree could
 * synchronize the device.)
 *   d               the matrix in the h2_desc format above, but every array
 *                   pointer is DEVICE memory owned by the caller
 *   n_dense_blocks  D_rowptr[2^q], the number of dense blocks (<= 2^20)
 *   x, y            device FP64, n x nv column-major (ldx, ldy >= n); y is
 *                   overwritten; x and y must not overlap
 * The working memory is one static 16 MiB device array in the library, held
 * by every GPU that loads it until the process exits. The call is rejected
 * with H2_ERR_UNSUPPORTED when k > 64, n_dense_blocks > 2^20, or unless
 *   256 + 2 * (2^(q+1) - 1) * nv * k * 8 + (n_dense_blocks + 1) * 8 <= 16 MiB.
 * The kernel first checks the structure arrays it indexes with (leaf offsets
 * from 0 to n with sizes 1..64, block row pointers from 0 and non-decreasing,
 * coupling columns on the row's level, dense columns among the leaves,
 * D_rowptr[2^q] == n_dense_blocks); if one fails it writes nothing but a
 * sticky error word and leaves y untouched: h2_matvec_static_check reports it.
 * Arithmetic is native FP64 (any finite values). Every call shares that
 * array; each word is written before it is read in the same call, so nothing
 * but the error word carries over, and calls that overlap on the GPU
 * (different streams, different threads) race and corrupt each other.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. One single-CTA kernel does all phases: it is
 * meant for small matrices, not for speed. FP64 storage only. Errors:
 * H2_ERR_INVALID, H2_ERR_UNSUPPORTED, H2_ERR_CUDA; message via h2_last_error.
 */
h2_status h2_matvec_static(const h2_desc* d, int64_t n_dense_blocks, int32_t nv, const double* x, int64_t ldx, double* y,
                           int64_t ldy, void* stream);

/*
 * Report a malformed description seen by h2_matvec_static since the last
 * check (the paper has no counterpart). Synchronizes `stream`, reads the
 * static array's error word and clears it; allocates nothing.
 * Returns H2_OK, H2_ERR_INVALID (some product since the last check found a
 * malformed description and left its y untouched) or H2_ERR_CUDA.
 */
h2_status h2_matvec_static_check(void* stream);

/*
 * Autotuning of the launch parameters of the scaled storage forms. Runs the
 * product y = A^H x with each candidate configuration (one warm-up and three
 * timed products, CUDA events on `stream`) and keeps the fastest for later
 * calls on this handle:
 *   dense consumer warps:   8 or 16 (16 only for passes of at most 8 vectors)
 *   coupling row chunks:    about 64, 128 or 256 coupling blocks per warp
 *   tree jobs:              subtrees at the default level (2^L >= twice the SMs)
 *                           or one or two levels higher (fewer, larger subtrees)
 * x, y, ldx, ldy, nv as for h2_matvec; y holds the product on return. The call
 * synchronizes `stream` (do not capture it in a graph). chosen[0] receives the
 * consumer warps, chosen[1] the chunk size, chosen[2] the leaves per tree CTA.
 * H2_FP64 handles have no options: chosen is all zero and nothing runs.
 * Errors: H2_ERR_INVALID, H2_ERR_CUDA.
 */
h2_status h2_tune(h2_handle h, int32_t nv, const double* x, int64_t ldx, double* y, int64_t ldy, void* stream,
                  int32_t chosen[3]);

/* Free all device memory of the handle (synchronizes the device first). NULL is a no-op. */
h2_status h2_destroy(h2_handle h);

/*
 * Batches: many independent H^2 matrices of uneven size multiplied together,
 * one launch per phase for the whole batch. The paper runs each phase of one
 * matrix as batched small operations over the nodes of a level (Sec. 3.1,
 * Sec. 4.2-4.4); a batch extends the same node-parallel phases across
 * matrices: the tree phases run over (matrix, subtree) jobs, the coupling
 * phase over the concatenated node rows of all matrices, and the dense phase
 * over one work list of every matrix's leaf rows, balanced across the SMs by
 * bytes.
 */
typedef struct h2_batch_s* h2_batch;

/*
 * Group `count` handles (host array, 1 <= count <= 2^23) into a batch.
 * The handles must be distinct, use the same scaled storage (H2_FP16_SCALED,
 * H2_BF16_SCALED or H2_INT16_SCALED, not H2_FP64), the same bases_fp32 choice
 * and the same rank k; their sizes and trees may differ. The batch refers to
 * the handles (it copies none of their blocks) and uses their work space:
 * keep them alive until h2_batch_destroy, and do not run a product of a
 * member handle, alone or in another batch, concurrently with a product of
 * this batch (order them on one stream). Errors: H2_ERR_INVALID (NULL,
 * duplicates, mixed forms or ranks), H2_ERR_UNSUPPORTED (H2_FP64 handles, or
 * handles made by h2_create_kernel_coupling),
 * H2_ERR_OOM, H2_ERR_CUDA.
 */
h2_status h2_batch_create(const h2_handle* hs, int32_t count, h2_batch* out);

/*
 * y_i = A_i x_i for every member i (host arrays of `count` entries each):
 *   nv[i]     vectors of matrix i (>= 0; 0 skips the matrix: its x[i] and
 *             y[i] are not touched and may be NULL)
 *   x[i]      device FP64, n_i x nv[i] column-major, leading dimension
 *             ldx[i] >= n_i
 *   y[i]      device FP64, n_i x nv[i], ldy[i] >= n_i; overwritten; must not
 *             overlap any x or another y
 * Works in passes of up to 16 vectors per matrix (as many as the largest
 * nv[i] needs). A pass launches ceil(count / 256) small kernels that write
 * the pointers into the batch's device table, then for each vector-count
 * bucket present among the members (1, 2, 3-4, 5-8, 9-16 vectors) one launch
 * of each tree and coupling phase (covering every member of the bucket), and
 * one launch of the dense phase for all members. Every launch goes to
 * `stream` (cudaStream_t, NULL = the default stream), so the call can be
 * captured in a CUDA graph (the pointers and counts are baked into the
 * graph). Asynchronous: bounded-wait failures surface through
 * h2_batch_check. Errors: H2_ERR_INVALID, H2_ERR_CUDA.
 */
h2_status h2_batch_matvec(h2_batch b, const int32_t* nv, const double* const* x, const int64_t* ldx,
                          double* const* y, const int64_t* ldy, void* stream);

/*
 * Autotuning of a batch: as h2_tune, over the candidates
 *   dense consumer warps:   8 or 16 (16 only when no member takes more than 8 vectors)
 *   coupling row chunks:    about 64, 128 or 256 coupling blocks per warp
 *   tree jobs:              subtrees of 16, 32 or 64 leaves per CTA
 * (one warm-up and two timed batched products each, arguments as for
 * h2_batch_matvec), then the split of the dense work items over the CTAs:
 * each leaf row weighed by its bytes times (1 + beta nv/16), nv its member's
 * vectors per pass, beta in {0, 1, 2, 4} (the fastest kept). chosen[0]
 * consumer warps, chosen[1] chunk size, chosen[2] leaves per tree CTA.
 * Synchronizes `stream`.
 */
h2_status h2_batch_tune(h2_batch b, const int32_t* nv, const double* const* x, const int64_t* ldx,
                        double* const* y, const int64_t* ldy, void* stream, int32_t chosen[3]);

/* Synchronize `stream`, then report H2_ERR_TIMEOUT (and clear it) if a bounded
 * device wait of a batched product ran out since the last check. */
h2_status h2_batch_check(h2_batch b, void* stream);

/*
 * info[0] members, [1] coupling rows (sum of the members' node counts),
 * [2] tree jobs (subtree CTAs of the tree phases), [3] dense work items,
 * [4] device bytes the batch itself holds, [5] kernel launches of one pass
 * whose members all fall in one vector-count bucket (each further bucket
 * present adds 3).
 */
h2_status h2_batch_info(h2_batch b, int64_t info[6]);

/* Per-phase timing of batched products, as h2_profile / h2_profile_read for a
 * handle: the phases are those of H2_NPHASES; the launch count includes the
 * pointer-table kernels. */
h2_status h2_batch_profile(h2_batch b, int32_t enable);
h2_status h2_batch_profile_read(h2_batch b, double ms[H2_NPHASES], int64_t* launches);

/* Free the batch's own tables (not the member handles). NULL is a no-op. */
h2_status h2_batch_destroy(h2_batch b);

/*
 * Algebraic compression (Sec. 5): a new, orthogonal and (with eps >= 0)
 * smaller representation of the same matrix.
 *
 *   orthogonalization (Sec. 5.2, Alg. 6)  U_i = Q_i T_i at the leaves (QR);
 *       Z_p = [T_c1 E_c1; T_c2 E_c2] = Q_Z T_p at inner nodes; the halves of
 *       Q_Z are the new transfers. Every explicit basis becomes orthonormal.
 *   projection (Alg. 7)                   S_ij <- T^U_i S_ij (T^V_j)^T
 *   basis generation (Sec. 5.3, Alg. 9)   R_i = triangular factor of
 *       [R_parent E_i^T; S_ij1^T; ...; S_ijb^T] (row tree; the column tree
 *       stacks [R_parent F_j^T; S_i1j; ...]), from R_root = 0 down
 *   truncation (Sec. 5.4, Alg. 10)        leading left singular vectors of
 *       W_i = U_i R_i^T (leaves) and W_p = Z_p R_p^T (inner nodes, Z_p from
 *       the children's new T), as many per node as the level's rank: the
 *       largest, over the level's nodes, count of singular values >= eps
 *       times that node's largest; T = Q^T U (leaves) or Q^T Z (inner nodes)
 *   projection again with the truncation's T
 * QR factors are taken with a non-negative diagonal in R. Where a node's
 * matrix has fewer singular vectors than the level rank, the missing ones
 * are zero. FP64 throughout (Householder QR, one-sided Jacobi SVD).
 *
 * The result has one uniform rank k_out, the largest level rank of either
 * tree (at least 1); levels of smaller rank are zero-padded, which leaves
 * the matrix unchanged. It is in the h2_desc layout at rank k_out, with the
 * input's structure and dense blocks, so it can be passed to h2_create.
 */
typedef struct h2_compressor_s* h2_compressor;

/*
 * Copy the matrix's bases, transfers and coupling blocks (FP64 storage form;
 * dense values are not needed and may be NULL) to the current device and
 * allocate the working arrays (about 4 x the coupling bytes in all).
 * Synchronous. Errors: as h2_create, H2_ERR_UNSUPPORTED for a scaled storage
 * form or 2^31 or more coupling blocks.
 */
h2_status h2_compress_create(const h2_desc* d, h2_compressor* out);

/*
 * Run on `stream` (asynchronous; nothing is allocated). eps < 0: only the
 * orthogonalization and projection (the result has rank k); 0 <= eps < 1:
 * the whole compression with relative threshold eps. Every run starts from
 * the matrix given to h2_compress_create and overwrites the previous
 * result. H2_ERR_INVALID for eps >= 1 or NaN, or another current device.
 */
h2_status h2_compress_run(h2_compressor c, double eps, void* stream);

/*
 * Wait for `stream`, then report the uniform rank of the result (k_out) and
 * the rank of every level l = 0..q of the row and column trees (ranks_u,
 * ranks_v: q + 1 entries each, may be NULL). After an eps < 0 run all are k.
 */
h2_status h2_compress_result(h2_compressor c, int32_t* k_out, int32_t* ranks_u, int32_t* ranks_v, void* stream);

/*
 * Copy one result array to host memory `dst` (count must be its exact size;
 * waits for `stream`). With K = k_out and k the input rank:
 *   H2C_U, H2C_V   leaf bases, n * K (layout of h2_desc.U at rank K)
 *   H2C_E, H2C_F   transfers, (2^(q+1) - 2) * K * K
 *   H2C_S          coupling blocks, nS * K * K
 *   H2C_T_ORTHO_U, H2C_T_ORTHO_V   the orthogonalization's T of every node,
 *                  (2^(q+1) - 1) * k * k, upper triangular (old = new * T)
 *   H2C_R_U, H2C_R_V               the basis generation's R of every node,
 *                  (2^(q+1) - 1) * k * k (after an eps >= 0 run)
 *   H2C_SIGMA_U, H2C_SIGMA_V       singular values of every node's W in
 *                  descending order, (2^(q+1) - 1) * k (after an eps >= 0 run)
 * V, F, T_ORTHO_V, R_V and SIGMA_V equal their U counterparts for a
 * symmetric matrix. H2_ERR_INVALID for an unknown array, a wrong count, or
 * before the first run.
 */
enum {
  H2C_U = 0, H2C_V = 1, H2C_E = 2, H2C_F = 3, H2C_S = 4, H2C_T_ORTHO_U = 5, H2C_T_ORTHO_V = 6,
  H2C_R_U = 7, H2C_R_V = 8, H2C_SIGMA_U = 9, H2C_SIGMA_V = 10
};
h2_status h2_compress_read(h2_compressor c, int32_t what, double* dst, int64_t count, void* stream);

/* Per-phase timing of h2_compress_run (CUDA events on its stream, recorded
 * while enabled): 0 orthogonalization, 1 projection, 2 basis generation,
 * 3 truncation, 4 second projection and repacking. h2_compress_profile_read
 * waits for the last run and gives its phase times and kernel launches. */
#define H2C_NPHASES 5
h2_status h2_compress_profile(h2_compressor c, int32_t enable);
h2_status h2_compress_profile_read(h2_compressor c, double ms[H2C_NPHASES], int64_t* launches);

/* info[0] most one-sided Jacobi sweeps a node took in the last run, [1] their
 * total over all nodes, [2] device bytes the compressor holds, [3] coupling
 * blocks, [4] q, [5] input rank k. Waits for the device. */
h2_status h2_compress_info(h2_compressor c, int64_t info[6]);

/* Free the compressor's device arrays. NULL is a no-op. */
h2_status h2_compress_destroy(h2_compressor c);

/*
 * Construction of a covariance H^2 matrix on the current device (Sec. 4.6):
 *   cluster tree  KD bisection: q is the smallest level with m 2^q >= n; level
 *                 by level a node's points are ordered by (coordinate along
 *                 the longest side of its tight box, the lowest dimension on a
 *                 tie; original index) and the first ceil(s/2) form the left
 *                 child. A leaf keeps the order of its parent's split.
 *   boxes, nodes  tight axis-aligned boxes; p first-kind Chebyshev nodes per
 *                 box side, (a+b)/2 + (b-a)/2 cos((2v+1) pi / (2p)), a side
 *                 shorter than 1e-10 widened to 1e-10 about its centre
 *   blocks        dual traversal from (root, root): a pair is a coupling
 *                 block when eta > 0, the boxes' Euclidean gap dist > 0 and
 *                 max(diam_i, diam_j) <= eta dist (diam = box diagonal);
 *                 else a dense block at the leaf level, else its four child
 *                 pairs. Block-sparse rows with ascending columns.
 *   values        (optional, FP64) U_i[a][nu] = L^i_nu(x_a) (tensor Lagrange
 *                 polynomials, dimension 0 slowest), E_c[mu][nu] =
 *                 L^parent_nu(xi^c_mu), S_ij[nu][mu] = K(xi_i^nu, xi_j^mu),
 *                 D_ij[a][b] = K(x_a, x_b), laid out as in h2_desc.
 * The structure is exact: boxes, diameters, distances and Chebyshev nodes use
 * the same rounded operations in the same order as the definitions above.
 * Kernel values (exp) may differ from a host evaluation in the last bit.
 */
typedef struct h2_built_s* h2_built;
enum { H2B_VALUES_U = 1, H2B_VALUES_E = 2, H2B_VALUES_S = 4, H2B_VALUES_D = 8 };
typedef struct {
  int64_t n;        /* points, 1 .. 2^31 - 1 */
  int32_t dim;      /* 1 .. 3 */
  int32_t m;        /* leaf size bound, 2 .. 64 */
  int32_t p;        /* Chebyshev nodes per dimension; rank k = p^dim <= 64 */
  int32_t kernel;   /* h2_kernel_kind */
  double eta;       /* admissibility parameter, >= 0 (0: dense blocks only) */
  double ell;       /* correlation length, > 0 */
  int32_t values;   /* mask of H2B_VALUES_*: which value arrays to build */
  int32_t reserved; /* 0 */
} h2_build_desc;

/*
 * Build from `points` (host FP64, n * dim, original order, point i at
 * points + i * dim). Synchronous; the device arrays live until
 * h2_built_destroy. Errors: H2_ERR_INVALID (NULL arguments, sizes or
 * parameters out of range, non-finite points), H2_ERR_UNSUPPORTED (p^dim > 64,
 * 2^31 or more blocks), H2_ERR_OOM, H2_ERR_CUDA.
 */
h2_status h2_build(const h2_build_desc* b, const double* points, h2_built* out);

/* info[0] q, [1] k, [2] coupling blocks, [3] dense blocks, [4] dense values,
 * [5] nodes, [6] leaves, [7] device bytes held */
h2_status h2_built_info(h2_built b, int64_t info[8]);

/* milliseconds of the build's device phases: [0] cluster tree, boxes and
 * Chebyshev nodes, [1] dual traversal and block-sparse rows, [2] values */
h2_status h2_built_times(h2_built b, double ms[3]);

/*
 * Copy one array to host memory (count must be its exact size):
 *   H2B_PERM        int64 [n]: original index of each cluster position
 *   H2B_LEAF_OFFSET int64 [2^q + 1]
 *   H2B_POINTS      double [n * dim]: the points in cluster order
 *   H2B_CHEB        double [nodes * dim * p]: node h, dimension d at (h dim + d) p
 *   H2B_S_ROWPTR, H2B_S_COLIDX, H2B_D_ROWPTR, H2B_D_COLIDX   int32, as h2_desc
 *   H2B_D_VALOFF    int64 [dense blocks + 1]: offset of each dense block's values
 *   H2B_U, H2B_E, H2B_S, H2B_D   double, as h2_desc (only those built)
 */
enum {
  H2B_PERM = 0, H2B_LEAF_OFFSET = 1, H2B_POINTS = 2, H2B_CHEB = 3, H2B_S_ROWPTR = 4, H2B_S_COLIDX = 5,
  H2B_D_ROWPTR = 6, H2B_D_COLIDX = 7, H2B_D_VALOFF = 8, H2B_U = 9, H2B_E = 10, H2B_S = 11, H2B_D = 12
};
h2_status h2_built_read(h2_built b, int32_t what, void* dst, int64_t count);

/*
 * A product handle (as h2_create) from a built matrix: storage and bases_fp32
 * as in h2_desc; flags: H2B_CREATE_KERNEL_COUPLING evaluates the coupling
 * blocks from the kernel in every product (h2_create_kernel_coupling),
 * adding H2B_CREATE_GENERATED_DENSE generates the dense blocks on the device
 * (h2_create_generated). Needs the U and E values, and S and D where they are
 * stored. The structure and the needed values pass through host memory once.
 * Errors: those of the create call; H2_ERR_INVALID for missing values or
 * flags outside the two above (generated dense blocks without kernel
 * coupling included).
 */
enum { H2B_CREATE_KERNEL_COUPLING = 1, H2B_CREATE_GENERATED_DENSE = 2 };
h2_status h2_create_built(h2_built b, int32_t storage, int32_t bases_fp32, int32_t flags, h2_handle* out);

/* Free the built matrix's device arrays. NULL is a no-op. */
h2_status h2_built_destroy(h2_built b);

/* Message of the calling thread's last failed call ("" if none). Valid until the next call. */
const char* h2_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* H2GB300_H */
