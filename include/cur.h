/*
 * cur.h - C ABI of libcur, a GB300 (sm_103a) implementation of the scalable
 * binary CUR cross: A ~ C U R with C = A(:,J), U = A(I,J)^dagger, R = A(I,:)
 * (arXiv 2502.11017, Section 1.1), where I and J are chosen by the blockwise
 * adaptive cross approximation (Algorithm 3), refined by block-wise maximal-volume
 * swaps (Section 1.2, Definition 1) and combined by a binary pairwise merge.
 *
 * Conventions shared by every call
 *  - Matrices are dense, row-major, in device memory of the handle's device:
 *    element (i, j) of a cur_mat lives at data + i*ld + j (elements, ld >= cols).
 *    Element offsets are 64-bit. Supported element types: CUR_F64, CUR_F32,
 *    CUR_BF16 (BF16 is read and widened to FP32).
 *  - Index vectors are int32, 0-based, device memory. Index sets are returned in
 *    submatrix-position order (position k of I is row k of A(I,J)).
 *  - Ownership: the caller allocates every input and output buffer. The library
 *    owns only the handle and the workspace allocated once by cur_create; no call
 *    allocates device memory.
 *  - Streams: every call enqueues its work on `stream` and returns without waiting
 *    for the GPU. Where the next step depends on a result (a singular start set, an
 *    inverse valid to inherit, a sweep that made no swap), a kernel takes the decision
 *    on the device; later steps run as no-ops when they are not needed. Outputs are
 *    complete once the stream reaches that point (cur_sync_status synchronises and
 *    returns the status). Calls that do wait for the GPU: cur_sync_status,
 *    cur_prof_read, cur_prof_refactors, and the first cur_cross_batched of each class of
 *    batch (its launch-shape tuning).
 *  - Errors: argument errors (CUR_ERR_ARG), workspace exhaustion (CUR_ERR_NOMEM)
 *    and CUDA launch errors (CUR_ERR_CUDA) are returned at once. Errors found on
 *    the device (CUR_ERR_SINGULAR, CUR_ERR_NONFINITE, CUR_ERR_NOCONV,
 *    CUR_ERR_TIMEOUT) and the early stop of the selection (CUR_WARN_RANK) are
 *    recorded in the handle's device status word; cur_sync_status returns the
 *    first one recorded since the previous cur_sync_status.
 *  - A handle serves one stream at a time; calls on one handle do not overlap.
 *  - Autotuning: cur_cross_batched (its Algorithm 3 launch: one or two CTAs per SM) times its
 *    candidate launch shapes on the first call of each shape class and keeps the fastest in
 *    the handle. Only shapes that leave every result unchanged are tuned.
 */
#ifndef CUR_H
#define CUR_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CUR_OK = 0,
    CUR_ERR_ARG = 1,        /* invalid argument: shape, rank, block size, pointer */
    CUR_ERR_SINGULAR = 2,   /* numerically singular A(I,J) where an inverse is needed */
    CUR_ERR_NONFINITE = 3,  /* NaN or Inf met in the data */
    CUR_ERR_NOCONV = 4,     /* maxvol did not converge within opts.max_swaps */
    CUR_ERR_TIMEOUT = 5,    /* a device-side wait ran out of time (no hang) */
    CUR_ERR_NOMEM = 6,      /* the handle's workspace is too small for this call */
    CUR_ERR_CUDA = 7,       /* a CUDA runtime call failed */
    CUR_WARN_RANK = 8       /* the residual reached rounding level before r picks */
} cur_status;

typedef enum { CUR_F64 = 0, CUR_F32 = 1, CUR_BF16 = 2 } cur_dtype;

/* A dense row-major matrix view (device memory). */
typedef struct {
    const void* data;
    int64_t rows, cols, ld;
    cur_dtype dtype;
} cur_mat;

/* Maxvol options. delta: swap while max|B_ij| > 1 + delta (default 1e-2).
 * max_swaps: cap on swaps per maxvol problem (<= 0 means 100 r).
 * nblocks: number of contiguous balanced row blocks of the tall basis.
 * flags: CUR_FLAG_POLISH runs maxvol over all rows after the merge (default on). */
typedef struct {
    double delta;
    int32_t max_swaps, nblocks;
    uint32_t flags;
} cur_opts;

#define CUR_FLAG_POLISH 1u
#define CUR_FLAG_PREC_BF16 2u   /* cur_maxvol_global: BF16 coefficient products first */
#define CUR_FLAG_PREC_FP8 4u    /* the same with E4M3 products (row-scaled); wins over BF16 */
/* FP32/BF16 data: factorise C(S,:) afresh at the start of every cycle of the swap iteration,
 * as the iteration of Section 1.2 is stated. Without it the kept double-float inverse is
 * carried across cycles while its drift bound, the sum over swaps of kappa_inf(C(S,:)), stays
 * at or below 2^18 (drift <= 2^-30 of an FP32 coefficient); FP64 data always factorises. */
#define CUR_FLAG_REFACTOR_ALWAYS 8u

/* Summary of one cur_cross call, written to DEVICE memory by cur_cross. */
typedef struct {
    double logvol;            /* log|det A(I,J)| of the returned cross */
    int32_t sweeps;           /* sweeps made (1..max) */
    int32_t swaps_total;      /* maxvol swaps over all stages */
    int32_t sweep_swaps[8];   /* swaps per sweep */
    int32_t aca_selected;     /* indices Algorithm 3 returned before padding */
    int32_t status;           /* cur_status of the whole call */
} cur_cross_info;

typedef struct cur_handle cur_handle;

/* Handle with `workspace_bytes` of device workspace on the current device.
 * cur_workspace_size gives the amount a problem of the given size needs. */
cur_status cur_create(cur_handle** h, size_t workspace_bytes);
cur_status cur_destroy(cur_handle* h);
size_t cur_workspace_size(int64_t m, int64_t n, int32_t r, cur_dtype dtype);

/* Algorithm 3 (Blockwise Adaptive Cross Approximation, Section 2.2).
 * axis = 1 selects r columns of A, axis = 0 selects r rows. Each round takes the
 * unselected row/column with the largest squared residual norm (lowest index on
 * ties) and projects it out of the residual. The residual is kept implicitly
 * (squared norms downdated by the projections onto an orthonormal basis of the
 * picks), which equals the paper's explicit blockwise projection up to rounding.
 * nblocks (>= 1) is Algorithm 3's block count; the result does not depend on it.
 * idx_out: r int32 (device); entries after an early stop are -1 and the status
 * word records CUR_WARN_RANK. */
cur_status cur_aca_select(cur_handle* h, const cur_mat* A, int axis, int32_t r,
                          int32_t nblocks, int32_t* idx_out, cudaStream_t stream);

/* Algorithm 1 (Section 1.3): adaptive cross approximation with full pivoting, the
 * paper's sequential baseline. From R_0 = A, step k takes (i, j) = argmax |R_k(i,j)|
 * (ties: the smallest row, then the smallest column) and eliminates
 * R_{k+1} = R_k - R_k(:,j) R_k(i,:) / R_k(i,j); r steps.
 * R_work: m x n row-major, contiguous device buffer of the compute type (double for
 * CUR_F64 data, float for CUR_F32 and CUR_BF16), owned by the caller; it receives the
 * residual R_r (rows I and columns J exactly zero). I_out, J_out: r int32 (device), the
 * pivots in selection order; piv_out: r doubles (device, may be NULL), the pivot values
 * R_k(i_k, j_k). A pivot at rounding level, |R_k(i,j)| <= max(m,n) eps max|A| with
 * eps = 2^-52, ends the loop: the remaining entries are -1 and the status word records
 * CUR_WARN_RANK; non-finite data records CUR_ERR_NONFINITE. 1 <= r <= min(m,n), else
 * CUR_ERR_ARG. Asynchronous. */
cur_status cur_aca_full(cur_handle* h, const cur_mat* A, int32_t r, void* R_work,
                        int32_t* I_out, int32_t* J_out, double* piv_out, cudaStream_t stream);

/* One matrix of a batch for cur_cross_batched. */
typedef struct {
    int64_t offset;              /* element offset of the matrix in the batch buffer */
    int64_t rows, cols, ld;      /* shape and leading dimension (row-major) */
    int32_t r, b_r, b_c;         /* rank, row blocks and column blocks of its cross */
} cur_batch_item;

/* Workspace bytes that cur_cross_batched needs for these items (host array). */
size_t cur_batch_workspace_size(const cur_batch_item* items, int32_t count);

/* The cross of every matrix of a batch: for each matrix what cur_cross computes (J0 by
 * Algorithm 3 on the columns, blockwise maxvol rows and columns with the binary merge,
 * global sweeps until none swaps), with every stage shared by all matrices: one launch
 * of Algorithm 3 for the whole batch, then the row selection (all blocks of all matrices
 * in one stage, each merge level of all matrices in one stage, all polishes in one
 * stage), the column selection the same way, and each half-sweep over the matrices that
 * have not converged. data: device buffer, CUR_F32 only; matrix t at data +
 * items[t].offset with leading dimension items[t].ld. items: host array of count entries
 * (count <= 65535), each with 1 <= r <= 64, r < min(rows, cols), rows <= 4096,
 * cols <= 1024, rows / b_r >= r and cols / b_c >= r, else CUR_ERR_ARG. IJ_out: device
 * int32; matrix t's I (r row ids) then J (r column ids) start at 2 (r_0 + ... + r_{t-1}).
 * info_out: device array of count cur_cross_info (may be NULL), each with that matrix's
 * status, log-volume, sweeps and swaps. The handle's status word records
 * CUR_ERR_SINGULAR or CUR_ERR_NOCONV if any matrix ended so, else CUR_WARN_RANK if
 * Algorithm 3 ran out early on any. Every decision per matrix (a merge node's next start,
 * the end of its sweeps, its status) is taken on the device and all sweeps are enqueued, so
 * the call only enqueues — except the first call of each class of batch (batch size and work
 * per matrix), which times the two launch shapes of Algorithm 3 and waits for them. After
 * that first call a batch of the same class can be captured in a CUDA graph and replayed. */
cur_status cur_cross_batched(cur_handle* h, const void* data, cur_dtype dtype,
                             const cur_batch_item* items, int32_t count, const cur_opts* opts,
                             int32_t* IJ_out, cur_cross_info* info_out, cudaStream_t stream);

/* Row selection for given columns J (r int32, device): maxvol on C = A(:,J).
 * C is split into opts->nblocks contiguous balanced row blocks (each >= r rows,
 * else CUR_ERR_ARG); each block starts from Algorithm 3 on its rows and runs
 * maxvol (B = C_k M^-1, swap while max|B_ij| > 1 + delta, Sherman-Morrison
 * updates; every r swaps a new cycle from C_k(S,:) factorised afresh); the block
 * sets are merged pairwise (binary
 * tournament, cur_merge) and, with CUR_FLAG_POLISH, refined by maxvol over all
 * rows. Outputs (device): I_out r int32, logvol_out 1 double (log|det C(I,:)|),
 * swaps_out 1 int32. */
cur_status cur_maxvol_rows(cur_handle* h, const cur_mat* A, const int32_t* J, int32_t r,
                           const cur_opts* opts, int32_t* I_out, double* logvol_out,
                           int32_t* swaps_out, cudaStream_t stream);

/* Column selection for given rows I: the same as cur_maxvol_rows on A(I,:)^T. */
cur_status cur_maxvol_cols(cur_handle* h, const cur_mat* A, const int32_t* I, int32_t r,
                           const cur_opts* opts, int32_t* J_out, double* logvol_out,
                           int32_t* swaps_out, cudaStream_t stream);

/* One level of the binary merge: the "binary parallel selection process" of Section 2.1,
 * which the paper names but does not define, read as a tournament of pairwise merges
 * in which each node runs the maximal-volume swap iteration (Section 1.2) on the union
 * of its two children. basis: p x r tall basis (device); cand: nsets x r
 * row indices of the basis (device, set t in row t). Node t merges sets 2t and
 * 2t+1 by maxvol on their 2r rows (left set first) started at the left set (the
 * right set if the left one is singular, Algorithm 3 on the union if both are);
 * an odd last set passes through. out: ceil(nsets/2) x r int32 (device). */
cur_status cur_merge(cur_handle* h, const cur_mat* basis, const int32_t* cand, int32_t nsets,
                     int32_t r, const cur_opts* opts, int32_t* out, cudaStream_t stream);

/* CUR assembly (Section 1.1): C = A(:,J) (m x r, A's dtype), R = A(I,:) (r x n, A's
 * dtype), U = A(I,J)^dagger (r x r double, row-major): the LU inverse (FP64,
 * partial pivoting) when rcond = 1/(|M|_1 |M^-1|_1) >= 1e-13, else the
 * pseudo-inverse by a one-sided Jacobi SVD with cutoff r eps s_max.
 * rcond_out: 1 double (device; 0 when M is singular). */
cur_status cur_assemble(cur_handle* h, const cur_mat* A, const int32_t* I, const int32_t* J,
                        int32_t r, void* C_out, double* U_out, void* R_out,
                        double* rcond_out, cudaStream_t stream);

/* Residual of the cross (Theorem 1; Section 3.1 error measure):
 * cheb_out = max_ij |A - C (U R)|, fro_rel_out = ||A - CUR||_F / ||A||_F (may be
 * NULL). C: m x r and R: r x n in A's dtype (as cur_assemble writes them), U: r x r
 * double. Arithmetic in FP32 for FP32/BF16 data, FP64 for FP64 data; sums are
 * carried in FP64. Outputs are device doubles. */
cur_status cur_residual_cheb(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                             const void* R, int32_t r, double* cheb_out, double* fro_rel_out,
                             cudaStream_t stream);

/* Allocation-free residual (the paper has no counterpart; the arithmetic is that of
 * cur_residual_cheb, with the same arguments and outputs but no handle). It is for
 * callers that cannot allocate device memory where they need the residual, e.g. after
 * handing all device memory to their own pool, or inside a loop that must not hit
 * cudaMalloc's implicit synchronisation. Its scratch (W = U R, r x n in the arithmetic
 * type, plus 32 bytes per CTA) lives in one 16 MiB array compiled into the library,
 * present on every device that loads it until the process exits; larger problems
 * (about r n > 4e6 for FP32/BF16 data, 2e6 for FP64) return CUR_ERR_NOMEM before any
 * launch. The array is shared by every call and keeps the last call's contents; calls
 * whose work overlaps on the GPU (other streams, other threads) race on it, so order
 * them. The first call on each device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first call before
 * any stream capture. Resetting the device (cudaDeviceReset, or releasing its primary
 * context) after that first call is not supported: the kept address would be stale. It
 * calls no cudaMalloc or cudaFree. A non-finite value in the data gives cheb_out = NaN (there
 * is no handle status word to record it). */
cur_status cur_residual_cheb_noalloc(const cur_mat* A, const void* C, const double* U,
                                     const void* R, int32_t r, double* cheb_out,
                                     double* fro_rel_out, cudaStream_t stream);

/* The whole cross (Algorithm 2 with blockwise maxvol refinement): J0 = Algorithm 3
 * on the columns (b_c blocks; padded with the lowest unused columns after an early
 * stop), sweep 1 = {I = cur_maxvol_rows(J0, b_r), J = cur_maxvol_cols(I, b_c)},
 * sweeps 2..8 = {maxvol on all rows of A(:,J) from I, maxvol on all columns of
 * A(I,:) from J} until a sweep makes no swap. I_out, J_out: r int32 (device);
 * info_out: one cur_cross_info (device, may be NULL). */
cur_status cur_cross(cur_handle* h, const cur_mat* A, int32_t r, int32_t b_r, int32_t b_c,
                     const cur_opts* opts, int32_t* I_out, int32_t* J_out,
                     cur_cross_info* info_out, cudaStream_t stream);

/* Maxvol over all p rows of a basis (p x r, contiguous: ld = cols = r; CUR_F32 or CUR_F64)
 * from the start rows S0 (r int32, device): B = C M^-1 with M = C(S,:), swap the row of
 * argmax |B_ij| into position j while |B_ij| > 1 + delta, Sherman-Morrison updates, a fresh
 * factorisation every r swaps (the swap iteration of Section 1.2's maximal-volume
 * refinement). With CUR_FLAG_PREC_BF16 in opts->flags (CUR_F32 basis, r a multiple of 16),
 * each iteration first forms B for all rows as a BF16 x BF16 -> FP32 tensor-core product
 * and takes its argmax, recomputes the winner exactly (FP64) and swaps only if the exact
 * value exceeds 1 + delta; the first winner that does not ends that phase, and the
 * FP32/FP64 iteration finishes from the set reached. CUR_FLAG_PREC_FP8 does the same with
 * E4M3 x E4M3 -> FP32 products, each row of C and of (M^-1)^T scaled to E4M3's range (448). Outputs (device): S_out r int32,
 * logvol_out 1 double (may be NULL), swaps_out 2 int32 (may be NULL): all swaps, and the
 * swaps of the BF16 phase. A singular C(S0,:) records CUR_ERR_SINGULAR (S_out = S0); more
 * than max_swaps records CUR_ERR_NOCONV. Asynchronous, with or without the low-precision
 * flags (their swap loop is one cooperative launch that ends itself on the device). */
cur_status cur_maxvol_global(cur_handle* h, const cur_mat* basis, const int32_t* S0, int32_t r,
                             const cur_opts* opts, int32_t* S_out, double* logvol_out,
                             int32_t* swaps_out, cudaStream_t stream);

/* The swap coefficients of the maximal-volume iteration (Section 1.2: B = C M^-1, whose entry
 * B_ij is the factor by which |det M| changes when row i replaces position j) on the tensor
 * cores: B_out (p x r FP32, contiguous) = basis (p x r FP32, contiguous) times minv (r x r
 * FP64, row-major, device), as 3xTF32 tcgen05 products (C and M^-1 each split into a TF32
 * high and low part; the low x low term is dropped, ~2^-22 relative). r must be 32 or 64,
 * else CUR_ERR_ARG. The swap engine forms the first cycle's B this way on FP32 stages of
 * at least 8192 rows with r = 32 or 64; this call exposes the product alone. Asynchronous. */
cur_status cur_coef_tf32(cur_handle* h, const cur_mat* basis, const double* minv, float* B_out,
                         cudaStream_t stream);

/* ---- Learned proposal (where the maxvol sweeps of Algorithm 2 start)
 *
 * A scoring network ranks the rows and the columns of A from a Gaussian sketch; the
 * r best-ranked of each are a proposed cross (I0, J0), which cur_cross_from refines by
 * the sweeps of global maxvol that end the cross (Section 3). Nothing here changes what
 * a converged cross is; the proposal only sets where the sweeps begin. */

/* Sketch features: Y = A S (m x k) and Zt = A^T T (n x k), row-major FP32, device, for
 * S (n x k) and T (m x k) row-major FP32 on the device (the caller draws them, e.g.
 * i.i.d. N(0, 1/k)). With normalize != 0, Y is divided by its largest row norm and Zt by
 * its own (unchanged if that is 0). A: any supported dtype (read as FP32). k must be 32;
 * S, T, Y, Zt 16-byte aligned; else CUR_ERR_ARG. FP32 accumulation, deterministic
 * (fixed summation order). Asynchronous. */
cur_status cur_sketch(cur_handle* h, const cur_mat* A, const float* S, const float* T, int32_t k,
                      float* Y, float* Zt, int32_t normalize, cudaStream_t stream);

/* The scoring network's parameters are one FP32 array of k*H + 2*H + 1 values: W1 (k x H,
 * row-major), b1 (H), w2 (H), b2. score(x) = relu(x W1 + b1) . w2 + b2 for a feature row
 * x (k values). k must be 32 and H a multiple of 32 in [32, 256]; X 16-byte aligned. */

/* scores[s] = score(X[s]) for the N rows of X (N x k, device). Asynchronous. */
cur_status cur_mlp_forward(cur_handle* h, const float* X, int64_t N, int32_t k, int32_t H,
                           const float* params, float* scores, cudaStream_t stream);

/* Gradient of the weighted mean binary cross-entropy
 *   L = (1/N) sum_s w_s [ y_s log(1 + e^-score_s) + (1 - y_s) log(1 + e^score_s) ],
 * w_s = pos_weight for y_s = 1 and 1 for y_s = 0, over the samples s = idx[0..N) (rows of
 * X, nrows x k, and entries of y, nrows; idx NULL: 0..N-1, N <= nrows). A sample index
 * outside [0, nrows) contributes nothing and records CUR_ERR_ARG. grads: same layout as
 * params (device); loss: one double (device, may be NULL). Deterministic. Asynchronous. */
cur_status cur_mlp_grad(cur_handle* h, const float* X, const float* y, int64_t nrows, const int64_t* idx,
                        int64_t N, int32_t k, int32_t H, const float* params, float pos_weight,
                        float* grads, double* loss, cudaStream_t stream);

/* One Adam step (Kingma and Ba, 2015) at step t >= 1 on count parameters, in place:
 * m1 = b1 m1 + (1 - b1) g, m2 = b2 m2 + (1 - b2) g^2,
 * params -= lr (m1 / (1 - b1^t)) / (sqrt(m2 / (1 - b2^t)) + eps). Asynchronous. */
cur_status cur_adam_step(cur_handle* h, float* params, const float* grads, float* m1, float* m2,
                         int64_t count, int32_t t, float lr, float beta1, float beta2, float eps,
                         cudaStream_t stream);

/* idx_out (r int32, device) = the indices of the r largest scores (N of them, device), in
 * decreasing score, equal scores by increasing index, NaN below every number.
 * 1 <= r <= N < 2^31. Asynchronous. */
cur_status cur_propose(cur_handle* h, const float* scores, int64_t N, int32_t r, int32_t* idx_out,
                       cudaStream_t stream);

/* Refinement of a proposed cross (I0, J0) (r int32 each, device): sweeps of global maxvol
 * on A(:,J) from I, then on A(I,:)^T from J, until a sweep makes no swap (at most 8), as
 * the sweeps that end cur_cross. If A(I0,J0) is singular nothing is refined: I = I0,
 * J = J0, info logvol = -inf, and CUR_ERR_SINGULAR is recorded (the caller falls back to
 * cur_cross). A sweep stage that ends SINGULAR or NOCONV records that status. info_out:
 * one cur_cross_info (device, may be NULL; aca_selected = 0, status = the end status).
 * 1 <= r <= 128, r < min(m, n). */
cur_status cur_cross_from(cur_handle* h, const cur_mat* A, int32_t r, const int32_t* I0,
                          const int32_t* J0, const cur_opts* opts, int32_t* I_out, int32_t* J_out,
                          cur_cross_info* info_out, cudaStream_t stream);

/* ---- Sharded cross: one process per GPU, each holding a contiguous slab of the rows of A
 *
 * The calls below are the per-rank steps of the cross when A is partitioned by rows over P
 * processes (Section 2.2 divides A into blocks handled by separate processes; Algorithm 3
 * reduces a (norm, index) pair over the blocks and broadcasts the pivot vector each round).
 * Each call works on the caller's slab only and enqueues on `stream`; the caller makes the
 * collectives between the calls (allreduce-sum, -max, -min of small device vectors) on its
 * own transport (NCCL between GPUs). The driver that strings them together is
 * paper_2502_11017_gb300.shard. BF16 slabs are accepted by the Algorithm 3 calls only. */

/* Algorithm 3 on the columns of A over row slabs. state: a caller-owned device buffer of
 * cur_shard_aca_state_bytes(h, A_k, r) bytes (the slab's share of the orthonormal basis Q,
 * the replicated squared norms and W = Q^T A, the pivot vector). A round t = 0 .. r-1 is
 *   pick(t, red) -> red2 ; allreduce-sum red2 (r doubles)
 *   commit(t, red2) -> red ; allreduce-sum red (n doubles)
 * after begin (-> red, the slab's squared column norms; allreduce-sum it). pick takes the
 * summed red (t = 0: the squared norms; t > 0: w = A^T q_{t-1}, so nu_j -= w_j^2), picks the
 * unpicked column of largest residual norm (lowest index on ties), forms the slab's part of
 * v = a_p - Q (Q^T a_p) and returns its partials of Q^T v (red2[0..t)) and of ||v||^2
 * (red2[t]). commit re-orthogonalises v once (CGS2: v -= Q (Q^T v)), whose squared norm is
 * red2[t] - ||red2[0..t)||^2 for orthonormal Q, stops the selection when that is <=
 * (max(m,n) eps ||A||_F)^2 (CUR_WARN_RANK in the status word; later calls do nothing), else
 * records p in idx_out[t], stores q_t = v / ||v|| and, while t + 1 < r, streams the slab once
 * for the next round's partial w. finish pads an early-stopped idx_out with the lowest unused
 * columns. m_global: rows of the whole A. idx_out: r int32 (device), -1 until picked. red: n
 * doubles, red2: r doubles (device). */
size_t cur_shard_aca_state_bytes(cur_handle* h, const cur_mat* A_k, int32_t r);
cur_status cur_shard_aca_begin(cur_handle* h, const cur_mat* A_k, int64_t m_global, int32_t r, void* state,
                               int32_t* idx_out, double* red, cudaStream_t stream);
cur_status cur_shard_aca_pick(cur_handle* h, const cur_mat* A_k, int32_t r, int32_t t, void* state,
                              const double* red, double* red2, cudaStream_t stream);
cur_status cur_shard_aca_commit(cur_handle* h, const cur_mat* A_k, int32_t r, int32_t t, void* state,
                                const double* red2, int32_t* idx_out, double* red, cudaStream_t stream);
cur_status cur_shard_aca_finish(cur_handle* h, const cur_mat* A_k, int32_t r, void* state, int32_t* idx_out,
                                cudaStream_t stream);

/* Maxvol over all rows of a basis C (p x r) distributed by row slabs: C_k (p_local x r,
 * contiguous, CUR_F32 or CUR_F64) holds global rows offset .. offset + p_local - 1. Every
 * rank holds the same S (r global row ids, position order) and M = C(S,:) (M_rows, r x r in
 * C's dtype, device). state: cur_dmv_state_bytes(p_local, r, dtype) bytes (B = C_k M^-1 in
 * C's dtype, M and its FP64 inverse, S, log|det M|, counters). The swap iteration:
 *   begin / refresh -> keyv (the slab's max |B_ij|; -1 if M is numerically singular,
 *       |u_kk| <= r eps max|M|, in which case the state's status is CUR_ERR_SINGULAR);
 *       begin loads S and M; both factorise M afresh in FP64 and form B.
 *   allreduce-max keyv; if it is <= 1 + delta the cycle ends (a cycle that ends with no swap
 *       ends the iteration; otherwise refresh starts the next cycle; cycles are r swaps);
 *   holder(keyv) -> keyi: the slab's flat index (global row * r + j) if it holds that value,
 *       else INT64_MAX; allreduce-min keyi (the lowest index wins a tie);
 *   fill(keyi) -> row: the winner's row of C if this slab owns it, else zeros; allreduce-sum;
 *   swap(keyi, row) -> keyv: b = row M^-1 in FP64, M^-1 -= M^-1(:,j) (b - e_j)^T / b_j,
 *       B -= B(:,j) (b - e_j)^T / b_j, S[j] = row id, log|det| += log|b_j|.
 * result writes S (r int32), log|det M| (1 double) and counts (2 int32: swaps, status);
 * any output may be NULL. Section 1.2's maximal-volume refinement; the same iteration as
 * cur_maxvol_global, with the ranks' agreement made by the caller. */
size_t cur_dmv_state_bytes(int64_t p_local, int32_t r, cur_dtype dtype);
cur_status cur_dmv_begin(cur_handle* h, const cur_mat* C_k, int64_t offset, const int32_t* S, const void* M_rows,
                         void* state, double* keyv_out, cudaStream_t stream);
cur_status cur_dmv_refresh(cur_handle* h, const cur_mat* C_k, int64_t offset, void* state, double* keyv_out,
                           cudaStream_t stream);
cur_status cur_dmv_holder(cur_handle* h, const cur_mat* C_k, void* state, const double* keyv_glob,
                          long long* keyi_out, cudaStream_t stream);
cur_status cur_dmv_fill(cur_handle* h, const cur_mat* C_k, int64_t offset, const long long* keyi_glob, void* row_out,
                        cudaStream_t stream);
cur_status cur_dmv_swap(cur_handle* h, const cur_mat* C_k, int64_t offset, void* state, const long long* keyi_glob,
                        const void* row, double* keyv_out, cudaStream_t stream);
cur_status cur_dmv_result(cur_handle* h, const cur_mat* C_k, void* state, int32_t* S_out, double* logvol_out,
                          int32_t* counts_out, cudaStream_t stream);

/* One node of the binary merge given by the two sets' rows: rows (2r x r, contiguous,
 * CUR_F32 or CUR_F64; the left set's r rows, then the right set's) and their ids (2r int32).
 * Maxvol on the 2r rows started at the left set (the right set if the left one is singular,
 * Algorithm 3 on the union if both are), as one node of cur_merge. ids_out: r int32; rows_out:
 * r x r in rows' dtype (the merged set's rows, position order); swaps_out: 1 int32 (may be
 * NULL). For a merge whose two sets live on different processes. */
cur_status cur_merge_pair(cur_handle* h, const cur_mat* rows, const int32_t* ids, const cur_opts* opts,
                          int32_t* ids_out, void* rows_out, int32_t* swaps_out, cudaStream_t stream);

/* out (count x X.cols, X's dtype, contiguous) row j = X(ids[j] - offset, :) when that row
 * lies in X (0 <= ids[j] - offset < X.rows), else zeros: the slab's share of A(I,:), whose
 * sum over the ranks is A(I,:). CUR_F32 or CUR_F64. */
cur_status cur_rows_at(cur_handle* h, const cur_mat* X, int64_t offset, const int32_t* ids, int32_t count,
                       void* out, cudaStream_t stream);
/* Xt_out (X.cols x X.rows, contiguous) = X^T. CUR_F32 or CUR_F64. */
cur_status cur_transpose(cur_handle* h, const cur_mat* X, void* Xt_out, cudaStream_t stream);
/* out[k] = ids[k] + offset (slab-local to global ids). */
cur_status cur_offset_ids(cur_handle* h, const int32_t* ids, int32_t count, int64_t offset, int32_t* out,
                          cudaStream_t stream);
/* C_out = A(:,J) (A.rows x r, contiguous) in the compute type: FP64 for CUR_F64 data, FP32
 * otherwise (Section 1.1's C). */
cur_status cur_gather_cols(cur_handle* h, const cur_mat* A, const int32_t* J, int32_t r, void* C_out,
                           cudaStream_t stream);
/* The residual's parts on A (a slab): parts_out = {max |A - C U R|, sum (A - CUR)^2, sum A^2}
 * (3 doubles, device), the terms of Theorem 1's Chebyshev norm and Section 3.1's relative
 * Frobenius error before the reduction over slabs (max, sum, sum). Arguments as
 * cur_residual_cheb. */
cur_status cur_residual_parts(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                              const void* R, int32_t r, double* parts_out, cudaStream_t stream);

/* Synchronise `stream` and return (and clear) the first device-side status. */
cur_status cur_sync_status(cur_handle* h, cudaStream_t stream);

/* Instrumentation (no counterpart in the paper). With cur_prof_enable(h, 1) the
 * library brackets every launch of the Algorithm 3 streaming pass with CUDA events
 * on the caller's stream. cur_prof_read synchronises `stream`, returns the summed
 * duration of those launches (pass_ms) and their number (pass_launches), the number
 * of kernels this library launched since the last read (kernel_launches, all
 * handles), and resets the three. Any output pointer may be NULL (host memory). */
cur_status cur_prof_enable(cur_handle* h, int on);
cur_status cur_prof_read(cur_handle* h, cudaStream_t stream, double* pass_ms,
                         int32_t* pass_launches, int64_t* kernel_launches);

/* Instrumentation: the number of factorisations of C(S,:) made at cycle boundaries of the
 * swap iteration (every cycle for FP64 data or with CUR_FLAG_REFACTOR_ALWAYS; for FP32/BF16
 * data otherwise only when the drift bound exceeds 2^18) by this handle's calls since the
 * last read. Synchronises `stream`, writes the count to *count (host) and resets it. */
cur_status cur_prof_refactors(cur_handle* h, cudaStream_t stream, int64_t* count);

/* Self-test of the bounded device waits (no counterpart in the paper): launches one CTA
 * that waits at a group barrier for a partner that does not exist. The wait gives up
 * after ~50 ms and records CUR_ERR_TIMEOUT in the status word (read it with
 * cur_sync_status); the context stays usable. Every spin-wait in this library has such a
 * limit (about 1-2 s in normal calls). */
cur_status cur_selftest_wait_timeout(cur_handle* h, cudaStream_t stream);

/* Default options: delta 1e-2, max_swaps 100 r, nblocks 1, CUR_FLAG_POLISH. */
cur_opts cur_default_opts(void);

const char* cur_status_string(cur_status s);

#ifdef __cplusplus
}
#endif
#endif /* CUR_H */
