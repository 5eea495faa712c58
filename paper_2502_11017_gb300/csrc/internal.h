// Host-side internals shared by the libcur translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "cur.h"

#define CUR_CK(x)                                                   \
    do {                                                            \
        cudaError_t e_ = (x);                                       \
        if (e_ != cudaSuccess) return CUR_ERR_CUDA;                 \
    } while (0)

#define CUR_TRY(x)                                                  \
    do {                                                            \
        cur_status s_ = (x);                                        \
        if (s_ != CUR_OK) return s_;                                \
    } while (0)

// Bump allocator over the handle's workspace; reset at the start of each call.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    bool ok = true;
    void* take(size_t bytes, size_t align = 256) {
        size_t o = (off + align - 1) / align * align;
        if (o + bytes > cap) {
            ok = false;
            return nullptr;
        }
        off = o + bytes;
        return base + o;
    }
    template <typename T>
    T* get(size_t count) {
        return static_cast<T*>(take(count * sizeof(T) + 16));
    }
};

// Counts kernel launches made by the library (all handles).
void note_launch(int n = 1);

struct cur_handle {
    // instrumentation: events around the Algorithm 3 pass launches
    int prof = 0;
    int prof_n = 0;
    cudaEvent_t prof_ev[2 * 4096] = {};
    int device = 0;
    int num_sms = 0;
    char* ws = nullptr;          // device workspace
    size_t ws_bytes = 0;
    int* status = nullptr;       // device status word (first error wins)
    char* host_stage = nullptr;  // pinned host buffer for small transfers
    size_t host_stage_bytes = 0;
    cudaEvent_t stage_ev = nullptr;  // recorded after the last copy that reads host_stage
    // Autotuner: the launch shape chosen for each shape class (key), by timing the candidates
    // on the first call of that class. Only shapes that leave results unchanged are tuned.
    struct TuneEntry {
        uint64_t key;
        int choice;
    };
    TuneEntry tune[64] = {};
    int ntune = 0;
    cudaEvent_t tune_ev[2] = {};    // timing events of the tuning runs
    Arena arena() const {
        Arena a;
        a.base = ws;
        a.cap = ws_bytes;
        return a;
    }
};

// The tuned choice for a shape class, or -1 if it has not been tuned yet.
inline int tune_lookup(const cur_handle* h, uint64_t key) {
    for (int i = 0; i < h->ntune; ++i)
        if (h->tune[i].key == key) return h->tune[i].choice;
    return -1;
}
inline void tune_store(cur_handle* h, uint64_t key, int choice) {
    for (int i = 0; i < h->ntune; ++i)
        if (h->tune[i].key == key) { h->tune[i].choice = choice; return; }
    const int slot = h->ntune < 64 ? h->ntune++ : (int)(key % 64);   // a full table reuses slots
    h->tune[slot].key = key;
    h->tune[slot].choice = choice;
}
// floor(log2(x)) for x >= 1 (0 otherwise): the size buckets of the tuning keys.
inline uint64_t tune_log2(uint64_t x) {
    uint64_t b = 0;
    while (x > 1) { x >>= 1; ++b; }
    return b;
}

// Element size of a cur_dtype.
inline size_t dtype_size(cur_dtype t) { return t == CUR_F64 ? 8 : (t == CUR_F32 ? 4 : 2); }

// ---- Algorithm 3 on a full matrix (aca.cu)
// Writes r indices (or -1 after an early stop) to idx_out and the number picked
// to *count_dev (both device). stop_dev (device int) is set on an early stop.
cur_status aca_select_full(cur_handle* h, const cur_mat* A, int axis, int r, int32_t* idx_out,
                           int32_t* count_dev, Arena& ar, cudaStream_t st);

// ---- maxvol pipelines (maxvol.cu)
//
// The pipelines only enqueue: every decision that depends on a result (a singular start, an
// inverse valid to inherit, the end of the sweeps) is taken by a kernel on the device.

// A maxvol call's result, written on the device for later kernels (the host never reads it).
struct MvDevResult {
    int32_t swaps;
    int32_t status;
    int32_t minv_valid;   // minv_out holds the final FP64 M^-1
    int32_t pad;
};
// An inverse handed between stages is minv_stride(r) doubles: M^-1 (r x r, row-major),
// then a bound on the rounding drift that Sherman-Morrison updates have added to it since
// it was last factorised (sum over swaps of kappa_inf(M)).
inline __host__ __device__ int64_t minv_stride(int r) { return (int64_t)r * r + 1; }

// Row selection on the tall basis `basis` (p x r, compute type of A's dtype,
// contiguous) with nblocks blocks, merge and optional polish. I_out: device r ints.
// With minv_out (minv_stride(r) doubles, device), the final FP64 M^-1 = C(I,:)^-1 is written
// there (res->minv_valid says whether it is valid). res: device, may be null. Nothing runs
// while *idle != 0 (device flag, may be null).
cur_status maxvol_basis_rows(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                             const cur_opts* o, int32_t* I_out, double* logvol_out,
                             int32_t* swaps_out, MvDevResult* res, Arena& ar, cudaStream_t st,
                             double* minv_out = nullptr, const int* idle = nullptr);
// Maxvol over all rows of a basis from the start rows S0 (device r ints, global
// rows). Writes the result to S_out (device, may alias S0).
// minv_in / lv_in (optional): M^-1 and log|det| of the start rows, given as is or as the
// transpose of the inverse (transpose_in) — a column stage's M^-1 is the transpose of the
// next row stage's; valid while *minv_in_valid != 0 (device; null: valid); no factorisation is
// made then. minv_out as for maxvol_basis_rows.
// If the set turns numerically singular, S_out is the start set, or with
// keep_singular_set the set reached at that point (the swap iteration's own result).
cur_status maxvol_global(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                         const cur_opts* o, const int32_t* S0, int32_t* S_out,
                         double* logvol_out, MvDevResult* res, Arena& ar, cudaStream_t st,
                         const double* minv_in = nullptr, const double* lv_in = nullptr,
                         const int* minv_in_valid = nullptr, bool transpose_in = false,
                         double* minv_out = nullptr, bool keep_singular_set = false,
                         const int* idle = nullptr);
// One merge level (cur_merge); its swaps are added to *acc_dev (device int).
cur_status merge_level(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                       const int32_t* cand, int nsets, const cur_opts* o, int32_t* out,
                       int* acc_dev, Arena& ar, cudaStream_t st);

// The sweeps of a cross on the device (cur_cross, cur_cross_from).
struct CrossCtl {
    int idle;             // nonzero: the remaining sweeps do nothing
    int abort;            // Algorithm 3 met an error: nothing after it runs
    int sweeps;
    int sweep_swaps[8];
    int last_status;      // a stage that ended NOCONV or SINGULAR
    int mc_valid;         // the last column stage's inverse is valid
    int singular_start;   // cur_cross_from: the proposed A(I0, J0) is singular
};
// Starts the control block; with check_status, an error already in the status word (from
// Algorithm 3) makes every later stage idle.
cur_status cross_begin(CrossCtl* ctl, const int* hstatus, bool check_status, cudaStream_t st);
// Sweep 1 of cur_cross (blockwise rows and columns) ended with these results.
cur_status cross_sweep_one(CrossCtl* ctl, const MvDevResult* rr, const MvDevResult* rc, cudaStream_t st);
// Sweeps first .. max_sweeps (all enqueued; idle once one makes no swap or ends with an error).
cur_status cross_sweeps(cur_handle* h, const cur_mat* A, int r, const cur_opts* o, int first, int max_sweeps,
                        bool from, int32_t* I, int32_t* J, void* Cb, void* Rb, double* Mr, double* Mc, double* lvr,
                        double* lv, CrossCtl* ctl, Arena& ar, cudaStream_t st);
// The cross's log-volume, status, outputs and info.
cur_status cross_end(cur_handle* h, const cur_mat* A, int r, bool from, const int32_t* I, const int32_t* J,
                     void* Rb, double* lv, CrossCtl* ctl, const int32_t* aca_count, int32_t* I_out, int32_t* J_out,
                     cur_cross_info* info_out, Arena& ar, cudaStream_t st);
// Gathers into the compute type: C = A(:,J) (m x r) and Rt = A(I,:)^T (n x r); nothing runs
// while *idle != 0.
cur_status gather_cols_compute(const cur_mat* A, const int32_t* J, int r, void* C, cudaStream_t st,
                               const int* idle = nullptr);
// The merge of two candidate sets given by their rows (2r x r, left set first) and ids
// (cur_merge_pair).
cur_status merge_pair_impl(cur_handle* h, cur_dtype dt, const void* rows, const int32_t* ids, int r,
                           const cur_opts* o, int32_t* ids_out, void* rows_out, int32_t* swaps_out, Arena& ar,
                           cudaStream_t st);
// The cross of every matrix of a batch (cur_cross_batched), FP32 data.
cur_status cross_batched_impl(cur_handle* h, const float* data, const cur_batch_item* items, int T,
                              const cur_opts* o, int32_t* IJ_out, cur_cross_info* info_out, Arena& ar,
                              cudaStream_t st);
// Algorithm 1 (ACA with full pivoting) into the caller's residual buffer R (m x n,
// compute type); see cur_aca_full.
cur_status aca_full_impl(cur_handle* h, const cur_mat* A, int r, void* R, int32_t* I, int32_t* J,
                         double* piv, Arena& ar, cudaStream_t st);
// log|det basis(rows,:)| (rows: device r ints) into *out (device), -inf for an exactly
// singular matrix; basis p x r contiguous in the compute type of dt (a row id outside
// [0, p) reads as a zero row).
cur_status logvol_rows(cur_dtype dt, const void* basis, int64_t p, int r, const int32_t* rows, double* out,
                       cudaStream_t st);
cur_status gather_rows_t_compute(const cur_mat* A, const int32_t* I, int r, void* Rt,
                                 cudaStream_t st, const int* idle = nullptr);
size_t compute_size(cur_dtype t);

// ---- low-precision coefficient phase of global maxvol (lowprec.cu)
// The BF16 (or, with CUR_FLAG_PREC_FP8, E4M3) phase alone, from S0 to S_out (device r ints,
// may alias), enqueued only. minv_in: the FP64 inverse of C(S0,:) (r x r), used when
// minv_flag is NULL or reads CUR_OK / CUR_ERR_NOCONV on the device, else (or when NULL)
// C(S0,:) is factorised; a singular start leaves S_out = S0. idle: a device word that skips the
// phase when set (may be NULL). *swaps_dev (device): the swaps the phase took.
cur_status lowprec_phase(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o, const int32_t* S0,
                         int32_t* S_out, int32_t* swaps_dev, Arena& ar, cudaStream_t st,
                         const double* minv_in, const int* minv_flag, const int* idle);
// Whether the stages of cur_cross take that phase (CUR_FLAG_PREC_BF16 or _FP8, FP32 basis,
// r a multiple of 16, and enough rows to fill the GPU).
bool lowprec_phase_applies(const cur_handle* h, const cur_opts* o, cur_dtype dt, int64_t p, int r);

// ---- learned proposal (proposal.cu)
// Workspace bytes of cur_sketch's split partials on a device with num_sms SMs.
size_t sketch_workspace_size(int num_sms, int64_t m, int64_t n);

// ---- assembly and residual (residual.cu)
cur_status assemble_impl(cur_handle* h, const cur_mat* A, const int32_t* I, const int32_t* J,
                         int r, void* C_out, double* U_out, void* R_out, double* rcond_out,
                         Arena& ar, cudaStream_t st);
// sums_out (2 doubles, device, may be NULL): sum (A - CUR)^2 and sum A^2 in FP64.
cur_status residual_impl(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                         const void* R, int r, double* cheb_out, double* fro_out, Arena& ar,
                         cudaStream_t st, double* sums_out = nullptr);

// tcgen05 residual for FP32 data, r = 32 or 64 (residual_tc.cu); CUR_ERR_ARG: not applicable.
cur_status residual_tc_impl(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                            const void* R, int r, double* cheb_out, double* fro_out, Arena& ar,
                            cudaStream_t st, double* sums_out = nullptr);

// Raises a kernel's dynamic shared-memory limit (on the current device) to at least `bytes`
// and never lowers it, so that calls from several host threads cannot shrink the limit
// under another thread's launch.
cur_status smem_attr(const void* fn, size_t bytes);

// Small host tables to device memory as kernel parameters (no host buffer outlives the
// call, the host never waits): maxvol.cu.
cur_status upload_table(void* dst, const void* src, size_t bytes, cudaStream_t st);

// ---- the coefficient product on the tensor cores (coef_tc.cu)
// A 128-row tile (rows row0 .. row0 + nrows - 1 of the basis) of problem prob.
struct CoefTile {
    int32_t prob;
    int32_t nrows;
    int64_t row0;
};
// FP32 bases with r = 32 or 64.
bool coef_tc_applies(cur_dtype dt, int r);
size_t coef_tc_smem(int r);
// B (prows x r, the basis's layout) = C M_prob^-1 on each tile, 3xTF32 tcgen05; minv64: P
// inverses (FP64, r x r, minv_stride apart); Wh, Wl: P r^2 floats of scratch; tiles of done
// problems are skipped.
cur_status coef_tc_launch(cur_handle* h, const float* basis, int64_t prows, int r, const double* minv64,
                          int64_t minv_stride_, int P, const CoefTile* tiles_dev, int ntiles, const int32_t* done,
                          float* Wh, float* Wl, float* B, cudaStream_t st);

// Cooperative launch helper (all CTAs co-resident).
cur_status launch_coop(const void* fn, dim3 grid, dim3 block, void** args, size_t smem,
                       cudaStream_t st);

// ---- the Algorithm 3 column pass alone (aca.cu), for the sharded selection (shard.cu)
// Row chunks of the pass over an m x n matrix: returns RC and sets *chunk (rows per chunk).
int aca_cols_chunks(int num_sms, int64_t m, int64_t n, cur_dtype dt, int64_t* chunk);
// part[rc * n + j] = sum over the rows of chunk rc of a_ij * q_i (dot != 0) or a_ij^2 (dot = 0):
// an FP64 value for FP64 data, a double-float pair (two floats) otherwise; q as q64 (FP64
// data) or qh + ql (two floats). Nothing runs while *stop != 0.
cur_status aca_cols_partials(const cur_mat* A, int dot, const double* q64, const float* qh,
                             const float* ql, void* part, int RC, int64_t chunk, const int* stop,
                             cudaStream_t st);
