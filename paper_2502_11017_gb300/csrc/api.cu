// C ABI of libcur: handle, workspace, argument checks and the cross driver.

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>

#include "common.cuh"
#include "internal.h"

cur_status pad_indices_dev(int32_t* idx, const int32_t* count, int r, int64_t size, cudaStream_t st);

namespace curk {

__global__ void iota_k(int32_t* x, int r) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) x[k] = k;
}

__global__ void set_status_k(int* st, int code) {
    if (threadIdx.x == 0 && blockIdx.x == 0) set_status(st, code);
}

// One CTA waits at a group barrier for a second CTA that is never launched: the
// bounded wait must run out, record CUR_ERR_TIMEOUT and return.
__global__ void selftest_wait_k(unsigned* ctr, int* status, long long limit) {
    group_barrier(ctr, 2u, status, limit);
}

}  // namespace curk

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cur_status smem_attr(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    CUR_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[std::make_pair(dev, fn)];
    if (bytes <= cur) return CUR_OK;
    CUR_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
    return CUR_OK;
}

cur_status launch_coop(const void* fn, dim3 grid, dim3 block, void** args, size_t smem,
                       cudaStream_t st) {
    CUR_CK(cudaLaunchCooperativeKernel(fn, grid, block, args, smem, st));
    return CUR_OK;
}

static bool mat_ok(const cur_mat* A) {
    if (!A || !A->data) return false;
    if (A->rows < 1 || A->cols < 1 || A->ld < A->cols) return false;
    if (A->dtype != CUR_F64 && A->dtype != CUR_F32 && A->dtype != CUR_BF16) return false;
    return true;
}

static cur_status peek_status(cur_handle* h, cudaStream_t st, int* out) {
    int* hs = reinterpret_cast<int*>(h->host_stage);
    CUR_CK(cudaMemcpyAsync(hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUR_CK(cudaStreamSynchronize(st));
    *out = hs[0];
    return CUR_OK;
}

extern "C" {

cur_opts cur_default_opts(void) {
    cur_opts o;
    o.delta = 1e-2;
    o.max_swaps = 0;
    o.nblocks = 1;
    o.flags = CUR_FLAG_POLISH;
    return o;
}

const char* cur_status_string(cur_status s) {
    switch (s) {
        case CUR_OK: return "ok";
        case CUR_ERR_ARG: return "invalid argument";
        case CUR_ERR_SINGULAR: return "singular submatrix";
        case CUR_ERR_NONFINITE: return "non-finite value in the data";
        case CUR_ERR_NOCONV: return "maxvol did not converge within max_swaps";
        case CUR_ERR_TIMEOUT: return "device-side wait timed out";
        case CUR_ERR_NOMEM: return "workspace too small";
        case CUR_ERR_CUDA: return "CUDA runtime error";
        case CUR_WARN_RANK: return "residual exhausted before r picks";
    }
    return "unknown status";
}

size_t cur_workspace_size(int64_t m, int64_t n, int32_t r, cur_dtype dtype) {
    if (m < 1 || n < 1 || r < 1) return 0;
    const size_t cs = dtype == CUR_F64 ? 8 : 4;
    const size_t mx = (size_t)std::max(m, n);
    const size_t R = (size_t)r;
    size_t b = (size_t)64 << 20;                              // tables, keys, small arrays
    b += 8 * ((size_t)4864 * 128 + 8 * mx);                   // Algorithm 3 partials and vectors
    b += 8 * R * mx * 2;                                      // W and Q of Algorithm 3
    b += cs * R * (size_t)(m + n) * 4;                        // bases, B, merge unions
    b += cs * R * mx;                                         // B in global memory for large r
    b += 8 * R * R * (size_t)((m + n) / R + 16) * 2;          // M^-1 per problem (two types)
    b += 8 * R * (size_t)n + 8 * 4 * (size_t)(m / 64 + 1) * 64;  // residual W and partials
    b += sketch_workspace_size(256, m, n);                    // sketch partials (<= 256 SMs)
    return b;
}

cur_status cur_create(cur_handle** hp, size_t workspace_bytes) {
    if (!hp) return CUR_ERR_ARG;
    *hp = nullptr;
    cur_handle* h = new (std::nothrow) cur_handle();
    if (!h) return CUR_ERR_NOMEM;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return CUR_ERR_CUDA;
    }
    h->ws_bytes = workspace_bytes;
    if (workspace_bytes && cudaMalloc(&h->ws, workspace_bytes) != cudaSuccess) {
        delete h;
        return CUR_ERR_NOMEM;
    }
    h->host_stage_bytes = (size_t)4 << 20;
    // two device words: the status word, then the count of cycle refactorisations
    if (cudaMalloc(&h->status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&h->host_stage, h->host_stage_bytes) != cudaSuccess ||
        cudaMemset(h->status, 0, 2 * sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->stage_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&h->tune_ev[0]) != cudaSuccess || cudaEventCreate(&h->tune_ev[1]) != cudaSuccess) {
        if (h->ws) cudaFree(h->ws);
        if (h->status) cudaFree(h->status);
        if (h->host_stage) cudaFreeHost(h->host_stage);
        if (h->stage_ev) cudaEventDestroy(h->stage_ev);
        for (auto& e : h->tune_ev)
            if (e) cudaEventDestroy(e);
        delete h;
        return CUR_ERR_CUDA;
    }
    *hp = h;
    return CUR_OK;
}

cur_status cur_destroy(cur_handle* h) {
    if (!h) return CUR_ERR_ARG;
    cudaDeviceSynchronize();
    for (auto& e : h->prof_ev)
        if (e) cudaEventDestroy(e);
    if (h->ws) cudaFree(h->ws);
    if (h->status) cudaFree(h->status);
    if (h->host_stage) cudaFreeHost(h->host_stage);
    if (h->stage_ev) cudaEventDestroy(h->stage_ev);
    for (auto& e : h->tune_ev)
        if (e) cudaEventDestroy(e);
    delete h;
    return CUR_OK;
}

cur_status cur_prof_enable(cur_handle* h, int on) {
    if (!h) return CUR_ERR_ARG;
    if (on && !h->prof_ev[0])
        for (auto& e : h->prof_ev) CUR_CK(cudaEventCreate(&e));
    h->prof = on ? 1 : 0;
    h->prof_n = 0;
    return CUR_OK;
}

cur_status cur_prof_read(cur_handle* h, cudaStream_t st, double* pass_ms, int32_t* pass_launches,
                         int64_t* kernel_launches) {
    if (!h) return CUR_ERR_ARG;
    CUR_CK(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (int k = 0; k < h->prof_n; ++k) {
        float ms = 0.f;
        CUR_CK(cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]));
        tot += ms;
    }
    if (pass_ms) *pass_ms = tot;
    if (pass_launches) *pass_launches = h->prof_n;
    const long long nl = g_launches.exchange(0);
    if (kernel_launches) *kernel_launches = nl;
    h->prof_n = 0;
    return CUR_OK;
}

cur_status cur_prof_refactors(cur_handle* h, cudaStream_t st, int64_t* count) {
    if (!h || !count) return CUR_ERR_ARG;
    CUR_CK(cudaStreamSynchronize(st));
    int v = 0;
    CUR_CK(cudaMemcpy(&v, h->status + 1, sizeof(int), cudaMemcpyDeviceToHost));
    CUR_CK(cudaMemset(h->status + 1, 0, sizeof(int)));
    *count = v;
    return CUR_OK;
}

cur_status cur_selftest_wait_timeout(cur_handle* h, cudaStream_t st) {
    if (!h) return CUR_ERR_ARG;
    Arena ar = h->arena();
    unsigned* ctr = ar.get<unsigned>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_CK(cudaMemsetAsync(ctr, 0, sizeof(unsigned), st));
    curk::selftest_wait_k<<<1, 32, 0, st>>>(ctr, h->status, 100000000LL);   // ~50 ms
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_sync_status(cur_handle* h, cudaStream_t st) {
    if (!h) return CUR_ERR_ARG;
    int v = 0;
    CUR_TRY(peek_status(h, st, &v));
    CUR_CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    CUR_CK(cudaStreamSynchronize(st));
    return (cur_status)v;
}

cur_status cur_aca_select(cur_handle* h, const cur_mat* A, int axis, int32_t r, int32_t nblocks,
                          int32_t* idx_out, cudaStream_t st) {
    if (!h || !mat_ok(A) || !idx_out || (axis != 0 && axis != 1) || nblocks < 1) return CUR_ERR_ARG;
    const int64_t size = axis == 1 ? A->cols : A->rows;
    if (r < 1 || r > 128 || r > size || nblocks > size) return CUR_ERR_ARG;
    Arena ar = h->arena();
    int32_t* cnt = ar.get<int32_t>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    return aca_select_full(h, A, axis, r, idx_out, cnt, ar, st);
}

size_t cur_batch_workspace_size(const cur_batch_item* items, int32_t count) {
    if (!items || count < 1) return 0;
    int rs = 1;
    for (int t = 0; t < count; ++t) rs = std::max(rs, (int)items[t].r);
    size_t b = (size_t)64 << 20;
    const size_t minv = ((size_t)rs * rs + 1) * 8 + (size_t)rs * 64;   // per stage problem
    for (int t = 0; t < count; ++t) {
        const cur_batch_item& it = items[t];
        if (it.r < 1 || it.rows < 1 || it.cols < 1) return 0;
        b += (size_t)(it.rows + it.cols) * it.r * 4 * 4;             // bases, unions, B
        b += minv * (size_t)(2 * (std::max(1, it.b_r) + std::max(1, it.b_c)) + 4);
        b += 512;
    }
    b += (size_t)std::min(count, 512) * 2 * 64 * 4096 * sizeof(float);   // Algorithm 3's Q slices
    b += (size_t)std::min(count, 512) * 64 * 1024 * sizeof(double);      // and its W slices
    return b;
}

cur_status cur_cross_batched(cur_handle* h, const void* data, cur_dtype dtype, const cur_batch_item* items,
                             int32_t count, const cur_opts* opts, int32_t* IJ_out, cur_cross_info* info_out,
                             cudaStream_t st) {
    if (!h || !data || !items || !IJ_out || count < 1 || count > 65535) return CUR_ERR_ARG;
    if (dtype != CUR_F32) return CUR_ERR_ARG;
    for (int t = 0; t < count; ++t) {
        const cur_batch_item& it = items[t];
        if (it.r < 1 || it.r > 64 || it.rows > 4096 || it.cols > 1024 || it.ld < it.cols || it.offset < 0) return CUR_ERR_ARG;
        if (it.r >= std::min(it.rows, it.cols) || it.b_r < 1 || it.b_c < 1) return CUR_ERR_ARG;
        if (it.rows / it.b_r < it.r || it.cols / it.b_c < it.r) return CUR_ERR_ARG;
    }
    cur_opts o = opts ? *opts : cur_default_opts();
    if (!(o.delta >= 0.0)) return CUR_ERR_ARG;
    Arena ar = h->arena();
    return cross_batched_impl(h, static_cast<const float*>(data), items, count, &o, IJ_out, info_out, ar, st);
}

cur_status cur_aca_full(cur_handle* h, const cur_mat* A, int32_t r, void* R_work, int32_t* I_out,
                        int32_t* J_out, double* piv_out, cudaStream_t st) {
    if (!h || !mat_ok(A) || !R_work || !I_out || !J_out) return CUR_ERR_ARG;
    if (r < 1 || r > std::min(A->rows, A->cols)) return CUR_ERR_ARG;
    Arena ar = h->arena();
    return aca_full_impl(h, A, r, R_work, I_out, J_out, piv_out, ar, st);
}

// NOCONV of a row or column selection goes to the status word.
__global__ void noconv_status_k(const MvDevResult* res, int* hstatus) {
    if (threadIdx.x == 0 && res->status == CUR_ERR_NOCONV) curk::set_status(hstatus, CUR_ERR_NOCONV);
}

static cur_status rows_common(cur_handle* h, const cur_mat* A, const int32_t* idx, int32_t r,
                              const cur_opts* opts, int32_t* out, double* logvol_out,
                              int32_t* swaps_out, bool cols, cudaStream_t st) {
    if (!h || !mat_ok(A) || !idx || !out) return CUR_ERR_ARG;
    const cur_opts o = opts ? *opts : cur_default_opts();
    const int64_t p = cols ? A->cols : A->rows;
    const int64_t other = cols ? A->rows : A->cols;
    if (r < 1 || r > 128 || r > other || o.nblocks < 1 || p / o.nblocks < r) return CUR_ERR_ARG;
    if (!(o.delta >= 0.0)) return CUR_ERR_ARG;
    Arena ar = h->arena();
    const cur_dtype cdt = A->dtype == CUR_F64 ? CUR_F64 : CUR_F32;
    void* basis = ar.take((size_t)p * r * compute_size(cdt));
    MvDevResult* res = ar.get<MvDevResult>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    if (cols) CUR_TRY(gather_rows_t_compute(A, idx, r, basis, st));
    else CUR_TRY(gather_cols_compute(A, idx, r, basis, st));
    CUR_TRY(maxvol_basis_rows(h, cdt, basis, p, r, &o, out, logvol_out, swaps_out, res, ar, st));
    noconv_status_k<<<1, 32, 0, st>>>(res, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_maxvol_rows(cur_handle* h, const cur_mat* A, const int32_t* J, int32_t r,
                           const cur_opts* opts, int32_t* I_out, double* logvol_out,
                           int32_t* swaps_out, cudaStream_t st) {
    return rows_common(h, A, J, r, opts, I_out, logvol_out, swaps_out, false, st);
}

cur_status cur_maxvol_cols(cur_handle* h, const cur_mat* A, const int32_t* I, int32_t r,
                           const cur_opts* opts, int32_t* J_out, double* logvol_out,
                           int32_t* swaps_out, cudaStream_t st) {
    return rows_common(h, A, I, r, opts, J_out, logvol_out, swaps_out, true, st);
}

cur_status cur_merge(cur_handle* h, const cur_mat* basis, const int32_t* cand, int32_t nsets,
                     int32_t r, const cur_opts* opts, int32_t* out, cudaStream_t st) {
    if (!h || !mat_ok(basis) || !cand || !out || nsets < 1) return CUR_ERR_ARG;
    if (basis->dtype == CUR_BF16) return CUR_ERR_ARG;
    if (r < 1 || r > 128 || basis->cols != r || basis->ld != r || basis->rows < r) return CUR_ERR_ARG;
    const cur_opts o = opts ? *opts : cur_default_opts();
    Arena ar = h->arena();
    int* acc = ar.get<int>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_CK(cudaMemsetAsync(acc, 0, sizeof(int), st));
    return merge_level(h, basis->dtype, basis->data, basis->rows, r, cand, nsets, &o, out, acc, ar, st);
}

cur_status cur_assemble(cur_handle* h, const cur_mat* A, const int32_t* I, const int32_t* J,
                        int32_t r, void* C_out, double* U_out, void* R_out, double* rcond_out,
                        cudaStream_t st) {
    if (!h || !mat_ok(A) || !I || !J || !U_out || !rcond_out) return CUR_ERR_ARG;
    if (r < 1 || r > 128 || r > A->rows || r > A->cols) return CUR_ERR_ARG;
    Arena ar = h->arena();
    return assemble_impl(h, A, I, J, r, C_out, U_out, R_out, rcond_out, ar, st);
}

cur_status cur_residual_cheb(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                             const void* R, int32_t r, double* cheb_out, double* fro_rel_out,
                             cudaStream_t st) {
    if (!h || !mat_ok(A) || !C || !U || !R || !cheb_out) return CUR_ERR_ARG;
    if (r < 1 || r > 128) return CUR_ERR_ARG;
    Arena ar = h->arena();
    return residual_impl(h, A, C, U, R, r, cheb_out, fro_rel_out, ar, st);
}

cur_status cur_residual_parts(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                              const void* R, int32_t r, double* parts_out, cudaStream_t st) {
    if (!h || !mat_ok(A) || !C || !U || !R || !parts_out) return CUR_ERR_ARG;
    if (r < 1 || r > 128) return CUR_ERR_ARG;
    Arena ar = h->arena();
    return residual_impl(h, A, C, U, R, r, parts_out, nullptr, ar, st, parts_out + 1);
}

cur_status cur_merge_pair(cur_handle* h, const cur_mat* rows, const int32_t* ids, const cur_opts* opts,
                          int32_t* ids_out, void* rows_out, int32_t* swaps_out, cudaStream_t st) {
    if (!h || !mat_ok(rows) || !ids || !ids_out || !rows_out) return CUR_ERR_ARG;
    if (rows->dtype == CUR_BF16) return CUR_ERR_ARG;
    const int64_t r = rows->cols;
    if (r < 1 || r > 128 || rows->ld != r || rows->rows != 2 * r) return CUR_ERR_ARG;
    const cur_opts o = opts ? *opts : cur_default_opts();
    Arena ar = h->arena();
    return merge_pair_impl(h, rows->dtype, rows->data, ids, (int)r, &o, ids_out, rows_out, swaps_out, ar, st);
}

cur_status cur_gather_cols(cur_handle* h, const cur_mat* A, const int32_t* J, int32_t r, void* C_out,
                           cudaStream_t st) {
    if (!h || !mat_ok(A) || !J || !C_out || r < 1 || r > A->cols) return CUR_ERR_ARG;
    return gather_cols_compute(A, J, r, C_out, st);
}

cur_status cur_cross(cur_handle* h, const cur_mat* A, int32_t r, int32_t b_r, int32_t b_c,
                     const cur_opts* opts, int32_t* I_out, int32_t* J_out,
                     cur_cross_info* info_out, cudaStream_t st) {
    if (!h || !mat_ok(A) || !I_out || !J_out) return CUR_ERR_ARG;
    const int64_t m = A->rows, n = A->cols;
    if (r < 1 || r > 128 || r >= std::min(m, n)) return CUR_ERR_ARG;
    if (b_r < 1 || b_c < 1 || m / b_r < r || n / b_c < r) return CUR_ERR_ARG;
    cur_opts o = opts ? *opts : cur_default_opts();
    if (!(o.delta >= 0.0)) return CUR_ERR_ARG;
    const int max_sweeps = 8;
    Arena ar = h->arena();
    const cur_dtype cdt = A->dtype == CUR_F64 ? CUR_F64 : CUR_F32;
    const size_t cs = compute_size(cdt);
    int32_t* J0 = ar.get<int32_t>(r);
    int32_t* cnt = ar.get<int32_t>(1);
    int32_t* I = ar.get<int32_t>(r);
    int32_t* J = ar.get<int32_t>(r);
    double* lv = ar.get<double>(1);
    void* Cb = ar.take((size_t)m * r * cs);
    void* Rb = ar.take((size_t)n * r * cs);
    // M^-1 of the last row stage (Mr = C(I,:)^-1) and column stage (Mc = R^T(J,:)^-1 =
    // (A(I,J)^T)^-1); each stage of a sweep starts from the other's inverse, transposed.
    double* Mr = ar.get<double>((size_t)minv_stride(r));
    double* Mc = ar.get<double>((size_t)minv_stride(r));
    double* lvr = ar.get<double>(1);
    CrossCtl* ctl = ar.get<CrossCtl>(1);
    MvDevResult* res = ar.get<MvDevResult>(2);
    if (!ar.ok) return CUR_ERR_NOMEM;
    // index sets start as 0..r-1, so that every gather reads inside A even when a stage idles
    curk::iota_k<<<1, 128, 0, st>>>(I, r);
    curk::iota_k<<<1, 128, 0, st>>>(J, r);
    CUR_CK(cudaGetLastError());
    note_launch(2);

    // J0: Algorithm 3 on the columns; an error it records makes everything after it idle
    CUR_TRY(aca_select_full(h, A, 1, r, J0, cnt, ar, st));
    CUR_TRY(cross_begin(ctl, h->status, true, st));
    CUR_TRY(pad_indices_dev(J0, cnt, r, n, st));

    // sweep 1: blockwise rows on A(:,J0), then blockwise columns on A(I,:)^T
    cur_opts orow = o;
    orow.nblocks = b_r;
    cur_opts ocol = o;
    ocol.nblocks = b_c;
    CUR_TRY(gather_cols_compute(A, J0, r, Cb, st, &ctl->abort));
    CUR_TRY(maxvol_basis_rows(h, cdt, Cb, m, r, &orow, I, nullptr, nullptr, &res[0], ar, st, nullptr, &ctl->abort));
    CUR_TRY(gather_rows_t_compute(A, I, r, Rb, st, &ctl->abort));
    CUR_TRY(maxvol_basis_rows(h, cdt, Rb, n, r, &ocol, J, lv, nullptr, &res[1], ar, st, Mc, &ctl->abort));
    CUR_TRY(cross_sweep_one(ctl, &res[0], &res[1], st));
    // sweeps 2 .. 8: global maxvol on the rows, then on the columns, until one swaps nothing
    CUR_TRY(cross_sweeps(h, A, r, &o, 2, max_sweeps, false, I, J, Cb, Rb, Mr, Mc, lvr, lv, ctl, ar, st));
    return cross_end(h, A, r, false, I, J, Rb, lv, ctl, cnt, I_out, J_out, info_out, ar, st);
}

}  // extern "C"
