// Algorithm 1 of the paper (Section 1.3): adaptive cross approximation with full
// pivoting, the sequential baseline that Algorithm 3 is set against.
//
// Step k picks (i, j) = argmax |R_k(i,j)| over the whole residual (ties: smallest
// row-major index) and eliminates R_{k+1} = R_k - R_k(:,j) R_k(i,:) / R_k(i,j). The
// residual is kept explicitly in a caller-owned m x n buffer (FP32 for FP32/BF16 data,
// FP64 for FP64 data), so a step is one streaming pass that reads and writes R once:
//   a1_update : R <- R - u v^T with u = R_k(:,j)/R_k(i,j), v = R_k(i,:), row i and
//               column j set to zero (exactly zero in exact arithmetic), and each
//               CTA's (max |R_{k+1}|, lowest index) in the same pass
//   a1_pick   : one CTA combines the CTA maxima in fixed order, applies the rounding
//               stop (|pivot| <= max(m,n) eps max|A|), records I, J and the pivot
//   a1_extract: u and v of the new pivot for the next update
// a1_init copies A into R and finds the first pivot's candidates. All steps are
// enqueued without host synchronisation; after a stop the remaining kernels return
// at once.

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace curk {

struct A1State {
    double amax;      // max |A|
    double piv;       // pivot value of the current step
    long long idx;    // its row-major index i n + j
    int stop;         // 1 once the loop has ended
};

constexpr int kA1Threads = 256;

// (value, index): larger value wins, then the smaller index
__device__ __forceinline__ void a1_better(double v, long long i, double& bv, long long& bi) {
    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

__device__ __forceinline__ void a1_block_argmax(double& bv, long long& bi, double* pv, long long* pi) {
    __shared__ double sv[32];
    __shared__ long long si[32];
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        a1_better(v2, i2, bv, bi);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sv[w] = bv; si[w] = bi; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        bv = lane < nw ? sv[lane] : -1.0;
        bi = lane < nw ? si[lane] : LLONG_MAX;
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            a1_better(v2, i2, bv, bi);
        }
        if (lane == 0) { pv[blockIdx.x] = bv; pi[blockIdx.x] = bi; }
    }
}

template <typename TR> struct Vec;
template <> struct Vec<float> { using T = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using T = double2; static constexpr int W = 2; };

template <typename TR>
__device__ __forceinline__ void vload(const TR* p, TR* x) {
    if constexpr (sizeof(TR) == 4) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
    } else {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        x[0] = t.x; x[1] = t.y;
    }
}
template <typename TR>
__device__ __forceinline__ void vstore(TR* p, const TR* x) {
    if constexpr (sizeof(TR) == 4) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(x[0], x[1], x[2], x[3]));
    } else {
        __stcs(reinterpret_cast<double2*>(p), make_double2(x[0], x[1]));
    }
}

template <typename TR, typename TA>
__device__ __forceinline__ TR a1_conv(TA x) {
    if constexpr (sizeof(TR) == 8) return to_d(x); else return to_f(x);
}

// R = A (converted), CTA argmax of |A|; non-finite data stops the loop. The scan
// compares in the residual's type; a thread visits increasing indices, so a strict
// '>' keeps the lowest index of its equal maxima.
template <typename TA, typename TR>
__global__ void __launch_bounds__(kA1Threads) a1_init(const TA* __restrict__ A, int64_t m, int64_t n,
                                                      int64_t ld, TR* __restrict__ R, double* pv,
                                                      long long* pi, int* status) {
    TR bv = (TR)-1;
    long long bi = LLONG_MAX;
    int bad = 0;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = e0 / n, c = e0 - i * n;
    const int64_t di = step / n, dc = step - di * n;
    for (; i < m;) {
        const TR x = a1_conv<TR>(A[i * ld + c]);
        const TR ax = fabs(x);
        if (!(ax <= (TR)INFINITY)) bad = 1;
        R[i * n + c] = x;
        if (ax > bv) { bv = ax; bi = i * n + c; }
        c += dc;
        i += di;
        if (c >= n) { c -= n; ++i; }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, CUR_ERR_NONFINITE);
    double dv = (double)bv;
    a1_block_argmax(dv, bi, pv, pi);
}

// One step's pivot: combine the CTA maxima, stop test, record (I, J, pivot).
template <typename TR>
__global__ void __launch_bounds__(1024) a1_pick(const TR* __restrict__ R, int64_t m, int64_t n, int k, int r,
                                                const double* pv, const long long* pi, int nparts,
                                                A1State* s, int32_t* I, int32_t* J, double* piv_out,
                                                int* status) {
    if (s->stop) return;
    double bv = -1.0;
    long long bi = LLONG_MAX;
    for (int c = threadIdx.x; c < nparts; c += blockDim.x) a1_better(pv[c], pi[c], bv, bi);
    __shared__ double sv;
    __shared__ long long si;
    // fixed-order combine: warp shuffles, then the warps' results
    {
        __shared__ double wv[32];
        __shared__ long long wi[32];
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            a1_better(v2, i2, bv, bi);
        }
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) { wv[w] = bv; wi[w] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = -1.0;
            long long ix = LLONG_MAX;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a1_better(wv[q], wi[q], v, ix);
            sv = v;
            si = ix;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (k == 0) s->amax = sv;
    const double tol = (double)max(m, n) * 2.220446049250313e-16 * s->amax;
    const int64_t ix = si;
    const double p = (ix >= 0 && ix < m * n) ? (double)R[ix] : 0.0;
    if (*status == CUR_ERR_NONFINITE || !(fabs(p) > tol) || !(sv > tol)) {
        s->stop = 1;
        for (int q = k; q < r; ++q) { I[q] = -1; J[q] = -1; if (piv_out) piv_out[q] = 0.0; }
        if (*status != CUR_ERR_NONFINITE) set_status(status, CUR_WARN_RANK);
        return;
    }
    I[k] = (int32_t)(ix / n);
    J[k] = (int32_t)(ix - (ix / n) * n);
    if (piv_out) piv_out[k] = p;
    s->piv = p;
    s->idx = ix;
}

// u = R(:, j) / R(i, j) and v = R(i, :) of the current pivot.
template <typename TR>
__global__ void a1_extract(const TR* __restrict__ R, int64_t m, int64_t n, const A1State* s,
                           TR* __restrict__ u, TR* __restrict__ v) {
    if (s->stop) return;
    const int64_t i0 = s->idx / n, j0 = s->idx - i0 * n;
    const TR p = (TR)s->piv;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m + n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < m) u[e] = R[e * n + j0] / p;
        else v[e - m] = R[i0 * n + (e - m)];
    }
}

// R <- R - u v^T with row i0 and column j0 zeroed; CTA argmax of the new |R|.
// VEC: W consecutive elements per access (n % W == 0), else 1. A thread takes U
// element groups a grid stride apart per iteration and issues their U loads before
// any store, so each SM keeps U x 16 bytes per thread in flight; the walk over
// (row, group) advances incrementally (no division in the loop). Within a thread the
// indices increase, so a strict '>' keeps the lowest index of equal maxima.
template <typename TR, bool VEC>
__global__ void __launch_bounds__(kA1Threads) a1_update(TR* __restrict__ R, int64_t m, int64_t n,
                                                        const A1State* s, const TR* __restrict__ u,
                                                        const TR* __restrict__ v, double* pv,
                                                        long long* pi) {
    if (s->stop) return;
    constexpr int W = VEC ? Vec<TR>::W : 1;
    constexpr int U = 4;
    const int64_t i0 = s->idx / n, j0 = s->idx - i0 * n;
    const int64_t ng = n / W;   // groups per row
    TR bv = (TR)-1;
    long long bi = LLONG_MAX;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = g0 / ng, cg = g0 - i * ng;
    const int64_t di = step / ng, dcg = step - di * ng;
    while (i < m) {
        int64_t ri[U], rc[U];
        TR x[U][W];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            ri[q] = i;
            rc[q] = cg * W;
            if (i < m) {
                const TR* p = R + i * n + cg * W;
                if constexpr (VEC) vload<TR>(p, x[q]); else x[q][0] = __ldcs(p);
            }
            cg += dcg;
            i += di;
            if (cg >= ng) { cg -= ng; ++i; }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (ri[q] >= m) break;
            const TR ui = u[ri[q]];
            const bool zrow = ri[q] == i0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int64_t c = rc[q] + w;
                TR y = fma(-ui, v[c], x[q][w]);
                if (zrow || c == j0) y = (TR)0;
                x[q][w] = y;
                const TR ay = fabs(y);
                if (ay > bv) { bv = ay; bi = ri[q] * n + c; }
            }
            TR* p = R + ri[q] * n + rc[q];
            if constexpr (VEC) vstore<TR>(p, x[q]); else __stcs(p, x[q][0]);
        }
    }
    double dv = (double)bv;
    a1_block_argmax(dv, bi, pv, pi);
}

template <typename TA, typename TR>
static cur_status aca_full_t(cur_handle* h, const cur_mat* A, int r, TR* R, int32_t* I, int32_t* J,
                             double* piv, Arena& ar, cudaStream_t st) {
    const int64_t m = A->rows, n = A->cols;
    // one wave of the update pass: every CTA resident (no tail wave)
    int occ = 0;
    CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, a1_update<TR, true>, kA1Threads, 0));
    const int G = h->num_sms * std::max(1, occ);
    double* pv = ar.get<double>(G);
    long long* pi = ar.get<long long>(G);
    TR* u = ar.get<TR>((size_t)m);
    TR* v = ar.get<TR>((size_t)n);
    A1State* s = ar.get<A1State>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_CK(cudaMemsetAsync(s, 0, sizeof(A1State), st));
    a1_init<TA, TR><<<G, kA1Threads, 0, st>>>(static_cast<const TA*>(A->data), m, n, A->ld, R, pv, pi,
                                              h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    constexpr int W = Vec<TR>::W;
    const bool vec = n % W == 0 && (reinterpret_cast<uintptr_t>(R) % 16) == 0;
    const unsigned ge = (unsigned)std::min<int64_t>((m + n + 255) / 256, (int64_t)h->num_sms * 4);
    for (int k = 0; k < r; ++k) {
        a1_pick<TR><<<1, 1024, 0, st>>>(R, m, n, k, r, pv, pi, G, s, I, J, piv, h->status);
        CUR_CK(cudaGetLastError());
        a1_extract<TR><<<ge, 256, 0, st>>>(R, m, n, s, u, v);
        CUR_CK(cudaGetLastError());
        const bool ev = h->prof && h->prof_n < 4096;
        if (ev) CUR_CK(cudaEventRecord(h->prof_ev[2 * h->prof_n], st));
        if (vec) a1_update<TR, true><<<G, kA1Threads, 0, st>>>(R, m, n, s, u, v, pv, pi);
        else a1_update<TR, false><<<G, kA1Threads, 0, st>>>(R, m, n, s, u, v, pv, pi);
        CUR_CK(cudaGetLastError());
        if (ev) CUR_CK(cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], st));
        if (ev) ++h->prof_n;
        note_launch(3);
    }
    return CUR_OK;
}

}  // namespace curk

cur_status aca_full_impl(cur_handle* h, const cur_mat* A, int r, void* R, int32_t* I, int32_t* J,
                         double* piv, Arena& ar, cudaStream_t st) {
    switch (A->dtype) {
        case CUR_F64:
            return curk::aca_full_t<double, double>(h, A, r, static_cast<double*>(R), I, J, piv, ar, st);
        case CUR_F32:
            return curk::aca_full_t<float, float>(h, A, r, static_cast<float*>(R), I, J, piv, ar, st);
        case CUR_BF16:
            return curk::aca_full_t<__nv_bfloat16, float>(h, A, r, static_cast<float*>(R), I, J, piv, ar, st);
    }
    return CUR_ERR_ARG;
}
