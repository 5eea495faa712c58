// CUR assembly (Section 1.1: C = A(:,J), U = A(I,J)^dagger, R = A(I,:)) and the
// residual of the cross (Theorem 1's Chebyshev norm max|A - CUR| and the relative
// Frobenius error of Section 3.1).
//
// The residual reads A exactly once. W = U R (r x n) is formed first in FP64 and
// rounded to the arithmetic type; each CTA then owns a 128-row panel, keeps its
// C rows in shared memory and walks the panel's column tiles: E = A - C W on a
// 128 x 128 tile, with |E| max, sum E^2 and sum A^2 folded in the epilogue.

#include <algorithm>
#include <climits>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace curk {

constexpr double kEpsR = 2.220446049250313e-16;

template <typename TA>
__global__ void gather_C_k(const TA* __restrict__ A, int64_t m, int64_t n, int64_t ld,
                           const int32_t* __restrict__ J, int r, TA* __restrict__ C, int* status) {
    const int64_t total = m * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int64_t j = J[e - i * r];
        if (j < 0 || j >= n) { set_status(status, CUR_ERR_ARG); C[e] = A[0]; continue; }
        C[e] = A[i * ld + j];
    }
}

template <typename TA>
__global__ void gather_R_k(const TA* __restrict__ A, int64_t m, int64_t n, int64_t ld,
                           const int32_t* __restrict__ I, int r, TA* __restrict__ R, int* status) {
    const int64_t total = (int64_t)r * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / n, j = e - k * n;
        const int64_t i = I[k];
        if (i < 0 || i >= m) { set_status(status, CUR_ERR_ARG); R[e] = A[0]; continue; }
        R[e] = A[i * ld + j];
    }
}

// One CTA: M = A(I,J) in FP64, LU with partial pivoting, inverse, rcond; if
// rcond < 1e-13 (or M is singular) the pseudo-inverse from a one-sided Jacobi SVD
// (round-robin pair order, one warp per pair) with cutoff r eps s_max.
// work: 3 r^2 doubles (global scratch).
template <typename TA>
__global__ void __launch_bounds__(256) assemble_inv_k(const TA* __restrict__ A, int64_t m,
                                                      int64_t n, int64_t ld,
                                                      const int32_t* __restrict__ I,
                                                      const int32_t* __restrict__ J, int r,
                                                      double* __restrict__ U, double* rcond_out,
                                                      double* __restrict__ work, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, nt = blockDim.x;
    double* M = reinterpret_cast<double*>(smem_raw);  // r x r, inverted in place
    double* colk = M + r * r;
    int* piv = reinterpret_cast<int*>(colk + r);
    double* X = work + r * r;    // r x r (Jacobi V)
    double* M0 = work + 2 * r * r;
    __shared__ int s_bad;
    __shared__ double s_max, s_n1, s_ni;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int e = tid; e < r * r; e += nt) {
        const int a = e / r, b = e - a * r;
        const int64_t i = I[a], j = J[b];
        double x = 0.0;
        if (i < 0 || i >= m || j < 0 || j >= n) s_bad = 1;
        else x = to_d(A[i * ld + j]);
        if (!isfinite(x)) s_bad = 2;
        M[e] = x;
        M0[e] = x;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            set_status(status, s_bad == 2 ? CUR_ERR_NONFINITE : CUR_ERR_ARG);
            *rcond_out = 0.0;
        }
        return;
    }
    {
        // max |M| and the 1-norm (largest column sum), one column per thread
        double mx = 0.0, cs = 0.0;
        for (int c = tid; c < r; c += nt) {
            double s = 0.0;
            for (int a = 0; a < r; ++a) { mx = fmax(mx, fabs(M[a * r + c])); s += fabs(M[a * r + c]); }
            cs = fmax(cs, s);
        }
        mx = block_max(mx);
        cs = block_max(cs);
        if (tid == 0) { s_max = mx; s_n1 = cs; }
        __syncthreads();
    }
    const int sing = gj_inverse(M, r, colk, piv, (double)r * kEpsR * s_max, nullptr);
    bool use_pinv = sing != 0;
    if (!use_pinv) {
        double cs = 0.0;
        for (int c = tid; c < r; c += nt) {
            double s = 0.0;
            for (int a = 0; a < r; ++a) s += fabs(M[a * r + c]);
            cs = fmax(cs, s);
        }
        cs = block_max(cs);
        if (tid == 0) {
            s_ni = cs;
            *rcond_out = 1.0 / (s_n1 * cs);
        }
        __syncthreads();
        use_pinv = !(1.0 / (s_n1 * s_ni) >= 1e-13);
        if (!use_pinv) {
            for (int e = tid; e < r * r; e += nt) U[e] = M[e];
            return;
        }
    } else if (tid == 0) {
        *rcond_out = 0.0;
    }
    // ---- pseudo-inverse: one-sided Jacobi on the columns of M0, V accumulates rotations
    double* Aj = M0;
    double* V = X;
    for (int e = tid; e < r * r; e += nt) V[e] = ((e / r) == (e % r)) ? 1.0 : 0.0;
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int rr = (r % 2 == 0) ? r : r + 1;  // round-robin over an even count (phantom column)
    __shared__ int s_rot;
    for (int sweep = 0; sweep < 80; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int step = 0; step < rr - 1; ++step) {
            for (int pr = warp; pr < rr / 2; pr += nw) {
                // pairs (a, b) of the round-robin schedule: position 0 fixed, others rotate
                int a, b;
                {
                    const int i1 = pr, i2 = rr - 1 - pr;
                    auto pos = [&](int i) { return i == 0 ? 0 : 1 + (i - 1 + step) % (rr - 1); };
                    a = pos(i1);
                    b = pos(i2);
                }
                if (a > b) { const int t = a; a = b; b = t; }
                if (b >= r) continue;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < r; i += 32) {
                    const double x = Aj[i * r + a], y = Aj[i * r + b];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                if (lane == 0) s_rot = 1;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = lane; i < r; i += 32) {
                    const double x = Aj[i * r + a], y = Aj[i * r + b];
                    Aj[i * r + a] = c * x - s * y;
                    Aj[i * r + b] = s * x + c * y;
                    const double vx = V[i * r + a], vy = V[i * r + b];
                    V[i * r + a] = c * vx - s * vy;
                    V[i * r + b] = s * vx + c * vy;
                }
            }
            __syncthreads();
        }
        const int rot = s_rot;
        __syncthreads();
        if (!rot) break;
    }
    // singular values, cutoff, U = V diag(1/s) Uhat^T with Uhat = Aj / s
    __shared__ double sv[128];
    for (int k = tid; k < r; k += nt) {
        double s = 0.0;
        for (int i = 0; i < r; ++i) s = fma(Aj[i * r + k], Aj[i * r + k], s);
        sv[k] = sqrt(s);
    }
    __syncthreads();
    if (tid == 0) {
        double smax = 0.0;
        for (int k = 0; k < r; ++k) smax = fmax(smax, sv[k]);
        s_max = (double)r * kEpsR * smax;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e - i * r;
        double s = 0.0;
        for (int k = 0; k < r; ++k)
            if (sv[k] > s_max) s += V[i * r + k] * (Aj[j * r + k] / sv[k]) / sv[k];
        U[e] = s;
    }
}

// W = U R (r x n) in FP64, rounded to TW. One thread per column.
template <typename TA, typename TW>
__global__ void __launch_bounds__(256) residual_w_k(const double* __restrict__ U,
                                                   const TA* __restrict__ R, int r, int64_t n,
                                                   TW* __restrict__ W) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* Us = reinterpret_cast<double*>(smem_raw);
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) Us[e] = U[e];
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double rc[128];
        for (int l = 0; l < r; ++l) rc[l] = to_d(R[(int64_t)l * n + j]);
        for (int k = 0; k < r; ++k) {
            double s = 0.0;
            for (int l = 0; l < r; ++l) s = fma(Us[k * r + l], rc[l], s);
            W[(int64_t)k * n + j] = (TW)s;
        }
    }
}

// N consecutive elements from 16-byte aligned memory as 16-byte loads.
template <typename T, int N>
__device__ __forceinline__ void ld_vec(const T* p, T (&x)[N]) {
    static_assert((N * sizeof(T)) % 16 == 0, "16-byte multiple");
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int c = 0; c < (int)(N * sizeof(T) / 16); ++c) {
        const uint4 v = q[c];
        memcpy(&x[c * (16 / sizeof(T))], &v, 16);
    }
}

// Residual tiles. TM x TN outputs per thread, 16 x 16 threads, tile (16 TM) x (16 TN).
// Grid: (panels, segments); CTA (p, s) takes rows [p*BM, p*BM+BM) and column tiles
// s, s + segs, ... Partials per CTA: max|E|, sum E^2, sum A^2, non-finite flag.
template <typename TA, typename TW, int TM, int TN>
__global__ void __launch_bounds__(256, 2) residual_k(const TA* __restrict__ A, int64_t m, int64_t n,
                                                  int64_t ld, const TA* __restrict__ C,
                                                  const TW* __restrict__ W, int r,
                                                  double* __restrict__ part, int vec) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TW* Ct = reinterpret_cast<TW*>(smem_raw);  // r x BM (transposed C panel)
    TW* Ws = Ct + (size_t)r * BM;              // r x BN
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * BM;
    const int segs = gridDim.y;
    for (int e = threadIdx.x; e < BM * r; e += blockDim.x) {
        const int k = e / BM, i = e - k * BM;
        Ct[k * BM + i] = (r0 + i < m) ? (TW)to_d(C[(r0 + i) * r + k]) : (TW)0;
    }
    double mx = 0.0, se = 0.0, sa = 0.0;
    int bad = 0;
    const int64_t ntile = (n + BN - 1) / BN;
    for (int64_t tn = blockIdx.y; tn < ntile; tn += segs) {
        const int64_t c0 = tn * BN;
        __syncthreads();
        for (int e = threadIdx.x; e < BN * r; e += blockDim.x) {
            const int k = e / BN, j = e - k * BN;
            Ws[k * BN + j] = (c0 + j < n) ? W[(int64_t)k * n + c0 + j] : (TW)0;
        }
        __syncthreads();
        TW acc[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) acc[a][b] = (TW)0;
#pragma unroll 4
        for (int k = 0; k < r; ++k) {
            TW x[TM], y[TN];
            ld_vec<TW, TM>(Ct + k * BM + ty * TM, x);
            // column pairs 2 tx + 32 b (+1): a half-warp reads 128 contiguous bytes per load
#pragma unroll
            for (int b = 0; b < TN / 2; ++b) {
                const TW* q = Ws + k * BN + 2 * tx + 32 * b;
                y[2 * b] = q[0];
                y[2 * b + 1] = q[1];
            }
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
        }
        TW tmx = (TW)0, tse = (TW)0, tsa = (TW)0;
#pragma unroll
        for (int a = 0; a < TM; ++a) {
            const int64_t i = r0 + ty * TM + a;
            if (i >= m) continue;
            const TA* arow = A + i * ld + c0;
            TA araw[TN];
#pragma unroll
            for (int b = 0; b < TN; ++b) {
                const int64_t cc = 2 * tx + 32 * (b >> 1) + (b & 1);
                araw[b] = (c0 + cc < n) ? arow[cc] : arow[0];
            }
#pragma unroll
            for (int b = 0; b < TN; ++b) {
                if (c0 + 2 * tx + 32 * (b >> 1) + (b & 1) >= n) continue;
                const TW av = (TW)to_d(araw[b]);
                const TW e = av - acc[a][b];
                if (!(fabs(e) <= (TW)INFINITY)) bad = 1;
                tmx = fmax(tmx, fabs(e));
                tse = fma(e, e, tse);
                tsa = fma(av, av, tsa);
            }
        }
        mx = fmax(mx, (double)tmx);
        se += (double)tse;
        sa += (double)tsa;
    }
    // CTA reduction
    __shared__ double rmx[8], rse[8], rsa[8];
    __shared__ int rbad;
    if (threadIdx.x == 0) rbad = 0;
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        se += __shfl_xor_sync(0xffffffffu, se, o);
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    __syncthreads();
    if (bad) rbad = 1;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { rmx[warp] = mx; rse[warp] = se; rsa[warp] = sa; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a1 = 0.0, a2 = 0.0, a3 = 0.0;
        for (int w = 0; w < 8; ++w) { a1 = fmax(a1, rmx[w]); a2 += rse[w]; a3 += rsa[w]; }
        const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        part[cta * 4 + 0] = a1;
        part[cta * 4 + 1] = a2;
        part[cta * 4 + 2] = a3;
        part[cta * 4 + 3] = rbad ? 1.0 : 0.0;
    }
}

// Combines the per-CTA partials in a fixed order (one CTA of 256 threads).
__global__ void residual_final_k(const double* part, int64_t nparts, double* cheb, double* fro,
                                 int* status, double* sums = nullptr) {
    __shared__ double s1[256], s2[256], s3[256];
    __shared__ int sb[256];
    const int tid = threadIdx.x;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int bad = 0;
    for (int64_t c = tid; c < nparts; c += blockDim.x) {
        a1 = fmax(a1, part[c * 4 + 0]);
        a2 += part[c * 4 + 1];
        a3 += part[c * 4 + 2];
        bad |= part[c * 4 + 3] != 0.0;
    }
    s1[tid] = a1; s2[tid] = a2; s3[tid] = a3; sb[tid] = bad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) {
            s1[tid] = fmax(s1[tid], s1[tid + o]);
            s2[tid] += s2[tid + o];
            s3[tid] += s3[tid + o];
            sb[tid] |= sb[tid + o];
        }
        __syncthreads();
    }
    if (tid != 0) return;
    a1 = s1[0];
    if (sb[0]) {
        set_status(status, CUR_ERR_NONFINITE);
        a1 = NAN;
    }
    *cheb = a1;
    if (fro) *fro = s3[0] > 0.0 ? sqrt(s2[0] / s3[0]) : 0.0;
    if (sums) { sums[0] = s2[0]; sums[1] = s3[0]; }
}

static inline unsigned nb(int64_t n, int t = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535));
}

template <typename TA>
static cur_status assemble_t(cur_handle* h, const cur_mat* Am, const int32_t* I, const int32_t* J,
                             int r, void* C_out, double* U_out, void* R_out, double* rcond_out,
                             Arena& ar, cudaStream_t st) {
    const TA* A = static_cast<const TA*>(Am->data);
    double* work = ar.get<double>((size_t)3 * r * r);
    if (!ar.ok) return CUR_ERR_NOMEM;
    if (C_out) {
        gather_C_k<TA><<<nb(Am->rows * r), 256, 0, st>>>(A, Am->rows, Am->cols, Am->ld, J, r, static_cast<TA*>(C_out), h->status);
        CUR_CK(cudaGetLastError());
    note_launch();
    }
    if (R_out) {
        gather_R_k<TA><<<nb(Am->cols * r), 256, 0, st>>>(A, Am->rows, Am->cols, Am->ld, I, r, static_cast<TA*>(R_out), h->status);
        CUR_CK(cudaGetLastError());
    note_launch();
    }
    const size_t sm = ((size_t)r * r + r) * sizeof(double) + (size_t)r * sizeof(int) + 64;
    CUR_TRY(smem_attr((const void*)assemble_inv_k<TA>, sm));
    assemble_inv_k<TA><<<1, 256, sm, st>>>(A, Am->rows, Am->cols, Am->ld, I, J, r, U_out, rcond_out, work, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

template <typename TA, typename TW, int TM, int TN>
static cur_status residual_t(cur_handle* h, const cur_mat* Am, const void* C, const double* U,
                             const void* R, int r, double* cheb, double* fro, Arena& ar,
                             cudaStream_t st, double* sums) {
    const int64_t m = Am->rows, n = Am->cols;
    TW* W = ar.get<TW>((size_t)r * n);
    constexpr int BM = 16 * TM, BN = 16 * TN;
    const int64_t panels = (m + BM - 1) / BM;
    const int64_t ntile = (n + BN - 1) / BN;
    const size_t sm = (size_t)r * (BM + BN) * sizeof(TW);
    CUR_TRY(smem_attr((const void*)residual_k<TA, TW, TM, TN>, sm));
    int occ = 1;
    CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, residual_k<TA, TW, TM, TN>, 256, sm));
    const int64_t want = (int64_t)h->num_sms * std::max(1, occ) * 4;
    int64_t segs = std::max<int64_t>(1, std::min<int64_t>(ntile, (want + panels - 1) / panels));
    segs = std::min<int64_t>(segs, 65535);
    if (panels > 2147483647LL) return CUR_ERR_ARG;
    double* part = ar.get<double>((size_t)panels * segs * 4);
    if (!ar.ok) return CUR_ERR_NOMEM;
    const size_t smw = (size_t)r * r * sizeof(double);
    CUR_TRY(smem_attr((const void*)residual_w_k<TA, TW>, smw));
    residual_w_k<TA, TW><<<nb(n), 256, smw, st>>>(U, static_cast<const TA*>(R), r, n, W);
    CUR_CK(cudaGetLastError());
    note_launch();
    const uintptr_t base = reinterpret_cast<uintptr_t>(Am->data);
    const int vec = (base % 16 == 0) && ((size_t)Am->ld * sizeof(TA)) % 16 == 0 ? 1 : 0;
    residual_k<TA, TW, TM, TN><<<dim3((unsigned)panels, (unsigned)segs), 256, sm, st>>>(
        static_cast<const TA*>(Am->data), m, n, Am->ld, static_cast<const TA*>(C), W, r, part, vec);
    CUR_CK(cudaGetLastError());
    note_launch();
    residual_final_k<<<1, 256, 0, st>>>(part, panels * segs, cheb, fro, h->status, sums);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

}  // namespace curk

cur_status assemble_impl(cur_handle* h, const cur_mat* A, const int32_t* I, const int32_t* J,
                         int r, void* C_out, double* U_out, void* R_out, double* rcond_out,
                         Arena& ar, cudaStream_t st) {
    switch (A->dtype) {
        case CUR_F64: return curk::assemble_t<double>(h, A, I, J, r, C_out, U_out, R_out, rcond_out, ar, st);
        case CUR_F32: return curk::assemble_t<float>(h, A, I, J, r, C_out, U_out, R_out, rcond_out, ar, st);
        case CUR_BF16: return curk::assemble_t<__nv_bfloat16>(h, A, I, J, r, C_out, U_out, R_out, rcond_out, ar, st);
    }
    return CUR_ERR_ARG;
}

cur_status residual_impl(cur_handle* h, const cur_mat* A, const void* C, const double* U,
                         const void* R, int r, double* cheb_out, double* fro_out, Arena& ar,
                         cudaStream_t st, double* sums_out) {
    if (A->dtype == CUR_F32) {
        // tensor-core (tcgen05) form where it applies; CUR_ERR_ARG means it does not
        const size_t mark = ar.off;
        const cur_status s = residual_tc_impl(h, A, C, U, R, r, cheb_out, fro_out, ar, st, sums_out);
        if (s != CUR_ERR_ARG) return s;
        ar.off = mark;
        ar.ok = true;
    }
    switch (A->dtype) {
        case CUR_F64: return curk::residual_t<double, double, 4, 4>(h, A, C, U, R, r, cheb_out, fro_out, ar, st, sums_out);
        case CUR_F32: return curk::residual_t<float, float, 8, 8>(h, A, C, U, R, r, cheb_out, fro_out, ar, st, sums_out);
        case CUR_BF16: return curk::residual_t<__nv_bfloat16, float, 8, 8>(h, A, C, U, R, r, cheb_out, fro_out, ar, st, sums_out);
    }
    return CUR_ERR_ARG;
}

// ---------------------------------------------------------------- allocation-free residual
//
// cur_residual_cheb needs a handle, and a handle allocates its workspace with cudaMalloc.
// Some callers cannot do that where they need the residual: code that runs after its
// device memory has been handed to a pool or allocator of its own, or a loop that must
// not hit cudaMalloc's implicit device synchronisation. For them
// cur_residual_cheb_noalloc keeps its scratch (W = U R and the per-CTA partial sums) in
// one array compiled into this library. The array's device address is looked up once
// per device, on the first call made with that device current, and kept until the
// process exits; a device reset after that first call is not supported (the kept
// address would no longer be valid).

#include <mutex>

namespace curk {
constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // 16 MiB on every device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
}  // namespace curk

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256] = {};

// Device address of the scratch array on the current device (set up on first use).
static cur_status noalloc_scratch(void** out) {
    int dev = 0;
    CUR_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return CUR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, curk::g_noalloc_scratch) != cudaSuccess || !p) return CUR_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return CUR_OK;
}

template <typename TA, typename TW, int TM, int TN>
static cur_status residual_noalloc_t(const cur_mat* Am, const void* C, const double* U,
                                     const void* R, int r, double* cheb, double* fro,
                                     cudaStream_t st) {
    using namespace curk;
    const int64_t m = Am->rows, n = Am->cols;
    constexpr int BM = 16 * TM, BN = 16 * TN;
    const int64_t panels = (m + BM - 1) / BM;
    const int64_t ntile = (n + BN - 1) / BN;
    if (panels > 65535LL * 32768LL) return CUR_ERR_ARG;
    int dev = 0, sms = 0;
    CUR_CK(cudaGetDevice(&dev));
    CUR_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t sm = (size_t)r * (BM + BN) * sizeof(TW);
    CUR_TRY(smem_attr((const void*)residual_k<TA, TW, TM, TN>, sm));
    int occ = 1;
    CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, residual_k<TA, TW, TM, TN>, 256, sm));
    const int64_t want = (int64_t)sms * std::max(1, occ) * 4;
    int64_t segs = std::max<int64_t>(1, std::min<int64_t>(ntile, (want + panels - 1) / panels));
    segs = std::min<int64_t>(segs, 65535);
    if (panels > 2147483647LL) return CUR_ERR_ARG;
    // scratch: W (r x n) then the partials (4 doubles per CTA), 256-byte aligned
    const size_t w_bytes = ((size_t)r * n * sizeof(TW) + 255) / 256 * 256;
    const size_t p_bytes = (size_t)panels * segs * 4 * sizeof(double);
    if (w_bytes + p_bytes > kNoallocScratchBytes) return CUR_ERR_NOMEM;
    void* base = nullptr;
    CUR_TRY(noalloc_scratch(&base));
    TW* W = static_cast<TW*>(base);
    double* part = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + w_bytes);
    const size_t smw = (size_t)r * r * sizeof(double);
    CUR_TRY(smem_attr((const void*)residual_w_k<TA, TW>, smw));
    residual_w_k<TA, TW><<<nb(n), 256, smw, st>>>(U, static_cast<const TA*>(R), r, n, W);
    CUR_CK(cudaGetLastError());
    const uintptr_t abase = reinterpret_cast<uintptr_t>(Am->data);
    const int vec = (abase % 16 == 0) && ((size_t)Am->ld * sizeof(TA)) % 16 == 0 ? 1 : 0;
    residual_k<TA, TW, TM, TN><<<dim3((unsigned)panels, (unsigned)segs), 256, sm, st>>>(
        static_cast<const TA*>(Am->data), m, n, Am->ld, static_cast<const TA*>(C), W, r, part, vec);
    CUR_CK(cudaGetLastError());
    residual_final_k<<<1, 256, 0, st>>>(part, panels * segs, cheb, fro, nullptr);
    CUR_CK(cudaGetLastError());
    return CUR_OK;
}

extern "C" cur_status cur_residual_cheb_noalloc(const cur_mat* A, const void* C, const double* U,
                                                const void* R, int32_t r, double* cheb_out,
                                                double* fro_rel_out, cudaStream_t stream) {
    if (!A || !A->data || A->rows < 1 || A->cols < 1 || A->ld < A->cols) return CUR_ERR_ARG;
    if (!C || !U || !R || !cheb_out || r < 1 || r > 128) return CUR_ERR_ARG;
    switch (A->dtype) {
        case CUR_F64: return residual_noalloc_t<double, double, 4, 4>(A, C, U, R, r, cheb_out, fro_rel_out, stream);
        case CUR_F32: return residual_noalloc_t<float, float, 8, 8>(A, C, U, R, r, cheb_out, fro_rel_out, stream);
        case CUR_BF16: return residual_noalloc_t<__nv_bfloat16, float, 8, 8>(A, C, U, R, r, cheb_out, fro_rel_out, stream);
    }
    return CUR_ERR_ARG;
}
