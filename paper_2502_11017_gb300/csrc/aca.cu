// Algorithm 3 (Blockwise Adaptive Cross Approximation, Section 2.2 of the paper)
// on a full m x n matrix, GB300 form.
//
// The paper keeps an explicit residual and, each round, (1) computes the squared
// norm of every row/column of every block, (2) reduces the block maxima to one
// pivot, (3) broadcasts the pivot vector v and (4) projects every block,
// R <- R - v (v^T R) / ||v||^2. In exact arithmetic this is column-pivoted
// Gram-Schmidt, so the same picks follow from an implicit residual:
//   nu_j = ||a_j||^2 - sum_k (q_k^T a_j)^2,   q_k = orthonormal basis of the picks,
// which needs one read of A per round (w = A^T q) instead of a read and a write.
// Each round is
//   pass   : w partials = A^T q_t over row chunks   (HBM stream, Dot2 accuracy)
//   pivot  : one cooperative kernel: reduce partials, W(t,:) = w, nu -= w^2,
//            argmax over unpicked (lowest index on ties), then the new direction
//            v = a_p - Q W(:,p), re-orthogonalised once (CGS2), q = v / ||v||.
// For axis 0 the roles of rows and columns swap (w = A q, row-dot products).

#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace curk {

enum { kNorm = 0, kDot = 1 };

// Threads of the pivot CTA (one per SM).
constexpr int kPivotThreads = 256;

template <typename TA>
using AccOf = typename std::conditional<std::is_same<TA, double>::value, DotD, Dot2>::type;

// Four consecutive elements, 16-byte (8-byte for BF16) vector loads, streaming.
__device__ __forceinline__ void load4(const float* p, float v[4]) {
    float4 x = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
    double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float v[4]) {
    uint2 x = __ldcs(reinterpret_cast<const uint2*>(p));
    v[0] = __uint_as_float(x.x << 16);
    v[1] = __uint_as_float(x.x & 0xffff0000u);
    v[2] = __uint_as_float(x.y << 16);
    v[3] = __uint_as_float(x.y & 0xffff0000u);
}
template <typename TA, typename TV>
__device__ __forceinline__ void load4_guard(const TA* row, int64_t col, int64_t n, TV v[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (col + k < n) ? (TV)to_d(row[col + k]) : (TV)0;
}

// Columns per lane of the column pass: 16 bytes of A per lane and row (8 for BF16).
template <typename TA> struct ColsPerLane { static constexpr int v = sizeof(TA) == 2 ? 8 : 4; };

__device__ __forceinline__ void loadc(const float* p, float* v) { load4(p, v); }
__device__ __forceinline__ void loadc(const double* p, double* v) { load4(p, v); }
__device__ __forceinline__ void loadc(const __nv_bfloat16* p, float* v) {
    const uint4 x = __ldcs(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
template <int CPL, typename TA, typename TV>
__device__ __forceinline__ void loadc_guard(const TA* row, int64_t col, int64_t n, TV* v) {
#pragma unroll
    for (int k = 0; k < CPL; ++k) v[k] = (col + k < n) ? (TV)to_d(row[col + k]) : (TV)0;
}

template <typename TA> struct ValT { using type = float; };
template <> struct ValT<double> { using type = double; };

__device__ __forceinline__ void acc_add(DotD& a, double x, int mode, double q, float, float) {
    if (mode == kNorm) a.add_sq(x); else a.add(x, q);
}
__device__ __forceinline__ void acc_add(Dot2& a, float x, int mode, double, float qh, float ql) {
    if (mode == kNorm) a.add_sq(x); else a.add(x, qh, ql);
}

// Partial sums travel as FP64 for FP64 data and as double-float pairs otherwise.
template <typename TA>
using PartT = typename std::conditional<std::is_same<TA, double>::value, double, df64>::type;

__device__ __forceinline__ df64 part_value(const Dot2& a) { return fast_two_sum(a.s, a.c); }
__device__ __forceinline__ double part_value(const DotD& a) { return a.s; }
__device__ __forceinline__ df64 part_add(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ double part_add(double a, double b) { return a + b; }
__device__ __forceinline__ double part_to_d(df64 a) { return df_to_d(a); }
__device__ __forceinline__ double part_to_d(double a) { return a; }
__device__ __forceinline__ df64 part_zero(df64) { return df64{0.f, 0.f}; }
__device__ __forceinline__ double part_zero(double) { return 0.0; }
__device__ __forceinline__ df64 shfl_xor(df64 v, int o) {
    return df64{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = part_add(v, shfl_xor(v, o));
    return v;
}

// part[rc * n + j] = sum over rows i of chunk rc of a_ij * q_i (kDot) or a_ij^2 (kNorm).
// grid = (ceil(n / (32 CPL)), RC), block = 256 (8 warps). Warp w takes rows r0 + w,
// r0 + w + 8, ...; lane l takes the CPL columns 32 CPL blockIdx.x + CPL l .. (CPL = 4,
// or 8 for BF16: 16 bytes per lane and row either way).
template <typename TA, int MODE, bool VEC>
__global__ void __launch_bounds__(256) aca_cols_pass(const TA* __restrict__ A, int64_t m, int64_t n,
                                                     int64_t ld, int64_t chunk,
                                                     const double* __restrict__ q64,
                                                     const float* __restrict__ qh,
                                                     const float* __restrict__ ql,
                                                     PartT<TA>* __restrict__ part,
                                                     const int* __restrict__ stop) {
    using V = typename ValT<TA>::type;
    using PT = PartT<TA>;
    constexpr int CPL = ColsPerLane<TA>::v, TW = 32 * CPL;
    __shared__ PT red[8][TW];
    if (*stop) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t col = (int64_t)blockIdx.x * TW + lane * CPL;
    const int64_t r0 = (int64_t)blockIdx.y * chunk;
    const int64_t r1 = min(r0 + chunk, m);
    const bool full = VEC && (col + CPL - 1 < n);
    AccOf<TA> acc[CPL];
    int64_t i = r0 + warp;
    if constexpr (std::is_same<TA, __nv_bfloat16>::value && MODE == kDot) {
        // BF16: about 12 FP32 operations per 2-byte element, so the sums of four rows take
        // long enough that the next four rows' loads are issued before them (same order of
        // summation as the loop below)
        if (full && i + 24 < r1) {
            uint4 xr[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xr[u] = __ldcs(reinterpret_cast<const uint4*>(A + (i + 8 * u) * ld + col));
            while (true) {
                const int64_t inext = i + 32;
                const bool more = inext + 24 < r1;
                uint4 xn[4];
                if (more) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        xn[u] = __ldcs(reinterpret_cast<const uint4*>(A + (inext + 8 * u) * ld + col));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float h = qh[i + 8 * u], l = ql[i + 8 * u];
                    const uint32_t w[4] = {xr[u].x, xr[u].y, xr[u].z, xr[u].w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc_add(acc[2 * k], __uint_as_float(w[k] << 16), MODE, 0.0, h, l);
                        acc_add(acc[2 * k + 1], __uint_as_float(w[k] & 0xffff0000u), MODE, 0.0, h, l);
                    }
                }
                i = inext;
                if (!more) break;
#pragma unroll
                for (int u = 0; u < 4; ++u) xr[u] = xn[u];
            }
        }
    }
    for (; i + 24 < r1; i += 32) {
        V x[4][CPL];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const TA* row = A + (i + 8 * u) * ld;
            if (full) loadc(row + col, x[u]); else loadc_guard<CPL>(row, col, n, x[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            double qd = 0.0; float h = 0.f, l = 0.f;
            if (MODE == kDot) {
                if (std::is_same<TA, double>::value) qd = q64[i + 8 * u];
                else { h = qh[i + 8 * u]; l = ql[i + 8 * u]; }
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc_add(acc[c], x[u][c], MODE, qd, h, l);
        }
    }
    for (; i < r1; i += 8) {
        V x[CPL];
        const TA* row = A + i * ld;
        if (full) loadc(row + col, x); else loadc_guard<CPL>(row, col, n, x);
        double qd = 0.0; float h = 0.f, l = 0.f;
        if (MODE == kDot) {
            if (std::is_same<TA, double>::value) qd = q64[i];
            else { h = qh[i]; l = ql[i]; }
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc_add(acc[c], x[c], MODE, qd, h, l);
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) red[warp][lane * CPL + c] = part_value(acc[c]);
    __syncthreads();
    if (threadIdx.x < TW) {
        const int64_t j = (int64_t)blockIdx.x * TW + threadIdx.x;
        if (j < n) {
            PT s0 = part_add(red[0][threadIdx.x], red[1][threadIdx.x]);
            PT s1 = part_add(red[2][threadIdx.x], red[3][threadIdx.x]);
            PT s2 = part_add(red[4][threadIdx.x], red[5][threadIdx.x]);
            PT s3 = part_add(red[6][threadIdx.x], red[7][threadIdx.x]);
            part[(int64_t)blockIdx.y * n + j] = part_add(part_add(s0, s1), part_add(s2, s3));
        }
    }
}

// out[i] = sum_j a_ij * q_j (kDot) or a_ij^2 (kNorm); one warp per row.
template <typename TA, int MODE, bool VEC>
__global__ void __launch_bounds__(256) aca_rows_pass(const TA* __restrict__ A, int64_t m, int64_t n,
                                                     int64_t ld, const double* __restrict__ q64,
                                                     const float* __restrict__ qh,
                                                     const float* __restrict__ ql,
                                                     PartT<TA>* __restrict__ out,
                                                     const int* __restrict__ stop) {
    using V = typename ValT<TA>::type;
    if (*stop) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t row = (int64_t)blockIdx.x * 8 + warp; row < m; row += (int64_t)gridDim.x * 8) {
        const TA* a = A + row * ld;
        AccOf<TA> acc;
        for (int64_t j = (int64_t)lane * 4; j < n; j += 128) {
            V x[4];
            if (VEC && j + 3 < n) load4(a + j, x); else load4_guard(a, j, n, x);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t jj = j + c;
                double qd = 0.0; float h = 0.f, l = 0.f;
                if (MODE == kDot && jj < n) {
                    if (std::is_same<TA, double>::value) qd = q64[jj];
                    else { h = qh[jj]; l = ql[jj]; }
                }
                acc_add(acc, x[c], MODE, qd, h, l);
            }
        }
        const PartT<TA> s = warp_sum_t(part_value(acc));
        if (lane == 0) out[row] = s;
    }
}

struct AcaParams {
    const void* A;
    int64_t m, n, ld;
    int axis, r;
    int64_t nsel, len;     // candidates (n for columns), vector length (m for columns)
    const void* part;      // RC x nsel partials (PartT)
    int RC;
    double* nu;
    unsigned char* mask;
    void* W;               // r x nsel: W(k, j) = q_k^T a_j (PartT)
    double* Q;             // r x len (column k contiguous): orthonormal directions; for
                           // FP32/BF16 data the same bytes hold them as double-float
                           // (r x len high words, then r x len low words)
    double* q64;
    float* qh;
    float* ql;
    double* v;             // len (double-float pairs for FP32/BF16 data)
    double* red1;          // G x r (double-float pairs for FP32/BF16 data)
    double* red2;          // G
    double* redf;          // G
    double* keyv;          // G
    long long* keyi;       // G
    unsigned* bar;
    double* frob2;
    int* count;
    int* stop;
    int* idx_out;
    int* status;
};

template <typename TA>
__device__ __forceinline__ double pivot_elem(const AcaParams& P, int64_t i, int64_t p) {
    const TA* A = static_cast<const TA*>(P.A);
    return P.axis == 1 ? to_d(A[i * P.ld + p]) : to_d(A[p * P.ld + i]);
}

// acc_a -= sum_kk Q(kk, ia) s(kk) and acc_b likewise for row ib. The Q values of eight
// directions are loaded before any arithmetic (32 loads in flight per thread), the next
// eight while the current ones are used (the sum is a chain over kk, so each batch would
// otherwise wait for its loads), and two interleaved chains per row (even and odd kk)
// keep four dependency chains in flight.
constexpr int kQB = 8;
__device__ __forceinline__ void qsub_load(const float* Qh, const float* Ql, int64_t len, int k, int k0,
                                          int64_t ia, int64_t ibb, float* ha, float* la, float* hb, float* lb) {
#pragma unroll
    for (int u = 0; u < kQB; ++u) {
        const int64_t o = (int64_t)min(k0 + u, k - 1) * len;   // past k: a valid row, not used
        ha[u] = Qh[o + ia];
        la[u] = Ql[o + ia];
        hb[u] = Qh[o + ibb];
        lb[u] = Ql[o + ibb];
    }
}
__device__ __forceinline__ void qsub_pair(const float* Qh, const float* Ql, int64_t len, int k,
                                          const df64* s, int64_t ia, int64_t ib, bool vb,
                                          df64& acc_a, df64& acc_b) {
    df64 a1{0.f, 0.f}, b1{0.f, 0.f};
    const int64_t ibb = vb ? ib : ia;
    float ha[kQB], la[kQB], hb[kQB], lb[kQB];
    qsub_load(Qh, Ql, len, k, 0, ia, ibb, ha, la, hb, lb);
    for (int k0 = 0; k0 < k; k0 += kQB) {
        float nha[kQB], nla[kQB], nhb[kQB], nlb[kQB];
        if (k0 + kQB < k) qsub_load(Qh, Ql, len, k, k0 + kQB, ia, ibb, nha, nla, nhb, nlb);
#pragma unroll
        for (int u = 0; u < kQB; u += 2) {
            const df64 s0 = k0 + u < k ? s[k0 + u] : df64{0.f, 0.f};
            const df64 s1 = k0 + u + 1 < k ? s[k0 + u + 1] : df64{0.f, 0.f};
            acc_a = df_sub(acc_a, df_mul(df64{ha[u], la[u]}, s0));
            acc_b = df_sub(acc_b, df_mul(df64{hb[u], lb[u]}, s0));
            a1 = df_sub(a1, df_mul(df64{ha[u + 1], la[u + 1]}, s1));
            b1 = df_sub(b1, df_mul(df64{hb[u + 1], lb[u + 1]}, s1));
        }
#pragma unroll
        for (int u = 0; u < kQB; ++u) {
            ha[u] = nha[u];
            la[u] = nla[u];
            hb[u] = nhb[u];
            lb[u] = nlb[u];
        }
    }
    acc_a = df_add(acc_a, a1);
    acc_b = df_add(acc_b, b1);
}

// One round of Algorithm 3 after its pass. `part` holds A^T q_t (t >= 0) or the
// squared norms (t = -1). Picks index k = t + 1; with `build`, also forms q_k.
// Cooperative launch; grid G <= co-resident CTAs, block 256. Two group barriers: after
// the partial sums of the pass (the pick), and after the partial dots of the first
// Gram-Schmidt projection. The barrier's counter is not reset between rounds: this
// round's barriers wait for bb + G and bb + 2G arrivals (bb = 2 G (t + 1)). A barrier that
// runs out of time stops the selection, so that no later round waits on a count that
// cannot be reached.
template <typename TA>
__global__ void __launch_bounds__(kPivotThreads) aca_pivot(AcaParams P, int t, int build, unsigned bb) {
    using PT = PartT<TA>;
    __shared__ double s_w[128];
    __shared__ PT s_q[4][64];
    __shared__ double s_tot;
    if (*P.stop) return;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    auto barrier = [&](unsigned n) {
        if (group_barrier(P.bar, bb + n * (unsigned)G, P.status)) return true;
        if (threadIdx.x == 0) *P.stop = 1;
        return false;
    };
    const int k = t + 1;
    const PT* part = static_cast<const PT*>(P.part);
    PT* W = static_cast<PT*>(P.W);

    // P0: reduce partials, downdate squared norms, local argmax over unpicked. The RC
    // partials of each column are summed by 4 threads in fixed order (deterministic).
    const int64_t j0 = P.nsel * g / G, j1 = P.nsel * (g + 1) / G;
    unsigned long long bk = dkey(-INFINITY);
    long long bi = LLONG_MAX;
    double fs = 0.0;
    int bad = 0;
    {
        const int lane64 = tid & 63, q4 = tid >> 6;   // 64 columns x 4 quarter-sums per pass (first 256 threads)
        for (int64_t jb = j0; jb < j1; jb += 64) {
            const int64_t j = jb + lane64;
            PT w0 = part_zero(PT{}), w1 = part_zero(PT{});
            if (j < j1 && q4 < 4) {
                const int rc0 = P.RC * q4 / 4, rc1 = P.RC * (q4 + 1) / 4;
                const PT* src = part + j;
                int rc = rc0;
                // even offsets into w0, odd into w1; up to kP0B loads in flight at a time
                constexpr int kP0B = 10;
                while (rc + 1 < rc1) {
                    const int nb = min(kP0B, (rc1 - rc) & ~1);
                    PT x[kP0B];
#pragma unroll
                    for (int i = 0; i < kP0B; ++i)
                        if (i < nb) x[i] = src[(int64_t)(rc + i) * P.nsel];
#pragma unroll
                    for (int i = 0; i < kP0B; i += 2)
                        if (i < nb) {
                            w0 = part_add(w0, x[i]);
                            w1 = part_add(w1, x[i + 1]);
                        }
                    rc += nb;
                }
                if (rc < rc1) w0 = part_add(w0, src[(int64_t)rc * P.nsel]);
            }
            if (q4 < 4) s_q[q4][lane64] = part_add(w0, w1);
            __syncthreads();
            if (q4 == 0 && j < j1) {
                const PT w = part_add(part_add(s_q[0][lane64], s_q[1][lane64]),
                                      part_add(s_q[2][lane64], s_q[3][lane64]));
                const double wd = part_to_d(w);
                double nu;
                if (t < 0) {
                    nu = wd;
                    fs += wd;
                    if (!isfinite(wd)) bad = 1;
                } else {
                    W[(int64_t)t * P.nsel + j] = w;
                    nu = P.nu[j] - wd * wd;
                }
                P.nu[j] = nu;
                const unsigned long long kj = dkey(nu);
                if (!P.mask[j] && better_key(kj, (long long)j, bk, bi)) { bk = kj; bi = j; }
            }
            __syncthreads();
        }
    }
    block_argmax_key(bk, bi);
    bad = __syncthreads_or(bad);
    if (t < 0) fs = block_sum(fs);
    if (tid == 0) {
        P.keyv[g] = dkey_value(bk);
        P.keyi[g] = bad ? -2LL : bi;
        P.redf[g] = fs;
    }
    if (!barrier(1u)) return;

    // P1: the global pick, identical in every CTA.
    unsigned long long pk = dkey(-INFINITY);
    long long pi = LLONG_MAX;
    int anybad = 0;
    for (int gg = tid; gg < G; gg += nt) {
        const long long ki = P.keyi[gg];
        const unsigned long long kg = dkey(P.keyv[gg]);
        if (ki == -2LL) anybad = 1;
        else if (better_key(kg, ki, pk, pi)) { pk = kg; pi = ki; }
    }
    anybad = __syncthreads_or(anybad);
    block_argmax_key(pk, pi);
    if (anybad) {
        if (g == 0 && tid == 0) { *P.stop = 1; set_status(P.status, CUR_ERR_NONFINITE); }
        return;
    }
    if (t < 0 && g == 0 && tid < 32) {
        const double f2 = warp_sum_strided(P.redf, G);
        if (tid == 0) *P.frob2 = f2;
    }
    if (pi == LLONG_MAX || pi < 0) {
        if (g == 0 && tid == 0) { *P.stop = 1; set_status(P.status, CUR_WARN_RANK); }
        return;
    }
    const int64_t p = pi;
    const int64_t i0 = P.len * g / G, i1 = P.len * (g + 1) / G;
    const int64_t len = P.len;
    const int r = P.r;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;

    if constexpr (!std::is_same<TA, double>::value) {
        // Double-float form (FP32/BF16 data): the Gram-Schmidt steps on the FP32 pipes;
        // Q, v and the partial dot products are stored as (high, low) FP32 pairs.
        float* Qh = reinterpret_cast<float*>(P.Q);
        float* Ql = Qh + (int64_t)r * len;
        float* vh = reinterpret_cast<float*>(P.v);
        float* vl = vh + len;
        df64* red1 = reinterpret_cast<df64*>(P.red1);
        __shared__ df64 s_df[128];
        __shared__ df64 s_wred[kPivotThreads / 32];
        __shared__ df64 s_inv;
        for (int kk = tid; kk < k; kk += nt) s_df[kk] = W[(int64_t)kk * P.nsel + p];
        __syncthreads();
        // P1b: v = a_p - Q W(:,p), two rows per thread, and this CTA's part of ||v||^2
        {
            df64 nv{0.f, 0.f};
            for (int64_t ia = i0 + tid; ia < i1; ia += 2 * nt) {
                const int64_t ib = ia + nt;
                const bool vb = ib < i1;
                df64 acc_a{(float)pivot_elem<TA>(P, ia, p), 0.f};
                df64 acc_b{vb ? (float)pivot_elem<TA>(P, ib, p) : 0.f, 0.f};
                qsub_pair(Qh, Ql, len, k, s_df, ia, ib, vb, acc_a, acc_b);
                vh[ia] = acc_a.h;
                vl[ia] = acc_a.l;
                nv = df_add(nv, df_mul(acc_a, acc_a));
                if (vb) {
                    vh[ib] = acc_b.h;
                    vl[ib] = acc_b.l;
                    nv = df_add(nv, df_mul(acc_b, acc_b));
                }
            }
            nv = warp_sum_t(nv);
            if (lane == 0) s_wred[warp] = nv;
            __syncthreads();
            if (tid == 0) {
                df64 sv{0.f, 0.f};
                for (int w = 0; w < nw; ++w) sv = df_add(sv, s_wred[w]);
                P.red2[g] = df_to_d(sv);
            }
        }
        // partial dots Q^T v: one warp per pair of directions; per iteration a lane loads
        // four rows of v and of both directions before the arithmetic (24 loads in flight)
        for (int kk = 2 * warp; kk < k; kk += 2 * nw) {
            const bool two = kk + 1 < k;
            const float* qh0 = Qh + (int64_t)kk * len;
            const float* ql0 = Ql + (int64_t)kk * len;
            const float* qh1 = Qh + (int64_t)(two ? kk + 1 : kk) * len;
            const float* ql1 = Ql + (int64_t)(two ? kk + 1 : kk) * len;
            df64 a0{0.f, 0.f}, a1{0.f, 0.f}, b0{0.f, 0.f}, b1{0.f, 0.f};
            // four rows per lane and step; the next step's loads issue before this step's sums
            float xh[4], xl[4], ph[4], pl[4], qh_[4], ql_[4];
            auto dload = [&](int64_t i, float* xh_, float* xl_, float* ph_, float* pl_, float* qa, float* qb) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t ii = i + 32 * u < i1 ? i + 32 * u : (i < i1 ? i : i0);
                    xh_[u] = vh[ii]; xl_[u] = vl[ii];
                    ph_[u] = qh0[ii]; pl_[u] = ql0[ii];
                    qa[u] = qh1[ii]; qb[u] = ql1[ii];
                }
            };
            if (i0 + lane < i1) dload(i0 + lane, xh, xl, ph, pl, qh_, ql_);
            for (int64_t i = i0 + lane; i < i1; i += 128) {
                float nxh[4], nxl[4], nph[4], npl[4], nqh[4], nql[4];
                if (i + 128 < i1) dload(i + 128, nxh, nxl, nph, npl, nqh, nql);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (i + 32 * u >= i1) break;
                    const df64 x{xh[u], xl[u]};
                    if (u & 1) {
                        a1 = df_add(a1, df_mul(df64{ph[u], pl[u]}, x));
                        b1 = df_add(b1, df_mul(df64{qh_[u], ql_[u]}, x));
                    } else {
                        a0 = df_add(a0, df_mul(df64{ph[u], pl[u]}, x));
                        b0 = df_add(b0, df_mul(df64{qh_[u], ql_[u]}, x));
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    xh[u] = nxh[u]; xl[u] = nxl[u];
                    ph[u] = nph[u]; pl[u] = npl[u];
                    qh_[u] = nqh[u]; ql_[u] = nql[u];
                }
            }
            const df64 acc0 = warp_sum_t(df_add(a0, a1));
            const df64 acc1 = warp_sum_t(df_add(b0, b1));
            if (lane == 0) {
                red1[(int64_t)g * r + kk] = acc0;
                if (two) red1[(int64_t)g * r + kk + 1] = acc1;
            }
        }
        if (!barrier(2u)) return;
        // P2: s = Q^T v, the CTAs' partial dots summed per direction in a fixed order (the
        // same in every CTA): D directions at a time, 256 / D threads per direction each
        // summing every (256 / D)-th CTA with up to kRB loads in flight, then the subsets
        // in order.
        {
            constexpr int kRB = 10;
            __shared__ df64 s_sub[kPivotThreads];
            const int D = k <= 32 ? 32 : 64, S = nt / D;
            const int dl = tid % D, gs = tid / D;
            for (int kb = 0; kb < k; kb += D) {
                const int kk = kb + dl;
                df64 acc{0.f, 0.f};
                if (kk < k) {
                    int gg = gs;
                    while (gg < G) {
                        df64 x[kRB];
#pragma unroll
                        for (int i = 0; i < kRB; ++i)
                            if (gg + i * S < G) x[i] = red1[(int64_t)(gg + i * S) * r + kk];
#pragma unroll
                        for (int i = 0; i < kRB; ++i)
                            if (gg + i * S < G) acc = df_add(acc, x[i]);
                        gg += kRB * S;
                    }
                }
                s_sub[tid] = acc;
                __syncthreads();
                if (gs == 0 && kk < k) {
                    df64 t = s_sub[dl];
                    for (int q = 1; q < S; ++q) t = df_add(t, s_sub[q * D + dl]);
                    s_df[kk] = t;
                }
                __syncthreads();
            }
        }
        // P3: ||v - Q s||^2 = ||v||^2 - ||s||^2 (Q orthonormal; s is ~eps ||a_p|| after the
        // first projection, so the difference loses nothing): the early-stop test and the
        // norm of q_k need no further reduction over the CTAs
        if (tid < 32) {
            const double vv = warp_sum_strided(P.red2, G);
            df64 ss{0.f, 0.f};
            for (int kk = tid; kk < k; kk += 32) ss = df_add(ss, df_mul(s_df[kk], s_df[kk]));
            ss = warp_sum_t(ss);
            if (tid == 0) s_tot = vv - df_to_d(ss);
        }
        __syncthreads();
        const double mx = (double)max(P.m, P.n) * 2.220446049250313e-16;
        if (!(s_tot > mx * mx * (*P.frob2))) {
            if (g == 0 && tid == 0) { *P.stop = 1; set_status(P.status, CUR_WARN_RANK); }
            return;
        }
        if (g == 0 && tid == 0) {
            P.idx_out[k] = (int)p;
            P.mask[p] = 1;
            *P.count = k + 1;
        }
        if (!build) return;
        if (tid == 0) s_inv = df_from_d(1.0 / sqrt(s_tot));
        __syncthreads();
        const df64 inv = s_inv;
        // second projection v -= Q s and q_k = v / ||v|| in one sweep
        for (int64_t ia = i0 + tid; ia < i1; ia += 2 * nt) {
            const int64_t ib = ia + nt;
            const bool vb = ib < i1;
            df64 acc_a{vh[ia], vl[ia]};
            df64 acc_b = vb ? df64{vh[ib], vl[ib]} : df64{0.f, 0.f};
            qsub_pair(Qh, Ql, len, k, s_df, ia, ib, vb, acc_a, acc_b);
            const df64 qa = df_mul(acc_a, inv);
            Qh[(int64_t)k * len + ia] = qa.h;
            Ql[(int64_t)k * len + ia] = qa.l;
            P.qh[ia] = qa.h;
            P.ql[ia] = qa.l;
            if (vb) {
                const df64 qb = df_mul(acc_b, inv);
                Qh[(int64_t)k * len + ib] = qb.h;
                Ql[(int64_t)k * len + ib] = qb.l;
                P.qh[ib] = qb.h;
                P.ql[ib] = qb.l;
            }
        }
    } else {
        // FP64 data: the same steps in FP64.
        const double* Wd = reinterpret_cast<const double*>(W);
        for (int kk = tid; kk < k; kk += nt) s_w[kk] = Wd[(int64_t)kk * P.nsel + p];
        __syncthreads();
        double nv = 0.0;
        for (int64_t i = i0 + tid; i < i1; i += nt) {
            double s = 0.0;
            for (int kk = 0; kk < k; ++kk) s = fma(P.Q[(int64_t)kk * len + i], s_w[kk], s);
            const double vi = pivot_elem<TA>(P, i, p) - s;
            P.v[i] = vi;
            nv = fma(vi, vi, nv);
        }
        nv = block_sum(nv);
        if (tid == 0) P.red2[g] = nv;
        for (int kk = warp; kk < k; kk += nw) {
            const double* qk = P.Q + (int64_t)kk * len;
            double acc = 0.0;
            for (int64_t i = i0 + lane; i < i1; i += 32) acc = fma(qk[i], P.v[i], acc);
            acc = warp_sum(acc);
            if (lane == 0) P.red1[(int64_t)g * r + kk] = acc;
        }
        if (!barrier(2u)) return;
        for (int kk = warp; kk < k; kk += nw) {
            const double sk = warp_sum_strided(P.red1 + kk, G, r);
            if (lane == 0) s_w[kk] = sk;
        }
        __syncthreads();
        // ||v - Q s||^2 = ||v||^2 - ||s||^2, as above
        if (tid < 32) {
            const double vv = warp_sum_strided(P.red2, G);
            double ss = 0.0;
            for (int kk = tid; kk < k; kk += 32) ss = fma(s_w[kk], s_w[kk], ss);
            ss = warp_sum(ss);
            if (tid == 0) s_tot = vv - ss;
        }
        __syncthreads();
        const double mx = (double)max(P.m, P.n) * 2.220446049250313e-16;
        if (!(s_tot > mx * mx * (*P.frob2))) {
            if (g == 0 && tid == 0) { *P.stop = 1; set_status(P.status, CUR_WARN_RANK); }
            return;
        }
        if (g == 0 && tid == 0) {
            P.idx_out[k] = (int)p;
            P.mask[p] = 1;
            *P.count = k + 1;
        }
        if (!build) return;
        const double inv = 1.0 / sqrt(s_tot);
        for (int64_t i = i0 + tid; i < i1; i += nt) {
            double s = 0.0;
            for (int kk = 0; kk < k; ++kk) s = fma(P.Q[(int64_t)kk * len + i], s_w[kk], s);
            const double q = (P.v[i] - s) * inv;
            P.Q[(int64_t)k * len + i] = q;
            P.q64[i] = q;
            float hi, lo;
            split_d(q, hi, lo);
            P.qh[i] = hi;
            P.ql[i] = lo;
        }
    }
}

template <typename TA>
static cur_status launch_pass(const AcaParams& P, int mode, int64_t chunk, int rc_count,
                              bool vec, cudaStream_t st) {
    const TA* A = static_cast<const TA*>(P.A);
    PartT<TA>* part = static_cast<PartT<TA>*>(const_cast<void*>(P.part));
    if (P.axis == 1) {
        constexpr int TW = 32 * ColsPerLane<TA>::v;
        dim3 grid((unsigned)((P.n + TW - 1) / TW), (unsigned)rc_count);
        if (mode == kNorm) {
            if (vec) aca_cols_pass<TA, kNorm, true><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, chunk, P.q64, P.qh, P.ql, part, P.stop);
            else aca_cols_pass<TA, kNorm, false><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, chunk, P.q64, P.qh, P.ql, part, P.stop);
        } else {
            if (vec) aca_cols_pass<TA, kDot, true><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, chunk, P.q64, P.qh, P.ql, part, P.stop);
            else aca_cols_pass<TA, kDot, false><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, chunk, P.q64, P.qh, P.ql, part, P.stop);
        }
    } else {
        const int64_t blocks = std::min<int64_t>((P.m + 7) / 8, 65535LL * 8);
        dim3 grid((unsigned)blocks);
        if (mode == kNorm) {
            if (vec) aca_rows_pass<TA, kNorm, true><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, P.q64, P.qh, P.ql, part, P.stop);
            else aca_rows_pass<TA, kNorm, false><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, P.q64, P.qh, P.ql, part, P.stop);
        } else {
            if (vec) aca_rows_pass<TA, kDot, true><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, P.q64, P.qh, P.ql, part, P.stop);
            else aca_rows_pass<TA, kDot, false><<<grid, 256, 0, st>>>(A, P.m, P.n, P.ld, P.q64, P.qh, P.ql, part, P.stop);
        }
    }
    CUR_CK(cudaGetLastError());
    return CUR_OK;
}

// The selection's state before its first pass: no index picked, no stop, the pivots'
// group-barrier counter at zero, idx_out[0..r) = -1.
__global__ void aca_init_k(unsigned char* mask, int64_t nsel, int* stop, int32_t* count, int32_t* idx_out, int r,
                           unsigned* bar) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nsel; j += (int64_t)gridDim.x * blockDim.x)
        mask[j] = 0;
    if (blockIdx.x != 0) return;
    for (int k = threadIdx.x; k < r; k += blockDim.x) idx_out[k] = -1;
    if (threadIdx.x == 0) {
        *stop = 0;
        *count = 0;
        *bar = 0u;
    }
}

template <typename TA>
static cur_status aca_run(cur_handle* h, const cur_mat* M, int axis, int r, int32_t* idx_out,
                          int32_t* count_dev, Arena& ar, cudaStream_t st) {
    AcaParams P{};
    P.A = M->data;
    P.m = M->rows;
    P.n = M->cols;
    P.ld = M->ld;
    P.axis = axis;
    P.r = r;
    P.nsel = axis == 1 ? P.n : P.m;
    P.len = axis == 1 ? P.m : P.n;
    const int G = h->num_sms;
    // Row chunks of the column pass: enough CTAs for ~32 per SM.
    int RC = 1;
    int64_t chunk = P.m;
    if (axis == 1) {
        const int64_t coltiles = (P.n + 32 * ColsPerLane<TA>::v - 1) / (32 * ColsPerLane<TA>::v);
        int64_t want = std::max<int64_t>(1, (int64_t)h->num_sms * 32 / coltiles);
        want = std::min<int64_t>(want, std::max<int64_t>(1, P.m / 64));
        want = std::min<int64_t>(want, 65535);
        RC = (int)want;
        chunk = (P.m + RC - 1) / RC;
        RC = (int)((P.m + chunk - 1) / chunk);
    }
    P.RC = RC;
    P.part = ar.get<double>((size_t)RC * P.nsel);   // PartT is 8 bytes either way
    P.nu = ar.get<double>(P.nsel);
    P.mask = ar.get<unsigned char>(P.nsel);
    P.W = ar.get<double>((size_t)r * P.nsel);
    P.Q = ar.get<double>((size_t)P.len * r);
    P.q64 = ar.get<double>(P.len);
    P.qh = ar.get<float>(P.len);
    P.ql = ar.get<float>(P.len);
    P.v = ar.get<double>(P.len);
    P.red1 = ar.get<double>((size_t)G * r);
    P.red2 = ar.get<double>(G);
    P.redf = ar.get<double>(G);
    P.keyv = ar.get<double>(G);
    P.keyi = ar.get<long long>(G);
    P.bar = ar.get<unsigned>(1);
    P.frob2 = ar.get<double>(1);
    P.stop = ar.get<int>(1);
    P.count = count_dev;
    P.idx_out = idx_out;
    P.status = h->status;
    if (!ar.ok) return CUR_ERR_NOMEM;

    const size_t es = sizeof(TA);
    const uintptr_t base = reinterpret_cast<uintptr_t>(M->data);
    const size_t va = 16;   // 16-byte vector loads on every row (8 columns of BF16, 4 of FP32)
    const bool vec = (base % va == 0) && ((size_t)(M->ld * es) % va == 0);

    aca_init_k<<<(unsigned)std::min<int64_t>((P.nsel + 255) / 256, 4LL * G), 256, 0, st>>>(
        P.mask, P.nsel, P.stop, count_dev, idx_out, r, P.bar);
    CUR_CK(cudaGetLastError());
    note_launch();

    CUR_TRY(launch_pass<TA>(P, kNorm, chunk, RC, vec, st));
    note_launch();
    for (int t = -1; t <= r - 2; ++t) {
        if (t >= 0) {
            const bool ev = h->prof && h->prof_n < 4096;
            if (ev) CUR_CK(cudaEventRecord(h->prof_ev[2 * h->prof_n], st));
            CUR_TRY(launch_pass<TA>(P, kDot, chunk, RC, vec, st));
            if (ev) CUR_CK(cudaEventRecord(h->prof_ev[2 * h->prof_n + 1], st));
            if (ev) ++h->prof_n;
            note_launch();
        }
        int build = (t + 1 < r - 1) ? 1 : 0;
        unsigned bb = 2u * (unsigned)G * (unsigned)(t + 1);
        void* args[] = {&P, &t, &build, &bb};
        CUR_TRY(launch_coop((const void*)aca_pivot<TA>, dim3(G), dim3(kPivotThreads), args, 0, st));
        note_launch();
    }
    return CUR_OK;
}

}  // namespace curk

cur_status aca_select_full(cur_handle* h, const cur_mat* A, int axis, int r, int32_t* idx_out,
                           int32_t* count_dev, Arena& ar, cudaStream_t st) {
    if (r > 128) return CUR_ERR_ARG;
    switch (A->dtype) {
        case CUR_F64: return curk::aca_run<double>(h, A, axis, r, idx_out, count_dev, ar, st);
        case CUR_F32: return curk::aca_run<float>(h, A, axis, r, idx_out, count_dev, ar, st);
        case CUR_BF16: return curk::aca_run<__nv_bfloat16>(h, A, axis, r, idx_out, count_dev, ar, st);
    }
    return CUR_ERR_ARG;
}

// ---- the column pass alone, for a row slab of A (the sharded Algorithm 3 in shard.cu)

int aca_cols_chunks(int num_sms, int64_t m, int64_t n, cur_dtype dt, int64_t* chunk) {
    const int cpl = dt == CUR_BF16 ? 8 : 4;
    const int64_t coltiles = (n + 32 * cpl - 1) / (32 * cpl);
    int64_t want = std::max<int64_t>(1, (int64_t)num_sms * 32 / coltiles);
    want = std::min<int64_t>(want, std::max<int64_t>(1, m / 64));
    want = std::min<int64_t>(want, 65535);
    const int64_t c = (m + want - 1) / want;
    *chunk = c;
    return (int)((m + c - 1) / c);
}

cur_status aca_cols_partials(const cur_mat* M, int dot, const double* q64, const float* qh,
                             const float* ql, void* part, int RC, int64_t chunk, const int* stop,
                             cudaStream_t st) {
    using namespace curk;
    AcaParams P{};
    P.A = M->data;
    P.m = M->rows;
    P.n = M->cols;
    P.ld = M->ld;
    P.axis = 1;
    P.q64 = const_cast<double*>(q64);
    P.qh = const_cast<float*>(qh);
    P.ql = const_cast<float*>(ql);
    P.part = part;
    P.stop = const_cast<int*>(stop);
    const uintptr_t base = reinterpret_cast<uintptr_t>(M->data);
    const bool vec = (base % 16 == 0) && ((size_t)M->ld * dtype_size(M->dtype)) % 16 == 0;
    const int mode = dot ? kDot : kNorm;
    cur_status s = CUR_ERR_ARG;
    switch (M->dtype) {
        case CUR_F64: s = launch_pass<double>(P, mode, chunk, RC, vec, st); break;
        case CUR_F32: s = launch_pass<float>(P, mode, chunk, RC, vec, st); break;
        case CUR_BF16: s = launch_pass<__nv_bfloat16>(P, mode, chunk, RC, vec, st); break;
    }
    if (s == CUR_OK) note_launch();
    return s;
}
