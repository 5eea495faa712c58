// Algorithm 3 (Section 2.2) on the columns of every matrix of a batch, one launch.
//
// The batch holds many small matrices of uneven shapes (up to a few thousand rows and a
// thousand columns, each a few MB), so each one is taken whole by one CTA: a persistent
// grid walks the batch, and a CTA runs all r rounds of its matrix with no grid-wide
// synchronisation. The rounds are those of the full-matrix kernels (the implicit
// residual nu_j = ||a_j||^2 - sum_k (q_k^T a_j)^2, one read of the matrix per round):
//   pass   : w_j = a_j^T q_t for every column (Dot2 with q as FP32 hi/lo pairs), the
//            512 threads split into n/4 four-column groups x as many row groups as fit
//            (2 for n = 1024, 16 for n = 128), every thread streaming; two CTAs
//            per SM, so one streams its matrix while the other runs its pivot step
//   pick   : nu_j -= w_j^2, masked argmax (lowest index on ties)
//   vector : v = a_p - Q W(:,p) with W = the passes' q^T a (the first Gram-Schmidt sweep
//            needs no Q^T a_p of its own), orthogonalised once more against q_1..q_t
//            (double-float), the early stop
//            on the recomputed ||v||^2 <= (max(m,n) eps ||A||_F)^2, q = v / ||v||
// Q lives in the CTA's slice of the workspace (r x m hi and lo floats); everything else
// in shared memory. Supports FP32 data, r <= 64, m <= 4096, n <= 1024.

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace curk {

constexpr int kBA_T = 512;      // threads per CTA (two CTAs per SM: one streams while the other pivots)
constexpr int kBA_RG = kBA_T / 256;   // partial-sum rows per column in shared memory: RG n <= kBA_RG kBA_MaxN
constexpr int kBA_MaxM = 4096;
constexpr int kBA_MaxN = 1024;
constexpr int kBA_MaxR = 64;

struct BatAcaItem {
    int64_t aoff, m, n, ld;   // matrix at data + aoff, row-major with leading dimension ld
    int32_t r;
    int64_t joff;             // its J0 at J + joff (r entries)
};

// shared-memory layout (bytes): nu n x 8 | part RG x n x 8 | v m x 8 | qh m x 4 | ql m x 4 |
// s kBA_MaxR x 8 | mask n
__host__ __device__ constexpr size_t bat_aca_smem() {
    return (size_t)kBA_MaxN * 8 + (size_t)kBA_RG * kBA_MaxN * 8 + (size_t)kBA_MaxM * 8 + (size_t)kBA_MaxM * 8 +
           (size_t)kBA_MaxR * 8 + kBA_MaxN + 64;
}

// (key, index) maximum over the CTA, integer keys (dkey order): no FP64 comparisons.
__device__ __forceinline__ void bat_argmax(unsigned long long& k, int& i) {
    long long li = i;
    block_argmax_key(k, li);
    i = (int)li;
}

__device__ __forceinline__ df64 bat_df_sum(df64 x) {
    __shared__ df64 sw[32];
    for (int o = 16; o > 0; o >>= 1)
        x = df_add(x, df64{__shfl_xor_sync(0xffffffffu, x.h, o), __shfl_xor_sync(0xffffffffu, x.l, o)});
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sw[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        df64 s{0.f, 0.f};
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s = df_add(s, sw[q]);
        sw[0] = s;
    }
    __syncthreads();
    const df64 out = sw[0];
    __syncthreads();
    return out;
}

// qs[k] = sum_i Q(k, i) v(i) for k < t (one warp per direction, double-float), then
// v(i) -= sum_k Q(k, i) qs[k].
__device__ void bat_project(const float* Qh, const float* Ql, int64_t m, int t, df64* v, df64* qs) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < t; k += nw) {
        const float* qh = Qh + (int64_t)k * m;
        const float* ql = Ql + (int64_t)k * m;
        df64 a0{0.f, 0.f}, a1{0.f, 0.f};
        for (int64_t i = lane; i < m; i += 64) {
            a0 = df_add(a0, df_mul(df64{qh[i], ql[i]}, v[i]));
            if (i + 32 < m) a1 = df_add(a1, df_mul(df64{qh[i + 32], ql[i + 32]}, v[i + 32]));
        }
        df64 s = df_add(a0, a1);
        for (int o = 16; o > 0; o >>= 1)
            s = df_add(s, df64{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)});
        if (lane == 0) qs[k] = s;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        df64 a0{0.f, 0.f}, a1{0.f, 0.f};
        int k = 0;
        for (; k + 1 < t; k += 2) {
            a0 = df_add(a0, df_mul(df64{Qh[(int64_t)k * m + i], Ql[(int64_t)k * m + i]}, qs[k]));
            a1 = df_add(a1, df_mul(df64{Qh[(int64_t)(k + 1) * m + i], Ql[(int64_t)(k + 1) * m + i]}, qs[k + 1]));
        }
        if (k < t) a0 = df_add(a0, df_mul(df64{Qh[(int64_t)k * m + i], Ql[(int64_t)k * m + i]}, qs[k]));
        v[i] = df_sub(v[i], df_add(a0, a1));
    }
    __syncthreads();
}

// order: the matrices by decreasing cost (r m n); queue: a zeroed counter. A CTA takes
// the next matrix of the order when it finishes one (largest first, so the tail is short).
__global__ void __launch_bounds__(kBA_T, 2) bat_aca_k(const float* __restrict__ data, const BatAcaItem* items,
                                                       const int32_t* order, int* queue, int count, int32_t* J,
                                                       int32_t* counts, float* Qws, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* nu = reinterpret_cast<double*>(smem_raw);
    df64* part = reinterpret_cast<df64*>(nu + kBA_MaxN);               // RG x n
    df64* v = part + kBA_RG * kBA_MaxN;                                  // m
    float* qh = reinterpret_cast<float*>(v + kBA_MaxM);                  // m
    float* ql = qh + kBA_MaxM;                                           // m
    df64* qs = reinterpret_cast<df64*>(ql + kBA_MaxM);                   // r
    unsigned char* mask = reinterpret_cast<unsigned char*>(qs + kBA_MaxR);
    __shared__ double s_frob2;
    __shared__ int s_next;
    const int tid = threadIdx.x;
    float* Qh = Qws + (int64_t)blockIdx.x * 2 * kBA_MaxR * kBA_MaxM;
    float* Ql = Qh + (int64_t)kBA_MaxR * kBA_MaxM;
    // W(t, j) = q_t^T a_j from the passes (the CTA's slice after all CTAs' Q slices)
    df64* W = reinterpret_cast<df64*>(Qws + (int64_t)gridDim.x * 2 * kBA_MaxR * kBA_MaxM) +
              (int64_t)blockIdx.x * kBA_MaxR * kBA_MaxN;

    while (true) {
        if (tid == 0) s_next = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_next;
        __syncthreads();
        if (q >= count) break;
        const int it = order[q];
        const BatAcaItem b = items[it];
        const float* A = data + b.aoff;
        const int64_t m = b.m, n = b.n, ld = b.ld;
        const int r = b.r;
        const bool vec = (n % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
        // column groups of 4 columns; as many row groups as the CTA's threads cover, so every
        // thread streams (a narrow matrix would otherwise leave most of them idle)
        const int cgn = (int)((n + 3) / 4);
        const int RG = max(1, min((int)blockDim.x / cgn, (int)(kBA_RG * kBA_MaxN / n)));
        const int cg = tid % cgn, rg = tid / cgn;
        const bool active = rg < RG;
        for (int j = tid; j < n; j += blockDim.x) mask[j] = 0;
        int picked = 0, bad = 0;
        for (int t = -1; t < r - 1; ++t) {
            // ---- pass: squared norms (t = -1) or w = A^T q_t
            const int64_t c0 = 4 * (int64_t)cg;
            Dot2 acc[4];
            if (active && c0 < n) {
                // four rows loaded before they are folded: 64 bytes in flight per thread
                for (int64_t i0 = rg; i0 < m; i0 += 4 * RG) {
                    float x[4][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t i = i0 + RG * u;
                        const float* row = A + (i < m ? i : i0) * ld + c0;
                        if (vec) {
                            const float4 y = __ldcs(reinterpret_cast<const float4*>(row));
                            x[u][0] = y.x; x[u][1] = y.y; x[u][2] = y.z; x[u][3] = y.w;
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; ++c) x[u][c] = c0 + c < n ? row[c] : 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t i = i0 + RG * u;
                        if (i >= m) break;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (t < 0) acc[c].add_sq(x[u][c]); else acc[c].add(x[u][c], qh[i], ql[i]);
                        }
                    }
                }
            }
            if (active && c0 < n)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (c0 + c < n) part[rg * n + c0 + c] = fast_two_sum(acc[c].s, acc[c].c);
            __syncthreads();
            // ---- pick
            unsigned long long bk = dkey(-INFINITY);
            int bi = INT_MAX;
            double fs = 0.0;
            for (int j = tid; j < n; j += blockDim.x) {
                df64 w = part[j];
                for (int g = 1; g < RG; ++g) w = df_add(w, part[g * n + j]);
                const double wd = df_to_d(w);
                double nuj;
                if (t < 0) {
                    nuj = wd;
                    fs += wd;
                    if (!isfinite(wd)) bad = 1;
                } else {
                    nuj = nu[j] - wd * wd;
                    W[(int64_t)t * n + j] = w;
                }
                nu[j] = nuj;
                const unsigned long long kj = dkey(nuj);
                if (!mask[j] && (kj > bk || (kj == bk && j < bi))) { bk = kj; bi = j; }
            }
            bad = __syncthreads_or(bad);
            if (t < 0) {
                const df64 f = bat_df_sum(df64{(float)fs, (float)(fs - (double)(float)fs)});
                if (tid == 0) s_frob2 = df_to_d(f);
            }
            bat_argmax(bk, bi);
            if (bad) {
                if (tid == 0) set_status(status, CUR_ERR_NONFINITE);
                break;
            }
            if (bi == INT_MAX) break;
            const int p = bi;
            // ---- vector: v = a_p - Q W(:,p) (the first projection's coefficients q^T a_p are
            // the passes' w, as in the full-matrix kernel), then orthogonalised once more
            const int k = t + 1;
            for (int kk = tid; kk < k; kk += blockDim.x) qs[kk] = W[(int64_t)kk * n + p];
            __syncthreads();
            for (int64_t i = tid; i < m; i += blockDim.x) {
                df64 a0{A[i * ld + p], 0.f}, a1{0.f, 0.f};
                int kk = 0;
                for (; kk + 1 < k; kk += 2) {
                    a0 = df_sub(a0, df_mul(df64{Qh[(int64_t)kk * m + i], Ql[(int64_t)kk * m + i]}, qs[kk]));
                    a1 = df_sub(a1, df_mul(df64{Qh[(int64_t)(kk + 1) * m + i], Ql[(int64_t)(kk + 1) * m + i]}, qs[kk + 1]));
                }
                if (kk < k) a0 = df_sub(a0, df_mul(df64{Qh[(int64_t)kk * m + i], Ql[(int64_t)kk * m + i]}, qs[kk]));
                v[i] = df_add(a0, a1);
            }
            __syncthreads();
            bat_project(Qh, Ql, m, k, v, qs);
            df64 nv{0.f, 0.f};
            for (int64_t i = tid; i < m; i += blockDim.x) nv = df_add(nv, df_mul(v[i], v[i]));
            const double s_tot = df_to_d(bat_df_sum(nv));
            const double mx = (double)max(m, n) * 2.220446049250313e-16;
            if (!(s_tot > mx * mx * s_frob2)) break;
            if (tid == 0) {
                J[b.joff + k] = p;
                mask[p] = 1;
            }
            picked = k + 1;
            if (k == r - 1) break;
            const df64 inv = df_from_d(1.0 / sqrt(s_tot));
            for (int64_t i = tid; i < m; i += blockDim.x) {
                const df64 q = df_mul(v[i], inv);
                Qh[(int64_t)k * m + i] = q.h;
                Ql[(int64_t)k * m + i] = q.l;
                qh[i] = q.h;
                ql[i] = q.l;
            }
            __syncthreads();
        }
        if (tid == 0) {
            counts[it] = picked;
            for (int k = picked; k < r; ++k) J[b.joff + k] = -1;
        }
        __syncthreads();
    }
}

}  // namespace curk

size_t bat_aca_workspace(int grid) {
    return (size_t)grid * 2 * curk::kBA_MaxR * curk::kBA_MaxM * sizeof(float) +
           (size_t)grid * curk::kBA_MaxR * curk::kBA_MaxN * sizeof(double);
}

cur_status bat_aca_launch(const float* data, const void* items_dev, const int32_t* order, int* queue, int count,
                          int32_t* J, int32_t* counts, float* Qws, int grid, int* status, cudaStream_t st) {
    using namespace curk;
    const size_t sm = bat_aca_smem();
    CUR_TRY(smem_attr((const void*)bat_aca_k, sm));
    CUR_CK(cudaMemsetAsync(queue, 0, sizeof(int), st));
    bat_aca_k<<<grid, kBA_T, sm, st>>>(data, static_cast<const BatAcaItem*>(items_dev), order, queue, count, J,
                                       counts, Qws, status);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

size_t bat_aca_item_size() { return sizeof(curk::BatAcaItem); }
