// Block-wise maximal-volume selection with a binary merge (GB300 form).
//
// The maximal-volume problem (Section 1.2, Definition 1) on a tall basis C
// (p x r) is attacked by the swap iteration: with M = C(S,:) and B = C M^-1,
// every entry B_ij is the factor by which |det M| changes when row i of C
// replaces position j of S. While max|B_ij| > 1 + delta the best swap is made
// and B is updated by Sherman-Morrison, B <- B - B(:,j) (B(i,:) - e_j^T) / B_ij;
// every r swaps, and before convergence is declared, a new cycle starts from B
// recomputed as C M^-1.
//
// Work is organised as "problems" (a row block of C, a merge node, or all of C),
// each handled by one CTA or by a group of co-resident CTAs:
//   mv_start  : Algorithm 3 (axis 0) on the problem's rows -> start set S
//               (implicit Gram-Schmidt, one group barrier per pick)
//   mv_lu     : one CTA per problem, FP64 Gauss-Jordan inverse of C(S,:) with
//               partial pivoting, log|det|
//   mv_engine : the whole swap iteration of a stage in one launch. Each CTA keeps
//               its slice of B in shared memory (FP32 for FP32/BF16 data, FP64 for
//               FP64 data; in global memory for a problem too large for that), and
//               a group agrees on argmax|B_ij| through one barrier per swap. The
//               first CTA recomputes the winning row of B from C and M^-1 and keeps
//               M^-1 current by the Sherman-Morrison update (double-float for FP32
//               data, FP64 for FP64 data). A cycle refactorises C(S,:) (FP64 data:
//               always; FP32 data: once the kept inverse's drift bound exceeds its
//               limit) and refreshes B = C M^-1. A merge node starts from its left
//               child's M^-1.
// A stage's problems may have different ranks (batches); single-CTA problems go in one
// plain launch, multi-CTA groups in cooperative launches of co-resident waves.

#include <algorithm>
#include <array>
#include <climits>
#include <initializer_list>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace curk {

constexpr double kEps = 2.220446049250313e-16;

struct MvProb {
    int64_t base;      // first row of the problem in the basis / B buffers
    int64_t boff;      // element offset of its basis rows (p x r, contiguous)
    int32_t r;         // its rank (<= the stage's r, which is the stride of per-problem arrays)
    int32_t gmode;     // 1: its B lives in global memory (a problem too large for shared memory)
    int64_t gid_base;  // global id of local row i = gid_base + i (when gid_arr == null)
    const int32_t* gid_arr;
    int32_t p;         // rows
    int32_t G;         // CTAs in its group
    int32_t rpc;       // rows per CTA
    int32_t group0;    // first slot of its group
};

struct MvArgs {
    const void* basis;  // rows x r (compute type), contiguous
    double* minv64;     // P x minv_stride(r): FP64 M^-1 of each problem, then its drift bound
    float* mdf;         // P x 2 r^2: double-float working copy when r > kMsMax (FP32 data)
    const MvProb* prob;
    int P, r;
    double delta;
    int max_swaps;
    double drift_max;          // refactorise once sum(swaps * kappa(M)) since the last factorisation exceeds it
    int keep_singular_set;     // 1: a set that turns singular stays as it is; 0: back to the start set
    void* bglob;               // rows x r B in global memory (compute type), or null: B in shared memory
    const void* bpre;          // rows x r: the first cycle's B from the tensor-core product, or null
    const int32_t* cta_prob;   // per CTA slot
    const int32_t* cta_part;
    int cta_base;              // first slot of this launch (waves)
    const int32_t* lu_mask;    // P: 1 = factorise C(S,:) in mv_lu
    int32_t* S;                // P x r local positions
    double* logvol;            // P
    int32_t* swaps;            // P
    int32_t* pstatus;          // P
    int32_t* done;             // P
    unsigned* bar;             // P
    double* keyv;              // slots x 2
    long long* keyi;           // slots x 2
    void* pub;                 // slots x 2 x r (compute type)
    double* aux;               // slots x 2 (start: frob partials)
    int* status;               // handle status word
    int* nrefactor;            // count of cycle refactorisations (instrumentation)
};

// ---------------------------------------------------------------- gathers

template <typename TA, typename TB>
__global__ void gather_cols_k(const TA* __restrict__ A, int64_t m, int64_t n, int64_t ld,
                              const int32_t* __restrict__ J, int r, TB* __restrict__ C,
                              int* status, const int* idle) {
    if (idle && *idle) return;
    const int64_t total = m * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int k = (int)(e - i * r);
        const int64_t j = J[k];
        if (j < 0 || j >= n) {
            set_status(status, CUR_ERR_ARG);
            C[e] = (TB)0;
            continue;
        }
        C[e] = (TB)to_d(A[i * ld + j]);
    }
}

// Rt(j, k) = A(I[k], j): 32 columns per CTA, transposed through shared memory.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) gather_rows_t_k(const TA* __restrict__ A, int64_t m,
                                                       int64_t n, int64_t ld,
                                                       const int32_t* __restrict__ I, int r,
                                                       TB* __restrict__ Rt, int* status, const int* idle) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (idle && *idle) return;
    TB* tile = reinterpret_cast<TB*>(smem_raw);  // r x 33
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    for (int k = ty; k < r; k += 8) {
        const int64_t i = I[k];
        const int64_t j = j0 + tx;
        TB v = (TB)0;
        if (i < 0 || i >= m) {
            if (tx == 0) set_status(status, CUR_ERR_ARG);
        } else if (j < n) {
            v = (TB)to_d(A[i * ld + j]);
        }
        tile[k * 33 + tx] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * r; e += blockDim.x) {
        const int jj = e / r, kk = e - jj * r;
        if (j0 + jj < n) Rt[(j0 + jj) * r + kk] = tile[kk * 33 + jj];
    }
}

// U rows (t*2r + i) = basis rows gid[t*2r + i].
template <typename TB>
__global__ void gather_union_k(const TB* __restrict__ basis, int64_t p, int r,
                               const int32_t* __restrict__ gid, int64_t nrows,
                               TB* __restrict__ U, int* status) {
    const int64_t total = nrows * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int c = (int)(e - i * r);
        const int64_t g = gid[i];
        if (g < 0 || g >= p) {
            set_status(status, CUR_ERR_ARG);
            U[e] = (TB)0;
            continue;
        }
        U[e] = basis[g * r + c];
    }
}

// ---------------------------------------------------------------- start: Algorithm 3 on rows

// The problem's rows sit in shared memory with an odd row stride, so that the 32 lanes of
// a warp, one row each, read 32 different banks.
__host__ __device__ __forceinline__ int start_ld(int r) { return r | 1; }

template <typename TB>
struct StartSmem {
    static size_t bytes(int nloc, int r) {
        size_t b = (size_t)nloc * start_ld(r) * sizeof(TB);
        b = (b + 15) / 16 * 16 + (size_t)nloc * sizeof(double);
        b += (size_t)r * r * sizeof(double);        // Q (FP64 data) or the projector P
        b += (size_t)10 * r * sizeof(double);       // v, sd, partial sums (8 r)
        b += (size_t)2 * r * sizeof(float);         // qh, ql
        b += (size_t)nloc + 16;                     // mask
        return b;
    }
};

// nu[i] = sum_c rows(i,c) * q(c) (mode 1: nu[i] -= that squared) or rows(i,c)^2 (mode 0),
// one thread per row, the columns in order (Dot2 for FP32 data, FP64 for FP64 data); the
// row's sum meets the FP64 pipe once, for the downdate.
template <typename TB>
__device__ __forceinline__ void rows_dot(const TB* rows, int ld, int nloc, int r, const double* q64,
                                         const float* qh, const float* ql, int mode,
                                         double* out, bool downdate) {
    for (int row = threadIdx.x; row < nloc; row += blockDim.x) {
        const TB* x = rows + (size_t)row * ld;
        double v;
        if constexpr (std::is_same<TB, double>::value) {
            DotD d;
            if (mode == 0) for (int c = 0; c < r; ++c) d.add_sq(x[c]);
            else for (int c = 0; c < r; ++c) d.add(x[c], q64[c]);
            v = d.value();
        } else {
            Dot2 d;
            if (mode == 0) for (int c = 0; c < r; ++c) d.add_sq(to_f(x[c]));
            else for (int c = 0; c < r; ++c) d.add(to_f(x[c]), qh[c], ql[c]);
            v = d.value();
        }
        if (downdate) out[row] -= v * v;
        else out[row] = v;
    }
}

// Threads of a block-start CTA: 16 warps for FP32/BF16 data (one row per thread for the
// 512-row slices of the row stage), 8 for FP64 data (its FP64 row sums need the registers).
template <typename TB> struct StartThreads { static constexpr int v = 512; };
template <> struct StartThreads<double> { static constexpr int v = 256; };

template <typename TB>
__global__ void __launch_bounds__(StartThreads<TB>::v, 1) mv_start(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int slot = a.cta_base + blockIdx.x;
    const int pb = a.cta_prob[slot], part = a.cta_part[slot];
    if (a.done[pb]) return;   // every CTA of the group leaves together: no barrier is left waiting
    const MvProb pr = a.prob[pb];
    const int r = pr.r, rs = a.r, G = pr.G;
    const int lo = part * pr.rpc, hi = min(pr.p, lo + pr.rpc), nloc = max(0, hi - lo);
    const TB* basis = static_cast<const TB*>(a.basis) + pr.boff;
    TB* rows = reinterpret_cast<TB*>(smem_raw);
    const int ld = start_ld(r);
    size_t off = ((size_t)nloc * ld * sizeof(TB) + 15) / 16 * 16;
    double* nu = reinterpret_cast<double*>(smem_raw + off); off += (size_t)nloc * sizeof(double);
    double* Q = reinterpret_cast<double*>(smem_raw + off); off += (size_t)r * r * sizeof(double);
    double* v = reinterpret_cast<double*>(smem_raw + off); off += (size_t)r * sizeof(double);
    double* sd = reinterpret_cast<double*>(smem_raw + off); off += (size_t)r * sizeof(double);
    double* red = reinterpret_cast<double*>(smem_raw + off); off += (size_t)8 * r * sizeof(double);
    float* qh = reinterpret_cast<float*>(smem_raw + off); off += (size_t)r * sizeof(float);
    float* ql = reinterpret_cast<float*>(smem_raw + off); off += (size_t)r * sizeof(float);
    unsigned char* msk = smem_raw + off;
    __shared__ double s_frob, s_inv;
    __shared__ int s_stop, s_p;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    int32_t* Sout = a.S + (int64_t)pb * rs;

    {
        Walk2 w(tid, nt, r);
        for (int e = tid; e < nloc * r; e += nt, w.next()) rows[w.i * ld + w.c] = basis[(int64_t)lo * r + e];
    }
    for (int i = tid; i < nloc; i += nt) msk[i] = 0;
    __syncthreads();
    rows_dot<TB>(rows, ld, nloc, r, v, qh, ql, 0, nu, false);
    if constexpr (!std::is_same<TB, double>::value) {
        df64* Pd = reinterpret_cast<df64*>(Q);
        for (int e = tid; e < r * r; e += nt) Pd[e] = df64{(e / r == e % r) ? 1.f : 0.f, 0.f};
    }
    __syncthreads();
    double fs = 0.0;
    for (int i = tid; i < nloc; i += nt) fs += nu[i];
    fs = block_sum(fs);
    int picked = 0;
    for (int k = 0; k < r; ++k) {
        unsigned long long bk = dkey(-INFINITY);
        long long bi = LLONG_MAX;
        for (int i = tid; i < nloc; i += nt) {
            const unsigned long long kk = dkey(nu[i]);
            if (!msk[i] && better_key(kk, (long long)(lo + i), bk, bi)) { bk = kk; bi = lo + i; }
        }
        block_argmax_key(bk, bi);
        const int par = k & 1;
        if (tid == 0) {
            a.keyv[(pr.group0 + part) * 2 + par] = dkey_value(bk);
            a.keyi[(pr.group0 + part) * 2 + par] = bi;
            if (k == 0) a.aux[(pr.group0 + part) * 2] = fs;
        }
        if (!group_barrier(&a.bar[pb], (unsigned)(G * (k + 1)), a.status)) return;
        if (warp == 0) {
            unsigned long long pk = dkey(-INFINITY);
            long long pi = LLONG_MAX;
            for (int g = lane; g < G; g += 32) {
                const unsigned long long kv = dkey(a.keyv[(pr.group0 + g) * 2 + par]);
                const long long ki = a.keyi[(pr.group0 + g) * 2 + par];
                if (better_key(kv, ki, pk, pi)) { pk = kv; pi = ki; }
            }
            warp_argmax_key(pk, pi);
            if (k == 0) {
                const double f = warp_sum_strided(a.aux + (int64_t)pr.group0 * 2, G, 2);
                if (lane == 0) s_frob = f;
            }
            if (lane == 0) {
                s_stop = (pi == LLONG_MAX) ? 1 : 0;
                s_p = s_stop ? 0 : (int)pi;
            }
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        // new direction: v = c_p - Q Q^T c_p, twice (CGS2); its norm is the recomputed
        // residual norm of row p, which decides an early stop before p is recorded.
        // FP32/BF16 data: double-float (Q, v and the dot products as FP32 pairs).
        const TB* cp = basis + (int64_t)p * r;
        if constexpr (std::is_same<TB, double>::value) {
            for (int c = tid; c < r; c += nt) v[c] = to_d(cp[c]);
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                for (int kk = warp; kk < k; kk += nw) {
                    double s = 0.0;
                    for (int c = lane; c < r; c += 32) s = fma(Q[kk * r + c], v[c], s);
                    s = warp_sum(s);
                    if (lane == 0) sd[kk] = s;
                }
                __syncthreads();
                for (int it = tid; it < 4 * r; it += nt) {
                    const int c = it % r, qt = it / r;
                    double s = 0.0;
                    for (int kk = k * qt / 4; kk < k * (qt + 1) / 4; ++kk) s = fma(Q[kk * r + c], sd[kk], s);
                    red[qt * r + c] = s;
                }
                __syncthreads();
                for (int c = tid; c < r; c += nt)
                    v[c] -= ((red[c] + red[r + c]) + red[2 * r + c]) + red[3 * r + c];
                __syncthreads();
            }
            if (warp == 0) {
                double s = 0.0;
                for (int c = lane; c < r; c += 32) s = fma(v[c], v[c], s);
                s = warp_sum(s);
                if (lane == 0) {
                    const double mx = (double)max(pr.p, r) * kEps;
                    s_stop = !(s > mx * mx * s_frob) ? 1 : 0;
                    s_inv = 1.0 / sqrt(s);
                }
            }
            __syncthreads();
            if (s_stop) break;
            if (part == 0 && tid == 0) Sout[k] = p;
            if (p >= lo && p < hi && tid == 0) msk[p - lo] = 1;
            picked = k + 1;
            if (k == r - 1) break;
            for (int c = tid; c < r; c += nt) {
                const double q = v[c] * s_inv;
                Q[k * r + c] = q;
                v[c] = q;
                split_d(q, qh[c], ql[c]);
            }
            __syncthreads();
        } else {
            // The projector P = I - sum_k q_k q_k^T (r x r, double-float, in the bytes of Q)
            // is kept current, so the two Gram-Schmidt sweeps are two products v <- P v with
            // all threads busy, instead of k dependent dot products each.
            df64* Pd = reinterpret_cast<df64*>(Q);
            df64* vd = reinterpret_cast<df64*>(v);
            df64* sdd = reinterpret_cast<df64*>(sd);
            df64* redd = reinterpret_cast<df64*>(red);
            for (int c = tid; c < r; c += nt) vd[c] = df64{to_f(cp[c]), 0.f};
            __syncthreads();
            for (int pass = 0; pass < 2 && k > 0; ++pass) {
                // quarter qt of the rows of P for column c, as two interleaved chains (even and
                // odd d); with 8 r threads or more each chain has its own thread
                if (nt >= 8 * r) {
                    df64* half = redd + 4 * r;   // the odd chains
                    for (int it = tid; it < 8 * r; it += nt) {
                        const int c = it % r, qt = (it / r) & 3, odd = it / (4 * r);
                        const int d0 = r * qt / 4, d1 = r * (qt + 1) / 4;
                        df64 sx{0.f, 0.f};
                        for (int d = d0 + odd; d < d1; d += 2)   // P symmetric: column c read as row c
                            sx = df_add(sx, df_mul(Pd[d * r + c], vd[d]));
                        (odd ? half : redd)[qt * r + c] = sx;
                    }
                    __syncthreads();
                    for (int c = tid; c < r; c += nt) {
                        df64 q[4];
#pragma unroll
                        for (int qt = 0; qt < 4; ++qt) q[qt] = df_add(redd[qt * r + c], half[qt * r + c]);
                        vd[c] = df_add(df_add(q[0], q[1]), df_add(q[2], q[3]));
                    }
                } else {
                    for (int it = tid; it < 4 * r; it += nt) {
                        const int c = it % r, qt = it / r;
                        df64 s0{0.f, 0.f}, s1{0.f, 0.f};
                        const int d0 = r * qt / 4, d1 = r * (qt + 1) / 4;
                        int d = d0;
                        for (; d + 1 < d1; d += 2) {   // P symmetric: column c read as row c
                            s0 = df_add(s0, df_mul(Pd[d * r + c], vd[d]));
                            s1 = df_add(s1, df_mul(Pd[(d + 1) * r + c], vd[d + 1]));
                        }
                        if (d < d1) s0 = df_add(s0, df_mul(Pd[d * r + c], vd[d]));
                        redd[qt * r + c] = df_add(s0, s1);
                    }
                    __syncthreads();
                    for (int c = tid; c < r; c += nt)
                        vd[c] = df_add(df_add(redd[c], redd[r + c]), df_add(redd[2 * r + c], redd[3 * r + c]));
                }
                __syncthreads();
            }
            if (warp == 0) {
                df64 s{0.f, 0.f};
                for (int c = lane; c < r; c += 32) s = df_add(s, df_mul(vd[c], vd[c]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const df64 t{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)};
                    s = df_add(s, t);
                }
                if (lane == 0) {
                    const double sn = df_to_d(s);
                    const double mx = (double)max(pr.p, r) * kEps;
                    s_stop = !(sn > mx * mx * s_frob) ? 1 : 0;
                    s_inv = 1.0 / sqrt(sn);
                }
            }
            __syncthreads();
            if (s_stop) break;
            if (part == 0 && tid == 0) Sout[k] = p;
            if (p >= lo && p < hi && tid == 0) msk[p - lo] = 1;
            picked = k + 1;
            if (k == r - 1) break;
            if (tid == 0) sdd[0] = df_from_d(s_inv);
            __syncthreads();
            const df64 inv = sdd[0];
            __syncthreads();
            for (int c = tid; c < r; c += nt) {
                const df64 q = df_mul(vd[c], inv);
                vd[c] = q;
                qh[c] = q.h;
                ql[c] = q.l;
            }
            __syncthreads();
            if (nt % r == 0) {   // P -= q q^T, one column per thread
                const int c = tid % r, di = nt / r;
                const df64 qc = vd[c];
                for (int i = tid / r; i < r; i += di) Pd[i * r + c] = df_sub(Pd[i * r + c], df_mul(vd[i], qc));
            } else {
                for (int e = tid; e < r * r; e += nt) {   // P -= q q^T
                    const int i = e / r, c = e - i * r;
                    Pd[e] = df_sub(Pd[e], df_mul(vd[i], vd[c]));
                }
            }
            __syncthreads();
        }
        // downdate: nu_i -= (c_i . q_k)^2
        rows_dot<TB>(rows, ld, nloc, r, v, qh, ql, 1, nu, true);
        __syncthreads();
    }
    // pad a short selection with the lowest unselected local rows
    if (part == 0 && tid == 0 && picked < r) {
        int fill = picked;
        for (int cand = 0; cand < pr.p && fill < r; ++cand) {
            bool used = false;
            for (int q = 0; q < fill; ++q) used |= (Sout[q] == cand);
            if (!used) Sout[fill++] = cand;
        }
    }
}

// ---------------------------------------------------------------- FP64 inverse of C(S,:)

template <typename TB>
__global__ void __launch_bounds__(512) mv_lu(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pb = blockIdx.x;
    if (threadIdx.x == 0) a.bar[pb] = 0u;   // the swap engine's group barrier starts from zero
    if (a.done[pb] || !a.lu_mask[pb]) return;
    const MvProb pr = a.prob[pb];
    const int r = pr.r, rs = a.r, tid = threadIdx.x, nt = blockDim.x;
    double* M = reinterpret_cast<double*>(smem_raw);  // r x r, inverted in place
    double* colk = M + r * r;
    int* piv = reinterpret_cast<int*>(colk + r);
    __shared__ double s_max;
    const TB* basis = static_cast<const TB*>(a.basis) + pr.boff;
    const int32_t* S = a.S + (int64_t)pb * rs;
    // C(S,:) in FP64; its maximum magnitude in the data's type (no FP64 comparisons)
    using TS = typename std::conditional<std::is_same<TB, double>::value, double, float>::type;
    TS mx = 0;
    int bad = 0;
    for (int e = tid; e < r * r; e += nt) {
        const int k = e / r, c = e - k * r;
        const int s = S[k];
        TS x = 0;
        if (s < 0 || s >= pr.p) bad = 1; else x = (TS)basis[(int64_t)s * r + c];
        if (!isfinite(x)) bad = 2;
        M[e] = (double)x;
        mx = fmax(mx, fabs(x));
    }
    bad = __syncthreads_or(bad);
    {
        __shared__ TS sm[32];
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) sm[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            TS t = 0;
            for (int w = 0; w < (nt >> 5); ++w) t = fmax(t, sm[w]);
            s_max = (double)t;
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) {
            a.pstatus[pb] = bad == 2 ? CUR_ERR_NONFINITE : CUR_ERR_ARG;
            a.done[pb] = 1;
            set_status(a.status, bad == 2 ? CUR_ERR_NONFINITE : CUR_ERR_ARG);
        }
        return;
    }
    double lv = 0.0;
    const int sing = gj_inverse(M, r, colk, piv, (double)r * kEps * s_max, &lv);
    if (sing) {
        if (tid == 0) { a.pstatus[pb] = CUR_ERR_SINGULAR; a.done[pb] = 1; a.logvol[pb] = -INFINITY; }
        return;
    }
    if (tid == 0) a.logvol[pb] = lv;
    double* out64 = a.minv64 + (int64_t)pb * minv_stride(rs);
    for (int e = tid; e < r * r; e += nt) out64[e] = M[e];
    if (tid == 0) out64[r * r] = 0.0;   // fresh: no drift
}

// ---------------------------------------------------------------- the swap iteration

// The first CTA of a group keeps M^-1 (FP64) in shared memory when r <= kMsMax.
constexpr int kMsMax = 64;

// Layout: [B slice | M^-1 (compute type) | colj | wrow] or, with the B slice in global
// memory (a stage whose B does not fit in the shared memory of co-resident CTAs),
// [M^-1 | colj | wrow | staging of kEngStage C rows]; while M^-1 is being refactorised,
// [C(S,:) in FP64 | pivot column | pivots] over the same bytes (all dead then); after it
// the first CTA's MinvKeeper.
constexpr int kEngStage = 32;

template <typename TB>
struct EngineSmem {
    __host__ __device__ static size_t head(int nloc, int r, bool gmode = false) {
        const size_t b = gmode ? ((size_t)r * r + nloc + r + (size_t)kEngStage * r) * sizeof(TB)
                               : ((size_t)nloc * r + (size_t)r * r + nloc + r) * sizeof(TB);
        const size_t gj = ((size_t)r * r + r) * sizeof(double) + (size_t)r * sizeof(int);
        return ((b > gj ? b : gj) + 15) / 16 * 16;
    }
    static size_t bytes(int nloc, int r, bool gmode = false) {
        size_t b = head(nloc, r, gmode) + (size_t)12 * r * sizeof(double) + 64;   // keeper vectors
        if (r <= kMsMax) b += (size_t)r * r * sizeof(double);
        return b;
    }
};

// Key of a coefficient magnitude (x >= 0, or -1 for none) in the order of its value: FP32
// coefficients compare by their bits in the high word, FP64 ones by dkey. No FP64
// arithmetic either way.
__device__ __forceinline__ unsigned long long coef_key(float x) { return (unsigned long long)fkey(x) << 32; }
__device__ __forceinline__ unsigned long long coef_key(double x) { return dkey(x); }
__device__ __forceinline__ double coef_key_value(unsigned long long k, float) {
    const unsigned f = (unsigned)(k >> 32);
    return (double)__uint_as_float((f >> 31) ? (f & 0x7fffffffu) : ~f);
}
__device__ __forceinline__ double coef_key_value(unsigned long long k, double) { return dkey_value(k); }

// Local argmax of |B| over the slice in the compute type; ties to the lowest index.
template <typename TB>
__device__ __forceinline__ void engine_scan(const TB* Bs, int nloc, int r, int lo, unsigned long long& bk,
                                            long long& bi, int& nan) {
    TB v = (TB)-1;
    int idx = INT_MAX;
    int bad = 0;
    Walk2 w(threadIdx.x, blockDim.x, r);
    for (int e = threadIdx.x; e < nloc * r; e += blockDim.x, w.next()) {
        const TB x = fabs(Bs[e]);
        if (!(x <= (TB)INFINITY)) bad = 1;
        const int id = (lo + w.i) * r + w.c;
        if (x > v || (x == v && id < idx)) { v = x; idx = id; }
    }
    bk = idx == INT_MAX ? coef_key((TB)-INFINITY) : coef_key(v);
    bi = idx == INT_MAX ? LLONG_MAX : (long long)idx;
    nan = bad;
}

// The first CTA's copy of M^-1 and its Sherman-Morrison update. For FP32/BF16 data it
// is kept in double-float (two FP32 words per entry, error-free transformations on the
// FP32 pipes; GB300's FP64 units run at ~1/64 of FP32 with 64-cycle latency); for
// FP64 data it stays in FP64. |det| is tracked as mantissa * 2^exponent.
template <typename TB>
struct MinvKeeper;

template <>
struct MinvKeeper<float> {
    float* Mh;
    float* Ml;
    df64* crow;   // r: C(i*,:)
    df64* brow;   // r: row i* of B
    df64* cj;     // r: column j* of M^-1, then divided by B(i*,j*)
    df64* red;    // 8 r: eighth-sums of brow
    LogAcc lacc;
    __device__ void setup(unsigned char* base, int r, double* Mg, bool in_smem, float* gdf) {
        crow = reinterpret_cast<df64*>(base);
        brow = crow + r;
        cj = brow + r;
        red = cj + r;
        Mh = in_smem ? reinterpret_cast<float*>(red + 8 * r) : gdf;
        Ml = Mh + r * r;
        lacc.init();
    }
    __device__ void load(const double* Mg, int r) {
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
            const df64 v = df_from_d(Mg[e]);
            Mh[e] = v.h;
            Ml[e] = v.l;
        }
    }
    __device__ void store(double* Mg, int r) const {
        for (int e = threadIdx.x; e < r * r; e += blockDim.x) Mg[e] = df_to_d(df64{Mh[e], Ml[e]});
    }
    __device__ float value(int e) const { return __fadd_rn(Mh[e], Ml[e]); }
    // The update for the winner (i*, j*) with C row `ci`, in four phases that the engine
    // separates by barriers and overlaps with its own work: load the row and column j* of
    // M^-1; the partial sums of the row i* of B = C(i*,:) M^-1; that row, B(i*,j*) and the
    // column divided by it (and the |det| factor); the rank-1 update of M^-1.
    __device__ void swap_load(const float* ci, int r, int jstar) {
        for (int c = threadIdx.x; c < r; c += blockDim.x) {
            crow[c] = df64{ci[c], 0.f};
            cj[c] = df64{Mh[c * r + jstar], Ml[c * r + jstar]};
        }
    }
    // brow = crow M^-1: eight partial sums per column, so each dependent chain is r/8 long
    __device__ void swap_partials(int r) {
        for (int it = threadIdx.x; it < 8 * r; it += blockDim.x) {
            const int c = it % r, qt = it / r;
            df64 s{0.f, 0.f};
            for (int k = r * qt / 8; k < r * (qt + 1) / 8; ++k)
                s = df_add(s, df_mul_f(df64{Mh[k * r + c], Ml[k * r + c]}, crow[k].h));
            red[qt * r + c] = s;
        }
    }
    __device__ df64 row_sum(int r, int c) const {
        return df_add(df_add(df_add(red[c], red[r + c]), df_add(red[2 * r + c], red[3 * r + c])),
                      df_add(df_add(red[4 * r + c], red[5 * r + c]), df_add(red[6 * r + c], red[7 * r + c])));
    }
    // every thread that needs B(i*,j*) forms the same sum as the thread of column j*
    __device__ void swap_finish_row(int r, int jstar) {
        const int tid = threadIdx.x, nt = blockDim.x;
        for (int c = tid; c < r; c += nt) {
            brow[c] = row_sum(r, c);
            cj[c] = df_div(cj[c], row_sum(r, jstar));
        }
        if (tid == nt - 1) lacc.mul(row_sum(r, jstar));
    }
    // M^-1 <- M^-1 - (M^-1(:,j) / B_ij) (B(i,:) - e_j^T)
    __device__ void swap_update(int r, int jstar) {
        const int tid = threadIdx.x, nt = blockDim.x;
        if (nt % r == 0) {   // one column per thread, four rows at a time
            const int c = tid % r, di = nt / r;
            const df64 wv = c == jstar ? df_sub(brow[c], df64{1.f, 0.f}) : brow[c];
            int i = tid / r;
            for (; i + 3 * di < r; i += 4 * di) {
                df64 m[4], q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = (i + u * di) * r + c;
                    m[u] = df64{Mh[e], Ml[e]};
                    q[u] = cj[i + u * di];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = (i + u * di) * r + c;
                    const df64 mv = df_sub(m[u], df_mul(q[u], wv));
                    Mh[e] = mv.h;
                    Ml[e] = mv.l;
                }
            }
            for (; i < r; i += di) {
                const int e = i * r + c;
                const df64 mv = df_sub(df64{Mh[e], Ml[e]}, df_mul(cj[i], wv));
                Mh[e] = mv.h;
                Ml[e] = mv.l;
            }
        } else {
            Walk2 w(tid, nt, r);
            for (int e = tid; e < r * r; e += nt, w.next()) {
                const df64 wv = w.c == jstar ? df_sub(brow[w.c], df64{1.f, 0.f}) : brow[w.c];
                const df64 mv = df_sub(df64{Mh[e], Ml[e]}, df_mul(cj[w.i], wv));
                Mh[e] = mv.h;
                Ml[e] = mv.l;
            }
        }
    }
    __device__ double dlog() const { return lacc.log_value(); }
};

template <>
struct MinvKeeper<double> {
    double* M;
    double* crow;
    double* brow;
    double* cj;
    double* red;
    LogAcc lacc;
    __device__ void setup(unsigned char* base, int r, double* Mg, bool in_smem, float*) {
        crow = reinterpret_cast<double*>(base);
        brow = crow + r;
        cj = brow + r;
        red = cj + r;
        M = in_smem ? red + 8 * r : Mg;
        lacc.init();
    }
    __device__ void load(const double* Mg, int r) {
        if (M != Mg)
            for (int e = threadIdx.x; e < r * r; e += blockDim.x) M[e] = Mg[e];
    }
    __device__ void store(double* Mg, int r) const {
        if (M != Mg)
            for (int e = threadIdx.x; e < r * r; e += blockDim.x) Mg[e] = M[e];
    }
    __device__ double value(int e) const { return M[e]; }
    __device__ void swap_load(const double* ci, int r, int jstar) {
        for (int c = threadIdx.x; c < r; c += blockDim.x) {
            crow[c] = ci[c];
            cj[c] = M[c * r + jstar];
        }
    }
    __device__ void swap_partials(int r) {
        for (int it = threadIdx.x; it < 8 * r; it += blockDim.x) {
            const int c = it % r, qt = it / r;
            double s = 0.0;
            for (int k = r * qt / 8; k < r * (qt + 1) / 8; ++k) s = fma(crow[k], M[k * r + c], s);
            red[qt * r + c] = s;
        }
    }
    __device__ double row_sum(int r, int c) const {
        return (((red[c] + red[r + c]) + (red[2 * r + c] + red[3 * r + c])) +
                ((red[4 * r + c] + red[5 * r + c]) + (red[6 * r + c] + red[7 * r + c])));
    }
    __device__ void swap_finish_row(int r, int jstar) {
        const int tid = threadIdx.x, nt = blockDim.x;
        for (int c = tid; c < r; c += nt) brow[c] = row_sum(r, c);
        if (tid == nt - 1) lacc.mul(df_from_d(row_sum(r, jstar)));
    }
    __device__ void swap_update(int r, int jstar) {
        const int tid = threadIdx.x, nt = blockDim.x;
        const double bb = brow[jstar];
        Walk2 w(tid, nt, r);
        for (int e = tid; e < r * r; e += nt, w.next()) {
            const double wv = brow[w.c] - (w.c == jstar ? 1.0 : 0.0);
            M[e] -= cj[w.i] * wv / bb;
        }
    }
    __device__ double dlog() const { return lacc.log_value(); }
};

// M^-1 of C(S,:) from scratch (FP64 Gauss-Jordan, the singularity rule of the start
// factorisation) into the keeper; W, colk, piv: shared scratch of r*r + r doubles and
// r ints. Returns 1 if C(S,:) is numerically singular. All threads of the CTA call it.
template <typename TB>
__device__ int engine_refactor(MinvKeeper<TB>& keep, const TB* basis, const int32_t* S, int r,
                               double* W, double* colk, int* piv, double* lv) {
    double mx = 0.0;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int k = e / r, c = e - k * r;
        const double x = to_d(basis[(int64_t)S[k] * r + c]);
        W[e] = x;
        mx = fmax(mx, fabs(x));
    }
    mx = block_max(mx);
    const int sing = gj_inverse(W, r, colk, piv, (double)r * kEps * mx, lv);
    if (!sing) {
        keep.load(W, r);
        if (threadIdx.x == 0) keep.lacc.init();
    }
    __syncthreads();
    return sing;
}

// kappa_inf(M) = ||C(S,:)||_inf ||M^-1||_inf with the kept inverse (all threads call it).
// It only scales the drift bound, so FP32 data sums in FP32 (no FP64 pipe work).
template <typename TB>
__device__ double engine_kappa(const MinvKeeper<TB>& keep, const TB* basis, const int32_t* S, int r) {
    using TS = typename std::conditional<std::is_same<TB, double>::value, double, float>::type;
    TS sm = 0, sx = 0;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = threadIdx.x >> 5; k < r; k += nw) {   // a warp per row
        TS a = 0, x = 0;
        const TB* row = basis + (int64_t)S[k] * r;
        for (int c = lane; c < r; c += 32) {
            a += fabs((TS)row[c]);
            x += fabs((TS)keep.value(k * r + c));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            x += __shfl_xor_sync(0xffffffffu, x, o);
        }
        sm = fmax(sm, a);
        sx = fmax(sx, x);
    }
    __shared__ TS s_m[32], s_x[32];
    const int warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { s_m[warp] = sm; s_x[warp] = sx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        TS m = 0, x = 0;
        for (int w = 0; w < nw; ++w) { m = fmax(m, s_m[w]); x = fmax(x, s_x[w]); }
        s_m[0] = m;
        s_x[0] = x;
    }
    __syncthreads();
    const double kap = (double)s_m[0] * (double)s_x[0];
    __syncthreads();
    return kap;
}

// Refresh of an FP32 B slice: B = C M^-1 for nloc rows (r = 32 or 64), the
// product of the engine's cycles after the first. C rows pass through shared memory
// (coalesced loads) in chunks of 8 rows per warp, staged in the chunk's own rows of B; each
// thread forms an 8 x (r/32) register tile (rows warp-uniform, columns lane + 32 j) with the
// C values read four k at a time as one broadcast 16-byte load, so a warp issues 8 + 4 r/32
// shared loads per 32 r/32 FMAs instead of two loads per FMA. Each entry is still one FMA
// chain over k in order, as a dot product.
template <int TN>
__device__ __noinline__ void refresh_tiled_tn(float* Bs, const float* Mi, const float* Cs, int nloc, int r) {
    constexpr int TM = 8;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int chunk = TM * nw;
    for (int i0 = 0; i0 < nloc; i0 += chunk) {
        const int nr = min(chunk, nloc - i0);
        float* stage = Bs + (size_t)i0 * r;
        for (int e = tid; e < nr * r; e += nt) stage[e] = Cs[(int64_t)i0 * r + e];
        __syncthreads();
        float acc[TM][TN];
#pragma unroll
        for (int q = 0; q < TM; ++q)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[q][j] = 0.f;
        const float* crow[TM];
#pragma unroll
        for (int q = 0; q < TM; ++q) crow[q] = stage + (size_t)min(warp * TM + q, nr - 1) * r;   // rows past nr: not stored
        for (int k = 0; k < r; k += 4) {
            float4 cv[TM];
#pragma unroll
            for (int q = 0; q < TM; ++q) cv[q] = *reinterpret_cast<const float4*>(crow[q] + k);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float mv[TN];
#pragma unroll
                for (int j = 0; j < TN; ++j) mv[j] = Mi[(k + kk) * r + lane + 32 * j];
#pragma unroll
                for (int q = 0; q < TM; ++q) {
                    const float c = kk == 0 ? cv[q].x : kk == 1 ? cv[q].y : kk == 2 ? cv[q].z : cv[q].w;
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[q][j] = fmaf(c, mv[j], acc[q][j]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TM; ++q) {
            const int i = warp * TM + q;
            if (i < nr)
#pragma unroll
                for (int j = 0; j < TN; ++j) stage[(size_t)i * r + lane + 32 * j] = acc[q][j];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void engine_refresh_tiled(float* Bs, const float* Mi, const float* Cs, int nloc, int r) {
    if (r == 32) refresh_tiled_tn<1>(Bs, Mi, Cs, nloc, r);
    else refresh_tiled_tn<2>(Bs, Mi, Cs, nloc, r);
}

// Problems that one CTA holds alone run with kSoloThreads threads (their swaps never wait on
// another CTA, so more threads only shorten each swap); groups of CTAs with 256 each.
constexpr int kSoloThreads = 512;

template <typename TB>
__global__ void __launch_bounds__(kSoloThreads, 1) mv_engine(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int slot = a.cta_base + blockIdx.x;
    const int pb = a.cta_prob[slot], part = a.cta_part[slot];
    if (a.done[pb]) return;
    const MvProb pr = a.prob[pb];
    const int r = pr.r, rs = a.r, G = pr.G, tid = threadIdx.x, nt = blockDim.x;
    const bool solo = G == 1;                   // one CTA: no inter-CTA exchange at all
    const int lo = part * pr.rpc, hi = min(pr.p, lo + pr.rpc), nloc = max(0, hi - lo);
    const bool gmode = a.bglob != nullptr && pr.gmode;
    TB* Bs = gmode ? static_cast<TB*>(a.bglob) + pr.boff + (int64_t)lo * r   // nloc x r slice of B
                   : reinterpret_cast<TB*>(smem_raw);
    TB* Mi = gmode ? reinterpret_cast<TB*>(smem_raw) : Bs + (size_t)nloc * r;   // r x r: M^-1 (compute type)
    TB* colj = Mi + (size_t)r * r;              // nloc
    TB* wrow = colj + nloc;                     // r: winning row of B, then B(i,:) - e_j
    TB* cstage = wrow + r;                      // global-memory mode: kEngStage C rows
    const size_t off = EngineSmem<TB>::head(nloc, r, gmode);
    double* Mg = a.minv64 + (int64_t)pb * minv_stride(rs);      // M^-1 in global memory (FP64)
    __shared__ long long s_w;
    __shared__ int s_nan, s_go;
    __shared__ MinvKeeper<TB> keep;
    __shared__ int32_t S0[128];      // the start set, restored if C(S,:) turns singular (unless kept)
    __shared__ double s_lv0;         // log|det| of the last factorisation
    __shared__ double s_drift;       // sum of swaps * kappa(M) since the last factorisation
    TB* pub = static_cast<TB*>(a.pub);
    const TB* basis = static_cast<const TB*>(a.basis) + pr.boff;
    const int myslot = pr.group0 + part;
    if (part == 0) {
        if (tid == 0)
            keep.setup(smem_raw + off, r, Mg, r <= kMsMax, a.mdf ? a.mdf + (int64_t)pb * 2 * rs * rs : nullptr);
        __syncthreads();
        keep.load(Mg, r);
        for (int k = tid; k < r; k += nt) S0[k] = a.S[(int64_t)pb * rs + k];
        // the inverse arrives with its drift bound (0 when just factorised)
        if (tid == 0) { s_lv0 = a.logvol[pb]; s_drift = Mg[(size_t)r * r]; }
    }
    int32_t* Sg = a.S + (int64_t)pb * rs;
    double* gjw = reinterpret_cast<double*>(smem_raw);   // refactorisation scratch over the B slice
    // First CTA only: M^-1 of C(S,:) afresh into the keeper; 1 if C(S,:) is singular.
    auto refactor = [&]() -> int {
        double lv = 0.0;
        const int sing = engine_refactor(keep, basis, Sg, r, gjw, gjw + (size_t)r * r,
                                         reinterpret_cast<int*>(gjw + (size_t)r * r + r), &lv);
        if (tid == 0 && !sing) { s_lv0 = lv; s_drift = 0.0; }
        if (tid == 0 && a.nrefactor) atomicAdd(a.nrefactor, 1);
        __syncthreads();
        return sing;
    };

    unsigned long long bk;   // argmax |B_ij| as an order key (coef_key), its flat index, a NaN seen
    long long bi;
    int nan;
    int par = 0, total = a.swaps[pb], made_last = 0;
    bool first_cycle = true;
    unsigned epoch = 0;
    int fin = 0, fstat = CUR_OK;
    auto publish = [&](int pp) {
        if (solo) return;
        if (tid == 0) {
            a.keyv[myslot * 2 + pp] = coef_key_value(bk, TB{});
            a.keyi[myslot * 2 + pp] = nan ? -2LL : bi;
        }
        if (!nan && bi != LLONG_MAX) {
            const int il = (int)(bi / r) - lo;
            for (int c = tid; c < r; c += nt) pub[((int64_t)myslot * 2 + pp) * rs + c] = Bs[il * r + c];
        }
    };
    // The swap test max|B_ij| > 1 + delta on order keys: for FP32 coefficients x > t holds
    // exactly when x exceeds the largest float <= t; group keys are of the published doubles.
    const unsigned long long thr_own = std::is_same<TB, double>::value
                                           ? dkey(1.0 + a.delta) : coef_key((TB)__double2float_rd(1.0 + a.delta));
    const unsigned long long thr_grp = dkey(1.0 + a.delta);
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    __shared__ unsigned long long r_k[32];
    __shared__ long long r_i[32];
    __shared__ int r_n[32];
    // The CTA's argmax of the threads' (bk, bi) and its NaN flag, then the decision for the
    // next swap in s_go (1 swap, 0 converged, -1 swap cap), s_w (winner) and s_nan: a solo
    // CTA decides on its own argmax (two barriers in all); a group publishes it, meets at
    // the group barrier and decides on the group's. False if the group barrier timed out.
    auto reduce_decide = [&]() -> bool {
        warp_argmax_key(bk, bi);
        const int wn = __any_sync(0xffffffffu, nan);
        if (lane == 0) { r_k[warp] = bk; r_i[warp] = bi; r_n[warp] = wn; }
        __syncthreads();
        if (warp == 0) {
            unsigned long long k = lane < nw ? r_k[lane] : 0ull;
            long long i = lane < nw ? r_i[lane] : LLONG_MAX;
            const int n = __any_sync(0xffffffffu, lane < nw ? r_n[lane] : 0);
            warp_argmax_key(k, i);
            if (lane == 0) {
                r_k[0] = k;
                r_i[0] = i;
                r_n[0] = n;
                if (solo) {
                    s_nan = n;
                    s_w = i;
                    s_go = (i == LLONG_MAX || !(k > thr_own)) ? 0 : (total >= a.max_swaps ? -1 : 1);
                }
            }
        }
        __syncthreads();
        if (solo) return true;
        bk = r_k[0];
        bi = r_i[0];
        nan = r_n[0];
        publish(par);
        ++epoch;
        if (!group_barrier(&a.bar[pb], (unsigned)G * epoch, a.status)) return false;
        if (tid < 32) {
            unsigned long long wk = dkey(-INFINITY);
            long long wi = LLONG_MAX;
            int anynan = 0;
            for (int g = tid; g < G; g += 32) {
                const long long ki = a.keyi[(pr.group0 + g) * 2 + par];
                const unsigned long long kv = dkey(a.keyv[(pr.group0 + g) * 2 + par]);
                if (ki == -2LL) anynan = 1;
                else if (better_key(kv, ki, wk, wi)) { wk = kv; wi = ki; }
            }
            anynan = __any_sync(0xffffffffu, anynan);
            warp_argmax_key(wk, wi);
            if (tid == 0) {
                s_nan = anynan;
                s_w = wi;
                s_go = (wi == LLONG_MAX || !(wk > thr_grp)) ? 0 : (total >= a.max_swaps ? -1 : 1);
            }
        }
        __syncthreads();
        return true;
    };
    while (true) {
        // refresh: B slice = C slice M^-1
        __syncthreads();
        if (part == 0) {
            for (int e = tid; e < r * r; e += nt) Mi[e] = (TB)keep.value(e);
        } else {
            for (int e = tid; e < r * r; e += nt) Mi[e] = (TB)Mg[e];
        }
        __syncthreads();
        bool tiled = false;
        if constexpr (std::is_same<TB, float>::value) {
            tiled = !(a.bpre && first_cycle) && !gmode && (r == 32 || r == 64);
            if (tiled) engine_refresh_tiled(Bs, Mi, basis + (int64_t)lo * r, nloc, r);
        }
        if (tiled) {
        } else if (a.bpre && first_cycle) {
            // the first cycle's B slice was formed on the tensor cores from the same M^-1
            const TB* src = static_cast<const TB*>(a.bpre) + pr.boff + (int64_t)lo * r;
            for (int e = tid; e < nloc * r; e += nt) Bs[e] = src[e];
        } else {
            // C rows pass through shared memory a chunk at a time (coalesced loads), then
            // B rows = C rows M^-1 with 8 outputs per thread in registers; the chunk's
            // own rows of Bs serve as the staging area (a separate one when B is global).
            const TB* Cs = basis + (int64_t)lo * r;
            const int chunk = max(1, min(kEngStage, 8 * nt / r));
            for (int i0 = 0; i0 < nloc; i0 += chunk) {
                const int nr = min(chunk, nloc - i0);
                TB* stage = gmode ? cstage : Bs + (size_t)i0 * r;
                for (int e = tid; e < nr * r; e += nt) stage[e] = Cs[(int64_t)i0 * r + e];
                __syncthreads();
                TB out[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = tid + u * nt;
                    TB sum = (TB)0;
                    if (e < nr * r) {
                        const int i = e / r, c = e - i * r;
                        const TB* ci = stage + (size_t)i * r;
                        for (int k = 0; k < r; ++k) sum = fma(ci[k], Mi[k * r + c], sum);
                    }
                    out[u] = sum;
                }
                __syncthreads();
                TB* dst = Bs + (size_t)i0 * r;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = tid + u * nt;
                    if (e < nr * r) dst[e] = out[u];
                }
                __syncthreads();
            }
        }
        first_cycle = false;
        __syncthreads();
        engine_scan(Bs, nloc, r, lo, bk, bi, nan);
        if (!reduce_decide()) { fin = 3; fstat = CUR_ERR_TIMEOUT; break; }
        int made = 0;
        while (true) {
            if (s_nan) { fin = 3; fstat = CUR_ERR_NONFINITE; break; }
            if (s_go == 0) { fin = made == 0 ? 1 : 2; break; }
            if (s_go < 0) { fin = 3; fstat = CUR_ERR_NOCONV; break; }
            const long long wi = s_w;
            const int istar = (int)(wi / r), jstar = (int)(wi - (long long)istar * r);
            const int owner = istar / pr.rpc;
            const TB* wsrc = solo ? Bs + (size_t)(istar - lo) * r
                                  : pub + ((int64_t)(pr.group0 + owner) * 2 + par) * rs;
            // the winner's row of B; the first CTA's update of M^-1 runs in four phases
            // between these barriers (see MinvKeeper)
            for (int c = tid; c < r; c += nt) wrow[c] = wsrc[c];
            if (part == 0) {
                keep.swap_load(basis + (int64_t)istar * r, r, jstar);
                if (tid == 0) a.S[(int64_t)pb * rs + jstar] = istar;
            }
            __syncthreads();
            const TB b = wrow[jstar];
            for (int i = tid; i < nloc; i += nt) colj[i] = Bs[i * r + jstar] / b;
            if (part == 0) keep.swap_partials(r);
            __syncthreads();
            if (part == 0) keep.swap_finish_row(r, jstar);
            __syncthreads();
            ++made;
            ++total;
            if (part == 0) keep.swap_update(r, jstar);
            // B <- B - (B(:,j) / B_ij) (B(i,:) - e_j^T), fused with the next local argmax
            {
                TB v = (TB)-1;
                int idx = INT_MAX, bad = 0;
                if (nt % r == 0) {
                    // each thread keeps one column (r divides the block): B(i,:) - e_j is read
                    // once, and its ids only grow, so the first maximum is the lowest id
                    const int c = tid % r, di = nt / r;
                    const TB wc = c == jstar ? wrow[c] - (TB)1 : wrow[c];
                    int i = tid / r, id = (lo + i) * r + c;
                    TB* bp = Bs + (size_t)i * r + c;
                    const size_t step = (size_t)di * r;
                    // four rows at a time: their loads issue before the arithmetic
                    for (; i + 3 * di < nloc; i += 4 * di, id += 4 * di * r, bp += 4 * step) {
                        const TB c0 = colj[i], c1 = colj[i + di], c2 = colj[i + 2 * di], c3 = colj[i + 3 * di];
                        const TB b0 = bp[0], b1 = bp[step], b2 = bp[2 * step], b3 = bp[3 * step];
                        const TB x0 = fma(-c0, wc, b0), x1 = fma(-c1, wc, b1), x2 = fma(-c2, wc, b2), x3 = fma(-c3, wc, b3);
                        bp[0] = x0;
                        bp[step] = x1;
                        bp[2 * step] = x2;
                        bp[3 * step] = x3;
                        const TB a0 = fabs(x0), a1 = fabs(x1), a2 = fabs(x2), a3 = fabs(x3);
                        bad |= !(a0 <= (TB)INFINITY) | !(a1 <= (TB)INFINITY) | !(a2 <= (TB)INFINITY) | !(a3 <= (TB)INFINITY);
                        if (a0 > v) { v = a0; idx = id; }
                        if (a1 > v) { v = a1; idx = id + di * r; }
                        if (a2 > v) { v = a2; idx = id + 2 * di * r; }
                        if (a3 > v) { v = a3; idx = id + 3 * di * r; }
                    }
                    for (; i < nloc; i += di, id += di * r, bp += step) {
                        const TB x = fma(-colj[i], wc, *bp);
                        *bp = x;
                        const TB ax = fabs(x);
                        bad |= !(ax <= (TB)INFINITY);
                        if (ax > v) { v = ax; idx = id; }
                    }
                } else {
                    Walk2 w(tid, nt, r);
                    for (int e = tid; e < nloc * r; e += nt, w.next()) {
                        const TB wc = w.c == jstar ? wrow[w.c] - (TB)1 : wrow[w.c];
                        const TB x = fma(-colj[w.i], wc, Bs[e]);
                        Bs[e] = x;
                        const TB ax = fabs(x);
                        if (!(ax <= (TB)INFINITY)) bad = 1;
                        const int id = (lo + w.i) * r + w.c;
                        if (ax > v || (ax == v && id < idx)) { v = ax; idx = id; }
                    }
                }
                bk = idx == INT_MAX ? coef_key((TB)-INFINITY) : coef_key(v);
                bi = idx == INT_MAX ? LLONG_MAX : (long long)idx;
                nan = bad;
            }
            par ^= 1;
            if (!reduce_decide()) { fin = 3; fstat = CUR_ERR_TIMEOUT; break; }
            if (made == r) { fin = 2; break; }
        }
        made_last = made;
        if (fin != 2) break;
        // A new cycle starts from M = C(S,:) factorised afresh once the Sherman-Morrison
        // updates carried since the last factorisation may have drifted: each swap adds
        // about kappa(M) u (u = unit roundoff of the kept inverse) to the refreshed B. With
        // drift_max = 0 (FP64 data) every cycle refactorises, as the iteration is stated;
        // for FP32 B the bound 2^18 keeps the drift below 2^-30. The first CTA decides and
        // refactorises; every CTA then refreshes from its M^-1.
        int sing = 0;
        if (part == 0) {
            __syncthreads();
            double drift = 0.0;
            if (a.drift_max > 0.0) {
                const double kap = engine_kappa(keep, basis, Sg, r);
                if (tid == 0) s_drift += (double)made * kap;
                __syncthreads();
                drift = s_drift;
            }
            if (a.drift_max <= 0.0 || !(drift <= a.drift_max)) {
                sing = refactor();
                if (tid == 0 && sing) a.pstatus[pb] = CUR_ERR_SINGULAR;   // seen by the group after the barrier
            }
            if (!solo && !sing) keep.store(Mg, r);
        }
        if (!solo) {
            ++epoch;
            if (!group_barrier(&a.bar[pb], (unsigned)G * epoch, a.status)) { fin = 3; fstat = CUR_ERR_TIMEOUT; break; }
            if (part != 0) sing = *reinterpret_cast<volatile int32_t*>(a.pstatus + pb) == CUR_ERR_SINGULAR;
        }
        if (sing) { fin = 3; fstat = CUR_ERR_SINGULAR; break; }
        fin = 0;
    }
    if (part == 0) {
        __syncthreads();
        // the stored inverse (inherited by merge nodes and later sweeps) leaves with its
        // drift bound, never above drift_max; only the swap cap can end a cycle with swaps
        if (fin == 3 && fstat == CUR_ERR_NOCONV && made_last > 0) {
            double drift = 0.0;
            if (a.drift_max > 0.0) {
                const double kap = engine_kappa(keep, basis, Sg, r);
                if (tid == 0) s_drift += (double)made_last * kap;
                __syncthreads();
                drift = s_drift;
            }
            if ((a.drift_max <= 0.0 || !(drift <= a.drift_max)) && refactor()) fstat = CUR_ERR_SINGULAR;
        }
        const bool sing = fin == 3 && fstat == CUR_ERR_SINGULAR;
        if (sing) {
            if (!a.keep_singular_set)
                for (int k = tid; k < r; k += nt) a.S[(int64_t)pb * rs + k] = S0[k];
        } else {
            keep.store(Mg, r);
            if (tid == 0) Mg[(size_t)r * r] = s_drift;
        }
        if (tid == 0) {
            a.swaps[pb] = total;
            a.logvol[pb] = sing ? -INFINITY : s_lv0 + keep.dlog();
            a.done[pb] = 1;
            a.pstatus[pb] = fin == 1 ? CUR_OK : fstat;
            if (fin == 3 && fstat != CUR_ERR_NOCONV && fstat != CUR_ERR_SINGULAR) set_status(a.status, fstat);
        }
    }
}

// dst = src^T (r x r), with the drift bound that follows the matrix.
__global__ void mv_transpose(const double* src, int r, double* dst) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= r * r; e += gridDim.x * blockDim.x) {
        const int a = e / r, b = e - a * r;
        dst[e] = e == r * r ? src[e] : src[b * r + a];
    }
}

// Global ids of the selected rows: out[pb * r + k] = gid(S[pb][k]).
__global__ void mv_emit(const MvProb* prob, const int32_t* S, int P, int r, int32_t* out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * r; e += gridDim.x * blockDim.x) {
        const int pb = e / r;
        const MvProb pr = prob[pb];
        const int s = S[e];
        out[e] = pr.gid_arr ? pr.gid_arr[s] : (int32_t)(pr.gid_base + s);
    }
}

// Local start positions from global ids: S[pb*r + k] = gid_start[pb*r + k] - gid_base.
__global__ void mv_set_start(const MvProb* prob, const int32_t* gstart, int P, int r, int32_t* S,
                             int* status) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * r; e += gridDim.x * blockDim.x) {
        const int pb = e / r;
        const MvProb pr = prob[pb];
        const int64_t s = (int64_t)gstart[e] - pr.gid_base;
        if (s < 0 || s >= pr.p) { set_status(status, CUR_ERR_ARG); S[e] = 0; }
        else S[e] = (int32_t)s;
    }
}

// S[pb*r + k] = off + k
__global__ void mv_iota(int32_t* S, int P, int r, int off) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * r; e += gridDim.x * blockDim.x)
        S[e] = off + (e % r);
}

// Pad idx (r entries, count valid, -1 after) with the lowest unused ids < size.
// log|det basis(rows,:)| (r x r) by LU with partial pivoting (first maximum |a_ik|,
// i >= k), the log-volume of Definition 1 for a set that may be numerically singular:
// a pivot that is exactly zero gives -inf, any other pivot counts however small.
template <typename TB>
__device__ void logvol_rows_dev(const TB* basis, int64_t p, int r, const int32_t* rows, double* out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* M = reinterpret_cast<double*>(smem_raw);
    __shared__ int s_p, s_zero;
    __shared__ double s_dinv;
    __shared__ LogAcc s_acc;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < r * r; e += nt) {
        const int k = e / r, c = e - k * r;
        const int64_t i = rows[k];
        M[e] = (i >= 0 && i < p) ? to_d(basis[i * r + c]) : 0.0;   // a row outside: a zero row
    }
    if (tid == 0) { s_zero = 0; s_acc.init(); }
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (tid < 32) {
            // first maximum |m_ik|, compared as integer keys (no FP64 comparisons)
            unsigned long long bk = 0ull;
            long long bi = k;
            for (int i = k + tid; i < r; i += 32) {
                const unsigned long long x = dkey(fabs(M[i * r + k]));
                if (x > bk) { bk = x; bi = i; }
            }
            warp_argmax_key(bk, bi);
            if (tid == 0) s_p = (int)bi;
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < r; j += nt) {
                const double t = M[k * r + j];
                M[k * r + j] = M[p * r + j];
                M[p * r + j] = t;
            }
        __syncthreads();
        const double d = M[k * r + k];
        if (d == 0.0 || !isfinite(d)) {
            if (tid == 0) s_zero = 1;
            continue;   // no elimination past a zero pivot (uniform: d is read by all)
        }
        if (tid == 0) { s_acc.mul(df_from_d(d)); s_dinv = 1.0 / d; }   // multipliers by the reciprocal, as LAPACK's LU
        __syncthreads();
        const double dinv = s_dinv;
        for (int i = k + 1 + tid; i < r; i += nt) M[i * r + k] *= dinv;
        __syncthreads();
        if (nt % r == 0) {   // one column per thread
            const int c = tid % r, di = nt / r;
            if (c > k) {
                const double akc = M[k * r + c];
                for (int i = k + 1 + (tid / r); i < r; i += di) M[i * r + c] = fma(-M[i * r + k], akc, M[i * r + c]);
            }
        } else {
            const int w = r - k - 1;
            for (int e = tid; e < w * w; e += nt) {
                const int i = k + 1 + e / w, j = k + 1 + e % w;
                M[i * r + j] = fma(-M[i * r + k], M[k * r + j], M[i * r + j]);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) *out = s_zero ? -INFINITY : s_acc.log_value();
}

template <typename TB>
__global__ void __launch_bounds__(512) logvol_rows_k(const TB* basis, int64_t p, int r, const int32_t* rows,
                                                     double* out) {
    logvol_rows_dev<TB>(basis, p, r, rows, out);
}

__global__ void pad_indices_k(int32_t* idx, const int32_t* count, int r, int64_t size) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int fill = *count;
    for (int64_t cand = 0; cand < size && fill < r; ++cand) {
        bool used = false;
        for (int q = 0; q < fill; ++q) used |= (idx[q] == cand);
        if (!used) idx[fill++] = (int32_t)cand;
    }
}

// ---------------------------------------------------------------- host side

static const size_t kSmemBudget = 200 * 1024;
static const int kSpreadRows = 64;   // fewest rows per CTA of a spread group

template <typename TB>
static int rows_cap(int r) {
    int lo = 1, hi = 1 << 20;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (EngineSmem<TB>::bytes(mid, r) <= kSmemBudget && StartSmem<TB>::bytes(mid, r) <= kSmemBudget) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename K>
static cur_status set_smem_attr(K* fn, size_t bytes) {
    CUR_TRY(smem_attr((const void*)fn, bytes));
    return CUR_OK;
}

static inline unsigned nblk(int64_t n, int t = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535));
}

// ---------------------------------------------------------------- uploads without waiting
//
// The stage tables (problem descriptors, CTA slots) are known on the host from the shapes
// alone. They reach the device as the parameters of a copy kernel: the launch takes its
// own copy of the parameters, so no host buffer has to outlive the call and the host
// never waits for the GPU before reusing one.
// Two parameter sizes: one short launch for the common small table, few launches of nearly
// the 32 KB parameter limit for the tables of large batches.
template <int N>
struct __align__(16) Blob {
    unsigned char* dst;
    int bytes;
    int pad;
    unsigned char data[N];
};
// 16-byte words where the destination allows (every table is 16-byte aligned in the arena),
// so a 30 KB parameter takes ~2000 reads instead of 30000.
template <int N>
__global__ void blob_k(const __grid_constant__ Blob<N> b) {
    const int nw = ((uintptr_t)b.dst % 16 == 0) ? b.bytes / 16 : 0;
    const uint4* src = reinterpret_cast<const uint4*>(b.data);
    uint4* dst = reinterpret_cast<uint4*>(b.dst);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    for (int i = 16 * nw + threadIdx.x; i < b.bytes; i += blockDim.x) b.dst[i] = b.data[i];
}
template <int N>
static cur_status upload_n(unsigned char* dst, const unsigned char* src, size_t bytes, cudaStream_t st) {
    Blob<N> b;
    for (size_t off = 0; off < bytes; off += N) {
        const size_t n = std::min<size_t>(N, bytes - off);
        b.dst = dst + off;
        b.bytes = (int)n;
        std::memcpy(b.data, src + off, n);
        blob_k<N><<<1, 256, 0, st>>>(b);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    return CUR_OK;
}
static cur_status upload(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    unsigned char* d = static_cast<unsigned char*>(dst);
    const unsigned char* s = static_cast<const unsigned char*>(src);
    if (bytes <= 2048) return upload_n<2048>(d, s, bytes, st);
    return upload_n<30720>(d, s, bytes, st);
}

// Several small tables in one launch: segment q goes to dst[q] from data + off[q] (offsets
// 16-byte aligned, so 16-byte words wherever the destination is aligned too).
constexpr int kUpSegs = 6;
template <int N>
struct __align__(16) BlobM {
    unsigned char* dst[kUpSegs];
    int off[kUpSegs];
    int bytes[kUpSegs];
    int nseg;
    int pad[3];
    unsigned char data[N];
};
template <int N>
__global__ void blobm_k(const __grid_constant__ BlobM<N> b) {
    for (int q = 0; q < b.nseg; ++q) {
        const int nw = ((uintptr_t)b.dst[q] % 16 == 0) ? b.bytes[q] / 16 : 0;
        const uint4* src = reinterpret_cast<const uint4*>(b.data + b.off[q]);
        uint4* dst = reinterpret_cast<uint4*>(b.dst[q]);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
        for (int i = 16 * nw + threadIdx.x; i < b.bytes[q]; i += blockDim.x) b.dst[q][i] = b.data[b.off[q] + i];
    }
}
struct UpSeg {
    void* dst;
    const void* src;
    size_t bytes;
};
template <int N>
static cur_status upload_multi_n(const UpSeg* seg, int n, cudaStream_t st) {
    BlobM<N> b;
    b.nseg = n;
    int off = 0;
    for (int q = 0; q < n; ++q) {
        b.dst[q] = static_cast<unsigned char*>(seg[q].dst);
        b.off[q] = off;
        b.bytes[q] = (int)seg[q].bytes;
        std::memcpy(b.data + off, seg[q].src, seg[q].bytes);
        off += (int)((seg[q].bytes + 15) / 16 * 16);
    }
    blobm_k<N><<<1, 256, 0, st>>>(b);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}
static cur_status upload_multi(std::initializer_list<UpSeg> segs, cudaStream_t st) {
    UpSeg v[kUpSegs];
    int n = 0;
    size_t tot = 0;
    for (const UpSeg& q : segs) {
        if (q.bytes == 0) continue;
        if (n == kUpSegs) return CUR_ERR_ARG;
        v[n++] = q;
        tot += (q.bytes + 15) / 16 * 16;
    }
    if (n == 0) return CUR_OK;
    if (tot <= 2048) return upload_multi_n<2048>(v, n, st);
    if (tot <= 30720) return upload_multi_n<30720>(v, n, st);
    for (int q = 0; q < n; ++q) CUR_TRY(upload(v[q].dst, v[q].src, v[q].bytes, st));
    return CUR_OK;
}

// Stages whose first B comes from the tensor-core product: FP32, r = 32 or 64, at least this
// many rows in all (below it the tiles are too few to pay for the extra launches).
constexpr int64_t kCoefMinRows = 8192;

// One stage: a set of problems on one basis buffer. The caller fills probs (base,
// gid_base, gid_arr, p); stage_setup plans the CTA groups and allocates per-problem
// state; stage_tables uploads the plan; stage_init sets the per-problem flags; decision
// kernels may then change them on the device; stage_launch runs the optional Algorithm 3
// start, the FP64 inverse where lu_mask is set, and the engine, for problems not done.
template <typename TB>
struct Stage {
    std::vector<MvProb> probs;
    int P = 0, slots = 0, max_rpc = 1;
    MvProb* dprob = nullptr;
    int32_t* dtab = nullptr;   // cta_prob | cta_part | lu_mask
    int32_t* S = nullptr;      // P x r
    double* minv64 = nullptr;  // P x minv_stride(r)
    float* mdf = nullptr;      // P x 2 r^2 (r > kMsMax only)
    double* logvol = nullptr;
    int32_t* swaps = nullptr;
    int32_t* pstatus = nullptr;
    int32_t* done = nullptr;
    int32_t* retry = nullptr;  // merge levels: which start a problem is on
    unsigned* bar = nullptr;
    double* keyv = nullptr;
    long long* keyi = nullptr;
    TB* pub = nullptr;
    double* aux = nullptr;
    int coop_slots = 0;         // slots [0, coop_slots) hold groups of several CTAs
    bool keep_singular_set = false;
    TB* bglob = nullptr;        // B in global memory when it cannot live in shared memory
    // the first cycle's B on the tensor cores (FP32, r = 32 or 64, large stages)
    float* bpre = nullptr;
    float* wh = nullptr;
    float* wl = nullptr;
    CoefTile* dtiles = nullptr;
    std::vector<CoefTile> tiles;
    int64_t rows_total = 0;
};

template <typename TB>
// starts: the stage runs the Algorithm 3 start (mv_start), which keeps each CTA's rows in
// shared memory, so its problems never take the global-memory form.
static cur_status stage_setup(cur_handle* h, int r, Stage<TB>& sg, Arena& ar, bool starts = false) {
    const int P = (int)sg.probs.size();
    sg.P = P;
    int capr[129] = {0};   // rows per CTA with B in shared memory, by rank
    auto cap_of = [&](int rr) {
        if (!capr[rr]) capr[rr] = rows_cap<TB>(rr);
        return capr[rr];
    };
    int64_t tot_p = 0;
    for (auto& pr : sg.probs) tot_p += pr.p;
    // A problem whose B does not fit one CTA's shared memory is spread over a group of
    // co-resident CTAs; with many problems in the stage (a batch), or when it would need
    // more than one CTA per SM, its B goes to global memory and one CTA takes it.
    const bool many = P >= 2 * h->num_sms;
    int64_t elems_end = 0;
    bool anyg = false;
    for (auto& pr : sg.probs) {
        const int cap = cap_of(pr.r);
        int64_t G = (pr.p + cap - 1) / cap;
        pr.gmode = 0;
        if (G > 1 && (many || G > h->num_sms) && !starts) pr.gmode = 1;
        if (pr.gmode && many) {
            G = 1;
        } else if (G > 1 || pr.gmode) {
            // spread large problems over the SMs in proportion to their size
            const int64_t spread = std::min<int64_t>((pr.p + kSpreadRows - 1) / kSpreadRows,
                                                     (int64_t)h->num_sms * pr.p / std::max<int64_t>(1, tot_p));
            G = std::max<int64_t>(pr.gmode ? 1 : G, spread);
            G = std::min<int64_t>(G, h->num_sms);
        }
        G = std::max<int64_t>(1, G);
        const int rpc = (int)((pr.p + G - 1) / G);
        G = (pr.p + rpc - 1) / rpc;
        pr.G = (int)G;
        pr.rpc = rpc;
        sg.max_rpc = std::max(sg.max_rpc, rpc);
        anyg |= pr.gmode != 0;
        elems_end = std::max<int64_t>(elems_end, pr.boff + (int64_t)pr.p * pr.r);
    }
    int slots = 0;
    // slots: the groups of several CTAs first (cooperative launches, co-resident), then
    // the single-CTA problems (one plain launch: they never wait on another CTA)
    for (int pass = 0; pass < 2; ++pass) {
        for (auto& pr : sg.probs)
            if ((pr.G > 1) == (pass == 0)) {
                pr.group0 = slots;
                slots += pr.G;
            }
        if (pass == 0) sg.coop_slots = slots;
    }
    sg.slots = slots;
    sg.dprob = ar.get<MvProb>(P);
    sg.dtab = ar.get<int32_t>((size_t)2 * slots + P);
    sg.S = ar.get<int32_t>((size_t)P * r);
    sg.minv64 = ar.get<double>((size_t)P * minv_stride(r));
    sg.mdf = r > kMsMax ? ar.get<float>((size_t)P * 2 * r * r) : nullptr;
    sg.logvol = ar.get<double>(P);
    sg.swaps = ar.get<int32_t>(P);
    sg.pstatus = ar.get<int32_t>(P);
    sg.done = ar.get<int32_t>(P);
    sg.retry = ar.get<int32_t>(P);
    sg.bar = ar.get<unsigned>(P);
    sg.keyv = ar.get<double>((size_t)2 * slots);
    sg.keyi = ar.get<long long>((size_t)2 * slots);
    sg.pub = ar.get<TB>((size_t)2 * slots * r);
    sg.aux = ar.get<double>((size_t)2 * slots);
    sg.bglob = anyg ? ar.get<TB>((size_t)elems_end) : nullptr;
    if (!ar.ok) return CUR_ERR_NOMEM;
    sg.tiles.clear();
    sg.bpre = nullptr;
    sg.rows_total = elems_end / std::max(1, r);
    bool same_r = true;
    for (auto& pr : sg.probs) same_r &= pr.r == r && pr.boff % r == 0;
    if (std::is_same<TB, float>::value && coef_tc_applies(CUR_F32, r) && same_r && sg.rows_total >= kCoefMinRows) {
        for (int pb = 0; pb < P; ++pb)
            for (int64_t i = 0; i < sg.probs[pb].p; i += 128)
                sg.tiles.push_back(CoefTile{pb, (int32_t)std::min<int64_t>(128, sg.probs[pb].p - i),
                                            sg.probs[pb].boff / r + i});
        const size_t mark = ar.off;
        sg.bpre = ar.get<float>((size_t)sg.rows_total * r);
        sg.wh = ar.get<float>((size_t)P * r * r);
        sg.wl = ar.get<float>((size_t)P * r * r);
        sg.dtiles = ar.get<CoefTile>(sg.tiles.size());
        if (!ar.ok) {   // no room: this stage forms its first B on the CUDA cores as the later ones
            ar.off = mark;
            ar.ok = true;
            sg.bpre = nullptr;
            sg.tiles.clear();
        }
    }
    return CUR_OK;
}

// The stage plan to the device: problem descriptors and the CTA slot tables.
template <typename TB>
static cur_status stage_tables(Stage<TB>& sg, cudaStream_t st) {
    const int P = sg.P, slots = sg.slots;
    std::vector<int32_t> tab((size_t)2 * slots);
    for (int pb = 0; pb < P; ++pb)
        for (int g = 0; g < sg.probs[pb].G; ++g) {
            tab[sg.probs[pb].group0 + g] = pb;
            tab[slots + sg.probs[pb].group0 + g] = g;
        }
    return upload_multi({{sg.dprob, sg.probs.data(), sizeof(MvProb) * P},
                         {sg.dtab, tab.data(), sizeof(int32_t) * tab.size()},
                         {sg.dtiles, sg.tiles.data(), sg.bpre ? sizeof(CoefTile) * sg.tiles.size() : 0}},
                        st);
}

// Per-problem defaults: factorise (lu_mask 1), not done (or all done while *idle != 0),
// no swaps, status OK.
// Per-problem flags and counters of a stage, its group-barrier counters, and (with S0) the
// start set S0[0..ns) copied into S.
__global__ void stage_init_k(int32_t* lu_mask, int32_t* done, int32_t* swaps, int32_t* pstatus, int32_t* retry,
                             unsigned* bar, int P, const int* idle, const int32_t* S0, int32_t* S, int ns) {
    const int sk = idle ? (*idle != 0) : 0;
    for (int pb = blockIdx.x * blockDim.x + threadIdx.x; pb < P; pb += gridDim.x * blockDim.x) {
        lu_mask[pb] = 1;
        done[pb] = sk;
        swaps[pb] = 0;
        pstatus[pb] = 0;
        retry[pb] = 0;
        bar[pb] = 0u;
    }
    if (S0)
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += gridDim.x * blockDim.x) S[k] = S0[k];
}

template <typename TB>
static cur_status stage_init(Stage<TB>& sg, const int* idle, cudaStream_t st, const int32_t* S0 = nullptr,
                             int ns = 0) {
    stage_init_k<<<nblk(std::max(sg.P, ns)), 256, 0, st>>>(sg.dtab + 2 * sg.slots, sg.done, sg.swaps, sg.pstatus,
                                                          sg.retry, sg.bar, sg.P, idle, S0, sg.S, ns);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

// The stage's kernels: the Algorithm 3 start (aca_start), the FP64 inverses where lu_mask is
// set, the swap engine; every kernel skips the problems marked done.
template <typename TB>
static cur_status stage_launch(cur_handle* h, const TB* basis, int r, const cur_opts* o, Stage<TB>& sg,
                               bool aca_start, cudaStream_t st) {
    const int P = sg.P, slots = sg.slots;
    MvArgs a{};
    a.basis = basis;
    a.minv64 = sg.minv64;
    a.mdf = sg.mdf;
    a.prob = sg.dprob;
    a.P = P;
    a.r = r;
    a.delta = o->delta;
    a.max_swaps = o->max_swaps > 0 ? o->max_swaps : 100 * r;
    // FP64 data (and CUR_FLAG_REFACTOR_ALWAYS): a fresh factorisation every cycle. FP32 B
    // (double-float inverse, u = 2^-48): the carried inverse while sum(swaps * kappa) <= 2^18,
    // i.e. drift <= 2^-30.
    a.drift_max = (std::is_same<TB, double>::value || (o->flags & CUR_FLAG_REFACTOR_ALWAYS)) ? 0.0 : 262144.0;
    a.nrefactor = h->status + 1;
    a.keep_singular_set = sg.keep_singular_set ? 1 : 0;
    a.bglob = sg.bglob;
    a.cta_prob = sg.dtab;
    a.cta_part = sg.dtab + slots;
    a.lu_mask = sg.dtab + 2 * slots;
    a.S = sg.S;
    a.logvol = sg.logvol;
    a.swaps = sg.swaps;
    a.pstatus = sg.pstatus;
    a.done = sg.done;
    a.bar = sg.bar;
    a.keyv = sg.keyv;
    a.keyi = sg.keyi;
    a.pub = sg.pub;
    a.aux = sg.aux;
    a.status = h->status;

    // shared memory of a launch: the largest any of its problems needs
    size_t sm_eng = 0, sm_start = 0;
    for (const auto& pr : sg.probs) {
        sm_eng = std::max(sm_eng, EngineSmem<TB>::bytes(pr.rpc, pr.r, pr.gmode != 0));
        sm_start = std::max(sm_start, StartSmem<TB>::bytes(pr.rpc, pr.r));
    }
    const size_t sm_lu = ((size_t)r * r + r) * sizeof(double) + (size_t)r * sizeof(int) + 64;
    CUR_TRY(set_smem_attr(mv_engine<TB>, sm_eng));
    CUR_TRY(set_smem_attr(mv_lu<TB>, sm_lu));
    int occ_eng = 0, occ_start = 1;
    CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_eng, mv_engine<TB>, 256, sm_eng));
    if (aca_start) {
        CUR_TRY(set_smem_attr(mv_start<TB>, sm_start));
        CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_start, mv_start<TB>, StartThreads<TB>::v, sm_start));
    }
    const int cap_eng = std::max(1, occ_eng) * h->num_sms;
    const int cap_start = std::max(1, occ_start) * h->num_sms;
    for (auto& pr : sg.probs)
        if (pr.G > cap_eng || (aca_start && pr.G > cap_start)) return CUR_ERR_ARG;
    // cooperative waves of whole multi-CTA groups, then one plain launch of the rest
    auto waves = [&](int capc) {
        std::vector<std::pair<int, int>> w;
        int first = 0, cnt = 0;
        for (int pb = 0; pb < P; ++pb) {
            const int G = sg.probs[pb].G;
            if (G == 1) continue;
            if (cnt + G > capc && cnt > 0) { w.push_back({first, cnt}); first += cnt; cnt = 0; }
            cnt += G;
        }
        if (cnt > 0) w.push_back({first, cnt});
        return w;
    };
    const int solo_slots = slots - sg.coop_slots;
    // the group-barrier counters are zero here: stage_init_k and the merge retry kernels
    // clear them before the Algorithm 3 start, mv_lu before the swap engine
    if (aca_start) {
        for (auto& w : waves(cap_start)) {
            MvArgs aw = a;
            aw.cta_base = w.first;
            void* args[] = {&aw};
            CUR_TRY(launch_coop((const void*)mv_start<TB>, dim3(w.second), dim3(StartThreads<TB>::v), args, sm_start, st));
            note_launch();
        }
        if (solo_slots > 0) {
            MvArgs aw = a;
            aw.cta_base = sg.coop_slots;
            mv_start<TB><<<solo_slots, StartThreads<TB>::v, sm_start, st>>>(aw);
            CUR_CK(cudaGetLastError());
            note_launch();
        }
    }
    mv_lu<TB><<<P, 512, sm_lu, st>>>(a);
    CUR_CK(cudaGetLastError());
    note_launch();
    if (sg.bpre) {
        // the first cycle's B = C M^-1 of every problem on the tensor cores
        CUR_TRY(coef_tc_launch(h, reinterpret_cast<const float*>(basis), sg.rows_total, r, sg.minv64, minv_stride(r), P,
                               sg.dtiles, (int)sg.tiles.size(), sg.done, sg.wh, sg.wl, sg.bpre, st));
        a.bpre = sg.bpre;
    }
    if (solo_slots > 0) {
        MvArgs aw = a;
        aw.cta_base = sg.coop_slots;
        mv_engine<TB><<<solo_slots, kSoloThreads, sm_eng, st>>>(aw);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    for (auto& w : waves(cap_eng)) {
        MvArgs aw = a;
        aw.cta_base = w.first;
        void* args[] = {&aw};
        CUR_TRY(launch_coop((const void*)mv_engine<TB>, dim3(w.second), dim3(256), args, sm_eng, st));
        note_launch();
    }
    return CUR_OK;
}

// ---------------------------------------------------------------- decisions on the device
//
// Where the next step depends on a result (a singular start, a valid inverse to inherit,
// whether a sweep swapped), a small kernel reads the result and sets the next stage's
// flags; nothing returns to the host, so the calls only enqueue.

// Where an inherited inverse comes from: M^-1 (minv_stride doubles) and log|det| of the
// start rows, valid when flag says so (mode 0: *flag != 0; mode 1: *flag is CUR_OK or
// CUR_ERR_NOCONV, the status of the stage that produced it; no flag: valid).
struct InheritSrc {
    const double* minv;
    const double* lv;
    const int* flag;
    int mode;
    int transpose;
};

// Problem t (one CTA each) starts from src[t]'s inverse when it is valid: copy (or transpose)
// it, take its log|det|, and skip the factorisation.
__global__ void inherit_k(const InheritSrc* __restrict__ src, int r, double* minv64, double* logvol,
                          int32_t* lu_mask, const int32_t* done) {
    const int t = blockIdx.x;
    const InheritSrc s = src[t];
    if (done[t] || !s.minv || !s.lv) return;
    const bool valid = !s.flag || (s.mode == 0 ? *s.flag != 0 : (*s.flag == CUR_OK || *s.flag == CUR_ERR_NOCONV));
    if (!valid) return;
    const int64_t stride = minv_stride(r);
    double* dst = minv64 + (int64_t)t * stride;
    for (int e = threadIdx.x; e <= r * r; e += blockDim.x) {
        const int a = e / r, b = e - a * r;
        dst[e] = (e == r * r || !s.transpose) ? s.minv[e] : s.minv[b * r + a];
    }
    if (threadIdx.x == 0) {
        logvol[t] = *s.lv;
        lu_mask[t] = 0;
    }
}

static cur_status launch_inherit(const std::vector<InheritSrc>& src, int r, double* minv64, double* logvol,
                                 int32_t* lu_mask, const int32_t* done, InheritSrc* dsrc, cudaStream_t st) {
    if (src.empty()) return CUR_OK;
    CUR_TRY(upload(dsrc, src.data(), sizeof(InheritSrc) * src.size(), st));
    inherit_k<<<(unsigned)src.size(), 1024, 0, st>>>(dsrc, r, minv64, logvol, lu_mask, done);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

// After attempt `attempt` of a merge level: a node whose start was singular moves on to the
// next start (after attempt 0: the right set, positions r..2r-1 of its union; after attempt
// 1: Algorithm 3 on the union, formed by mv_start); the swaps of a node that finished are
// added to *acc, those of an abandoned attempt are not counted.
__global__ void merge_retry_k(int attempt, int P, int r, int32_t* pstatus, int32_t* swaps, int32_t* done,
                              int32_t* lu_mask, int32_t* S, int32_t* retry, int* acc, unsigned* bar) {
    for (int pb = blockIdx.x * blockDim.x + threadIdx.x; pb < P; pb += gridDim.x * blockDim.x) {
        bar[pb] = 0u;   // for the next attempt's Algorithm 3 start
        if (attempt > 0 && retry[pb] != attempt) continue;
        const bool sing = pstatus[pb] == CUR_ERR_SINGULAR;
        if (attempt < 2 && sing) {
            retry[pb] = attempt + 1;
            pstatus[pb] = CUR_OK;
            swaps[pb] = 0;
            done[pb] = 0;
            lu_mask[pb] = 1;
            if (attempt == 0)
                for (int k = 0; k < r; ++k) S[(int64_t)pb * r + k] = r + k;
        } else {
            retry[pb] = 0;
            atomicAdd(acc, swaps[pb]);
        }
    }
}

// acc += sum of swaps[0..P)
__global__ void acc_swaps_k(const int32_t* swaps, int P, int* acc) {
    int s = 0;
    for (int pb = threadIdx.x; pb < P; pb += blockDim.x) s += swaps[pb];
    atomicAdd(acc, s);
}

// The end of a global maxvol stage: the set (the start set again if the iteration turned
// singular, unless keep), log|det|, the final inverse and the device result.
__global__ void global_finish_k(const int32_t* pstatus, const int32_t* swaps, const int32_t* Sst, const int32_t* S0,
                                int r, int keep, int32_t* S_out, const double* lv_st, double* logvol_out,
                                const double* minv64, double* minv_out, MvDevResult* res, const int* idle) {
    if (idle && *idle) return;
    const int stv = pstatus[0];
    const bool ok = stv != CUR_ERR_SINGULAR && stv != CUR_ERR_ARG && stv != CUR_ERR_NONFINITE && stv != CUR_ERR_TIMEOUT;
    const bool use_stage = (stv != CUR_ERR_SINGULAR || keep) && stv != CUR_ERR_ARG;
    for (int k = threadIdx.x; k < r; k += blockDim.x) S_out[k] = use_stage ? Sst[k] : S0[k];
    if (minv_out && ok)
        for (int e = threadIdx.x; e <= r * r; e += blockDim.x) minv_out[e] = minv64[e];
    if (threadIdx.x == 0) {
        if (logvol_out) *logvol_out = *lv_st;
        if (res) {
            res->swaps = swaps[0];
            res->status = stv;
            res->minv_valid = (ok && minv_out) ? 1 : 0;
        }
    }
}

// Row selection without the polish: the merged set, its inverse and log|det| (when the root
// problem's status makes them valid; else the log-volume taken directly, lv_direct).
__global__ void rows_root_k(const int32_t* root, int r, int32_t* I_out, const double* root_minv, const double* root_lv,
                            const int* root_stat, const double* lv_direct, double* logvol_out, double* minv_out,
                            const int* acc, int32_t* swaps_out, MvDevResult* res, const int* idle) {
    if (idle && *idle) return;
    const bool valid = root_minv && root_lv && (!root_stat || *root_stat == CUR_OK || *root_stat == CUR_ERR_NOCONV);
    for (int k = threadIdx.x; k < r; k += blockDim.x) I_out[k] = root[k];
    if (minv_out && valid)
        for (int e = threadIdx.x; e <= r * r; e += blockDim.x) minv_out[e] = root_minv[e];
    if (threadIdx.x == 0) {
        if (logvol_out) *logvol_out = valid ? *root_lv : *lv_direct;
        if (swaps_out) *swaps_out = *acc;
        if (res) {
            res->swaps = *acc;
            res->status = CUR_OK;
            res->minv_valid = (valid && minv_out) ? 1 : 0;
        }
    }
}

// Row selection with the polish: the counts add up.
__global__ void rows_polish_k(const int* acc, const MvDevResult* pol, int32_t* swaps_out, MvDevResult* res,
                              const int* idle) {
    if (idle && *idle) return;
    if (threadIdx.x != 0) return;
    const int tot = *acc + pol->swaps;
    if (swaps_out) *swaps_out = tot;
    if (res) {
        res->swaps = tot;
        res->status = pol->status;
        res->minv_valid = pol->minv_valid;
    }
}

// After the polish's low-precision phase: its swaps into *acc; *iflag = CUR_OK while the
// merge's inverse of the set still holds (no swap taken and its status word valid), else
// CUR_ERR_SINGULAR (the finish factorises afresh).
__global__ void lp_after_k(const int32_t* lp_swaps, const int* root_flag, int* acc, int* iflag) {
    if (threadIdx.x != 0) return;
    const int n = *lp_swaps;
    *acc += n;
    const bool valid = n == 0 && (!root_flag || *root_flag == CUR_OK || *root_flag == CUR_ERR_NOCONV);
    *iflag = valid ? CUR_OK : CUR_ERR_SINGULAR;
}

// One merge level on `basis` (p x r): sets in cand (nsets x r, global rows). in_src[k]
// describes, per input set, where its M^-1 and log|det| are (when known) and whether they
// are valid; node t then starts from its left set's M^-1 instead of a new factorisation.
// out_src describes the output sets. Swaps are added to *acc (device).
template <typename TB>
static cur_status merge_level_t(cur_handle* h, const TB* basis, int64_t p, int r,
                                const int32_t* cand, int nsets, const cur_opts* o, int32_t* out,
                                int* acc, const std::vector<InheritSrc>& in_src, Stage<TB>& lv,
                                std::vector<InheritSrc>& out_src, const int* idle, Arena& ar,
                                cudaStream_t st) {
    const int npairs = nsets / 2;
    out_src.clear();
    if (npairs == 0) {
        CUR_CK(cudaMemcpyAsync(out, cand, sizeof(int32_t) * r * nsets, cudaMemcpyDeviceToDevice, st));
        out_src = in_src;
        return CUR_OK;
    }
    const int64_t nrows = (int64_t)npairs * 2 * r;
    TB* U = ar.get<TB>((size_t)nrows * r);
    InheritSrc* dsrc = ar.get<InheritSrc>(npairs);
    if (!ar.ok) return CUR_ERR_NOMEM;
    gather_union_k<TB><<<nblk(nrows * r), 256, 0, st>>>(basis, p, r, cand, nrows, U, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    lv.probs.clear();
    for (int t = 0; t < npairs; ++t) {
        MvProb pr{};
        pr.base = (int64_t)t * 2 * r;
        pr.boff = pr.base * r;
        pr.r = r;
        pr.gid_arr = cand + (int64_t)t * 2 * r;
        pr.gid_base = 0;
        pr.p = 2 * r;
        lv.probs.push_back(pr);
    }
    CUR_TRY(stage_setup<TB>(h, r, lv, ar));
    CUR_TRY(stage_tables(lv, st));
    CUR_TRY(stage_init(lv, idle, st));
    mv_iota<<<nblk(npairs * r), 256, 0, st>>>(lv.S, npairs, r, 0);
    CUR_CK(cudaGetLastError());
    note_launch();
    // node t starts from its left set (2t) with that set's inverse when it is valid
    std::vector<InheritSrc> src(npairs);
    for (int t = 0; t < npairs; ++t) {
        const int k = 2 * t;
        src[t] = k < (int)in_src.size() ? in_src[k] : InheritSrc{nullptr, nullptr, nullptr, 0, 0};
        src[t].transpose = 0;
    }
    CUR_TRY(launch_inherit(src, r, lv.minv64, lv.logvol, lv.dtab + 2 * lv.slots, lv.done, dsrc, st));
    // attempt 0: the left set; 1: the right set where the left one is singular; 2: Algorithm 3
    // on the union where both are
    for (int attempt = 0; attempt < 3; ++attempt) {
        CUR_TRY(stage_launch<TB>(h, U, r, o, lv, attempt == 2, st));
        merge_retry_k<<<nblk(npairs), 256, 0, st>>>(attempt, npairs, r, lv.pstatus, lv.swaps, lv.done,
                                                    lv.dtab + 2 * lv.slots, lv.S, lv.retry, acc, lv.bar);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    mv_emit<<<nblk(npairs * r), 256, 0, st>>>(lv.dprob, lv.S, npairs, r, out);
    CUR_CK(cudaGetLastError());
    note_launch();
    for (int t = 0; t < npairs; ++t)
        out_src.push_back(InheritSrc{lv.minv64 + (int64_t)t * minv_stride(r), lv.logvol + t, lv.pstatus + t, 1, 0});
    if (nsets % 2 == 1) {
        CUR_CK(cudaMemcpyAsync(out + (int64_t)npairs * r, cand + (int64_t)(nsets - 1) * r,
                               sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
        out_src.push_back(nsets - 1 < (int)in_src.size() ? in_src[nsets - 1]
                                                         : InheritSrc{nullptr, nullptr, nullptr, 0, 0});
    }
    return CUR_OK;
}

// Maxvol over all p rows of the basis, started at S0 (global rows). With `inherit` (M^-1
// and log|det| of exactly the rows S0 in that order, or the transpose of that inverse, valid
// per its flag) no new factorisation is made. minv_out receives the final M^-1; res (device)
// the swaps, the status and whether minv_out is valid. Nothing runs while *idle != 0.
template <typename TB>
static cur_status global_t(cur_handle* h, const TB* basis, int64_t p, int r, const cur_opts* o,
                           const int32_t* S0, int32_t* S_out, double* logvol_out, MvDevResult* res,
                           Arena& ar, cudaStream_t st, InheritSrc inherit, double* minv_out,
                           bool keep_singular_set, const int* idle) {
    Stage<TB> sg;
    sg.keep_singular_set = keep_singular_set;
    MvProb pr{};
    pr.base = 0;
    pr.boff = 0;
    pr.r = r;
    pr.gid_base = 0;
    pr.gid_arr = nullptr;
    pr.p = (int32_t)p;
    sg.probs.push_back(pr);
    CUR_TRY(stage_setup<TB>(h, r, sg, ar));
    InheritSrc* dsrc = ar.get<InheritSrc>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(stage_tables(sg, st));
    CUR_TRY(stage_init(sg, idle, st, S0, r));
    if (inherit.minv && inherit.lv)
        CUR_TRY(launch_inherit(std::vector<InheritSrc>{inherit}, r, sg.minv64, sg.logvol, sg.dtab + 2 * sg.slots,
                               sg.done, dsrc, st));
    CUR_TRY(stage_launch<TB>(h, basis, r, o, sg, false, st));
    global_finish_k<<<1, 256, 0, st>>>(sg.pstatus, sg.swaps, sg.S, S0, r, keep_singular_set ? 1 : 0, S_out, sg.logvol,
                                       logvol_out, sg.minv64, minv_out, res, idle);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

template <typename TB>
static cur_status rows_t(cur_handle* h, const TB* basis, int64_t p, int r, const cur_opts* o,
                         int32_t* I_out, double* logvol_out, int32_t* swaps_out, MvDevResult* res,
                         Arena& ar, cudaStream_t st, double* minv_out, const int* idle) {
    const int nb = std::max(1, o->nblocks);
    const int64_t base_sz = p / nb, extra = p % nb;
    if (base_sz < r) return CUR_ERR_ARG;
    int32_t* setsA = ar.get<int32_t>((size_t)nb * r);
    int32_t* setsB = ar.get<int32_t>((size_t)nb * r);
    int* acc = ar.get<int>(1);
    MvDevResult* pol = ar.get<MvDevResult>(1);
    double* lv_direct = ar.get<double>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_CK(cudaMemsetAsync(acc, 0, sizeof(int), st));
    // Stage objects (and their workspace) stay alive until the end of the call, so a
    // merge node can start from its left set's M^-1.
    std::vector<Stage<TB>> stages;
    stages.reserve(64);
    stages.emplace_back();
    Stage<TB>& sb = stages[0];
    int64_t s0 = 0;
    for (int k = 0; k < nb; ++k) {
        const int64_t sz = base_sz + (k < extra ? 1 : 0);
        MvProb pr{};
        pr.base = s0;
        pr.boff = s0 * r;
        pr.r = r;
        pr.gid_base = s0;
        pr.gid_arr = nullptr;
        pr.p = (int32_t)sz;
        sb.probs.push_back(pr);
        s0 += sz;
    }
    CUR_TRY(stage_setup<TB>(h, r, sb, ar, true));
    CUR_TRY(stage_tables(sb, st));
    CUR_TRY(stage_init(sb, idle, st));
    mv_iota<<<nblk(nb * r), 256, 0, st>>>(sb.S, nb, r, 0);   // valid rows even when nothing runs
    CUR_CK(cudaGetLastError());
    note_launch();
    CUR_TRY(stage_launch<TB>(h, basis, r, o, sb, true, st));
    acc_swaps_k<<<1, 256, 0, st>>>(sb.swaps, nb, acc);
    CUR_CK(cudaGetLastError());
    mv_emit<<<nblk(nb * r), 256, 0, st>>>(sb.dprob, sb.S, nb, r, setsA);
    CUR_CK(cudaGetLastError());
    note_launch(2);
    std::vector<InheritSrc> src, src2;
    for (int k = 0; k < nb; ++k)
        src.push_back(InheritSrc{sb.minv64 + (int64_t)k * minv_stride(r), sb.logvol + k, sb.pstatus + k, 1, 0});
    int nsets = nb;
    int32_t* cur = setsA;
    int32_t* nxt = setsB;
    while (nsets > 1) {
        stages.emplace_back();
        CUR_TRY(merge_level_t<TB>(h, basis, p, r, cur, nsets, o, nxt, acc, src, stages.back(), src2, idle, ar, st));
        nsets = (nsets + 1) / 2;
        std::swap(cur, nxt);
        src.swap(src2);
    }
    const InheritSrc root = src.empty() ? InheritSrc{nullptr, nullptr, nullptr, 0, 0} : src[0];
    if (o->flags & CUR_FLAG_POLISH) {
        InheritSrc start = root;
        if constexpr (std::is_same<TB, float>::value) {
            // with CUR_FLAG_PREC_BF16 / _FP8 on a large basis, low-precision products take the
            // polish's swaps first; the FP32 engine then finishes, from the merge's inverse if
            // that phase took no swap, else from a fresh factorisation (decided on the device)
            if (lowprec_phase_applies(h, o, CUR_F32, p, r)) {
                int32_t* lp_swaps = ar.get<int32_t>(1);
                int* iflag = ar.get<int>(1);
                if (!ar.ok) return CUR_ERR_NOMEM;
                CUR_TRY(lowprec_phase(h, basis, p, r, o, cur, cur, lp_swaps, ar, st, root.minv, root.flag, idle));
                lp_after_k<<<1, 32, 0, st>>>(lp_swaps, root.flag, acc, iflag);
                CUR_CK(cudaGetLastError());
                note_launch();
                start = InheritSrc{root.minv, root.lv, iflag, 1, 0};
            }
        }
        CUR_TRY(global_t<TB>(h, basis, p, r, o, cur, I_out, logvol_out, pol, ar, st, start, minv_out, false, idle));
        rows_polish_k<<<1, 32, 0, st>>>(acc, pol, swaps_out, res, idle);
        CUR_CK(cudaGetLastError());
        note_launch();
    } else {
        CUR_TRY(logvol_rows(std::is_same<TB, double>::value ? CUR_F64 : CUR_F32, basis, p, r, cur, lv_direct, st));
        rows_root_k<<<1, 256, 0, st>>>(cur, r, I_out, root.minv, root.lv, root.flag, lv_direct, logvol_out,
                                       minv_out, acc, swaps_out, res, idle);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    return CUR_OK;
}

}  // namespace curk

size_t compute_size(cur_dtype t) { return t == CUR_F64 ? 8 : 4; }

cur_status maxvol_basis_rows(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                             const cur_opts* o, int32_t* I_out, double* logvol_out,
                             int32_t* swaps_out, MvDevResult* res, Arena& ar, cudaStream_t st,
                             double* minv_out, const int* idle) {
    // the workspace a call takes is free again for the next call on the stream (stream order)
    const size_t mark = ar.off;
    cur_status s;
    if (dt == CUR_F64)
        s = curk::rows_t<double>(h, static_cast<const double*>(basis), p, r, o, I_out, logvol_out, swaps_out, res, ar,
                                 st, minv_out, idle);
    else
        s = curk::rows_t<float>(h, static_cast<const float*>(basis), p, r, o, I_out, logvol_out, swaps_out, res, ar,
                                st, minv_out, idle);
    ar.off = mark;
    ar.ok = true;
    return s;
}

cur_status maxvol_global(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                         const cur_opts* o, const int32_t* S0, int32_t* S_out,
                         double* logvol_out, MvDevResult* res, Arena& ar, cudaStream_t st,
                         const double* minv_in, const double* lv_in, const int* minv_in_valid,
                         bool transpose_in, double* minv_out, bool keep_singular_set, const int* idle) {
    const curk::InheritSrc src{minv_in, lv_in, minv_in_valid, 0, transpose_in ? 1 : 0};
    const size_t mark = ar.off;
    cur_status s;
    if (dt == CUR_F64)
        s = curk::global_t<double>(h, static_cast<const double*>(basis), p, r, o, S0, S_out, logvol_out, res, ar, st,
                                   src, minv_out, keep_singular_set, idle);
    else
        s = curk::global_t<float>(h, static_cast<const float*>(basis), p, r, o, S0, S_out, logvol_out, res, ar, st,
                                  src, minv_out, keep_singular_set, idle);
    ar.off = mark;
    ar.ok = true;
    return s;
}

template <typename TB>
static cur_status merge_one(cur_handle* h, const TB* basis, int64_t p, int r, const int32_t* cand,
                            int nsets, const cur_opts* o, int32_t* out, int* acc, Arena& ar,
                            cudaStream_t st) {
    curk::Stage<TB> lv;
    std::vector<curk::InheritSrc> none, os;
    return curk::merge_level_t<TB>(h, basis, p, r, cand, nsets, o, out, acc, none, lv, os, nullptr, ar, st);
}

cur_status upload_table(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return curk::upload(dst, src, bytes, st);
}

cur_status merge_level(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                       const int32_t* cand, int nsets, const cur_opts* o, int32_t* out,
                       int* acc_dev, Arena& ar, cudaStream_t st) {
    if (dt == CUR_F64)
        return merge_one<double>(h, static_cast<const double*>(basis), p, r, cand, nsets, o, out, acc_dev, ar, st);
    return merge_one<float>(h, static_cast<const float*>(basis), p, r, cand, nsets, o, out, acc_dev, ar, st);
}


// ---------------------------------------------------------------- the sweeps of a cross
//
// Sweeps of global maxvol on the rows of A(:,J) from I, then on the columns of A(I,:)^T
// from J, until a sweep makes no swap (reading 17). Every sweep up to the cap is enqueued;
// the control block's idle flag, set on the device by the sweep that ends the loop, makes
// the later sweeps' kernels return at once.

namespace curk {

__global__ void cross_begin_k(CrossCtl* ctl, const int* hstatus, int check_status) {
    if (threadIdx.x != 0) return;
    int idle = 0;
    if (check_status) {
        const int s = *hstatus;
        idle = (s != CUR_OK && s != CUR_WARN_RANK) ? 1 : 0;   // Algorithm 3 met an error
    }
    ctl->idle = idle;
    ctl->abort = idle;
    ctl->sweeps = 0;
    for (int k = 0; k < 8; ++k) ctl->sweep_swaps[k] = 0;
    ctl->last_status = CUR_OK;
    ctl->mc_valid = 0;
    ctl->singular_start = 0;
}

// Sweep 1 of cur_cross (the blockwise row and column selections) is over.
__global__ void sweep_one_k(CrossCtl* ctl, const MvDevResult* rr, const MvDevResult* rc) {
    if (threadIdx.x != 0 || ctl->abort) return;
    ctl->sweeps = 1;
    ctl->sweep_swaps[0] = rr->swaps + rc->swaps;
    if (rr->status != CUR_OK) ctl->last_status = rr->status;
    if (rc->status != CUR_OK) ctl->last_status = rc->status;
    ctl->mc_valid = rc->minv_valid;
}

// cur_cross_from, sweep 1: a singular proposed A(I0, J0) (the row stage's start, no swap)
// leaves nothing to refine.
__global__ void from_start_k(CrossCtl* ctl, const MvDevResult* r1) {
    if (threadIdx.x != 0 || ctl->idle) return;
    if (r1->status == CUR_ERR_SINGULAR && r1->swaps == 0) {
        ctl->last_status = CUR_ERR_SINGULAR;
        ctl->singular_start = 1;
        ctl->sweeps = 1;
        ctl->idle = 1;
    }
}

__global__ void sweep_end_k(CrossCtl* ctl, const MvDevResult* r1, const MvDevResult* r2, int s) {
    if (threadIdx.x != 0 || ctl->idle) return;
    ctl->sweeps = s;
    ctl->sweep_swaps[s - 1] = r1->swaps + r2->swaps;
    ctl->mc_valid = r2->minv_valid;
    if (r1->status != CUR_OK || r2->status != CUR_OK) {
        ctl->last_status = r1->status != CUR_OK ? r1->status : r2->status;
        ctl->idle = 1;
    } else if (r1->swaps + r2->swaps == 0) {
        ctl->idle = 1;
    }
}

// The cross's log-volume (taken directly when a stage ended with an error: such a stage
// leaves no log|det| of its own; -inf for a singular proposal), its status and its info.
__global__ void cross_end_k(CrossCtl* ctl, double* lv, const double* lv_direct, cur_cross_info* info,
                            const int32_t* aca_count, int* hstatus, int from, const int32_t* I, const int32_t* J,
                            int r, int32_t* I_out, int32_t* J_out) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        I_out[k] = I[k];
        J_out[k] = J[k];
    }
    if (threadIdx.x != 0) return;
    if (ctl->singular_start) *lv = -INFINITY;
    else if (ctl->last_status != CUR_OK) *lv = *lv_direct;
    if (ctl->last_status == CUR_ERR_NOCONV || ctl->last_status == CUR_ERR_SINGULAR)
        set_status(hstatus, ctl->last_status);
    if (!info) return;
    int tot = 0;
    for (int k = 0; k < 8; ++k) tot += ctl->sweep_swaps[k];
    info->logvol = *lv;
    info->sweeps = ctl->sweeps;
    info->swaps_total = tot;
    for (int k = 0; k < 8; ++k) info->sweep_swaps[k] = ctl->sweep_swaps[k];
    info->aca_selected = aca_count ? *aca_count : 0;
    info->status = from ? ctl->last_status : *hstatus;
}

}  // namespace curk

cur_status cross_begin(CrossCtl* ctl, const int* hstatus, bool check_status, cudaStream_t st) {
    curk::cross_begin_k<<<1, 32, 0, st>>>(ctl, hstatus, check_status ? 1 : 0);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cross_sweep_one(CrossCtl* ctl, const MvDevResult* rr, const MvDevResult* rc, cudaStream_t st) {
    curk::sweep_one_k<<<1, 32, 0, st>>>(ctl, rr, rc);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cross_sweeps(cur_handle* h, const cur_mat* A, int r, const cur_opts* o, int first, int max_sweeps,
                        bool from, int32_t* I, int32_t* J, void* Cb, void* Rb, double* Mr, double* Mc, double* lvr,
                        double* lv, CrossCtl* ctl, Arena& ar, cudaStream_t st) {
    const cur_dtype cdt = A->dtype == CUR_F64 ? CUR_F64 : CUR_F32;
    const int64_t m = A->rows, n = A->cols;
    MvDevResult* res = ar.get<MvDevResult>(2);
    if (!ar.ok) return CUR_ERR_NOMEM;
    for (int s = first; s <= max_sweeps; ++s) {
        CUR_TRY(gather_cols_compute(A, J, r, Cb, st, &ctl->idle));
        CUR_TRY(maxvol_global(h, cdt, Cb, m, r, o, I, I, lvr, &res[0], ar, st, Mc, lv, &ctl->mc_valid, true, Mr, true,
                              &ctl->idle));
        if (from && s == 1) {
            curk::from_start_k<<<1, 32, 0, st>>>(ctl, &res[0]);
            CUR_CK(cudaGetLastError());
            note_launch();
        }
        CUR_TRY(gather_rows_t_compute(A, I, r, Rb, st, &ctl->idle));
        CUR_TRY(maxvol_global(h, cdt, Rb, n, r, o, J, J, lv, &res[1], ar, st, Mr, lvr, &res[0].minv_valid, true, Mc,
                              true, &ctl->idle));
        curk::sweep_end_k<<<1, 32, 0, st>>>(ctl, &res[0], &res[1], s);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    return CUR_OK;
}

cur_status cross_end(cur_handle* h, const cur_mat* A, int r, bool from, const int32_t* I, const int32_t* J,
                     void* Rb, double* lv, CrossCtl* ctl, const int32_t* aca_count, int32_t* I_out, int32_t* J_out,
                     cur_cross_info* info_out, Arena& ar, cudaStream_t st) {
    const cur_dtype cdt = A->dtype == CUR_F64 ? CUR_F64 : CUR_F32;
    double* lv_direct = ar.get<double>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(gather_rows_t_compute(A, I, r, Rb, st));
    CUR_TRY(logvol_rows(cdt, Rb, A->cols, r, J, lv_direct, st));
    curk::cross_end_k<<<1, 128, 0, st>>>(ctl, lv, lv_direct, info_out, aca_count, h->status, from ? 1 : 0, I, J, r,
                                         I_out, J_out);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}


namespace curk {
// ids_out[k] = ids[pos[k]], rows_out[k, :] = rows[pos[k], :] (the merged set's ids and rows).
template <typename TB>
__global__ void pair_emit_k(const TB* __restrict__ rows, const int32_t* __restrict__ ids,
                            const int32_t* __restrict__ pos, int r, int32_t* __restrict__ ids_out,
                            TB* __restrict__ rows_out, int32_t* swaps_out, const int* acc) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int k = e / r, c = e - k * r;
        rows_out[e] = rows[(int64_t)pos[k] * r + c];
    }
    for (int k = threadIdx.x; k < r; k += blockDim.x) ids_out[k] = ids[pos[k]];
    if (threadIdx.x == 0 && swaps_out) *swaps_out = *acc;
}
}  // namespace curk

cur_status merge_pair_impl(cur_handle* h, cur_dtype dt, const void* rows, const int32_t* ids, int r,
                           const cur_opts* o, int32_t* ids_out, void* rows_out, int32_t* swaps_out, Arena& ar,
                           cudaStream_t st) {
    int32_t* cand = ar.get<int32_t>((size_t)2 * r);
    int32_t* pos = ar.get<int32_t>((size_t)r);
    int* acc = ar.get<int>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    curk::mv_iota<<<1, 256, 0, st>>>(cand, 1, 2 * r, 0);
    CUR_CK(cudaGetLastError());
    note_launch();
    CUR_CK(cudaMemsetAsync(acc, 0, sizeof(int), st));
    CUR_TRY(merge_level(h, dt, rows, 2 * r, r, cand, 2, o, pos, acc, ar, st));
    if (dt == CUR_F64)
        curk::pair_emit_k<double><<<1, 256, 0, st>>>(static_cast<const double*>(rows), ids, pos, r, ids_out,
                                                     static_cast<double*>(rows_out), swaps_out, acc);
    else
        curk::pair_emit_k<float><<<1, 256, 0, st>>>(static_cast<const float*>(rows), ids, pos, r, ids_out,
                                                    static_cast<float*>(rows_out), swaps_out, acc);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

template <typename TA>
static cur_status gather_cols_t(const cur_mat* A, const int32_t* J, int r, void* C, cudaStream_t st, const int* idle) {
    const TA* a = static_cast<const TA*>(A->data);
    const int64_t total = A->rows * r;
    if (A->dtype == CUR_F64)
        curk::gather_cols_k<TA, double><<<curk::nblk(total), 256, 0, st>>>(a, A->rows, A->cols, A->ld, J, r, static_cast<double*>(C), nullptr, idle);
    else
        curk::gather_cols_k<TA, float><<<curk::nblk(total), 256, 0, st>>>(a, A->rows, A->cols, A->ld, J, r, static_cast<float*>(C), nullptr, idle);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status gather_cols_compute(const cur_mat* A, const int32_t* J, int r, void* C, cudaStream_t st, const int* idle) {
    switch (A->dtype) {
        case CUR_F64: return gather_cols_t<double>(A, J, r, C, st, idle);
        case CUR_F32: return gather_cols_t<float>(A, J, r, C, st, idle);
        case CUR_BF16: return gather_cols_t<__nv_bfloat16>(A, J, r, C, st, idle);
    }
    return CUR_ERR_ARG;
}

template <typename TA>
static cur_status gather_rows_t_t(const cur_mat* A, const int32_t* I, int r, void* Rt, cudaStream_t st, const int* idle) {
    const TA* a = static_cast<const TA*>(A->data);
    const unsigned grid = (unsigned)((A->cols + 31) / 32);
    if (A->dtype == CUR_F64) {
        const size_t sm = (size_t)r * 33 * sizeof(double);
        CUR_TRY(smem_attr((const void*)curk::gather_rows_t_k<TA, double>, sm));
        curk::gather_rows_t_k<TA, double><<<grid, 256, sm, st>>>(a, A->rows, A->cols, A->ld, I, r, static_cast<double*>(Rt), nullptr, idle);
    } else {
        const size_t sm = (size_t)r * 33 * sizeof(float);
        CUR_TRY(smem_attr((const void*)curk::gather_rows_t_k<TA, float>, sm));
        curk::gather_rows_t_k<TA, float><<<grid, 256, sm, st>>>(a, A->rows, A->cols, A->ld, I, r, static_cast<float*>(Rt), nullptr, idle);
    }
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status gather_rows_t_compute(const cur_mat* A, const int32_t* I, int r, void* Rt, cudaStream_t st, const int* idle) {
    switch (A->dtype) {
        case CUR_F64: return gather_rows_t_t<double>(A, I, r, Rt, st, idle);
        case CUR_F32: return gather_rows_t_t<float>(A, I, r, Rt, st, idle);
        case CUR_BF16: return gather_rows_t_t<__nv_bfloat16>(A, I, r, Rt, st, idle);
    }
    return CUR_ERR_ARG;
}

cur_status logvol_rows(cur_dtype dt, const void* basis, int64_t p, int r, const int32_t* rows, double* out,
                       cudaStream_t st) {
    const size_t sm = (size_t)r * r * sizeof(double);
    if (dt == CUR_F64) {
        CUR_TRY(curk::set_smem_attr(curk::logvol_rows_k<double>, sm));
        curk::logvol_rows_k<double><<<1, 512, sm, st>>>(static_cast<const double*>(basis), p, r, rows, out);
    } else {
        CUR_TRY(curk::set_smem_attr(curk::logvol_rows_k<float>, sm));
        curk::logvol_rows_k<float><<<1, 512, sm, st>>>(static_cast<const float*>(basis), p, r, rows, out);
    }
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status pad_indices_dev(int32_t* idx, const int32_t* count, int r, int64_t size, cudaStream_t st) {
    curk::pad_indices_k<<<1, 32, 0, st>>>(idx, count, r, size);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

// ================================================================ batches of matrices
//
// The cross of every matrix of a batch with each stage shared by all matrices: one launch
// of Algorithm 3 for all of them (batched_aca.cu), then the row selection (every block of
// every matrix in one stage, each merge level of all matrices in one stage, every polish
// in one stage), the column selection the same way, and the sweeps (one stage per
// half-sweep over the matrices that have not converged). FP32 data; each problem keeps
// its own rank, the stage's stride is the largest.

namespace curk {

struct BatGItem {         // matrix t of the batch, for the gathers
    int64_t aoff, m, n, ld;
    int32_t r;
    int64_t coff;         // its basis at C + coff (m x r for columns J, n x r for rows I)
    int64_t ioff;         // its indices at idx + ioff
};

// C(i, k) = A(i, J_k), m x r, for matrix blockIdx.y.
__global__ void bat_gather_cols_k(const float* __restrict__ data, const BatGItem* items,
                                  const int32_t* __restrict__ J, float* __restrict__ C) {
    const BatGItem b = items[blockIdx.y];
    const int64_t total = b.m * b.r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / b.r;
        const int k = (int)(e - i * b.r);
        C[b.coff + e] = data[b.aoff + i * b.ld + J[b.ioff + k]];
    }
}

// Rt(j, k) = A(I_k, j), n x r, for matrix blockIdx.y (reads along rows of A).
__global__ void bat_gather_rows_t_k(const float* __restrict__ data, const BatGItem* items,
                                    const int32_t* __restrict__ I, float* __restrict__ Rt) {
    const BatGItem b = items[blockIdx.y];
    const int64_t total = b.n * b.r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / b.n);
        const int64_t j = e - (int64_t)k * b.n;
        Rt[b.coff + j * b.r + k] = data[b.aoff + (int64_t)I[b.ioff + k] * b.ld + j];
    }
}

// out[pb rs + k] = global id of S[pb rs + k] for k < r(pb), -1 after.
__global__ void bat_emit_k(const MvProb* prob, const int32_t* S, int P, int rs, int32_t* out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * rs; e += gridDim.x * blockDim.x) {
        const int pb = e / rs, k = e - pb * rs;
        const MvProb pr = prob[pb];
        if (k >= pr.r) { out[e] = -1; continue; }
        const int s = S[e];
        out[e] = pr.gid_arr ? pr.gid_arr[s] : (int32_t)(pr.gid_base + s);
    }
}

// Start rows of the flagged problems: k (left set) or r(pb) + k (right set).
__global__ void bat_iota_k(const int32_t* rr, const int32_t* flag, int P, int rs, int right, int32_t* S) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * rs; e += gridDim.x * blockDim.x) {
        const int pb = e / rs, k = e - pb * rs;
        if (flag && !flag[pb]) continue;
        S[e] = right ? rr[pb] + k : k;
    }
}

// dst row d (rs entries) = src row idx[d].
__global__ void bat_rows_copy_k(const int32_t* src, const int32_t* idx, int D, int rs, int32_t* dst) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D * rs; e += gridDim.x * blockDim.x) {
        const int d = e / rs, k = e - d * rs;
        dst[e] = src[(int64_t)idx[d] * rs + k];
    }
}

// dst row idx[d] = src row d.
__global__ void bat_rows_scatter_k(const int32_t* src, const int32_t* idx, int D, int rs, int32_t* dst) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D * rs; e += gridDim.x * blockDim.x) {
        const int d = e / rs, k = e - d * rs;
        dst[(int64_t)idx[d] * rs + k] = src[e];
    }
}

struct BatUnion {
    int64_t uoff;     // union rows at U + uoff (2 r x r)
    int64_t boff;     // the matrix's basis at basis + boff (p x r)
    int32_t r, p;
    int32_t left, right;   // set rows in the current set array
};

// cand[q 2rs + x] = left set (x < r), right set (r <= x < 2r); U = basis rows of cand.
__global__ void bat_union_k(const float* __restrict__ basis, const BatUnion* un, const int32_t* sets, int rs,
                            int32_t* cand, float* __restrict__ U, int* status) {
    const BatUnion u = un[blockIdx.y];
    int32_t* cq = cand + (int64_t)blockIdx.y * 2 * rs;
    for (int x = threadIdx.x; x < 2 * u.r; x += blockDim.x)
        cq[x] = x < u.r ? sets[(int64_t)u.left * rs + x] : sets[(int64_t)u.right * rs + x - u.r];
    __syncthreads();
    const int64_t total = (int64_t)2 * u.r * u.r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e / u.r), c = (int)(e - (int64_t)x * u.r);
        const int32_t g = cq[x];
        if (g < 0 || g >= u.p) { set_status(status, CUR_ERR_ARG); U[u.uoff + e] = 0.f; continue; }
        U[u.uoff + e] = basis[u.boff + (int64_t)g * u.r + c];
    }
}

// Pad J0 of each matrix (count[t] valid entries) with its lowest unused column ids.
__global__ void bat_pad_k(int32_t* J, const int64_t* joff, const int32_t* rr, const int64_t* nn,
                          const int32_t* count, int T) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int32_t* j = J + joff[t];
        const int r = rr[t];
        int fill = count[t];
        for (int64_t cand = 0; cand < nn[t] && fill < r; ++cand) {
            bool used = false;
            for (int q = 0; q < fill; ++q) used |= j[q] == cand;
            if (!used) j[fill++] = (int32_t)cand;
        }
    }
}

// Unpacked per-matrix indices (stride rs) to the packed output and back.
__global__ void bat_pack_k(const int32_t* src, const int64_t* off, const int32_t* rr, int T, int rs,
                           int32_t* dst, int to_packed) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < T * rs; e += gridDim.x * blockDim.x) {
        const int t = e / rs, k = e - t * rs;
        if (k >= rr[t]) continue;
        if (to_packed) dst[off[t] + k] = src[e];
        else dst[e] = src[off[t] + k];
    }
}

struct BatBasis {
    int64_t boff;       // basis of matrix t at basis + boff, p x r
    int32_t p, r, nb;   // rows, rank, blocks
};

// Tables of a batch reach the device as kernel parameters (upload_table): no host wait.
static cur_status bat_upload(cur_handle*, void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return upload(dst, src, bytes, st);
}

// ---- per-matrix bookkeeping on the device: every decision of the batched cross (a merge
// node's next start, the end of a matrix's sweeps, its status) is taken by these kernels,
// so cur_cross_batched only enqueues (once its launch shape is tuned).

// acc_m[item[pb]] += swaps[pb]
__global__ void bat_acc_k(const int32_t* swaps, const int32_t* item, int P, int32_t* acc_m) {
    for (int pb = blockIdx.x * blockDim.x + threadIdx.x; pb < P; pb += gridDim.x * blockDim.x)
        atomicAdd(&acc_m[item[pb]], swaps[pb]);
}

// merge_retry_k for nodes of per-problem rank rr and per-matrix swap counts.
__global__ void bat_merge_retry_k(int attempt, int P, int rs, const int32_t* rr, const int32_t* item,
                                  int32_t* pstatus, int32_t* swaps, int32_t* done, int32_t* lu_mask, int32_t* S,
                                  int32_t* retry, int32_t* acc_m, unsigned* bar) {
    for (int pb = blockIdx.x * blockDim.x + threadIdx.x; pb < P; pb += gridDim.x * blockDim.x) {
        bar[pb] = 0u;   // for the next attempt's Algorithm 3 start
        if (attempt > 0 && retry[pb] != attempt) continue;
        if (attempt < 2 && pstatus[pb] == CUR_ERR_SINGULAR) {
            retry[pb] = attempt + 1;
            pstatus[pb] = CUR_OK;
            swaps[pb] = 0;
            done[pb] = 0;
            lu_mask[pb] = 1;
            if (attempt == 0)
                for (int k = 0; k < rr[pb]; ++k) S[(int64_t)pb * rs + k] = rr[pb] + k;
        } else {
            retry[pb] = 0;
            atomicAdd(&acc_m[item[pb]], swaps[pb]);
        }
    }
}

// The polish of each matrix: its status, and its swaps added.
__global__ void bat_polish_end_k(const int32_t* pstatus, const int32_t* swaps, int T, int32_t* side_stat,
                                 int32_t* acc_m) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        side_stat[t] = pstatus[t];
        acc_m[t] += swaps[t];
    }
}

// A sweep stage runs only the matrices still sweeping.
__global__ void bat_live_done_k(const int32_t* live, int T, int32_t* done) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) done[t] = live[t] ? 0 : 1;
}

__global__ void bat_copy_lv_k(const double* src, const int32_t* live, int T, double* lv) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        if (live[t]) lv[t] = src[t];
}

// Algorithm 3 ran out before r picks: CUR_WARN_RANK for that matrix.
__global__ void bat_warn_k(const int32_t* cnt, const int32_t* rr, int T, int32_t* mstat) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        mstat[t] = cnt[t] < rr[t] ? CUR_WARN_RANK : CUR_OK;
}

// Sweep 1 (blockwise rows, then columns) of every matrix is over.
__global__ void bat_sweep1_k(int T, const int32_t* st_r, const int32_t* sw_r, const int32_t* st_c,
                             const int32_t* sw_c, int32_t* mstat, int32_t* msw, int32_t* msweeps, int32_t* live) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        for (int k = 0; k < 8; ++k) msw[t * 8 + k] = 0;
        msw[t * 8] = sw_r[t] + sw_c[t];
        msweeps[t] = 1;
        if (st_r[t] != CUR_OK) mstat[t] = st_r[t];
        if (st_c[t] != CUR_OK) mstat[t] = st_c[t];
        live[t] = 1;
    }
}

// A later sweep of the matrices still sweeping: it ends a matrix's sweeps if a stage ended
// with an error or nothing was swapped.
__global__ void bat_sweep_end_k(int sweep, int T, const int32_t* q1, const int32_t* s1, const int32_t* q2,
                                const int32_t* s2, int32_t* live, int32_t* msweeps, int32_t* msw, int32_t* mstat) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        if (!live[t]) continue;
        msweeps[t] = sweep;
        msw[t * 8 + sweep - 1] = s1[t] + s2[t];
        if (q1[t] != CUR_OK || q2[t] != CUR_OK) {
            mstat[t] = q1[t] != CUR_OK ? q1[t] : q2[t];
            live[t] = 0;
        } else if (s1[t] + s2[t] == 0) {
            live[t] = 0;
        }
    }
}

// log|det A(I,J)| of each matrix whose cross ended with an error (one CTA per matrix): such a
// stage leaves no log|det| of its own.
__global__ void __launch_bounds__(256) bat_logvol_k(const float* Rt, const BatBasis* brt, const int32_t* J, int rs,
                                                    const int32_t* mstat, double* lvf) {
    const int t = blockIdx.x;
    const int sv = mstat[t];
    if (sv == CUR_OK || sv == CUR_WARN_RANK) return;
    const BatBasis b = brt[t];
    logvol_rows_dev<float>(Rt + b.boff, b.p, b.r, J + (int64_t)t * rs, lvf + t);
}

// The host-visible outcome: the status word (the last SINGULAR / NOCONV in matrix order, else
// CUR_WARN_RANK if any matrix's Algorithm 3 ran out) and each matrix's cur_cross_info.
__global__ void bat_finish_k(int T, const int32_t* mstat, const int32_t* cnt, const int32_t* msweeps,
                             const int32_t* msw, const double* lvc, const double* lvf, cur_cross_info* info,
                             int* hstatus) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int worst = CUR_OK, warn = 0;
        for (int t = 0; t < T; ++t) {
            if (mstat[t] == CUR_ERR_SINGULAR || mstat[t] == CUR_ERR_NOCONV) worst = mstat[t];
            if (mstat[t] == CUR_WARN_RANK) warn = 1;
        }
        if (worst != CUR_OK) set_status(hstatus, worst);
        else if (warn) set_status(hstatus, CUR_WARN_RANK);
    }
    if (!info) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        cur_cross_info f;
        const int sv = mstat[t];
        f.logvol = (sv != CUR_OK && sv != CUR_WARN_RANK) ? lvf[t] : lvc[t];
        f.sweeps = msweeps[t];
        f.swaps_total = 0;
        for (int k = 0; k < 8; ++k) {
            f.sweep_swaps[k] = msw[t * 8 + k];
            f.swaps_total += msw[t * 8 + k];
        }
        f.aca_selected = cnt[t];
        f.status = sv;
        info[t] = f;
    }
}

// Maxvol row selection (blocks, binary merge, polish) on every basis of `bs`. out: device,
// row t at t rs (local row ids); logvol: device, one double per matrix; side_stat: device,
// the polish's status per matrix; acc_m: device, swaps added per matrix.
static cur_status bat_rows(cur_handle* h, const float* basis, const std::vector<BatBasis>& bs, int rs,
                           const cur_opts* o, int32_t* out, double* logvol, int32_t* side_stat, int32_t* acc_m,
                           Arena& ar, cudaStream_t st) {
    const int T = (int)bs.size();
    const size_t mark = ar.off;
    // ---- blocks: Algorithm 3 start and maxvol on each block of each matrix
    std::vector<std::vector<int>> sets(T);
    std::vector<int32_t> item;
    Stage<float> sb;
    for (int t = 0; t < T; ++t) {
        const int64_t base_sz = bs[t].p / bs[t].nb, extra = bs[t].p % bs[t].nb;
        int64_t s0 = 0;
        for (int k = 0; k < bs[t].nb; ++k) {
            const int64_t sz = base_sz + (k < extra ? 1 : 0);
            MvProb pr{};
            pr.base = s0;
            pr.boff = bs[t].boff + s0 * bs[t].r;
            pr.r = bs[t].r;
            pr.p = (int32_t)sz;
            pr.gid_base = s0;
            sets[t].push_back((int)sb.probs.size());
            sb.probs.push_back(pr);
            item.push_back(t);
            s0 += sz;
        }
    }
    CUR_TRY(stage_setup<float>(h, rs, sb, ar, true));
    int32_t* ditem = ar.get<int32_t>(item.size());
    int32_t* cur = ar.get<int32_t>((size_t)sb.P * rs);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(stage_tables(sb, st));
    CUR_TRY(stage_init(sb, nullptr, st));
    CUR_TRY(stage_launch<float>(h, basis, rs, o, sb, true, st));
    CUR_TRY(bat_upload(h, ditem, item.data(), sizeof(int32_t) * item.size(), st));
    bat_acc_k<<<nblk(sb.P), 256, 0, st>>>(sb.swaps, ditem, sb.P, acc_m);
    bat_emit_k<<<nblk((int64_t)sb.P * rs), 256, 0, st>>>(sb.dprob, sb.S, sb.P, rs, cur);
    CUR_CK(cudaGetLastError());
    note_launch(2);
    // ---- merge levels: node (2u, 2u+1) of every matrix that still has two sets or more
    std::vector<Stage<float>> keep;   // stages stay alive while their memory is in use
    keep.reserve(16);
    while (true) {
        std::vector<BatUnion> un;
        std::vector<int32_t> node_item, pass_src, hr;
        std::vector<std::vector<int>> nsets(T);
        int64_t uoff = 0;
        for (int t = 0; t < T; ++t) {
            const auto& L = sets[t];
            for (size_t u = 0; u + 1 < L.size(); u += 2) {
                BatUnion b{};
                b.uoff = uoff;
                b.boff = bs[t].boff;
                b.r = bs[t].r;
                b.p = bs[t].p;
                b.left = L[u];
                b.right = L[u + 1];
                nsets[t].push_back((int)un.size());
                un.push_back(b);
                node_item.push_back(t);
                hr.push_back(b.r);
                uoff += (int64_t)2 * b.r * b.r;
            }
        }
        const int Q = (int)un.size();
        if (Q == 0) break;
        for (int t = 0; t < T; ++t)
            if (sets[t].size() % 2 == 1 && sets[t].size() > 1) {
                nsets[t].push_back(Q + (int)pass_src.size());
                pass_src.push_back(sets[t].back());
            } else if (sets[t].size() == 1) {
                nsets[t].push_back(Q + (int)pass_src.size());
                pass_src.push_back(sets[t][0]);
            }
        BatUnion* dun = ar.get<BatUnion>(Q);
        int32_t* cand = ar.get<int32_t>((size_t)Q * 2 * rs);
        float* U = ar.get<float>((size_t)uoff);
        int32_t* rr = ar.get<int32_t>(Q);
        int32_t* nitem = ar.get<int32_t>(Q);
        int32_t* nxt = ar.get<int32_t>((size_t)(Q + pass_src.size()) * rs);
        int32_t* psrc = ar.get<int32_t>(pass_src.size() + 1);
        if (!ar.ok) return CUR_ERR_NOMEM;
        CUR_TRY(bat_upload(h, dun, un.data(), sizeof(BatUnion) * Q, st));
        CUR_TRY(bat_upload(h, rr, hr.data(), sizeof(int32_t) * Q, st));
        CUR_TRY(bat_upload(h, nitem, node_item.data(), sizeof(int32_t) * Q, st));
        bat_union_k<<<dim3(4, Q), 256, 0, st>>>(basis, dun, cur, rs, cand, U, h->status);
        CUR_CK(cudaGetLastError());
        note_launch();
        keep.emplace_back();
        Stage<float>& lv = keep.back();
        for (int q = 0; q < Q; ++q) {
            MvProb pr{};
            pr.base = 0;
            pr.boff = un[q].uoff;
            pr.r = un[q].r;
            pr.p = 2 * un[q].r;
            pr.gid_arr = cand + (int64_t)q * 2 * rs;
            lv.probs.push_back(pr);
        }
        CUR_TRY(stage_setup<float>(h, rs, lv, ar));
        CUR_TRY(stage_tables(lv, st));
        CUR_TRY(stage_init(lv, nullptr, st));
        bat_iota_k<<<nblk((int64_t)Q * rs), 256, 0, st>>>(rr, nullptr, Q, rs, 0, lv.S);
        CUR_CK(cudaGetLastError());
        note_launch();
        // the left set; where it is singular, the right set; where both are, Algorithm 3 on
        // the union (the swaps of an abandoned attempt are not counted)
        for (int attempt = 0; attempt < 3; ++attempt) {
            CUR_TRY(stage_launch<float>(h, U, rs, o, lv, attempt == 2, st));
            bat_merge_retry_k<<<nblk(Q), 256, 0, st>>>(attempt, Q, rs, rr, nitem, lv.pstatus, lv.swaps, lv.done,
                                                       lv.dtab + 2 * lv.slots, lv.S, lv.retry, acc_m, lv.bar);
            CUR_CK(cudaGetLastError());
            note_launch();
        }
        bat_emit_k<<<nblk((int64_t)Q * rs), 256, 0, st>>>(lv.dprob, lv.S, Q, rs, nxt);
        CUR_CK(cudaGetLastError());
        note_launch();
        if (!pass_src.empty()) {
            CUR_TRY(bat_upload(h, psrc, pass_src.data(), sizeof(int32_t) * pass_src.size(), st));
            bat_rows_copy_k<<<nblk((int64_t)pass_src.size() * rs), 256, 0, st>>>(cur, psrc, (int)pass_src.size(), rs,
                                                                                nxt + (int64_t)Q * rs);
            CUR_CK(cudaGetLastError());
            note_launch();
        }
        cur = nxt;
        sets.swap(nsets);
    }
    // ---- polish: maxvol over all rows of each matrix from its merged set
    Stage<float> sp;
    std::vector<int32_t> src(T);
    for (int t = 0; t < T; ++t) {
        MvProb pr{};
        pr.base = 0;
        pr.boff = bs[t].boff;
        pr.r = bs[t].r;
        pr.p = bs[t].p;
        sp.probs.push_back(pr);
        src[t] = sets[t][0];
    }
    CUR_TRY(stage_setup<float>(h, rs, sp, ar));
    int32_t* dsrc = ar.get<int32_t>(T);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(stage_tables(sp, st));
    CUR_TRY(stage_init(sp, nullptr, st));
    CUR_TRY(bat_upload(h, dsrc, src.data(), sizeof(int32_t) * T, st));
    bat_rows_copy_k<<<nblk((int64_t)T * rs), 256, 0, st>>>(cur, dsrc, T, rs, sp.S);
    CUR_CK(cudaGetLastError());
    note_launch();
    cur_opts o2 = *o;
    if (!(o->flags & CUR_FLAG_POLISH)) o2.delta = 1e300;   // no swap: one factorisation for log|det|
    CUR_TRY(stage_launch<float>(h, basis, rs, &o2, sp, false, st));
    bat_polish_end_k<<<nblk(T), 256, 0, st>>>(sp.pstatus, sp.swaps, T, side_stat, acc_m);
    CUR_CK(cudaGetLastError());
    note_launch();
    CUR_CK(cudaMemcpyAsync(out, sp.S, sizeof(int32_t) * T * rs, cudaMemcpyDeviceToDevice, st));
    CUR_CK(cudaMemcpyAsync(logvol, sp.logvol, sizeof(double) * T, cudaMemcpyDeviceToDevice, st));
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

// Global maxvol over all rows of every basis from S (device, row t at t rs), in place, for
// the matrices still sweeping (live); a set that turns singular stays as reached (the swap
// iteration's own result). stat, swaps: device, per matrix; lv (may be null): log|det| of the
// live matrices.
static cur_status bat_global(cur_handle* h, const float* basis, const std::vector<BatBasis>& bs, int rs,
                             const cur_opts* o, int32_t* S, double* lv, const int32_t* live, int32_t* stat,
                             int32_t* swaps, Arena& ar, cudaStream_t st) {
    const int T = (int)bs.size();
    const size_t mark = ar.off;
    Stage<float> sg;
    sg.keep_singular_set = true;
    for (int t = 0; t < T; ++t) {
        MvProb pr{};
        pr.boff = bs[t].boff;
        pr.r = bs[t].r;
        pr.p = bs[t].p;
        sg.probs.push_back(pr);
    }
    CUR_TRY(stage_setup<float>(h, rs, sg, ar));
    CUR_TRY(stage_tables(sg, st));
    CUR_TRY(stage_init(sg, nullptr, st));
    bat_live_done_k<<<nblk(T), 256, 0, st>>>(live, T, sg.done);
    CUR_CK(cudaGetLastError());
    note_launch();
    CUR_CK(cudaMemcpyAsync(sg.S, S, sizeof(int32_t) * T * rs, cudaMemcpyDeviceToDevice, st));
    CUR_TRY(stage_launch<float>(h, basis, rs, o, sg, false, st));
    CUR_CK(cudaMemcpyAsync(S, sg.S, sizeof(int32_t) * T * rs, cudaMemcpyDeviceToDevice, st));
    CUR_CK(cudaMemcpyAsync(stat, sg.pstatus, sizeof(int32_t) * T, cudaMemcpyDeviceToDevice, st));
    CUR_CK(cudaMemcpyAsync(swaps, sg.swaps, sizeof(int32_t) * T, cudaMemcpyDeviceToDevice, st));
    if (lv) {
        bat_copy_lv_k<<<nblk(T), 256, 0, st>>>(sg.logvol, live, T, lv);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

}  // namespace curk

size_t bat_aca_workspace(int grid);
size_t bat_aca_item_size();
cur_status bat_aca_launch(const float* data, const void* items_dev, const int32_t* order, int* queue, int count,
                          int32_t* J, int32_t* counts, float* Qws, int grid, int* status, cudaStream_t st);

// The cross of every matrix of the batch (see cur_cross_batched).
cur_status cross_batched_impl(cur_handle* h, const float* data, const cur_batch_item* items, int T,
                              const cur_opts* o, int32_t* IJ_out, cur_cross_info* info_out, Arena& ar,
                              cudaStream_t st) {
    using namespace curk;
    int rs = 1;
    int64_t sum_r = 0, sum_mr = 0, sum_nr = 0;
    for (int t = 0; t < T; ++t) {
        rs = std::max(rs, (int)items[t].r);
        sum_r += items[t].r;
        sum_mr += items[t].rows * items[t].r;
        sum_nr += items[t].cols * items[t].r;
    }
    // ---- per-matrix tables
    struct AcaIt { int64_t aoff, m, n, ld; int32_t r; int64_t joff; };
    std::vector<AcaIt> ai(T);
    std::vector<BatGItem> gc(T), gr(T);
    std::vector<BatBasis> bc(T), brt(T);
    std::vector<int64_t> joff(T), nn(T), io(T), jo2(T);
    std::vector<int32_t> rr(T);
    int64_t jo = 0, co = 0, ro = 0;
    for (int t = 0; t < T; ++t) {
        const cur_batch_item& b = items[t];
        ai[t] = AcaIt{b.offset, b.rows, b.cols, b.ld, b.r, jo};
        joff[t] = jo;
        io[t] = 2 * jo;
        jo2[t] = 2 * jo + b.r;
        nn[t] = b.cols;
        rr[t] = b.r;
        gc[t] = BatGItem{b.offset, b.rows, b.cols, b.ld, b.r, co, (int64_t)t * rs};
        gr[t] = BatGItem{b.offset, b.rows, b.cols, b.ld, b.r, ro, (int64_t)t * rs};
        bc[t] = BatBasis{co, (int32_t)b.rows, b.r, b.b_r};
        brt[t] = BatBasis{ro, (int32_t)b.cols, b.r, b.b_c};
        jo += b.r;
        co += b.rows * b.r;
        ro += b.cols * b.r;
    }
    static_assert(sizeof(AcaIt) == 48, "BatAcaItem layout");
    if (bat_aca_item_size() != sizeof(AcaIt)) return CUR_ERR_ARG;
    // Algorithm 3 launch shape: one or two CTAs per SM (a CTA runs a whole matrix, so the
    // result does not depend on it), tuned per class of batch size and work per matrix
    double work = 0.0;
    for (int t = 0; t < T; ++t) work += (double)items[t].rows * items[t].cols * items[t].r;
    const uint64_t tkey = (1ull << 56) | (tune_log2((uint64_t)T) << 8) | tune_log2((uint64_t)(work / T) + 1);
    const int grid_max = std::min(T, 2 * h->num_sms);
    void* dai = ar.take(sizeof(AcaIt) * T);
    BatGItem* dgc = ar.get<BatGItem>(T);
    BatGItem* dgr = ar.get<BatGItem>(T);
    BatBasis* dbrt = ar.get<BatBasis>(T);
    int64_t* djoff = ar.get<int64_t>(T);
    int64_t* dnn = ar.get<int64_t>(T);
    int64_t* dio = ar.get<int64_t>(T);
    int64_t* djo = ar.get<int64_t>(T);
    int32_t* drr = ar.get<int32_t>(T);
    int32_t* J0 = ar.get<int32_t>(sum_r);
    int32_t* cnt = ar.get<int32_t>(T);
    float* Qws = static_cast<float*>(ar.take(bat_aca_workspace(grid_max)));
    float* C = ar.get<float>(sum_mr);
    float* Rt = ar.get<float>(sum_nr);
    int32_t* I = ar.get<int32_t>((size_t)T * rs);
    int32_t* J = ar.get<int32_t>((size_t)T * rs);
    double* lvc = ar.get<double>(T);
    double* lvf = ar.get<double>(T);
    int32_t* dorder = ar.get<int32_t>(T);
    int* queue = ar.get<int>(1);
    // per-matrix state on the device: status, sweeps, swaps per sweep, still sweeping; the
    // two sides' polish statuses and swap counts; the sweep stages' statuses and swaps
    int32_t* mstat = ar.get<int32_t>(T);
    int32_t* msweeps = ar.get<int32_t>(T);
    int32_t* msw = ar.get<int32_t>((size_t)8 * T);
    int32_t* live = ar.get<int32_t>(T);
    int32_t* acc = ar.get<int32_t>((size_t)2 * T);   // swaps of sweep 1: rows, columns
    int32_t* sst = ar.get<int32_t>((size_t)2 * T);   // polish statuses of sweep 1: rows, columns
    int32_t* qs = ar.get<int32_t>((size_t)4 * T);    // a later sweep: q1, s1, q2, s2
    if (!ar.ok) return CUR_ERR_NOMEM;
    {
        std::vector<int32_t> order(T);
        for (int t = 0; t < T; ++t) order[t] = t;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return items[x].rows * items[x].cols * items[x].r > items[y].rows * items[y].cols * items[y].r;
        });
        CUR_TRY(bat_upload(h, dorder, order.data(), sizeof(int32_t) * T, st));
    }
    CUR_TRY(bat_upload(h, dai, ai.data(), sizeof(AcaIt) * T, st));
    CUR_TRY(bat_upload(h, dgc, gc.data(), sizeof(BatGItem) * T, st));
    CUR_TRY(bat_upload(h, dgr, gr.data(), sizeof(BatGItem) * T, st));
    CUR_TRY(bat_upload(h, dbrt, brt.data(), sizeof(BatBasis) * T, st));
    CUR_TRY(bat_upload(h, djoff, joff.data(), sizeof(int64_t) * T, st));
    CUR_TRY(bat_upload(h, dnn, nn.data(), sizeof(int64_t) * T, st));
    CUR_TRY(bat_upload(h, dio, io.data(), sizeof(int64_t) * T, st));
    CUR_TRY(bat_upload(h, djo, jo2.data(), sizeof(int64_t) * T, st));
    CUR_TRY(bat_upload(h, drr, rr.data(), sizeof(int32_t) * T, st));
    // ---- J0: Algorithm 3 on the columns of every matrix, padded per matrix
    const int tuned = tune_lookup(h, tkey);
    if (tuned >= 0) {
        CUR_TRY(bat_aca_launch(data, dai, dorder, queue, T, J0, cnt, Qws, std::min(T, tuned * h->num_sms),
                               h->status, st));
    } else {
        // first batch of this class: time both shapes (each computes the same J0), keep the
        // faster; this first call waits for the two timed launches
        float best_ms = 0.f;
        int best = 2;
        for (int per_sm = 1; per_sm <= 2; ++per_sm) {
            CUR_CK(cudaEventRecord(h->tune_ev[0], st));
            CUR_TRY(bat_aca_launch(data, dai, dorder, queue, T, J0, cnt, Qws, std::min(T, per_sm * h->num_sms),
                                   h->status, st));
            CUR_CK(cudaEventRecord(h->tune_ev[1], st));
            CUR_CK(cudaEventSynchronize(h->tune_ev[1]));
            float ms = 0.f;
            CUR_CK(cudaEventElapsedTime(&ms, h->tune_ev[0], h->tune_ev[1]));
            if (per_sm == 1 || ms < best_ms) { best_ms = ms; best = per_sm; }
        }
        tune_store(h, tkey, best);
    }
    bat_warn_k<<<nblk(T), 256, 0, st>>>(cnt, drr, T, mstat);
    bat_pad_k<<<nblk(T, 128), 128, 0, st>>>(J0, djoff, drr, dnn, cnt, T);
    bat_pack_k<<<nblk((int64_t)T * rs), 256, 0, st>>>(J0, djoff, drr, T, rs, J, 0);
    CUR_CK(cudaGetLastError());
    note_launch(3);
    auto gather_c = [&](const int32_t* Jd) -> cur_status {
        bat_gather_cols_k<<<dim3(8, T), 256, 0, st>>>(data, dgc, Jd, C);
        CUR_CK(cudaGetLastError());
        note_launch();
        return CUR_OK;
    };
    auto gather_r = [&](const int32_t* Id) -> cur_status {
        bat_gather_rows_t_k<<<dim3(8, T), 256, 0, st>>>(data, dgr, Id, Rt);
        CUR_CK(cudaGetLastError());
        note_launch();
        return CUR_OK;
    };
    // ---- sweep 1: blockwise rows on A(:,J0), then blockwise columns on A(I,:)^T
    CUR_CK(cudaMemsetAsync(acc, 0, sizeof(int32_t) * 2 * T, st));
    CUR_TRY(gather_c(J));
    CUR_TRY(bat_rows(h, C, bc, rs, o, I, lvc, sst, acc, ar, st));
    CUR_TRY(gather_r(I));
    CUR_TRY(bat_rows(h, Rt, brt, rs, o, J, lvc, sst + T, acc + T, ar, st));
    bat_sweep1_k<<<nblk(T), 256, 0, st>>>(T, sst, acc, sst + T, acc + T, mstat, msw, msweeps, live);
    CUR_CK(cudaGetLastError());
    note_launch();
    // ---- sweeps 2..8: global rows from I, global columns from J, for the matrices still
    // sweeping (every sweep is enqueued; a matrix that has stopped takes no part)
    for (int sweep = 2; sweep <= 8; ++sweep) {
        CUR_TRY(gather_c(J));
        CUR_TRY(bat_global(h, C, bc, rs, o, I, nullptr, live, qs, qs + T, ar, st));
        CUR_TRY(gather_r(I));
        CUR_TRY(bat_global(h, Rt, brt, rs, o, J, lvc, live, qs + 2 * T, qs + 3 * T, ar, st));
        bat_sweep_end_k<<<nblk(T), 256, 0, st>>>(sweep, T, qs, qs + T, qs + 2 * T, qs + 3 * T, live, msweeps, msw,
                                                 mstat);
        CUR_CK(cudaGetLastError());
        note_launch();
    }
    // ---- outputs; a matrix whose cross did not end OK reports log|det A(I,J)| taken directly
    bat_pack_k<<<nblk((int64_t)T * rs), 256, 0, st>>>(I, dio, drr, T, rs, IJ_out, 1);
    bat_pack_k<<<nblk((int64_t)T * rs), 256, 0, st>>>(J, djo, drr, T, rs, IJ_out, 1);
    CUR_CK(cudaGetLastError());
    CUR_TRY(smem_attr((const void*)bat_logvol_k, (size_t)rs * rs * sizeof(double)));
    bat_logvol_k<<<T, 256, (size_t)rs * rs * sizeof(double), st>>>(Rt, dbrt, J, rs, mstat, lvf);
    CUR_CK(cudaGetLastError());
    bat_finish_k<<<nblk(T), 256, 0, st>>>(T, mstat, cnt, msweeps, msw, lvc, lvf, info_out, h->status);
    CUR_CK(cudaGetLastError());
    note_launch(4);
    return CUR_OK;
}
