// Block-wise maximal-volume selection with a binary merge (GB300 form).
//
// The maximal-volume problem (Section 1.2, Definition 1) on a tall basis C
// (p x r) is attacked by the swap iteration: with M = C(S,:) and B = C M^-1,
// every entry B_ij is the factor by which |det M| changes when row i of C
// replaces position j of S. While max|B_ij| > 1 + delta the best swap is made
// and B is updated by Sherman-Morrison, B <- B - B(:,j) (B(i,:) - e_j^T) / B_ij;
// every r swaps, and before declaring convergence, M^-1 and B are recomputed.
//
// Work is organised as "problems" (a row block of C, a merge node, or all of C),
// each handled by a group of CTAs:
//   mv_start : Algorithm 3 (axis 0) on the problem's rows -> start set S
//              (implicit Gram-Schmidt, one group barrier per pick)
//   mv_lu    : one CTA per problem, FP64 LU with partial pivoting of C(S,:),
//              inverse and log|det|
//   mv_coef  : B = C M^-1 for all problems (the coefficient product)
//   mv_swap  : the swap loop; each CTA keeps its slice of B in shared memory,
//              the group agrees on the argmax through one barrier per swap
// A host loop repeats lu -> coef -> swap until every problem has converged on a
// freshly recomputed B.

#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace curk {

constexpr double kEps = 2.220446049250313e-16;

struct MvProb {
    int64_t base;      // first row of the problem in the basis / B buffers
    int64_t gid_base;  // global id of local row i = gid_base + i (when gid_arr == null)
    const int32_t* gid_arr;
    int32_t p;         // rows
    int32_t G;         // CTAs in its group
    int32_t rpc;       // rows per CTA
    int32_t group0;    // first slot of its group
};

struct MvArgs {
    const void* basis;  // rows x r (compute type), contiguous
    void* B;            // rows x r (compute type)
    void* minv;         // P x r x r (compute type)
    double* minv64;     // P x r x r (FP64 inverse)
    const MvProb* prob;
    int P, r;
    double delta;
    int max_swaps;
    const int32_t* cta_prob;   // per CTA slot
    const int32_t* cta_part;
    int cta_base;              // first slot of this launch (waves)
    const int32_t* tile_prob;  // coef tiles
    const int32_t* tile_row0;
    int32_t* S;                // P x r local positions
    double* logvol;            // P
    int32_t* swaps;            // P
    int32_t* pstatus;          // P
    int32_t* done;             // P
    unsigned* bar;             // P
    int* pending;              // 1
    double* keyv;              // slots x 2
    long long* keyi;           // slots x 2
    void* pub;                 // slots x 2 x r (compute type)
    double* aux;               // slots x 2 (start: frob partials)
    int* status;               // handle status word
};

// ---------------------------------------------------------------- gathers

template <typename TA, typename TB>
__global__ void gather_cols_k(const TA* __restrict__ A, int64_t m, int64_t n, int64_t ld,
                              const int32_t* __restrict__ J, int r, TB* __restrict__ C,
                              int* status) {
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
                                                       TB* __restrict__ Rt, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
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

template <typename TB>
struct StartSmem {
    static size_t bytes(int nloc, int r) {
        size_t b = (size_t)nloc * r * sizeof(TB);
        b = (b + 15) / 16 * 16 + (size_t)nloc * sizeof(double);
        b += (size_t)r * r * sizeof(double);        // Q
        b += (size_t)4 * r * sizeof(double);        // v, s, scratch
        b += (size_t)2 * r * sizeof(float);         // qh, ql
        b += (size_t)nloc + 16;                     // mask
        return b;
    }
};

template <typename TB>
__global__ void __launch_bounds__(256) mv_start(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int slot = a.cta_base + blockIdx.x;
    const int pb = a.cta_prob[slot], part = a.cta_part[slot];
    const MvProb pr = a.prob[pb];
    const int r = a.r, G = pr.G;
    const int lo = part * pr.rpc, hi = min(pr.p, lo + pr.rpc), nloc = max(0, hi - lo);
    const TB* basis = static_cast<const TB*>(a.basis) + pr.base * r;
    TB* rows = reinterpret_cast<TB*>(smem_raw);
    size_t off = ((size_t)nloc * r * sizeof(TB) + 15) / 16 * 16;
    double* nu = reinterpret_cast<double*>(smem_raw + off); off += (size_t)nloc * sizeof(double);
    double* Q = reinterpret_cast<double*>(smem_raw + off); off += (size_t)r * r * sizeof(double);
    double* v = reinterpret_cast<double*>(smem_raw + off); off += (size_t)r * sizeof(double);
    double* sd = reinterpret_cast<double*>(smem_raw + off); off += (size_t)r * sizeof(double);
    double* scr = reinterpret_cast<double*>(smem_raw + off); off += (size_t)2 * r * sizeof(double);
    float* qh = reinterpret_cast<float*>(smem_raw + off); off += (size_t)r * sizeof(float);
    float* ql = reinterpret_cast<float*>(smem_raw + off); off += (size_t)r * sizeof(float);
    unsigned char* msk = smem_raw + off;
    __shared__ double s_frob;
    __shared__ int s_stop, s_p;
    const int tid = threadIdx.x, nt = blockDim.x;
    int32_t* Sout = a.S + (int64_t)pb * r;

    for (int e = tid; e < nloc * r; e += nt) rows[e] = basis[(int64_t)lo * r + e];
    for (int i = tid; i < nloc; i += nt) msk[i] = 0;
    __syncthreads();
    // squared norms of the rows
    double fs = 0.0;
    for (int i = tid; i < nloc; i += nt) {
        double s;
        if (std::is_same<TB, double>::value) {
            DotD d;
            for (int c = 0; c < r; ++c) d.add_sq(to_d(rows[i * r + c]));
            s = d.value();
        } else {
            Dot2 d;
            for (int c = 0; c < r; ++c) d.add_sq(to_f(rows[i * r + c]));
            s = d.value();
        }
        nu[i] = s;
        fs += s;
    }
    fs = block_sum(fs);
    int picked = 0;
    for (int k = 0; k < r; ++k) {
        double bv = -INFINITY;
        long long bi = LLONG_MAX;
        for (int i = tid; i < nloc; i += nt)
            if (!msk[i] && better(nu[i], (long long)(lo + i), bv, bi)) { bv = nu[i]; bi = lo + i; }
        block_argmax(bv, bi);
        const int par = k & 1;
        if (tid == 0) {
            a.keyv[(pr.group0 + part) * 2 + par] = bv;
            a.keyi[(pr.group0 + part) * 2 + par] = bi;
            if (k == 0) a.aux[(pr.group0 + part) * 2] = fs;
        }
        if (!group_barrier(&a.bar[pb], (unsigned)(G * (k + 1)), a.status)) return;
        if (tid == 0) {
            double pv = -INFINITY;
            long long pi = LLONG_MAX;
            for (int g = 0; g < G; ++g) {
                const double kv = a.keyv[(pr.group0 + g) * 2 + par];
                const long long ki = a.keyi[(pr.group0 + g) * 2 + par];
                if (better(kv, ki, pv, pi)) { pv = kv; pi = ki; }
            }
            if (k == 0) {
                double f = 0.0;
                for (int g = 0; g < G; ++g) f += a.aux[(pr.group0 + g) * 2];
                s_frob = f;
            }
            s_stop = (pi == LLONG_MAX) ? 1 : 0;
            s_p = s_stop ? 0 : (int)pi;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        // new direction: v = c_p - Q Q^T c_p, twice (CGS2); its norm is the recomputed
        // residual norm of row p, which decides an early stop before p is recorded
        const TB* cp = basis + (int64_t)p * r;
        for (int c = tid; c < r; c += nt) v[c] = to_d(cp[c]);
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            for (int kk = tid; kk < k; kk += nt) {
                double s = 0.0;
                for (int c = 0; c < r; ++c) s = fma(Q[kk * r + c], v[c], s);
                sd[kk] = s;
            }
            __syncthreads();
            for (int c = tid; c < r; c += nt) {
                double s = 0.0;
                for (int kk = 0; kk < k; ++kk) s = fma(Q[kk * r + c], sd[kk], s);
                scr[r + c] = v[c] - s;
            }
            __syncthreads();
            for (int c = tid; c < r; c += nt) v[c] = scr[r + c];
            __syncthreads();
        }
        if (tid == 0) {
            double s = 0.0;
            for (int c = 0; c < r; ++c) s = fma(v[c], v[c], s);
            const double mx = (double)max(pr.p, r) * kEps;
            s_stop = !(s > mx * mx * s_frob) ? 1 : 0;
            scr[1] = 1.0 / sqrt(s);
        }
        __syncthreads();
        if (s_stop) break;
        if (part == 0 && tid == 0) Sout[k] = p;
        if (p >= lo && p < hi && tid == 0) msk[p - lo] = 1;
        picked = k + 1;
        if (k == r - 1) break;
        for (int c = tid; c < r; c += nt) {
            const double q = v[c] * scr[1];
            Q[k * r + c] = q;
            split_d(q, qh[c], ql[c]);
        }
        __syncthreads();
        // downdate: nu_i -= (c_i . q_k)^2
        for (int i = tid; i < nloc; i += nt) {
            double w;
            if (std::is_same<TB, double>::value) {
                DotD d;
                for (int c = 0; c < r; ++c) d.add(to_d(rows[i * r + c]), Q[k * r + c]);
                w = d.value();
            } else {
                Dot2 d;
                for (int c = 0; c < r; ++c) d.add(to_f(rows[i * r + c]), qh[c], ql[c]);
                w = d.value();
            }
            nu[i] -= w * w;
        }
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

// ---------------------------------------------------------------- FP64 LU and inverse

template <typename TB>
__global__ void __launch_bounds__(256) mv_lu(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pb = blockIdx.x;
    if (a.done[pb]) return;
    const MvProb pr = a.prob[pb];
    const int r = a.r, tid = threadIdx.x, nt = blockDim.x;
    double* M = reinterpret_cast<double*>(smem_raw);  // r x r
    int* perm = reinterpret_cast<int*>(M + r * r);
    double* X = a.minv64 + (int64_t)pb * r * r;       // r x r (inverse, one column per thread)
    __shared__ int s_piv, s_sing;
    __shared__ double s_max;
    const TB* basis = static_cast<const TB*>(a.basis) + pr.base * r;
    const int32_t* S = a.S + (int64_t)pb * r;
    double mx = 0.0;
    int bad = 0;
    for (int e = tid; e < r * r; e += nt) {
        const int k = e / r, c = e - k * r;
        const int s = S[k];
        double x = 0.0;
        if (s < 0 || s >= pr.p) bad = 1; else x = to_d(basis[(int64_t)s * r + c]);
        if (!isfinite(x)) bad = 2;
        M[e] = x;
        mx = fmax(mx, fabs(x));
    }
    for (int k = tid; k < r; k += nt) perm[k] = k;
    bad = __syncthreads_or(bad);
    {
        __shared__ double sm[32];
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) sm[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (nt >> 5); ++w) t = fmax(t, sm[w]);
            s_max = t;
            s_sing = 0;
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
    const double thresh = (double)r * kEps * s_max;
    for (int k = 0; k < r; ++k) {
        if (tid < 32) {
            double bv = -1.0;
            int bi = k;
            for (int i = k + tid; i < r; i += 32) {
                const double x = fabs(M[i * r + k]);
                if (x > bv) { bv = x; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
            }
            if (tid == 0) s_piv = bi;
        }
        __syncthreads();
        const int pv = s_piv;
        if (pv != k) {
            for (int c = tid; c < r; c += nt) {
                const double t = M[k * r + c];
                M[k * r + c] = M[pv * r + c];
                M[pv * r + c] = t;
            }
            if (tid == 0) { const int t = perm[k]; perm[k] = perm[pv]; perm[pv] = t; }
        }
        __syncthreads();
        const double d = M[k * r + k];
        if (!(fabs(d) > thresh)) {
            if (tid == 0) s_sing = 1;
        }
        if (d != 0.0) {
            for (int i = k + 1 + tid; i < r; i += nt) M[i * r + k] /= d;
            __syncthreads();
            const int w = r - k - 1;
            for (int e = tid; e < w * w; e += nt) {
                const int i = k + 1 + e / w, j = k + 1 + e % w;
                M[i * r + j] -= M[i * r + k] * M[k * r + j];
            }
        }
        __syncthreads();
    }
    if (s_sing) {
        if (tid == 0) { a.pstatus[pb] = CUR_ERR_SINGULAR; a.done[pb] = 1; }
        return;
    }
    if (tid == 0) {
        double lv = 0.0;
        for (int k = 0; k < r; ++k) lv += log(fabs(M[k * r + k]));
        a.logvol[pb] = lv;
    }
    // inverse: column c solves L y = P e_c, U x = y
    for (int c = tid; c < r; c += nt) {
        for (int i = 0; i < r; ++i) {
            double s = (perm[i] == c) ? 1.0 : 0.0;
            for (int j = 0; j < i; ++j) s -= M[i * r + j] * X[j * r + c];
            X[i * r + c] = s;
        }
        for (int i = r - 1; i >= 0; --i) {
            double s = X[i * r + c];
            for (int j = i + 1; j < r; ++j) s -= M[i * r + j] * X[j * r + c];
            X[i * r + c] = s / M[i * r + i];
        }
    }
    __syncthreads();
    TB* out = static_cast<TB*>(a.minv) + (int64_t)pb * r * r;
    for (int e = tid; e < r * r; e += nt) out[e] = (TB)X[e];
}

// ---------------------------------------------------------------- coefficients B = C M^-1

template <typename TB>
__global__ void __launch_bounds__(256) mv_coef(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pb = a.tile_prob[blockIdx.x];
    if (a.done[pb]) return;
    const MvProb pr = a.prob[pb];
    const int r = a.r, tid = threadIdx.x, nt = blockDim.x;
    const int row0 = a.tile_row0[blockIdx.x];
    const int nrow = min(64, pr.p - row0);
    TB* Mi = reinterpret_cast<TB*>(smem_raw);  // r x r
    TB* Ct = Mi + r * r;                       // 64 x r
    const TB* src = static_cast<const TB*>(a.minv) + (int64_t)pb * r * r;
    for (int e = tid; e < r * r; e += nt) Mi[e] = src[e];
    const TB* basis = static_cast<const TB*>(a.basis) + (pr.base + row0) * r;
    for (int e = tid; e < nrow * r; e += nt) Ct[e] = basis[e];
    __syncthreads();
    TB* B = static_cast<TB*>(a.B) + (pr.base + row0) * r;
    for (int e = tid; e < nrow * r; e += nt) {
        const int i = e / r, c = e - i * r;
        TB s = (TB)0;
        for (int k = 0; k < r; ++k) s = fma(Ct[i * r + k], Mi[k * r + c], s);
        B[e] = s;
    }
}

// ---------------------------------------------------------------- swap loop

template <typename TB>
__device__ __forceinline__ void scan_slice(const TB* Bs, int nloc, int r, int lo, double& bv,
                                           long long& bi, int& nan) {
    for (int e = threadIdx.x; e < nloc * r; e += blockDim.x) {
        const double x = fabs(to_d(Bs[e]));
        if (!(x <= INFINITY)) nan = 1;
        const int i = e / r, c = e - i * r;
        const long long idx = (long long)(lo + i) * r + c;
        if (better(x, idx, bv, bi)) { bv = x; bi = idx; }
    }
}

template <typename TB>
__global__ void __launch_bounds__(256) mv_swap(MvArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int slot = a.cta_base + blockIdx.x;
    const int pb = a.cta_prob[slot], part = a.cta_part[slot];
    if (a.done[pb]) return;
    const MvProb pr = a.prob[pb];
    const int r = a.r, G = pr.G, tid = threadIdx.x, nt = blockDim.x;
    const int lo = part * pr.rpc, hi = min(pr.p, lo + pr.rpc), nloc = max(0, hi - lo);
    TB* Bs = reinterpret_cast<TB*>(smem_raw);
    TB* colj = Bs + (size_t)nloc * r;
    TB* wrow = colj + nloc;
    __shared__ double s_b;
    __shared__ long long s_w;
    __shared__ int s_state, s_nan;
    TB* pub = static_cast<TB*>(a.pub);
    const TB* Bg = static_cast<const TB*>(a.B) + (pr.base + lo) * r;
    for (int e = tid; e < nloc * r; e += nt) Bs[e] = Bg[e];
    __syncthreads();

    double bv = -INFINITY;
    long long bi = LLONG_MAX;
    int nan = 0;
    scan_slice(Bs, nloc, r, lo, bv, bi, nan);
    nan = __syncthreads_or(nan);
    block_argmax(bv, bi);
    int par = 0;
    const int myslot = pr.group0 + part;
    auto publish = [&](int pp) {
        if (tid == 0) {
            a.keyv[myslot * 2 + pp] = bv;
            a.keyi[myslot * 2 + pp] = nan ? -2LL : bi;
        }
        if (!nan && bi != LLONG_MAX) {
            const int il = (int)(bi / r) - lo;
            for (int c = tid; c < r; c += nt) pub[((int64_t)myslot * 2 + pp) * r + c] = Bs[il * r + c];
        }
    };
    publish(par);

    int made = 0, total = a.swaps[pb];
    double lv_inc = 0.0;
    unsigned epoch = 0;
    int fin = 0;  // 0 running, 1 converged, 2 refresh, 3 error
    int fstat = CUR_OK;
    while (true) {
        ++epoch;
        if (!group_barrier(&a.bar[pb], (unsigned)G * epoch, a.status)) { fin = 3; fstat = CUR_ERR_TIMEOUT; break; }
        if (tid == 0) {
            double wv = -INFINITY;
            long long wi = LLONG_MAX;
            int anynan = 0;
            for (int g = 0; g < G; ++g) {
                const long long ki = a.keyi[(pr.group0 + g) * 2 + par];
                const double kv = a.keyv[(pr.group0 + g) * 2 + par];
                if (ki == -2LL) anynan = 1;
                else if (better(kv, ki, wv, wi)) { wv = kv; wi = ki; }
            }
            s_nan = anynan;
            s_w = wi;
            s_b = wv;
        }
        __syncthreads();
        if (s_nan) { fin = 3; fstat = CUR_ERR_NONFINITE; break; }
        const long long wi = s_w;
        const double wv = s_b;
        if (wi == LLONG_MAX || !(wv > 1.0 + a.delta)) { fin = made == 0 ? 1 : 2; break; }
        if (total >= a.max_swaps) { fin = 3; fstat = CUR_ERR_NOCONV; break; }
        const int istar = (int)(wi / r), jstar = (int)(wi - (long long)istar * r);
        const int owner = istar / pr.rpc;
        const TB* wsrc = pub + ((int64_t)(pr.group0 + owner) * 2 + par) * r;
        for (int c = tid; c < r; c += nt) wrow[c] = wsrc[c];
        for (int i = tid; i < nloc; i += nt) colj[i] = Bs[i * r + jstar];
        __syncthreads();
        const TB b = wrow[jstar];
        if (part == 0 && tid == 0) {
            a.S[(int64_t)pb * r + jstar] = istar;
            lv_inc += log(fabs(to_d(b)));
        }
        __syncthreads();
        if (tid == 0) wrow[jstar] = wrow[jstar] - (TB)1;
        __syncthreads();
        ++made;
        ++total;
        // B <- B - B(:,j) (B(i,:) - e_j^T) / B_ij, fused with the next local argmax
        bv = -INFINITY;
        bi = LLONG_MAX;
        nan = 0;
        for (int e = tid; e < nloc * r; e += nt) {
            const int i = e / r, c = e - i * r;
            const TB f = colj[i] / b;
            const TB x = fma(-f, wrow[c], Bs[e]);
            Bs[e] = x;
            const double ax = fabs(to_d(x));
            if (!(ax <= INFINITY)) nan = 1;
            const long long idx = (long long)(lo + i) * r + c;
            if (better(ax, idx, bv, bi)) { bv = ax; bi = idx; }
        }
        nan = __syncthreads_or(nan);
        block_argmax(bv, bi);
        par ^= 1;
        publish(par);
        if (made == r) { fin = 2; break; }
    }
    if (part == 0 && tid == 0) {
        a.swaps[pb] = total;
        a.logvol[pb] += lv_inc;
        if (fin == 1) { a.done[pb] = 1; a.pstatus[pb] = CUR_OK; }
        else if (fin == 3) {
            a.done[pb] = 1;
            a.pstatus[pb] = fstat;
            if (fstat != CUR_ERR_NOCONV) set_status(a.status, fstat);
        } else {
            atomicAdd(a.pending, 1);
        }
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

template <typename TB>
static size_t swap_smem(int nloc, int r) { return ((size_t)nloc * r + nloc + r) * sizeof(TB) + 64; }

static const size_t kSmemBudget = 200 * 1024;

template <typename TB>
static int rows_cap(int r) {
    int lo = 1, hi = 1 << 20;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (swap_smem<TB>(mid, r) <= kSmemBudget && StartSmem<TB>::bytes(mid, r) <= kSmemBudget) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename K>
static cur_status set_smem_attr(K* fn, size_t bytes) {
    CUR_CK(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return CUR_OK;
}

struct Stage {
    std::vector<MvProb> probs;  // base, gid_base, gid_arr, p filled by the caller
};

// Runs maxvol on every problem of the stage. S (device, P x r local positions) holds
// the start unless aca_start. skip (host, may be empty) marks problems to leave alone.
// Per-problem results stay in the arrays of `out`.
struct StageOut {
    int32_t* S;
    double* logvol;
    int32_t* swaps;
    int32_t* pstatus;
    int32_t* done;
    MvProb* dprob;
    int P;
};

template <typename TB>
static cur_status run_stage(cur_handle* h, const TB* basis, int64_t total_rows, int r,
                            const cur_opts* o, Stage& sg, bool aca_start,
                            const std::vector<int>& skip, int32_t* S, StageOut* so, Arena& ar,
                            cudaStream_t st, bool lu_only = false) {
    const int P = (int)sg.probs.size();
    if (P == 0) return CUR_OK;
    // group sizes
    const int cap = rows_cap<TB>(r);
    int64_t tot_p = 0;
    for (auto& pr : sg.probs) tot_p += pr.p;
    int slots = 0;
    for (auto& pr : sg.probs) {
        int64_t G = (pr.p + cap - 1) / cap;
        const int64_t spread = std::min<int64_t>((pr.p + 63) / 64,
                                                 (int64_t)h->num_sms * pr.p / std::max<int64_t>(1, tot_p));
        G = std::max<int64_t>(G, std::max<int64_t>(1, spread));
        int rpc = (int)((pr.p + G - 1) / G);
        G = (pr.p + rpc - 1) / rpc;
        pr.G = (int)G;
        pr.rpc = rpc;
        pr.group0 = slots;
        slots += (int)G;
    }
    int max_rpc = 1;
    for (auto& pr : sg.probs) max_rpc = std::max(max_rpc, pr.rpc);
    std::vector<int32_t> cta_prob(slots), cta_part(slots);
    for (int pb = 0; pb < P; ++pb)
        for (int g = 0; g < sg.probs[pb].G; ++g) {
            cta_prob[sg.probs[pb].group0 + g] = pb;
            cta_part[sg.probs[pb].group0 + g] = g;
        }
    std::vector<int32_t> tile_prob, tile_row0;
    for (int pb = 0; pb < P; ++pb)
        for (int row0 = 0; row0 < sg.probs[pb].p; row0 += 64) {
            tile_prob.push_back(pb);
            tile_row0.push_back(row0);
        }
    const int ntiles = (int)tile_prob.size();

    MvArgs a{};
    a.basis = basis;
    a.B = ar.get<TB>((size_t)total_rows * r);
    a.minv = ar.get<TB>((size_t)P * r * r);
    a.minv64 = ar.get<double>((size_t)P * r * r);
    MvProb* dprob = ar.get<MvProb>(P);
    int32_t* d_tables = ar.get<int32_t>((size_t)2 * slots + 2 * ntiles);
    a.prob = dprob;
    a.P = P;
    a.r = r;
    a.delta = o->delta;
    a.max_swaps = o->max_swaps > 0 ? o->max_swaps : 100 * r;
    a.cta_prob = d_tables;
    a.cta_part = d_tables + slots;
    a.tile_prob = d_tables + 2 * slots;
    a.tile_row0 = d_tables + 2 * slots + ntiles;
    a.S = S;
    a.logvol = ar.get<double>(P);
    a.swaps = ar.get<int32_t>(P);
    a.pstatus = ar.get<int32_t>(P);
    a.done = ar.get<int32_t>(P);
    a.bar = ar.get<unsigned>(P);
    a.pending = ar.get<int>(1);
    a.keyv = ar.get<double>((size_t)2 * slots);
    a.keyi = ar.get<long long>((size_t)2 * slots);
    a.pub = ar.get<TB>((size_t)2 * slots * r);
    a.aux = ar.get<double>((size_t)2 * slots);
    a.status = h->status;
    if (!ar.ok) return CUR_ERR_NOMEM;

    // upload descriptors and tables through the pinned staging buffer
    const size_t need = sizeof(MvProb) * P + sizeof(int32_t) * (2 * slots + 2 * ntiles) +
                        sizeof(int32_t) * P + 64;
    if (need > h->host_stage_bytes) return CUR_ERR_NOMEM;
    CUR_CK(cudaStreamSynchronize(st));  // the staging buffer may still feed an earlier copy
    char* hs = h->host_stage;
    std::memcpy(hs, sg.probs.data(), sizeof(MvProb) * P);
    int32_t* ht = reinterpret_cast<int32_t*>(hs + sizeof(MvProb) * P);
    std::memcpy(ht, cta_prob.data(), sizeof(int32_t) * slots);
    std::memcpy(ht + slots, cta_part.data(), sizeof(int32_t) * slots);
    std::memcpy(ht + 2 * slots, tile_prob.data(), sizeof(int32_t) * ntiles);
    std::memcpy(ht + 2 * slots + ntiles, tile_row0.data(), sizeof(int32_t) * ntiles);
    int32_t* hdone = ht + 2 * slots + 2 * ntiles;
    for (int pb = 0; pb < P; ++pb) hdone[pb] = (!skip.empty() && skip[pb]) ? 1 : 0;
    CUR_CK(cudaMemcpyAsync(dprob, hs, sizeof(MvProb) * P, cudaMemcpyHostToDevice, st));
    CUR_CK(cudaMemcpyAsync(d_tables, ht, sizeof(int32_t) * (2 * slots + 2 * ntiles),
                           cudaMemcpyHostToDevice, st));
    CUR_CK(cudaMemcpyAsync(a.done, hdone, sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
    CUR_CK(cudaMemsetAsync(a.swaps, 0, sizeof(int32_t) * P, st));
    CUR_CK(cudaMemsetAsync(a.pstatus, 0, sizeof(int32_t) * P, st));
    CUR_CK(cudaMemsetAsync(a.logvol, 0, sizeof(double) * P, st));

    // kernel attributes and co-residency per launch wave
    const size_t sm_swap = swap_smem<TB>(max_rpc, r);
    const size_t sm_start = StartSmem<TB>::bytes(max_rpc, r);
    const size_t sm_lu = (size_t)r * r * sizeof(double) + (size_t)r * sizeof(int) + 64;
    const size_t sm_coef = ((size_t)r * r + 64 * (size_t)r) * sizeof(TB) + 64;
    CUR_TRY(set_smem_attr(mv_swap<TB>, sm_swap));
    CUR_TRY(set_smem_attr(mv_start<TB>, sm_start));
    CUR_TRY(set_smem_attr(mv_lu<TB>, sm_lu));
    CUR_TRY(set_smem_attr(mv_coef<TB>, sm_coef));
    int occ_swap = 0, occ_start = 0;
    CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_swap, mv_swap<TB>, 256, sm_swap));
    CUR_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_start, mv_start<TB>, 256, sm_start));
    const int cap_swap = std::max(1, occ_swap) * h->num_sms;
    const int cap_start = std::max(1, occ_start) * h->num_sms;
    // waves: consecutive whole groups within the capacity
    auto waves = [&](int capc) {
        std::vector<std::pair<int, int>> w;  // (first slot, count)
        int first = 0, cnt = 0;
        for (int pb = 0; pb < P; ++pb) {
            const int G = sg.probs[pb].G;
            if (cnt + G > capc && cnt > 0) { w.push_back({first, cnt}); first += cnt; cnt = 0; }
            cnt += G;
        }
        if (cnt > 0) w.push_back({first, cnt});
        return w;
    };
    for (auto& pr : sg.probs)
        if (pr.G > cap_swap || pr.G > cap_start) return CUR_ERR_ARG;

    if (aca_start) {
        CUR_CK(cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * P, st));
        for (auto& w : waves(cap_start)) {
            MvArgs aw = a;
            aw.cta_base = w.first;
            void* args[] = {&aw};
            CUR_TRY(launch_coop((const void*)mv_start<TB>, dim3(w.second), dim3(256), args, sm_start, st));
            note_launch();
        }
    }
    const int max_cycles = a.max_swaps / r + 4;
    int* hpend = reinterpret_cast<int*>(hs + need - 32);
    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        mv_lu<TB><<<P, 256, sm_lu, st>>>(a);
        CUR_CK(cudaGetLastError());
    note_launch();
        if (lu_only) break;
        mv_coef<TB><<<ntiles, 256, sm_coef, st>>>(a);
        CUR_CK(cudaGetLastError());
    note_launch();
        CUR_CK(cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * P, st));
        CUR_CK(cudaMemsetAsync(a.pending, 0, sizeof(int), st));
        for (auto& w : waves(cap_swap)) {
            MvArgs aw = a;
            aw.cta_base = w.first;
            void* args[] = {&aw};
            CUR_TRY(launch_coop((const void*)mv_swap<TB>, dim3(w.second), dim3(256), args, sm_swap, st));
            note_launch();
        }
        CUR_CK(cudaMemcpyAsync(hpend, a.pending, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUR_CK(cudaStreamSynchronize(st));
        if (*hpend == 0) break;
    }
    so->S = S;
    so->logvol = a.logvol;
    so->swaps = a.swaps;
    so->pstatus = a.pstatus;
    so->done = a.done;
    so->dprob = dprob;
    so->P = P;
    return CUR_OK;
}

// Reads per-problem statuses and swap counts to the host (stream synchronised).
static cur_status read_stage(cur_handle* h, const StageOut& so, std::vector<int>& stat,
                             std::vector<int>& sw, cudaStream_t st) {
    const int P = so.P;
    if ((size_t)P * 8 + 64 > h->host_stage_bytes) return CUR_ERR_NOMEM;
    int32_t* hs = reinterpret_cast<int32_t*>(h->host_stage);
    CUR_CK(cudaMemcpyAsync(hs, so.pstatus, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, st));
    CUR_CK(cudaMemcpyAsync(hs + P, so.swaps, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, st));
    CUR_CK(cudaStreamSynchronize(st));
    stat.assign(hs, hs + P);
    sw.assign(hs + P, hs + 2 * P);
    return CUR_OK;
}

static inline unsigned nblk(int64_t n, int t = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535));
}

template <typename TB>
static cur_status merge_level_t(cur_handle* h, const TB* basis, int64_t p, int r,
                                const int32_t* cand, int nsets, const cur_opts* o, int32_t* out,
                                int* swaps, Arena& ar, cudaStream_t st) {
    const int npairs = nsets / 2;
    *swaps = 0;
    if (npairs == 0) {
        CUR_CK(cudaMemcpyAsync(out, cand, sizeof(int32_t) * r * nsets, cudaMemcpyDeviceToDevice, st));
        return CUR_OK;
    }
    const size_t mark = ar.off;
    const int64_t nrows = (int64_t)npairs * 2 * r;
    TB* U = ar.get<TB>((size_t)nrows * r);
    int32_t* S = ar.get<int32_t>((size_t)npairs * r);
    int32_t* S2 = ar.get<int32_t>((size_t)npairs * r);
    if (!ar.ok) return CUR_ERR_NOMEM;
    // the union of pair t is cand rows 2t, 2t+1: contiguous in cand
    gather_union_k<TB><<<nblk(nrows * r), 256, 0, st>>>(basis, p, r, cand, nrows, U, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    Stage sg;
    for (int t = 0; t < npairs; ++t) {
        MvProb pr{};
        pr.base = (int64_t)t * 2 * r;
        pr.gid_arr = cand + (int64_t)t * 2 * r;
        pr.gid_base = 0;
        pr.p = 2 * r;
        sg.probs.push_back(pr);
    }
    mv_iota<<<nblk(npairs * r), 256, 0, st>>>(S, npairs, r, 0);
    CUR_CK(cudaGetLastError());
    note_launch();
    StageOut so{};
    std::vector<int> none;
    CUR_TRY(run_stage<TB>(h, U, nrows, r, o, sg, false, none, S, &so, ar, st));
    std::vector<int> stat, sw;
    CUR_TRY(read_stage(h, so, stat, sw, st));
    for (int v : sw) *swaps += v;
    // singular left start: start at the right child; then Algorithm 3 on the union
    std::vector<int> skip(npairs, 1);
    bool any = false;
    for (int t = 0; t < npairs; ++t)
        if (stat[t] == CUR_ERR_SINGULAR) { skip[t] = 0; any = true; }
    if (any) {
        mv_iota<<<nblk(npairs * r), 256, 0, st>>>(S2, npairs, r, r);
        CUR_CK(cudaGetLastError());
    note_launch();
        Stage sg2 = sg;
        StageOut so2{};
        CUR_TRY(run_stage<TB>(h, U, nrows, r, o, sg2, false, skip, S2, &so2, ar, st));
        std::vector<int> stat2, sw2;
        CUR_TRY(read_stage(h, so2, stat2, sw2, st));
        std::vector<int> skip3(npairs, 1);
        bool any3 = false;
        for (int t = 0; t < npairs; ++t) {
            if (skip[t]) continue;
            *swaps += sw2[t];
            if (stat2[t] == CUR_ERR_SINGULAR) { skip3[t] = 0; any3 = true; }
            CUR_CK(cudaMemcpyAsync(S + (int64_t)t * r, S2 + (int64_t)t * r, sizeof(int32_t) * r,
                                   cudaMemcpyDeviceToDevice, st));
        }
        if (any3) {
            Stage sg3 = sg;
            StageOut so3{};
            CUR_TRY(run_stage<TB>(h, U, nrows, r, o, sg3, true, skip3, S2, &so3, ar, st));
            std::vector<int> stat3, sw3;
            CUR_TRY(read_stage(h, so3, stat3, sw3, st));
            for (int t = 0; t < npairs; ++t) {
                if (skip3[t]) continue;
                *swaps += sw3[t];
                CUR_CK(cudaMemcpyAsync(S + (int64_t)t * r, S2 + (int64_t)t * r, sizeof(int32_t) * r,
                                       cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    mv_emit<<<nblk(npairs * r), 256, 0, st>>>(so.dprob, S, npairs, r, out);
    CUR_CK(cudaGetLastError());
    note_launch();
    if (nsets % 2 == 1)
        CUR_CK(cudaMemcpyAsync(out + (int64_t)npairs * r, cand + (int64_t)(nsets - 1) * r,
                               sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

template <typename TB>
static cur_status global_t(cur_handle* h, const TB* basis, int64_t p, int r, const cur_opts* o,
                           const int32_t* S0, int32_t* S_out, double* logvol_out, MvResult* res,
                           Arena& ar, cudaStream_t st, bool lu_only = false) {
    const size_t mark = ar.off;
    int32_t* S = ar.get<int32_t>(r);
    if (!ar.ok) return CUR_ERR_NOMEM;
    Stage sg;
    MvProb pr{};
    pr.base = 0;
    pr.gid_base = 0;
    pr.gid_arr = nullptr;
    pr.p = (int32_t)p;
    sg.probs.push_back(pr);
    CUR_CK(cudaMemcpyAsync(S, S0, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    StageOut so{};
    std::vector<int> none;
    CUR_TRY(run_stage<TB>(h, basis, p, r, o, sg, false, none, S, &so, ar, st, lu_only));
    std::vector<int> stat, sw;
    CUR_TRY(read_stage(h, so, stat, sw, st));
    if (res) { res->swaps = sw[0]; res->status = stat[0]; }
    if (stat[0] != CUR_ERR_SINGULAR && stat[0] != CUR_ERR_ARG)
        CUR_CK(cudaMemcpyAsync(S_out, S, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    else if (S_out != S0)
        CUR_CK(cudaMemcpyAsync(S_out, S0, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    if (logvol_out) CUR_CK(cudaMemcpyAsync(logvol_out, so.logvol, sizeof(double), cudaMemcpyDeviceToDevice, st));
    CUR_CK(cudaStreamSynchronize(st));
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

template <typename TB>
static cur_status rows_t(cur_handle* h, const TB* basis, int64_t p, int r, const cur_opts* o,
                         int32_t* I_out, double* logvol_out, int32_t* swaps_out, MvResult* res,
                         Arena& ar, cudaStream_t st) {
    const int nb = std::max(1, o->nblocks);
    const int64_t base_sz = p / nb, extra = p % nb;
    if (base_sz < r) return CUR_ERR_ARG;
    const size_t mark = ar.off;
    int32_t* S = ar.get<int32_t>((size_t)nb * r);
    int32_t* setsA = ar.get<int32_t>((size_t)nb * r);
    int32_t* setsB = ar.get<int32_t>((size_t)nb * r);
    if (!ar.ok) return CUR_ERR_NOMEM;
    Stage sg;
    int64_t s0 = 0;
    for (int k = 0; k < nb; ++k) {
        const int64_t sz = base_sz + (k < extra ? 1 : 0);
        MvProb pr{};
        pr.base = s0;
        pr.gid_base = s0;
        pr.gid_arr = nullptr;
        pr.p = (int32_t)sz;
        sg.probs.push_back(pr);
        s0 += sz;
    }
    StageOut so{};
    std::vector<int> none;
    CUR_TRY(run_stage<TB>(h, basis, p, r, o, sg, true, none, S, &so, ar, st));
    std::vector<int> stat, sw;
    CUR_TRY(read_stage(h, so, stat, sw, st));
    int total = 0;
    for (int v : sw) total += v;
    mv_emit<<<nblk(nb * r), 256, 0, st>>>(so.dprob, S, nb, r, setsA);
    CUR_CK(cudaGetLastError());
    note_launch();
    int nsets = nb;
    int32_t* cur = setsA;
    int32_t* nxt = setsB;
    while (nsets > 1) {
        int msw = 0;
        CUR_TRY(merge_level_t<TB>(h, basis, p, r, cur, nsets, o, nxt, &msw, ar, st));
        total += msw;
        nsets = (nsets + 1) / 2;
        std::swap(cur, nxt);
    }
    int fstat = CUR_OK;
    if (o->flags & CUR_FLAG_POLISH) {
        MvResult gr;
        CUR_TRY(global_t<TB>(h, basis, p, r, o, cur, I_out, logvol_out, &gr, ar, st));
        total += gr.swaps;
        fstat = gr.status;
    } else {
        CUR_CK(cudaMemcpyAsync(I_out, cur, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
        if (logvol_out) {
            // log|det| of the merged set through one LU
            MvResult gr;
            int32_t* tmp = ar.get<int32_t>(r);
            if (!ar.ok) return CUR_ERR_NOMEM;
            CUR_TRY(global_t<TB>(h, basis, p, r, o, cur, tmp, logvol_out, &gr, ar, st, true));
        }
    }
    if (swaps_out) {
        int32_t* hs = reinterpret_cast<int32_t*>(h->host_stage);
        CUR_CK(cudaStreamSynchronize(st));
        hs[0] = total;
        CUR_CK(cudaMemcpyAsync(swaps_out, hs, sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CUR_CK(cudaStreamSynchronize(st));
    }
    if (res) { res->swaps = total; res->status = fstat; }
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

}  // namespace curk

size_t compute_size(cur_dtype t) { return t == CUR_F64 ? 8 : 4; }

cur_status maxvol_basis_rows(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                             const cur_opts* o, int32_t* I_out, double* logvol_out,
                             int32_t* swaps_out, MvResult* res, Arena& ar, cudaStream_t st) {
    if (dt == CUR_F64)
        return curk::rows_t<double>(h, static_cast<const double*>(basis), p, r, o, I_out, logvol_out, swaps_out, res, ar, st);
    return curk::rows_t<float>(h, static_cast<const float*>(basis), p, r, o, I_out, logvol_out, swaps_out, res, ar, st);
}

cur_status maxvol_global(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                         const cur_opts* o, const int32_t* S0, int32_t* S_out,
                         double* logvol_out, MvResult* res, Arena& ar, cudaStream_t st) {
    if (dt == CUR_F64)
        return curk::global_t<double>(h, static_cast<const double*>(basis), p, r, o, S0, S_out, logvol_out, res, ar, st);
    return curk::global_t<float>(h, static_cast<const float*>(basis), p, r, o, S0, S_out, logvol_out, res, ar, st);
}

cur_status merge_level(cur_handle* h, cur_dtype dt, const void* basis, int64_t p, int r,
                       const int32_t* cand, int nsets, const cur_opts* o, int32_t* out,
                       int* swaps, Arena& ar, cudaStream_t st) {
    if (dt == CUR_F64)
        return curk::merge_level_t<double>(h, static_cast<const double*>(basis), p, r, cand, nsets, o, out, swaps, ar, st);
    return curk::merge_level_t<float>(h, static_cast<const float*>(basis), p, r, cand, nsets, o, out, swaps, ar, st);
}

template <typename TA>
static cur_status gather_cols_t(const cur_mat* A, const int32_t* J, int r, void* C, cudaStream_t st) {
    const TA* a = static_cast<const TA*>(A->data);
    const int64_t total = A->rows * r;
    if (A->dtype == CUR_F64)
        curk::gather_cols_k<TA, double><<<curk::nblk(total), 256, 0, st>>>(a, A->rows, A->cols, A->ld, J, r, static_cast<double*>(C), nullptr);
    else
        curk::gather_cols_k<TA, float><<<curk::nblk(total), 256, 0, st>>>(a, A->rows, A->cols, A->ld, J, r, static_cast<float*>(C), nullptr);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status gather_cols_compute(const cur_mat* A, const int32_t* J, int r, void* C, cudaStream_t st) {
    switch (A->dtype) {
        case CUR_F64: return gather_cols_t<double>(A, J, r, C, st);
        case CUR_F32: return gather_cols_t<float>(A, J, r, C, st);
        case CUR_BF16: return gather_cols_t<__nv_bfloat16>(A, J, r, C, st);
    }
    return CUR_ERR_ARG;
}

template <typename TA>
static cur_status gather_rows_t_t(const cur_mat* A, const int32_t* I, int r, void* Rt, cudaStream_t st) {
    const TA* a = static_cast<const TA*>(A->data);
    const unsigned grid = (unsigned)((A->cols + 31) / 32);
    if (A->dtype == CUR_F64) {
        const size_t sm = (size_t)r * 33 * sizeof(double);
        CUR_CK(cudaFuncSetAttribute((const void*)curk::gather_rows_t_k<TA, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        curk::gather_rows_t_k<TA, double><<<grid, 256, sm, st>>>(a, A->rows, A->cols, A->ld, I, r, static_cast<double*>(Rt), nullptr);
    } else {
        const size_t sm = (size_t)r * 33 * sizeof(float);
        CUR_CK(cudaFuncSetAttribute((const void*)curk::gather_rows_t_k<TA, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        curk::gather_rows_t_k<TA, float><<<grid, 256, sm, st>>>(a, A->rows, A->cols, A->ld, I, r, static_cast<float*>(Rt), nullptr);
    }
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status gather_rows_t_compute(const cur_mat* A, const int32_t* I, int r, void* Rt, cudaStream_t st) {
    switch (A->dtype) {
        case CUR_F64: return gather_rows_t_t<double>(A, I, r, Rt, st);
        case CUR_F32: return gather_rows_t_t<float>(A, I, r, Rt, st);
        case CUR_BF16: return gather_rows_t_t<__nv_bfloat16>(A, I, r, Rt, st);
    }
    return CUR_ERR_ARG;
}

cur_status pad_indices_dev(int32_t* idx, const int32_t* count, int r, int64_t size, cudaStream_t st) {
    curk::pad_indices_k<<<1, 32, 0, st>>>(idx, count, r, size);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}
