// The cross over row slabs of A, one process per GPU (the sharded form).
//
// Rank k of P holds a contiguous slab A_k of the rows of A. Algorithm 3 (Section 2.2)
// needs, per round, a global reduction and the pivot vector: on row slabs the column
// statistics are sums over the ranks, so a round is
//   pick   : red = sum over ranks of the slab partials (the caller's allreduce);
//            W(t-1,:) = red, nu -= red^2 (t = 0: nu = red, the squared norms), masked
//            argmax (lowest index) -> p; v_k = A_k(:,p) - Q_k^T W(:t,p);
//            red2 = (Q_k v_k, ||v_k||^2)
//   commit : c = sum of red2[0..t); rank-stop test on ||v - Q^T c||^2 = sum of red2[t] -
//            ||c||^2 (Q orthonormal); q_t = (v_k - Q_k^T c) / ||v|| (CGS2, second pass);
//            red = A_k^T q_t (the next round's pass: the HBM stream, Dot2 accuracy as on
//            one GPU)
// with two allreduces per round (n and r doubles) made by the caller between calls.
//
// Maxvol over all rows of a basis distributed by row slabs (the polish and the sweeps):
// every rank keeps the r x r matrix M = C(S,:) and its FP64 inverse (identical on every
// rank) and the slab of B = C_k M^-1. Per swap the ranks agree on argmax |B_ij| by two
// allreduces (MAX of the value, then MIN of the flat index (global row * r + j) among
// the ranks that hold that value), and the owner's row of C reaches every rank through an
// allreduce-sum of a vector that only the owner fills. Each cycle of r swaps starts from a
// fresh FP64 factorisation of M, as the oracle's iteration does.
//
// Everything here enqueues on the caller's stream and returns; per-call state lives in
// caller-owned device buffers (cur_shard_aca_state_bytes, cur_dmv_state_bytes).

#include <algorithm>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

cur_status pad_indices_dev(int32_t* idx, const int32_t* count, int r, int64_t size, cudaStream_t st);

namespace curk {

constexpr int kShardG = 152;   // CTAs of the slab kernels (one wave on 152 SMs)

static inline unsigned nbs(int64_t n, int t = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535));
}
static inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// ---------------------------------------------------------------- Algorithm 3 state

struct AcaHdr {
    int stop, count, p, pad;
    double frob2;
    int64_t m_global;
};

struct AcaLayout {
    int64_t m, n;
    int r, RC;
    int64_t chunk;
    size_t hdr, nu, mask, W, Q, q64, qh, ql, v, part, cta, total;
};

static AcaLayout aca_layout(const cur_handle* h, const cur_mat* A, int r) {
    AcaLayout L{};
    L.m = A->rows;
    L.n = A->cols;
    L.r = r;
    L.RC = aca_cols_chunks(h->num_sms, L.m, L.n, A->dtype, &L.chunk);
    size_t o = 0;
    L.hdr = o; o += al256(sizeof(AcaHdr));
    L.nu = o; o += al256(8 * (size_t)L.n);
    L.mask = o; o += al256((size_t)L.n);
    L.W = o; o += al256(8 * (size_t)r * L.n);
    L.Q = o; o += al256(8 * (size_t)r * L.m);
    L.q64 = o; o += al256(8 * (size_t)L.m);
    L.qh = o; o += al256(4 * (size_t)L.m);
    L.ql = o; o += al256(4 * (size_t)L.m);
    L.v = o; o += al256(8 * (size_t)L.m);
    L.part = o; o += al256(8 * (size_t)L.RC * L.n);
    L.cta = o; o += al256(8 * (size_t)kShardG * (r + 1));
    L.total = o;
    return L;
}

template <typename T> __device__ __forceinline__ double part_d(T x);
template <> __device__ __forceinline__ double part_d<double>(double x) { return x; }
template <> __device__ __forceinline__ double part_d<df64>(df64 x) { return (double)x.h + (double)x.l; }

// red[j] = sum over the RC row chunks of part[rc][j], in chunk order.
template <typename PT>
__global__ void sa_reduce_k(const PT* __restrict__ part, int RC, int64_t n, double* __restrict__ red,
                            const int* stop) {
    if (*stop) return;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int rc = 0; rc < RC; ++rc) s += part_d(part[(int64_t)rc * n + j]);
        red[j] = s;
    }
}

// The global pick of round t (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) sa_pick_k(const double* __restrict__ red, int64_t n, int t,
                                                  double* nu, double* W, unsigned char* mask, AcaHdr* hdr,
                                                  int* status) {
    if (hdr->stop) return;
    double bv = -INFINITY;
    long long bi = LLONG_MAX;
    double fs = 0.0;
    int bad = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double x = red[j];
        double v;
        if (t == 0) {
            v = x;
            fs += x;
            if (!isfinite(x)) bad = 1;
        } else {
            W[(int64_t)(t - 1) * n + j] = x;
            v = nu[j] - x * x;
        }
        nu[j] = v;
        if (!mask[j] && better(v, (long long)j, bv, bi)) { bv = v; bi = j; }
    }
    block_argmax(bv, bi);
    bad = __syncthreads_or(bad);
    if (t == 0) fs = block_sum(fs);
    if (threadIdx.x != 0) return;
    if (t == 0) hdr->frob2 = fs;
    if (bad) { hdr->stop = 1; set_status(status, CUR_ERR_NONFINITE); return; }
    if (bi == LLONG_MAX) { hdr->stop = 1; set_status(status, CUR_WARN_RANK); return; }
    hdr->p = (int)bi;
}

// v = A_k(:,p) - Q^T W(:t,p) over the slab's rows; per-CTA partials of Q v (t values) and
// of ||v||^2 (at index t).
template <typename TA>
__global__ void __launch_bounds__(256) sa_vec_k(const TA* __restrict__ A, int64_t m, int64_t n, int64_t ld,
                                                int t, int r, const double* __restrict__ Q,
                                                const double* __restrict__ W, double* __restrict__ v,
                                                double* __restrict__ cta, const AcaHdr* hdr) {
    __shared__ double s_w[128];
    if (hdr->stop) return;
    const int g = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
    const int64_t p = hdr->p;
    for (int k = tid; k < t; k += blockDim.x) s_w[k] = W[(int64_t)k * n + p];
    __syncthreads();
    const int64_t i0 = m * g / G, i1 = m * (g + 1) / G;
    double nv = 0.0;
    for (int64_t i = i0 + tid; i < i1; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < t; ++k) s = fma(Q[(int64_t)k * m + i], s_w[k], s);
        const double vi = to_d(A[i * ld + p]) - s;
        v[i] = vi;
        nv = fma(vi, vi, nv);
    }
    nv = block_sum(nv);
    if (tid == 0) cta[(int64_t)g * r + t] = nv;
    const int warp = tid >> 5, lane = tid & 31;
    for (int k = warp; k < t; k += blockDim.x >> 5) {
        double acc = 0.0;
        for (int64_t i = i0 + lane; i < i1; i += 32) acc = fma(Q[(int64_t)k * m + i], v[i], acc);
        acc = warp_sum(acc);
        if (lane == 0) cta[(int64_t)g * r + k] = acc;
    }
}

// out[k] = sum over CTAs g of cta[g * stride + k] (CTA order) for k < cnt; 0 for cnt <= k < len.
__global__ void sa_sum_k(const double* __restrict__ cta, int G, int stride, int cnt, int len,
                         double* __restrict__ out, const AcaHdr* hdr) {
    if (hdr && hdr->stop) return;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        double s = 0.0;
        if (k < cnt)
            for (int g = 0; g < G; ++g) s += cta[(int64_t)g * stride + k];
        out[k] = s;
    }
}

// The round's end from red2 (summed over the ranks: Q^T v at [0, t), ||v||^2 at t): the
// rank-stop test on ||v - Q c||^2 = ||v||^2 - ||c||^2 (c = Q^T v, Q orthonormal), then the
// pick, the second Gram-Schmidt pass v -= Q^T c and q_t = v / ||v|| in one sweep.
__global__ void __launch_bounds__(256) sa_commit_k(int64_t m, int64_t n, int t, const double* __restrict__ red2,
                                                   const double* __restrict__ v, double* __restrict__ Q,
                                                   double* __restrict__ q64, float* __restrict__ qh,
                                                   float* __restrict__ ql, unsigned char* mask, int32_t* idx_out,
                                                   AcaHdr* hdr, int* status) {
    __shared__ double s_c[128];
    __shared__ double s_s;
    if (hdr->stop) return;
    const int g = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
    for (int k = tid; k < t; k += blockDim.x) s_c[k] = red2[k];
    if (tid < 32) {
        double cc = 0.0;
        for (int k = tid; k < t; k += 32) cc = fma(red2[k], red2[k], cc);
        cc = warp_sum(cc);
        if (tid == 0) s_s = red2[t] - cc;
    }
    __syncthreads();
    const double s = s_s;
    const double mx = (double)max(hdr->m_global, n) * 2.220446049250313e-16;
    if (!(s > mx * mx * hdr->frob2)) {
        __syncthreads();
        if (g == 0 && tid == 0) { hdr->stop = 1; set_status(status, CUR_WARN_RANK); }
        return;
    }
    const int p = hdr->p;
    __syncthreads();
    if (g == 0 && tid == 0) {
        idx_out[t] = p;
        mask[p] = 1;
        hdr->count = t + 1;
    }
    const double inv = 1.0 / sqrt(s);
    const int64_t i0 = m * g / G, i1 = m * (g + 1) / G;
    for (int64_t i = i0 + tid; i < i1; i += blockDim.x) {
        double sq = 0.0;
        for (int k = 0; k < t; ++k) sq = fma(Q[(int64_t)k * m + i], s_c[k], sq);
        const double q = (v[i] - sq) * inv;
        Q[(int64_t)t * m + i] = q;
        q64[i] = q;
        float hi, lo;
        split_d(q, hi, lo);
        qh[i] = hi;
        ql[i] = lo;
    }
}

// ---------------------------------------------------------------- distributed maxvol state

struct DmvHdr {
    int swaps, status, singular, pad;
    double logvol;
    double keyv;
    long long keyi;
};

struct DmvLayout {
    int64_t p;
    int r;
    size_t hdr, M, Minv, S, b, colj, B, ckv, cki, total;
};

static DmvLayout dmv_layout(int64_t p, int r, cur_dtype dt) {
    DmvLayout L{};
    L.p = p;
    L.r = r;
    size_t o = 0;
    L.hdr = o; o += al256(sizeof(DmvHdr));
    L.M = o; o += al256(8 * (size_t)r * r);
    L.Minv = o; o += al256(8 * (size_t)r * r);
    L.S = o; o += al256(4 * (size_t)r);
    L.b = o; o += al256(8 * (size_t)r);
    L.colj = o; o += al256(8 * (size_t)r);
    L.B = o; o += al256(compute_size(dt) * (size_t)p * r);
    L.ckv = o; o += al256(8 * (size_t)kShardG);
    L.cki = o; o += al256(8 * (size_t)kShardG);
    L.total = o;
    return L;
}

template <typename TB>
__global__ void dmv_load_k(const int32_t* __restrict__ S, const TB* __restrict__ Mrows, int r,
                           int32_t* __restrict__ Sd, double* __restrict__ Md, DmvHdr* hdr) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) Md[e] = to_d(Mrows[e]);
    for (int e = threadIdx.x; e < r; e += blockDim.x) Sd[e] = S[e];
    if (threadIdx.x == 0) { hdr->swaps = 0; hdr->status = CUR_OK; hdr->singular = 0; }
}

// Fresh factorisation of M (one CTA): Minv, log|det|; a pivot with |u_kk| <= r eps max|M|
// marks the set numerically singular (the oracle's LU test).
__global__ void __launch_bounds__(256) dmv_factor_k(const double* __restrict__ M, int r,
                                                    double* __restrict__ Minv, DmvHdr* hdr) {
    extern __shared__ double sm[];
    double* A = sm;
    double* colk = A + r * r;
    int* piv = reinterpret_cast<int*>(colk + r);
    __shared__ double s_mx;
    double mx = 0.0;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        A[e] = M[e];
        mx = fmax(mx, fabs(M[e]));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) s_mx = mx;
    __syncthreads();
    double lad = 0.0;
    const int sing = gj_inverse(A, r, colk, piv, (double)r * 2.220446049250313e-16 * s_mx, &lad);
    __syncthreads();
    if (sing) {
        if (threadIdx.x == 0) { hdr->singular = 1; hdr->status = CUR_ERR_SINGULAR; hdr->logvol = -INFINITY; }
        return;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) Minv[e] = A[e];
    if (threadIdx.x == 0) { hdr->singular = 0; hdr->logvol = lad; }
}

// B = C_k Minv (FP64 products, stored in the compute type) and each CTA's argmax |B_ij|
// (key = global row * r + j; the smaller key wins a tie).
template <typename TB>
__global__ void __launch_bounds__(256) dmv_coef_k(const TB* __restrict__ C, int64_t p, int64_t off, int r,
                                                  const double* __restrict__ Minv, TB* __restrict__ B,
                                                  double* ckv, long long* cki, const DmvHdr* hdr) {
    extern __shared__ double sMi[];
    double bv = -1.0;
    long long bi = LLONG_MAX;
    if (hdr->singular) {
        if (threadIdx.x == 0) { ckv[blockIdx.x] = -1.0; cki[blockIdx.x] = LLONG_MAX; }
        return;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sMi[e] = Minv[e];
    __syncthreads();
    const int64_t tot = p * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int c = (int)(e - i * r);
        const TB* ci = C + i * r;
        double s = 0.0;
        for (int k = 0; k < r; ++k) s = fma(to_d(ci[k]), sMi[k * r + c], s);
        const TB b = (TB)s;
        B[e] = b;
        const double a = fabs(to_d(b));
        const long long key = (off + i) * r + c;
        if (better(a, key, bv, bi)) { bv = a; bi = key; }
    }
    block_argmax(bv, bi);
    if (threadIdx.x == 0) { ckv[blockIdx.x] = bv; cki[blockIdx.x] = bi; }
}

__global__ void dmv_key_k(const double* ckv, const long long* cki, int G, DmvHdr* hdr, double* keyv_out) {
    double bv = -1.0;
    long long bi = LLONG_MAX;
    for (int g = threadIdx.x; g < G; g += blockDim.x)
        if (better(ckv[g], cki[g], bv, bi)) { bv = ckv[g]; bi = cki[g]; }
    block_argmax(bv, bi);
    if (threadIdx.x != 0) return;
    if (hdr->singular) { bv = -1.0; bi = LLONG_MAX; }
    hdr->keyv = bv;
    hdr->keyi = bi;
    *keyv_out = bv;
}

__global__ void dmv_holder_k(const DmvHdr* hdr, const double* keyv_glob, long long* keyi_out) {
    if (threadIdx.x == 0) *keyi_out = (hdr->keyv == *keyv_glob) ? hdr->keyi : LLONG_MAX;
}

template <typename TB>
__global__ void dmv_fill_k(const TB* __restrict__ C, int64_t p, int64_t off, int r, const long long* keyi,
                           TB* __restrict__ row) {
    const long long k = *keyi;
    const long long i = k == LLONG_MAX ? -1 : k / r;
    const bool own = i >= off && i < off + p;
    for (int c = threadIdx.x; c < r; c += blockDim.x) row[c] = own ? C[(i - off) * r + c] : (TB)0;
}

// The swap of global row i = keyi / r into position j = keyi % r (one CTA): b = c Minv in
// FP64 from the owner's row c, Minv -= Minv(:,j) (b - e_j)^T / b_j, M(j,:) = c, S[j] = i.
template <typename TB>
__global__ void __launch_bounds__(256) dmv_row_k(const TB* __restrict__ row, const long long* keyi, int r,
                                                 double* __restrict__ M, double* __restrict__ Minv,
                                                 int32_t* __restrict__ S, double* __restrict__ b,
                                                 double* __restrict__ colj, DmvHdr* hdr) {
    __shared__ double s_c[128], s_b[128], s_cj[128];
    const long long key = *keyi;
    const int j = (int)(key % r);
    const long long i = key / r;
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        s_c[k] = to_d(row[k]);
        s_cj[k] = Minv[k * r + j];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < r; ++k) s = fma(s_c[k], Minv[k * r + c], s);
        s_b[c] = s;
    }
    __syncthreads();
    const double bj = s_b[j];
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int a = e / r, c = e - a * r;
        const double w = (s_b[c] - (c == j ? 1.0 : 0.0)) / bj;
        Minv[e] -= s_cj[a] * w;
    }
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
        M[j * r + c] = s_c[c];
        b[c] = s_b[c];
        colj[c] = s_cj[c];
    }
    if (threadIdx.x == 0) {
        S[j] = (int32_t)i;
        hdr->logvol += log(fabs(bj));
        hdr->swaps += 1;
    }
}

// B -= B(:,j) (b - e_j)^T / b_j over the slab, and each CTA's new argmax.
template <typename TB>
__global__ void __launch_bounds__(256) dmv_update_k(TB* __restrict__ B, int64_t p, int64_t off, int r,
                                                    const long long* keyi, const double* __restrict__ b,
                                                    double* ckv, long long* cki) {
    __shared__ double s_w[128];
    const int j = (int)(*keyi % r);
    const double bj = b[j];
    for (int c = threadIdx.x; c < r; c += blockDim.x) s_w[c] = (b[c] - (c == j ? 1.0 : 0.0)) / bj;
    __syncthreads();
    double bv = -1.0;
    long long bi = LLONG_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        TB* bi_row = B + i * r;
        const double x = to_d(bi_row[j]);
        for (int c = 0; c < r; ++c) {
            const TB nb = (TB)(to_d(bi_row[c]) - x * s_w[c]);
            bi_row[c] = nb;
            const double a = fabs(to_d(nb));
            const long long key = (off + i) * r + c;
            if (better(a, key, bv, bi)) { bv = a; bi = key; }
        }
    }
    block_argmax(bv, bi);
    if (threadIdx.x == 0) { ckv[blockIdx.x] = bv; cki[blockIdx.x] = bi; }
}

__global__ void dmv_result_k(const DmvHdr* hdr, const int32_t* S, int r, int32_t* S_out, double* logvol_out,
                             int32_t* counts_out) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) if (S_out) S_out[k] = S[k];
    if (threadIdx.x == 0) {
        if (logvol_out) *logvol_out = hdr->logvol;
        if (counts_out) { counts_out[0] = hdr->swaps; counts_out[1] = hdr->status; }
    }
}

// ---------------------------------------------------------------- small gathers

// out[j, :] = X(ids[j] - off, :) when that row is in the slab, else zeros.
template <typename T>
__global__ void rows_at_k(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, int64_t off,
                          const int32_t* __restrict__ ids, int count, T* __restrict__ out) {
    const int64_t tot = (int64_t)count * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / cols);
        const int64_t c = e - (int64_t)j * cols;
        const int64_t i = (int64_t)ids[j] - off;
        out[e] = (i >= 0 && i < rows) ? X[i * ld + c] : (T)0;
    }
}

// Xt (cols x rows, contiguous) = X^T, 32 x 32 tiles through shared memory.
template <typename T>
__global__ void transpose_k(const T* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, T* __restrict__ Xt) {
    __shared__ T tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t i = r0 + k, c = c0 + threadIdx.x;
        if (i < rows && c < cols) tile[k][threadIdx.x] = X[i * ld + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, i = r0 + threadIdx.x;
        if (c < cols && i < rows) Xt[c * rows + i] = tile[threadIdx.x][k];
    }
}

__global__ void sa_init_k(AcaHdr* hdr, int64_t m_global) {
    if (threadIdx.x != 0) return;
    hdr->stop = 0;
    hdr->count = 0;
    hdr->p = -1;
    hdr->frob2 = 0.0;
    hdr->m_global = m_global;
}

__global__ void offset_ids_k(const int32_t* in, int count, int64_t off, int32_t* out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x)
        out[k] = (int32_t)(in[k] + off);
}

}  // namespace curk

using namespace curk;

static bool slab_ok(const cur_mat* A) {
    return A && A->data && A->rows >= 1 && A->cols >= 1 && A->ld >= A->cols &&
           (A->dtype == CUR_F64 || A->dtype == CUR_F32 || A->dtype == CUR_BF16);
}
static bool basis_ok(const cur_mat* C, int r) {
    return C && C->data && C->rows >= 1 && C->cols == r && C->ld == r &&
           (C->dtype == CUR_F64 || C->dtype == CUR_F32);
}

#define SH_ENTER(h)                                                  \
    do {                                                             \
        if (!(h)) return CUR_ERR_ARG;                                \
        CUR_CK(cudaSetDevice((h)->device));                          \
    } while (0)

template <typename TA>
static cur_status sa_pass(cur_handle* h, const cur_mat* A, const AcaLayout& L, char* base, int dot,
                          double* red, cudaStream_t st) {
    using PT = typename std::conditional<std::is_same<TA, double>::value, double, df64>::type;
    AcaHdr* hdr = reinterpret_cast<AcaHdr*>(base + L.hdr);
    CUR_TRY(aca_cols_partials(A, dot, reinterpret_cast<double*>(base + L.q64), reinterpret_cast<float*>(base + L.qh),
                              reinterpret_cast<float*>(base + L.ql), base + L.part, L.RC, L.chunk, &hdr->stop, st));
    sa_reduce_k<PT><<<nbs(L.n), 256, 0, st>>>(reinterpret_cast<const PT*>(base + L.part), L.RC, L.n, red, &hdr->stop);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

static cur_status sa_pass_any(cur_handle* h, const cur_mat* A, const AcaLayout& L, char* base, int dot,
                              double* red, cudaStream_t st) {
    switch (A->dtype) {
        case CUR_F64: return sa_pass<double>(h, A, L, base, dot, red, st);
        case CUR_F32: return sa_pass<float>(h, A, L, base, dot, red, st);
        case CUR_BF16: return sa_pass<__nv_bfloat16>(h, A, L, base, dot, red, st);
    }
    return CUR_ERR_ARG;
}

template <typename TA>
static cur_status sa_vec_launch(const cur_mat* A, const AcaLayout& L, char* base, int t, cudaStream_t st) {
    sa_vec_k<TA><<<kShardG, 256, 0, st>>>(static_cast<const TA*>(A->data), L.m, L.n, A->ld, t, L.r,
                                          reinterpret_cast<const double*>(base + L.Q),
                                          reinterpret_cast<const double*>(base + L.W),
                                          reinterpret_cast<double*>(base + L.v),
                                          reinterpret_cast<double*>(base + L.cta),
                                          reinterpret_cast<const AcaHdr*>(base + L.hdr));
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

template <typename TB>
static cur_status dmv_coef_launch(const cur_mat* C, int64_t off, const DmvLayout& L, char* base, double* keyv_out,
                                  cudaStream_t st) {
    const int r = L.r;
    DmvHdr* hdr = reinterpret_cast<DmvHdr*>(base + L.hdr);
    const size_t smf = ((size_t)r * r + r) * sizeof(double) + (size_t)r * sizeof(int) + 64;
    CUR_TRY(smem_attr((const void*)dmv_factor_k, smf));
    dmv_factor_k<<<1, 256, smf, st>>>(reinterpret_cast<const double*>(base + L.M), r,
                                      reinterpret_cast<double*>(base + L.Minv), hdr);
    CUR_CK(cudaGetLastError());
    const size_t smc = (size_t)r * r * sizeof(double);
    CUR_TRY(smem_attr((const void*)dmv_coef_k<TB>, smc));
    dmv_coef_k<TB><<<kShardG, 256, smc, st>>>(static_cast<const TB*>(C->data), L.p, off, r,
                                             reinterpret_cast<const double*>(base + L.Minv),
                                             reinterpret_cast<TB*>(base + L.B), reinterpret_cast<double*>(base + L.ckv),
                                             reinterpret_cast<long long*>(base + L.cki), hdr);
    CUR_CK(cudaGetLastError());
    dmv_key_k<<<1, 256, 0, st>>>(reinterpret_cast<const double*>(base + L.ckv),
                                 reinterpret_cast<const long long*>(base + L.cki), kShardG, hdr, keyv_out);
    CUR_CK(cudaGetLastError());
    note_launch(3);
    return CUR_OK;
}

template <typename TB>
static cur_status dmv_swap_launch(const cur_mat* C, int64_t off, const DmvLayout& L, char* base, const long long* keyi,
                                  const void* row, double* keyv_out, cudaStream_t st) {
    const int r = L.r;
    DmvHdr* hdr = reinterpret_cast<DmvHdr*>(base + L.hdr);
    dmv_row_k<TB><<<1, 256, 0, st>>>(static_cast<const TB*>(row), keyi, r, reinterpret_cast<double*>(base + L.M),
                                     reinterpret_cast<double*>(base + L.Minv), reinterpret_cast<int32_t*>(base + L.S),
                                     reinterpret_cast<double*>(base + L.b), reinterpret_cast<double*>(base + L.colj), hdr);
    CUR_CK(cudaGetLastError());
    dmv_update_k<TB><<<kShardG, 256, 0, st>>>(reinterpret_cast<TB*>(base + L.B), L.p, off, r, keyi,
                                              reinterpret_cast<const double*>(base + L.b),
                                              reinterpret_cast<double*>(base + L.ckv),
                                              reinterpret_cast<long long*>(base + L.cki));
    CUR_CK(cudaGetLastError());
    dmv_key_k<<<1, 256, 0, st>>>(reinterpret_cast<const double*>(base + L.ckv),
                                 reinterpret_cast<const long long*>(base + L.cki), kShardG, hdr, keyv_out);
    CUR_CK(cudaGetLastError());
    note_launch(3);
    return CUR_OK;
}

extern "C" {

// ---- Algorithm 3 on the columns of a row slab

size_t cur_shard_aca_state_bytes(cur_handle* h, const cur_mat* A_k, int32_t r) {
    if (!h || !slab_ok(A_k) || r < 1 || r > 128) return 0;
    return aca_layout(h, A_k, r).total;
}

cur_status cur_shard_aca_begin(cur_handle* h, const cur_mat* A_k, int64_t m_global, int32_t r, void* state,
                               int32_t* idx_out, double* red, cudaStream_t stream) {
    SH_ENTER(h);
    if (!slab_ok(A_k) || !state || !idx_out || !red || r < 1 || r > 128 || r > A_k->cols ||
        m_global < A_k->rows)
        return CUR_ERR_ARG;
    const AcaLayout L = aca_layout(h, A_k, r);
    char* base = static_cast<char*>(state);
    sa_init_k<<<1, 32, 0, stream>>>(reinterpret_cast<AcaHdr*>(base + L.hdr), m_global);
    CUR_CK(cudaGetLastError());
    note_launch();
    CUR_CK(cudaMemsetAsync(base + L.mask, 0, (size_t)L.n, stream));
    CUR_CK(cudaMemsetAsync(idx_out, 0xff, sizeof(int32_t) * r, stream));
    return sa_pass_any(h, A_k, L, base, 0, red, stream);
}

cur_status cur_shard_aca_pick(cur_handle* h, const cur_mat* A_k, int32_t r, int32_t t, void* state,
                              const double* red, double* red2, cudaStream_t stream) {
    SH_ENTER(h);
    if (!slab_ok(A_k) || !state || !red || !red2 || r < 1 || r > 128 || t < 0 || t >= r) return CUR_ERR_ARG;
    const AcaLayout L = aca_layout(h, A_k, r);
    char* base = static_cast<char*>(state);
    AcaHdr* hdr = reinterpret_cast<AcaHdr*>(base + L.hdr);
    sa_pick_k<<<1, 1024, 0, stream>>>(red, L.n, t, reinterpret_cast<double*>(base + L.nu),
                                      reinterpret_cast<double*>(base + L.W),
                                      reinterpret_cast<unsigned char*>(base + L.mask), hdr, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    switch (A_k->dtype) {
        case CUR_F64: CUR_TRY(sa_vec_launch<double>(A_k, L, base, t, stream)); break;
        case CUR_F32: CUR_TRY(sa_vec_launch<float>(A_k, L, base, t, stream)); break;
        case CUR_BF16: CUR_TRY(sa_vec_launch<__nv_bfloat16>(A_k, L, base, t, stream)); break;
    }
    sa_sum_k<<<1, 128, 0, stream>>>(reinterpret_cast<const double*>(base + L.cta), kShardG, r, t + 1, r, red2, hdr);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_shard_aca_commit(cur_handle* h, const cur_mat* A_k, int32_t r, int32_t t, void* state,
                                const double* red2, int32_t* idx_out, double* red, cudaStream_t stream) {
    SH_ENTER(h);
    if (!slab_ok(A_k) || !state || !red2 || !idx_out || !red || r < 1 || r > 128 || t < 0 || t >= r)
        return CUR_ERR_ARG;
    const AcaLayout L = aca_layout(h, A_k, r);
    char* base = static_cast<char*>(state);
    AcaHdr* hdr = reinterpret_cast<AcaHdr*>(base + L.hdr);
    // the rounding-level test uses max(m, n) of the whole matrix (m from the header)
    sa_commit_k<<<kShardG, 256, 0, stream>>>(L.m, L.n, t, red2, reinterpret_cast<const double*>(base + L.v),
                                             reinterpret_cast<double*>(base + L.Q),
                                             reinterpret_cast<double*>(base + L.q64),
                                             reinterpret_cast<float*>(base + L.qh),
                                             reinterpret_cast<float*>(base + L.ql),
                                             reinterpret_cast<unsigned char*>(base + L.mask), idx_out, hdr,
                                             h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    if (t + 1 < r) return sa_pass_any(h, A_k, L, base, 1, red, stream);
    return CUR_OK;
}

cur_status cur_shard_aca_finish(cur_handle* h, const cur_mat* A_k, int32_t r, void* state, int32_t* idx_out,
                                cudaStream_t stream) {
    SH_ENTER(h);
    if (!slab_ok(A_k) || !state || !idx_out || r < 1 || r > 128) return CUR_ERR_ARG;
    const AcaLayout L = aca_layout(h, A_k, r);
    char* base = static_cast<char*>(state);
    return pad_indices_dev(idx_out, reinterpret_cast<const int32_t*>(base + L.hdr + offsetof(AcaHdr, count)), r, L.n,
                           stream);
}

// ---- maxvol over a basis distributed by row slabs

size_t cur_dmv_state_bytes(int64_t p_local, int32_t r, cur_dtype dt) {
    if (p_local < 1 || r < 1 || r > 128 || (dt != CUR_F32 && dt != CUR_F64)) return 0;
    return dmv_layout(p_local, r, dt).total;
}

cur_status cur_dmv_begin(cur_handle* h, const cur_mat* C_k, int64_t offset, const int32_t* S, const void* M_rows,
                         void* state, double* keyv_out, cudaStream_t stream) {
    SH_ENTER(h);
    if (!C_k || C_k->cols < 1 || C_k->cols > 128 || !basis_ok(C_k, (int)C_k->cols) || offset < 0 || !S ||
        !M_rows || !state || !keyv_out)
        return CUR_ERR_ARG;
    const int r = (int)C_k->cols;
    const DmvLayout L = dmv_layout(C_k->rows, r, C_k->dtype);
    char* base = static_cast<char*>(state);
    DmvHdr* hdr = reinterpret_cast<DmvHdr*>(base + L.hdr);
    if (C_k->dtype == CUR_F64)
        dmv_load_k<double><<<1, 256, 0, stream>>>(S, static_cast<const double*>(M_rows), r,
                                                  reinterpret_cast<int32_t*>(base + L.S),
                                                  reinterpret_cast<double*>(base + L.M), hdr);
    else
        dmv_load_k<float><<<1, 256, 0, stream>>>(S, static_cast<const float*>(M_rows), r,
                                                 reinterpret_cast<int32_t*>(base + L.S),
                                                 reinterpret_cast<double*>(base + L.M), hdr);
    CUR_CK(cudaGetLastError());
    note_launch();
    if (C_k->dtype == CUR_F64) return dmv_coef_launch<double>(C_k, offset, L, base, keyv_out, stream);
    return dmv_coef_launch<float>(C_k, offset, L, base, keyv_out, stream);
}

cur_status cur_dmv_refresh(cur_handle* h, const cur_mat* C_k, int64_t offset, void* state, double* keyv_out,
                           cudaStream_t stream) {
    SH_ENTER(h);
    if (!C_k || C_k->cols < 1 || C_k->cols > 128 || !basis_ok(C_k, (int)C_k->cols) || offset < 0 || !state ||
        !keyv_out)
        return CUR_ERR_ARG;
    const DmvLayout L = dmv_layout(C_k->rows, (int)C_k->cols, C_k->dtype);
    char* base = static_cast<char*>(state);
    if (C_k->dtype == CUR_F64) return dmv_coef_launch<double>(C_k, offset, L, base, keyv_out, stream);
    return dmv_coef_launch<float>(C_k, offset, L, base, keyv_out, stream);
}

cur_status cur_dmv_holder(cur_handle* h, const cur_mat* C_k, void* state, const double* keyv_glob,
                          long long* keyi_out, cudaStream_t stream) {
    SH_ENTER(h);
    if (!C_k || C_k->cols < 1 || C_k->cols > 128 || !basis_ok(C_k, (int)C_k->cols) || !state || !keyv_glob ||
        !keyi_out)
        return CUR_ERR_ARG;
    const DmvLayout L = dmv_layout(C_k->rows, (int)C_k->cols, C_k->dtype);
    dmv_holder_k<<<1, 32, 0, stream>>>(reinterpret_cast<const DmvHdr*>(static_cast<char*>(state) + L.hdr), keyv_glob,
                                       keyi_out);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_dmv_fill(cur_handle* h, const cur_mat* C_k, int64_t offset, const long long* keyi_glob, void* row_out,
                        cudaStream_t stream) {
    SH_ENTER(h);
    if (!C_k || C_k->cols < 1 || C_k->cols > 128 || !basis_ok(C_k, (int)C_k->cols) || offset < 0 || !keyi_glob ||
        !row_out)
        return CUR_ERR_ARG;
    const int r = (int)C_k->cols;
    if (C_k->dtype == CUR_F64)
        dmv_fill_k<double><<<1, 128, 0, stream>>>(static_cast<const double*>(C_k->data), C_k->rows, offset, r,
                                                  keyi_glob, static_cast<double*>(row_out));
    else
        dmv_fill_k<float><<<1, 128, 0, stream>>>(static_cast<const float*>(C_k->data), C_k->rows, offset, r,
                                                 keyi_glob, static_cast<float*>(row_out));
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_dmv_swap(cur_handle* h, const cur_mat* C_k, int64_t offset, void* state, const long long* keyi_glob,
                        const void* row, double* keyv_out, cudaStream_t stream) {
    SH_ENTER(h);
    if (!C_k || C_k->cols < 1 || C_k->cols > 128 || !basis_ok(C_k, (int)C_k->cols) || offset < 0 || !state ||
        !keyi_glob || !row || !keyv_out)
        return CUR_ERR_ARG;
    const DmvLayout L = dmv_layout(C_k->rows, (int)C_k->cols, C_k->dtype);
    char* base = static_cast<char*>(state);
    if (C_k->dtype == CUR_F64) return dmv_swap_launch<double>(C_k, offset, L, base, keyi_glob, row, keyv_out, stream);
    return dmv_swap_launch<float>(C_k, offset, L, base, keyi_glob, row, keyv_out, stream);
}

cur_status cur_dmv_result(cur_handle* h, const cur_mat* C_k, void* state, int32_t* S_out, double* logvol_out,
                          int32_t* counts_out, cudaStream_t stream) {
    SH_ENTER(h);
    if (!C_k || C_k->cols < 1 || C_k->cols > 128 || !basis_ok(C_k, (int)C_k->cols) || !state) return CUR_ERR_ARG;
    const DmvLayout L = dmv_layout(C_k->rows, (int)C_k->cols, C_k->dtype);
    char* base = static_cast<char*>(state);
    dmv_result_k<<<1, 128, 0, stream>>>(reinterpret_cast<const DmvHdr*>(base + L.hdr),
                                        reinterpret_cast<const int32_t*>(base + L.S), L.r, S_out, logvol_out,
                                        counts_out);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

// ---- gathers and index maps

cur_status cur_rows_at(cur_handle* h, const cur_mat* X, int64_t offset, const int32_t* ids, int32_t count,
                       void* out, cudaStream_t stream) {
    SH_ENTER(h);
    if (!slab_ok(X) || !ids || !out || count < 1 || X->dtype == CUR_BF16) return CUR_ERR_ARG;
    const int64_t tot = (int64_t)count * X->cols;
    if (X->dtype == CUR_F64)
        rows_at_k<double><<<nbs(tot), 256, 0, stream>>>(static_cast<const double*>(X->data), X->rows, X->cols, X->ld,
                                                        offset, ids, count, static_cast<double*>(out));
    else
        rows_at_k<float><<<nbs(tot), 256, 0, stream>>>(static_cast<const float*>(X->data), X->rows, X->cols, X->ld,
                                                       offset, ids, count, static_cast<float*>(out));
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_transpose(cur_handle* h, const cur_mat* X, void* Xt_out, cudaStream_t stream) {
    SH_ENTER(h);
    if (!slab_ok(X) || !Xt_out || X->dtype == CUR_BF16) return CUR_ERR_ARG;
    const dim3 grid((unsigned)((X->cols + 31) / 32), (unsigned)((X->rows + 31) / 32));
    if (grid.y > 65535) return CUR_ERR_ARG;
    if (X->dtype == CUR_F64)
        transpose_k<double><<<grid, dim3(32, 8), 0, stream>>>(static_cast<const double*>(X->data), X->rows, X->cols,
                                                              X->ld, static_cast<double*>(Xt_out));
    else
        transpose_k<float><<<grid, dim3(32, 8), 0, stream>>>(static_cast<const float*>(X->data), X->rows, X->cols,
                                                             X->ld, static_cast<float*>(Xt_out));
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_offset_ids(cur_handle* h, const int32_t* ids, int32_t count, int64_t offset, int32_t* out,
                          cudaStream_t stream) {
    SH_ENTER(h);
    if (!ids || !out || count < 1) return CUR_ERR_ARG;
    offset_ids_k<<<nbs(count), 256, 0, stream>>>(ids, count, offset, out);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

}  // extern "C"
