// Shared device helpers for libcur (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#include "cur.h"
#include "df64.cuh"

namespace curk {

constexpr int kWarp = 32;
// Upper bound on one device-side wait (~2 s at 2 GHz). A wait that runs out sets
// CUR_ERR_TIMEOUT in the status word and returns; nothing spins forever.
constexpr long long kWaitCycles = 4000000000LL;

// ---------------------------------------------------------------- element types

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(double x) { return (float)x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// Compute type of the maxvol coefficients for a given element type.
template <typename T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

// ---------------------------------------------------------------- status word

// The first error wins; an error replaces an earlier CUR_WARN_RANK, never the reverse.
__device__ __forceinline__ void set_status(int* st, int code) {
    if (!st) return;
    const int old = atomicCAS(st, 0, code);
    if (old == CUR_WARN_RANK && code != CUR_WARN_RANK) atomicCAS(st, CUR_WARN_RANK, code);
}

// ---------------------------------------------------------------- accurate dot products
//
// Error-free transformations in FP32: TwoProduct through FMA and Knuth's TwoSum
// (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 26(6), 2005, algorithm Dot2). The explicit _rn intrinsics are never contracted
// into FMAs by the compiler, which the transformations rely on. q is given as an
// unevaluated sum qh + ql of two floats, so that the FP32 products carry the
// accuracy of a double-precision q. The result is as if computed in about twice
// FP32 precision and then rounded: error ~ 2^-48 sum|a_i q_i| + 2^-24 |result|,
// and the result is read out in double.
struct Dot2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float qh, float ql) {
        float p = __fmul_rn(a, qh);
        float e = __fmaf_rn(a, qh, -p);
        e = __fmaf_rn(a, ql, e);
        float t = __fadd_rn(s, p);
        float bp = __fsub_rn(t, s);
        float sg = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(sg, e));
    }
    __device__ __forceinline__ void add_sq(float a) { add(a, a, 0.f); }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Plain double accumulator with the same interface (FP64 data).
struct DotD {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double q) { s = fma(a, q, s); }
    __device__ __forceinline__ void add_sq(double a) { s = fma(a, a, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// Split a double into hi + lo floats (hi = fl32(x), lo = fl32(x - hi)).
__device__ __forceinline__ void split_d(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (value, index) maximum: larger value wins, then the smaller index.
__device__ __forceinline__ bool better(double v1, long long i1, double v2, long long i2) {
    return v1 > v2 || (v1 == v2 && i1 < i2);
}

// Order-preserving integer key of a double: dkey(a) < dkey(b) iff a < b, for numbers a, b
// (-0 and +0 share one key); NaN takes key 0, below -inf, so it is never a maximum. Only
// integer operations: GB300's FP64 pipe runs at about 1/64 of the FP32 rate, and the
// comparisons of a (value, index) reduction in FP64 were the slow part of every argmax.
__device__ __forceinline__ unsigned long long dkey(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if ((b << 1) == 0ull) return 1ull << 63;
    if ((b & 0x7ff0000000000000ull) == 0x7ff0000000000000ull && (b & 0x000fffffffffffffull) != 0ull) return 0ull;
    return (b >> 63) ? ~b : (b | (1ull << 63));
}
__device__ __forceinline__ double dkey_value(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & ~(1ull << 63)) : ~k;
    return __longlong_as_double((long long)b);
}
// Key of a float, in the same order (for values that never meet a double's key).
__device__ __forceinline__ unsigned fkey(float v) {
    const unsigned b = __float_as_uint(v);
    if ((b << 1) == 0u) return 1u << 31;
    if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu) != 0u) return 0u;
    return (b >> 31) ? ~b : (b | (1u << 31));
}
__device__ __forceinline__ bool better_key(unsigned long long k1, long long i1, unsigned long long k2, long long i2) {
    return k1 > k2 || (k1 == k2 && i1 < i2);
}

// Warp-wide (key, index) maximum by four redux.sync steps: the largest key, then among its
// holders the smallest index (signed order). All 32 lanes call it; every lane gets the result.
__device__ __forceinline__ void warp_argmax_key(unsigned long long& k, long long& i) {
    const unsigned full = 0xffffffffu;
    const unsigned kh = (unsigned)(k >> 32), kl = (unsigned)k;
    const unsigned mh = __reduce_max_sync(full, kh);
    const unsigned ml = __reduce_max_sync(full, kh == mh ? kl : 0u);
    const bool cand = kh == mh && kl == ml;
    const unsigned long long u = cand ? ((unsigned long long)i ^ (1ull << 63)) : ~0ull;
    const unsigned uh = __reduce_min_sync(full, (unsigned)(u >> 32));
    const unsigned ul = __reduce_min_sync(full, (unsigned)(u >> 32) == uh ? (unsigned)u : ~0u);
    k = ((unsigned long long)mh << 32) | ml;
    i = (long long)((((unsigned long long)uh << 32) | ul) ^ (1ull << 63));
}

__device__ __forceinline__ void warp_argmax(double& v, long long& i) {
    unsigned long long k = dkey(v);
    warp_argmax_key(k, i);
    v = dkey_value(k);
}

// Block-wide (key, index) maximum; every thread gets the result. blockDim.x must be a
// multiple of 32 and at most 1024. Uses 2 x 32 words of static shared memory.
__device__ __forceinline__ void block_argmax_key(unsigned long long& k, long long& i) {
    __shared__ unsigned long long sk[32];
    __shared__ long long si[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    warp_argmax_key(k, i);
    __syncthreads();
    if (lane == 0) { sk[warp] = k; si[warp] = i; }
    __syncthreads();
    if (warp == 0) {
        k = lane < nw ? sk[lane] : 0ull;
        i = lane < nw ? si[lane] : (long long)0x7fffffffffffffffLL;
        warp_argmax_key(k, i);
        if (lane == 0) { sk[0] = k; si[0] = i; }
    }
    __syncthreads();
    k = sk[0];
    i = si[0];
    __syncthreads();
}

// Block-wide (value, index) maximum of doubles (larger value, then smaller index).
__device__ __forceinline__ void block_argmax(double& v, long long& i) {
    unsigned long long k = dkey(v);
    block_argmax_key(k, i);
    v = dkey_value(k);
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sb[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sb[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) sb[0] = v;
    }
    __syncthreads();
    v = sb[0];
    __syncthreads();
    return v;
}

// Sum of x[0..n) by one warp: lane l adds x[l], x[l+32], ... in order, then a fixed
// xor tree. Every lane returns the same value, identical in every CTA that calls it.
__device__ __forceinline__ double warp_sum_strided(const double* x, int n, int64_t stride = 1) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    int g = lane;
    for (; g + 96 < n; g += 128) {   // four loads in flight, summed in index order
        const double x0 = x[(int64_t)g * stride], x1 = x[(int64_t)(g + 32) * stride];
        const double x2 = x[(int64_t)(g + 64) * stride], x3 = x[(int64_t)(g + 96) * stride];
        s += x0;
        s += x1;
        s += x2;
        s += x3;
    }
    for (; g < n; g += 32) s += x[(int64_t)g * stride];
    return warp_sum(s);
}

// Walks the flat index e = tid, tid + nt, ... of an nloc x r array as (row, column)
// without a division per step.
struct Walk2 {
    int i, c, di, dc, r;
    __device__ __forceinline__ Walk2(int e0, int step, int r_) : r(r_) {
        i = e0 / r_;
        c = e0 - i * r_;
        di = step / r_;
        dc = step - di * r_;
    }
    __device__ __forceinline__ void next() {
        i += di;
        c += dc;
        if (c >= r) { c -= r; ++i; }
    }
};

__device__ __forceinline__ double block_max(double v) {
    __shared__ double sb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sb[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sb[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sb[0] = v;
    }
    __syncthreads();
    v = sb[0];
    __syncthreads();
    return v;
}

// ---------------------------------------------------------------- group barrier
//
// CTAs of one group (all co-resident: cooperative launch) meet here. `ctr` is a
// counter zeroed before the launch; the n-th barrier of a group of G CTAs waits
// for ctr >= n * G. Returns false (and sets CUR_ERR_TIMEOUT) if the wait runs out.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool group_barrier(unsigned* ctr, unsigned target, int* status,
                                              long long limit = kWaitCycles) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(ctr, 1u);
        const long long t0 = clock64();
        while (ld_acquire_u32(ctr) < target) {
            if (clock64() - t0 > limit) {
                ok = 0;
                set_status(status, CUR_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    const int ok = s_ok;
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------- small dense inverse
//
// In-place Gauss-Jordan inverse of the r x r row-major matrix A (shared memory),
// FP64, partial pivoting by rows (first maximum |a_ik|, i >= k). The k-th pivot is
// the k-th pivot of LU with partial pivoting, so |pivot| <= thresh flags the same
// numerical singularity and sum log|pivot| = log|det A|. Columns are unscrambled at
// the end in the reverse order of the row interchanges. colk: r doubles, piv: r ints
// of shared memory. Returns 1 if singular (A then holds no inverse).
__device__ __forceinline__ int gj_inverse(double* A, int r, double* colk, int* piv,
                                          double thresh, double* logabsdet) {
    __shared__ int s_sing, s_p;
    __shared__ double s_dinv;
    __shared__ double s_prow[128];   // the step's pivot row, scaled (r <= 128)
    __shared__ double s_colk[128];   // the other buffer of the pivot column (steps alternate)
    __shared__ LogAcc s_lacc;        // log|det| without a logarithm per step
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    // One warp: the pivot of column k (its first maximum |a_ik|, i >= k, compared as integer
    // keys), its test, the log|det| factor and its reciprocal (one FP64 division), and the
    // column k as it will be after the row interchange. Step k's elimination runs this for
    // column k + 1 as soon as that column is final, so it overlaps the rest of the elimination.
    auto pivot_of = [&](int k, double* ck) {
        unsigned long long bk = 0ull;
        long long bi = k;
        for (int i = k + lane; i < r; i += 32) {
            const unsigned long long x = dkey(fabs(A[i * r + k]));
            if (x > bk) { bk = x; bi = i; }
        }
        warp_argmax_key(bk, bi);
        const int p = (int)bi;
        for (int i = lane; i < r; i += 32) ck[i] = A[(i == k ? p : (i == p ? k : i)) * r + k];
        if (lane == 0) {
            const double d = A[p * r + k];
            s_p = p;
            if (!(fabs(d) > thresh)) s_sing = 1;
            else { s_lacc.mul(df_from_d(d)); s_dinv = 1.0 / d; }
        }
        __syncwarp();
    };
    if (tid == 0) { s_sing = 0; s_lacc.init(); }
    __syncthreads();
    if (tid < 32) pivot_of(0, colk);
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (s_sing) return 1;
        const int p = s_p;
        const double dinv = s_dinv;
        const double* ck = (k & 1) ? s_colk : colk;   // the column k after the interchange
        // every thread: rows k and p interchanged, and the scaled pivot row (from row p)
        for (int c = tid; c < r; c += nt) {
            const double ak = A[k * r + c], ap = A[p * r + c];
            s_prow[c] = (c == k ? 1.0 : ap) * dinv;
            if (p != k) {
                A[k * r + c] = ap;
                A[p * r + c] = ak;
            }
        }
        if (tid == 0) piv[k] = p;
        __syncthreads();
        // elimination: warp 0 finishes column k + 1 and finds the next pivot while the
        // other warps eliminate every other column
        const int kn = k + 1;
        if (tid < 32) {
            if (kn < r) {
                const double akc = s_prow[kn];
                for (int i = lane; i < r; i += 32)
                    A[i * r + kn] = i == k ? akc : fma(-ck[i], akc, A[i * r + kn]);
                __syncwarp();
                pivot_of(kn, (kn & 1) ? s_colk : colk);
            }
        } else {
            Walk2 w(tid - 32, nt - 32, r);
            for (int e = tid - 32; e < r * r; e += nt - 32, w.next())
                if (w.c != kn) A[e] = w.i == k ? s_prow[w.c] : fma(-ck[w.i], s_prow[w.c], w.c == k ? 0.0 : A[e]);
        }
        __syncthreads();
    }
    for (int k = r - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int i = tid; i < r; i += nt) {
                const double t = A[i * r + k];
                A[i * r + k] = A[i * r + p];
                A[i * r + p] = t;
            }
        __syncthreads();
    }
    if (logabsdet) *logabsdet = s_lacc.log_value();
    return 0;
}

}  // namespace curk
