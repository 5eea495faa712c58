// Global maxvol with low-precision coefficient products (the precision option of the swap
// iteration of Section 1.2's maximal-volume refinement).
//
// Each iteration forms B = C M^-1 for all p rows of the basis as a BF16 x BF16 -> FP32
// tcgen05 product (kind::f16), or E4M3 x E4M3 -> FP32 (kind::f8f6f4) with every row of C and
// of (M^-1)^T scaled to E4M3's range, and reduces argmax |B_ij| in the epilogue without
// writing B. C is rounded once; (M^-1)^T after every swap. The product kernel is warp
// specialised: one lane streams 128-row tiles of C through a ring of TMA stages, one lane
// issues the MMAs into two TMEM accumulators, four warps read them back. Each CTA then
// evaluates its two candidate entries exactly, b_ij = C(i,:) M^-1(:,j) with M^-1 held as a
// double-float pair (hi + lo floats, about 2^-48 relative), the products formed by the
// error-free Dot2 sums on the FP32 pipes and read out in FP64 (GB300's FP64 rate is a small
// fraction of its FP32 rate, so FP64-class arithmetic runs on the FP32 pipes, as in the swap
// engine). One CTA takes the row of the largest exact entry over all CTAs, recomputes it in
// full, and swaps on its largest entry only if |b_j| > 1 + delta (the exact argmax unless
// rounding pushed it below its CTA's two best rows); M^-1 gets its Sherman-Morrison update in
// double-float. The start is factorised in FP64 (or handed over). The first winner whose
// exact value does not pass ends this phase, and the FP32/FP64 swap engine (maxvol.cu)
// finishes from the set reached, so the result is dominant to the same standard as the
// plain path's. Every accepted swap raises the volume by |b_j| > 1 + delta, so the phase
// cannot cycle.

#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace curk {

constexpr int kLpBM = 128;           // rows of C per tile (MMA M)
constexpr int kLpKC = 64;            // BF16 elements per 128-byte swizzled K chunk
constexpr int kLpChunkC = kLpBM * 128;  // bytes of one K chunk of a C tile
constexpr int kLpEpiWarps = 4;        // warps reading the accumulators
constexpr int kLpThreadsWS = 32 * (2 + kLpEpiWarps);
constexpr int kLpBatch = 16;         // iterations launched between two reads of the control block

// Instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulator, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor: kind::f8f6f4 with E4M3 A and B, FP32 accumulator, both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_e4m3(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// The largest finite E4M3 value; each row of a scaled FP8 operand is stretched to it.
constexpr float kE4M3Max = 448.f;
__device__ __forceinline__ unsigned char to_e4m3(float x) {
    return (unsigned char)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

struct LpCtl {           // control block of one call (device)
    int done;            // the BF16 phase is over
    int swaps;           // swaps it took
    int status;          // CUR_OK or CUR_ERR_SINGULAR (start set)
    int pad;
    double logvol;       // log|det C(S,:)|
};

struct LpCand {          // a CTA's largest exact |b_ij| over its two candidate entries (-1: none)
    double v;
    int i, j;
};

__device__ __forceinline__ bool lp_better(float v, int i, int j, float v2, int i2, int j2) {
    return v > v2 || (v == v2 && (i < i2 || (i == i2 && j < j2)));
}

// Cq (p x ldk BF16) = C (p x r FP32), zero past column r.
__global__ void lp_quant_c(const float* __restrict__ C, int64_t p, int r, int ldk, __nv_bfloat16* __restrict__ Cq) {
    const int64_t total = p * ldk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldk;
        const int k = (int)(e - i * ldk);
        Cq[e] = __float2bfloat16_rn(k < r ? C[i * r + k] : 0.f);
    }
}

// Cq (p x ldk E4M3) = C s_i with s_i = 448 / max_k |C_ik| per row (1 for a zero row),
// cinv[i] = 1 / s_i; zero past column r. One warp per row.
__global__ void lp_quant_c8(const float* __restrict__ C, int64_t p, int r, int ldk, unsigned char* __restrict__ Cq,
                            float* __restrict__ cinv) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < p; i += nw) {
        float mx = 0.f;
        for (int k = lane; k < r; k += 32) mx = fmaxf(mx, fabsf(C[i * r + k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float sc = mx > 0.f && isfinite(mx) ? kE4M3Max / mx : 1.f;
        for (int k = lane; k < ldk; k += 32) Cq[i * ldk + k] = k < r ? to_e4m3(C[i * r + k] * sc) : (unsigned char)0;
        if (lane == 0) cinv[i] = 1.f / sc;
    }
}

// W (r x ldk) = (M^-1)^T from its hi part (M^-1[k][n] at M[k * pitch + n]), zero past column
// r: BF16 rounded, or E4M3 with row n scaled by t_n = 448 / max_k |M^-1[k][n]| and
// winv[n] = 1 / t_n. Ends with the block synchronised.
template <bool F8>
__device__ __forceinline__ void lp_requant(const float* M, int pitch, int r, int ldk, void* W, float* winv) {
    if constexpr (!F8) {
        __nv_bfloat16* Wb = static_cast<__nv_bfloat16*>(W);
        for (int n = threadIdx.x >> 5; n < r; n += blockDim.x >> 5)
            for (int k = threadIdx.x & 31; k < ldk; k += 32)
                Wb[n * ldk + k] = __float2bfloat16_rn(k < r ? M[k * pitch + n] : 0.f);
    } else {
        unsigned char* W8 = static_cast<unsigned char*>(W);
        const int lane = threadIdx.x & 31;
        for (int n = threadIdx.x >> 5; n < r; n += blockDim.x >> 5) {
            float mx = 0.f;
            for (int k = lane; k < r; k += 32) mx = fmaxf(mx, fabsf(M[k * pitch + n]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const float t = mx > 0.f && isfinite(mx) ? kE4M3Max / mx : 1.f;
            for (int k = lane; k < ldk; k += 32) W8[n * ldk + k] = k < r ? to_e4m3(M[k * pitch + n] * t) : (unsigned char)0;
            if (lane == 0) winv[n] = 1.f / t;
        }
    }
    __syncthreads();
}

// M = C(S,:) in FP64, its inverse (as hi + lo floats) and log|det|; one CTA.
template <bool F8>
__global__ void lp_setup_k(const float* __restrict__ C, int r, int ldk, const int32_t* S, void* W, float* winv,
                           float* Mh, float* Ml, LpCtl* ctl) {
    extern __shared__ double lsm[];
    double* M = lsm;                   // r x r
    double* colk = M + r * r;          // r
    int* piv = reinterpret_cast<int*>(colk + r);
    const int tid = threadIdx.x;
    double mx = 0.0;
    for (int e = tid; e < r * r; e += blockDim.x) {
        const double x = (double)C[(int64_t)S[e / r] * r + (e % r)];
        M[e] = x;
        mx = fmax(mx, fabs(x));
    }
    mx = block_max(mx);
    double lv = 0.0;
    const int sing = gj_inverse(M, r, colk, piv, (double)r * 2.220446049250313e-16 * mx, &lv);
    if (sing) {
        if (tid == 0) { ctl->status = CUR_ERR_SINGULAR; ctl->done = 1; ctl->logvol = -INFINITY; }
        return;
    }
    for (int e = tid; e < r * r; e += blockDim.x) split_d(M[e], Mh[e], Ml[e]);
    __syncthreads();
    lp_requant<F8>(Mh, r, r, ldk, W, winv);
    if (tid == 0) { ctl->status = CUR_OK; ctl->done = 0; ctl->swaps = 0; ctl->logvol = lv; }
}

// The same from a given FP64 inverse of C(S,:) (r x r, row-major): split and rounded only.
template <bool F8>
__global__ void lp_setup_from_k(const double* __restrict__ minv, int r, int ldk, void* W, float* winv, float* Mh,
                                float* Ml, LpCtl* ctl) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) split_d(minv[e], Mh[e], Ml[e]);
    __syncthreads();
    lp_requant<F8>(Mh, r, r, ldk, W, winv);
    if (threadIdx.x == 0) { ctl->status = CUR_OK; ctl->done = 0; ctl->swaps = 0; ctl->logvol = 0.0; }
}

// argmax |B_ij| over all rows of C for B = Cq Wq^T: persistent CTAs over 128-row tiles, warp
// specialised. Warp 0 (one lane) streams the tiles of C through a ring of NS shared-
// memory stages with TMA; warp 1 (one lane) issues the MMAs of each tile into one of two TMEM
// accumulators; warps 2..5 read an accumulator back (warp w: TMEM lanes 32 (w % 4) ...) while
// the next tile is loaded and multiplied, and keep the CTA's two best rows. At the end the
// candidate entries of those two rows are evaluated exactly (warps 0 and 1).
template <bool F8, int NS>
__global__ void __launch_bounds__(kLpThreadsWS) lp_argmax_k(const __grid_constant__ CUtensorMap mC,
                                                            const __grid_constant__ CUtensorMap mW, int64_t p, int r,
                                                            int kc, int tcols, const float* __restrict__ cinv,
                                                            const float* __restrict__ winv, const float* __restrict__ C,
                                                            const float* __restrict__ Mh, const float* __restrict__ Ml,
                                                            const LpCtl* ctl, LpCand* cand, int* status) {
    extern __shared__ unsigned char lp_raw[];
    __shared__ uint64_t full[NS], empty[NS], accf[2], acce[2], wbar;
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ float red_v[2 * kLpEpiWarps];
    __shared__ int red_i[2 * kLpEpiWarps], red_j[2 * kLpEpiWarps];
    __shared__ float s_winv[128];
    __shared__ int s_rows[2], s_cols[2];
    __shared__ double s_ev[2];
    __shared__ int s_ei[2], s_ej[2];
    if (ctl->done) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* WS = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(lp_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t wchunk = (uint32_t)r * 128;
    unsigned char* CS = WS + (size_t)kc * wchunk;
    const uint32_t cbuf = (uint32_t)kc * kLpChunkC;     // one stage: a 128-row tile of C
    const int64_t ntiles = (p + kLpBM - 1) / kLpBM;
    const int nloc = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    constexpr int kEl = F8 ? 128 : kLpKC;   // elements of one 128-byte K chunk
    const int rpad = (r + 31) / 32 * 32;    // TMEM columns of one accumulator
    if constexpr (F8)
        for (int j = tid; j < r; j += blockDim.x) s_winv[j] = winv[j];
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kLpEpiWarps);
        }
        mbar_init(&wbar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tslot, tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int issued[NS] = {};
            mbar_expect_tx(&wbar, (uint32_t)kc * wchunk);
            for (int c = 0; c < kc; ++c) tma_load_2d(WS + (size_t)c * wchunk, &mW, &wbar, kEl * c, 0);
            for (int k = 0; k < nloc && !abort_flag; ++k) {
                const int s = k % NS, u = k / NS;
                if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) { abort_flag = 1; break; }
                const int64_t tile = blockIdx.x + (int64_t)k * gridDim.x;
                mbar_expect_tx(&full[s], cbuf);
                for (int c = 0; c < kc; ++c)
                    tma_load_2d(CS + (size_t)s * cbuf + (size_t)c * kLpChunkC, &mC, &full[s], kEl * c,
                                (int)(tile * kLpBM));
                ++issued[s];
            }
            // every load issued has landed before the CTA's memory goes away
            mbar_wait(&wbar, 0);
            for (int s = 0; s < NS; ++s)
                if (issued[s] > 0) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1));
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = F8 ? idesc_e4m3(kLpBM, r) : idesc_bf16(kLpBM, r);
            bool ok = mbar_wait(&wbar, 0);
            int last = -1;
            for (int k = 0; k < nloc && ok && !abort_flag; ++k) {
                const int s = k % NS, u = k / NS, b = k & 1, v = k >> 1;
                if (!mbar_wait(&full[s], (uint32_t)(u & 1))) { ok = false; break; }
                if (v > 0 && !mbar_wait(&acce[b], (uint32_t)((v - 1) & 1))) { ok = false; break; }
                tc_fence_after();
                const uint32_t ca = su32(CS + (size_t)s * cbuf), wa = su32(WS);
                const uint32_t d = tmem + (uint32_t)(b * rpad);
                for (int q = 0; q < kc * 4; ++q) {
                    const uint32_t oc = (uint32_t)(q >> 2) * kLpChunkC + (uint32_t)(q & 3) * 32;
                    const uint32_t ow = (uint32_t)(q >> 2) * wchunk + (uint32_t)(q & 3) * 32;
                    if constexpr (F8) mma_e4m3(d, sdesc_k128(ca + oc), sdesc_k128(wa + ow), idesc, q != 0);
                    else mma_bf16(d, sdesc_k128(ca + oc), sdesc_k128(wa + ow), idesc, q != 0);
                }
                mma_commit(&empty[s]);
                mma_commit(&accf[b]);
                last = k;
            }
            if (!ok) abort_flag = 1;
            // every MMA issued has completed once the last commit has arrived
            if (last >= 0) mbar_wait(&accf[last & 1], (uint32_t)((last >> 1) & 1));
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int q = warp & 3;   // TMEM lane quarter of this warp
        float tv[2] = {-1.f, -1.f};
        int ti[2] = {INT_MAX, INT_MAX}, tj[2] = {INT_MAX, INT_MAX};
        for (int k = 0; k < nloc; ++k) {
            const int b = k & 1, v = k >> 1;
            if (!mbar_wait(&accf[b], (uint32_t)(v & 1))) { abort_flag = 1; break; }
            tc_fence_after();
            const int64_t tile = blockIdx.x + (int64_t)k * gridDim.x;
            const int64_t row = tile * kLpBM + 32 * q + lane;
            const float ci = F8 ? (row < p ? cinv[row] : 0.f) : 1.f;
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * rpad);
            float bv = -1.f;
            int bj = INT_MAX;
            for (int c0 = 0; c0 < r; c0 += 16) {
                float x[16];
                tmem_ld16(taddr + (uint32_t)c0, x);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float a = F8 ? fabsf(x[u]) * ci * s_winv[c0 + u] : fabsf(x[u]);
                    if (a > bv) { bv = a; bj = c0 + u; }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
            int bi = row < p ? (int)row : INT_MAX;
            if (row >= p) { bv = -1.f; bj = INT_MAX; }
            // this tile's two best rows of the warp, merged into the warp's running two
            for (int t = 0; t < 2; ++t) {
                float wv = bv;
                int wi = bi, wj = bj;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float v2 = __shfl_xor_sync(0xffffffffu, wv, o);
                    const int i2 = __shfl_xor_sync(0xffffffffu, wi, o);
                    const int j2 = __shfl_xor_sync(0xffffffffu, wj, o);
                    if (lp_better(v2, i2, j2, wv, wi, wj)) { wv = v2; wi = i2; wj = j2; }
                }
                if (bi == wi) { bv = -2.f; bi = INT_MAX; bj = INT_MAX; }
                if (lp_better(wv, wi, wj, tv[0], ti[0], tj[0])) {
                    tv[1] = tv[0]; ti[1] = ti[0]; tj[1] = tj[0];
                    tv[0] = wv; ti[0] = wi; tj[0] = wj;
                } else if (lp_better(wv, wi, wj, tv[1], ti[1], tj[1])) {
                    tv[1] = wv; ti[1] = wi; tj[1] = wj;
                }
            }
        }
        if (lane == 0) {
            const int e = 2 * (warp - 2);
            red_v[e] = tv[0]; red_i[e] = ti[0]; red_j[e] = tj[0];
            red_v[e + 1] = tv[1]; red_i[e + 1] = ti[1]; red_j[e + 1] = tj[1];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        float bv[2] = {-1.f, -1.f};
        int bi[2] = {INT_MAX, INT_MAX}, bj[2] = {INT_MAX, INT_MAX};
        if (abort_flag) {
            set_status(status, CUR_ERR_TIMEOUT);
        } else {
            for (int e = 0; e < 2 * kLpEpiWarps; ++e) {
                const float v = red_v[e];
                const int i = red_i[e], j = red_j[e];
                if (lp_better(v, i, j, bv[0], bi[0], bj[0])) {
                    bv[1] = bv[0]; bi[1] = bi[0]; bj[1] = bj[0];
                    bv[0] = v; bi[0] = i; bj[0] = j;
                } else if (lp_better(v, i, j, bv[1], bi[1], bj[1])) {
                    bv[1] = v; bi[1] = i; bj[1] = j;
                }
            }
        }
        for (int t = 0; t < 2; ++t) {
            s_rows[t] = bv[t] >= 0.f ? bi[t] : -1;
            s_cols[t] = bj[t];
        }
    }
    __syncthreads();
    // the exact value of each candidate entry, b_ij = C(i,:) M^-1(:,j) with M^-1 as hi + lo
    // floats (one warp per entry, Dot2 partial sums per lane, double-float warp reduction)
    if (warp < 2) {
        double ev = -1.0;
        int ei = INT_MAX, ej = INT_MAX;
        if (s_rows[warp] >= 0) {
            const int row = s_rows[warp], col = s_cols[warp];
            const float* a = C + (int64_t)row * r;
            Dot2 d;
            for (int l = lane; l < r; l += 32) d.add(__ldg(a + l), Mh[l * r + col], Ml[l * r + col]);
            df64 v = fast_two_sum(d.s, d.c);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v = df_add(v, df64{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
            ev = fabs(df_to_d(v));
            ei = row;
            ej = col;
        }
        if (lane == 0) { s_ev[warp] = ev; s_ei[warp] = ei; s_ej[warp] = ej; }
    }
    __syncthreads();
    if (tid == 0) {
        double ev = s_ev[0];
        int ei = s_ei[0], ej = s_ej[0];
        if (s_ev[1] > ev || (s_ev[1] == ev && (s_ei[1] < ei || (s_ei[1] == ei && s_ej[1] < ej)))) {
            ev = s_ev[1]; ei = s_ei[1]; ej = s_ej[1];
        }
        LpCand c;
        c.v = ev;
        c.i = ei;
        c.j = ej;
        cand[blockIdx.x] = c;
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// The winner of the CTAs' exact candidates; its swap and the double-float Sherman-Morrison
// update of M^-1 if it passes, else the end of the phase. One CTA.
template <bool F8>
__global__ void __launch_bounds__(1024) lp_swap_k(const float* __restrict__ C, int64_t p, int r, int ldk,
                                                  const LpCand* cand, int ncand, float* Mh, float* Ml, int32_t* S,
                                                  void* W, float* winv, LpCtl* ctl, double delta, int max_swaps) {
    extern __shared__ double lsm[];
    double* b = lsm;                                                // exact row i of B (r)
    df64* mcol = reinterpret_cast<df64*>(lsm + r);                  // column j of M^-1 (r)
    df64* g = mcol + r;                                             // (b - e_j) / b_j (r)
    const int rp = r + 1;                                           // padded row pitch of M^-1
    float* sh = reinterpret_cast<float*>(g + r);                    // M^-1 hi, r x rp
    float* sl = sh + r * rp;                                        // M^-1 lo, r x rp
    __shared__ double wv[32];
    __shared__ int wi[32], wj[32];
    __shared__ int si, sj;
    __shared__ double sv;
    if (ctl->done) return;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (int l = warp; l < r; l += nt >> 5)
        for (int c = lane; c < r; c += 32) {
            sh[l * rp + c] = Mh[l * r + c];
            sl[l * rp + c] = Ml[l * r + c];
        }
    double bv = -1.0;
    int bi = INT_MAX, bj = INT_MAX;
    for (int c = tid; c < ncand; c += nt) {
        const LpCand x = cand[c];
        if (x.v > bv || (x.v == bv && (x.i < bi || (x.i == bi && x.j < bj)))) { bv = x.v; bi = x.i; bj = x.j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
        if (v2 > bv || (v2 == bv && (i2 < bi || (i2 == bi && j2 < bj)))) { bv = v2; bi = i2; bj = j2; }
    }
    if (lane == 0) { wv[warp] = bv; wi[warp] = bi; wj[warp] = bj; }
    __syncthreads();
    if (tid < 32) {
        bv = tid < (nt >> 5) ? wv[tid] : -1.0;
        bi = tid < (nt >> 5) ? wi[tid] : INT_MAX;
        bj = tid < (nt >> 5) ? wj[tid] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
            if (v2 > bv || (v2 == bv && (i2 < bi || (i2 == bi && j2 < bj)))) { bv = v2; bi = i2; bj = j2; }
        }
        if (tid == 0) { sv = bv; si = bi; sj = bj; }
    }
    __syncthreads();
    const int i = si;
    if (!(sv >= 0.0) || i < 0 || (int64_t)i >= p) {
        if (tid == 0) ctl->done = 1;
        return;
    }
    // the winner's row, exactly, and its largest entry (lowest column on ties)
    for (int c = tid; c < r; c += nt) {
        const float* a = C + (int64_t)i * r;
        Dot2 d;
#pragma unroll 4
        for (int l = 0; l < r; ++l) d.add(a[l], sh[l * rp + c], sl[l * rp + c]);
        b[c] = d.value();
    }
    __syncthreads();
    if (tid < 32) {
        double bv2 = -1.0;
        int bj2 = INT_MAX;
        for (int c = tid; c < r; c += 32) {
            const double x = fabs(b[c]);
            if (x > bv2) { bv2 = x; bj2 = c; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, bv2, o);
            const int j2 = __shfl_xor_sync(0xffffffffu, bj2, o);
            if (v2 > bv2 || (v2 == bv2 && j2 < bj2)) { bv2 = v2; bj2 = j2; }
        }
        if (tid == 0) sj = bj2;
    }
    __syncthreads();
    const int j = sj;
    const double bjv = b[j];
    if (!(fabs(bjv) > 1.0 + delta)) {
        if (tid == 0) ctl->done = 1;
        return;
    }
    if (tid < r) {
        mcol[tid] = df_make(sh[tid * rp + j], sl[tid * rp + j]);
        g[tid] = df_div(df_from_d(b[tid] - (tid == j ? 1.0 : 0.0)), df_from_d(bjv));
    }
    __syncthreads();
    for (int l = warp; l < r; l += nt >> 5)
        for (int c = lane; c < r; c += 32) {
            const df64 v = df_sub(df_make(sh[l * rp + c], sl[l * rp + c]), df_mul(mcol[l], g[c]));
            sh[l * rp + c] = v.h;
            sl[l * rp + c] = v.l;
            Mh[l * r + c] = v.h;
            Ml[l * r + c] = v.l;
        }
    __syncthreads();
    // W from the updated M^-1 (the padded pitch keeps a warp's column reads conflict-free)
    lp_requant<F8>(sh, rp, r, ldk, W, winv);
    if (tid == 0) {
        S[j] = i;
        ctl->logvol += log(fabs(bjv));
        if (++ctl->swaps >= max_swaps) ctl->done = 1;
    }
}

__global__ void lp_finish_k(int32_t* swaps_out, const LpCtl* ctl, int exact_swaps, int code, int* hstatus) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (swaps_out) {
        swaps_out[0] = ctl->swaps + exact_swaps;
        swaps_out[1] = ctl->swaps;
    }
    if (code == CUR_ERR_SINGULAR || code == CUR_ERR_NOCONV || code == CUR_ERR_NONFINITE) set_status(hstatus, code);
}

// The same with the exact engine's result on the device.
__global__ void lp_finish_dev_k(int32_t* swaps_out, const LpCtl* ctl, const MvDevResult* res, int* hstatus) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (swaps_out) {
        swaps_out[0] = ctl->swaps + res->swaps;
        swaps_out[1] = ctl->swaps;
    }
    const int code = res->status;
    if (code == CUR_ERR_SINGULAR || code == CUR_ERR_NOCONV || code == CUR_ERR_NONFINITE) set_status(hstatus, code);
}

static PFN_cuTensorMapEncodeTiled_v12000 lp_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// rows x ldk elements of es bytes (ldk es a multiple of 128), boxes of 128 bytes x box_rows
// rows, 128-byte swizzle; BF16 (es = 2) or E4M3 bytes (es = 1).
static bool lp_map(CUtensorMap* map, const void* base, int64_t rows, int ldk, int box_rows, int es) {
    auto enc = lp_encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)ldk * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
               const_cast<void*>(base), gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace curk

// The stages of cur_cross take the low-precision phase only where its product has at least
// this many 128-row tiles per SM; below that the FP32 engine's shared-memory B is faster.
constexpr int64_t kBf16MinTilesPerSm = 4;

// The low-precision phase alone (BF16, or E4M3 with fp8), from S0 to S_out (device r
// ints; may alias). *swaps: the swaps it took; *status: CUR_OK or CUR_ERR_SINGULAR (a singular
// C(S0,:); S_out = S0). Synchronises the stream. C: p x r FP32 (contiguous, device), r a
// multiple of 16.
template <bool F8>
static cur_status lowprec_phase_t(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o,
                                  const int32_t* S0, int32_t* S_out, int* swaps, int* status, Arena& ar,
                                  cudaStream_t st, const double* minv_in) {
    using namespace curk;
    const size_t mark = ar.off;
    constexpr int es = F8 ? 1 : 2, kEl = 128 / es;
    const int kc = (r + kEl - 1) / kEl, ldk = kc * kEl;
    // two accumulators of rpad = r rounded up to 32 columns; TMEM is allocated in powers of 2
    const int rpad = (r + 31) / 32 * 32;
    const int tcols = 2 * rpad <= 64 ? 64 : (2 * rpad <= 128 ? 128 : 256);
    const int64_t ntiles = (p + kLpBM - 1) / kLpBM;
    // launch shapes of the product kernel: TMA stages (2 or 4) and CTAs per SM (1 or 2), as far
    // as shared memory (227 KB per SM) and TMEM (512 columns per SM) allow; the autotuner
    // picks one per class of (precision, r, p) by timing them (the results do not depend on it)
    struct Shape { int ns, per_sm; };
    const Shape shapes[4] = {{4, 2}, {4, 1}, {2, 2}, {2, 1}};
    auto smem_of = [&](int ns) { return 1024 + (size_t)kc * r * 128 + (size_t)ns * kc * kLpChunkC; };
    auto fits = [&](Shape c) {
        return (size_t)c.per_sm * smem_of(c.ns) <= (size_t)227 * 1024 && c.per_sm * tcols <= 512;
    };
    auto grid_of = [&](Shape c) { return (int)std::min<int64_t>({ntiles, (int64_t)c.per_sm * h->num_sms, 1024}); };
    const int grid_max = (int)std::min<int64_t>({ntiles, 2LL * h->num_sms, 1024});
    void* Cq = ar.take((size_t)p * ldk * es);
    void* W = ar.take((size_t)r * ldk * es);
    float* cinv = ar.get<float>(F8 ? (size_t)p : 1);
    float* winv = ar.get<float>((size_t)r);
    float* Mh = ar.get<float>((size_t)r * r);
    float* Ml = ar.get<float>((size_t)r * r);
    int32_t* S = ar.get<int32_t>(r);
    LpCand* cand = ar.get<LpCand>((size_t)grid_max);
    LpCtl* ctl = ar.get<LpCtl>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUtensorMap mC, mW;
    if (!lp_map(&mC, Cq, p, ldk, kLpBM, es) || !lp_map(&mW, W, r, ldk, r, es)) return CUR_ERR_ARG;
    CUR_CK(cudaMemsetAsync(ctl, 0, sizeof(LpCtl), st));
    CUR_CK(cudaMemcpyAsync(S, S0, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    const unsigned qgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p * ldk + 255) / 256, 8LL * h->num_sms));
    if constexpr (F8)
        lp_quant_c8<<<qgrid, 256, 0, st>>>(C, p, r, ldk, static_cast<unsigned char*>(Cq), cinv);
    else
        lp_quant_c<<<qgrid, 256, 0, st>>>(C, p, r, ldk, static_cast<__nv_bfloat16*>(Cq));
    CUR_CK(cudaGetLastError());
    if (minv_in) {
        lp_setup_from_k<F8><<<1, 256, 0, st>>>(minv_in, r, ldk, W, winv, Mh, Ml, ctl);
    } else {
        const size_t sm_setup = (size_t)r * r * sizeof(double) + (size_t)r * sizeof(double) + (size_t)r * sizeof(int) + 64;
        CUR_TRY(smem_attr((const void*)lp_setup_k<F8>, sm_setup));
        lp_setup_k<F8><<<1, 256, sm_setup, st>>>(C, r, ldk, S, W, winv, Mh, Ml, ctl);
    }
    CUR_CK(cudaGetLastError());
    note_launch(2);
    CUR_TRY(smem_attr((const void*)lp_argmax_k<F8, 4>, smem_of(4)));
    CUR_TRY(smem_attr((const void*)lp_argmax_k<F8, 2>, smem_of(2)));
    auto launch_argmax = [&](Shape c) -> cur_status {
        const int g = grid_of(c);
        if (c.ns == 4)
            lp_argmax_k<F8, 4><<<g, kLpThreadsWS, smem_of(4), st>>>(mC, mW, p, r, kc, tcols, cinv, winv, C, Mh, Ml,
                                                                   ctl, cand, h->status);
        else
            lp_argmax_k<F8, 2><<<g, kLpThreadsWS, smem_of(2), st>>>(mC, mW, p, r, kc, tcols, cinv, winv, C, Mh, Ml,
                                                                   ctl, cand, h->status);
        CUR_CK(cudaGetLastError());
        return CUR_OK;
    };
    const uint64_t tkey = (2ull << 56) | ((uint64_t)F8 << 48) | ((uint64_t)r << 16) | tune_log2((uint64_t)p);
    int choice = tune_lookup(h, tkey);
    if (choice < 0) {
        // time each shape that fits over three launches on the current inverse, keep the fastest
        float best_ms = 0.f;
        choice = -1;
        for (int c = 0; c < 4; ++c) {
            if (!fits(shapes[c])) continue;
            CUR_CK(cudaEventRecord(h->tune_ev[0], st));
            for (int rep = 0; rep < 3; ++rep) CUR_TRY(launch_argmax(shapes[c]));
            CUR_CK(cudaEventRecord(h->tune_ev[1], st));
            CUR_CK(cudaEventSynchronize(h->tune_ev[1]));
            float ms = 0.f;
            CUR_CK(cudaEventElapsedTime(&ms, h->tune_ev[0], h->tune_ev[1]));
            note_launch(3);
            if (choice < 0 || ms < best_ms) { best_ms = ms; choice = c; }
        }
        if (choice < 0) return CUR_ERR_ARG;
        tune_store(h, tkey, choice);
    }
    const Shape shape = shapes[choice];
    const int grid = grid_of(shape);
    const size_t sm_swap = (size_t)r * sizeof(double) + 2 * (size_t)r * sizeof(df64) +
                           2 * (size_t)r * (r + 1) * sizeof(float) + 16;
    CUR_TRY(smem_attr((const void*)lp_swap_k<F8>, sm_swap));
    const int max_swaps = o->max_swaps > 0 ? o->max_swaps : 100 * r;
    LpCtl* hc = reinterpret_cast<LpCtl*>(h->host_stage);
    CUR_CK(cudaEventSynchronize(h->stage_ev));   // host_stage is free once its last copy has run
    for (;;) {
        for (int q = 0; q < kLpBatch; ++q) {
            CUR_TRY(launch_argmax(shape));
            lp_swap_k<F8><<<1, 1024, sm_swap, st>>>(C, p, r, ldk, cand, grid, Mh, Ml, S, W, winv, ctl, o->delta,
                                                    max_swaps);
            CUR_CK(cudaGetLastError());
        }
        note_launch(2 * kLpBatch);
        CUR_CK(cudaMemcpyAsync(hc, ctl, sizeof(LpCtl), cudaMemcpyDeviceToHost, st));
        CUR_CK(cudaStreamSynchronize(st));
        if (hc->done) break;
    }
    *swaps = hc->swaps;
    *status = hc->status;
    CUR_CK(cudaEventRecord(h->stage_ev, st));
    CUR_CK(cudaMemcpyAsync(S_out, *status == CUR_ERR_SINGULAR ? S0 : S, sizeof(int32_t) * r,
                           cudaMemcpyDeviceToDevice, st));
    CUR_CK(cudaStreamSynchronize(st));
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

cur_status lowprec_phase(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o, const int32_t* S0,
                         int32_t* S_out, int* swaps, int* status, Arena& ar, cudaStream_t st, const double* minv_in) {
    if (o->flags & CUR_FLAG_PREC_FP8)
        return lowprec_phase_t<true>(h, C, p, r, o, S0, S_out, swaps, status, ar, st, minv_in);
    return lowprec_phase_t<false>(h, C, p, r, o, S0, S_out, swaps, status, ar, st, minv_in);
}

bool lowprec_phase_applies(const cur_handle* h, const cur_opts* o, cur_dtype dt, int64_t p, int r) {
    return (o->flags & (CUR_FLAG_PREC_BF16 | CUR_FLAG_PREC_FP8)) && dt == CUR_F32 && r % 16 == 0 && r >= 16 && r <= 128 &&
           p >= (int64_t)kBf16MinTilesPerSm * curk::kLpBM * h->num_sms && p <= INT_MAX - 256;
}

// The low-precision phase, then the exact engine from the set it reached.
static cur_status maxvol_global_bf16(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o,
                                     const int32_t* S0, int32_t* S_out, double* logvol_out, int32_t* swaps_out,
                                     Arena& ar, cudaStream_t st) {
    using namespace curk;
    int lp_swaps = 0, lp_status = CUR_OK;
    CUR_TRY(lowprec_phase(h, C, p, r, o, S0, S_out, &lp_swaps, &lp_status, ar, st, nullptr));
    LpCtl* ctl = ar.get<LpCtl>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    LpCtl hv{};
    hv.swaps = lp_swaps;
    hv.logvol = -INFINITY;
    CUR_CK(cudaMemcpyAsync(ctl, &hv, sizeof(LpCtl), cudaMemcpyHostToDevice, st));
    if (lp_status == CUR_ERR_SINGULAR) {
        if (logvol_out) CUR_CK(cudaMemcpyAsync(logvol_out, &ctl->logvol, sizeof(double), cudaMemcpyDeviceToDevice, st));
        lp_finish_k<<<1, 32, 0, st>>>(swaps_out, ctl, 0, CUR_ERR_SINGULAR, h->status);
        CUR_CK(cudaGetLastError());
        note_launch();
        CUR_CK(cudaStreamSynchronize(st));
        return CUR_OK;
    }
    MvDevResult* res = ar.get<MvDevResult>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(maxvol_global(h, CUR_F32, C, p, r, o, S_out, S_out, logvol_out, res, ar, st));
    lp_finish_dev_k<<<1, 32, 0, st>>>(swaps_out, ctl, res, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

extern "C" {

cur_status cur_maxvol_global(cur_handle* h, const cur_mat* basis, const int32_t* S0, int32_t r,
                             const cur_opts* opts, int32_t* S_out, double* logvol_out, int32_t* swaps_out,
                             cudaStream_t st) {
    if (!h || !basis || !basis->data || !S0 || !S_out) return CUR_ERR_ARG;
    const int64_t p = basis->rows;
    if (r < 1 || r > 128 || basis->cols != r || basis->ld != r || p < r || p > INT_MAX - 256) return CUR_ERR_ARG;
    cur_opts o = opts ? *opts : cur_default_opts();
    if (!(o.delta >= 0.0)) return CUR_ERR_ARG;
    Arena ar = h->arena();
    if (o.flags & (CUR_FLAG_PREC_BF16 | CUR_FLAG_PREC_FP8)) {
        if (basis->dtype != CUR_F32 || r % 16 != 0) return CUR_ERR_ARG;
        return maxvol_global_bf16(h, static_cast<const float*>(basis->data), p, r, &o, S0, S_out, logvol_out,
                                  swaps_out, ar, st);
    }
    if (basis->dtype != CUR_F32 && basis->dtype != CUR_F64) return CUR_ERR_ARG;
    MvDevResult* res = ar.get<MvDevResult>(1);
    curk::LpCtl* ctl = ar.get<curk::LpCtl>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(maxvol_global(h, basis->dtype, basis->data, p, r, &o, S0, S_out, logvol_out, res, ar, st));
    CUR_CK(cudaMemsetAsync(ctl, 0, sizeof(curk::LpCtl), st));
    curk::lp_finish_dev_k<<<1, 32, 0, st>>>(swaps_out, ctl, res, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

}  // extern "C"
