// Global maxvol with low-precision coefficient products (the precision option of the swap
// iteration of Section 1.2's maximal-volume refinement).
//
// Each iteration forms B = C M^-1 for all p rows of the basis as a BF16 x BF16 -> FP32
// tcgen05 product (kind::f16), or E4M3 x E4M3 -> FP32 (kind::f8f6f4) with every row of C and
// of (M^-1)^T scaled to E4M3's range, and reduces argmax |B_ij| in the epilogue without
// writing B. C is rounded once; (M^-1)^T after every swap. The whole loop is one persistent
// cooperative launch (one CTA per SM, warp specialised): one lane streams the CTA's 128-row
// tiles of C through a ring of TMA stages, one lane issues the MMAs into two TMEM
// accumulators, eight warps read them back and keep their threads' two best rows. Each CTA
// then evaluates its two best candidate entries exactly, b_ij = C(i,:) M^-1(:,j) with M^-1
// held as a double-float pair (hi + lo floats, about 2^-48 relative), the products formed by
// the error-free Dot2 sums on the FP32 pipes and read out in FP64 (GB300's FP64 rate is a
// small fraction of its FP32 rate, so FP64-class arithmetic runs on the FP32 pipes, as in the
// swap engine). Between grid barriers every CTA takes the row of the largest exact entry
// over all CTAs, the CTAs recompute that row in full (an entry each), and the swap is made on
// its largest entry only if |b_j| > 1 + delta (the exact argmax unless rounding pushed it
// below its CTA's two best rows): each CTA updates the rows of M^-1 it owns by
// Sherman-Morrison in double-float, with their part of W = (M^-1)^T. The start is factorised
// in FP64 (or handed over) on the device. The first winner whose exact value does not pass
// ends the loop, and the FP32/FP64 swap engine (maxvol.cu) finishes from the set reached, so
// the result is dominant to the same standard as the plain path's. Every accepted swap raises
// the volume by |b_j| > 1 + delta, so the phase cannot cycle. Nothing waits on the host.

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
constexpr int kLpEpiWarps = 8;        // warps reading the accumulators (lane quarter x column half)
constexpr int kLpThreadsWS = 32 * (2 + kLpEpiWarps);

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

// The start of the phase, on the device (one CTA): S = S0; nothing more when `idle` is set;
// the given FP64 inverse of C(S0,:) when it is valid (minv_flag NULL, CUR_OK or
// CUR_ERR_NOCONV); else C(S0,:) in FP64, its inverse and log|det| (a singular start ends the
// phase with CUR_ERR_SINGULAR). M^-1 is kept as hi + lo floats; W = (M^-1)^T rounded. Also
// clears the loop's grid-barrier counter.
template <bool F8>
__global__ void lp_setup_k(const float* __restrict__ C, int r, int ldk, const int32_t* S0, int32_t* S,
                           const double* minv_in, const int* minv_flag, const int* idle, void* W, float* winv,
                           float* Mh, float* Ml, LpCtl* ctl, unsigned* gbar) {
    extern __shared__ double lsm[];
    double* M = lsm;                   // r x r
    double* colk = M + r * r;          // r
    int* piv = reinterpret_cast<int*>(colk + r);
    const int tid = threadIdx.x;
    for (int k = tid; k < r; k += blockDim.x) S[k] = S0[k];
    if (tid == 0) {
        *gbar = 0u;
        ctl->status = CUR_OK;
        ctl->done = 0;
        ctl->swaps = 0;
        ctl->logvol = 0.0;
    }
    if (idle && *idle) {
        if (tid == 0) ctl->done = 1;
        return;
    }
    const bool given = minv_in && (!minv_flag || *minv_flag == CUR_OK || *minv_flag == CUR_ERR_NOCONV);
    if (given) {
        for (int e = tid; e < r * r; e += blockDim.x) split_d(minv_in[e], Mh[e], Ml[e]);
    } else {
        double mx = 0.0;
        for (int e = tid; e < r * r; e += blockDim.x) {
            const double x = (double)C[(int64_t)S0[e / r] * r + (e % r)];
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
        if (tid == 0) ctl->logvol = lv;
    }
    __syncthreads();
    lp_requant<F8>(Mh, r, r, ldk, W, winv);
}

// Barrier of the eight epilogue warps (named barrier 1, 256 threads); returns the OR of v over
// them, so that every one of them takes the same branch after it.
__device__ __forceinline__ bool epi_sync_or(bool v) {
    int res;
    asm volatile("{ .reg .pred p, q; setp.ne.b32 q, %1, 0; bar.red.or.pred p, 1, 256, q; selp.u32 %0, 1, 0, p; }"
                 : "=r"(res) : "r"((int)v) : "memory");
    return res != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Grid barrier of the loop: the calling thread (one per CTA) arrives on the counter and waits
// for `target` arrivals (G times the barrier's ordinal, counted alike in every CTA). False
// after the time limit.
__device__ __forceinline__ bool lp_grid_sync(unsigned* ctr, unsigned target) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const long long t0 = clock64();
    while (ld_acquire_u32(ctr) < target) {
        if (clock64() - t0 > kWaitCycles) return false;
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// Waits (bounded) until iteration `it` is released or the loop ends; false on the time limit.
__device__ __forceinline__ bool lp_wait_go(volatile int* go, volatile int* quit, int64_t it) {
    const long long t0 = clock64();
    while (*go < it && !*quit) {
        if (clock64() - t0 > kTcWait) return false;
        __nanosleep(64);
    }
    return true;
}

struct LpLoop {          // arguments of the swap loop
    int64_t p;
    int r, kc, ldk, tcols;
    const float* cinv;   // FP8: 1 / scale of each row of C
    float* winv;         // FP8: 1 / scale of each row of W (rewritten by the swaps)
    const float* C;      // p x r FP32 basis
    float* Mh;           // M^-1, hi and lo floats (r x r)
    float* Ml;
    void* W;             // (M^-1)^T rounded (r x ldk)
    int32_t* S;
    LpCtl* ctl;
    LpCand* cand;        // one per CTA
    double* brow;        // r: the winner's exact row of B
    unsigned* gbar;      // grid-barrier counter, zero at launch
    double delta;
    int max_swaps;
    int* status;
};

// The whole swap loop of the phase in one persistent cooperative launch (one CTA per SM).
// Each iteration: B = Cq Wq^T for all p rows with the argmax |B_ij| in the epilogue (warp 0,
// one lane: TMA loads of W and of the CTA's 128-row tiles of C through a ring of NS stages,
// the first NS tiles of the next iteration loaded during this one's swap; warp 1, one lane:
// the MMAs into two TMEM accumulators; warps 2..9: the accumulators read back, each warp a lane
// quarter and half of the columns, each thread keeping the two best of its rows over the
// iteration; then the CTA's two best rows, their candidate entries evaluated exactly). Then,
// on the epilogue warps of every
// CTA, between grid barriers: the winner over all CTAs' candidates (every CTA alike); its
// exact row b = C(i,:) M^-1, one entry per CTA; the swap test |b_j| > 1 + delta on its largest
// entry; the double-float Sherman-Morrison update of the rows of M^-1 each CTA owns, with
// their columns of W. C and W are read from L2 (ld.global.cg) where another CTA wrote them.
template <bool F8, int NS>
__global__ void __launch_bounds__(kLpThreadsWS, 1) lp_loop_k(const __grid_constant__ CUtensorMap mC,
                                                             const __grid_constant__ CUtensorMap mW, LpLoop a) {
    extern __shared__ unsigned char lp_raw[];
    __shared__ uint64_t full[NS], empty[NS], accf[2], acce[2], wbar;
    __shared__ uint32_t tslot;
    __shared__ volatile int s_go, s_quit;   // iteration released to the TMA and MMA lanes; end of the loop
    __shared__ float red_v[2 * kLpEpiWarps];
    __shared__ int red_i[2 * kLpEpiWarps], red_j[2 * kLpEpiWarps];
    __shared__ float s_winv[128];
    __shared__ int s_rows[2], s_cols[2];
    __shared__ double s_ev[2];
    __shared__ int s_ei[2], s_ej[2];
    __shared__ double s_wv[kLpEpiWarps];
    __shared__ int s_wi[kLpEpiWarps];
    __shared__ double s_b[128];
    __shared__ df64 s_g[128];
    __shared__ int s_i, s_j;
    __shared__ double s_bj;
    if (a.ctl->done) return;   // a singular (or skipped) start: every CTA leaves
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = a.r, kc = a.kc, G = gridDim.x;
    unsigned char* WS = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(lp_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t wchunk = (uint32_t)r * 128;
    unsigned char* CS = WS + (size_t)kc * wchunk;
    const uint32_t cbuf = (uint32_t)kc * kLpChunkC;     // one stage: a 128-row tile of C
    const int64_t ntiles = (a.p + kLpBM - 1) / kLpBM;
    const int nloc = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / G + 1) : 0;
    constexpr int kEl = F8 ? 128 : kLpKC;   // elements of one 128-byte K chunk
    const int rpad = (r + 31) / 32 * 32;    // TMEM columns of one accumulator
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
        s_go = 0;
        s_quit = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tslot, a.tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int issued[NS] = {};
            int nw = 0;
            bool ok = true;
            const int pre = min(NS, nloc);
            auto issue = [&](int64_t it, int k) -> bool {
                const int64_t gk = it * nloc + k;
                const int s = (int)(gk % NS);
                const int64_t u = gk / NS;
                if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1))) return false;
                const int64_t tile = blockIdx.x + (int64_t)k * G;
                mbar_expect_tx(&full[s], cbuf);
                for (int c = 0; c < kc; ++c)
                    tma_load_2d(CS + (size_t)s * cbuf + (size_t)c * kLpChunkC, &mC, &full[s], kEl * c,
                                (int)(tile * kLpBM));
                ++issued[s];
                return true;
            };
            for (int64_t it = 0; ok; ++it) {
                if (it > 0) {
                    if (!lp_wait_go(&s_go, &s_quit, it)) { ok = false; break; }
                    if (s_quit) break;
                }
                // W of this iteration (written by the epilogue warps of every CTA before the release)
                asm volatile("fence.proxy.async.global;" ::: "memory");
                mbar_expect_tx(&wbar, (uint32_t)kc * wchunk);
                for (int c = 0; c < kc; ++c) tma_load_2d(WS + (size_t)c * wchunk, &mW, &wbar, kEl * c, 0);
                ++nw;
                for (int k = it > 0 ? pre : 0; k < nloc && ok; ++k) ok = issue(it, k);
                // C does not change: the next iteration's first tiles load during this one's swap
                for (int k = 0; k < pre && ok; ++k) ok = issue(it + 1, k);
            }
            if (!ok) set_status(a.status, CUR_ERR_TIMEOUT);
            // every load issued has landed before the CTA's memory goes away
            if (nw > 0) mbar_wait(&wbar, (uint32_t)((nw - 1) & 1));
            for (int s = 0; s < NS; ++s)
                if (issued[s] > 0) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1));
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = F8 ? idesc_e4m3(kLpBM, r) : idesc_bf16(kLpBM, r);
            bool ok = true;
            int64_t last = -1;
            for (int64_t it = 0; ok; ++it) {
                if (it > 0) {
                    if (!lp_wait_go(&s_go, &s_quit, it)) { ok = false; break; }
                    if (s_quit) break;
                }
                if (!mbar_wait(&wbar, (uint32_t)(it & 1))) { ok = false; break; }
                for (int k = 0; k < nloc; ++k) {
                    const int64_t gk = it * nloc + k;
                    const int s = (int)(gk % NS), b = (int)(gk & 1);
                    const int64_t u = gk / NS, v = gk >> 1;
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
                    last = gk;
                }
            }
            if (!ok) set_status(a.status, CUR_ERR_TIMEOUT);
            // every MMA issued has completed once the last commit has arrived
            if (last >= 0) mbar_wait(&accf[last & 1], (uint32_t)((last >> 1) & 1));
        }
    } else {
        // ---------------------------------------------------------------- epilogue and swap
        const int q = warp & 3;        // TMEM lane quarter of this warp
        const int ew = warp - 2;       // 0..7
        const int et = tid - 64;       // 0..255
        // this warp's columns: the first or second half of the 16-column groups
        const int ng = (r + 15) / 16, hsplit = (ng + 1) / 2;
        const int cb = ew < 4 ? 0 : 16 * hsplit, ce = ew < 4 ? min(r, 16 * hsplit) : r;
        int64_t gk = 0;
        unsigned ep = 0;               // grid barriers passed
        int swaps = 0;
        for (int64_t it = 0;; ++it) {
            if constexpr (F8)
                for (int j = et; j < r; j += 256) s_winv[j] = __ldcg(a.winv + j);
            epi_sync();
            // the two best (|b|, row, column) of this thread's rows and columns
            float tv[2] = {-1.f, -1.f};
            int ti[2] = {INT_MAX, INT_MAX}, tj[2] = {INT_MAX, INT_MAX};
            bool ok = true;
            for (int k = 0; k < nloc; ++k, ++gk) {
                const int b = (int)(gk & 1);
                if (!mbar_wait(&accf[b], (uint32_t)((gk >> 1) & 1))) { ok = false; break; }
                tc_fence_after();
                const int64_t tile = blockIdx.x + (int64_t)k * G;
                const int64_t row = tile * kLpBM + 32 * q + lane;
                const float ci = F8 ? (row < a.p ? a.cinv[row] : 0.f) : 1.f;
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * rpad);
                float bv = -1.f;
                int bj = INT_MAX;
                for (int c0 = cb; c0 < ce; c0 += 32) {
                    if (c0 + 32 <= ce) {
                        float x[32];
                        tmem_ld32(taddr + (uint32_t)c0, x);
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            const float av = F8 ? fabsf(x[u]) * ci * s_winv[c0 + u] : fabsf(x[u]);
                            if (av > bv) { bv = av; bj = c0 + u; }
                        }
                    } else {
                        float x[16];
                        tmem_ld16(taddr + (uint32_t)c0, x);
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const float av = F8 ? fabsf(x[u]) * ci * s_winv[c0 + u] : fabsf(x[u]);
                            if (av > bv) { bv = av; bj = c0 + u; }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[b]);
                if (row < a.p && bj != INT_MAX) {
                    const int bi = (int)row;
                    if (lp_better(bv, bi, bj, tv[0], ti[0], tj[0])) {
                        tv[1] = tv[0]; ti[1] = ti[0]; tj[1] = tj[0];
                        tv[0] = bv; ti[0] = bi; tj[0] = bj;
                    } else if (lp_better(bv, bi, bj, tv[1], ti[1], tj[1])) {
                        tv[1] = bv; ti[1] = bi; tj[1] = bj;
                    }
                }
            }
            // the warp's two best entries (its rows are distinct: one per lane and tile)
            {
                int row1 = -1;
                for (int t = 0; t < 2; ++t) {
                    const int u = (t == 1 && ti[0] == row1) ? 1 : 0;
                    float wv = tv[u];
                    int wi = ti[u], wj = tj[u];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float v2 = __shfl_xor_sync(0xffffffffu, wv, o);
                        const int i2 = __shfl_xor_sync(0xffffffffu, wi, o);
                        const int j2 = __shfl_xor_sync(0xffffffffu, wj, o);
                        if (lp_better(v2, i2, j2, wv, wi, wj)) { wv = v2; wi = i2; wj = j2; }
                    }
                    if (lane == 0) { red_v[2 * ew + t] = wv; red_i[2 * ew + t] = wi; red_j[2 * ew + t] = wj; }
                    row1 = wi;
                }
            }
            if (epi_sync_or(!ok)) { set_status(a.status, CUR_ERR_TIMEOUT); break; }
            // the CTA's two best rows (distinct), each with its best column: every row's best
            // entry over the two column halves is among the warps' two best
            if (ew == 0) {
                int row1 = -1;
                for (int t = 0; t < 2; ++t) {
                    float wv = -1.f;
                    int wi = INT_MAX, wj = INT_MAX;
                    for (int e = lane; e < 2 * kLpEpiWarps; e += 32) {
                        const float v = red_v[e];
                        const int i = red_i[e], j = red_j[e];
                        if (v >= 0.f && i != row1 && lp_better(v, i, j, wv, wi, wj)) { wv = v; wi = i; wj = j; }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float v2 = __shfl_xor_sync(0xffffffffu, wv, o);
                        const int i2 = __shfl_xor_sync(0xffffffffu, wi, o);
                        const int j2 = __shfl_xor_sync(0xffffffffu, wj, o);
                        if (lp_better(v2, i2, j2, wv, wi, wj)) { wv = v2; wi = i2; wj = j2; }
                    }
                    if (lane == 0) {
                        s_rows[t] = wv >= 0.f ? wi : -1;
                        s_cols[t] = wj;
                    }
                    row1 = wv >= 0.f ? wi : -2;
                }
            }
            epi_sync();
            // the exact value of each candidate entry, b_ij = C(i,:) M^-1(:,j) with M^-1 as hi + lo
            // floats (one warp per entry, Dot2 partial sums per lane, double-float warp reduction)
            if (ew < 2) {
                double ev = -1.0;
                int ei = INT_MAX, ej = INT_MAX;
                if (s_rows[ew] >= 0) {
                    const int row = s_rows[ew], col = s_cols[ew];
                    const float* ar = a.C + (int64_t)row * r;
                    Dot2 d;
                    for (int l = lane; l < r; l += 32) d.add(__ldg(ar + l), __ldcg(a.Mh + l * r + col), __ldcg(a.Ml + l * r + col));
                    df64 v = fast_two_sum(d.s, d.c);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        v = df_add(v, df64{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
                    ev = fabs(df_to_d(v));
                    ei = row;
                    ej = col;
                }
                if (lane == 0) { s_ev[ew] = ev; s_ei[ew] = ei; s_ej[ew] = ej; }
            }
            epi_sync();
            bool gfail = false;
            if (et == 0) {
                double ev = s_ev[0];
                int ei = s_ei[0], ej = s_ej[0];
                if (s_ev[1] > ev || (s_ev[1] == ev && (s_ei[1] < ei || (s_ei[1] == ei && s_ej[1] < ej)))) {
                    ev = s_ev[1]; ei = s_ei[1]; ej = s_ej[1];
                }
                LpCand c;
                c.v = ev;
                c.i = ei;
                c.j = ej;
                a.cand[blockIdx.x] = c;
                gfail = !lp_grid_sync(a.gbar, (unsigned)G * ++ep);
            }
            if (epi_sync_or(gfail)) { set_status(a.status, CUR_ERR_TIMEOUT); break; }
            // the winner over every CTA's exact candidate (the same in every CTA)
            {
                double bv = -1.0;
                int bi = INT_MAX, bj = INT_MAX;
                for (int c = et; c < G; c += 256) {
                    const double xv = __ldcg(&a.cand[c].v);
                    const int xi = __ldcg(&a.cand[c].i), xj = __ldcg(&a.cand[c].j);
                    if (xv > bv || (xv == bv && (xi < bi || (xi == bi && xj < bj)))) { bv = xv; bi = xi; bj = xj; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
                    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                    const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
                    if (v2 > bv || (v2 == bv && (i2 < bi || (i2 == bi && j2 < bj)))) { bv = v2; bi = i2; bj = j2; }
                }
                if (lane == 0) { s_wv[ew] = bv; s_wi[ew] = bi; red_j[ew] = bj; }
                epi_sync();
                if (et == 0) {
                    bv = s_wv[0]; bi = s_wi[0]; bj = red_j[0];
                    for (int w = 1; w < kLpEpiWarps; ++w) {
                        const double v2 = s_wv[w];
                        const int i2 = s_wi[w], j2 = red_j[w];
                        if (v2 > bv || (v2 == bv && (i2 < bi || (i2 == bi && j2 < bj)))) { bv = v2; bi = i2; bj = j2; }
                    }
                    s_i = (bv >= 0.0 && bi >= 0 && (int64_t)bi < a.p) ? bi : -1;
                }
                epi_sync();
            }
            const int i = s_i;
            if (i < 0) break;   // no candidate: the phase ends
            // the winner's exact row, b_c = C(i,:) M^-1(:,c): the entries c = blockIdx.x + G w of
            // this CTA, one warp each
            for (int c = blockIdx.x + G * ew; c < r; c += G * kLpEpiWarps) {
                const float* ar = a.C + (int64_t)i * r;
                Dot2 d;
                for (int l = lane; l < r; l += 32) d.add(__ldg(ar + l), __ldcg(a.Mh + l * r + c), __ldcg(a.Ml + l * r + c));
                df64 v = fast_two_sum(d.s, d.c);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    v = df_add(v, df64{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
                if (lane == 0) a.brow[c] = df_to_d(v);
            }
            epi_sync();
            gfail = false;
            if (et == 0) gfail = !lp_grid_sync(a.gbar, (unsigned)G * ++ep);
            if (epi_sync_or(gfail)) { set_status(a.status, CUR_ERR_TIMEOUT); break; }
            // its largest entry (lowest column on ties) and the swap test
            for (int c = et; c < r; c += 256) s_b[c] = __ldcg(a.brow + c);
            epi_sync();
            if (ew == 0) {
                double bv2 = -1.0;
                int bj2 = INT_MAX;
                for (int c = lane; c < r; c += 32) {
                    const double x = fabs(s_b[c]);
                    if (x > bv2) { bv2 = x; bj2 = c; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, bv2, o);
                    const int j2 = __shfl_xor_sync(0xffffffffu, bj2, o);
                    if (v2 > bv2 || (v2 == bv2 && j2 < bj2)) { bv2 = v2; bj2 = j2; }
                }
                if (lane == 0) { s_j = bj2; s_bj = s_b[bj2]; }
            }
            epi_sync();
            const int j = s_j;
            const double bjv = s_bj;
            if (!(fabs(bjv) > 1.0 + a.delta)) break;   // the winner does not pass: the phase ends
            // Sherman-Morrison on the rows l = blockIdx.x, blockIdx.x + G, ... of M^-1 (double-
            // float) and, for BF16, their columns of W = (M^-1)^T
            for (int c = et; c < r; c += 256) s_g[c] = df_div(df_from_d(s_b[c] - (c == j ? 1.0 : 0.0)), df_from_d(bjv));
            epi_sync();
            for (int l = blockIdx.x; l < r; l += G) {
                const df64 ml = df_make(__ldcg(a.Mh + l * r + j), __ldcg(a.Ml + l * r + j));
                epi_sync();   // every thread has M^-1(l, j) before it is overwritten
                for (int c = et; c < r; c += 256) {
                    const df64 v = df_sub(df_make(__ldcg(a.Mh + l * r + c), __ldcg(a.Ml + l * r + c)), df_mul(ml, s_g[c]));
                    a.Mh[l * r + c] = v.h;
                    a.Ml[l * r + c] = v.l;
                    if constexpr (!F8) static_cast<__nv_bfloat16*>(a.W)[(int64_t)c * a.ldk + l] = __float2bfloat16_rn(v.h);
                }
            }
            if constexpr (F8) {
                // each row n of W takes its scale from all of column n of M^-1: after a barrier,
                // the rows n = blockIdx.x, blockIdx.x + G, ..., one warp each
                epi_sync();
                gfail = false;
                if (et == 0) gfail = !lp_grid_sync(a.gbar, (unsigned)G * ++ep);
                if (epi_sync_or(gfail)) { set_status(a.status, CUR_ERR_TIMEOUT); break; }
                unsigned char* W8 = static_cast<unsigned char*>(a.W);
                for (int n = blockIdx.x + G * ew; n < r; n += G * kLpEpiWarps) {
                    float mx = 0.f;
                    for (int k = lane; k < r; k += 32) mx = fmaxf(mx, fabsf(__ldcg(a.Mh + k * r + n)));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    const float t = mx > 0.f && isfinite(mx) ? kE4M3Max / mx : 1.f;
                    for (int k = lane; k < a.ldk; k += 32)
                        W8[(int64_t)n * a.ldk + k] = k < r ? to_e4m3(__ldcg(a.Mh + k * r + n) * t) : (unsigned char)0;
                    if (lane == 0) a.winv[n] = 1.f / t;
                }
            }
            if (blockIdx.x == 0 && et == 0) {
                a.S[j] = i;
                a.ctl->logvol += log(fabs(bjv));
                a.ctl->swaps = swaps + 1;
            }
            ++swaps;
            if (swaps >= a.max_swaps) break;
            // W reaches the next iteration's TMA load through the grid barrier
            asm volatile("fence.proxy.async.global;" ::: "memory");
            epi_sync();
            gfail = false;
            if (et == 0) gfail = !lp_grid_sync(a.gbar, (unsigned)G * ++ep);
            if (epi_sync_or(gfail)) { set_status(a.status, CUR_ERR_TIMEOUT); break; }
            if (et == 0) s_go = (int)(it + 1);
        }
        if (et == 0) {
            s_quit = 1;
            if (blockIdx.x == 0) a.ctl->done = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tcols);
    }
}

// S_out = S0 after a singular start, else the set the loop reached (S_out may alias S0);
// *swaps = the swaps the loop took.
__global__ void lp_out_k(const LpCtl* ctl, const int32_t* S0, const int32_t* S, int32_t* S_out, int r,
                         int32_t* swaps) {
    const bool sing = ctl->status == CUR_ERR_SINGULAR;
    for (int k = threadIdx.x; k < r; k += blockDim.x) S_out[k] = sing ? S0[k] : S[k];
    if (threadIdx.x == 0) *swaps = ctl->swaps;
}

// swaps_out = {lp_swaps + exact swaps, lp_swaps} and the exact engine's status (lp_swaps
// NULL: no low-precision phase ran).
__global__ void lp_finish_dev_k(int32_t* swaps_out, const int32_t* lp_swaps, const MvDevResult* res, int* hstatus) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int lp = lp_swaps ? *lp_swaps : 0;
    if (swaps_out) {
        swaps_out[0] = lp + res->swaps;
        swaps_out[1] = lp;
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

// The low-precision phase alone (BF16, or E4M3 with fp8), from S0 to S_out (device r ints;
// may alias), enqueued: C rounded once, the start set up on the device, the whole swap loop in
// one cooperative launch, the result chosen on the device. C: p x r FP32 (contiguous,
// device), r a multiple of 16.
template <bool F8>
static cur_status lowprec_phase_t(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o,
                                  const int32_t* S0, int32_t* S_out, int32_t* swaps_dev, Arena& ar,
                                  cudaStream_t st, const double* minv_in, const int* minv_flag, const int* idle) {
    using namespace curk;
    const size_t mark = ar.off;
    constexpr int es = F8 ? 1 : 2, kEl = 128 / es;
    const int kc = (r + kEl - 1) / kEl, ldk = kc * kEl;
    // two accumulators of rpad = r rounded up to 32 columns; TMEM is allocated in powers of 2
    const int rpad = (r + 31) / 32 * 32;
    const int tcols = 2 * rpad <= 64 ? 64 : (2 * rpad <= 128 ? 128 : 256);
    const int64_t ntiles = (p + kLpBM - 1) / kLpBM;
    auto smem_of = [&](int ns) { return 1024 + (size_t)kc * r * 128 + (size_t)ns * kc * kLpChunkC; };
    const bool four = smem_of(4) <= (size_t)227 * 1024;   // TMA stages: 4 where they fit, else 2
    const int grid = (int)std::min<int64_t>(ntiles, h->num_sms);
    void* Cq = ar.take((size_t)p * ldk * es);
    void* W = ar.take((size_t)r * ldk * es);
    float* cinv = ar.get<float>(F8 ? (size_t)p : 1);
    float* winv = ar.get<float>((size_t)r);
    float* Mh = ar.get<float>((size_t)r * r);
    float* Ml = ar.get<float>((size_t)r * r);
    int32_t* S = ar.get<int32_t>(r);
    LpCand* cand = ar.get<LpCand>((size_t)grid);
    double* brow = ar.get<double>((size_t)r);
    LpCtl* ctl = ar.get<LpCtl>(1);
    unsigned* gbar = ar.get<unsigned>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUtensorMap mC, mW;
    if (!lp_map(&mC, Cq, p, ldk, kLpBM, es) || !lp_map(&mW, W, r, ldk, r, es)) return CUR_ERR_ARG;
    const unsigned qgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p * ldk + 255) / 256, 8LL * h->num_sms));
    if constexpr (F8)
        lp_quant_c8<<<qgrid, 256, 0, st>>>(C, p, r, ldk, static_cast<unsigned char*>(Cq), cinv);
    else
        lp_quant_c<<<qgrid, 256, 0, st>>>(C, p, r, ldk, static_cast<__nv_bfloat16*>(Cq));
    CUR_CK(cudaGetLastError());
    const size_t sm_setup = (size_t)r * r * sizeof(double) + (size_t)r * sizeof(double) + (size_t)r * sizeof(int) + 64;
    CUR_TRY(smem_attr((const void*)lp_setup_k<F8>, sm_setup));
    lp_setup_k<F8><<<1, 256, sm_setup, st>>>(C, r, ldk, S0, S, minv_in, minv_flag, idle, W, winv, Mh, Ml, ctl, gbar);
    CUR_CK(cudaGetLastError());
    LpLoop la{};
    la.p = p;
    la.r = r;
    la.kc = kc;
    la.ldk = ldk;
    la.tcols = tcols;
    la.cinv = cinv;
    la.winv = winv;
    la.C = C;
    la.Mh = Mh;
    la.Ml = Ml;
    la.W = W;
    la.S = S;
    la.ctl = ctl;
    la.cand = cand;
    la.brow = brow;
    la.gbar = gbar;
    la.delta = o->delta;
    la.max_swaps = o->max_swaps > 0 ? o->max_swaps : 100 * r;
    la.status = h->status;
    void* args[] = {&mC, &mW, &la};
    if (four) {
        CUR_TRY(smem_attr((const void*)lp_loop_k<F8, 4>, smem_of(4)));
        CUR_TRY(launch_coop((const void*)lp_loop_k<F8, 4>, dim3(grid), dim3(kLpThreadsWS), args, smem_of(4), st));
    } else {
        CUR_TRY(smem_attr((const void*)lp_loop_k<F8, 2>, smem_of(2)));
        CUR_TRY(launch_coop((const void*)lp_loop_k<F8, 2>, dim3(grid), dim3(kLpThreadsWS), args, smem_of(2), st));
    }
    lp_out_k<<<1, 128, 0, st>>>(ctl, S0, S, S_out, r, swaps_dev);
    CUR_CK(cudaGetLastError());
    note_launch(4);
    ar.off = mark;
    ar.ok = true;
    return CUR_OK;
}

cur_status lowprec_phase(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o, const int32_t* S0,
                         int32_t* S_out, int32_t* swaps_dev, Arena& ar, cudaStream_t st, const double* minv_in,
                         const int* minv_flag, const int* idle) {
    if (o->flags & CUR_FLAG_PREC_FP8)
        return lowprec_phase_t<true>(h, C, p, r, o, S0, S_out, swaps_dev, ar, st, minv_in, minv_flag, idle);
    return lowprec_phase_t<false>(h, C, p, r, o, S0, S_out, swaps_dev, ar, st, minv_in, minv_flag, idle);
}

bool lowprec_phase_applies(const cur_handle* h, const cur_opts* o, cur_dtype dt, int64_t p, int r) {
    return (o->flags & (CUR_FLAG_PREC_BF16 | CUR_FLAG_PREC_FP8)) && dt == CUR_F32 && r % 16 == 0 && r >= 16 && r <= 128 &&
           p >= (int64_t)kBf16MinTilesPerSm * curk::kLpBM * h->num_sms && p <= INT_MAX - 256;
}

// The low-precision phase, then the exact engine from the set it reached (after a singular
// start the exact engine meets the same singular C(S0,:) and reports it).
static cur_status maxvol_global_bf16(cur_handle* h, const float* C, int64_t p, int r, const cur_opts* o,
                                     const int32_t* S0, int32_t* S_out, double* logvol_out, int32_t* swaps_out,
                                     Arena& ar, cudaStream_t st) {
    using namespace curk;
    int32_t* lp_swaps = ar.get<int32_t>(1);
    MvDevResult* res = ar.get<MvDevResult>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(lowprec_phase(h, C, p, r, o, S0, S_out, lp_swaps, ar, st, nullptr, nullptr, nullptr));
    CUR_TRY(maxvol_global(h, CUR_F32, C, p, r, o, S_out, S_out, logvol_out, res, ar, st));
    lp_finish_dev_k<<<1, 32, 0, st>>>(swaps_out, lp_swaps, res, h->status);
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
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_TRY(maxvol_global(h, basis->dtype, basis->data, p, r, &o, S0, S_out, logvol_out, res, ar, st));
    curk::lp_finish_dev_k<<<1, 32, 0, st>>>(swaps_out, nullptr, res, h->status);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

}  // extern "C"
