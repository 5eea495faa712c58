// Residual of the cross on the tensor cores (tcgen05, sm_103a): max|A - C W| and
// sum (A - C W)^2, sum A^2 with W = U R, for FP32 data and r = 32 or 64 (whole
// 128-byte swizzle rows); other shapes use the CUDA-core kernel of residual.cu.
//
// The product D = C W (m x n, K = r) runs as 3xTF32 on tcgen05.mma (kind::tf32):
// C = Ch + Cl and W = Wh + Wl with Ch, Wh rounded to TF32 and Cl, Wl the rounded
// remainders; D = Ch Wh + Cl Wh + Ch Wl keeps ~22 bits, i.e. FP32-level accuracy
// (the dropped Cl Wl term is ~2^-22 relative). Tile by tile (M = 128 rows of A,
// N = 128 columns, K = r) the C panel is the MMA's A operand, read from tensor memory,
// and the tile's W^T the B operand, read from shared memory; a TMEM lane is a row of A.
//
// Per CTA (persistent, one per SM, 608 threads; its tiles run along row panels):
//   TMEM         two accumulators (128 columns each) and two C panels (hi in 64
//                columns, lo in the next 64): the next panel is split and stored while
//                the current one is in use
//   warp 0       TMA producer of W^T (128 columns of A x r, hi and lo, 128-byte swizzle,
//                K-major) into two stages, so the next tile's W loads during this one's MMAs
//   warp 1       MMA issuer (one thread): 3 passes x r/8 MMAs per tile into one of the
//                two accumulators
//   warp 18      TMA producer of A: 32-row x 128-column sub-tiles (16 KB, four 32 x 32
//                boxes with 128-byte swizzle) into a ring of up to 10 slots; A is read
//                from HBM exactly once
//   warps 2..17  epilogue: warp (lane quarter q, column group g) reads its 32 rows x 32
//                accumulator columns with tcgen05.ld and the same block of A from shared
//                memory (16-byte loads, conflict-free through the swizzle), and folds
//                max|E|, sum E^2, sum A^2; the same warps split C rows into TF32 hi and
//                lo and store them into TMEM with tcgen05.st when a panel begins
// Out-of-range rows and columns read as zeros from every operand (TMA fill; zero C rows),
// so E = 0 there and no element needs a mask.
// Waits are bounded; on a timeout the CTA records CUR_ERR_TIMEOUT, waits (bounded) for
// the copies and MMAs it issued, frees its TMEM and returns.

#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstring>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"
#include "tc.cuh"

namespace curk {

constexpr int kTcBM = 128;            // rows of A per tile (MMA M, TMEM lanes)
constexpr int kTcBN = 128;            // columns of A per tile (MMA N)
constexpr int kChunk = 16384;         // one 128-row x 32-element FP32 swizzled chunk of W^T

// Wt[j][k] = (U R)(k, j) = sum_l U(k, l) R(l, j), split into TF32 hi and lo, rows padded
// to ldk. A block (256 threads) takes 2 * (256 / ceil(r/4)) columns j and every k: U (as
// double-float, l-major) and the block's columns of R are staged in shared memory, and
// each thread sums 4 k x 2 j entries over l in double-float (eight independent chains on
// the FP32 pipes, ~48-bit accuracy).
__host__ __device__ constexpr int prep_w_cols(int r) { return 2 * (256 / ((r + 3) / 4)); }
__host__ __device__ constexpr size_t prep_w_smem(int r) {
    return (size_t)r * (4 * ((r + 3) / 4)) * sizeof(df64) + (size_t)r * prep_w_cols(r) * sizeof(float);
}
template <typename TA>
__global__ void __launch_bounds__(256) tc_prep_w(const double* __restrict__ U, const TA* __restrict__ R,
                                                 int r, int64_t n, int ldk, float* __restrict__ Wh,
                                                 float* __restrict__ Wl) {
    extern __shared__ __align__(16) unsigned char prep_raw[];
    const int kgn = (r + 3) >> 2, kp = 4 * kgn, jt = prep_w_cols(r);
    df64* Us = reinterpret_cast<df64*>(prep_raw);                      // Us[l * kp + k] = U(k, l)
    float* Rs = reinterpret_cast<float*>(Us + (size_t)r * kp);          // Rs[l * jt + jj] = R(l, j0 + jj)
    const int64_t j0 = (int64_t)blockIdx.x * jt;
    for (int e = threadIdx.x; e < r * kp; e += blockDim.x) {
        const int l = e / kp, k = e - l * kp;
        Us[e] = k < r ? df_from_d(U[(int64_t)k * r + l]) : df64{0.f, 0.f};
    }
    for (int e = threadIdx.x; e < r * jt; e += blockDim.x) {
        const int l = e / jt, jj = e - l * jt;
        Rs[e] = j0 + jj < n ? to_f(R[(int64_t)l * n + j0 + jj]) : 0.f;
    }
    __syncthreads();
    const int kg = threadIdx.x % kgn, jg = threadIdx.x / kgn;
    if (2 * jg >= jt) return;
    df64 acc[2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[0][i] = acc[1][i] = df64{0.f, 0.f};
    for (int l = 0; l < r; ++l) {
        const df64* ul = Us + l * kp + 4 * kg;
        const float r0 = Rs[l * jt + 2 * jg], r1 = Rs[l * jt + 2 * jg + 1];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const df64 u = ul[i];
            acc[0][i] = df_add(acc[0][i], df_mul_f(u, r0));
            acc[1][i] = df_add(acc[1][i], df_mul_f(u, r1));
        }
    }
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
        const int64_t j = j0 + 2 * jg + jj;
        if (j >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = 4 * kg + i;
            if (k >= ldk) continue;
            float hi = 0.f, lo = 0.f;
            if (k < r) {
                const df64 w = acc[jj][i];
                hi = to_tf32(__fadd_rn(w.h, w.l));
                const df64 rem = df_sub(w, df64{hi, 0.f});
                lo = to_tf32(__fadd_rn(rem.h, rem.l));
            }
            Wh[j * ldk + k] = hi;
            Wl[j * ldk + k] = lo;
        }
    }
}

constexpr int kAR = 32;                     // rows of A per staged sub-tile (one lane quarter)
constexpr int kABox = kAR * 32 * 4;         // 4 KB: 32 rows x 32 columns FP32, 128-byte swizzle
constexpr int kASub = 4 * kABox;            // 16 KB: 32 rows x 128 columns
constexpr int kNAMax = 10;                  // A ring slots at most
constexpr int kEpiWarps = 16;               // epilogue: 4 lane quarters x 4 column groups
constexpr int kTmemCols = 512;              // accumulators at 0 and 128, C panels at 256 and 384
constexpr int kCLo = 64;                    // TMEM column offset of a panel's lo words

struct TcArgs {
    int64_t m, n;
    const float* C;   // m x r, row-major
    int r, nch, ksteps, na;
    int64_t ntile_n, ntiles;
    double* part;   // 4 doubles per CTA
    int* status;
};

// 8 consecutive TMEM columns of this thread's lane (32x32b shape); no wait.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                    "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                    "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// D (+)= A B with A (M x K, K-major) in tensor memory and B described in shared memory.
__device__ __forceinline__ void mma_tf32_ts(uint32_t dtmem, uint32_t atmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p; }"
                 :: "r"(dtmem), "r"(atmem), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

// One epilogue warp's share of a C panel: its lane quarter's 32 rows, K columns
// [kq, kq + r/4), split into TF32 hi (TMEM column cbase + k) and lo (cbase + kCLo + k).
// Rows past m are zeros. Ends with the stores complete and fenced for the MMA thread.
__device__ __forceinline__ void store_c_panel(const TcArgs& a, int64_t panel, uint32_t trow, uint32_t cbase,
                                              int q, int g, int lane) {
    const int64_t row = panel * kTcBM + 32 * q + lane;
    const bool rv = row < a.m;
    const int kw = a.r >> 2;   // 8 or 16 columns per warp
    const float* src = a.C + (rv ? row : 0) * a.r;
    for (int k0 = g * kw; k0 < (g + 1) * kw; k0 += 8) {
        float hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float c = rv ? __ldg(src + k0 + i) : 0.f;
            hi[i] = to_tf32(c);
            lo[i] = to_tf32(c - hi[i]);
        }
        tmem_st8(trow + cbase + (uint32_t)k0, hi);
        tmem_st8(trow + cbase + (uint32_t)(kCLo + k0), lo);
    }
    tmem_wait_st();
    tc_fence_before();
}

__global__ void __launch_bounds__(608, 1) residual_tc_k(const __grid_constant__ CUtensorMap mWh,
                                                        const __grid_constant__ CUtensorMap mWl,
                                                        const __grid_constant__ CUtensorMap mA,
                                                        TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nch = a.nch, na = a.na;
    const uint32_t half_bytes = (uint32_t)nch * kChunk;   // W^T hi (or lo) of one tile
    unsigned char* WB = sm;                     // 2 stages x (hi, lo)
    unsigned char* AS = WB + 4 * (size_t)half_bytes;   // ring of na A sub-tiles
    __shared__ __align__(8) uint64_t wfull[2], wempty[2], cfull[2], accf[2], acce[2], af[kNAMax], ae[kNAMax];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ double rmx[kEpiWarps], rse[kEpiWarps], rsa[kEpiWarps];
    __shared__ int rbad[kEpiWarps];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t G = gridDim.x;
    const int64_t t0 = a.ntiles * blockIdx.x / G, t1 = a.ntiles * (blockIdx.x + 1) / G;

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&wfull[s], 1);
            mbar_init(&wempty[s], 1);
            mbar_init(&cfull[s], kEpiWarps);
            mbar_init(&accf[s], 1);
            mbar_init(&acce[s], kEpiWarps);
        }
        for (int s = 0; s < na; ++s) {
            mbar_init(&af[s], 1);
            mbar_init(&ae[s], 4);   // the four column-group warps of one lane quarter
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // ------------------------------------------------------------ W^T producer
        if (lane == 0) {
            int64_t nw = 0;   // tiles whose W was issued
            bool ok = true;
            for (int64_t t = t0; t < t1 && !abort_flag; ++t, ++nw) {
                const int64_t ct = t % a.ntile_n;
                const int s = (int)(nw & 1);
                const int64_t u = nw >> 1;
                if (u > 0 && !mbar_wait(&wempty[s], (uint32_t)((u - 1) & 1))) { ok = false; break; }
                unsigned char* dst = WB + (size_t)s * 2 * half_bytes;
                mbar_expect_tx(&wfull[s], 2 * half_bytes);
                for (int c = 0; c < nch; ++c) {
                    tma_load_2d(dst + c * kChunk, &mWh, &wfull[s], 32 * c, (int)(ct * kTcBN));
                    tma_load_2d(dst + half_bytes + c * kChunk, &mWl, &wfull[s], 32 * c, (int)(ct * kTcBN));
                }
            }
            if (!ok) { abort_flag = 1; set_status(a.status, CUR_ERR_TIMEOUT); }
            // after an abort, wait (bounded) for the last copy into each stage: the MMA
            // warp consumed every full barrier otherwise
            if (abort_flag)
                for (int64_t q = nw - 1; q >= 0 && q >= nw - 2; --q) mbar_wait(&wfull[q & 1], (uint32_t)((q >> 1) & 1));
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(kTcBM, kTcBN);
            int64_t cur_panel = -1, pc = -1, it = 0;
            bool ok = true;
            uint64_t* last_bar = nullptr;   // the barrier of the last commit and its phase
            uint32_t last_par = 0;
            for (int64_t t = t0; t < t1 && !abort_flag; ++t, ++it) {
                const int64_t panel = t / a.ntile_n;
                if (panel != cur_panel) {
                    ++pc;
                    cur_panel = panel;
                    if (!mbar_wait(&cfull[pc & 1], (uint32_t)((pc >> 1) & 1))) { ok = false; break; }
                }
                const int b = (int)(it & 1);
                const int64_t u = it >> 1;
                if (u > 0 && !mbar_wait(&acce[b], (uint32_t)((u - 1) & 1))) { ok = false; break; }
                if (!mbar_wait(&wfull[b], (uint32_t)(u & 1))) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kTcBN);
                const uint32_t cpan = tmem + 256u + (uint32_t)((pc & 1) * 128);
                const uint32_t wh = su32(WB + (size_t)b * 2 * half_bytes), wl = wh + half_bytes;
                // Ch Wh, Cl Wh, Ch Wl
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t aop = cpan + (pass == 1 ? (uint32_t)kCLo : 0u);
                    const uint32_t bop = pass == 2 ? wl : wh;
                    for (int k = 0; k < a.ksteps; ++k) {
                        const uint32_t off = (uint32_t)((k >> 2) * kChunk + (k & 3) * 32);
                        mma_tf32_ts(d, aop + (uint32_t)(8 * k), sdesc_k128(bop + off), idesc, (pass | k) != 0);
                    }
                }
                mma_commit(&wempty[b]);
                mma_commit(&accf[b]);
                last_bar = &accf[b];
                last_par = (uint32_t)(u & 1);
            }
            if (!ok) { abort_flag = 1; set_status(a.status, CUR_ERR_TIMEOUT); }
            // every MMA issued has finished once the last commit has arrived
            if (last_bar) mbar_wait(last_bar, last_par);
        }
    } else if (warp == 2 + kEpiWarps) {
        // ------------------------------------------------------------ A producer
        if (lane == 0) {
            int64_t idx = 0;
            bool ok = true;
            for (int64_t t = t0; t < t1 && ok && !abort_flag; ++t) {
                const int64_t panel = t / a.ntile_n, ct = t - panel * a.ntile_n;
                for (int k = 0; k < kTcBM / kAR; ++k, ++idx) {
                    const int slot = (int)(idx % na);
                    const int64_t use = idx / na;
                    if (use > 0 && !mbar_wait(&ae[slot], (uint32_t)((use - 1) & 1))) { ok = false; break; }
                    mbar_expect_tx(&af[slot], (uint32_t)kASub);
                    for (int g = 0; g < 4; ++g)
                        tma_load_2d(AS + (size_t)slot * kASub + g * kABox, &mA, &af[slot],
                                    (int)(ct * kTcBN + 32 * g), (int)(panel * kTcBM + kAR * k));
                }
            }
            if (!ok) { abort_flag = 1; set_status(a.status, CUR_ERR_TIMEOUT); }
            if (abort_flag)
                for (int64_t q = idx - 1; q >= 0 && q >= idx - na; --q)
                    mbar_wait(&af[q % na], (uint32_t)((q / na) & 1));
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..17)
        const int q = warp & 3;              // TMEM lane quarter of this warp = rows 32 q .. 32 q + 31
        const int g = (warp - 2) >> 2;       // column group: columns 32 g .. 32 g + 31 of the tile
        const int ew = warp - 2;
        const uint32_t trow = (uint32_t)(32 * q) << 16;
        float mx = 0.f;
        double se = 0.0, sa = 0.0;
        int bad = 0;
        if (t0 < t1) {
            // the first two panels; later ones are stored when the panel before them begins
            const int64_t p0 = t0 / a.ntile_n, plast = (t1 - 1) / a.ntile_n;
            store_c_panel(a, p0, trow, 256u, q, g, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&cfull[0]);
            if (plast > p0) {
                store_c_panel(a, p0 + 1, trow, 384u, q, g, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(&cfull[1]);
            }
        }
        int64_t it = 0, cur_panel = -1, pc = -1;
        const int64_t plast = t1 > t0 ? (t1 - 1) / a.ntile_n : -1;
        for (int64_t t = t0; t < t1; ++t, ++it) {
            const int64_t panel = t / a.ntile_n;
            const bool fresh = panel != cur_panel;
            if (fresh) { ++pc; cur_panel = panel; }
            const int b = (int)(it & 1);
            if (!mbar_wait(&accf[b], (uint32_t)((it >> 1) & 1))) {
                abort_flag = 1;
                set_status(a.status, CUR_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            if (fresh && pc >= 1 && panel + 1 <= plast) {
                // every MMA of the panel before this one has completed (this tile's commit
                // follows them), so its TMEM columns take the panel after this one
                store_c_panel(a, panel + 1, trow, 256u + (uint32_t)(((pc + 1) & 1) * 128), q, g, lane);
                __syncwarp();
                if (lane == 0) mbar_arrive(&cfull[(pc + 1) & 1]);
            }
            const int64_t idx = 4 * it + q;
            const int slot = (int)(idx % na);
            if (!mbar_wait(&af[slot], (uint32_t)((idx / na) & 1))) {
                abort_flag = 1;
                set_status(a.status, CUR_ERR_TIMEOUT);
                break;
            }
            __syncwarp();
            // the 32 x 32 block: accumulator columns b*128 + 32 g .. + 31 of this warp's
            // lanes, and row `lane` of A box g (16-byte chunk c stored at c ^ (lane & 7))
            float dall[32];
            tmem_ld32(tmem + trow + (uint32_t)(b * kTcBN + 32 * g), dall);
            const unsigned char* arow = AS + (size_t)slot * kASub + g * kABox + lane * 128;
            // four independent chains per sum; a NaN anywhere makes the group's sum of
            // squares NaN (fmaxf alone would drop it)
            float m4[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f}, a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 x4 = *reinterpret_cast<const float4*>(arow + ((c ^ (lane & 7)) << 4));
                const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float e = xs[i] - dall[4 * c + i];
                    m4[i] = fmaxf(m4[i], fabsf(e));
                    s4[i] = fmaf(e, e, s4[i]);
                    a4[i] = fmaf(xs[i], xs[i], a4[i]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ae[slot]);
            const float gs = (s4[0] + s4[1]) + (s4[2] + s4[3]);
            if (gs != gs) bad = 1;
            mx = fmaxf(mx, fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3])));
            se += (double)gs;
            sa += (double)((a4[0] + a4[1]) + (a4[2] + a4[3]));
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
            if (abort_flag) break;
        }
        // reduce over the epilogue threads
        double dmx = mx;
        for (int o = 16; o > 0; o >>= 1) {
            dmx = fmax(dmx, __shfl_xor_sync(0xffffffffu, dmx, o));
            se += __shfl_xor_sync(0xffffffffu, se, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (lane == 0) { rmx[ew] = dmx; rse[ew] = se; rsa[ew] = sa; rbad[ew] = bad; }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        double m1 = 0.0, m2 = 0.0, m3 = 0.0;
        int bd = 0;
        for (int w = 0; w < kEpiWarps; ++w) { m1 = fmax(m1, rmx[w]); m2 += rse[w]; m3 += rsa[w]; bd |= rbad[w]; }
        a.part[blockIdx.x * 4 + 0] = m1;
        a.part[blockIdx.x * 4 + 1] = m2;
        a.part[blockIdx.x * 4 + 2] = m3;
        a.part[blockIdx.x * 4 + 3] = bd ? 1.0 : 0.0;
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Combines the per-CTA partials (same as the SIMT path's final step).
__global__ void tc_final_k(const double* part, int64_t nparts, double* cheb, double* fro, int* status,
                           double* sums) {
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

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// A (m x n FP32, leading dimension ld), boxes of 32 columns x 32 rows with 128-byte
// swizzle: in a staged box, row i's 16-byte chunk c sits at chunk c ^ (i & 7) of its
// 128-byte row. Needs a 16-byte aligned base and ld % 4 == 0.
static bool make_map_a(CUtensorMap* map, const float* base, int64_t m, int64_t n, int64_t ld) {
    auto enc = encode_fn();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld & 3) != 0) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t gstr[1] = {(cuuint64_t)ld * sizeof(float)};
    cuuint32_t box[2] = {32, (cuuint32_t)kAR};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// rows x ldk FP32, boxes of 32 elements x 128 rows, 128-byte swizzle.
static bool make_map(CUtensorMap* map, const float* base, int64_t rows, int r, int ldk) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)r, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)ldk * sizeof(float)};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace curk

// Returns CUR_ERR_ARG when this path does not apply (the caller then uses the SIMT path).
cur_status residual_tc_impl(cur_handle* h, const cur_mat* Am, const void* C, const double* U,
                            const void* R, int r, double* cheb, double* fro, Arena& ar,
                            cudaStream_t st, double* sums) {
    using namespace curk;
    if (Am->dtype != CUR_F32 || (r != 32 && r != 64)) return CUR_ERR_ARG;
    const int64_t m = Am->rows, n = Am->cols;
    if ((m + kTcBM - 1) / kTcBM > INT_MAX / kTcBM || (n + kTcBN - 1) / kTcBN > INT_MAX / kTcBN) return CUR_ERR_ARG;
    const int ldk = (r + 3) / 4 * 4;           // 16-byte row pitch for the tensor maps
    const int nch = (r + 31) / 32;
    float* Wh = ar.get<float>((size_t)n * ldk);
    float* Wl = ar.get<float>((size_t)n * ldk);
    const int G = h->num_sms;
    double* part = ar.get<double>((size_t)G * 4);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUtensorMap mWh, mWl, mA;
    if (!make_map_a(&mA, static_cast<const float*>(Am->data), m, n, Am->ld)) return CUR_ERR_ARG;
    if (!make_map(&mWh, Wh, n, r, ldk) || !make_map(&mWl, Wl, n, r, ldk)) return CUR_ERR_ARG;
    const size_t smw = prep_w_smem(r);
    CUR_TRY(smem_attr((const void*)tc_prep_w<float>, smw));
    tc_prep_w<float><<<(unsigned)((n + prep_w_cols(r) - 1) / prep_w_cols(r)), 256, smw, st>>>(
        U, static_cast<const float*>(R), r, n, ldk, Wh, Wl);
    CUR_CK(cudaGetLastError());
    note_launch();
    TcArgs a{};
    a.m = m;
    a.n = n;
    a.C = static_cast<const float*>(C);
    a.r = r;
    a.nch = nch;
    a.ksteps = (r + 7) / 8;
    a.ntile_n = (n + kTcBN - 1) / kTcBN;
    a.ntiles = ((m + kTcBM - 1) / kTcBM) * a.ntile_n;
    a.part = part;
    a.status = h->status;
    const int grid = (int)std::min<int64_t>(G, a.ntiles);
    // two stages of the W^T tile (hi and lo each), then as many 16 KB A slots as fit
    const size_t fixed = (size_t)4 * nch * kChunk + 1024;
    const size_t budget = 225 * 1024;
    a.na = (int)std::min<size_t>(kNAMax, (budget - fixed) / kASub);
    if (a.na < 4) return CUR_ERR_ARG;
    const size_t sm = fixed + (size_t)a.na * kASub;
    CUR_TRY(smem_attr((const void*)residual_tc_k, sm));
    residual_tc_k<<<grid, 32 * (3 + kEpiWarps), sm, st>>>(mWh, mWl, mA, a);
    CUR_CK(cudaGetLastError());
    note_launch();
    tc_final_k<<<1, 256, 0, st>>>(part, grid, cheb, fro, h->status, sums);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}
