// Residual of the cross on the tensor cores (tcgen05, sm_103a): max|A - C W| and
// sum (A - C W)^2, sum A^2 with W = U R, for FP32 data and r = 32 or 64 (whole
// 128-byte swizzle rows); other shapes use the CUDA-core kernel of residual.cu.
//
// The product D = C W (m x n, K = r) runs as 3xTF32 on tcgen05.mma (kind::tf32):
// C = Ch + Cl and W = Wh + Wl with Ch, Wh rounded to TF32 and Cl, Wl the rounded
// remainders; D = Ch Wh + Ch Wl + Cl Wh keeps ~22 bits, i.e. FP32-level accuracy
// (the dropped Cl Wl term is ~2^-22 relative). The MMA computes D^T tile by tile
// (M = 128 columns of A, N = 128 rows, K = r) so that a TMEM lane is a column of A.
//
// Per CTA (persistent, one per SM, 608 threads):
//   warp 0       TMA producer: the C panel (128 rows x r, hi and lo, resident while
//                the CTA stays on the panel) and the tile's W^T (128 x r) as two
//                buffers, hi (released after MMA passes 0 and 1) and lo (after pass 2),
//                128-byte swizzled, K-major
//   warp 1       MMA issuer (one thread): 3 passes x r/8 MMAs per tile into one of two
//                TMEM accumulators (128 lanes x 128 FP32 columns each)
//   warp 18      TMA producer of A: 32-row x 128-column sub-tiles (16 KB, unswizzled)
//                into a ring of up to 8 slots (6 for r = 64), so A stays in flight
//                while earlier ones are folded; A is read from HBM exactly once
//   warps 2..17  epilogue: warp (sub-tile k, column quarter q) reads its 32 accumulator
//                columns with tcgen05.ld, its column of the staged A rows from shared
//                memory (conflict-free), and folds max|E|, sum E^2, sum A^2 with
//                independent chains
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

constexpr int kTcBM = 128;            // rows of A per tile (MMA N)
constexpr int kTcBN = 128;            // columns of A per tile (MMA M)
constexpr int kChunk = 16384;         // one 128-row x 32-element FP32 swizzled chunk

// Wt[j][k] = (U R)(k, j), split into TF32 hi and lo, rows padded to ldk. One thread per
// entry (k fastest, so the stores are coalesced); the r-term sum runs in double-float
// (U converted once per CTA), i.e. on the FP32 pipes with ~48-bit accuracy.
template <typename TA>
__global__ void __launch_bounds__(256) tc_prep_w(const double* __restrict__ U, const TA* __restrict__ R,
                                                 int r, int64_t n, int ldk, float* __restrict__ Wh,
                                                 float* __restrict__ Wl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    df64* Ut = reinterpret_cast<df64*>(smem_raw);   // U^T: lanes with consecutive k read consecutive words
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int k = e / r, l = e - k * r;
        Ut[l * r + k] = df_from_d(U[e]);
    }
    __syncthreads();
    const int64_t total = n * ldk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / ldk;
        const int k = (int)(e - j * ldk);
        float hi = 0.f, lo = 0.f;
        if (k < r) {
            df64 s0{0.f, 0.f}, s1{0.f, 0.f};
            int l = 0;
            for (; l + 1 < r; l += 2) {
                s0 = df_add(s0, df_mul_f(Ut[l * r + k], to_f(R[(int64_t)l * n + j])));
                s1 = df_add(s1, df_mul_f(Ut[(l + 1) * r + k], to_f(R[(int64_t)(l + 1) * n + j])));
            }
            if (l < r) s0 = df_add(s0, df_mul_f(Ut[l * r + k], to_f(R[(int64_t)l * n + j])));
            const df64 w = df_add(s0, s1);
            hi = to_tf32(__fadd_rn(w.h, w.l));
            const df64 rem = df_sub(w, df64{hi, 0.f});
            lo = to_tf32(__fadd_rn(rem.h, rem.l));
        }
        Wh[e] = hi;
        Wl[e] = lo;
    }
}

// Ch/Cl (m x ldk): C split into TF32 hi and lo, rows padded to ldk.
template <typename TA>
__global__ void tc_prep_c(const TA* __restrict__ C, int64_t m, int r, int ldk, float* __restrict__ Ch,
                          float* __restrict__ Cl) {
    const int64_t total = m * ldk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldk;
        const int k = (int)(e - i * ldk);
        float hi = 0.f, lo = 0.f;
        if (k < r) {
            const float c = to_f(C[i * r + k]);
            hi = to_tf32(c);
            lo = to_tf32(c - hi);
        }
        Ch[e] = hi;
        Cl[e] = lo;
    }
}

constexpr int kAR = 32;                     // rows of A per staged sub-tile
constexpr int kASub = kAR * kTcBN * 4;      // 16 KB: 32 rows x 128 columns, FP32
constexpr int kNAMax = 8;                   // A ring slots at most
constexpr int kEpiWarps = 16;               // epilogue: 4 row sub-tiles x 4 column quarters

struct TcArgs {
    int64_t m, n;
    int r, nch, ksteps, na;
    int64_t ntile_n, ntiles;
    double* part;   // 4 doubles per CTA
    int* status;
};

__global__ void __launch_bounds__(608, 1) residual_tc_k(const __grid_constant__ CUtensorMap mWh,
                                                        const __grid_constant__ CUtensorMap mWl,
                                                        const __grid_constant__ CUtensorMap mCh,
                                                        const __grid_constant__ CUtensorMap mCl,
                                                        const __grid_constant__ CUtensorMap mA,
                                                        TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nch = a.nch, na = a.na;
    unsigned char* CH = sm;                     // C panel, TF32 hi (resident per row panel)
    unsigned char* CL = CH + nch * kChunk;      // C panel, TF32 lo
    unsigned char* WH = CL + nch * kChunk;      // W^T tile, hi (released after MMA passes 0, 1)
    unsigned char* WL = WH + nch * kChunk;      // W^T tile, lo (released after pass 2)
    unsigned char* AS = WL + nch * kChunk;      // ring of na A sub-tiles (32 x 128 FP32)
    __shared__ __align__(8) uint64_t whf, whe, wlf, wle, cfull, cempty, accf[2], acce[2], af[kNAMax],
        ae[kNAMax];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ double rmx[kEpiWarps], rse[kEpiWarps], rsa[kEpiWarps];
    __shared__ int rbad[kEpiWarps];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t G = gridDim.x;
    const int64_t t0 = a.ntiles * blockIdx.x / G, t1 = a.ntiles * (blockIdx.x + 1) / G;
    const uint32_t half_bytes = (uint32_t)nch * kChunk;

    if (tid == 0) {
        mbar_init(&whf, 1);
        mbar_init(&whe, 1);
        mbar_init(&wlf, 1);
        mbar_init(&wle, 1);
        mbar_init(&cfull, 1);
        mbar_init(&cempty, 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&accf[s], 1);
            mbar_init(&acce[s], kEpiWarps);
        }
        for (int s = 0; s < na; ++s) {
            mbar_init(&af[s], 1);
            mbar_init(&ae[s], 4);   // the four column-quarter warps of one row sub-tile
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tslot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // ------------------------------------------------------------ C panel and W^T producer
        if (lane == 0) {
            int64_t cur_panel = -1, it = 0, nwh = 0, nwl = 0;   // tiles, hi and lo loads issued
            int cuse = 0;
            bool ok = true;
            for (int64_t t = t0; t < t1 && ok && !abort_flag; ++t, ++it) {
                const int64_t panel = t / a.ntile_n, ct = t - panel * a.ntile_n;
                if (panel != cur_panel) {
                    if (cuse > 0 && !mbar_wait(&cempty, (cuse - 1) & 1)) { ok = false; break; }
                    mbar_expect_tx(&cfull, 2 * half_bytes);
                    for (int c = 0; c < nch; ++c) {
                        tma_load_2d(CH + c * kChunk, &mCh, &cfull, 32 * c, (int)(panel * kTcBM));
                        tma_load_2d(CL + c * kChunk, &mCl, &cfull, 32 * c, (int)(panel * kTcBM));
                    }
                    ++cuse;
                    cur_panel = panel;
                }
                // hi, then lo, in the order the MMAs free them
                for (int part = 0; part < 2; ++part) {
                    uint64_t* fb = part ? &wlf : &whf;
                    uint64_t* eb = part ? &wle : &whe;
                    if (it > 0 && !mbar_wait(eb, (uint32_t)((it - 1) & 1))) { ok = false; break; }
                    mbar_expect_tx(fb, half_bytes);
                    for (int c = 0; c < nch; ++c)
                        tma_load_2d((part ? WL : WH) + c * kChunk, part ? &mWl : &mWh, fb, 32 * c, (int)(ct * kTcBN));
                    ++(part ? nwl : nwh);
                }
            }
            if (!ok) { abort_flag = 1; set_status(a.status, CUR_ERR_TIMEOUT); }
            // after an abort, wait (bounded) for the last copy into each buffer: the MMA
            // warp consumed every full barrier otherwise
            if (abort_flag) {
                if (nwh > 0) mbar_wait(&whf, (uint32_t)((nwh - 1) & 1));
                if (nwl > 0) mbar_wait(&wlf, (uint32_t)((nwl - 1) & 1));
                if (cuse > 0) mbar_wait(&cfull, (uint32_t)((cuse - 1) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32(kTcBN, kTcBM);
            int64_t cur_panel = -1, it = 0;
            int cuse = 0;
            bool ok = true;
            const uint32_t ch = su32(CH), cl = su32(CL), wh = su32(WH), wl = su32(WL);
            uint64_t* last_bar = nullptr;   // the barrier of the last commit and its phase
            uint32_t last_par = 0;
            for (int64_t t = t0; t < t1 && !abort_flag; ++t, ++it) {
                const int64_t panel = t / a.ntile_n;
                if (panel != cur_panel) {
                    if (cuse > 0) mma_commit(&cempty);
                    if (!mbar_wait(&cfull, cuse & 1)) { ok = false; break; }
                    ++cuse;
                    cur_panel = panel;
                }
                const int b = (int)(it & 1);
                const int64_t u = it >> 1;
                if (u > 0 && !mbar_wait(&acce[b], (uint32_t)((u - 1) & 1))) { ok = false; break; }
                const uint32_t d = tmem + (uint32_t)(b * kTcBM);
                bool fine = true;
                // passes 0 and 1 (Wh Ch, Wh Cl) release the hi buffer; pass 2 (Wl Ch) the lo
                for (int part = 0; part < 2; ++part) {
                    uint64_t* fb = part ? &wlf : &whf;
                    uint64_t* eb = part ? &wle : &whe;
                    if (!mbar_wait(fb, (uint32_t)(it & 1))) { fine = false; break; }
                    tc_fence_after();
                    const uint32_t wop = part ? wl : wh;
                    for (int pass = part ? 2 : 0; pass < (part ? 3 : 2); ++pass) {
                        const uint32_t bop = pass == 1 ? cl : ch;
                        for (int k = 0; k < a.ksteps; ++k) {
                            const uint32_t off = (uint32_t)((k >> 2) * kChunk + (k & 3) * 32);
                            mma_tf32(d, sdesc_k128(wop + off), sdesc_k128(bop + off), idesc, (pass | k) != 0);
                        }
                    }
                    mma_commit(eb);
                    last_bar = eb;
                    last_par = (uint32_t)(it & 1);
                }
                if (!fine) { ok = false; break; }
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
                    tma_load_2d(AS + (size_t)slot * kASub, &mA, &af[slot], (int)(ct * kTcBN),
                                (int)(panel * kTcBM + kAR * k));
                }
            }
            if (!ok) { abort_flag = 1; set_status(a.status, CUR_ERR_TIMEOUT); }
            if (abort_flag)
                for (int64_t q = idx - 1; q >= 0 && q >= idx - na; --q)
                    mbar_wait(&af[q % na], (uint32_t)((q / na) & 1));
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..17)
        const int q = warp & 3;              // TMEM lane quarter of this warp = column quarter
        const int k = (warp - 2) >> 2;       // row sub-tile: rows 32 k .. 32 k + 31 of the tile
        const int jl = 32 * q + lane;        // column within the tile = TMEM lane
        const int ew = warp - 2;
        float mx = 0.f;
        double se = 0.0, sa = 0.0;
        int bad = 0;
        int64_t it = 0;
        for (int64_t t = t0; t < t1; ++t, ++it) {
            const int64_t panel = t / a.ntile_n, ct = t - panel * a.ntile_n;
            const int64_t j = ct * kTcBN + jl;
            const int64_t rbase = panel * kTcBM + kAR * k;
            const bool jv = j < a.n;
            const bool full = jv && rbase + kAR <= a.m;   // every row of the sub-tile exists
            const int b = (int)(it & 1);
            if (!mbar_wait(&accf[b], (uint32_t)((it >> 1) & 1))) {
                abort_flag = 1;
                set_status(a.status, CUR_ERR_TIMEOUT);
                break;
            }
            const int64_t idx = 4 * it + k;
            const int slot = (int)(idx % na);
            if (!mbar_wait(&af[slot], (uint32_t)((idx / na) & 1))) {
                abort_flag = 1;
                set_status(a.status, CUR_ERR_TIMEOUT);
                break;
            }
            __syncwarp();
            tc_fence_after();
            const float* As = reinterpret_cast<const float*>(AS + (size_t)slot * kASub) + jl;
            float tse = 0.f, tsa = 0.f;
            // the sub-tile's 32 accumulator columns in one TMEM load (one wait)
            float dall[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTcBM + kAR * k), dall);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float* dv = dall + 16 * c;
                if (full) {
                    // four independent chains per sum; a NaN anywhere makes the group's
                    // sum of squares NaN (fmaxf alone would drop it)
                    float m4[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f},
                          a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float x = As[(16 * c + i) * kTcBN];
                        const float e = x - dv[i];
                        m4[i & 3] = fmaxf(m4[i & 3], fabsf(e));
                        s4[i & 3] = fmaf(e, e, s4[i & 3]);
                        a4[i & 3] = fmaf(x, x, a4[i & 3]);
                    }
                    const float gs = (s4[0] + s4[1]) + (s4[2] + s4[3]);
                    if (gs != gs) bad = 1;
                    mx = fmaxf(mx, fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3])));
                    tse += gs;
                    tsa += (a4[0] + a4[1]) + (a4[2] + a4[3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float x = As[(16 * c + i) * kTcBN];
                        if (jv && rbase + 16 * c + i < a.m) {
                            const float e = x - dv[i];
                            if (!(fabsf(e) <= INFINITY)) bad = 1;
                            mx = fmaxf(mx, fabsf(e));
                            tse = fmaf(e, e, tse);
                            tsa = fmaf(x, x, tsa);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ae[slot]);
            se += (double)tse;
            sa += (double)tsa;
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
        tmem_dealloc(tmem, 256);
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

// A (m x n FP32, leading dimension ld), boxes of 128 columns x 32 rows, no swizzle:
// a staged sub-tile is row-major 32 x 128 in shared memory. Needs a 16-byte aligned base
// and ld % 4 == 0.
static bool make_map_a(CUtensorMap* map, const float* base, int64_t m, int64_t n, int64_t ld) {
    auto enc = encode_fn();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld & 3) != 0) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t gstr[1] = {(cuuint64_t)ld * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kTcBN, (cuuint32_t)kAR};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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

static inline unsigned nbk(int64_t n, int t = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535));
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
    float* Ch = ar.get<float>((size_t)m * ldk);
    float* Cl = ar.get<float>((size_t)m * ldk);
    const int G = h->num_sms;
    double* part = ar.get<double>((size_t)G * 4);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUtensorMap mWh, mWl, mCh, mCl, mA;
    if (!make_map_a(&mA, static_cast<const float*>(Am->data), m, n, Am->ld)) return CUR_ERR_ARG;
    if (!make_map(&mWh, Wh, n, r, ldk) || !make_map(&mWl, Wl, n, r, ldk) || !make_map(&mCh, Ch, m, r, ldk) ||
        !make_map(&mCl, Cl, m, r, ldk))
        return CUR_ERR_ARG;
    const size_t smw = (size_t)r * r * sizeof(df64);
    CUR_TRY(smem_attr((const void*)tc_prep_w<float>, smw));
    tc_prep_w<float><<<(unsigned)std::min<int64_t>((n * ldk + 255) / 256, 8 * G), 256, smw, st>>>(
        U, static_cast<const float*>(R), r, n, ldk, Wh, Wl);
    CUR_CK(cudaGetLastError());
    note_launch();
    tc_prep_c<float><<<nbk(m * ldk), 256, 0, st>>>(static_cast<const float*>(C), m, r, ldk, Ch, Cl);
    CUR_CK(cudaGetLastError());
    note_launch();
    TcArgs a{};
    a.m = m;
    a.n = n;
    a.r = r;
    a.nch = nch;
    a.ksteps = (r + 7) / 8;
    a.ntile_n = (n + kTcBN - 1) / kTcBN;
    a.ntiles = ((m + kTcBM - 1) / kTcBM) * a.ntile_n;
    a.part = part;
    a.status = h->status;
    const int grid = (int)std::min<int64_t>(G, a.ntiles);
    // C panel and W^T tile (hi and lo each), then as many 16 KB A slots as fit
    const size_t fixed = (size_t)4 * nch * kChunk + 1024;
    const size_t budget = 225 * 1024;
    a.na = (int)std::min<size_t>(kNAMax, (budget - fixed) / kASub);
    if (a.na < 4) return CUR_ERR_ARG;
    const size_t sm = fixed + (size_t)a.na * kASub;
    CUR_TRY(smem_attr((const void*)residual_tc_k, sm));
    residual_tc_k<<<grid, 32 * (3 + kEpiWarps), sm, st>>>(mWh, mWl, mCh, mCl, mA, a);
    CUR_CK(cudaGetLastError());
    note_launch();
    tc_final_k<<<1, 256, 0, st>>>(part, grid, cheb, fro, h->status, sums);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}
