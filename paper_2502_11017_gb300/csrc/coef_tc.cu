// The coefficient product of the maxvol iteration, B = C M^-1 (Section 1.2's swap
// coefficients), on the tensor cores (tcgen05, sm_103a) for FP32 bases with r = 32 or 64.
//
// A stage's problems each own a run of rows of the basis C and an inverse M^-1 (FP64, as
// mv_lu or an inherited inverse leaves it). The product runs as 3xTF32 on
// tcgen05.mma.kind::tf32: C = Ch + Cl and W = M^-1 = Wh + Wl with Ch, Wh rounded to TF32
// and Cl, Wl the rounded remainders; D = Ch Wh + Ch Wl + Cl Wh keeps ~22 bits (FP32 level;
// the dropped Cl Wl is ~2^-22 relative). Tiles are 128 rows of one problem (they never
// straddle problems). A persistent CTA per SM takes every G-th tile through two
// shared-memory stages and two TMEM accumulators:
//   warp 0     TMA: the FP32 C tile (128 rows x r, 128-byte swizzle, K-major) and the
//              problem's W^T hi and lo (r rows x r) into the free stage
//   warps 6-9  split the landed C tile into TF32 hi (in place) and lo (the same swizzled
//              positions), then a proxy fence for the tensor core
//   warp 1     one thread: 3 passes x r/8 MMAs (M = 128 rows, N = r) per tile
//   warps 2-5  epilogue: tcgen05.ld of the thread's row (TMEM lane = row) into the consumed
//              C stage (swizzled), then one TMA tensor store of the B tile
// so the copy of tile i + 1, the split and MMAs of tile i and the epilogue of tile i - 1
// overlap. Persistent CTA, 320 threads.
// HBM traffic: C read once, B written once (W comes from L2). Waits are bounded: on a
// timeout the CTA records CUR_ERR_TIMEOUT, waits (bounded) for what it issued, frees its
// TMEM and returns.

#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace curk {

constexpr int kCoefBM = 128;                // rows per tile (MMA M)
constexpr int kCoefChunk = kCoefBM * 128;   // one 128-row x 32-element FP32 swizzled chunk

// W^T of problem pb (r rows x r, row n = column n of M^-1) split into TF32 hi and lo.
__global__ void coef_prep_w(const double* __restrict__ minv64, int64_t stride, int P, int r,
                            float* __restrict__ Wh, float* __restrict__ Wl, const int32_t* done) {
    const int64_t total = (int64_t)P * r * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int pb = (int)(e / ((int64_t)r * r));
        const int rem = (int)(e - (int64_t)pb * r * r);
        const int n = rem / r, k = rem - n * r;
        float hi = 0.f, lo = 0.f;
        if (!done || !done[pb]) {
            const double w = minv64[(int64_t)pb * stride + (int64_t)k * r + n];
            hi = to_tf32((float)w);
            lo = to_tf32((float)(w - (double)hi));
        }
        Wh[e] = hi;
        Wl[e] = lo;
    }
}

// All 128 epilogue threads agree (named barrier 1, AND-reduction): a wait that ran out in any
// of them ends the loop in all, so none is left at the next named barrier.
__device__ __forceinline__ bool epi_all(bool v) {
    uint32_t res;
    asm volatile("{ .reg .pred p, q; setp.ne.u32 q, %1, 0; bar.red.and.pred p, 1, 128, q; selp.u32 %0, 1, 0, p; }"
                 : "=r"(res) : "r"((uint32_t)v) : "memory");
    return res != 0;
}

constexpr int kCoefThreads = 320;        // warp 0: TMA, warp 1: MMA, warps 2..5: epilogue, 6..9: split
constexpr int kCoefEpi = 128;            // threads of the epilogue warps (one per tile row), and of the split
constexpr int kCoefMaxTiles = 128;       // tiles per CTA at most (the launch makes enough CTAs)

// Persistent: CTA c takes tiles c, c + G, ... Two shared-memory stages (C hi, C lo, W^T hi,
// W^T lo) and two TMEM accumulators, so the copy of tile i + 1, the split and MMAs of tile i
// and the epilogue of tile i - 1 overlap.
__global__ void __launch_bounds__(kCoefThreads, 1) coef_tc_k(const __grid_constant__ CUtensorMap mC,
                                                            const __grid_constant__ CUtensorMap mWh,
                                                            const __grid_constant__ CUtensorMap mWl,
                                                            const __grid_constant__ CUtensorMap mB,
                                                            const CoefTile* __restrict__ tiles, int ntiles, int r,
                                                            float* __restrict__ B, const int32_t* __restrict__ done,
                                                            int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nch = r / 32;
    const int wchunk = r * 128;                          // a 32-element chunk of W^T: r rows x 128 bytes
    const int cbytes = nch * kCoefChunk, wbytes = nch * wchunk;
    const int stage_bytes = 2 * cbytes + 2 * wbytes;
    auto CH = [&](int s) { return sm + s * stage_bytes; };
    auto CL = [&](int s) { return sm + s * stage_bytes + cbytes; };
    auto WH = [&](int s) { return sm + s * stage_bytes + 2 * cbytes; };
    auto WL = [&](int s) { return sm + s * stage_bytes + 2 * cbytes + wbytes; };
    __shared__ __align__(8) uint64_t full[2], split[2], mmad[2], accf[2], sfree[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ CoefTile s_tiles[kCoefMaxTiles];   // this CTA's tiles (prob -1: a done problem's)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncols = 2 * r;                             // two accumulators of r columns (64 or 128)
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&split[s], kCoefEpi);
            mbar_init(&mmad[s], 1);
            mbar_init(&accf[s], kCoefEpi);
            mbar_init(&sfree[s], 1);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tslot, ncols);
    // this CTA's tiles blockIdx.x, + gridDim.x, ... (at most kCoefMaxTiles: the launch makes
    // enough CTAs), read once; every role walks the same list
    const int my = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    for (int k = tid; k < my; k += blockDim.x) {
        CoefTile T = tiles[blockIdx.x + (int64_t)k * gridDim.x];
        if (done && done[T.prob]) T.prob = -1;
        s_tiles[k] = T;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int i = 0, issued = 0;
            for (int k = 0; k < my && !abort_flag; ++k) {
                const CoefTile T = s_tiles[k];
                if (T.prob < 0) continue;
                const int s = i & 1, u = i >> 1;
                // the stage is free once the epilogue of tile i - 2 is done with it
                if (u > 0 && !mbar_wait(&sfree[s], (uint32_t)((u - 1) & 1))) { abort_flag = 1; set_status(status, CUR_ERR_TIMEOUT); break; }
                mbar_expect_tx(&full[s], (uint32_t)(cbytes + 2 * wbytes));
                for (int c = 0; c < nch; ++c) {
                    tma_load_2d(CH(s) + c * kCoefChunk, &mC, &full[s], 32 * c, (int)T.row0);
                    tma_load_2d(WH(s) + c * wchunk, &mWh, &full[s], 32 * c, T.prob * r);
                    tma_load_2d(WL(s) + c * wchunk, &mWl, &full[s], 32 * c, T.prob * r);
                }
                ++i;
                issued = i;
            }
            // after an abort, wait (bounded) for the copies still in flight
            if (abort_flag)
                for (int q = issued - 1; q >= 0 && q >= issued - 2; --q) mbar_wait(&full[q & 1], (uint32_t)((q >> 1) & 1));
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kCoefBM, r);
            int i = 0;
            uint64_t* last = nullptr;
            uint32_t last_par = 0;
            for (int k = 0; k < my && !abort_flag; ++k) {
                if (s_tiles[k].prob < 0) continue;
                const int s = i & 1, u = i >> 1;
                if (!mbar_wait(&split[s], (uint32_t)(u & 1))) { abort_flag = 1; set_status(status, CUR_ERR_TIMEOUT); break; }
                if (u > 0 && !mbar_wait(&accf[s], (uint32_t)((u - 1) & 1))) { abort_flag = 1; set_status(status, CUR_ERR_TIMEOUT); break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(s * r);
                const uint32_t ch0 = su32(CH(s)), cl0 = su32(CL(s)), wh0 = su32(WH(s)), wl0 = su32(WL(s));
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t aop = pass == 2 ? cl0 : ch0;   // Ch Wh, Ch Wl, Cl Wh
                    const uint32_t bop = pass == 1 ? wl0 : wh0;
                    for (int k = 0; k < r / 8; ++k) {
                        const uint32_t offc = (uint32_t)((k >> 2) * kCoefChunk + (k & 3) * 32);
                        const uint32_t offw = (uint32_t)((k >> 2) * wchunk + (k & 3) * 32);
                        mma_tf32(d, sdesc_k128(aop + offc), sdesc_k128(bop + offw), idesc, (pass | k) != 0);
                    }
                }
                mma_commit(&mmad[s]);
                last = &mmad[s];
                last_par = (uint32_t)(u & 1);
                ++i;
            }
            if (last) mbar_wait(last, last_par);   // every MMA issued has finished
        }
    } else if (warp < 6) {
        // ---------------------------------------------------------------- epilogue (warps 2..5)
        // A full tile goes out through the consumed C stage: each thread writes its row into
        // the 128-byte-swizzled layout of the B tensor map, one thread stores the tile by TMA
        // and frees the stage once the copy has read it. A tile that ends a problem early is
        // stored row by row (a box store cannot stop at the problem's last row).
        const int lq = (warp & 3) * 32;                     // this warp's TMEM lanes = tile rows
        const int row = lq + lane;
        const int et = tid - 64;
        int i = 0;
        bool ok = true;
        for (int k = 0; k < my && !abort_flag; ++k) {
            const CoefTile T = s_tiles[k];
            if (T.prob < 0) continue;
            const int s = i & 1, u = i >> 1;
            if (!epi_all(mbar_wait(&mmad[s], (uint32_t)(u & 1)))) { ok = false; break; }
            tc_fence_after();
            if (T.nrows == kCoefBM) {
                unsigned char* stg = CH(s);
                for (int c0 = 0; c0 < r; c0 += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)lq << 16) + (uint32_t)(s * r + c0), v);
                    unsigned char* base = stg + (c0 / 32) * kCoefChunk + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(base + ((q ^ (row & 7)) << 4)) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                tc_fence_before();
                mbar_arrive(&accf[s]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (et == 0) {
                    for (int c = 0; c < nch; ++c) tma_store_2d(&mB, stg + c * kCoefChunk, 32 * c, (int)T.row0);
                    tma_store_commit();
                    tma_store_wait_read();
                    mbar_arrive(&sfree[s]);
                }
            } else {
                if (et == 0) mbar_arrive(&sfree[s]);
                for (int c0 = 0; c0 < r; c0 += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)lq << 16) + (uint32_t)(s * r + c0), v);
                    if (row < T.nrows) {
                        float4* dst = reinterpret_cast<float4*>(B + (T.row0 + row) * r + c0);
#pragma unroll
                        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&accf[s]);
            }
            ++i;
        }
        if (et == 0) tma_store_wait_all();                  // the tile stores have completed
        if (!ok) { abort_flag = 1; set_status(status, CUR_ERR_TIMEOUT); }
    } else {
        // ---------------------------------------------------------------- split (warps 6..9)
        const int et = tid - 192;
        int i = 0;
        bool ok = true;
        for (int k = 0; k < my && !abort_flag; ++k) {
            if (s_tiles[k].prob < 0) continue;
            const int s = i & 1, u = i >> 1;
            if (!mbar_wait(&full[s], (uint32_t)(u & 1))) { ok = false; break; }
            float4* ch = reinterpret_cast<float4*>(CH(s));
            float4* cl = reinterpret_cast<float4*>(CL(s));
            for (int e = et; e < nch * kCoefChunk / 16; e += kCoefEpi) {
                const float4 x = ch[e];
                float4 hi, lo;
                hi.x = to_tf32(x.x); lo.x = to_tf32(x.x - hi.x);
                hi.y = to_tf32(x.y); lo.y = to_tf32(x.y - hi.y);
                hi.z = to_tf32(x.z); lo.z = to_tf32(x.z - hi.z);
                hi.w = to_tf32(x.w); lo.w = to_tf32(x.w - hi.w);
                ch[e] = hi;
                cl[e] = lo;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&split[s]);
            ++i;
        }
        if (!ok) { abort_flag = 1; set_status(status, CUR_ERR_TIMEOUT); }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

static PFN_cuTensorMapEncodeTiled_v12000 coef_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// rows x r FP32 (pitch r), boxes of 32 elements x box_rows, 128-byte swizzle.
static bool coef_map(CUtensorMap* map, const float* base, int64_t rows, int r, int box_rows) {
    auto enc = coef_encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)r, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)r * sizeof(float)};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstr, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace curk

bool coef_tc_applies(cur_dtype dt, int r) { return dt == CUR_F32 && (r == 32 || r == 64); }

size_t coef_tc_smem(int r) {
    const int nch = r / 32;
    return 1024 + 2 * (2 * (size_t)nch * curk::kCoefChunk + 2 * (size_t)nch * r * 128);
}

cur_status coef_tc_launch(cur_handle* h, const float* basis, int64_t prows, int r, const double* minv64,
                          int64_t minv_stride_, int P, const CoefTile* tiles_dev, int ntiles, const int32_t* done,
                          float* Wh, float* Wl, float* B, cudaStream_t st) {
    using namespace curk;
    if (!coef_tc_applies(CUR_F32, r) || ntiles < 1) return CUR_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(basis) % 16 || reinterpret_cast<uintptr_t>(Wh) % 16 ||
        reinterpret_cast<uintptr_t>(Wl) % 16 || reinterpret_cast<uintptr_t>(B) % 16)
        return CUR_ERR_ARG;
    CUtensorMap mC, mWh, mWl, mB;
    if (!coef_map(&mC, basis, prows, r, kCoefBM) || !coef_map(&mWh, Wh, (int64_t)P * r, r, r) ||
        !coef_map(&mWl, Wl, (int64_t)P * r, r, r) || !coef_map(&mB, B, prows, r, kCoefBM))
        return CUR_ERR_ARG;
    const int64_t wtot = (int64_t)P * r * r;
    const unsigned wg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((wtot + 255) / 256, 4LL * h->num_sms));
    coef_prep_w<<<wg, 256, 0, st>>>(minv64, minv_stride_, P, r, Wh, Wl, done);
    CUR_CK(cudaGetLastError());
    const size_t sm = coef_tc_smem(r);
    CUR_TRY(smem_attr((const void*)coef_tc_k, sm));
    const int grid = std::max(std::min(ntiles, h->num_sms), (ntiles + kCoefMaxTiles - 1) / kCoefMaxTiles);
    coef_tc_k<<<grid, kCoefThreads, sm, st>>>(mC, mWh, mWl, mB, tiles_dev, ntiles, r, B, done, h->status);
    CUR_CK(cudaGetLastError());
    note_launch(2);
    return CUR_OK;
}

extern "C" cur_status cur_coef_tf32(cur_handle* h, const cur_mat* basis, const double* minv, float* B_out,
                                    cudaStream_t st) {
    if (!h || !basis || !basis->data || !minv || !B_out) return CUR_ERR_ARG;
    const int64_t p = basis->rows;
    const int r = (int)basis->cols;
    if (basis->dtype != CUR_F32 || basis->ld != basis->cols || !coef_tc_applies(CUR_F32, r) || p < 1 ||
        p > INT_MAX - 256)
        return CUR_ERR_ARG;
    Arena ar = h->arena();
    const int64_t ntiles = (p + curk::kCoefBM - 1) / curk::kCoefBM;
    CoefTile* tiles = ar.get<CoefTile>((size_t)ntiles);
    float* Wh = ar.get<float>((size_t)r * r);
    float* Wl = ar.get<float>((size_t)r * r);
    if (!ar.ok) return CUR_ERR_NOMEM;
    std::vector<CoefTile> ht((size_t)ntiles);
    for (int64_t t = 0; t < ntiles; ++t)
        ht[t] = CoefTile{0, (int32_t)std::min<int64_t>(curk::kCoefBM, p - t * curk::kCoefBM), t * curk::kCoefBM};
    CUR_TRY(upload_table(tiles, ht.data(), sizeof(CoefTile) * ht.size(), st));
    return coef_tc_launch(h, static_cast<const float*>(basis->data), p, r, minv, (int64_t)r * r, 1, tiles,
                          (int)ntiles, nullptr, Wh, Wl, B_out, st);
}
