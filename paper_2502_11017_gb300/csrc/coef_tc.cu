// The coefficient product of the maxvol iteration, B = C M^-1 (Section 1.2's swap
// coefficients), on the tensor cores (tcgen05, sm_103a) for FP32 bases with r = 32 or 64.
//
// A stage's problems each own a run of rows of the basis C and an inverse M^-1 (FP64, as
// mv_lu or an inherited inverse leaves it). The product runs as 3xTF32 on
// tcgen05.mma.kind::tf32: C = Ch + Cl and W = M^-1 = Wh + Wl with Ch, Wh rounded to TF32
// and Cl, Wl the rounded remainders; D = Ch Wh + Ch Wl + Cl Wh keeps ~22 bits (FP32 level;
// the dropped Cl Wl is ~2^-22 relative). One CTA per 128-row tile of a problem (tiles never
// straddle problems), 128 threads:
//   thread 0   TMA: the FP32 C tile (128 rows x r, 128-byte swizzle, K-major) and the
//              problem's W^T hi and lo (r rows x r); one mbarrier with the byte count
//   all        split the C tile in shared memory into TF32 hi (in place) and lo (the same
//              swizzled positions), then a proxy fence for the tensor core
//   thread 0   3 passes x r/8 MMAs (M = 128 rows, N = r) into one TMEM accumulator
//   all        tcgen05.ld of the thread's row (TMEM lane = row), store B rows
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

__global__ void __launch_bounds__(128, 2) coef_tc_k(const __grid_constant__ CUtensorMap mC,
                                                    const __grid_constant__ CUtensorMap mWh,
                                                    const __grid_constant__ CUtensorMap mWl,
                                                    const CoefTile* __restrict__ tiles, int r, float* __restrict__ B,
                                                    const int32_t* __restrict__ done, int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nch = r / 32;
    const int wchunk = r * 128;                 // one 32-element chunk of W^T: r rows x 128 bytes
    unsigned char* CH = sm;
    unsigned char* CL = CH + nch * kCoefChunk;
    unsigned char* WH = CL + nch * kCoefChunk;
    unsigned char* WL = WH + nch * wchunk;
    __shared__ __align__(8) uint64_t full, mmad;
    __shared__ uint32_t tslot;
    const CoefTile T = tiles[blockIdx.x];
    if (done && done[T.prob]) return;           // the whole CTA leaves: nothing issued yet
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ncols = r < 32 ? 32 : r;          // TMEM columns (a power of two >= 32)
    if (tid == 0) {
        mbar_init(&full, 1);
        mbar_init(&mmad, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tslot, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    if (tid == 0) {
        mbar_expect_tx(&full, (uint32_t)(nch * kCoefChunk + 2 * nch * wchunk));
        for (int c = 0; c < nch; ++c) {
            tma_load_2d(CH + c * kCoefChunk, &mC, &full, 32 * c, (int)T.row0);
            tma_load_2d(WH + c * wchunk, &mWh, &full, 32 * c, T.prob * r);
            tma_load_2d(WL + c * wchunk, &mWl, &full, 32 * c, T.prob * r);
        }
    }
    bool ok = mbar_wait(&full, 0);
    ok = __syncthreads_and(ok);
    if (ok) {
        // split C into TF32 hi (in place) and lo at the same swizzled positions
        float* ch = reinterpret_cast<float*>(CH);
        float* cl = reinterpret_cast<float*>(CL);
        for (int e = tid; e < nch * kCoefChunk / 4; e += blockDim.x) {
            const float x = ch[e];
            const float hi = to_tf32(x);
            ch[e] = hi;
            cl[e] = to_tf32(x - hi);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t idesc = idesc_tf32(kCoefBM, r);
            const uint32_t ch0 = su32(CH), cl0 = su32(CL), wh0 = su32(WH), wl0 = su32(WL);
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t aop = pass == 2 ? cl0 : ch0;   // Ch Wh, Ch Wl, Cl Wh
                const uint32_t bop = pass == 1 ? wl0 : wh0;
                for (int k = 0; k < r / 8; ++k) {
                    const uint32_t offc = (uint32_t)((k >> 2) * kCoefChunk + (k & 3) * 32);
                    const uint32_t offw = (uint32_t)((k >> 2) * wchunk + (k & 3) * 32);
                    mma_tf32(tmem, sdesc_k128(aop + offc), sdesc_k128(bop + offw), idesc, (pass | k) != 0);
                }
            }
            mma_commit(&mmad);
        }
        bool fine = mbar_wait(&mmad, 0);
        fine = __syncthreads_and(fine);
        tc_fence_after();
        if (fine) {
            const int64_t row = T.row0 + tid;
            for (int c0 = 0; c0 < r; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
                if (tid < T.nrows) {
                    float4* dst = reinterpret_cast<float4*>(B + row * r + c0);
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        } else if (tid == 0) {
            set_status(status, CUR_ERR_TIMEOUT);
            mbar_wait(&mmad, 0);   // bounded: the MMAs it issued
        }
    } else if (tid == 0) {
        set_status(status, CUR_ERR_TIMEOUT);
        mbar_wait(&full, 0);       // bounded: the copies it issued
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
    return 1024 + 2 * (size_t)nch * curk::kCoefChunk + 2 * (size_t)nch * r * 128;
}

cur_status coef_tc_launch(cur_handle* h, const float* basis, int64_t prows, int r, const double* minv64,
                          int64_t minv_stride_, int P, const CoefTile* tiles_dev, int ntiles, const int32_t* done,
                          float* Wh, float* Wl, float* B, cudaStream_t st) {
    using namespace curk;
    if (!coef_tc_applies(CUR_F32, r) || ntiles < 1) return CUR_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(basis) % 16 || reinterpret_cast<uintptr_t>(Wh) % 16 ||
        reinterpret_cast<uintptr_t>(Wl) % 16 || reinterpret_cast<uintptr_t>(B) % 16)
        return CUR_ERR_ARG;
    CUtensorMap mC, mWh, mWl;
    if (!coef_map(&mC, basis, prows, r, kCoefBM) || !coef_map(&mWh, Wh, (int64_t)P * r, r, r) ||
        !coef_map(&mWl, Wl, (int64_t)P * r, r, r))
        return CUR_ERR_ARG;
    const int64_t wtot = (int64_t)P * r * r;
    const unsigned wg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((wtot + 255) / 256, 4LL * h->num_sms));
    coef_prep_w<<<wg, 256, 0, st>>>(minv64, minv_stride_, P, r, Wh, Wl, done);
    CUR_CK(cudaGetLastError());
    const size_t sm = coef_tc_smem(r);
    CUR_TRY(smem_attr((const void*)coef_tc_k, sm));
    coef_tc_k<<<ntiles, 128, sm, st>>>(mC, mWh, mWl, tiles_dev, r, B, done, h->status);
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
