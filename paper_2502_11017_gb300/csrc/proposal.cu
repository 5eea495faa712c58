// Learned proposal for the maxvol cross: Gaussian sketch features of the rows and the
// columns of A, a 2-layer scoring network (forward pass, cross-entropy gradients, Adam),
// the r best-scored indices, and maxvol refinement of a proposed cross. The selection
// itself stays the paper's maxvol (Section 3, Algorithm 2's sweeps); the network only
// chooses where the sweeps start.
//
// Sketch (Y = A S, Zt = A^T T, k = 32 features): two one-pass register-tiled FP32
// contractions. A CTA owns 128 rows (or 128 columns) and a contiguous range of the
// contraction, a thread an 8 x 4 block of outputs; the split partials are summed in a
// fixed order, so the features are deterministic. At 16 flops per element of A the pair
// is bound by the FP32 FMA rate, not HBM; a one-pass kernel computing both would read A
// once but do the same FMAs.
//
// Network (k -> H -> 1, ReLU): a CTA of H threads, thread h owns hidden unit h and holds
// column h of W1 in registers; 32 samples at a time are staged in shared memory, the
// score of each is a block reduction (a transposing butterfly in each warp). Gradients
// are per-CTA partials summed in a fixed order by a second kernel.

#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace curk {

constexpr int kSkK = 32;        // features per row / column
constexpr int kSkT = 128;       // rows (or columns) of A per CTA
constexpr int kSkC = 32;        // contraction chunk
constexpr int kSkThreads = 128;
constexpr int kSkPad = 4;       // shared-memory row padding (floats)
constexpr int kMlpMaxH = 256;   // hidden units (one thread each; registers bound the CTA)

template <typename TA>
__device__ __forceinline__ float4 load4(const TA* p) {
    return make_float4(to_f(p[0]), to_f(p[1]), to_f(p[2]), to_f(p[3]));
}
template <>
__device__ __forceinline__ float4 load4<float>(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
template <>
__device__ __forceinline__ float4 load4<__nv_bfloat16>(const __nv_bfloat16* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&u.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&u.y);
    const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 load4<double>(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// Four consecutive elements p[0..3] of a row whose valid part ends at `lim` elements from p
// (zeros past it); vec: the four are in range and 4-element aligned.
template <typename TA>
__device__ __forceinline__ float4 load4_guard(const TA* p, int64_t lim, bool vec) {
    if (vec && lim >= 4) return load4(p);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lim > 0) v.x = to_f(p[0]);
    if (lim > 1) v.y = to_f(p[1]);
    if (lim > 2) v.z = to_f(p[2]);
    if (lim > 3) v.w = to_f(p[3]);
    return v;
}

// Partial row sketch: Yp[split][i][c] = sum over the split's columns j of A[i][j] S[j][c].
// grid (ceil(m / 128), splits); the split's columns are chunks [c0, c1) of 32.
template <typename TA>
__global__ void __launch_bounds__(kSkThreads) sk_rows_k(const TA* __restrict__ A, int64_t m, int64_t n,
                                                        int64_t ld, bool vec, const float* __restrict__ S,
                                                        int chunks_per_split, float* __restrict__ Yp) {
    __shared__ __align__(16) float As[kSkT][kSkC + kSkPad];
    __shared__ __align__(16) float Ss[kSkC][kSkK];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int rg = lane >> 3, cg = lane & 7;
    const int64_t i0 = (int64_t)blockIdx.x * kSkT;
    const int64_t nchunks = (n + kSkC - 1) / kSkC;
    const int64_t c0 = (int64_t)blockIdx.y * chunks_per_split;
    const int64_t c1 = c0 + chunks_per_split < nchunks ? c0 + chunks_per_split : nchunks;
    float acc[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
    float4 ra[8], rs[2];
    auto fetch = [&](int64_t ch) {
        const int64_t j0 = ch * kSkC;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = t + kSkThreads * u, row = e >> 3, c4 = e & 7;
            const int64_t i = i0 + row, j = j0 + 4 * c4;
            ra[u] = i < m ? load4_guard(A + i * ld + j, n - j, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + kSkThreads * u, row = e >> 3, c4 = e & 7;
            const int64_t j = j0 + row;
            rs[u] = j < n ? __ldg(reinterpret_cast<const float4*>(S + j * kSkK) + c4)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if (c0 < c1) fetch(c0);
    for (int64_t ch = c0; ch < c1; ++ch) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = t + kSkThreads * u;
            *reinterpret_cast<float4*>(&As[e >> 3][4 * (e & 7)]) = ra[u];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + kSkThreads * u;
            *reinterpret_cast<float4*>(&Ss[e >> 3][4 * (e & 7)]) = rs[u];
        }
        __syncthreads();
        if (ch + 1 < c1) fetch(ch + 1);
#pragma unroll
        for (int kk = 0; kk < kSkC; kk += 4) {
            float4 s[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] = *reinterpret_cast<const float4*>(&Ss[kk + q][4 * cg]);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 a = *reinterpret_cast<const float4*>(&As[warp * 32 + rg + 4 * q][kk]);
                acc[q][0] = fmaf(a.x, s[0].x, fmaf(a.y, s[1].x, fmaf(a.z, s[2].x, fmaf(a.w, s[3].x, acc[q][0]))));
                acc[q][1] = fmaf(a.x, s[0].y, fmaf(a.y, s[1].y, fmaf(a.z, s[2].y, fmaf(a.w, s[3].y, acc[q][1]))));
                acc[q][2] = fmaf(a.x, s[0].z, fmaf(a.y, s[1].z, fmaf(a.z, s[2].z, fmaf(a.w, s[3].z, acc[q][2]))));
                acc[q][3] = fmaf(a.x, s[0].w, fmaf(a.y, s[1].w, fmaf(a.z, s[2].w, fmaf(a.w, s[3].w, acc[q][3]))));
            }
        }
    }
    float* out = Yp + (int64_t)blockIdx.y * m * kSkK;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t i = i0 + warp * 32 + rg + 4 * q;
        if (i < m)
            *reinterpret_cast<float4*>(out + i * kSkK + 4 * cg) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
    }
}

// Partial column sketch: Zp[split][j][c] = sum over the split's rows i of A[i][j] T[i][c].
// grid (ceil(n / 128), splits); the split's rows are chunks [c0, c1) of 32.
template <typename TA>
__global__ void __launch_bounds__(kSkThreads) sk_cols_k(const TA* __restrict__ A, int64_t m, int64_t n,
                                                        int64_t ld, bool vec, const float* __restrict__ T,
                                                        int chunks_per_split, float* __restrict__ Zp) {
    __shared__ __align__(16) float As[kSkC][kSkT + kSkPad];
    __shared__ __align__(16) float Ts[kSkC][kSkK];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int jg = lane >> 3, cg = lane & 7;
    const int64_t j0 = (int64_t)blockIdx.x * kSkT;
    const int64_t nchunks = (m + kSkC - 1) / kSkC;
    const int64_t c0 = (int64_t)blockIdx.y * chunks_per_split;
    const int64_t c1 = c0 + chunks_per_split < nchunks ? c0 + chunks_per_split : nchunks;
    float acc[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = 0.f;
    float4 ra[8], rt[2];
    auto fetch = [&](int64_t ch) {
        const int64_t r0 = ch * kSkC;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = t + kSkThreads * u, row = e >> 5, c4 = e & 31;
            const int64_t i = r0 + row, j = j0 + 4 * c4;
            ra[u] = i < m ? load4_guard(A + i * ld + j, n - j, vec) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + kSkThreads * u, row = e >> 3, c4 = e & 7;
            const int64_t i = r0 + row;
            rt[u] = i < m ? __ldg(reinterpret_cast<const float4*>(T + i * kSkK) + c4)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if (c0 < c1) fetch(c0);
    for (int64_t ch = c0; ch < c1; ++ch) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = t + kSkThreads * u;
            *reinterpret_cast<float4*>(&As[e >> 5][4 * (e & 31)]) = ra[u];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = t + kSkThreads * u;
            *reinterpret_cast<float4*>(&Ts[e >> 3][4 * (e & 7)]) = rt[u];
        }
        __syncthreads();
        if (ch + 1 < c1) fetch(ch + 1);
#pragma unroll 8
        for (int ii = 0; ii < kSkC; ++ii) {
            const float4 tv = *reinterpret_cast<const float4*>(&Ts[ii][4 * cg]);
            const float4 a0 = *reinterpret_cast<const float4*>(&As[ii][warp * 32 + jg * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[ii][warp * 32 + jg * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                acc[q][0] = fmaf(av[q], tv.x, acc[q][0]);
                acc[q][1] = fmaf(av[q], tv.y, acc[q][1]);
                acc[q][2] = fmaf(av[q], tv.z, acc[q][2]);
                acc[q][3] = fmaf(av[q], tv.w, acc[q][3]);
            }
        }
    }
    float* out = Zp + (int64_t)blockIdx.y * n * kSkK;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t j = j0 + warp * 32 + jg * 8 + q;
        if (j < n)
            *reinterpret_cast<float4*>(out + j * kSkK + 4 * cg) = make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
    }
}

// out[i][:] = sum over s of part[s][i][:] (s in order); the largest squared row norm goes
// to *maxsq (as the bits of a non-negative float, so an integer maximum orders them).
// Eight threads per row, each one float4.
__global__ void sk_reduce_k(const float* __restrict__ part, int splits, int64_t rows, float* __restrict__ out,
                            unsigned* maxsq) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = g >> 3;
    const int c4 = (int)(g & 7);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < rows) {
        for (int p = 0; p < splits; ++p) {
            const float4 v = reinterpret_cast<const float4*>(part + ((int64_t)p * rows + i) * kSkK)[c4];
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
        reinterpret_cast<float4*>(out + i * kSkK)[c4] = s;
    }
    float nsq = s.x * s.x + s.y * s.y + s.z * s.z + s.w * s.w;
    nsq += __shfl_xor_sync(0xffffffffu, nsq, 1);
    nsq += __shfl_xor_sync(0xffffffffu, nsq, 2);
    nsq += __shfl_xor_sync(0xffffffffu, nsq, 4);
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) nsq = fmaxf(nsq, __shfl_xor_sync(0xffffffffu, nsq, o));
    if ((threadIdx.x & 31) == 0 && nsq > 0.f) atomicMax(maxsq, __float_as_uint(nsq));
}

// x *= 1 / sqrt(max squared row norm), when that is positive and finite.
__global__ void sk_scale_k(float* __restrict__ x, int64_t count, const unsigned* maxsq) {
    const float mx = __uint_as_float(*maxsq);
    if (!(mx > 0.f) || !isfinite(mx)) return;
    const float inv = 1.0f / sqrtf(mx);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        x[e] *= inv;
}

// ---------------------------------------------------------------- scoring network

// v[0..31] per lane -> returns, in lane l, the sum over the warp's lanes of v[l].
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float send = upper ? v[i] : v[i + off];
            const float keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}

struct MlpCtx {
    float w[kSkK];   // column h of W1
    float b1, w2;
};

// The row of X for sample sg (idx[sg], or sg), or -1 if it lies outside [0, nrows).
__device__ __forceinline__ int64_t mlp_row(const int64_t* idx, int64_t sg, int64_t nrows) {
    const int64_t row = idx ? idx[sg] : sg;
    return row >= 0 && row < nrows ? row : -1;
}

// Stages samples [s0, s0 + 32) (rows idx[s] of X, or s) in Xs; zeros past N and for a row
// outside X (recorded as CUR_ERR_ARG).
__device__ __forceinline__ void mlp_stage(float (*Xs)[kSkK], const float* __restrict__ X, const int64_t* idx,
                                          int64_t N, int64_t nrows, int64_t s0, int* status) {
    for (int e = threadIdx.x; e < 32 * (kSkK / 4); e += blockDim.x) {
        const int s = e / (kSkK / 4), c4 = e % (kSkK / 4);
        const int64_t sg = s0 + s;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sg < N) {
            const int64_t row = mlp_row(idx, sg, nrows);
            if (row >= 0) v = __ldg(reinterpret_cast<const float4*>(X + row * kSkK) + c4);
            else if (c4 == 0) set_status(status, CUR_ERR_ARG);
        }
        *reinterpret_cast<float4*>(&Xs[s][4 * c4]) = v;
    }
}

// Scores of the 32 staged samples: z[s] = pre-activation of unit h; returns in red[] the
// per-warp partial sums of relu(z) w2 (red[warp][s]); the caller sums them.
__device__ __forceinline__ void mlp_hidden(const float (*Xs)[kSkK], const MlpCtx& c, float (&z)[32],
                                           float (*red)[32]) {
    float v[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        float a = c.b1;
#pragma unroll
        for (int k = 0; k < kSkK; ++k) a = fmaf(Xs[s][k], c.w[k], a);
        z[s] = a;
        v[s] = fmaxf(a, 0.f) * c.w2;
    }
    const float ws = warp_transpose_sum(v);
    red[threadIdx.x >> 5][threadIdx.x & 31] = ws;
}

__device__ __forceinline__ void mlp_load(MlpCtx& c, const float* __restrict__ P, int H) {
    const int h = threadIdx.x;
#pragma unroll
    for (int k = 0; k < kSkK; ++k) c.w[k] = P[(int64_t)k * H + h];
    c.b1 = P[(int64_t)kSkK * H + h];
    c.w2 = P[(int64_t)kSkK * H + H + h];
}

// scores[s] = relu(X[s] W1 + b1) w2 + b2 for all N samples. blockDim = H.
__global__ void __launch_bounds__(kMlpMaxH) mlp_fwd_k(const float* __restrict__ X, int64_t N, const float* __restrict__ P, int H,
                          float* __restrict__ scores) {
    __shared__ __align__(16) float Xs[32][kSkK];
    __shared__ float red[32][32];
    MlpCtx c;
    mlp_load(c, P, H);
    const float b2 = P[(int64_t)kSkK * H + 2 * H];
    const int nw = H >> 5;
    float z[32];
    for (int64_t s0 = (int64_t)blockIdx.x * 32; s0 < N; s0 += (int64_t)gridDim.x * 32) {
        __syncthreads();
        mlp_stage(Xs, X, nullptr, N, N, s0, nullptr);
        __syncthreads();
        mlp_hidden(Xs, c, z, red);
        __syncthreads();
        if (threadIdx.x < 32) {
            float sc = b2;
            for (int w = 0; w < nw; ++w) sc += red[w][threadIdx.x];
            if (s0 + threadIdx.x < N) scores[s0 + threadIdx.x] = sc;
        }
    }
}

__device__ __forceinline__ float softplus(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// Per-CTA partial gradients of the weighted mean cross-entropy; gp row = [dW1 (k x H),
// db1 (H), dw2 (H), db2, loss]. blockDim = H.
__global__ void __launch_bounds__(kMlpMaxH) mlp_grad_k(const float* __restrict__ X, const float* __restrict__ y, const int64_t* idx,
                           int64_t N, int64_t nrows, const float* __restrict__ P, int H, float pos_weight, float invN,
                           float* __restrict__ gp, int* status) {
    __shared__ __align__(16) float Xs[32][kSkK];
    __shared__ float red[32][32];
    __shared__ float dss[32];
    MlpCtx c;
    mlp_load(c, P, H);
    const float b2 = P[(int64_t)kSkK * H + 2 * H];
    const int nw = H >> 5;
    float dW[kSkK];
#pragma unroll
    for (int k = 0; k < kSkK; ++k) dW[k] = 0.f;
    float db1 = 0.f, dw2 = 0.f, db2 = 0.f, loss = 0.f;
    float z[32];
    for (int64_t s0 = (int64_t)blockIdx.x * 32; s0 < N; s0 += (int64_t)gridDim.x * 32) {
        __syncthreads();
        mlp_stage(Xs, X, idx, N, nrows, s0, status);
        __syncthreads();
        mlp_hidden(Xs, c, z, red);
        __syncthreads();
        if (threadIdx.x < 32) {
            const int64_t sg = s0 + threadIdx.x;
            float ds = 0.f;
            const int64_t row = sg < N ? mlp_row(idx, sg, nrows) : -1;
            if (row >= 0) {
                float sc = b2;
                for (int w = 0; w < nw; ++w) sc += red[w][threadIdx.x];
                const float lab = y[row];
                const float wt = lab > 0.5f ? pos_weight : 1.f;
                const float sig = 1.f / (1.f + expf(-sc));
                ds = wt * (sig - lab) * invN;
                loss += wt * (lab * softplus(-sc) + (1.f - lab) * softplus(sc));
            }
            dss[threadIdx.x] = ds;
            db2 += ds;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 32; ++s) {
            const float ds = dss[s];
            dw2 = fmaf(fmaxf(z[s], 0.f), ds, dw2);
            const float dh = z[s] > 0.f ? ds * c.w2 : 0.f;
            db1 += dh;
#pragma unroll
            for (int k = 0; k < kSkK; ++k) dW[k] = fmaf(Xs[s][k], dh, dW[k]);
        }
    }
    const int64_t Pn = (int64_t)kSkK * H + 2 * H + 1;
    float* g = gp + (int64_t)blockIdx.x * (Pn + 1);
    const int h = threadIdx.x;
#pragma unroll
    for (int k = 0; k < kSkK; ++k) g[(int64_t)k * H + h] = dW[k];
    g[(int64_t)kSkK * H + h] = db1;
    g[(int64_t)kSkK * H + H + h] = dw2;
    if (threadIdx.x < 32) {
        for (int o = 16; o > 0; o >>= 1) {
            db2 += __shfl_xor_sync(0xffffffffu, db2, o);
            loss += __shfl_xor_sync(0xffffffffu, loss, o);
        }
        if (threadIdx.x == 0) {
            g[Pn - 1] = db2;
            g[Pn] = loss * invN;
        }
    }
}

// grads[p] = sum over CTAs b (in order) of gp[b][p]; *loss likewise, in double.
__global__ void mlp_grad_reduce_k(const float* __restrict__ gp, int nb, int64_t Pn, float* __restrict__ grads,
                                  double* loss) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > Pn) return;
    if (p < Pn) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += gp[(int64_t)b * (Pn + 1) + p];
        grads[p] = s;
    } else if (loss) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += (double)gp[(int64_t)b * (Pn + 1) + p];
        *loss = s;
    }
}

// Adam (Kingma and Ba, 2015): m1 = b1 m1 + (1 - b1) g, m2 = b2 m2 + (1 - b2) g^2,
// p -= lr (m1 / c1) / (sqrt(m2 / c2) + eps) with c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void adam_k(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int64_t count, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float a = b1 * m1[e] + (1.f - b1) * ge;
        const float v = b2 * m2[e] + (1.f - b2) * ge * ge;
        m1[e] = a;
        m2[e] = v;
        p[e] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// ---------------------------------------------------------------- top-r proposal

// Order-preserving key of (score, index): a larger score wins, then the smaller index;
// NaN ranks below everything.
__device__ __forceinline__ unsigned long long prop_key(float s, int64_t i) {
    const unsigned b = __float_as_uint(s == 0.f ? 0.f : s);   // -0 ranks as +0
    const unsigned o = isnan(s) ? 0u : ((b & 0x80000000u) ? ~b : (b | 0x80000000u));
    return ((unsigned long long)o << 32) | (unsigned long long)(0xffffffffu - (unsigned)i);
}

// idx[t] = index of the (t+1)-th largest key; every key is distinct, so round t takes the
// largest key below round t-1's. One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) propose_k(const float* __restrict__ scores, int64_t N, int r,
                                                  int32_t* __restrict__ idx) {
    __shared__ unsigned long long wmax[32];
    unsigned long long prev = ~0ull;
    for (int t = 0; t < r; ++t) {
        unsigned long long best = 0ull;
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
            const unsigned long long k = prop_key(scores[i], i);
            if (k < prev && k > best) best = k;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k = __shfl_xor_sync(0xffffffffu, best, o);
            best = k > best ? k : best;
        }
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
        __syncthreads();
        best = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) best = wmax[w] > best ? wmax[w] : best;
        __syncthreads();
        prev = best;
        if (threadIdx.x == 0) idx[t] = (int32_t)(0xffffffffu - (unsigned)(best & 0xffffffffull));
    }
}

// Closes cur_cross_from: records a SINGULAR / NOCONV end in the status word, sets the
// log-volume of a singular proposal to -inf, and fills the caller's info.
}  // namespace curk

namespace {

// Column and row splits of the two sketch kernels: enough CTAs for about four per SM.
void sketch_splits(int num_sms, int64_t m, int64_t n, int* sr, int* cpr, int* sc, int* cpc) {
    const int64_t tr = (m + curk::kSkT - 1) / curk::kSkT, tc = (n + curk::kSkT - 1) / curk::kSkT;
    const int64_t nr = (n + curk::kSkC - 1) / curk::kSkC, nc = (m + curk::kSkC - 1) / curk::kSkC;
    const int64_t want = 4LL * num_sms;
    int64_t s = std::max<int64_t>(1, std::min<int64_t>((want + tr - 1) / tr, nr));
    *cpr = (int)((nr + s - 1) / s);
    *sr = (int)((nr + *cpr - 1) / *cpr);
    s = std::max<int64_t>(1, std::min<int64_t>((want + tc - 1) / tc, nc));
    *cpc = (int)((nc + s - 1) / s);
    *sc = (int)((nc + *cpc - 1) / *cpc);
}

template <typename TA>
cur_status sketch_launch(const cur_mat* A, const float* S, const float* T, float* Yp, float* Zp, int sr, int cpr,
                         int sc, int cpc, cudaStream_t st) {
    const TA* a = static_cast<const TA*>(A->data);
    const bool vec = (A->ld % 4 == 0) &&
                     (reinterpret_cast<uintptr_t>(A->data) % (4 * sizeof(TA)) == 0);
    const dim3 gr((unsigned)((A->rows + curk::kSkT - 1) / curk::kSkT), (unsigned)sr);
    curk::sk_rows_k<TA><<<gr, curk::kSkThreads, 0, st>>>(a, A->rows, A->cols, A->ld, vec, S, cpr, Yp);
    CUR_CK(cudaGetLastError());
    const dim3 gc((unsigned)((A->cols + curk::kSkT - 1) / curk::kSkT), (unsigned)sc);
    curk::sk_cols_k<TA><<<gc, curk::kSkThreads, 0, st>>>(a, A->rows, A->cols, A->ld, vec, T, cpc, Zp);
    CUR_CK(cudaGetLastError());
    note_launch(2);
    return CUR_OK;
}

bool aligned16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

int mlp_grid(int num_sms, int64_t N) {
    const int64_t chunks = (N + 31) / 32;
    return (int)std::max<int64_t>(1, std::min<int64_t>(chunks, num_sms));
}

bool mlp_shape_ok(int32_t k, int32_t H) { return k == curk::kSkK && H >= 32 && H <= curk::kMlpMaxH && H % 32 == 0; }

}  // namespace

size_t sketch_workspace_size(int num_sms, int64_t m, int64_t n) {
    int sr, cpr, sc, cpc;
    sketch_splits(num_sms, m, n, &sr, &cpr, &sc, &cpc);
    return sizeof(float) * curk::kSkK * ((size_t)sr * m + (size_t)sc * n) + 4096;
}

extern "C" {

cur_status cur_sketch(cur_handle* h, const cur_mat* A, const float* S, const float* T, int32_t k, float* Y,
                      float* Zt, int32_t normalize, cudaStream_t st) {
    if (!h || !A || !A->data || !S || !T || !Y || !Zt) return CUR_ERR_ARG;
    if (A->rows < 1 || A->cols < 1 || A->ld < A->cols) return CUR_ERR_ARG;
    if (A->dtype != CUR_F64 && A->dtype != CUR_F32 && A->dtype != CUR_BF16) return CUR_ERR_ARG;
    if (k != curk::kSkK) return CUR_ERR_ARG;
    if (!aligned16(S) || !aligned16(T) || !aligned16(Y) || !aligned16(Zt)) return CUR_ERR_ARG;
    const int64_t m = A->rows, n = A->cols;
    int sr, cpr, sc, cpc;
    sketch_splits(h->num_sms, m, n, &sr, &cpr, &sc, &cpc);
    Arena ar = h->arena();
    float* Yp = ar.get<float>((size_t)sr * m * curk::kSkK);
    float* Zp = ar.get<float>((size_t)sc * n * curk::kSkK);
    unsigned* mx = ar.get<unsigned>(2);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_CK(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned), st));
    if (A->dtype == CUR_F32) CUR_TRY(sketch_launch<float>(A, S, T, Yp, Zp, sr, cpr, sc, cpc, st));
    else if (A->dtype == CUR_BF16) CUR_TRY(sketch_launch<__nv_bfloat16>(A, S, T, Yp, Zp, sr, cpr, sc, cpc, st));
    else CUR_TRY(sketch_launch<double>(A, S, T, Yp, Zp, sr, cpr, sc, cpc, st));
    const int tb = 256;
    curk::sk_reduce_k<<<(unsigned)((8 * m + tb - 1) / tb), tb, 0, st>>>(Yp, sr, m, Y, mx);
    CUR_CK(cudaGetLastError());
    curk::sk_reduce_k<<<(unsigned)((8 * n + tb - 1) / tb), tb, 0, st>>>(Zp, sc, n, Zt, mx + 1);
    CUR_CK(cudaGetLastError());
    note_launch(2);
    if (normalize) {
        const unsigned g = (unsigned)std::max(1, 4 * h->num_sms);
        curk::sk_scale_k<<<g, tb, 0, st>>>(Y, m * curk::kSkK, mx);
        CUR_CK(cudaGetLastError());
        curk::sk_scale_k<<<g, tb, 0, st>>>(Zt, n * curk::kSkK, mx + 1);
        CUR_CK(cudaGetLastError());
        note_launch(2);
    }
    return CUR_OK;
}

cur_status cur_mlp_forward(cur_handle* h, const float* X, int64_t N, int32_t k, int32_t H, const float* params,
                           float* scores, cudaStream_t st) {
    if (!h || !X || !params || !scores || N < 1 || !mlp_shape_ok(k, H) || !aligned16(X)) return CUR_ERR_ARG;
    curk::mlp_fwd_k<<<(unsigned)std::min<int64_t>((N + 31) / 32, 8LL * h->num_sms), H, 0, st>>>(X, N, params, H,
                                                                                                   scores);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_mlp_grad(cur_handle* h, const float* X, const float* y, int64_t nrows, const int64_t* idx, int64_t N,
                        int32_t k, int32_t H, const float* params, float pos_weight, float* grads, double* loss,
                        cudaStream_t st) {
    if (!h || !X || !y || !params || !grads || N < 1 || nrows < 1 || !mlp_shape_ok(k, H) || !aligned16(X))
        return CUR_ERR_ARG;
    if (!idx && N > nrows) return CUR_ERR_ARG;
    if (!(pos_weight > 0.f)) return CUR_ERR_ARG;
    const int nb = mlp_grid(h->num_sms, N);
    const int64_t Pn = (int64_t)k * H + 2 * H + 1;
    Arena ar = h->arena();
    float* gp = ar.get<float>((size_t)nb * (Pn + 1));
    if (!ar.ok) return CUR_ERR_NOMEM;
    curk::mlp_grad_k<<<nb, H, 0, st>>>(X, y, idx, N, nrows, params, H, pos_weight, (float)(1.0 / (double)N), gp,
                                       h->status);
    CUR_CK(cudaGetLastError());
    curk::mlp_grad_reduce_k<<<(unsigned)((Pn + 1 + 255) / 256), 256, 0, st>>>(gp, nb, Pn, grads, loss);
    CUR_CK(cudaGetLastError());
    note_launch(2);
    return CUR_OK;
}

cur_status cur_adam_step(cur_handle* h, float* params, const float* grads, float* m1, float* m2, int64_t count,
                         int32_t t, float lr, float beta1, float beta2, float eps, cudaStream_t st) {
    if (!h || !params || !grads || !m1 || !m2 || count < 1 || t < 1) return CUR_ERR_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f)) return CUR_ERR_ARG;
    const float c1 = (float)(1.0 - pow((double)beta1, (double)t));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)t));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 4LL * h->num_sms));
    curk::adam_k<<<g, 256, 0, st>>>(params, grads, m1, m2, count, lr, beta1, beta2, eps, c1, c2);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_propose(cur_handle* h, const float* scores, int64_t N, int32_t r, int32_t* idx_out,
                       cudaStream_t st) {
    if (!h || !scores || !idx_out || r < 1 || N < r || N > 0x7fffffffLL) return CUR_ERR_ARG;
    curk::propose_k<<<1, 1024, 0, st>>>(scores, N, r, idx_out);
    CUR_CK(cudaGetLastError());
    note_launch();
    return CUR_OK;
}

cur_status cur_cross_from(cur_handle* h, const cur_mat* A, int32_t r, const int32_t* I0, const int32_t* J0,
                          const cur_opts* opts, int32_t* I_out, int32_t* J_out, cur_cross_info* info_out,
                          cudaStream_t st) {
    if (!h || !A || !A->data || !I0 || !J0 || !I_out || !J_out) return CUR_ERR_ARG;
    if (A->rows < 1 || A->cols < 1 || A->ld < A->cols) return CUR_ERR_ARG;
    if (A->dtype != CUR_F64 && A->dtype != CUR_F32 && A->dtype != CUR_BF16) return CUR_ERR_ARG;
    const int64_t m = A->rows, n = A->cols;
    if (r < 1 || r > 128 || r >= std::min(m, n)) return CUR_ERR_ARG;
    cur_opts o = opts ? *opts : cur_default_opts();
    if (!(o.delta >= 0.0)) return CUR_ERR_ARG;
    const int max_sweeps = 8;
    Arena ar = h->arena();
    const cur_dtype cdt = A->dtype == CUR_F64 ? CUR_F64 : CUR_F32;
    const size_t cs = compute_size(cdt);
    int32_t* I = ar.get<int32_t>(r);
    int32_t* J = ar.get<int32_t>(r);
    double* lv = ar.get<double>(1);
    double* lvr = ar.get<double>(1);
    double* Mr = ar.get<double>((size_t)minv_stride(r));
    double* Mc = ar.get<double>((size_t)minv_stride(r));
    void* Cb = ar.take((size_t)m * r * cs);
    void* Rb = ar.take((size_t)n * r * cs);
    CrossCtl* ctl = ar.get<CrossCtl>(1);
    if (!ar.ok) return CUR_ERR_NOMEM;
    CUR_CK(cudaMemcpyAsync(I, I0, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    CUR_CK(cudaMemcpyAsync(J, J0, sizeof(int32_t) * r, cudaMemcpyDeviceToDevice, st));
    // sweeps 1 .. 8 from the proposal (no inverse to inherit at first: mc_valid starts at 0)
    CUR_TRY(cross_begin(ctl, h->status, false, st));
    CUR_TRY(cross_sweeps(h, A, r, &o, 1, max_sweeps, true, I, J, Cb, Rb, Mr, Mc, lvr, lv, ctl, ar, st));
    return cross_end(h, A, r, true, I, J, Rb, lv, ctl, nullptr, I_out, J_out, info_out, ar, st);
}

}  // extern "C"
