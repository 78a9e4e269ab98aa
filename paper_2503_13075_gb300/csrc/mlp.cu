// mlp.cu -- learned warm start for the ILVES Newton solve.
//
// The paper starts Newton from lambda_0 = 0 (supplement Sec. 2.3).  This file adds a
// small network that predicts lambda_0 from local geometry, trained on multipliers of
// the plain solver; the Newton loop is unchanged and still decides convergence.
//
//   features  16 per constraint (own violation / alignment / masses, 4 line-graph
//             neighbour slots with their violation, coupling cosine and shared mass)
//   network   16 -> 128 -> ReLU -> 128 -> ReLU -> 1, bfloat16 weights and inputs,
//             float32 accumulation, on the tensor cores (mma.sync m16n8k16): the first
//             layer's accumulators are rounded to bfloat16 and reused in registers as the
//             second layer's A operand, the third layer is a quad-shuffle dot product
//   target    y = lambda * scale, scale = 4 (w_i + w_j) s.rho / d^2  -> lambda_0 = y / scale
//   training  forward on the tensor cores storing activations, backward on the float32
//             pipes (one thread per hidden unit, register accumulators, one atomic flush
//             per block), Adam on float32 master weights, bfloat16 copies refreshed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

#include "devmath.cuh"
#include "ilves.h"
#include "internal.h"
#include "topology_impl.h"

namespace ilves {

constexpr int NF = ILVES_MLP_FEATURES, NH = ILVES_MLP_HIDDEN;
constexpr int P_W1 = 0, P_B1 = P_W1 + NH * NF, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH,
              P_B3 = P_W3 + NH, P_N = P_B3 + 1;
static_assert(P_N == ILVES_MLP_PARAMS, "parameter count");
constexpr int W1_LD = NF + 8;   // padded shared-memory row (bf16) -> conflict-free B fragments
constexpr int W2_LD = NH + 8;
constexpr int FWD_WARPS = 4;

// ------------------------------------------------------------------------------------
// features
// ------------------------------------------------------------------------------------
struct FeatArgs {
    const double* x_old;
    const double* x_unc;
    const double* inv_mass;
    const double* d;
    const int32_t* con_i;
    const int32_t* con_j;
    const int32_t* nbr;
    const int32_t* nbr_atom;
    float4* ws_con;    // per constraint: (s.xyz, sigma0 / d^2), (rho.xyz, d)
    float* ws_atom;    // per atom: inverse mass
    int32_t n_c;
    int32_t n_atoms;
};

__device__ __forceinline__ float3 ld3(const double* x, int64_t a) {
    return make_float3(narrow(x[3 * a]), narrow(x[3 * a + 1]), narrow(x[3 * a + 2]));
}
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Prep pass: per-constraint float32 geometry and per-atom weights into the topology's
// warm-start workspace, so the feature stage gathers 32 bytes per neighbour instead of
// four float64 atom positions.
__global__ void k_ws_prep(FeatArgs F) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < F.n_c) {
        const int i = F.con_i[k], j = F.con_j[k];
        const float3 s = sub3(ld3(F.x_unc, i), ld3(F.x_unc, j));
        const float3 r = sub3(ld3(F.x_old, i), ld3(F.x_old, j));
        const float dk = narrow(F.d[k]), d2 = dk * dk;
        F.ws_con[2 * k] = make_float4(s.x, s.y, s.z, (dot3(s, s) - d2) / d2);
        F.ws_con[2 * k + 1] = make_float4(r.x, r.y, r.z, dk);
    }
    if (k < F.n_atoms) F.ws_atom[k] = narrow(F.inv_mass[k]);
}

// Features of constraint k from the workspace; `half` selects which half of the 16
// features this lane writes (two lanes per row): half 0 = own terms + slots 0-1,
// half 1 = slots 2-3 (the scale is produced by half 0).
__device__ __forceinline__ void ws_features(const FeatArgs& F, int k, int half, float* f, float& scale) {
    const float4 s4 = F.ws_con[2 * k], r4 = F.ws_con[2 * k + 1];
    const int i = F.con_i[k], j = F.con_j[k];
    const float wi = F.ws_atom[i], wj = F.ws_atom[j], W = wi + wj;
    const float inv_w = W > 0.f ? 1.0f / W : 0.f;
    const float dk = r4.w, inv_d2 = 1.0f / (dk * dk);
    const float3 s = make_float3(s4.x, s4.y, s4.z), r = make_float3(r4.x, r4.y, r4.z);
    const float sr = dot3(s, r);
    if (half == 0) {
        const float3 sm = sub3(s, r);
        f[0] = s4.w;
        f[1] = sr * inv_d2 - 1.0f;
        f[2] = (wi - wj) * inv_w;
        f[3] = dot3(sm, sm) * inv_d2;
        scale = 4.0f * W * sr * inv_d2;
    }
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * half + qq;
        const int l = F.nbr[4 * k + q];
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (l >= 0) {
            const int a = F.nbr_atom[4 * k + q];
            const float4 sl4 = F.ws_con[2 * l], rl4 = F.ws_con[2 * l + 1];
            const float sgn = ((a == i) == (a == F.con_i[l])) ? 1.f : -1.f;
            g0 = sl4.w;
            g1 = sgn * dot3(s, make_float3(rl4.x, rl4.y, rl4.z)) / (dk * rl4.w);
            g2 = F.ws_atom[a] * inv_w;
        }
        f[4 + 3 * q] = g0;
        f[5 + 3 * q] = g1;
        f[6 + 3 * q] = g2;
    }
}

__global__ void k_features(FeatArgs F, float* __restrict__ feat, float* __restrict__ scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F.n_c) return;
    float f[NF], sc = 0.f;
    ws_features(F, k, 0, f, sc);
    ws_features(F, k, 1, f, sc);
#pragma unroll
    for (int q = 0; q < NF; ++q) feat[(int64_t)k * NF + q] = f[q];
    if (scale) scale[k] = sc;
}

// Jacobi guess lambda_0 = sigma_0 / A_kk at x_unc (no network): y = f0, own terms only.
__global__ void k_diag_guess(FeatArgs F, float* __restrict__ lambda0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F.n_c) return;
    const int i = F.con_i[k], j = F.con_j[k];
    const float3 s = sub3(ld3(F.x_unc, i), ld3(F.x_unc, j));
    const float3 r = sub3(ld3(F.x_old, i), ld3(F.x_old, j));
    const float dk = narrow(F.d[k]), d2 = dk * dk;
    const float W = narrow(F.inv_mass[i]) + narrow(F.inv_mass[j]);
    const float a = 4.0f * W * dot3(s, r);
    const float l0 = (dot3(s, s) - d2) / a;
    lambda0[k] = (a != 0.f && isfinite(l0)) ? l0 : 0.f;
}

// ------------------------------------------------------------------------------------
// tensor-core forward
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float& d0, float& d1, float& d2, float& d3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct MlpWeights {
    const __nv_bfloat16* w1;  // [NH][NF]  (out x in) bfloat16
    const __nv_bfloat16* w2;  // [NH][NH]
    const float* params;      // float32 master parameters (biases, w3, b3 read from here)
};

// Input rows come either from a feature matrix (training / explicit inference) or are
// computed on the fly from the topology (fused warm start, output = lambda_0).
template <bool kFused, bool kTrain>
__global__ void __launch_bounds__(FWD_WARPS * 32)
k_mlp_forward(MlpWeights Wt, const float* __restrict__ X, int n, FeatArgs F, float* __restrict__ out,
              __nv_bfloat16* __restrict__ h1_out, float* __restrict__ h2_out) {
    __shared__ __align__(16) __nv_bfloat16 w1s[NH * W1_LD];
    __shared__ __align__(16) __nv_bfloat16 w2s[NH * W2_LD];
    __shared__ float b1s[NH], b2s[NH], w3s[NH];
    __shared__ float fs[FWD_WARPS][16][NF + 1];
    __shared__ float scs[FWD_WARPS][16];
    {  // stage the bfloat16 weights with 16-byte loads (8 values), all loads issued before the stores
        const uint4* g1 = reinterpret_cast<const uint4*>(Wt.w1);
        const uint4* g2 = reinterpret_cast<const uint4*>(Wt.w2);
        constexpr int N1 = NH * NF / 8, N2 = NH * NH / 8, PER = N2 / (FWD_WARPS * 32);
        uint4 v[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) v[u] = __ldg(g2 + threadIdx.x + u * FWD_WARPS * 32);
        for (int e = threadIdx.x; e < N1; e += blockDim.x) {
            const int row = (e * 8) / NF, col = (e * 8) % NF;
            *reinterpret_cast<uint4*>(w1s + row * W1_LD + col) = __ldg(g1 + e);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * FWD_WARPS * 32;
            const int row = (e * 8) / NH, col = (e * 8) % NH;
            *reinterpret_cast<uint4*>(w2s + row * W2_LD + col) = v[u];
        }
    }
    for (int e = threadIdx.x; e < NH; e += blockDim.x) {
        b1s[e] = Wt.params[P_B1 + e];
        b2s[e] = Wt.params[P_B2 + e];
        w3s[e] = Wt.params[P_W3 + e];
    }
    const float b3 = Wt.params[P_B3];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    const int n_tiles = (n + 15) / 16;
    for (int tile = blockIdx.x * FWD_WARPS + warp; tile < n_tiles; tile += gridDim.x * FWD_WARPS) {
        const int r0 = tile * 16;
        // ---- input rows into shared memory; in the fused mode two lanes build each row's
        //      features from the warm-start workspace (lane r: own terms + slots 0-1,
        //      lane r + 16: slots 2-3)
        {
            const int rl = lane & 15, half = lane >> 4, row = r0 + rl;
            float f[NF], sc = 0.f;
#pragma unroll
            for (int c = 0; c < NF; ++c) f[c] = 0.f;
            if (row < n) {
                if constexpr (kFused) {
                    ws_features(F, row, half, f, sc);
                } else if (half == 0) {
#pragma unroll
                    for (int c = 0; c < NF; ++c) f[c] = X[(int64_t)row * NF + c];
                }
            }
            if (half == 0) {
#pragma unroll
                for (int c = 0; c < 10; ++c) fs[warp][rl][c] = f[c];
                scs[warp][rl] = sc;
            }
            if (kFused ? half == 1 : half == 0) {
#pragma unroll
                for (int c = 10; c < NF; ++c) fs[warp][rl][c] = f[c];
            }
        }
        __syncwarp();
        const uint32_t a0 = pack_bf16(fs[warp][g][2 * q], fs[warp][g][2 * q + 1]);
        const uint32_t a1 = pack_bf16(fs[warp][g + 8][2 * q], fs[warp][g + 8][2 * q + 1]);
        const uint32_t a2 = pack_bf16(fs[warp][g][2 * q + 8], fs[warp][g][2 * q + 9]);
        const uint32_t a3 = pack_bf16(fs[warp][g + 8][2 * q + 8], fs[warp][g + 8][2 * q + 9]);
        // ---- layer 1: 16 n-tiles of 8 hidden units; ReLU; bfloat16 A operand of layer 2
        uint32_t h[NH / 16][4];
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) {
            const __nv_bfloat16* wrow = w1s + (8 * nt + g) * W1_LD;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wrow + 2 * q);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wrow + 2 * q + 8);
            const int c = 8 * nt + 2 * q;
            float d0 = b1s[c], d1 = b1s[c + 1], d2 = b1s[c], d3 = b1s[c + 1];
            mma_bf16(d0, d1, d2, d3, a0, a1, a2, a3, b0, b1);
            const uint32_t lo = pack_bf16(fmaxf(d0, 0.f), fmaxf(d1, 0.f));
            const uint32_t hi = pack_bf16(fmaxf(d2, 0.f), fmaxf(d3, 0.f));
            h[nt >> 1][(nt & 1) * 2 + 0] = lo;  // a0 / a2 of k-tile nt/2
            h[nt >> 1][(nt & 1) * 2 + 1] = hi;  // a1 / a3
            if constexpr (kTrain) {
                if (r0 + g < n) *reinterpret_cast<uint32_t*>(h1_out + (int64_t)(r0 + g) * NH + c) = lo;
                if (r0 + g + 8 < n) *reinterpret_cast<uint32_t*>(h1_out + (int64_t)(r0 + g + 8) * NH + c) = hi;
            }
        }
        // ---- layer 2 + layer 3
        float y_lo = 0.f, y_hi = 0.f;
#pragma unroll 4
        for (int nt = 0; nt < NH / 8; ++nt) {
            const int c = 8 * nt + 2 * q;
            float d0 = b2s[c], d1 = b2s[c + 1], d2 = b2s[c], d3 = b2s[c + 1];
            const __nv_bfloat16* wrow = w2s + (8 * nt + g) * W2_LD;
#pragma unroll
            for (int kt = 0; kt < NH / 16; ++kt) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wrow + 16 * kt + 2 * q);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wrow + 16 * kt + 2 * q + 8);
                mma_bf16(d0, d1, d2, d3, h[kt][0], h[kt][1], h[kt][2], h[kt][3], b0, b1);
            }
            d0 = fmaxf(d0, 0.f);
            d1 = fmaxf(d1, 0.f);
            d2 = fmaxf(d2, 0.f);
            d3 = fmaxf(d3, 0.f);
            y_lo = fmaf(d0, w3s[c], fmaf(d1, w3s[c + 1], y_lo));
            y_hi = fmaf(d2, w3s[c], fmaf(d3, w3s[c + 1], y_hi));
            if constexpr (kTrain) {
                if (r0 + g < n) *reinterpret_cast<float2*>(h2_out + (int64_t)(r0 + g) * NH + c) = make_float2(d0, d1);
                if (r0 + g + 8 < n) *reinterpret_cast<float2*>(h2_out + (int64_t)(r0 + g + 8) * NH + c) = make_float2(d2, d3);
            }
        }
        y_lo += __shfl_xor_sync(0xFFFFFFFFu, y_lo, 1);
        y_lo += __shfl_xor_sync(0xFFFFFFFFu, y_lo, 2);
        y_hi += __shfl_xor_sync(0xFFFFFFFFu, y_hi, 1);
        y_hi += __shfl_xor_sync(0xFFFFFFFFu, y_hi, 2);
        if (q == 0) {
            for (int half = 0; half < 2; ++half) {
                const int rl = g + 8 * half, row = r0 + rl;
                if (row >= n) continue;
                const float y = (half ? y_hi : y_lo) + b3;
                if constexpr (kFused) {
                    const float sc = scs[warp][rl];
                    const float l0 = y / sc;
                    out[row] = (sc != 0.f && isfinite(l0)) ? l0 : 0.f;
                } else {
                    out[row] = y;
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------
// float32 backward: one thread per hidden unit, rows streamed through shared memory
// ------------------------------------------------------------------------------------
constexpr int BWD_ROWS = 128;

__global__ void __launch_bounds__(NH)
k_mlp_backward(const float* __restrict__ X, const float* __restrict__ t, int n, const float* __restrict__ y,
               const __nv_bfloat16* __restrict__ h1, const float* __restrict__ h2, const __nv_bfloat16* __restrict__ w2b,
               const float* __restrict__ params, float* __restrict__ grad, float* __restrict__ loss) {
    __shared__ __nv_bfloat16 w2s[NH * NH];  // [c][k], the bfloat16 weights the forward used
    __shared__ float dz2s[NH], h1s[NH], xs[NF], dys;
    const int c = threadIdx.x;  // hidden unit of layer 2 (and of layer 1 for the input side)
    for (int e = c; e < NH * NH; e += NH) w2s[e] = w2b[e];
    const float w3c = params[P_W3 + c];
    float gw2[NH];
#pragma unroll
    for (int k = 0; k < NH; ++k) gw2[k] = 0.f;
    float gw1[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) gw1[f] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
    const float inv_n = 1.0f / (float)n;
    const int rb = blockIdx.x * BWD_ROWS, re = min(n, rb + BWD_ROWS);
    __syncthreads();
    for (int r = rb; r < re; ++r) {
        if (c == 0) {
            const float res = y[r] - t[r];
            dys = 2.0f * res * inv_n;
            lsum += res * res * inv_n;
        }
        h1s[c] = __bfloat162float(h1[(int64_t)r * NH + c]);
        if (c < NF) xs[c] = X[(int64_t)r * NF + c];
        __syncthreads();
        const float dy = dys;
        const float h2c = h2[(int64_t)r * NH + c];
        const float dz2 = h2c > 0.f ? dy * w3c : 0.f;
        gw3 += dy * h2c;
        gb2 += dz2;
        gb3 += dy;
        dz2s[c] = dz2;
#pragma unroll
        for (int k = 0; k < NH; ++k) gw2[k] = fmaf(dz2, h1s[k], gw2[k]);
        __syncthreads();
        // this thread now plays hidden unit k = c of layer 1
        float dh1 = 0.f;
#pragma unroll 8
        for (int cc = 0; cc < NH; ++cc) dh1 = fmaf(dz2s[cc], __bfloat162float(w2s[cc * NH + c]), dh1);
        const float dz1 = h1s[c] > 0.f ? dh1 : 0.f;
        gb1 += dz1;
#pragma unroll
        for (int f = 0; f < NF; ++f) gw1[f] = fmaf(dz1, xs[f], gw1[f]);
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NH; ++k) atomicAdd(grad + P_W2 + c * NH + k, gw2[k]);
#pragma unroll
    for (int f = 0; f < NF; ++f) atomicAdd(grad + P_W1 + c * NF + f, gw1[f]);
    atomicAdd(grad + P_B1 + c, gb1);
    atomicAdd(grad + P_B2 + c, gb2);
    atomicAdd(grad + P_W3 + c, gw3);
    if (c == 0) {
        atomicAdd(grad + P_B3, gb3);
        if (loss) atomicAdd(loss, lsum);
    }
}

__global__ void k_zero(float* __restrict__ p, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.f;
}

// Adam on the float32 master parameters; refreshes the bfloat16 weight copies.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1c, float b2c, __nv_bfloat16* __restrict__ w1b,
                       __nv_bfloat16* __restrict__ w2b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P_N) return;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / b1c) / (sqrtf(vi / b2c) + eps);
    p[i] = pi;
    if (i < P_B1) w1b[i - P_W1] = __float2bfloat16_rn(pi);
    else if (i >= P_W2 && i < P_B2) w2b[i - P_W2] = __float2bfloat16_rn(pi);
}

__global__ void k_refresh_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ w1b,
                               __nv_bfloat16* __restrict__ w2b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NH * NF) w1b[i] = __float2bfloat16_rn(p[P_W1 + i]);
    if (i < NH * NH) w2b[i] = __float2bfloat16_rn(p[P_W2 + i]);
}

}  // namespace ilves

using namespace ilves;

struct ilves_mlp {
    int32_t device = -1;
    int32_t max_batch = 0;
    int64_t step = 0;
    float* params = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;
    float* y = nullptr;
    __nv_bfloat16* w1b = nullptr;
    __nv_bfloat16* w2b = nullptr;
    __nv_bfloat16* h1 = nullptr;
    float* h2 = nullptr;
};

static ilves_status mlp_status(cudaError_t e) {
    if (e == cudaSuccess) return ILVES_OK;
    return e == cudaErrorMemoryAllocation ? ILVES_ERR_OOM : ILVES_ERR_CUDA;
}

static FeatArgs feat_args(const ilves_topology* T, const double* x_old, const double* x_unc, const double* inv_mass,
                          const double* d) {
    FeatArgs F;
    F.x_old = x_old;
    F.x_unc = x_unc;
    F.inv_mass = inv_mass;
    F.d = d;
    F.con_i = T->d_con_i;
    F.con_j = T->d_con_j;
    F.nbr = T->d_nbr;
    F.nbr_atom = T->d_nbr_atom;
    F.ws_con = reinterpret_cast<float4*>(T->d_ws_con);
    F.ws_atom = T->d_ws_atom;
    F.n_c = T->n_c;
    F.n_atoms = T->n_atoms;
    return F;
}

// one wave of persistent blocks (4 per SM fit the 47 KB of shared memory each)
static int fwd_grid(int n) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + 15) / 16;
    return std::max(1, std::min((tiles + FWD_WARPS - 1) / FWD_WARPS, sms * 4));
}

extern "C" int64_t ilves_mlp_param_count(void) { return P_N; }

extern "C" ilves_status ilves_mlp_create(int32_t max_batch, uint64_t seed, ilves_mlp** out) {
    if (!out || max_batch <= 0) return ILVES_ERR_INVALID_ARG;
    *out = nullptr;
    ilves_mlp* M = new ilves_mlp();
    cudaGetDevice(&M->device);
    M->max_batch = max_batch;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void**)&M->params, P_N * sizeof(float));
    alloc((void**)&M->m, P_N * sizeof(float));
    alloc((void**)&M->v, P_N * sizeof(float));
    alloc((void**)&M->grad, P_N * sizeof(float));
    alloc((void**)&M->loss, sizeof(float));
    alloc((void**)&M->y, (size_t)max_batch * sizeof(float));
    alloc((void**)&M->w1b, NH * NF * sizeof(__nv_bfloat16));
    alloc((void**)&M->w2b, NH * NH * sizeof(__nv_bfloat16));
    alloc((void**)&M->h1, (size_t)max_batch * NH * sizeof(__nv_bfloat16));
    alloc((void**)&M->h2, (size_t)max_batch * NH * sizeof(float));
    if (e != cudaSuccess) {
        ilves_mlp_destroy(M);
        return mlp_status(e);
    }
    // He-uniform weights, zero biases
    std::vector<float> h(P_N, 0.f);
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<float> u(-1.f, 1.f);
    for (int i = 0; i < NH * NF; ++i) h[P_W1 + i] = u(rng) * std::sqrt(6.f / NF);
    for (int i = 0; i < NH * NH; ++i) h[P_W2 + i] = u(rng) * std::sqrt(6.f / NH);
    for (int i = 0; i < NH; ++i) h[P_W3 + i] = u(rng) * std::sqrt(3.f / NH);
    ilves_status s = ilves_mlp_set_params(M, h.data());
    if (s != ILVES_OK) {
        ilves_mlp_destroy(M);
        return s;
    }
    *out = M;
    return ILVES_OK;
}

extern "C" void ilves_mlp_destroy(ilves_mlp* M) {
    if (!M) return;
    for (void* p : {(void*)M->params, (void*)M->m, (void*)M->v, (void*)M->grad, (void*)M->loss, (void*)M->y,
                    (void*)M->w1b, (void*)M->w2b, (void*)M->h1, (void*)M->h2})
        if (p) cudaFree(p);
    delete M;
}

extern "C" ilves_status ilves_mlp_set_params(ilves_mlp* M, const float* host_params) {
    if (!M || !host_params) return ILVES_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(M->params, host_params, P_N * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->m, 0, P_N * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(M->v, 0, P_N * sizeof(float));
    if (e != cudaSuccess) return mlp_status(e);
    M->step = 0;
    k_refresh_bf16<<<(NH * NH + 255) / 256, 256>>>(M->params, M->w1b, M->w2b);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return mlp_status(e);
}

extern "C" ilves_status ilves_mlp_get_params(const ilves_mlp* M, float* host_params) {
    if (!M || !host_params) return ILVES_ERR_INVALID_ARG;
    return mlp_status(cudaMemcpy(host_params, M->params, P_N * sizeof(float), cudaMemcpyDeviceToHost));
}

extern "C" ilves_status ilves_mlp_features(const ilves_topology* T, const double* x_old, const double* x_unc,
                                           const double* inv_mass, const double* d, float* features, float* scale,
                                           void* stream) {
    if (!T || !T->on_device || !features) return ILVES_ERR_INVALID_ARG;
    if (T->n_c == 0) return ILVES_OK;
    if (!x_old || !x_unc || !inv_mass || !d) return ILVES_ERR_INVALID_ARG;
    const FeatArgs F = feat_args(T, x_old, x_unc, inv_mass, d);
    const int np = std::max(T->n_c, T->n_atoms);
    k_ws_prep<<<(np + 255) / 256, 256, 0, (cudaStream_t)stream>>>(F);
    k_features<<<(T->n_c + 127) / 128, 128, 0, (cudaStream_t)stream>>>(F, features, scale);
    return mlp_status(cudaGetLastError());
}

extern "C" ilves_status ilves_mlp_forward(const ilves_mlp* M, const float* features, int32_t n, float* y,
                                          void* stream) {
    if (!M || n < 0 || (n > 0 && (!features || !y))) return ILVES_ERR_INVALID_ARG;
    if (n == 0) return ILVES_OK;
    const MlpWeights Wt{M->w1b, M->w2b, M->params};
    FeatArgs F{};
    k_mlp_forward<false, false><<<fwd_grid(n), FWD_WARPS * 32, 0, (cudaStream_t)stream>>>(Wt, features, n, F, y,
                                                                                           nullptr, nullptr);
    return mlp_status(cudaGetLastError());
}

extern "C" ilves_status ilves_warm_start(const ilves_mlp* M, const ilves_topology* T, const double* x_old,
                                         const double* x_unc, const double* inv_mass, const double* d,
                                         float* lambda0, void* stream) {
    if (!T || !T->on_device || (T->n_c > 0 && !lambda0)) return ILVES_ERR_INVALID_ARG;
    if (T->n_c == 0) return ILVES_OK;
    if (!x_old || !x_unc || !inv_mass || !d) return ILVES_ERR_INVALID_ARG;
    const FeatArgs F = feat_args(T, x_old, x_unc, inv_mass, d);
    if (!M) {
        k_diag_guess<<<(T->n_c + 127) / 128, 128, 0, (cudaStream_t)stream>>>(F, lambda0);
    } else {
        const MlpWeights Wt{M->w1b, M->w2b, M->params};
        const int np = std::max(T->n_c, T->n_atoms);
        k_ws_prep<<<(np + 255) / 256, 256, 0, (cudaStream_t)stream>>>(F);
        k_mlp_forward<true, false><<<fwd_grid(T->n_c), FWD_WARPS * 32, 0, (cudaStream_t)stream>>>(
            Wt, nullptr, T->n_c, F, lambda0, nullptr, nullptr);
    }
    return mlp_status(cudaGetLastError());
}

// forward with stored activations + backward into M->grad (and the loss into M->loss)
static ilves_status mlp_gradient(ilves_mlp* M, const float* X, const float* t, int32_t n, cudaStream_t s) {
    const MlpWeights Wt{M->w1b, M->w2b, M->params};
    FeatArgs F{};
    k_mlp_forward<false, true><<<fwd_grid(n), FWD_WARPS * 32, 0, s>>>(Wt, X, n, F, M->y, M->h1, M->h2);
    k_zero<<<(P_N + 255) / 256, 256, 0, s>>>(M->grad, P_N);
    k_zero<<<1, 32, 0, s>>>(M->loss, 1);
    k_mlp_backward<<<(n + BWD_ROWS - 1) / BWD_ROWS, NH, 0, s>>>(X, t, n, M->y, M->h1, M->h2, M->w2b, M->params,
                                                               M->grad, M->loss);
    return mlp_status(cudaGetLastError());
}

extern "C" ilves_status ilves_mlp_gradient(ilves_mlp* M, const float* features, const float* target, int32_t n,
                                           float* grad_out, float* loss_out, void* stream) {
    if (!M || n <= 0 || n > M->max_batch || !features || !target) return ILVES_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    ilves_status st = mlp_gradient(M, features, target, n, s);
    if (st != ILVES_OK) return st;
    cudaError_t e = cudaSuccess;
    if (grad_out) e = cudaMemcpyAsync(grad_out, M->grad, P_N * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, M->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return mlp_status(e);
}

extern "C" ilves_status ilves_mlp_train_step(ilves_mlp* M, const float* features, const float* target, int32_t n,
                                             float lr, float* loss_out, void* stream) {
    if (!M || n <= 0 || n > M->max_batch || !features || !target || !(lr >= 0.f)) return ILVES_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    ilves_status st = mlp_gradient(M, features, target, n, s);
    if (st != ILVES_OK) return st;
    M->step += 1;
    const float b1c = 1.f - std::pow(0.9f, (float)M->step), b2c = 1.f - std::pow(0.999f, (float)M->step);
    k_adam<<<(P_N + 255) / 256, 256, 0, s>>>(M->params, M->m, M->v, M->grad, lr, b1c, b2c, M->w1b, M->w2b);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, M->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return mlp_status(e);
}
