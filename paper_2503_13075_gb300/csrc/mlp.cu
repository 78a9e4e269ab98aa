// mlp.cu -- learned warm start for the ILVES Newton solve.
//
// The paper starts Newton from lambda_0 = 0 (supplement Sec. 2.3).  This file adds a
// small network that predicts lambda_0 from local geometry, trained on multipliers of
// the plain solver; the Newton loop is unchanged and still decides convergence.
//
//   features  16 per constraint (own violation / alignment / masses, 4 line-graph
//             neighbour slots with their violation, coupling cosine and shared mass)
//   network   16 -> 128 -> ReLU -> 128 -> ReLU -> 1, bfloat16 weights and inputs,
//             float32 accumulation, on the 5th-generation tensor cores (tcgen05.mma,
//             operands in shared memory, accumulators in tensor memory): per 128-row tile
//             one MMA for layer 1, its epilogue writes the bfloat16 A tile of layer 2
//             (eight MMAs), whose epilogue does the third layer as a per-row dot product
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
constexpr int TILE = 128;  // rows per tensor-core tile (M of the MMA), one thread per row

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
// tensor-core forward (tcgen05: operands in shared memory, accumulators in tensor memory)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

struct MlpWeights {
    const __nv_bfloat16* w1;  // [NH][NF]  (out x in) bfloat16
    const __nv_bfloat16* w2;  // [NH][NH]
    const float* params;      // float32 master parameters (biases, w3, b3 read from here)
};

// Operand tiles use the tensor cores' canonical K-major layout without swizzling: the
// tile is cut into core matrices of 8 rows x 16 bytes (8 bfloat16 of K), each stored as
// 128 contiguous bytes; core (row group g, K chunk c) sits at g * SBO + c * 128.
__device__ __forceinline__ uint32_t core_offset(int row, int kchunk, int kchunks) {
    return (uint32_t)((row >> 3) * (kchunks * 128) + kchunk * 128 + (row & 7) * 16);
}
// shared-memory matrix descriptor: start >> 4, leading (K) byte offset >> 4, stride (row
// group) byte offset >> 4, descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: f32 accumulator (bits 4-5 = 1), bf16 A and B (bits
// 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NH >> 3) << 17) |
                                ((uint32_t)(TILE >> 4) << 24);
// one 128-column accumulator: layer 2 reuses the columns once layer 1's epilogue has
// moved them to shared memory
constexpr uint32_t kTmemCols = NH;

__device__ __forceinline__ uint32_t saddr_of(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
// bounded wait for the mbarrier phase of the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
// 32 consecutive accumulator columns of this thread's row (warp w reads lanes 32w..32w+31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// shared-memory plan of the forward kernel (bytes from a 128-byte aligned base); about
// 74 KB, so at most three CTAs share an SM and their tensor memory (3 x 128 of 512
// columns) always fits
constexpr uint32_t SM_W1 = 0, SM_W2 = SM_W1 + NH * NF * 2, SM_A1 = SM_W2 + NH * NH * 2,
                   SM_A2 = SM_A1 + TILE * NF * 2, SM_B = SM_A2 + TILE * NH * 2, SM_BAR = SM_B + 3 * NH * 4,
                   SM_USED = SM_BAR + 16;
constexpr uint32_t SM_REQUEST = SM_USED + 128;
static_assert(4 * (SM_REQUEST + 1024) > 228 * 1024 && kTmemCols * 3 <= 512, "at most three CTAs per SM");

// Persistent forward over 128-row tiles.  Per tile: rows -> bfloat16 A tile; one MMA
// (K = 16) into the 128 tensor-memory columns; epilogue (+b1, ReLU, bfloat16) writes the
// second A tile; eight MMAs (K = 128) into the same columns; epilogue (+b2, ReLU, dot
// with w3, +b3) gives y.  One thread per row: thread t of warp w owns row 32 w + t, which
// is tensor-memory lane 32 w + t.  Input rows come from a feature matrix or, fused, are
// built from the topology (output lambda_0 = y / scale); in training mode the hidden
// activations are stored for the backward pass.  A wait that gives up counts in *err and
// ends the kernel after freeing its tensor memory.
template <bool kFused, bool kTrain>
__global__ void __launch_bounds__(TILE)
k_mlp_forward(MlpWeights Wt, const float* __restrict__ X, int n, FeatArgs F, float* __restrict__ out,
              __nv_bfloat16* __restrict__ h1_out, float* __restrict__ h2_out, int* __restrict__ err,
              int wait_test) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float* b1s = reinterpret_cast<float*>(sm + SM_B);
    float* b2s = b1s + NH;
    float* w3s = b2s + NH;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + SM_BAR);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar = saddr_of(bar);
    if (warp == 0) {  // 256 tensor-memory columns for this CTA
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr_of(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights into the canonical layout: 16-byte chunks of 8 K values
    for (int e = tid; e < NH * NF / 8; e += TILE) {
        const int row = e / (NF / 8), kc = e % (NF / 8);
        *reinterpret_cast<uint4*>(sm + SM_W1 + core_offset(row, kc, NF / 8)) =
            __ldg(reinterpret_cast<const uint4*>(Wt.w1) + e);
    }
    for (int e = tid; e < NH * NH / 8; e += TILE) {
        const int row = e / (NH / 8), kc = e % (NH / 8);
        *reinterpret_cast<uint4*>(sm + SM_W2 + core_offset(row, kc, NH / 8)) =
            __ldg(reinterpret_cast<const uint4*>(Wt.w2) + e);
    }
    for (int e = tid; e < NH; e += TILE) {
        b1s[e] = Wt.params[P_B1 + e];
        b2s[e] = Wt.params[P_B2 + e];
        w3s[e] = Wt.params[P_W3 + e];
    }
    const float b3 = Wt.params[P_B3];
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_lane = (uint32_t)(32 * warp) << 16;
    const uint64_t dA1 = smem_desc(saddr_of(sm + SM_A1), 128, (NF / 8) * 128);
    const uint64_t dW1 = smem_desc(saddr_of(sm + SM_W1), 128, (NF / 8) * 128);
    const uint64_t dA2 = smem_desc(saddr_of(sm + SM_A2), 128, (NH / 8) * 128);
    const uint64_t dW2 = smem_desc(saddr_of(sm + SM_W2), 128, (NH / 8) * 128);
    uint32_t parity = 0;
    bool ok = true;
    const int n_tiles = (n + TILE - 1) / TILE;
    if (wait_test) {  // testing: wait on a phase nothing completes (no MMA in flight), so the wait runs out
        ok = __syncthreads_and(mbar_wait(mbar, parity)) != 0;
    }
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int row = tile * TILE + tid;
        // ---- input row -> bfloat16 A tile
        float f[NF], sc = 0.f;
#pragma unroll
        for (int c = 0; c < NF; ++c) f[c] = 0.f;
        if (row < n) {
            if constexpr (kFused) {
                ws_features(F, row, 0, f, sc);
                ws_features(F, row, 1, f, sc);
            } else {
                const float4* xr = reinterpret_cast<const float4*>(X + (int64_t)row * NF);
#pragma unroll
                for (int c = 0; c < NF / 4; ++c) {
                    const float4 v = __ldg(xr + c);
                    f[4 * c] = v.x;
                    f[4 * c + 1] = v.y;
                    f[4 * c + 2] = v.z;
                    f[4 * c + 3] = v.w;
                }
            }
        }
#pragma unroll
        for (int kc = 0; kc < NF / 8; ++kc)
            *reinterpret_cast<uint4*>(sm + SM_A1 + core_offset(tid, kc, NF / 8)) =
                make_uint4(pack_bf16(f[8 * kc], f[8 * kc + 1]), pack_bf16(f[8 * kc + 2], f[8 * kc + 3]),
                           pack_bf16(f[8 * kc + 4], f[8 * kc + 5]), pack_bf16(f[8 * kc + 6], f[8 * kc + 7]));
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 1: one MMA, K = 16
        if (tid == 0) {
            tc_mma(tmem, dA1, dW1, 0u);
            tc_commit(mbar);
        }
        ok = __syncthreads_and(mbar_wait(mbar, parity)) != 0;  // one decision for the whole CTA
        parity ^= 1u;
        tc_fence_after();
        if (!ok) break;
#pragma unroll 1
        for (int ch = 0; ch < NH / 32; ++ch) {
            float v[32];
            tmem_ld32(tmem + t_lane + 32 * ch, v);
            uint32_t hb[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
                hb[j] = pack_bf16(fmaxf(v[2 * j] + b1s[32 * ch + 2 * j], 0.f),
                                  fmaxf(v[2 * j + 1] + b1s[32 * ch + 2 * j + 1], 0.f));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 u = make_uint4(hb[4 * q], hb[4 * q + 1], hb[4 * q + 2], hb[4 * q + 3]);
                *reinterpret_cast<uint4*>(sm + SM_A2 + core_offset(tid, 4 * ch + q, NH / 8)) = u;
                if constexpr (kTrain) {
                    if (row < n) reinterpret_cast<uint4*>(h1_out + (int64_t)row * NH + 32 * ch)[q] = u;
                }
            }
        }
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 2: eight MMAs along K = 128 (16 per step: two core matrices, 256 bytes)
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NH / 16; ++k) tc_mma(tmem, dA2 + (uint64_t)(k * 16), dW2 + (uint64_t)(k * 16), k > 0);
            tc_commit(mbar);
        }
        ok = __syncthreads_and(mbar_wait(mbar, parity)) != 0;
        parity ^= 1u;
        tc_fence_after();
        if (!ok) break;
        float y = 0.f;
#pragma unroll 1
        for (int ch = 0; ch < NH / 32; ++ch) {
            float v[32];
            tmem_ld32(tmem + t_lane + 32 * ch, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                v[j] = fmaxf(v[j] + b2s[32 * ch + j], 0.f);
                y = fmaf(v[j], w3s[32 * ch + j], y);
            }
            if constexpr (kTrain) {
                if (row < n) {
                    float4* h2r = reinterpret_cast<float4*>(h2_out + (int64_t)row * NH + 32 * ch);
#pragma unroll
                    for (int q = 0; q < 8; ++q) h2r[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
        if (row < n) {
            y += b3;
            if constexpr (kFused) {
                const float l0 = y / sc;
                out[row] = (sc != 0.f && isfinite(l0)) ? l0 : 0.f;
            } else {
                out[row] = y;
            }
        }
        tc_fence_before();
    }
    if (!ok && tid == 0) atomicAdd(err, 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                                : "memory");
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
    int* err = nullptr;  // tensor-core waits that gave up (see ilves_mlp_check)
    int32_t wait_test = 0;  // testing: forward kernels wait on a phase nothing completes
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

// Launches the tensor-core forward: persistent CTAs, at most three per SM (the shared
// memory request guarantees it), one 128-row tile at a time.
template <bool kFused, bool kTrain>
static cudaError_t launch_forward(const MlpWeights& Wt, const float* X, int n, const FeatArgs& F, float* out,
                                  __nv_bfloat16* h1, float* h2, int* err, int wait_test, cudaStream_t s) {
    static bool attr_set[64] = {};
    int dev = 0, sms = 152;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(k_mlp_forward<kFused, kTrain>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SM_REQUEST);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const int tiles = (n + TILE - 1) / TILE;
    const int grid = std::max(1, std::min(tiles, 3 * sms));
    k_mlp_forward<kFused, kTrain><<<grid, TILE, SM_REQUEST, s>>>(Wt, X, n, F, out, h1, h2, err, wait_test);
    return cudaGetLastError();
}

extern "C" int64_t ilves_mlp_param_count(void) { return P_N; }

extern "C" ilves_status ilves_mlp_check(const ilves_mlp* M, int32_t* waits_given_up) {
    if (!M || !waits_given_up) return ILVES_ERR_INVALID_ARG;
    int v = 0;
    const cudaError_t e = cudaMemcpy(&v, M->err, sizeof(int), cudaMemcpyDeviceToHost);
    *waits_given_up = v;
    if (e != cudaSuccess) return mlp_status(e);
    return v ? ILVES_ERR_TIMEOUT : ILVES_OK;
}

extern "C" ilves_status ilves_mlp_set_wait_test(ilves_mlp* M, int32_t on) {
    if (!M) return ILVES_ERR_INVALID_ARG;
    M->wait_test = on ? 1 : 0;
    return ILVES_OK;
}

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
    alloc((void**)&M->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(M->err, 0, sizeof(int));
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
                    (void*)M->w1b, (void*)M->w2b, (void*)M->h1, (void*)M->h2, (void*)M->err})
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
    if (reinterpret_cast<uintptr_t>(features) & 15u) return ILVES_ERR_INVALID_ARG;
    const MlpWeights Wt{M->w1b, M->w2b, M->params};
    FeatArgs F{};
    return mlp_status(
        launch_forward<false, false>(Wt, features, n, F, y, nullptr, nullptr, M->err, M->wait_test, (cudaStream_t)stream));
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
        const cudaError_t e =
            launch_forward<true, false>(Wt, nullptr, T->n_c, F, lambda0, nullptr, nullptr, M->err, M->wait_test,
                                        (cudaStream_t)stream);
        if (e != cudaSuccess) return mlp_status(e);
    }
    return mlp_status(cudaGetLastError());
}

// forward with stored activations + backward into M->grad (and the loss into M->loss)
static ilves_status mlp_gradient(ilves_mlp* M, const float* X, const float* t, int32_t n, cudaStream_t s) {
    const MlpWeights Wt{M->w1b, M->w2b, M->params};
    FeatArgs F{};
    if (reinterpret_cast<uintptr_t>(X) & 15u) return ILVES_ERR_INVALID_ARG;
    const cudaError_t e = launch_forward<false, true>(Wt, X, n, F, M->y, M->h1, M->h2, M->err, M->wait_test, s);
    if (e != cudaSuccess) return mlp_status(e);
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
