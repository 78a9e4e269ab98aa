// solve.cu -- sm_103a kernels and C ABI of the ILVES-M constraint solver.
//
// One Newton solve per molecule (supplement Sec. 2.3, ILVES-M):
//   S1  rho_k = x_old,i - x_old,j;  x = x_unc - M^-1 G(x_old)^T lambda0
//   S2  sigma_k = |x_i - x_j|^2 - d_k^2; stop when max |sigma_k| / d_k^2 <= tol (Sec. 4)
//   S3  A = G(x) M^-1 G(x_old)^T assembled on the fly inside the factor tasks:
//         A_kk = 4 (w_i + w_j) r_k . rho_k,   A_kl = 4 s_k(a) s_l(a) w_a r_k . rho_l
//   S4  sparse LU (Crout form Lt * Ut) in the planner's elimination order, level by level
//   S5  forward substitution fused into the DIAG tasks, backward substitution by level;
//       lambda += delta
//   S6  x_a -= w_a sum_{k at a} s_k(a) 2 delta_k rho_k;  back to S2
// All of a molecule's state lives next to its program: in shared memory for molecules
// run by one warp (the batched persistent kernel), in a global workspace for large
// molecules run by a whole CTA.  No host round trip happens inside the Newton loop.
//
// Precision modes: FP64 runs every step in float64.  MIXED keeps S2, the lambda
// accumulation and S6 in float64 and runs S3-S5 in float32 (the outer Newton loop is
// the iterative refinement).  On this GPU the float64 pipe issues about two FMAs per
// clock per SM and also executes f64<->f32 conversions, so the conversions between
// the two precisions are done with integer bit operations (exact widening, truncating
// narrowing) instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ilves.h"
#include "internal.h"
#include "topology_impl.h"
#include "devmath.cuh"

namespace ilves {

// ------------------------------------------------------------------------------------
// precision policies
// ------------------------------------------------------------------------------------
struct ModeFP64 {
    using LP = double;
    struct V4 { double x, y, z, w; };
    static constexpr int id = ILVES_PREC_FP64;
    static constexpr bool df = false;
    static constexpr double pivot_rel = 1e-13;
};
struct ModeMixed {
    using LP = float;
    using V4 = float4;
    static constexpr int id = ILVES_PREC_MIXED;
    static constexpr bool df = false;
    static constexpr float pivot_rel = 1e-5f;
};
struct ModeMixedDF {
    using LP = float;
    using V4 = float4;
    static constexpr int id = ILVES_PREC_MIXED_DF;
    static constexpr bool df = true;
    static constexpr float pivot_rel = 1e-5f;
};

template <class LP> __device__ __forceinline__ LP to_lp(double v);
template <> __device__ __forceinline__ float to_lp<float>(double v) { return narrow(v); }
template <> __device__ __forceinline__ double to_lp<double>(double v) { return v; }
__device__ __forceinline__ double to_hp(float v) { return widen(v); }
__device__ __forceinline__ double to_hp(double v) { return v; }

// |s| <= t for t >= 0 by comparing bit patterns (NaN compares false)
__device__ __forceinline__ bool abs_le(double s, double t) {
    const long long sb = __double_as_longlong(s) & 0x7FFFFFFFFFFFFFFFll;
    return sb <= __double_as_longlong(t);
}
__device__ __forceinline__ bool nonfinite(double s) {
    return (__double_as_longlong(s) & 0x7FF0000000000000ll) == 0x7FF0000000000000ll;
}
__device__ __forceinline__ bool nonfinite(float s) { return (__float_as_uint(s) & 0x7F800000u) == 0x7F800000u; }
__device__ __forceinline__ float lp_abs(float v) { return fabsf(v); }
__device__ __forceinline__ double lp_abs(double v) { return fabs(v); }
__device__ __forceinline__ float lp_rcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double lp_rcp(double a) { return 1.0 / a; }

// ------------------------------------------------------------------------------------
// float-float arithmetic: a value is the unevaluated sum hi + lo of two float32 words
// with |lo| <= ulp(hi) / 2.  Building blocks: Knuth's two-sum, Dekker's fast two-sum
// (|a| >= |b|) and the FMA-based exact product.  Additions use the short form
// (two-sum of the high words, low words added once): its absolute error is about
// 2^-24 |lo| parts, i.e. 2^-48 of the operands, which is what the error budget of the
// displacement formulation needs.
// ------------------------------------------------------------------------------------
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    fast_two_sum(s, e, s, e);
    return {s, e};
}
__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) { return df_add(a, dfloat{-b.hi, -b.lo}); }
__device__ __forceinline__ dfloat df_add_f(dfloat a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e = __fadd_rn(e, a.lo);
    fast_two_sum(s, e, s, e);
    return {s, e};
}
__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    fast_two_sum(p, e, p, e);
    return {p, e};
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    fast_two_sum(p, e, p, e);
    return {p, e};
}
// float64 -> float-float: hi = the truncated leading 24 bits (integer pipe), lo = the
// rounded remainder (one float64 subtraction)
__device__ __forceinline__ dfloat df_split(double v) {
    const float hi = narrow(v);
    return {hi, __double2float_rn(v - widen(hi))};
}
__device__ __forceinline__ double df_join(dfloat a) { return widen(a.hi) + widen(a.lo); }
__device__ __forceinline__ dfloat as_df(double v) { return *reinterpret_cast<dfloat*>(&v); }
__device__ __forceinline__ double as_bits(dfloat v) { return *reinterpret_cast<double*>(&v); }

// ------------------------------------------------------------------------------------
// teams
// ------------------------------------------------------------------------------------
struct WarpTeam {
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ bool all(bool p) const { return __all_sync(0xFFFFFFFFu, p); }
    __device__ __forceinline__ bool any(bool p) const { return __any_sync(0xFFFFFFFFu, p); }
};
struct BlockTeam {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool all(bool p) const { return __syncthreads_and(p) != 0; }
    __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
};

struct SolveArgs {
    const double* x_old;
    const double* x_unc;
    const double* inv_mass;
    const double* d;
    const float* lambda0;
    double* x_out;
    double* lambda_out;
    int32_t* iterations_out;
    int32_t* status_out;
    const int32_t* atom_gid;
    double tol;
    int32_t max_iter;
};

// ------------------------------------------------------------------------------------
// one molecule, one team
// ------------------------------------------------------------------------------------
// Float64-class arrays (X, W, RHO, S, D2, LAM) hold float64 values, or in the
// float-float mode dfloat pairs stored in the same 8 bytes.  In the float64 modes X
// holds absolute positions; in the float-float mode it holds displacements x - x_unc
// and S holds s_k = x_unc,i - x_unc,j, so that r_k = s_k + (dx_i - dx_j).
template <class Mode, class IdxT, class Team>
__device__ void solve_molecule(const Team& tm, const MolDesc& D, const uint8_t* prog, uint8_t* st,
                               const SolveArgs& A) {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    constexpr bool DF = Mode::df;
    const int na = D.na, nc = D.nc;
    const ProgLayout PL = prog_layout<IdxT>(na, nc, D.ntask, D.nterm, D.nlevel);
    const StateLayout SL = state_layout(na, nc, D.ntask, sizeof(LP), DF);
    const ConA<IdxT>* con = reinterpret_cast<const ConA<IdxT>*>(prog + PL.con_atoms);
    const int32_t* con_gid = reinterpret_cast<const int32_t*>(prog + PL.con_gid);
    const Piv<IdxT>* piv = reinterpret_cast<const Piv<IdxT>*>(prog + PL.piv);
    const IdxT* lvl_task = reinterpret_cast<const IdxT*>(prog + PL.lvl_task);
    const IdxT* lvl_piv = reinterpret_cast<const IdxT*>(prog + PL.lvl_piv);
    const IdxT* inc_ptr = reinterpret_cast<const IdxT*>(prog + PL.inc_ptr);
    const IdxT* inc = reinterpret_cast<const IdxT*>(prog + PL.inc);
    const Task<IdxT>* tasks = reinterpret_cast<const Task<IdxT>*>(prog + PL.tasks);
    using TO = TermOf<IdxT>;
    const typename TO::T* terms = reinterpret_cast<const typename TO::T*>(prog + PL.terms);
    double* X = reinterpret_cast<double*>(st + SL.x);  // SoA x | y | z
    double* W = reinterpret_cast<double*>(st + SL.w);
    LP* WL = reinterpret_cast<LP*>(st + SL.wl);  // assembly weights (factor precision)
    double* RHO = reinterpret_cast<double*>(st + SL.rho);  // SoA
    double* SK = reinterpret_cast<double*>(st + SL.s);     // SoA (float-float mode)
    double* D2 = reinterpret_cast<double*>(st + SL.d2);
    const double tol = A.tol;
    const float tolf = (float)A.tol;
    double* LAM = reinterpret_cast<double*>(st + SL.lam);
    V4* RHOF = reinterpret_cast<V4*>(st + SL.rhof);
    V4* RF = reinterpret_cast<V4*>(st + SL.rf);
    LP* INV = reinterpret_cast<LP*>(st + SL.inv);
    LP* Y = reinterpret_cast<LP*>(st + SL.y);
    LP* V = reinterpret_cast<LP*>(st + SL.vals);
    const int r0 = tm.rank(), ts = tm.size();

    auto gid_of = [&](int a) -> int64_t {
        return D.atom_base >= 0 ? (int64_t)D.atom_base + a : (int64_t)A.atom_gid[D.gid_off + a];
    };
    // ---- S1: reference geometry (x_old staged through X), weights
    for (int a = r0; a < na; a += ts) {
        const int64_t g = gid_of(a);
        X[a] = A.x_old[3 * g];
        X[na + a] = A.x_old[3 * g + 1];
        X[2 * na + a] = A.x_old[3 * g + 2];
        const double w = A.inv_mass[g];
        W[a] = DF ? as_bits(df_split(w)) : w;
        WL[a] = to_lp<LP>(w);
    }
    if (r0 == 0) {  // zero-weight atom referenced by fill entries
        W[na] = 0.0;
        WL[na] = LP(0);
    }
    tm.sync();
    for (int p = r0; p < nc; p += ts) {
        const int i = con[p].i, j = con[p].j;
        const double rx = X[i] - X[j], ry = X[na + i] - X[na + j], rz = X[2 * na + i] - X[2 * na + j];
        V4 v;
        v.x = to_lp<LP>(rx);
        v.y = to_lp<LP>(ry);
        v.z = to_lp<LP>(rz);
        v.w = LP(0);
        RHOF[p] = v;
        const int32_t g = con_gid[p];
        const double dd = A.d[g];
        if constexpr (DF) {
            RHO[p] = as_bits(df_split(rx));
            RHO[nc + p] = as_bits(df_split(ry));
            RHO[2 * nc + p] = as_bits(df_split(rz));
            D2[p] = as_bits(df_split(dd * dd));
        } else {
            RHO[p] = rx;
            RHO[nc + p] = ry;
            RHO[2 * nc + p] = rz;
            D2[p] = dd * dd;
        }
        WL[na + 1 + p] = WL[i] + WL[j];
        const float l0 = A.lambda0 ? A.lambda0[g] : 0.0f;
        LAM[p] = DF ? as_bits(dfloat{l0, 0.0f}) : widen(l0);
        Y[p] = (LP)l0;
    }
    tm.sync();
    for (int a = r0; a < na; a += ts) {
        if constexpr (DF) {  // displacements start at zero
            X[a] = 0.0;
            X[na + a] = 0.0;
            X[2 * na + a] = 0.0;
        } else {
            const int64_t g = gid_of(a);
            X[a] = A.x_unc[3 * g];
            X[na + a] = A.x_unc[3 * g + 1];
            X[2 * na + a] = A.x_unc[3 * g + 2];
        }
    }
    if constexpr (DF) {
        for (int p = r0; p < nc; p += ts) {
            const int64_t gi = gid_of(con[p].i), gj = gid_of(con[p].j);
            SK[p] = as_bits(df_split(A.x_unc[3 * gi] - A.x_unc[3 * gj]));
            SK[nc + p] = as_bits(df_split(A.x_unc[3 * gi + 1] - A.x_unc[3 * gj + 1]));
            SK[2 * nc + p] = as_bits(df_split(A.x_unc[3 * gi + 2] - A.x_unc[3 * gj + 2]));
        }
    }
    tm.sync();

    // ---- S6: x -= M^-1 G(x_old)^T Y   (Y holds delta, or lambda0 before the loop)
    auto update_positions = [&]() {
        for (int a = r0; a < na; a += ts) {
            const int e1 = inc_ptr[a + 1];
            if constexpr (DF) {
                dfloat ax{0.f, 0.f}, ay{0.f, 0.f}, az{0.f, 0.f};
                for (int e = inc_ptr[a]; e < e1; ++e) {
                    const unsigned v = inc[e];
                    const int p = (int)(v >> 1);
                    const float dl = (float)Y[p];
                    const float c = (v & 1u) ? -(dl + dl) : (dl + dl);
                    ax = df_add(ax, df_mul_f(as_df(RHO[p]), c));
                    ay = df_add(ay, df_mul_f(as_df(RHO[nc + p]), c));
                    az = df_add(az, df_mul_f(as_df(RHO[2 * nc + p]), c));
                }
                const dfloat w = as_df(W[a]);
                X[a] = as_bits(df_sub(as_df(X[a]), df_mul(w, ax)));
                X[na + a] = as_bits(df_sub(as_df(X[na + a]), df_mul(w, ay)));
                X[2 * na + a] = as_bits(df_sub(as_df(X[2 * na + a]), df_mul(w, az)));
            } else {
                double ax = 0.0, ay = 0.0, az = 0.0;
                for (int e = inc_ptr[a]; e < e1; ++e) {
                    const unsigned v = inc[e];
                    const int p = (int)(v >> 1);
                    const LP dl = Y[p];
                    const double c = to_hp((v & 1u) ? -(dl + dl) : (dl + dl));
                    ax = fma(c, RHO[p], ax);
                    ay = fma(c, RHO[nc + p], ay);
                    az = fma(c, RHO[2 * nc + p], az);
                }
                const double w = W[a];
                X[a] = fma(-w, ax, X[a]);
                X[na + a] = fma(-w, ay, X[na + a]);
                X[2 * na + a] = fma(-w, az, X[2 * na + a]);
            }
        }
    };
    if (A.lambda0) {
        update_positions();
        tm.sync();
    }

    int status = ILVES_MOL_MAX_ITER, iters = A.max_iter;
    for (int it = 0;; ++it) {
        // ---- S2: violations (float64 class), Jacobian rows and right-hand side
        bool conv = true, bad = false;
        for (int p = r0; p < nc; p += ts) {
            const int i = con[p].i, j = con[p].j;
            V4 v;
            if constexpr (DF) {
                const dfloat rx = df_add(as_df(SK[p]), df_sub(as_df(X[i]), as_df(X[j])));
                const dfloat ry = df_add(as_df(SK[nc + p]), df_sub(as_df(X[na + i]), as_df(X[na + j])));
                const dfloat rz = df_add(as_df(SK[2 * nc + p]), df_sub(as_df(X[2 * na + i]), as_df(X[2 * na + j])));
                const dfloat d2 = as_df(D2[p]);
                // |r|^2 - d^2: exact products of the high words, two-sums of the big terms,
                // every rounding error collected in a small tail
                const float px = __fmul_rn(rx.hi, rx.hi), ex = __fmaf_rn(rx.hi, rx.hi, -px);
                const float py = __fmul_rn(ry.hi, ry.hi), ey = __fmaf_rn(ry.hi, ry.hi, -py);
                const float pz = __fmul_rn(rz.hi, rz.hi), ez = __fmaf_rn(rz.hi, rz.hi, -pz);
                float s1, e1, s2, e2, s3, e3;
                two_sum(px, py, s1, e1);
                two_sum(s1, pz, s2, e2);
                two_sum(s2, -d2.hi, s3, e3);
                float cross = __fmul_rn(rx.hi, rx.lo);
                cross = __fmaf_rn(ry.hi, ry.lo, cross);
                cross = __fmaf_rn(rz.hi, rz.lo, cross);
                const float tail = ((ex + ey) + (ez + e1)) + ((e2 + e3) - d2.lo) + (cross + cross);
                const float sg = s3 + tail;
                conv = conv && fabsf(sg) <= tolf * d2.hi;
                bad = bad || nonfinite(sg);
                v.x = rx.hi;
                v.y = ry.hi;
                v.z = rz.hi;
                Y[p] = sg;
            } else {
                const double rx = X[i] - X[j], ry = X[na + i] - X[na + j], rz = X[2 * na + i] - X[2 * na + j];
                const double d2 = D2[p];
                const double sg = fma(rx, rx, fma(ry, ry, fma(rz, rz, -d2)));
                conv = conv && abs_le(sg, tol * d2);
                bad = bad || nonfinite(sg);
                v.x = to_lp<LP>(rx);
                v.y = to_lp<LP>(ry);
                v.z = to_lp<LP>(rz);
                Y[p] = to_lp<LP>(sg);
            }
            v.w = LP(0);
            RF[p] = v;
        }
        if (tm.any(bad)) {
            status = ILVES_MOL_NONFINITE;
            iters = it;
            break;
        }
        if (tm.all(conv)) {
            status = ILVES_MOL_CONVERGED;
            iters = it;
            break;
        }
        if (it >= A.max_iter) break;
        tm.sync();
        // ---- S3 + S4 + forward half of S5, one level at a time
        bool singular = false;
        for (int l = 0; l < D.nlevel; ++l) {
            const int p0 = lvl_piv[l], np = lvl_piv[l + 1] - p0;
            const int t0 = lvl_task[l], t1 = lvl_task[l + 1];
            // one pass over the level's tasks with a single code path: the first np tasks are
            // the DIAG tasks of the level's pivots (their "shared atom" is the pseudo-atom
            // carrying w_i + w_j), which also produce 1 / pivot and the forward-solve entry
            for (int t = t0 + r0; t < t1; t += ts) {
                const Task<IdxT> tk = tasks[t];
                const bool diag = t < t0 + np;
                const int e1 = tasks[t + 1].tstart;
                const V4 rr = RF[tk.row], pp = RHOF[tk.col];
                const int at = tk.atomsign >> 1;
                const LP wv = WL[at];
                const LP c = (tk.atomsign & 1) ? LP(-4) * wv : LP(4) * wv;
                const LP a = c * (rr.x * pp.x + rr.y * pp.y + rr.z * pp.z);
                LP s = a, yv = LP(0);
#pragma unroll 2
                for (int e = tk.tstart; e < e1; ++e) {
                    const auto tr = terms[e];
                    const int m = TO::m(tr);
                    const LP li = V[TO::l(tr)] * INV[m];
                    s -= li * V[TO::u(tr)];
                    yv += li * Y[m];
                }
                V[t] = s;
                if (diag) {
                    singular = singular || !(lp_abs(s) > Mode::pivot_rel * lp_abs(a));
                    INV[tk.row] = lp_rcp(s);
                    Y[tk.row] -= yv;
                }
            }
            tm.sync();
        }
        if (tm.any(singular)) {
            status = ILVES_MOL_SINGULAR_PIVOT;
            iters = it;
            break;
        }
        // ---- backward half of S5
        for (int l = D.nlevel - 1; l >= 0; --l) {
            const int p1 = lvl_piv[l + 1];
            for (int p = lvl_piv[l] + r0; p < p1; p += ts) {
                const int us = piv[p].diag, nu = piv[p].nup;
                LP dl = Y[p];
                for (int k = 0; k < nu; ++k) dl -= V[us + k] * Y[tasks[us + k].col];
                Y[p] = dl * INV[p];
            }
            tm.sync();
        }
        // ---- lambda += delta (float64 class), S6
        for (int p = r0; p < nc; p += ts) {
            if constexpr (DF) LAM[p] = as_bits(df_add_f(as_df(LAM[p]), (float)Y[p]));
            else LAM[p] += to_hp(Y[p]);
        }
        update_positions();
        tm.sync();
    }
    // ---- S7: outputs
    for (int a = r0; a < na; a += ts) {
        const int64_t g = gid_of(a);
        if constexpr (DF) {
            A.x_out[3 * g] = A.x_unc[3 * g] + df_join(as_df(X[a]));
            A.x_out[3 * g + 1] = A.x_unc[3 * g + 1] + df_join(as_df(X[na + a]));
            A.x_out[3 * g + 2] = A.x_unc[3 * g + 2] + df_join(as_df(X[2 * na + a]));
        } else {
            A.x_out[3 * g] = X[a];
            A.x_out[3 * g + 1] = X[na + a];
            A.x_out[3 * g + 2] = X[2 * na + a];
        }
    }
    if (A.lambda_out)
        for (int p = r0; p < nc; p += ts) A.lambda_out[con_gid[p]] = DF ? df_join(as_df(LAM[p])) : LAM[p];
    if (r0 == 0) {
        if (A.iterations_out) A.iterations_out[D.mol_id] = iters;
        if (A.status_out) A.status_out[D.mol_id] = status;
    }
}

// ------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------
struct SmallSched {
    const int32_t* cta_slot_ptr;
    const int32_t* slot_ptr;
    const int32_t* slot_mol;
    const int32_t* slot_off;
};

// Persistent batched kernel: warp w of CTA c owns one slot (a fixed slice of the CTA's
// shared-memory arena) and solves its queue of molecules one after the other; warps
// never wait for each other.  Each molecule's program blob is staged into the slice
// with 16-byte loads before its Newton loop.
template <class Mode>
__global__ void __launch_bounds__(1024, 1)
k_solve_small(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob, SmallSched S,
              SolveArgs A) {
    extern __shared__ __align__(16) uint8_t arena[];
    const WarpTeam tm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = S.cta_slot_ptr[blockIdx.x] + warp;
    if (slot >= S.cta_slot_ptr[blockIdx.x + 1]) return;
    uint8_t* slice = arena + S.slot_off[slot];
    const int q1 = S.slot_ptr[slot + 1];
    for (int q = S.slot_ptr[slot]; q < q1; ++q) {
        const MolDesc D = desc[S.slot_mol[q]];
        const ProgLayout PL = prog_layout<uint16_t>(D.na, D.nc, D.ntask, D.nterm, D.nlevel);
        const uint4* src = reinterpret_cast<const uint4*>(blob + D.blob_off);
        uint4* dst = reinterpret_cast<uint4*>(slice);
        const int n16 = (int)(PL.bytes >> 4);
        int k = lane;
        for (; k + 96 < n16; k += 128) {  // four independent 16-byte loads in flight per lane
            const uint4 a0 = __ldg(src + k), a1 = __ldg(src + k + 32), a2 = __ldg(src + k + 64),
                        a3 = __ldg(src + k + 96);
            dst[k] = a0;
            dst[k + 32] = a1;
            dst[k + 64] = a2;
            dst[k + 96] = a3;
        }
        for (; k < n16; k += 32) dst[k] = __ldg(src + k);
        __syncwarp();
        solve_molecule<Mode, uint16_t, WarpTeam>(tm, D, slice, slice + PL.bytes, A);
        __syncwarp();
    }
}

// Large molecules: one CTA per molecule, program and state in global memory.
template <class Mode>
__global__ void __launch_bounds__(512, 1)
k_solve_large(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob, uint8_t* work,
              SolveArgs A) {
    const BlockTeam tm;
    const MolDesc D = desc[blockIdx.x];
    solve_molecule<Mode, uint32_t, BlockTeam>(tm, D, blob + D.blob_off, work + D.work_off, A);
}

__global__ void k_copy_free(const int32_t* __restrict__ idx, int n, const double* __restrict__ x_unc,
                            double* __restrict__ x_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int64_t g = idx[i];
        x_out[3 * g] = x_unc[3 * g];
        x_out[3 * g + 1] = x_unc[3 * g + 1];
        x_out[3 * g + 2] = x_unc[3 * g + 2];
    }
}

// ------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------
template <class T>
static cudaError_t upload(T** dptr, const std::vector<T>& v) {
    *dptr = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dptr, v.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_device(ilves_topology* T) {
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    f(T->d_desc);
    f(T->d_blob);
    f(T->d_atom_gid);
    f(T->d_free_atoms);
    f(T->d_con_i);
    f(T->d_con_j);
    f(T->d_nbr);
    f(T->d_nbr_atom);
    f(T->d_ws_con);
    f(T->d_ws_atom);
    f(T->d_work);
    for (auto& s : T->sched) {
        f(s.cta_slot_ptr);
        f(s.slot_ptr);
        f(s.slot_mol);
        f(s.slot_off);
        s = DeviceSchedule{};
    }
    if (T->side_stream) cudaStreamDestroy((cudaStream_t)T->side_stream);
    if (T->ev_fork) cudaEventDestroy((cudaEvent_t)T->ev_fork);
    if (T->ev_join) cudaEventDestroy((cudaEvent_t)T->ev_join);
    T->d_desc = nullptr;
    T->d_blob = nullptr;
    T->d_atom_gid = nullptr;
    T->d_free_atoms = nullptr;
    T->d_con_i = T->d_con_j = T->d_nbr = T->d_nbr_atom = nullptr;
    T->d_ws_con = T->d_ws_atom = nullptr;
    T->d_work = nullptr;
    T->side_stream = T->ev_fork = T->ev_join = nullptr;
}

template <class Mode>
static const void* small_kernel() {
    return (const void*)k_solve_small<Mode>;
}

static ilves_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return ILVES_OK;
    if (e == cudaErrorMemoryAllocation) return ILVES_ERR_OOM;
    return ILVES_ERR_CUDA;
}

static ilves_status upload_topology(ilves_topology* T, const ilves_setup_opts& o) {
    cudaError_t e;
    int dev = o.device;
    if (dev < 0) {
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return to_status(e);
    } else if ((e = cudaSetDevice(dev)) != cudaSuccess) {
        return to_status(e);
    }
    T->device = dev;
    int n_sm = 0, smem_optin = 0, smem_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    T->n_sm = n_sm;
    const int ctas_per_sm = o.ctas_per_sm > 0 ? std::min(o.ctas_per_sm, 4) : 1;
    const int arena = std::min(smem_optin, smem_sm / ctas_per_sm - 1024) & ~15;
    // molecules whose slice does not fit an arena take the CTA-per-molecule path
    for (auto& M : T->mols)
        if (!M.large && footprint(M, ILVES_PREC_FP64) > (uint32_t)arena) M.large = true;
    // descriptors, program blobs, atom ids
    std::vector<int32_t> order;
    for (int32_t m = 0; m < T->n_mol; ++m)
        if (!T->mols[m].large) order.push_back(m);
    T->n_small = (int32_t)order.size();
    for (int32_t m = 0; m < T->n_mol; ++m)
        if (T->mols[m].large) order.push_back(m);
    T->n_large = T->n_mol - T->n_small;
    std::vector<int32_t> desc_index(T->n_mol);
    std::vector<MolDesc> desc(T->n_mol);
    std::vector<int32_t> gids;
    int64_t boff = 0, woff = 0;
    for (int32_t k = 0; k < T->n_mol; ++k) {
        const int32_t m = order[k];
        const MolHost& M = T->mols[m];
        desc_index[m] = k;
        MolDesc& D = desc[k];
        D.blob_off = boff;
        boff += (program_blob_bytes(T, m) + 15) & ~int64_t(15);
        const int32_t na = (int32_t)M.atoms.size();
        D.atom_base = (M.atoms.back() - M.atoms.front() == na - 1) ? M.atoms.front() : -1;
        D.gid_off = (int32_t)gids.size();
        gids.insert(gids.end(), M.atoms.begin(), M.atoms.end());
        D.mol_id = m;
        D.nterm = M.nterm;
        D.ntask = M.ntask;
        D.na = na;
        D.nc = (int32_t)M.cons.size();
        D.nlevel = M.nlevel;
        D.pad = 0;
        D.work_off = 0;
        if (M.large) {
            D.work_off = woff;
            woff += (std::max(state_layout(na, D.nc, M.ntask, 8, false).bytes, state_layout(na, D.nc, M.ntask, 4, true).bytes) + 255) & ~int64_t(255);
        }
    }
    std::vector<uint8_t> blob((size_t)std::max<int64_t>(boff, 16), 0);
    for (int32_t k = 0; k < T->n_mol; ++k) program_write_blob(T, order[k], blob.data() + desc[k].blob_off);
    T->blob_bytes = boff;
    T->work_bytes = woff;
    if ((e = upload(&T->d_desc, desc)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_blob, blob)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_atom_gid, gids)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_free_atoms, T->free_atoms)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_con_i, T->con_i)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_con_j, T->con_j)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_nbr, T->nbr)) != cudaSuccess) return to_status(e);
    if ((e = upload(&T->d_nbr_atom, T->nbr_atom)) != cudaSuccess) return to_status(e);
    if (T->n_c > 0 && (e = cudaMalloc((void**)&T->d_ws_con, (size_t)T->n_c * 8 * sizeof(float))) != cudaSuccess)
        return to_status(e);
    if (T->n_atoms > 0 && (e = cudaMalloc((void**)&T->d_ws_atom, (size_t)T->n_atoms * sizeof(float))) != cudaSuccess)
        return to_status(e);
    if (woff > 0 && (e = cudaMalloc((void**)&T->d_work, woff)) != cudaSuccess) return to_status(e);
    // persistent schedules, one per precision mode
    for (int mode = 0; mode < 3; ++mode) {
        std::vector<uint32_t> fps;
        for (int32_t m = 0; m < T->n_mol; ++m)
            if (!T->mols[m].large) fps.push_back(footprint(T->mols[m], mode));
        // auto: the largest warp count per CTA whose slices fit the arena (searched downwards)
        int warps = o.warps_per_cta > 0 ? o.warps_per_cta : 32;
        warps = std::max(1, std::min(32, warps));
        HostSchedule HS;
        build_schedule(T, mode, n_sm * ctas_per_sm, warps, arena, HS);
        for (auto& km : HS.slot_mol) km = desc_index[km];
        DeviceSchedule& DS = T->sched[mode];
        DS.n_cta = HS.n_cta;
        DS.warps = HS.warps;
        DS.arena = HS.arena;
        if ((e = upload(&DS.cta_slot_ptr, HS.cta_slot_ptr)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.slot_ptr, HS.slot_ptr)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.slot_mol, HS.slot_mol)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.slot_off, HS.slot_off)) != cudaSuccess) return to_status(e);
    }
    if (T->n_large > 0) {
        cudaStream_t s;
        cudaEvent_t a, b;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return to_status(e);
        T->side_stream = s;
        if ((e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming)) != cudaSuccess) return to_status(e);
        T->ev_fork = a;
        if ((e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming)) != cudaSuccess) return to_status(e);
        T->ev_join = b;
    }
    T->on_device = true;
    return ILVES_OK;
}

template <class Mode>
static ilves_status launch_mode(ilves_topology* T, const SolveArgs& A, cudaStream_t stream) {
    cudaError_t e;
    int launches = 0;
    const DeviceSchedule& DS = T->sched[Mode::id];
    if (!T->smem_attr_set[Mode::id]) {
        e = cudaFuncSetAttribute(small_kernel<Mode>(), cudaFuncAttributeMaxDynamicSharedMemorySize, DS.arena);
        if (e != cudaSuccess) return to_status(e);
        T->smem_attr_set[Mode::id] = true;
    }
    if (T->n_large > 0) {
        cudaStream_t side = (cudaStream_t)T->side_stream;
        if ((e = cudaEventRecord((cudaEvent_t)T->ev_fork, stream)) != cudaSuccess) return to_status(e);
        if ((e = cudaStreamWaitEvent(side, (cudaEvent_t)T->ev_fork, 0)) != cudaSuccess) return to_status(e);
        k_solve_large<Mode><<<T->n_large, T->large_threads, 0, side>>>(T->d_desc + T->n_small, T->d_blob,
                                                                       T->d_work, A);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
        if ((e = cudaEventRecord((cudaEvent_t)T->ev_join, side)) != cudaSuccess) return to_status(e);
    }
    if (T->n_small > 0) {
        SmallSched S{DS.cta_slot_ptr, DS.slot_ptr, DS.slot_mol, DS.slot_off};
        k_solve_small<Mode><<<DS.n_cta, DS.warps * 32, DS.arena, stream>>>(T->d_desc, T->d_blob, S, A);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
    }
    const int nf = (int)T->free_atoms.size();
    if (nf > 0 && A.x_out != A.x_unc) {
        k_copy_free<<<(nf + 255) / 256, 256, 0, stream>>>(T->d_free_atoms, nf, A.x_unc, A.x_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
    }
    if (T->n_large > 0) {
        if ((e = cudaStreamWaitEvent(stream, (cudaEvent_t)T->ev_join, 0)) != cudaSuccess) return to_status(e);
    }
    T->last_launches = launches;
    return ILVES_OK;
}

// ------------------------------------------------------------------------------------
// Allocation-free variant (see ilves_solve_static_scratch in ilves.h).  The state of
// CTA-per-molecule solves lives in this file-scope device array instead of the
// topology's workspace.  Host code must not pass the symbol itself to a kernel (in host
// code it names a host-side stand-in); its device address is looked up once per device.
// ------------------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mutex;
static void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up on first use).
static ilves_status static_scratch_address(int dev, uint8_t** out) {
    if (dev < 0 || dev >= kMaxDevices) return ILVES_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return ILVES_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = reinterpret_cast<uint8_t*>(g_scratch_addr[dev]);
    return ILVES_OK;
}

template <class Mode>
static ilves_status launch_mode_static(ilves_topology* T, const SolveArgs& A, cudaStream_t stream,
                                       uint8_t* scratch) {
    cudaError_t e;
    int launches = 0;
    const DeviceSchedule& DS = T->sched[Mode::id];
    if (!T->smem_attr_set[Mode::id]) {
        e = cudaFuncSetAttribute(small_kernel<Mode>(), cudaFuncAttributeMaxDynamicSharedMemorySize, DS.arena);
        if (e != cudaSuccess) return to_status(e);
        T->smem_attr_set[Mode::id] = true;
    }
    if (T->n_large > 0) {
        cudaStream_t side = (cudaStream_t)T->side_stream;
        if ((e = cudaEventRecord((cudaEvent_t)T->ev_fork, stream)) != cudaSuccess) return to_status(e);
        if ((e = cudaStreamWaitEvent(side, (cudaEvent_t)T->ev_fork, 0)) != cudaSuccess) return to_status(e);
        k_solve_large<Mode><<<T->n_large, T->large_threads, 0, side>>>(T->d_desc + T->n_small, T->d_blob, scratch, A);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
        if ((e = cudaEventRecord((cudaEvent_t)T->ev_join, side)) != cudaSuccess) return to_status(e);
    }
    if (T->n_small > 0) {
        SmallSched S{DS.cta_slot_ptr, DS.slot_ptr, DS.slot_mol, DS.slot_off};
        k_solve_small<Mode><<<DS.n_cta, DS.warps * 32, DS.arena, stream>>>(T->d_desc, T->d_blob, S, A);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
    }
    const int nf = (int)T->free_atoms.size();
    if (nf > 0 && A.x_out != A.x_unc) {
        k_copy_free<<<(nf + 255) / 256, 256, 0, stream>>>(T->d_free_atoms, nf, A.x_unc, A.x_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
    }
    if (T->n_large > 0) {
        if ((e = cudaStreamWaitEvent(stream, (cudaEvent_t)T->ev_join, 0)) != cudaSuccess) return to_status(e);
    }
    T->last_launches = launches;
    return ILVES_OK;
}

}  // namespace ilves

using namespace ilves;

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" void ilves_default_opts(ilves_setup_opts* o) {
    if (!o) return;
    o->ordering = 0;
    o->degree_slack = 2;
    o->warps_per_cta = 0;
    o->ctas_per_sm = 0;
    o->device = -1;
    o->max_warp_constraints = 0;
}

extern "C" ilves_status ilves_setup_topology(int32_t n_atoms, int32_t n_constraints, const int32_t* atom_i,
                                             const int32_t* atom_j, const ilves_setup_opts* opts,
                                             ilves_topology** out) {
    if (!out) return ILVES_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_atoms < 0 || n_constraints < 0) return ILVES_ERR_INVALID_ARG;
    if (n_constraints > 0 && (!atom_i || !atom_j)) return ILVES_ERR_INVALID_ARG;
    ilves_setup_opts o;
    ilves_default_opts(&o);
    if (opts) o = *opts;
    if (o.ordering < 0 || o.ordering > 2 || o.degree_slack < 0 || o.warps_per_cta < 0 ||
        o.warps_per_cta > 32 || o.ctas_per_sm < 0 || o.ctas_per_sm > 4)
        return ILVES_ERR_INVALID_ARG;
    ilves_topology* T = new ilves_topology();
    ilves_status s = plan_topology(T, n_atoms, n_constraints, atom_i, atom_j, o);
    if (s == ILVES_OK && o.device != -2) s = upload_topology(T, o);
    if (s != ILVES_OK) {
        free_device(T);
        free_programs(T);
        delete T;
        return s;
    }
    *out = T;
    return ILVES_OK;
}

extern "C" ilves_status ilves_solve(ilves_topology* T, const double* x_old, const double* x_unc,
                                    const double* inv_mass, const double* d, double tol, int32_t max_iter,
                                    int32_t precision, const float* lambda0, double* x_out, double* lambda_out,
                                    int32_t* iterations_out, int32_t* mol_status_out, void* stream) {
    if (!T || !T->on_device) return ILVES_ERR_INVALID_ARG;
    if (max_iter < 0 || !(tol >= 0.0)) return ILVES_ERR_INVALID_ARG;
    if (T->n_atoms > 0 && (!x_old || !x_unc || !inv_mass || !x_out)) return ILVES_ERR_INVALID_ARG;
    if (T->n_c > 0 && !d) return ILVES_ERR_INVALID_ARG;
    SolveArgs A;
    A.x_old = x_old;
    A.x_unc = x_unc;
    A.inv_mass = inv_mass;
    A.d = d;
    A.lambda0 = lambda0;
    A.x_out = x_out;
    A.lambda_out = lambda_out;
    A.iterations_out = iterations_out;
    A.status_out = mol_status_out;
    A.atom_gid = T->d_atom_gid;
    A.tol = tol;
    A.max_iter = max_iter;
    cudaStream_t s = (cudaStream_t)stream;
    T->last_launches = 0;
    switch (precision) {
        case ILVES_PREC_FP64: return launch_mode<ModeFP64>(T, A, s);
        case ILVES_PREC_MIXED: return launch_mode<ModeMixed>(T, A, s);
        case ILVES_PREC_MIXED_DF: return launch_mode<ModeMixedDF>(T, A, s);
        default: return ILVES_ERR_INVALID_ARG;
    }
}

extern "C" ilves_status ilves_solve_static_scratch(ilves_topology* T, const double* x_old, const double* x_unc,
                                                   const double* inv_mass, const double* d, double tol,
                                                   int32_t max_iter, int32_t precision, const float* lambda0,
                                                   double* x_out, double* lambda_out, int32_t* iterations_out,
                                                   int32_t* mol_status_out, void* stream) {
    if (!T || !T->on_device) return ILVES_ERR_INVALID_ARG;
    if (max_iter < 0 || !(tol >= 0.0)) return ILVES_ERR_INVALID_ARG;
    if (T->n_atoms > 0 && (!x_old || !x_unc || !inv_mass || !x_out)) return ILVES_ERR_INVALID_ARG;
    if (T->n_c > 0 && !d) return ILVES_ERR_INVALID_ARG;
    if (precision < ILVES_PREC_FP64 || precision > ILVES_PREC_MIXED_DF) return ILVES_ERR_INVALID_ARG;
    if ((uint64_t)T->work_bytes > (uint64_t)kStaticScratchBytes) return ILVES_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ILVES_ERR_CUDA;
    if (dev != T->device) return ILVES_ERR_INVALID_ARG;
    uint8_t* scratch = nullptr;
    ilves_status st = static_scratch_address(dev, &scratch);
    if (st != ILVES_OK) return st;
    SolveArgs A;
    A.x_old = x_old;
    A.x_unc = x_unc;
    A.inv_mass = inv_mass;
    A.d = d;
    A.lambda0 = lambda0;
    A.x_out = x_out;
    A.lambda_out = lambda_out;
    A.iterations_out = iterations_out;
    A.status_out = mol_status_out;
    A.atom_gid = T->d_atom_gid;
    A.tol = tol;
    A.max_iter = max_iter;
    cudaStream_t s = (cudaStream_t)stream;
    T->last_launches = 0;
    switch (precision) {
        case ILVES_PREC_FP64: return launch_mode_static<ModeFP64>(T, A, s, scratch);
        case ILVES_PREC_MIXED: return launch_mode_static<ModeMixed>(T, A, s, scratch);
        default: return launch_mode_static<ModeMixedDF>(T, A, s, scratch);
    }
}

extern "C" int64_t ilves_static_scratch_bytes(void) { return (int64_t)kStaticScratchBytes; }

extern "C" int64_t ilves_topology_workspace_bytes(const ilves_topology* T) { return T ? T->work_bytes : 0; }

extern "C" ilves_status ilves_topology_info(const ilves_topology* T, int32_t* n_molecules, int64_t* nnz_factor,
                                            int32_t* max_levels, int64_t* n_fill, int32_t* n_large) {
    if (!T) return ILVES_ERR_INVALID_ARG;
    int64_t nnz = 0, fill = 0;
    int32_t ml = 0, nl = 0;
    for (const auto& M : T->mols) {
        nnz += M.ntask;
        fill += M.n_fill;
        ml = std::max(ml, M.nlevel);
        nl += M.large ? 1 : 0;
    }
    if (n_molecules) *n_molecules = T->n_mol;
    if (nnz_factor) *nnz_factor = nnz;
    if (max_levels) *max_levels = ml;
    if (n_fill) *n_fill = fill;
    if (n_large) *n_large = nl;
    return ILVES_OK;
}

extern "C" ilves_status ilves_topology_molecules(const ilves_topology* T, int32_t* atoms, int32_t* constraints,
                                                 int32_t* levels, int32_t* first_atom) {
    if (!T) return ILVES_ERR_INVALID_ARG;
    for (int32_t m = 0; m < T->n_mol; ++m) {
        const MolHost& M = T->mols[m];
        if (atoms) atoms[m] = (int32_t)M.atoms.size();
        if (constraints) constraints[m] = (int32_t)M.cons.size();
        if (levels) levels[m] = M.nlevel;
        if (first_atom) first_atom[m] = M.atoms.front();
    }
    return ILVES_OK;
}

extern "C" ilves_status ilves_topology_export_molecule(const ilves_topology* T, int32_t mol, int32_t* pos_gid,
                                                       int32_t* level, int32_t* up_ptr, int32_t* up_idx) {
    if (!T || mol < 0 || mol >= T->n_mol) return ILVES_ERR_INVALID_ARG;
    program_export(T, mol, pos_gid, level, up_ptr, up_idx);
    return ILVES_OK;
}

extern "C" void ilves_destroy_topology(ilves_topology* T) {
    if (!T) return;
    if (T->on_device) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (T->device >= 0 && cur != T->device) cudaSetDevice(T->device);
        free_device(T);
        if (cur >= 0 && cur != T->device) cudaSetDevice(cur);
    }
    free_programs(T);
    delete T;
}

extern "C" const char* ilves_status_string(int32_t s) {
    switch (s) {
        case ILVES_OK: return "ok";
        case ILVES_ERR_INVALID_ARG: return "invalid argument";
        case ILVES_ERR_TOPOLOGY: return "invalid topology";
        case ILVES_ERR_CUDA: return "CUDA error";
        case ILVES_ERR_OOM: return "out of device memory";
        case ILVES_ERR_TIMEOUT: return "device wait timed out";
        case ILVES_ERR_TOO_LARGE: return "scratch needed exceeds the static maximum";
        default: return "unknown status";
    }
}

extern "C" int32_t ilves_last_launch_count(const ilves_topology* T) { return T ? T->last_launches : 0; }
