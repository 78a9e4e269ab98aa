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
#include <type_traits>
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
// v = hi + lo with hi = v truncated to float (narrow) and lo = the rest rounded to float.
// For 2^-75 <= |v| < 2^128 the rest is exactly the 29 mantissa bits below hi's, times
// 2^(exponent - 52), and lo stays in float's normal range: lo is built from those bits on the
// integer pipe (one int-to-float conversion, then the power of two added to its exponent
// field), bit for bit what rounding v - hi would give; smaller, huge and non-finite v take
// the float64 route.
__device__ __forceinline__ dfloat df_split(double v) {
    const float hi = narrow(v);
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FFu);
    if (e <= 948 || e >= 1151) return {hi, __double2float_rn(v - widen(hi))};
    const unsigned rem = (unsigned)(b & 0x1FFFFFFFull);
    const unsigned fb = __float_as_uint(__uint2float_rn(rem));  // 0, or its exponent field in [127, 156]
    const unsigned lb = (fb & 0x007FFFFFu) | ((unsigned)((int)(fb >> 23) + (e - 1075)) << 23);
    return {hi, __uint_as_float(rem != 0u ? (lb | ((unsigned)(b >> 32) & 0x80000000u)) : 0u)};
}
__device__ __forceinline__ double df_join(dfloat a) { return widen(a.hi) + widen(a.lo); }
__device__ __forceinline__ dfloat as_df(double v) { return *reinterpret_cast<dfloat*>(&v); }
__device__ __forceinline__ double as_bits(dfloat v) { return *reinterpret_cast<double*>(&v); }

// ------------------------------------------------------------------------------------
// teams
// ------------------------------------------------------------------------------------
// The kThreads threads (whole warps) of a batched-kernel slot: kSlotThreads for the wide
// slots, one warp for the narrow ones; more than one warp synchronises on named barrier
// 1 + slot (barrier 0 is the CTA's).
template <int kThreads>
struct SlotTeamT {
    static constexpr int kSize = kThreads;
    __device__ __forceinline__ int rank() const { return threadIdx.x % kThreads; }
    __device__ __forceinline__ int size() const { return kThreads; }
    __device__ __forceinline__ int id() const { return threadIdx.x / kThreads; }
    __device__ __forceinline__ void sync() const {
        if constexpr (kThreads == 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(id() + 1), "n"(kThreads) : "memory");
    }
    __device__ __forceinline__ bool all(bool p) const {
        if constexpr (kThreads == 32) {
            return __all_sync(0xFFFFFFFFu, p);
        } else {
            unsigned r;
            asm volatile("{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.and.pred po, %2, %3, pi;\n"
                         "selp.u32 %0, 1, 0, po;\n}\n"
                         : "=r"(r)
                         : "r"((unsigned)p), "r"(id() + 1), "n"(kThreads)
                         : "memory");
            return r != 0;
        }
    }
    __device__ __forceinline__ bool any(bool p) const {
        if constexpr (kThreads == 32) {
            return __any_sync(0xFFFFFFFFu, p);
        } else {
            unsigned r;
            asm volatile("{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.or.pred po, %2, %3, pi;\n"
                         "selp.u32 %0, 1, 0, po;\n}\n"
                         : "=r"(r)
                         : "r"((unsigned)p), "r"(id() + 1), "n"(kThreads)
                         : "memory");
            return r != 0;
        }
    }
};
using SlotTeam = SlotTeamT<kSlotThreads>;
using NarrowTeam = SlotTeamT<kNarrowThreads>;
template <class T> struct IsSlotTeam : std::false_type {};
template <int N> struct IsSlotTeam<SlotTeamT<N>> : std::true_type {};
struct BlockTeam {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool all(bool p) const { return __syncthreads_and(p) != 0; }
    __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
};

// Asynchronous global -> shared copies (cp.async): every copy of a batch is in flight at
// once and lands without passing through registers; wait_all + a team barrier makes the
// batch visible.  Both addresses are aligned to the copy size.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// hint: bring the 128-byte line holding p into L2 (no register, no fault on a valid address)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

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
    int32_t chord;       // ILVES-F: factorise A(x_old, x_old) once, reuse it every iteration
    int32_t start_diag;  // lambda0 = the diagonal guess, computed in S1 (lambda0 is NULL)
    __host__ __device__ bool has_start() const { return lambda0 != nullptr || start_diag != 0; }
};

// The diagonal (Jacobi) start of constraint k: lambda0_k = sigma_k(x_unc) / A_kk with
// A_kk = 4 (w_i + w_j) (s_k . r_k), s = x_unc,i - x_unc,j, r = x_old,i - x_old,j (one
// Newton step on the diagonal of A(x_unc, x_old)); float32 arithmetic on coordinates
// rounded to float32, as the stand-alone warm start (ilves_warm_start without a network)
// computes it, so both routes give the same lambda0.
__device__ __forceinline__ float f32_of(float v) { return v; }
__device__ __forceinline__ float f32_of(double v) { return narrow(v); }
__device__ __forceinline__ float diag_start(float sx, float sy, float sz, float rx, float ry, float rz, float d,
                                           float w_ij) {
    const float d2 = d * d;
    const float a = 4.0f * w_ij * (sx * rx + sy * ry + sz * rz);
    const float l0 = ((sx * sx + sy * sy + sz * sz) - d2) / a;
    return (a != 0.f && isfinite(l0)) ? l0 : 0.f;
}

// ------------------------------------------------------------------------------------
// per-item operations on one molecule's program and state
// ------------------------------------------------------------------------------------
// Float64-class arrays (X, W, RHO, S, D2, LAM) hold float64 values, or in the
// float-float mode dfloat pairs stored in the same 8 bytes.  In the float64 modes X
// holds absolute positions; in the float-float mode it holds displacements x - x_unc
// and S holds s_k = x_unc,i - x_unc,j, so that r_k = s_k + (dx_i - dx_j).
//
// kCoh: the state lives in global memory and other CTAs write parts of it (partitioned
// molecules), so state another CTA may have written is read through L2 (ld.global.cg)
// and never from a possibly stale L1 line (see ldf); the program is read-only and read
// through the texture path.
template <bool kCoh, class T>
__device__ __forceinline__ T lds(const T* p) {
    if constexpr (kCoh) {
        if constexpr (sizeof(T) == 32) {
            T v;
            const double2* q = reinterpret_cast<const double2*>(p);
            *reinterpret_cast<double2*>(&v) = __ldcg(q);
            reinterpret_cast<double2*>(&v)[1] = __ldcg(q + 1);
            return v;
        } else {
            return __ldcg(p);
        }
    } else {
        return *p;
    }
}
// State loads of a partitioned molecule: values written by another CTA ("foreign": the
// separator block and its atoms) are read through L2; everything else -- the CTA's own
// parts, and arrays fixed since set-up -- through L1.  Plain loads in the other modes.
template <bool kCoh, class T>
__device__ __forceinline__ T ldf(const T* p, bool foreign) {
    if constexpr (kCoh) {
        if (foreign) return lds<true>(p);
    }
    return *p;
}
template <bool kCoh, class T>
__device__ __forceinline__ T ldp(const T* p) {
    if constexpr (kCoh) {
        T v;
        if constexpr (sizeof(T) == 16) *reinterpret_cast<uint4*>(&v) = __ldg(reinterpret_cast<const uint4*>(p));
        else if constexpr (sizeof(T) == 8) *reinterpret_cast<uint2*>(&v) = __ldg(reinterpret_cast<const uint2*>(p));
        else if constexpr (sizeof(T) == 4) *reinterpret_cast<unsigned*>(&v) = __ldg(reinterpret_cast<const unsigned*>(p));
        else *reinterpret_cast<unsigned short*>(&v) = __ldg(reinterpret_cast<const unsigned short*>(p));
        return v;
    } else {
        return *p;
    }
}

template <class Mode, class IdxT, bool kCoh>
struct MolView {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    using TO = TermOf<IdxT>;
    using TaskT = typename TO::TaskT;
    static constexpr bool DF = Mode::df;
    static constexpr bool kCompact = sizeof(IdxT) == 2;
    int na, nc;
    const SegRow* seg;
    const ConA<IdxT>* con;
    const int32_t* con_gid;
    const Piv<IdxT>* piv;
    const IdxT* lvl_task;
    const IdxT* lvl_piv;
    const IdxT* lane_term;
    const IdxT* inc_ptr;
    const IdxT* inc;
    const IdxT* aslot;  // batched molecules: local atom of each atom slot
    const TaskT* tasks;
    const typename TO::T* terms;
    double *X, *W, *RHO, *SK, *D2, *LAM;
    float* RHOL;  // float-float mode: low parts of rho (SoA); the high parts are RHOF.xyz
    LP *WL, *Y, *V;
    V4 *RHOF, *RF;  // RHOF[p].w = w_i + w_j, RF[p].w = 1 / pivot p
    // partitioned molecules: Schur contribution tables and their values (4 per separator
    // task: two partial sums of L inv U, two of L inv y), in the workspace after the state
    const SepInfo* sep_info;
    const int32_t* cptr;
    const Contrib* cent;
    LP* CT;
    int sep_t0;
    int sep_p0;    // first separator position (nc if not partitioned)
    bool cohall;   // every state load is foreign (the separator phase)
    double* STG;  // x_old gathered AoS (warp path set-up only; aliases RF and later arrays)
    const MolDesc* D;
    const SolveArgs* A;
    float tolf;  // tol in float (float-float convergence test)

    // prog: the program (in shared memory for warp molecules); gprog: its global copy,
    // which alone holds con_gid
    __device__ __forceinline__ void init(const MolDesc& d, const uint8_t* prog, uint8_t* st, const SolveArgs& a,
                                         const uint8_t* gprog) {
        D = &d;
        A = &a;
        tolf = (float)a.tol;
        na = d.na;
        nc = d.nc;
        const ProgLayout PL =
            prog_layout<IdxT>(na, nc, d.ntask, d.nterm, d.nlevel, d.n_seg, d.n_sept, d.n_cent, d.pprog_bytes);
        const StateLayout SL = state_layout(na, nc, d.ntask, sizeof(LP), DF);
        seg = reinterpret_cast<const SegRow*>(prog + PL.seg);
        con = reinterpret_cast<const ConA<IdxT>*>(prog + PL.con_atoms);
        con_gid = reinterpret_cast<const int32_t*>(gprog + PL.con_gid);
        piv = reinterpret_cast<const Piv<IdxT>*>(prog + PL.piv);
        lvl_task = reinterpret_cast<const IdxT*>(prog + PL.lvl_task);
        lvl_piv = reinterpret_cast<const IdxT*>(prog + PL.lvl_piv);
        lane_term = reinterpret_cast<const IdxT*>(prog + PL.lane_term);
        inc_ptr = reinterpret_cast<const IdxT*>(prog + PL.inc_ptr);
        inc = reinterpret_cast<const IdxT*>(prog + PL.inc);
        aslot = reinterpret_cast<const IdxT*>(prog + PL.atom_off);
        tasks = reinterpret_cast<const TaskT*>(prog + PL.tasks);
        terms = reinterpret_cast<const typename TO::T*>(prog + PL.terms);
        X = reinterpret_cast<double*>(st + SL.x);
        W = reinterpret_cast<double*>(st + SL.w);
        WL = reinterpret_cast<LP*>(st + SL.wl);
        RHO = reinterpret_cast<double*>(st + SL.rho);
        RHOL = reinterpret_cast<float*>(st + SL.rho);
        SK = reinterpret_cast<double*>(st + SL.s);
        D2 = reinterpret_cast<double*>(st + SL.d2);
        LAM = reinterpret_cast<double*>(st + SL.lam);
        RHOF = reinterpret_cast<V4*>(st + SL.rhof);
        RF = reinterpret_cast<V4*>(st + SL.rf);
        Y = reinterpret_cast<LP*>(st + SL.y);
        V = reinterpret_cast<LP*>(st + SL.vals);
        STG = reinterpret_cast<double*>(st + SL.stage);
        sep_info = reinterpret_cast<const SepInfo*>(prog + PL.sep_info);
        cptr = reinterpret_cast<const int32_t*>(prog + PL.cptr);
        cent = reinterpret_cast<const Contrib*>(prog + PL.cent);
        CT = reinterpret_cast<LP*>(st + SL.bytes);
        sep_t0 = d.ntask - d.n_sept;
        sep_p0 = d.n_seg > 1 ? ldp<kCoh>(&seg[d.n_seg - 1].piv) : nc;
        cohall = false;
    }
    // global atom of atom slot o (the molecule's atoms in ascending global order); in
    //      large molecules local atom a sits in slot a, in batched molecules in the slot
    //      whose entry of aslot is a (their local atoms are ordered by degree)
    __device__ __forceinline__ int64_t slot_gid(int o) const {
        return D->atom_base >= 0 ? (int64_t)D->atom_base + o : (int64_t)A->atom_gid[D->gid_off + o];
    }
    __device__ __forceinline__ int64_t gid(int a) const {
        static_assert(!kCompact, "batched molecules address their atoms by slot");
        return slot_gid(a);
    }
    __device__ __forceinline__ ConA<IdxT> cons(int p) const { return ldp<kCoh>(con + p); }
    __device__ __forceinline__ int32_t gid_of_con(int p) const { return __ldg(con_gid + p); }
    __device__ __forceinline__ LP* inv_ptr(int p) const { return reinterpret_cast<LP*>(RF + p) + 3; }
    __device__ __forceinline__ bool foreign(int p) const { return cohall || p >= sep_p0; }

    // ---- partitioned molecules with one part per CTA: shared-memory copies of the CTA's
    //      own part (positions [P0, P1), atoms [A0, A1), tasks [T0, T1)) of the values it
    //      writes and reads back within a phase -- Y, RF (with 1/pivot), V, X.  Stores
    //      go to both copies, so other CTAs keep reading the global state; loads of the
    //      own part come from shared memory.  Off (XS == nullptr) in the other modes.
    int P0 = 0, P1 = 0, A0 = 0, A1 = 0, T0 = 0, T1 = 0;
    double* XS = nullptr;  // SoA with stride A1 - A0
    LP* YS = nullptr;
    V4* RFS = nullptr;
    LP* VS = nullptr;
    __device__ __forceinline__ bool in_p(int p) const {
        if constexpr (kCoh) return XS != nullptr && p >= P0 && p < P1;
        else return false;
    }
    __device__ __forceinline__ bool in_a(int a) const {
        if constexpr (kCoh) return XS != nullptr && a >= A0 && a < A1;
        else return false;
    }
    __device__ __forceinline__ bool in_t(int t) const {
        if constexpr (kCoh) return XS != nullptr && t >= T0 && t < T1;
        else return false;
    }
    __device__ __forceinline__ LP y_ld(int p) const { return in_p(p) ? YS[p - P0] : ldf<kCoh>(Y + p, foreign(p)); }
    // wt: the part's values must also reach global memory (another CTA reads them: the
    //     separator phase's terms of interior pivots beyond the contribution slots)
    bool wt = true;
    __device__ __forceinline__ void y_st(int p, LP v) {
        if (!in_p(p)) {
            Y[p] = v;
            return;
        }
        if (wt) Y[p] = v;
        YS[p - P0] = v;
    }
    __device__ __forceinline__ V4 rf_ld(int p) const { return in_p(p) ? RFS[p - P0] : ldf<kCoh>(RF + p, foreign(p)); }
    __device__ __forceinline__ void rf_st(int p, const V4& v) {
        if (!in_p(p)) {
            RF[p] = v;
            return;
        }
        if (wt) RF[p] = v;
        RFS[p - P0] = v;
    }
    __device__ __forceinline__ LP inv(int p) const {
        return in_p(p) ? reinterpret_cast<const LP*>(RFS + (p - P0))[3] : ldf<kCoh>(inv_ptr(p), foreign(p));
    }
    __device__ __forceinline__ void inv_st(int p, LP v) {
        if (!in_p(p)) {
            *inv_ptr(p) = v;
            return;
        }
        if (wt) *inv_ptr(p) = v;
        reinterpret_cast<LP*>(RFS + (p - P0))[3] = v;
    }
    // task values: slots of tasks of pivot m are foreign when m is
    __device__ __forceinline__ LP v_ld(int t, bool fgn) const { return in_t(t) ? VS[t - T0] : ldf<kCoh>(V + t, fgn); }
    __device__ __forceinline__ void v_st(int t, LP v) {
        if (!in_t(t)) {
            V[t] = v;
            return;
        }
        if (wt) V[t] = v;
        VS[t - T0] = v;
    }
    // coordinate c of atom a (float64 class)
    __device__ __forceinline__ double x_ld(int c, int a, bool fgn) const {
        return in_a(a) ? XS[c * (A1 - A0) + (a - A0)] : ldf<kCoh>(X + c * na + a, fgn);
    }
    __device__ __forceinline__ void x_st(int c, int a, double v) {
        X[c * na + a] = v;
        if (in_a(a)) XS[c * (A1 - A0) + (a - A0)] = v;
    }

    // ---- partitioned molecules, one part per CTA, with the part's program staged in
    //      shared memory (PartProgHeader): 16-bit part-local task words, terms and pivot
    //      records; a position code c is the part position P0 + c, or, with kPartSep
    //      set, the separator PST[c & ~kPartSep], whose rows and solution values are staged
    //      in SEPRF / SEPREF / SEPY once per phase.  RHS and WLS hold the part's reference
    //      rows and weights (fixed for the solve).  Off (PH == nullptr) otherwise.
    const PartProgHeader* PH = nullptr;
    const uint16_t *PLP = nullptr, *PLT = nullptr;
    const int32_t* PST = nullptr;
    const uint32_t *PLANE = nullptr, *PPIV = nullptr;
    const uint16_t* PAORD = nullptr;  // the part's atoms in update order (offsets from A0)
    const uint2 *PTK = nullptr, *PTM = nullptr;
    const uint2 *PCB = nullptr, *PCT = nullptr;  // the part's contributions and their terms
    V4* RHS = nullptr;
    LP* WLS = nullptr;
    V4 *SEPRF = nullptr, *SEPREF = nullptr;  // the separators' current and reference rows
    LP* SEPY = nullptr;                      // and solution values (scratch after the program)
    __device__ __forceinline__ void part_prog_bind(const uint8_t* sp) {
        PH = reinterpret_cast<const PartProgHeader*>(sp);
        const PartProgLayout L =
            part_prog_layout(PH->np, PH->nt, PH->na, PH->nlev, PH->nsep, PH->nterm, PH->ncontrib, PH->ncterm);
        PLP = reinterpret_cast<const uint16_t*>(sp + L.lvl_piv);
        PLT = reinterpret_cast<const uint16_t*>(sp + L.lvl_task);
        PST = reinterpret_cast<const int32_t*>(sp + L.septab);
        PLANE = reinterpret_cast<const uint32_t*>(sp + L.lane_term);
        PPIV = reinterpret_cast<const uint32_t*>(sp + L.piv);
        PAORD = reinterpret_cast<const uint16_t*>(sp + L.aorder);
        PTK = reinterpret_cast<const uint2*>(sp + L.tasks);
        PTM = reinterpret_cast<const uint2*>(sp + L.terms);
        PCB = reinterpret_cast<const uint2*>(sp + L.contribs);
        PCT = reinterpret_cast<const uint2*>(sp + L.cterms);
        uint8_t* sc = const_cast<uint8_t*>(sp) + L.scratch;
        SEPRF = reinterpret_cast<V4*>(sc);
        SEPREF = SEPRF + PH->nsep;
        SEPY = reinterpret_cast<LP*>(SEPREF + PH->nsep);
    }
    // current Jacobian row / reference row of the constraint with position code c
    __device__ __forceinline__ V4 prow(uint32_t c) const { return (c & kPartSep) ? SEPRF[c & ~kPartSep] : RFS[c]; }
    __device__ __forceinline__ V4 pref(uint32_t c) const { return (c & kPartSep) ? SEPREF[c & ~kPartSep] : RHS[c]; }
    // one level of the part's factorisation: local tasks t0 + r + kPartThreads k, DIAG
    //      tasks first (np of them, pivots p0 + ...); thread r walks its terms from offset e
    __device__ __forceinline__ void part_level(int t0, int t1, int np, int r, int& e, bool& singular) {
        for (int t = t0 + r; t < t1; t += kPartThreads) {
            const uint2 w = PTK[t];
            const uint32_t rc = w.x & 0xFFFFu, cc = w.x >> 16, ac = w.y & 0xFFFFu;
            const int n = (int)(w.y >> 24);
            const bool diag = t < t0 + np;
            const V4 rr = prow(rc), pp = pref(cc);
            const LP wv = diag ? pp.w : (ac == kPartNoAtom ? LP(0) : WLS[ac]);
            const LP cf = ((w.y >> 16) & 1u) ? LP(-4) * wv : LP(4) * wv;
            const LP a = cf * (rr.x * pp.x + rr.y * pp.y + rr.z * pp.z);
            LP sacc = a, yv = LP(0);
#pragma unroll 2
            for (int k = e; k < e + n; ++k) {
                const uint2 tr = PTM[k];
                const uint32_t m = tr.y;
                const LP li = VS[tr.x & 0xFFFFu] * reinterpret_cast<const LP*>(RFS + m)[3];
                sacc -= li * VS[tr.x >> 16];
                if (diag) yv += li * YS[m];
            }
            e += n;
            VS[t] = sacc;
            if (wt) V[T0 + t] = sacc;
            if (diag) {  // rc is a part position
                singular = singular || !(lp_abs(sacc) > Mode::pivot_rel * lp_abs(a));
                const LP ri = lp_rcp(sacc);
                reinterpret_cast<LP*>(RFS + rc)[3] = ri;
                const LP ny = YS[rc] - yv;
                YS[rc] = ny;
                if (wt) {
                    *inv_ptr(P0 + (int)rc) = ri;
                    Y[P0 + (int)rc] = ny;
                }
            }
        }
    }
    // contribution c of the part to the separator block (as contrib, from the part program)
    __device__ __forceinline__ void part_contrib(int c, bool factor) {
        const uint2 E = PCB[c];
        const bool diag = (E.x >> 31) != 0u;
        const int e0 = (int)(E.y & 0xFFFFu), e1 = e0 + (int)(E.y >> 16);
        LP sv = LP(0), sy = LP(0);
        for (int k = e0; k < e1; ++k) {
            const uint2 tr = PCT[k];
            const uint32_t m = tr.y;
            const LP li = VS[tr.x & 0xFFFFu] * reinterpret_cast<const LP*>(RFS + m)[3];
            if (factor) sv += li * VS[tr.x >> 16];
            if (diag) sy += li * YS[m];
        }
        LP* ct = CT + (E.x & 0x7FFFFFFFu);
        if (factor) ct[0] = sv;
        if (diag) ct[2] = sy;
    }
    // forward substitution alone (ILVES-F with its stored factor): the DIAG tasks of a level
    __device__ __forceinline__ void part_forward_level(int t0, int t1, int p0, int np, int r, int& e) {
        for (int t = t0 + r; t < t1; t += kPartThreads) {
            const int n = (int)(PTK[t].y >> 24);
            if (t < t0 + np) {
                const int pl = p0 + (t - t0);
                LP yv = LP(0);
                for (int k = e; k < e + n; ++k) {
                    const uint2 tr = PTM[k];
                    const uint32_t m = tr.y;
                    yv += VS[tr.x & 0xFFFFu] * reinterpret_cast<const LP*>(RFS + m)[3] * YS[m];
                }
                const LP ny = YS[pl] - yv;
                YS[pl] = ny;
                if (wt) Y[P0 + pl] = ny;
            }
            e += n;
        }
    }
    // backward substitution for part pivot pl (local position)
    __device__ __forceinline__ void part_backward(int pl) {
        const uint32_t pv = PPIV[pl];
        const int us = (int)(pv & 0xFFFFu), nu = (int)(pv >> 16);
        LP dl = YS[pl];
        for (int k = 0; k < nu; ++k) {
            const uint32_t q = PTK[us + k].x >> 16;
            const LP yq = (q & kPartSep) ? SEPY[q & ~kPartSep] : YS[q];
            dl -= VS[us + k] * yq;
        }
        const LP r = dl * reinterpret_cast<const LP*>(RFS + pl)[3];
        YS[pl] = r;
        if (wt) Y[P0 + pl] = r;
    }

    // ---- S1
    // weights of atom a; with stage_ref, x_old is staged in X for s1_constraint
    __device__ __forceinline__ void s1_atom(int a, bool stage_ref) {
        const int64_t g = gid(a);
        if (stage_ref) {
            X[a] = A->x_old[3 * g];
            X[na + a] = A->x_old[3 * g + 1];
            X[2 * na + a] = A->x_old[3 * g + 2];
        }
        const double w = A->inv_mass[g];
        W[a] = DF ? as_bits(df_split(w)) : w;
        WL[a] = to_lp<LP>(w);
    }
    __device__ __forceinline__ void s1_dummy() {
        W[na] = 0.0;
        WL[na] = LP(0);
    }
    // rho, assembly data, lambda0 of constraint p; ref_staged: x_old staged in X (else
    // global); part_staged (partitioned, both atoms in the CTA's part): x_old in X, x_unc
    // in the part copy XS, weights in WL, so the inputs are read once per atom, in order
    __device__ __forceinline__ void s1_constraint(int p, bool ref_staged, bool part_staged = false) {
        const ConA<IdxT> c = cons(p);
        const int i = c.i, j = c.j;
        const int64_t gi = gid(i), gj = gid(j);
        ref_staged = ref_staged || part_staged;
        auto unc = [&](int cc, int a, int64_t ga) {
            return part_staged ? XS[cc * (A1 - A0) + (a - A0)] : A->x_unc[3 * ga + cc];
        };
        double rx, ry, rz;
        if (ref_staged) {
            rx = X[i] - X[j];
            ry = X[na + i] - X[na + j];
            rz = X[2 * na + i] - X[2 * na + j];
        } else {
            rx = A->x_old[3 * gi] - A->x_old[3 * gj];
            ry = A->x_old[3 * gi + 1] - A->x_old[3 * gj + 1];
            rz = A->x_old[3 * gi + 2] - A->x_old[3 * gj + 2];
        }
        V4 v;
        v.x = to_lp<LP>(rx);
        v.y = to_lp<LP>(ry);
        v.z = to_lp<LP>(rz);
        v.w = part_staged ? *(WL + i) + *(WL + j) : to_lp<LP>(A->inv_mass[gi]) + to_lp<LP>(A->inv_mass[gj]);
        RHOF[p] = v;
        const int32_t g = gid_of_con(p);
        const double dd = A->d[g];
        if constexpr (DF) {
            RHOL[p] = df_split(rx).lo;
            RHOL[nc + p] = df_split(ry).lo;
            RHOL[2 * nc + p] = df_split(rz).lo;
            D2[p] = as_bits(df_split(dd * dd));
            SK[p] = as_bits(df_split(unc(0, i, gi) - unc(0, j, gj)));
            SK[nc + p] = as_bits(df_split(unc(1, i, gi) - unc(1, j, gj)));
            SK[2 * nc + p] = as_bits(df_split(unc(2, i, gi) - unc(2, j, gj)));
        } else {
            RHO[p] = rx;
            RHO[nc + p] = ry;
            RHO[2 * nc + p] = rz;
            D2[p] = dd * dd;
        }
        float l0 = A->lambda0 ? A->lambda0[g] : 0.0f;
        if (A->start_diag) {
            float o[6];  // x_old,i - x_old,j and x_unc,i - x_unc,j, per coordinate rounded first
            for (int c = 0; c < 3; ++c) {
                o[c] = ref_staged ? narrow(X[c * na + i]) - narrow(X[c * na + j])
                                  : narrow(A->x_old[3 * gi + c]) - narrow(A->x_old[3 * gj + c]);
                o[3 + c] = narrow(unc(c, i, gi)) - narrow(unc(c, j, gj));
            }
            l0 = diag_start(o[3], o[4], o[5], o[0], o[1], o[2], narrow(dd),
                            part_staged ? f32_of(*(WL + i)) + f32_of(*(WL + j))
                                        : narrow(A->inv_mass[gi]) + narrow(A->inv_mass[gj]));
        }
        LAM[p] = DF ? as_bits(dfloat{l0, 0.0f}) : widen(l0);
        y_st(p, (LP)l0);
    }
    // partitioned S1 with part copies: x_unc of atom a into the part copy XS only (raw
    // values, every mode), then, after the constraints, into X (s1_atom_unc_staged)
    __device__ __forceinline__ void s1_stage_unc(int a) {
        const int64_t g = gid(a);
        for (int c = 0; c < 3; ++c) XS[c * (A1 - A0) + (a - A0)] = A->x_unc[3 * g + c];
    }
    __device__ __forceinline__ void s1_atom_unc_staged(int a) {
        for (int c = 0; c < 3; ++c) x_st(c, a, DF ? 0.0 : XS[c * (A1 - A0) + (a - A0)]);
    }
    __device__ __forceinline__ void s1_atom_unc(int a) {
        if constexpr (DF) {  // displacements start at zero
            x_st(0, a, 0.0);
            x_st(1, a, 0.0);
            x_st(2, a, 0.0);
        } else {
            const int64_t g = gid(a);
            x_st(0, a, A->x_unc[3 * g]);
            x_st(1, a, A->x_unc[3 * g + 1]);
            x_st(2, a, A->x_unc[3 * g + 2]);
        }
    }

    // ---- S1, shared-memory state: one batch of asynchronous gathers, then local passes.
    // x_old -> STG (AoS); x_unc -> X (SoA; AoS in the float-float mode, where X is free
    // until the displacements start); inv_mass -> W, d -> D2, lambda0 -> Y as raw values.
    //      The reads run over atom slots, so consecutive lanes read consecutive addresses.
    __device__ __forceinline__ void s1_gather(int r0, int ts) {
        for (int e = r0; e < 3 * na; e += ts) {
            const int o = e / 3, c = e - 3 * o, a = (int)aslot[o];
            const int64_t g = 3 * slot_gid(o) + c;
            cp_async8(STG + 3 * a + c, A->x_old + g);
            cp_async8(DF ? X + 3 * a + c : X + c * na + a, A->x_unc + g);
        }
        for (int o = r0; o < na; o += ts) cp_async8(W + aslot[o], A->inv_mass + slot_gid(o));
        for (int p = r0; p < nc; p += ts) {
            const int32_t g = gid_of_con(p);
            cp_async8(D2 + p, A->d + g);
            if (A->lambda0 && !A->start_diag) cp_async4(reinterpret_cast<float*>(Y + p), A->lambda0 + g);
        }
        cp_async_wait_all();
    }
    __device__ __forceinline__ void s1_atom_local(int a) {
        const double w = *(W + a);
        if constexpr (DF) W[a] = as_bits(df_split(w));
        WL[a] = to_lp<LP>(w);
    }
    __device__ __forceinline__ void s1_constraint_local(int p) {
        const ConA<IdxT> c = cons(p);
        const int i = c.i, j = c.j;
        const double rx = *(STG + 3 * i) - *(STG + 3 * j);
        const double ry = *(STG + 3 * i + 1) - *(STG + 3 * j + 1);
        const double rz = *(STG + 3 * i + 2) - *(STG + 3 * j + 2);
        V4 v;
        v.x = to_lp<LP>(rx);
        v.y = to_lp<LP>(ry);
        v.z = to_lp<LP>(rz);
        v.w = *(WL + i) + *(WL + j);
        RHOF[p] = v;
        const double dd = *(D2 + p);
        if constexpr (DF) {
            RHOL[p] = df_split(rx).lo;
            RHOL[nc + p] = df_split(ry).lo;
            RHOL[2 * nc + p] = df_split(rz).lo;
            D2[p] = as_bits(df_split(dd * dd));
            SK[p] = as_bits(df_split(*(X + 3 * i) - *(X + 3 * j)));
            SK[nc + p] = as_bits(df_split(*(X + 3 * i + 1) - *(X + 3 * j + 1)));
            SK[2 * nc + p] = as_bits(df_split(*(X + 3 * i + 2) - *(X + 3 * j + 2)));
        } else {
            RHO[p] = rx;
            RHO[nc + p] = ry;
            RHO[2 * nc + p] = rz;
            D2[p] = dd * dd;
        }
        float l0 = A->lambda0 ? *(reinterpret_cast<const float*>(Y + p)) : 0.0f;
        if (A->start_diag) {  // x_unc is in X (AoS in the float-float mode, else SoA)
            float u[3];
            for (int c = 0; c < 3; ++c)
                u[c] = DF ? narrow(*(X + 3 * i + c)) - narrow(*(X + 3 * j + c))
                          : narrow(*(X + c * na + i)) - narrow(*(X + c * na + j));
            l0 = diag_start(u[0], u[1], u[2], narrow(*(STG + 3 * i)) - narrow(*(STG + 3 * j)),
                            narrow(*(STG + 3 * i + 1)) - narrow(*(STG + 3 * j + 1)),
                            narrow(*(STG + 3 * i + 2)) - narrow(*(STG + 3 * j + 2)), narrow(dd),
                            f32_of(*(WL + i)) + f32_of(*(WL + j)));
        }
        LAM[p] = DF ? as_bits(dfloat{l0, 0.0f}) : widen(l0);
        Y[p] = (LP)l0;
    }

    // ---- S6: x_a -= w_a sum_k s_k(a) 2 Y_k rho_k   (Y holds delta, or lambda0).
    //      upd_eval computes the new coordinates (float64 class, as bit patterns),
    //      upd_store writes them.
    struct Upd { double x, y, z; };
    __device__ __forceinline__ Upd upd_eval(int a) const {
        const int e1 = ldp<kCoh>(inc_ptr + a + 1);
        if constexpr (DF) {
            dfloat ax{0.f, 0.f}, ay{0.f, 0.f}, az{0.f, 0.f};
            for (int e = ldp<kCoh>(inc_ptr + a); e < e1; ++e) {
                const unsigned v = ldp<kCoh>(inc + e);
                const int p = (int)(v >> 1);
                const float dl = (float)y_ld(p);
                const float c = (v & 1u) ? -(dl + dl) : (dl + dl);
                const V4 hi = *(RHOF + p);
                ax = df_add(ax, df_mul_f(dfloat{hi.x, *(RHOL + p)}, c));
                ay = df_add(ay, df_mul_f(dfloat{hi.y, *(RHOL + nc + p)}, c));
                az = df_add(az, df_mul_f(dfloat{hi.z, *(RHOL + 2 * nc + p)}, c));
            }
            const dfloat w = as_df(*(W + a));
            return {as_bits(df_sub(as_df(x_ld(0, a, false)), df_mul(w, ax))),
                    as_bits(df_sub(as_df(x_ld(1, a, false)), df_mul(w, ay))),
                    as_bits(df_sub(as_df(x_ld(2, a, false)), df_mul(w, az)))};
        } else {
            double ax = 0.0, ay = 0.0, az = 0.0;
            for (int e = ldp<kCoh>(inc_ptr + a); e < e1; ++e) {
                const unsigned v = ldp<kCoh>(inc + e);
                const int p = (int)(v >> 1);
                const LP dl = y_ld(p);
                const double c = to_hp((v & 1u) ? -(dl + dl) : (dl + dl));
                ax = fma(c, *(RHO + p), ax);
                ay = fma(c, *(RHO + nc + p), ay);
                az = fma(c, *(RHO + 2 * nc + p), az);
            }
            const double w = *(W + a);
            return {fma(-w, ax, x_ld(0, a, false)), fma(-w, ay, x_ld(1, a, false)), fma(-w, az, x_ld(2, a, false))};
        }
    }
    __device__ __forceinline__ void upd_store(int a, const Upd& u) {
        x_st(0, a, u.x);
        x_st(1, a, u.y);
        x_st(2, a, u.z);
    }
    __device__ __forceinline__ void update_atom(int a) { upd_store(a, upd_eval(a)); }

    // ---- S2: violation of constraint p (float64 class), Jacobian row, right-hand side.
    //      viol_eval computes, viol_store writes (rows = false keeps RF: ILVES-F after its
    //      first iteration, where RF.w holds the stored factor's reciprocal pivots and the
    //      Jacobian rows are not needed).
    struct Viol { V4 v; LP y; bool conv, bad; };
    __device__ __forceinline__ Viol viol_eval(int p) const {
        const ConA<IdxT> cc = cons(p);
        const int i = cc.i, j = cc.j;
        const bool fx = foreign(p);
        Viol o;
        if constexpr (DF) {
            const dfloat rx = df_add(as_df(*(SK + p)), df_sub(as_df(x_ld(0, i, fx)), as_df(x_ld(0, j, fx))));
            const dfloat ry = df_add(as_df(*(SK + nc + p)),
                                     df_sub(as_df(x_ld(1, i, fx)), as_df(x_ld(1, j, fx))));
            const dfloat rz = df_add(as_df(*(SK + 2 * nc + p)),
                                     df_sub(as_df(x_ld(2, i, fx)), as_df(x_ld(2, j, fx))));
            const dfloat d2 = as_df(*(D2 + p));
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
            o.conv = fabsf(sg) <= tolf * d2.hi;
            o.bad = nonfinite(sg);
            o.v.x = rx.hi;
            o.v.y = ry.hi;
            o.v.z = rz.hi;
            o.y = sg;
        } else {
            const double rx = x_ld(0, i, fx) - x_ld(0, j, fx);
            const double ry = x_ld(1, i, fx) - x_ld(1, j, fx);
            const double rz = x_ld(2, i, fx) - x_ld(2, j, fx);
            const double d2 = *(D2 + p);
            const double sg = fma(rx, rx, fma(ry, ry, fma(rz, rz, -d2)));
            o.conv = abs_le(sg, A->tol * d2);
            o.bad = nonfinite(sg);
            o.v.x = to_lp<LP>(rx);
            o.v.y = to_lp<LP>(ry);
            o.v.z = to_lp<LP>(rz);
            o.y = to_lp<LP>(sg);
        }
        o.v.w = LP(0);
        return o;
    }
    __device__ __forceinline__ void viol_store(int p, const Viol& o, bool rows) {
        y_st(p, o.y);
        if (rows) rf_st(p, o.v);
    }
    __device__ __forceinline__ void violation(int p, bool& conv, bool& bad, bool rows = true) {
        const Viol o = viol_eval(p);
        conv = conv && o.conv;
        bad = bad || o.bad;
        viol_store(p, o, rows);
    }

    // ---- S3 + S4 + forward S5: one task writing value slot t, with terms [e0, e1);
    //      DIAG tasks (diag = true) also produce 1/pivot and the forward-solve entry.
    //      Every entry is a - sum_m Lt[row,m] inv_m U[m,col], a = 4 s s' w_atom r_row . rho_col
    //      (for DIAG entries w_atom = w_i + w_j, kept in RHOF[row].w).
    __device__ __forceinline__ LP assemble(int row, int col, int atom, bool neg, bool diag) const {
        const V4 rr = rf_ld(row), pp = *(RHOF + col);
        const LP wv = diag ? pp.w : *(WL + atom);
        const LP c = neg ? LP(-4) * wv : LP(4) * wv;
        return c * (rr.x * pp.x + rr.y * pp.y + rr.z * pp.z);
    }
    __device__ __forceinline__ void task_core(int t, int row, int col, int atom, bool neg, int e0, int e1, bool diag,
                                              bool& singular) {
        finish(t, row, assemble(row, col, atom, neg, diag), e0, e1, diag, singular);
    }
    // a - sum over terms [e0, e1) -> value slot t (and, for DIAG, 1/pivot and y_row)
    __device__ __forceinline__ void finish(int t, int row, LP a, int e0, int e1, bool diag, bool& singular) {
        LP sacc = a, yv = LP(0);
#pragma unroll 2
        for (int e = e0; e < e1; ++e) {
            const auto tr = ldp<kCoh>(terms + e);
            const int m = TO::m(tr);
            const bool fm = foreign(m);
            const LP li = v_ld(TO::l(tr), fm) * inv(m);
            sacc -= li * v_ld(TO::u(tr), fm);
            if (diag) yv += li * y_ld(m);
        }
        v_st(t, sacc);
        if (diag) {
            singular = singular || !(lp_abs(sacc) > Mode::pivot_rel * lp_abs(a));
            inv_st(row, lp_rcp(sacc));
            y_st(row, y_ld(row) - yv);
        }
    }
    // large molecules: task records with term pointers
    __device__ __forceinline__ void task(int t, bool diag, bool& singular) {
        const TaskT tk = ldp<kCoh>(tasks + t);
        const int e1 = ldp<kCoh>(tasks + t + 1).tstart;
        task_core(t, tk.row, tk.col, tk.atomsign >> 1, tk.atomsign & 1, tk.tstart, e1, diag, singular);
    }
    // batched molecules: one level's tasks t0 + lane + kTeam k for a team of kTeam threads
    //      (the width the program was laid out for); the lane walks its terms from offset e
    template <int kTeam>
    __device__ __forceinline__ void level_tasks(int t0, int t1, int np, int lane, int& e, bool& singular) {
        for (int t = t0 + lane; t < t1; t += kTeam) {
            const uint32_t w = lds<kCoh>(tasks + t);
            const int n = (int)TaskWord::nterm(w);
            const bool diag = t < t0 + np;
            finish(t, TaskWord::row(w),
                   assemble(TaskWord::row(w), TaskWord::col(w), TaskWord::atom(w), TaskWord::neg(w), diag), e, e + n,
                   diag, singular);
            e += n;
        }
    }

    // ---- forward S5 alone (ILVES-F iterations after the first): y_p -= sum_m L[p,m] y_m,
    //      with the terms [e0, e1) of pivot p's DIAG task
    __device__ __forceinline__ void forward_terms(int p, int e0, int e1) {
        LP yv = LP(0);
        for (int e = e0; e < e1; ++e) {
            const auto tr = ldp<kCoh>(terms + e);
            const int m = TO::m(tr);
            const bool fm = foreign(m);
            yv += v_ld(TO::l(tr), fm) * inv(m) * y_ld(m);
        }
        y_st(p, y_ld(p) - yv);
    }
    __device__ __forceinline__ void forward(int t, int p) {
        forward_terms(p, ldp<kCoh>(tasks + t).tstart, ldp<kCoh>(tasks + t + 1).tstart);
    }
    // ILVES-F assembles A(x_old, x_old): the Jacobian rows are the reference bonds
    __device__ __forceinline__ void chord_rows(int p) { rf_st(p, *(RHOF + p)); }

    // ---- backward S5 for pivot p: delta_p = inv_p (y_p - sum_q U[p,q] delta_q)
    __device__ __forceinline__ int task_col(int t) const {
        if constexpr (kCompact) return (int)TaskWord::col(ldp<kCoh>(tasks + t));
        else return (int)ldp<kCoh>(tasks + t).col;
    }
    __device__ __forceinline__ void backward(int p) {
        const Piv<IdxT> pv = ldp<kCoh>(piv + p);
        const int us = pv.diag, nu = pv.nup;
        const bool fp = foreign(p);
        LP dl = y_ld(p);
        for (int k = 0; k < nu; ++k) {
            const int q = task_col(us + k);
            dl -= v_ld(us + k, fp) * y_ld(q);
        }
        y_st(p, dl * inv(p));
    }
    // ---- partitioned molecules: part-side Schur contribution entry c (factor: the L inv U
    //      sum as well; DIAG tasks: the L inv y sum of the forward solve)
    __device__ __forceinline__ void contrib(int c, bool factor) {
        const Contrib E = ldp<kCoh>(cent + c);
        const TaskT tk = ldp<kCoh>(tasks + E.task);
        const bool diag = tk.row == tk.col;
        LP sv = LP(0), sy = LP(0);
        for (uint32_t e = E.e0; e < E.e1; ++e) {
            const auto tr = ldp<kCoh>(terms + e);
            const int m = TO::m(tr);
            const bool fm = foreign(m);
            const LP li = v_ld(TO::l(tr), fm) * inv(m);
            if (factor) sv += li * v_ld(TO::u(tr), fm);
            if (diag) sy += li * y_ld(m);
        }
        LP* ct = CT + 4 * (E.task - sep_t0);
        if (factor) ct[E.slot] = sv;
        if (diag) ct[2 + E.slot] = sy;
    }
    // separator task t: the parts' contributions, then its remaining terms
    __device__ __forceinline__ void task_sep(int t, bool diag, bool& singular) {
        const TaskT tk = ldp<kCoh>(tasks + t);
        const int e1 = ldp<kCoh>(tasks + t + 1).tstart;
        const SepInfo si = ldp<kCoh>(sep_info + (t - sep_t0));
        const LP a = assemble(tk.row, tk.col, tk.atomsign >> 1, tk.atomsign & 1, diag);
        const LP* ct = CT + 4 * (t - sep_t0);
        LP sacc = a, yv = LP(0);
        for (uint32_t g = 0; g < si.ngroups; ++g) {
            sacc -= lds<kCoh>(ct + g);
            if (diag) yv += lds<kCoh>(ct + 2 + g);
        }
        for (int e = (int)si.b_start; e < e1; ++e) {
            const auto tr = ldp<kCoh>(terms + e);
            const int m = TO::m(tr);
            const LP li = lds<kCoh>(V + TO::l(tr)) * inv(m);
            sacc -= li * lds<kCoh>(V + TO::u(tr));
            if (diag) yv += li * lds<kCoh>(Y + m);
        }
        V[t] = sacc;
        if (diag) {
            singular = singular || !(lp_abs(sacc) > Mode::pivot_rel * lp_abs(a));
            *inv_ptr(tk.row) = lp_rcp(sacc);
            Y[tk.row] = lds<kCoh>(Y + tk.row) - yv;
        }
    }
    // forward solve alone for separator pivot p (DIAG task t)
    __device__ __forceinline__ void forward_sep(int t, int p) {
        const SepInfo si = ldp<kCoh>(sep_info + (t - sep_t0));
        const LP* ct = CT + 4 * (t - sep_t0);
        LP yv = LP(0);
        for (uint32_t g = 0; g < si.ngroups; ++g) yv += lds<kCoh>(ct + 2 + g);
        const int e1 = ldp<kCoh>(tasks + t + 1).tstart;
        for (int e = (int)si.b_start; e < e1; ++e) {
            const auto tr = ldp<kCoh>(terms + e);
            const int m = TO::m(tr);
            yv += lds<kCoh>(V + TO::l(tr)) * inv(m) * lds<kCoh>(Y + m);
        }
        Y[p] = lds<kCoh>(Y + p) - yv;
    }

    // ---- the separator phase in shared memory (one CTA), from the separator program
    //      (SepProgHeader; SLP .. STM point into its shared-memory copy): SV = values of
    //      the separator tasks, SRF = Jacobian rows of the separators (.w = 1 / pivot), SY
    //      = their right-hand side / solution; indices local to the separator block.
    //      Terms of interior pivots beyond the parts' contributions read the global state.
    //      SP = the separators' reference rows, SC = each task's assembly coefficient
    //      (4 s s' w), both fixed for the whole solve.
    const uint16_t *SLP = nullptr, *SLT = nullptr;
    const uint32_t* SPV = nullptr;
    const uint2 *STK = nullptr, *STM = nullptr;
    __device__ __forceinline__ void sep_prog_bind(const uint8_t* sp) {
        const SepProgHeader* h = reinterpret_cast<const SepProgHeader*>(sp);
        const SepProgLayout L = sep_prog_layout(h->nsep, h->nt, h->nlev, h->nterm);
        SLP = reinterpret_cast<const uint16_t*>(sp + L.lvl_piv);
        SLT = reinterpret_cast<const uint16_t*>(sp + L.lvl_task);
        SPV = reinterpret_cast<const uint32_t*>(sp + L.piv);
        STK = reinterpret_cast<const uint2*>(sp + L.tasks);
        STM = reinterpret_cast<const uint2*>(sp + L.terms);
    }
    // the factors of one term: L[row,m] inv_m, U[m,col] and y_m
    __device__ __forceinline__ void sep_term(const uint2 tr, const LP* SV, const V4* SRF, const LP* SY, LP& li, LP& u,
                                             LP& ym) const {
        if (tr.x != kSepInterior) {
            const uint32_t m = tr.y;
            li = SV[tr.x & 0xFFFFu] * reinterpret_cast<const LP*>(SRF + m)[3];
            u = SV[tr.x >> 16];
            ym = SY[m];
        } else {  // an interior pivot past the parts' two contribution slots
            const auto g = ldp<kCoh>(terms + tr.y);
            const int m = TO::m(g);
            li = lds<kCoh>(V + TO::l(g)) * lds<kCoh>(inv_ptr(m));
            u = lds<kCoh>(V + TO::u(g));
            ym = lds<kCoh>(Y + m);
        }
    }
    __device__ __forceinline__ static int sep_e(const uint2 w) { return (int)(w.y & 0x3FFFFFFFu); }
    // separator task tl (local), one thread
    __device__ __forceinline__ void sep_task_smem(int tl, bool diag, bool& singular, LP* SV, V4* SRF, LP* SY,
                                                  const V4* SP, const LP* SC) const {
        const uint2 w = STK[tl];
        const int e1 = sep_e(STK[tl + 1]);
        const int row = (int)(w.x & 0xFFFFu), col = (int)(w.x >> 16);
        const V4 rr = SRF[row], pp = SP[col];
        const LP a = SC[tl] * (rr.x * pp.x + rr.y * pp.y + rr.z * pp.z);
        LP sacc = a + SV[tl], yv = LP(0);  // SV, SY hold minus the parts' contributions
        for (int e = sep_e(w); e < e1; ++e) {
            LP li, u, ym;
            sep_term(STM[e], SV, SRF, SY, li, u, ym);
            sacc -= li * u;
            if (diag) yv += li * ym;
        }
        SV[tl] = sacc;
        if (diag) {
            singular = singular || !(lp_abs(sacc) > Mode::pivot_rel * lp_abs(a));
            reinterpret_cast<LP*>(SRF + row)[3] = lp_rcp(sacc);
            SY[row] -= yv;
        }
    }
    // one level with g lanes per task (g a power of two up to 32; the narrow last levels,
    //      where few pivots carry many terms): the lanes of a group split the task's
    //      terms and reduce them with shuffles within the group.  Every thread runs the
    //      same number of passes, so the shuffles see whole warps.
    __device__ __forceinline__ void sep_level_groups(int t0, int t1, int np, int g, int r0, int ts, bool& singular,
                                                     LP* SV, V4* SRF, LP* SY, const V4* SP, const LP* SC) const {
        const int sub = r0 & (g - 1), per_pass = ts / g;
        for (int tb = t0; tb < t1; tb += per_pass) {
            const int tl = tb + r0 / g;
            const bool act = tl < t1, diag = tl < t0 + np;
            LP ps = LP(0), py = LP(0);
            uint2 w = make_uint2(0u, 0u);
            if (act) {
                w = STK[tl];
                const int e1 = sep_e(STK[tl + 1]);
                for (int e = sep_e(w) + sub; e < e1; e += g) {
                    LP li, u, ym;
                    sep_term(STM[e], SV, SRF, SY, li, u, ym);
                    ps += li * u;
                    if (diag) py += li * ym;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                if (o < g) {  // uniform over the warp
                    ps += __shfl_xor_sync(0xFFFFFFFFu, ps, o);
                    py += __shfl_xor_sync(0xFFFFFFFFu, py, o);
                }
            }
            if (act && sub == 0) {
                const int row = (int)(w.x & 0xFFFFu), col = (int)(w.x >> 16);
                const V4 rr = SRF[row], pp = SP[col];
                const LP a = SC[tl] * (rr.x * pp.x + rr.y * pp.y + rr.z * pp.z);
                const LP sacc = a + SV[tl] - ps;
                SV[tl] = sacc;
                if (diag) {
                    singular = singular || !(lp_abs(sacc) > Mode::pivot_rel * lp_abs(a));
                    reinterpret_cast<LP*>(SRF + row)[3] = lp_rcp(sacc);
                    SY[row] -= py;
                }
            }
        }
    }
    // forward substitution alone for separator pivot pl (its DIAG task tl)
    __device__ __forceinline__ void sep_forward_smem(int tl, int pl, const LP* SV, const V4* SRF, LP* SY) const {
        LP yv = LP(0);
        const int e1 = sep_e(STK[tl + 1]);
        for (int e = sep_e(STK[tl]); e < e1; ++e) {
            LP li, u, ym;
            sep_term(STM[e], SV, SRF, SY, li, u, ym);
            yv += li * ym;
        }
        SY[pl] -= yv;
    }
    // staging of separator task tl: the parts' contributions CS (4 per task: two partial
    //      sums of L inv U, two of L inv y), summed, go into SV (as its negative start
    //      value, factor iterations only) and, for a DIAG task, into the right-hand side
    //      SY of its pivot
    //      (CS in shared memory, or the global CT when cs_global)
    __device__ __forceinline__ void sep_stage_smem(int tl, bool factor, const LP* CS, bool cs_global, LP* SV,
                                                   LP* SY) const {
        const uint2 w = STK[tl];
        const uint32_t ng = w.y >> 30;
        LP cv = LP(0), cy = LP(0);
        for (uint32_t g = 0; g < ng; ++g) {
            cv += cs_global ? lds<kCoh>(CS + 4 * tl + g) : CS[4 * tl + g];
            cy += cs_global ? lds<kCoh>(CS + 4 * tl + 2 + g) : CS[4 * tl + 2 + g];
        }
        if (factor) SV[tl] = -cv;
        if ((w.x & 0xFFFFu) == (w.x >> 16)) SY[w.x & 0xFFFFu] -= cy;
    }
    // assembly coefficient 4 s s' w of separator task tl (w_i + w_j for a pivot)
    __device__ __forceinline__ LP sep_coef(int tl) const {
        const TaskT tk = ldp<kCoh>(tasks + sep_t0 + tl);
        const LP wv = tk.row == tk.col ? lds<kCoh>(RHOF + tk.row).w : lds<kCoh>(WL + (tk.atomsign >> 1));
        return (tk.atomsign & 1) ? LP(-4) * wv : LP(4) * wv;
    }
    __device__ __forceinline__ void sep_backward_smem(int pl, const LP* SV, const V4* SRF, LP* SY) const {
        const uint32_t pv = SPV[pl];
        const int us = (int)(pv & 0xFFFFu), nu = (int)(pv >> 16);
        LP dl = SY[pl];
        for (int k = 0; k < nu; ++k) dl -= SV[us + k] * SY[STK[us + k].x >> 16];
        SY[pl] = dl * reinterpret_cast<const LP*>(SRF + pl)[3];
    }

    __device__ __forceinline__ void lambda_acc(int p) {
        const LP dl = y_ld(p);
        if constexpr (DF) LAM[p] = as_bits(df_add_f(as_df(*(LAM + p)), (float)dl));
        else LAM[p] = *(LAM + p) + to_hp(dl);
    }

    // ---- S7
    __device__ __forceinline__ void out_atom(int a) {
        const int64_t g = gid(a);
        if constexpr (DF) {
            A->x_out[3 * g] = A->x_unc[3 * g] + df_join(as_df(*(X + a)));
            A->x_out[3 * g + 1] = A->x_unc[3 * g + 1] + df_join(as_df(*(X + na + a)));
            A->x_out[3 * g + 2] = A->x_unc[3 * g + 2] + df_join(as_df(*(X + 2 * na + a)));
        } else {
            A->x_out[3 * g] = *(X + a);
            A->x_out[3 * g + 1] = *(X + na + a);
            A->x_out[3 * g + 2] = *(X + 2 * na + a);
        }
    }
    // batched molecules: the positions, one coordinate per lane in global order
    __device__ __forceinline__ void out_atoms_by_slot(int r0, int ts) {
        for (int e = r0; e < 3 * na; e += ts) {
            const int o = e / 3, c = e - 3 * o, a = (int)aslot[o];
            const int64_t g = 3 * slot_gid(o) + c;
            if constexpr (DF) A->x_out[g] = A->x_unc[g] + df_join(as_df(*(X + c * na + a)));
            else A->x_out[g] = *(X + c * na + a);
        }
    }
    __device__ __forceinline__ void out_lambda(int p) {
        const double l = *(LAM + p);
        A->lambda_out[gid_of_con(p)] = DF ? df_join(as_df(l)) : l;
    }
};

// ------------------------------------------------------------------------------------
// one molecule, one team (a warp with state in shared memory, or a CTA with state in a
// global workspace)
// ------------------------------------------------------------------------------------
template <class Mode, class IdxT, class Team>
__device__ void solve_molecule(const Team& tm, const MolDesc& D, const uint8_t* prog, uint8_t* st,
                               const SolveArgs& A, const uint8_t* gprog) {
    constexpr bool kCompact = sizeof(IdxT) == 2;  // batched-kernel molecules (a SlotTeamT)
    MolView<Mode, IdxT, false> M;
    M.init(D, prog, st, A, gprog);
    const int na = D.na, nc = D.nc;
    const int r0 = tm.rank(), ts = tm.size();
    // ---- S1
    if constexpr (IsSlotTeam<Team>::value) {
        M.s1_gather(r0, ts);
        tm.sync();
        for (int a = r0; a < na; a += ts) M.s1_atom_local(a);
        if (r0 == 0) M.s1_dummy();
        tm.sync();
        for (int p = r0; p < nc; p += ts) M.s1_constraint_local(p);
        tm.sync();
        if constexpr (Mode::df) {
            for (int a = r0; a < na; a += ts) M.s1_atom_unc(a);
            tm.sync();
        }
    } else {
        for (int a = r0; a < na; a += ts) M.s1_atom(a, true);
        if (r0 == 0) M.s1_dummy();
        tm.sync();
        for (int p = r0; p < nc; p += ts) M.s1_constraint(p, true);
        tm.sync();
        for (int a = r0; a < na; a += ts) M.s1_atom_unc(a);
        tm.sync();
    }
    if (A.has_start()) {  // x = x_unc - M^-1 G(x_old)^T lambda0
        for (int a = r0; a < na; a += ts) M.update_atom(a);
        tm.sync();
    }
    int status = ILVES_MOL_MAX_ITER, iters = A.max_iter;
    for (int it = 0;; ++it) {
        bool conv = true, bad = false;
        for (int p = r0; p < nc; p += ts) M.violation(p, conv, bad, !A.chord || it == 0);
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
        if (!A.chord || it == 0) {
            if (A.chord) {  // ILVES-F: factorise A(x_old, x_old) once
                for (int p = r0; p < nc; p += ts) M.chord_rows(p);
                tm.sync();
            }
            // one pass per level; the first np tasks of a level are its DIAG tasks; a warp
            // lane walks its terms with a running offset
            bool singular = false;
            int e = kCompact ? (int)M.lane_term[r0] : 0;
            for (int l = 0; l < D.nlevel; ++l) {
                const int p0 = M.lvl_piv[l], np = M.lvl_piv[l + 1] - p0;
                const int t0 = M.lvl_task[l], t1 = M.lvl_task[l + 1];
                if constexpr (kCompact) {
                    M.template level_tasks<Team::kSize>(t0, t1, np, r0, e, singular);
                } else {
                    for (int t = t0 + r0; t < t1; t += ts) M.task(t, t < t0 + np, singular);
                }
                tm.sync();
            }
            if (tm.any(singular)) {
                status = ILVES_MOL_SINGULAR_PIVOT;
                iters = it;
                break;
            }
        } else {  // ILVES-F: forward substitution with the stored factor
            int e = kCompact ? (int)M.lane_term[r0] : 0;
            for (int l = 0; l < D.nlevel; ++l) {
                const int p0 = M.lvl_piv[l], p1 = M.lvl_piv[l + 1], t0 = M.lvl_task[l];
                if constexpr (kCompact) {  // DIAG tasks: t0 + (p - p0); skip the others' terms
                    const int t1 = M.lvl_task[l + 1];
                    for (int t = t0 + r0; t < t1; t += ts) {
                        const int n = (int)TaskWord::nterm(M.tasks[t]);
                        if (t < t0 + (p1 - p0)) M.forward_terms(p0 + (t - t0), e, e + n);
                        e += n;
                    }
                } else {
                    for (int p = p0 + r0; p < p1; p += ts) M.forward(t0 + (p - p0), p);
                }
                tm.sync();
            }
        }
        for (int l = D.nlevel - 1; l >= 0; --l) {
            const int p1 = M.lvl_piv[l + 1];
            for (int p = M.lvl_piv[l] + r0; p < p1; p += ts) M.backward(p);
            tm.sync();
        }
        for (int p = r0; p < nc; p += ts) M.lambda_acc(p);
        for (int a = r0; a < na; a += ts) M.update_atom(a);
        tm.sync();
    }
    if constexpr (kCompact) M.out_atoms_by_slot(r0, ts);
    else
        for (int a = r0; a < na; a += ts) M.out_atom(a);
    if (A.lambda_out)
        for (int p = r0; p < nc; p += ts) M.out_lambda(p);
    if (r0 == 0) {
        if (A.iterations_out) A.iterations_out[D.mol_id] = iters;
        if (A.status_out) A.status_out[D.mol_id] = status;
    }
}

// ------------------------------------------------------------------------------------
// partitioned molecule: all CTAs of a cooperative launch (supplement Sec. 3: private
// partitions eliminated in parallel, contributions to the shared partition, the shared
// block factorised by one worker, back substitution in parallel)
// ------------------------------------------------------------------------------------
constexpr long long kSpinBudget = 1ll << 22;  // bounded wait: ~0.3 s of polling per launch

// Arrive on a monotone 64-bit counter and wait (bounded) until every CTA of this barrier
// generation arrived.  Returns false if the wait gave up.
__device__ __forceinline__ bool grid_sync(unsigned long long* ctr, unsigned n_blocks, long long& budget) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long arrived = atomicAdd(ctr, 1ull) + 1ull;
        const unsigned long long target = ((arrived + n_blocks - 1) / n_blocks) * (unsigned long long)n_blocks;
        int good = 1;
        while (*reinterpret_cast<volatile unsigned long long*>(ctr) < target) {
            if (--budget <= 0) {
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Shared memory of the separator phase: rows (V4) and right-hand sides of the
// separators, values of the separator tasks; the separators' reference rows and the
// tasks' assembly coefficients; with stage_ct, a copy of the parts' contributions (4 per
// task); the separator program.  Used when it fits kPartedSmemMax.
template <class Mode>
__host__ __device__ inline uint32_t sep_smem_bytes(int nsep, int n_sept, int sprog_bytes, bool stage_ct) {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    return 2 * align16((uint32_t)sizeof(V4) * nsep) + align16((uint32_t)sizeof(LP) * nsep) +
           2 * align16((uint32_t)sizeof(LP) * n_sept) + (stage_ct ? align16(4u * (uint32_t)sizeof(LP) * n_sept) : 0u) +
           align16((uint32_t)sprog_bytes);
}

// Shared memory of a part's own copies (X, Y, RF, V) for the largest part.
template <class Mode>
__host__ __device__ inline uint32_t part_smem_bytes(int na, int np, int nt) {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    return align16(24u * na) + align16((uint32_t)sizeof(LP) * np) + align16((uint32_t)sizeof(V4) * np) +
           align16((uint32_t)sizeof(LP) * nt);
}
// The same with the part program staged too: the part's reference rows and weights, then
// the largest part program.
template <class Mode>
__host__ __device__ inline uint32_t part_prog_smem_bytes(int na, int np, int nt, int prog_max) {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    return part_smem_bytes<Mode>(na, np, nt) + align16((uint32_t)sizeof(V4) * np) +
           align16((uint32_t)sizeof(LP) * na) + (uint32_t)prog_max;
}
constexpr uint32_t kPartedSmemMax = 72 * 1024;  // three CTAs per SM still fit

// Dynamic shared memory of a partitioned launch: the separator block (0 = it stays in
// global memory) of CTA sep_cta, and the part copies (0 = off; on only with one part per
// CTA).  With a CTA of its own for the separator block (sep_cta == number of parts) both
// regions start at offset 0 of their CTAs and a launch needs only the larger one, which
// leaves more of each SM's L1 to the parts' programs; otherwise CTA 0 holds both.
struct PartedSmem {
    uint32_t sep_bytes, part_bytes;
    int32_t sep_cta;
    uint32_t prog;    // nonzero: part programs staged too (part_bytes counts them)
    uint32_t sep_ct;  // nonzero: the separator CTA stages the contributions (sep_bytes counts them)
    uint32_t wt;      // nonzero: parts write their factor values, reciprocal pivots, rows and
                      // solve vector through to global memory (the separator phase reads some)
    uint32_t phantom; // testing: CTAs the grid barriers wait for beyond the launch's (never arrive)
};

struct PartSync {
    unsigned long long barrier;
    int notconv[4];
    int bad[4];
    int singular[4];
    int timeout;
};

template <class Mode>
__global__ void __launch_bounds__(256, 3)
k_solve_parted(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob, uint8_t* work, PartSync* sync,
               SolveArgs A, PartedSmem cfg) {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    extern __shared__ __align__(16) uint8_t sep_smem[];
    const MolDesc D = *desc;
    MolView<Mode, uint32_t, true> M;
    M.init(D, blob + D.blob_off, work + D.work_off, A, blob + D.blob_off);
    const int n_parts = D.n_seg - 1;
    const SegRow* seg = M.seg;
    const int sep0 = __ldg(&seg[n_parts].piv), nsep = D.nc - sep0;
    // separator block in shared memory when it fits (the host sized the launch alike)
    const bool sep_in_smem = cfg.sep_bytes > 0;
    V4* SRF = reinterpret_cast<V4*>(sep_smem);
    LP* SY = reinterpret_cast<LP*>(sep_smem + align16((uint32_t)sizeof(V4) * nsep));
    LP* SV = reinterpret_cast<LP*>(sep_smem + align16((uint32_t)sizeof(V4) * nsep) +
                                   align16((uint32_t)sizeof(LP) * nsep));
    V4* SP = reinterpret_cast<V4*>(reinterpret_cast<uint8_t*>(SV) + align16((uint32_t)sizeof(LP) * D.n_sept));
    LP* SC = reinterpret_cast<LP*>(reinterpret_cast<uint8_t*>(SP) + align16((uint32_t)sizeof(V4) * nsep));
    LP* CS = reinterpret_cast<LP*>(reinterpret_cast<uint8_t*>(SC) + align16((uint32_t)sizeof(LP) * D.n_sept));
    uint8_t* SPROG =
        reinterpret_cast<uint8_t*>(CS) + (cfg.sep_ct ? align16(4u * (uint32_t)sizeof(LP) * D.n_sept) : 0u);
    // segment programs: part q's is [poff[q], poff[q + 1]) of the pprog section, the
    // separator block's follows
    const ProgLayout PL = prog_layout<uint32_t>(D.na, D.nc, D.ntask, D.nterm, D.nlevel, D.n_seg, D.n_sept, D.n_cent,
                                                D.pprog_bytes);
    const uint8_t* gp = blob + D.blob_off;
    const uint32_t* poff = reinterpret_cast<const uint32_t*>(gp + PL.pprog_off);
    if (cfg.part_bytes > 0 && (int)blockIdx.x < n_parts) {  // this CTA's part, copied in shared memory
        const int q = blockIdx.x;
        const SegRow s0 = seg[q], s1 = seg[q + 1];
        M.P0 = s0.piv;
        M.P1 = s1.piv;
        M.A0 = s0.atom;
        M.A1 = s1.atom;
        M.T0 = __ldg(M.lvl_task + s0.lvl);
        M.T1 = __ldg(M.lvl_task + s1.lvl - 1);
        uint8_t* pb = sep_smem + (cfg.sep_cta == 0 ? align16(cfg.sep_bytes) : 0u);
        const int pna = M.A1 - M.A0, pnp = M.P1 - M.P0;
        M.XS = reinterpret_cast<double*>(pb);
        pb += align16(24u * pna);
        M.YS = reinterpret_cast<LP*>(pb);
        pb += align16((uint32_t)sizeof(LP) * pnp);
        M.RFS = reinterpret_cast<V4*>(pb);
        pb += align16((uint32_t)sizeof(V4) * pnp);
        M.VS = reinterpret_cast<LP*>(pb);
        M.wt = cfg.wt != 0;
        if (cfg.prog) {
            pb += align16((uint32_t)sizeof(LP) * (M.T1 - M.T0));
            M.RHS = reinterpret_cast<V4*>(pb);
            pb += align16((uint32_t)sizeof(V4) * pnp);
            M.WLS = reinterpret_cast<LP*>(pb);
            pb += align16((uint32_t)sizeof(LP) * pna);
            const uint32_t o0 = __ldg(poff + q), o1 = __ldg(poff + q + 1);
            for (uint32_t o = 16u * threadIdx.x; o < o1 - o0; o += 16u * blockDim.x)
                cp_async16(pb + o, gp + PL.pprog + o0 + o);
            cp_async_wait_all();
            __syncthreads();
            M.part_prog_bind(pb);
        }
    }
    const int G = gridDim.x, b = blockIdx.x, r0 = threadIdx.x, ts = blockDim.x;
    const unsigned nb = gridDim.x + cfg.phantom;
    long long budget = kSpinBudget;
    auto part_atoms = [&](int q, int& a0, int& a1) {
        a0 = __ldg(&seg[q].atom);
        a1 = __ldg(&seg[q + 1].atom);
    };
    // constraints owned by this CTA: the interior pivots of its parts, and every G-th separator
    auto for_owned = [&](auto&& f) {
        for (int q = b; q < n_parts; q += G) {
            const int p1 = __ldg(&seg[q + 1].piv);
            for (int p = __ldg(&seg[q].piv) + r0; p < p1; p += ts) f(p);
        }
        for (int k = b + G * r0; k < nsep; k += G * ts) f(sep0 + k);
    };
    auto for_my_atoms = [&](auto&& f) {
        for (int q = b; q < n_parts; q += G) {
            int a0, a1;
            part_atoms(q, a0, a1);
            for (int a = a0 + r0; a < a1; a += ts) f(a);
        }
    };
    // the position updates, in the part program's order when there is one (atoms of equal
    // degree side by side, so a warp's float64 incidence loops run equally long)
    auto for_update_atoms = [&](auto&& f) {
        if (M.PH) {
            for (int k = r0; k < M.A1 - M.A0; k += ts) f(M.A0 + (int)M.PAORD[k]);
        } else {
            for_my_atoms(f);
        }
    };
    // ---- S1.  With part copies the inputs of the part's atoms are read once each, in
    //      order (x_old into X, x_unc into XS), and the part's constraints built from
    //      them; separators (atoms of two parts) read the inputs directly.
    if (M.XS) {
        for_my_atoms([&](int a) {
            M.s1_atom(a, true);
            M.s1_stage_unc(a);
        });
        if (b == 0 && r0 == 0) M.s1_dummy();
        __syncthreads();
        for_owned([&](int p) { M.s1_constraint(p, false, p < sep0); });
        __syncthreads();
        for_my_atoms([&](int a) { M.s1_atom_unc_staged(a); });
    } else {
        for_my_atoms([&](int a) { M.s1_atom(a, false); });
        if (b == 0 && r0 == 0) M.s1_dummy();
        for_owned([&](int p) { M.s1_constraint(p, false); });
        for_my_atoms([&](int a) { M.s1_atom_unc(a); });
    }
    bool alive = grid_sync(&sync->barrier, nb, budget);
    if (M.PH) {  // the part's reference rows and weights (written by this CTA in S1), the
                 // separators' reference rows (written by their owners)
        for (int k = r0; k < M.P1 - M.P0; k += ts) M.RHS[k] = *(M.RHOF + M.P0 + k);
        for (int a = r0; a < M.A1 - M.A0; a += ts) M.WLS[a] = *(M.WL + M.A0 + a);
        for (int k = r0; k < (int)M.PH->nsep; k += ts) M.SEPREF[k] = lds<true>(M.RHOF + M.PST[k]);
        __syncthreads();
    }
    if (b == cfg.sep_cta && sep_in_smem) {  // the separator program, reference rows, coefficients
        const uint32_t o0 = __ldg(poff + n_parts), o1 = __ldg(poff + n_parts + 1);
        for (uint32_t o = 16u * r0; o < o1 - o0; o += 16u * ts) cp_async16(SPROG + o, gp + PL.pprog + o0 + o);
        for (int k = r0; k < nsep; k += ts) SP[k] = lds<true>(M.RHOF + sep0 + k);
        for (int tl = r0; tl < D.n_sept; tl += ts) SC[tl] = M.sep_coef(tl);
        cp_async_wait_all();
        __syncthreads();
        M.sep_prog_bind(SPROG);
    }
    if (alive && A.has_start()) {
        for_update_atoms([&](int a) { M.update_atom(a); });
        alive = grid_sync(&sync->barrier, nb, budget);
    }
    int status = ILVES_MOL_MAX_ITER, iters = A.max_iter;
    for (int it = 0; alive; ++it) {
        const int slot = it & 3;
        // ---- violations of owned constraints, global vote
        bool conv = true, bad = false;
        for_owned([&](int p) { M.violation(p, conv, bad, !A.chord || it == 0); });
        const int nconv_block = __syncthreads_count(!conv);
        const int bad_block = __syncthreads_or(bad);
        if (r0 == 0) {
            if (nconv_block) atomicAdd(&sync->notconv[slot], nconv_block);
            if (bad_block) atomicOr(&sync->bad[slot], 1);
        }
        if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
        const int any_bad = __ldcg(&sync->bad[slot]), any_nc = __ldcg(&sync->notconv[slot]);
        if (b == 0 && r0 == 0) {  // free the slot used two iterations from now
            sync->notconv[(it + 2) & 3] = 0;
            sync->bad[(it + 2) & 3] = 0;
            sync->singular[(it + 2) & 3] = 0;
        }
        if (any_bad) {
            status = ILVES_MOL_NONFINITE;
            iters = it;
            break;
        }
        if (any_nc == 0) {
            status = ILVES_MOL_CONVERGED;
            iters = it;
            break;
        }
        if (it >= A.max_iter) break;
        const bool factor = !A.chord || it == 0;
        if (A.chord && it == 0) {  // ILVES-F: assemble A(x_old, x_old) (rows of owned constraints)
            for_owned([&](int p) { M.chord_rows(p); });
            if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
        }
        // ---- phase A: every part factorises its interior (and its rows/columns towards
        //      the separators) level by level; ILVES-F iterations only substitute forward.
        //      Meanwhile the separator CTA stages the separator rows (their factor's
        //      reciprocal pivots stay in SRF.w across ILVES-F iterations) and right-hand
        //      sides, which phase A does not change.
        if (b == cfg.sep_cta && sep_in_smem)
            for (int k = r0; k < nsep; k += ts) {
                if (factor) SRF[k] = lds<true>(M.RF + sep0 + k);
                SY[k] = lds<true>(M.Y + sep0 + k);
            }
        bool singular = false;
        for (int q = b; q < n_parts; q += G) {
            if (M.PH) {  // the part program in shared memory (one part per CTA)
                if (factor) {  // current rows of the separators the part's entries touch
                    for (int k = r0; k < (int)M.PH->nsep; k += ts) M.SEPRF[k] = lds<true>(M.RF + M.PST[k]);
                    __syncthreads();
                }
                const int nl = (int)M.PH->nlev;
                int e = (int)M.PLANE[r0];
                for (int l = 0; l < nl; ++l) {
                    const int p0 = M.PLP[l], np = M.PLP[l + 1] - p0, t0 = M.PLT[l], t1 = M.PLT[l + 1];
                    if (factor) M.part_level(t0, t1, np, r0, e, singular);
                    else M.part_forward_level(t0, t1, p0, np, r0, e);
                    __syncthreads();
                }
            } else {
                const int l0 = __ldg(&seg[q].lvl), l1 = __ldg(&seg[q + 1].lvl) - 1;
                for (int l = l0; l < l1; ++l) {
                    const int p0 = __ldg(M.lvl_piv + l), p1 = __ldg(M.lvl_piv + l + 1), np = p1 - p0;
                    const int t0 = __ldg(M.lvl_task + l), t1 = __ldg(M.lvl_task + l + 1);
                    if (factor)
                        for (int t = t0 + r0; t < t1; t += ts) M.task(t, t < t0 + np, singular);
                    else
                        for (int p = p0 + r0; p < p1; p += ts) M.forward(t0 + (p - p0), p);
                    __syncthreads();
                }
            }
            // this part's contributions to the separator block (Schur complement)
            if (M.PH) {
                for (int c = r0; c < (int)M.PH->ncontrib; c += ts) M.part_contrib(c, factor);
            } else {
                const int c1 = __ldg(M.cptr + q + 1);
                for (int c = __ldg(M.cptr + q) + r0; c < c1; c += ts) M.contrib(c, factor);
            }
        }
        if (__syncthreads_or(singular) && r0 == 0) atomicOr(&sync->singular[slot], 1);
        if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
        // ---- phase B: CTA 0 factorises the separator block (the Schur complement) and
        //      solves it forward and backward
        if (b == cfg.sep_cta && sep_in_smem) {
            // the parts' contributions (the separator rows and right-hand sides were staged
            // during phase A), then the solve in shared memory; publish the solution
            if (cfg.sep_ct) {
                const int n16 = (int)(4u * (uint32_t)sizeof(LP) * D.n_sept / 16u);
                for (int k = r0; k < n16; k += ts)
                    cp_async16(reinterpret_cast<uint8_t*>(CS) + 16 * k, reinterpret_cast<const uint8_t*>(M.CT) + 16 * k);
            }
            cp_async_wait_all();
            __syncthreads();
            for (int tl = r0; tl < D.n_sept; tl += ts)
                M.sep_stage_smem(tl, factor, cfg.sep_ct ? CS : M.CT, !cfg.sep_ct, SV, SY);
            __syncthreads();
            bool sing = false;
            const int nl = (int)reinterpret_cast<const SepProgHeader*>(SPROG)->nlev;
            for (int l = 0; l < nl; ++l) {
                const int p0 = M.SLP[l], p1 = M.SLP[l + 1], np = p1 - p0;
                const int t0 = M.SLT[l], t1 = M.SLT[l + 1];
                int g = 1;  // narrow level: g >= 4 lanes per task, one pass
                while (g < 32 && 2 * g * (t1 - t0) <= ts) g *= 2;
                if (factor && g >= 4) {
                    M.sep_level_groups(t0, t1, np, g, r0, ts, sing, SV, SRF, SY, SP, SC);
                } else if (factor)
                    for (int t = t0 + r0; t < t1; t += ts) M.sep_task_smem(t, t < t0 + np, sing, SV, SRF, SY, SP, SC);
                else
                    for (int p = p0 + r0; p < p1; p += ts) M.sep_forward_smem(t0 + (p - p0), p, SV, SRF, SY);
                __syncthreads();
            }
            if (__syncthreads_or(sing) && r0 == 0) atomicOr(&sync->singular[slot], 1);
            for (int l = nl - 1; l >= 0; --l) {
                const int p1 = M.SLP[l + 1];
                for (int p = M.SLP[l] + r0; p < p1; p += ts) M.sep_backward_smem(p, SV, SRF, SY);
                __syncthreads();
            }
            for (int k = r0; k < nsep; k += ts) M.Y[sep0 + k] = SY[k];
        } else if (b == cfg.sep_cta) {
            M.cohall = true;  // the separator block: every value may come from another CTA
            bool sing = false;
            const int l0 = __ldg(&seg[n_parts].lvl), l1 = __ldg(&seg[n_parts + 1].lvl) - 1;
            for (int l = l0; l < l1; ++l) {
                const int p0 = __ldg(M.lvl_piv + l), p1 = __ldg(M.lvl_piv + l + 1), np = p1 - p0;
                const int t0 = __ldg(M.lvl_task + l), t1 = __ldg(M.lvl_task + l + 1);
                if (factor)
                    for (int t = t0 + r0; t < t1; t += ts) M.task_sep(t, t < t0 + np, sing);
                else
                    for (int p = p0 + r0; p < p1; p += ts) M.forward_sep(t0 + (p - p0), p);
                __syncthreads();
            }
            if (__syncthreads_or(sing) && r0 == 0) atomicOr(&sync->singular[slot], 1);
            for (int l = l1 - 1; l >= l0; --l) {
                const int p1 = __ldg(M.lvl_piv + l + 1);
                for (int p = __ldg(M.lvl_piv + l) + r0; p < p1; p += ts) M.backward(p);
                __syncthreads();
            }
            M.cohall = false;
        }
        if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
        if (__ldcg(&sync->singular[slot])) {
            status = ILVES_MOL_SINGULAR_PIVOT;
            iters = it;
            break;
        }
        // ---- phase D: back substitution inside every part, multipliers, positions
        for (int q = b; q < n_parts; q += G) {
            if (M.PH) {
                for (int k = r0; k < (int)M.PH->nsep; k += ts) M.SEPY[k] = lds<true>(M.Y + M.PST[k]);
                __syncthreads();
                for (int l = (int)M.PH->nlev - 1; l >= 0; --l) {
                    const int p1 = M.PLP[l + 1];
                    for (int p = M.PLP[l] + r0; p < p1; p += ts) M.part_backward(p);
                    __syncthreads();
                }
                continue;
            }
            const int l0 = __ldg(&seg[q].lvl), l1 = __ldg(&seg[q + 1].lvl) - 1;
            for (int l = l1 - 1; l >= l0; --l) {
                const int p1 = __ldg(M.lvl_piv + l + 1);
                for (int p = __ldg(M.lvl_piv + l) + r0; p < p1; p += ts) M.backward(p);
                __syncthreads();
            }
        }
        for_owned([&](int p) { M.lambda_acc(p); });
        for_update_atoms([&](int a) { M.update_atom(a); });
        if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
    }
    if (!alive) {
        status = ILVES_MOL_WAIT_TIMEOUT;
        if (r0 == 0) atomicOr(&sync->timeout, 1);
    }
    for_my_atoms([&](int a) { M.out_atom(a); });
    if (A.lambda_out) for_owned([&](int p) { M.out_lambda(p); });
    if (b == 0 && r0 == 0) {
        if (A.iterations_out) A.iterations_out[D.mol_id] = iters;
        if (A.status_out) A.status_out[D.mol_id] = status;
    }
}

// ------------------------------------------------------------------------------------
// overlapping domains (supplement Sec. 3, the Overlapping Partitioning Method): one CTA
// per domain of a cooperative launch.  Each iteration every domain evaluates the violations
// of its constraints at the current positions, factorises A(x, x_old) restricted to them
// and solves it in shared memory -- a local approximation of z = A^-1 sigma -- and keeps
// the corrections of the constraints it owns; after a grid barrier the owners add them to
// lambda and move their atoms; a second barrier publishes the positions.  A quasi-Newton
// iteration on the exact constraint equations: it converges to the same root as ILVES-M.
// The workspace holds the molecule's positions (SoA; displacements x - x_unc as float-float
// pairs in the float-float mode), the owned corrections and lambda.
// ------------------------------------------------------------------------------------
template <class Mode>
__global__ void __launch_bounds__(kPartThreads, 3)
k_solve_opm(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob, uint8_t* work, PartSync* sync,
            SolveArgs A, uint32_t phantom, uint32_t staged) {
    using LP = typename Mode::LP;
    using V4 = typename Mode::V4;
    constexpr bool DF = Mode::df;  // float-float: displacements x - x_unc, float-float pairs
    extern __shared__ __align__(16) uint8_t dsm[];
    const MolDesc D = *desc;
    const uint8_t* mb = blob + D.blob_off;
    const uint32_t n_dom = reinterpret_cast<const OpmBlobHeader*>(mb)->n_dom;
    const uint32_t* dom_off = reinterpret_cast<const uint32_t*>(mb + sizeof(OpmBlobHeader));
    const int32_t* con_gid =
        reinterpret_cast<const int32_t*>(mb + align16((uint32_t)sizeof(OpmBlobHeader) + 4u * (n_dom + 1)));
    const int dm = blockIdx.x, r0 = threadIdx.x, ts = blockDim.x;
    const uint8_t* prog = mb + __ldg(dom_off + dm);  // the domain's program: in shared memory if staged
    if (staged) {
        const uint32_t nbytes = __ldg(dom_off + dm + 1) - __ldg(dom_off + dm);
        for (uint32_t o = 16u * r0; o < nbytes; o += 16u * ts) cp_async16(dsm + o, prog + o);
        cp_async_wait_all();
        __syncthreads();
        prog = dsm;
    }
    const DomProgHeader H = *reinterpret_cast<const DomProgHeader*>(prog);
    const DomProgLayout L = dom_prog_layout(H.na, H.na_own, H.nc, H.nt, H.nterm, H.nlev, H.n_inc);
    const uint8_t* dsmp = prog;
    const uint16_t* LPV = reinterpret_cast<const uint16_t*>(dsmp + L.lvl_piv);
    const uint16_t* LTK = reinterpret_cast<const uint16_t*>(dsmp + L.lvl_task);
    const uint32_t* LANE = reinterpret_cast<const uint32_t*>(dsmp + L.lane_term);
    const uint32_t* PV = reinterpret_cast<const uint32_t*>(dsmp + L.piv);
    const uint32_t* CON = reinterpret_cast<const uint32_t*>(dsmp + L.con);
    const uint32_t* CML = reinterpret_cast<const uint32_t*>(dsmp + L.con_ml);
    const int32_t* AML = reinterpret_cast<const int32_t*>(dsmp + L.atom_ml);
    const uint16_t* IP = reinterpret_cast<const uint16_t*>(dsmp + L.inc_ptr);
    const uint16_t* IV = reinterpret_cast<const uint16_t*>(dsmp + L.inc);
    const uint16_t* AORD = reinterpret_cast<const uint16_t*>(dsmp + L.aorder);
    const uint2* TK = reinterpret_cast<const uint2*>(dsmp + L.tasks);
    const uint32_t* TM = reinterpret_cast<const uint32_t*>(dsmp + L.terms);
    const int na = (int)H.na, no = (int)H.na_own, nc = (int)H.nc;
    const DomStateLayout S = dom_state_layout(H.na, H.na_own, H.nc, H.nt, (uint32_t)sizeof(LP), DF);
    uint8_t* st = staged ? dsm + L.bytes : dsm;
    double* X = reinterpret_cast<double*>(st + S.x);
    LP* WL = reinterpret_cast<LP*>(st + S.wl);
    double* W = reinterpret_cast<double*>(st + S.w);
    double* RHO = reinterpret_cast<double*>(st + S.rho);
    float* RHOL = reinterpret_cast<float*>(st + S.rho);  // float-float mode: low parts of rho (SoA)
    double* SK = reinterpret_cast<double*>(st + S.sk);   // float-float mode: x_unc,i - x_unc,j
    V4* RHOF = reinterpret_cast<V4*>(st + S.rhof);
    V4* RF = reinterpret_cast<V4*>(st + S.rf);
    double* D2 = reinterpret_cast<double*>(st + S.d2);
    LP* Y = reinterpret_cast<LP*>(st + S.y);
    LP* V = reinterpret_cast<LP*>(st + S.v);
    const int na_m = D.na, nc_m = D.nc;
    double* GX = reinterpret_cast<double*>(work + D.work_off);          // positions, SoA
    LP* GDL = reinterpret_cast<LP*>(work + D.work_off + 24 * (int64_t)na_m);  // owned corrections
    double* GLAM = reinterpret_cast<double*>(work + D.work_off + 24 * (int64_t)na_m + 8 * (int64_t)nc_m);
    auto gid = [&](int al) -> int64_t {
        return D.atom_base >= 0 ? (int64_t)D.atom_base + al : (int64_t)A.atom_gid[D.gid_off + al];
    };
    auto inv = [&](int p) -> LP { return reinterpret_cast<const LP*>(RF + p)[3]; };
    const unsigned nb = gridDim.x + phantom;
    long long budget = kSpinBudget;
    // ---- S1: x_old of the domain's atoms (staged in X), weights
    for (int k = r0; k < na; k += ts) {
        const int64_t g = gid(AML[k]);
        for (int c = 0; c < 3; ++c) X[c * na + k] = A.x_old[3 * g + c];
        const double w = A.inv_mass[g];
        WL[k] = to_lp<LP>(w);
        if (k < no) W[k] = DF ? as_bits(df_split(w)) : w;
    }
    if (r0 == 0) WL[na] = LP(0);
    __syncthreads();
    // rho, reference rows, d^2; starting multipliers of the owned constraints
    for (int p = r0; p < nc; p += ts) {
        const int i = (int)(CON[p] & 0xFFFFu), j = (int)(CON[p] >> 16);
        const double rx = X[i] - X[j], ry = X[na + i] - X[na + j], rz = X[2 * na + i] - X[2 * na + j];
        if constexpr (DF) {
            RHOL[p] = df_split(rx).lo;
            RHOL[nc + p] = df_split(ry).lo;
            RHOL[2 * nc + p] = df_split(rz).lo;
            const int64_t gi = gid(AML[i]), gj = gid(AML[j]);
            for (int c = 0; c < 3; ++c) SK[c * nc + p] = as_bits(df_split(A.x_unc[3 * gi + c] - A.x_unc[3 * gj + c]));
        } else {
            RHO[p] = rx;
            RHO[nc + p] = ry;
            RHO[2 * nc + p] = rz;
        }
        V4 v;
        v.x = to_lp<LP>(rx);
        v.y = to_lp<LP>(ry);
        v.z = to_lp<LP>(rz);
        v.w = WL[i] + WL[j];
        RHOF[p] = v;
        const uint32_t cm = CML[p];
        const int cl = (int)(cm & 0x7FFFFFFFu);
        const int32_t g = __ldg(con_gid + cl);
        const double dd = A.d[g];
        D2[p] = DF ? as_bits(df_split(dd * dd)) : dd * dd;
        if (cm >> 31) {
            float l0 = A.lambda0 ? A.lambda0[g] : 0.0f;
            if (A.start_diag) {
                const int64_t gi = gid(AML[i]), gj = gid(AML[j]);
                float u[3], o[3];
                for (int c = 0; c < 3; ++c) {
                    u[c] = narrow(A.x_unc[3 * gi + c]) - narrow(A.x_unc[3 * gj + c]);
                    o[c] = narrow(X[c * na + i]) - narrow(X[c * na + j]);
                }
                l0 = diag_start(u[0], u[1], u[2], o[0], o[1], o[2], narrow(dd), f32_of(WL[i]) + f32_of(WL[j]));
            }
            GDL[cl] = (LP)l0;
            GLAM[cl] = DF ? as_bits(dfloat{l0, 0.0f}) : widen(l0);
        }
    }
    __syncthreads();
    for (int k = r0; k < no; k += ts) {  // owned atoms start at x_unc (displacement 0)
        const int al = AML[k];
        const int64_t g = gid(al);
        for (int c = 0; c < 3; ++c) {
            const double v = DF ? 0.0 : A.x_unc[3 * g + c];
            X[c * na + k] = v;
            GX[c * (int64_t)na_m + al] = v;
        }
    }
    // x_a -= w_a sum_p s_p(a) 2 delta_p rho_p over the owned atom's constraints, with the
    // owners' corrections (own ones from Y)
    auto update_owned = [&](bool from_y) {
        for (int kk = r0; kk < no; kk += ts) {
            const int k = (int)AORD[kk];
            double x, y, z;
            if constexpr (DF) {
                dfloat ax{0.f, 0.f}, ay{0.f, 0.f}, az{0.f, 0.f};
                for (int e = IP[k]; e < IP[k + 1]; ++e) {
                    const uint32_t v = IV[e];
                    const int p = (int)(v >> 1);
                    const uint32_t cm = CML[p];
                    const float dl = (float)((from_y && (cm >> 31)) ? Y[p] : __ldcg(GDL + (cm & 0x7FFFFFFFu)));
                    const float c = (v & 1u) ? -(dl + dl) : (dl + dl);
                    const V4 hi = RHOF[p];
                    ax = df_add(ax, df_mul_f(dfloat{hi.x, RHOL[p]}, c));
                    ay = df_add(ay, df_mul_f(dfloat{hi.y, RHOL[nc + p]}, c));
                    az = df_add(az, df_mul_f(dfloat{hi.z, RHOL[2 * nc + p]}, c));
                }
                const dfloat w = as_df(W[k]);
                x = as_bits(df_sub(as_df(X[k]), df_mul(w, ax)));
                y = as_bits(df_sub(as_df(X[na + k]), df_mul(w, ay)));
                z = as_bits(df_sub(as_df(X[2 * na + k]), df_mul(w, az)));
            } else {
                double ax = 0.0, ay = 0.0, az = 0.0;
                for (int e = IP[k]; e < IP[k + 1]; ++e) {
                    const uint32_t v = IV[e];
                    const int p = (int)(v >> 1);
                    const uint32_t cm = CML[p];
                    const LP dl = (from_y && (cm >> 31)) ? Y[p] : __ldcg(GDL + (cm & 0x7FFFFFFFu));
                    const double c = to_hp((v & 1u) ? -(dl + dl) : (dl + dl));
                    ax = fma(c, RHO[p], ax);
                    ay = fma(c, RHO[nc + p], ay);
                    az = fma(c, RHO[2 * nc + p], az);
                }
                const double w = W[k];
                x = fma(-w, ax, X[k]);
                y = fma(-w, ay, X[na + k]);
                z = fma(-w, az, X[2 * na + k]);
            }
            const int al = AML[k];
            X[k] = x;
            X[na + k] = y;
            X[2 * na + k] = z;
            GX[al] = x;
            GX[(int64_t)na_m + al] = y;
            GX[2 * (int64_t)na_m + al] = z;
        }
    };
    bool alive = grid_sync(&sync->barrier, nb, budget);
    if (alive && A.has_start()) {  // x = x_unc - M^-1 G(x_old)^T lambda0
        update_owned(false);
        alive = grid_sync(&sync->barrier, nb, budget);
    }
    int status = ILVES_MOL_MAX_ITER, iters = A.max_iter;
    for (int it = 0; alive; ++it) {
        const int slot = it & 3;
        for (int k = no + r0; k < na; k += ts) {  // the halo's current positions
            const int al = AML[k];
            for (int c = 0; c < 3; ++c) X[c * na + k] = __ldcg(GX + c * (int64_t)na_m + al);
        }
        __syncthreads();
        // ---- violations of the domain's constraints (the owned ones vote), Jacobian rows
        const bool rows = !A.chord || it == 0;
        bool conv = true, bad = false;
        for (int p = r0; p < nc; p += ts) {
            const int i = (int)(CON[p] & 0xFFFFu), j = (int)(CON[p] >> 16);
            V4 v;
            if constexpr (DF) {  // r = s + (dx_i - dx_j) and |r|^2 - d^2 by error-free transformations
                const dfloat rx = df_add(as_df(SK[p]), df_sub(as_df(X[i]), as_df(X[j])));
                const dfloat ry = df_add(as_df(SK[nc + p]), df_sub(as_df(X[na + i]), as_df(X[na + j])));
                const dfloat rz = df_add(as_df(SK[2 * nc + p]), df_sub(as_df(X[2 * na + i]), as_df(X[2 * na + j])));
                const dfloat d2 = as_df(D2[p]);
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
                if (CML[p] >> 31) {
                    conv = conv && fabsf(sg) <= (float)A.tol * d2.hi;
                    bad = bad || nonfinite(sg);
                }
                Y[p] = (LP)sg;
                v.x = rx.hi;
                v.y = ry.hi;
                v.z = rz.hi;
            } else {
                const double rx = X[i] - X[j], ry = X[na + i] - X[na + j], rz = X[2 * na + i] - X[2 * na + j];
                const double d2 = D2[p];
                const double sg = fma(rx, rx, fma(ry, ry, fma(rz, rz, -d2)));
                if (CML[p] >> 31) {
                    conv = conv && abs_le(sg, A.tol * d2);
                    bad = bad || nonfinite(sg);
                }
                Y[p] = to_lp<LP>(sg);
                v.x = to_lp<LP>(rx);
                v.y = to_lp<LP>(ry);
                v.z = to_lp<LP>(rz);
            }
            v.w = LP(0);
            if (rows) RF[p] = v;
        }
        const int nconv = __syncthreads_count(!conv);
        const int anybad = __syncthreads_or(bad);
        if (r0 == 0) {
            if (nconv) atomicAdd(&sync->notconv[slot], nconv);
            if (anybad) atomicOr(&sync->bad[slot], 1);
        }
        // ---- the domain's Newton step (speculative: the vote is read after the barrier)
        bool singular = false;
        if (A.chord && it == 0) {  // ILVES-F: the reference rows, factorised once
            for (int p = r0; p < nc; p += ts) RF[p] = RHOF[p];
            __syncthreads();
        }
        int e = (int)LANE[r0];
        for (int l = 0; l < (int)H.nlev; ++l) {
            const int p0 = LPV[l], np = LPV[l + 1] - p0, t0 = LTK[l], t1 = LTK[l + 1];
            for (int t = t0 + r0; t < t1; t += ts) {
                const uint2 w = TK[t];
                const int n = (int)(w.y >> 24);
                const bool diag = t < t0 + np;
                if (!rows) {  // ILVES-F after its first iteration: forward substitution only
                    if (diag) {
                        LP yv = LP(0);
                        for (int k = e; k < e + n; ++k) {
                            const uint32_t tr = TM[k];
                            yv += V[DomTerm::l(tr)] * inv((int)DomTerm::m(tr)) * Y[DomTerm::m(tr)];
                        }
                        Y[p0 + (t - t0)] -= yv;
                    }
                    e += n;
                    continue;
                }
                const uint32_t rc = w.x & 0xFFFFu, cc = w.x >> 16, ac = w.y & 0xFFFFu;
                const V4 rr = RF[rc], pp = RHOF[cc];
                const LP wv = diag ? pp.w : (ac == 0xFFFFu ? LP(0) : WL[ac]);
                const LP cf = ((w.y >> 16) & 1u) ? LP(-4) * wv : LP(4) * wv;
                const LP a = cf * (rr.x * pp.x + rr.y * pp.y + rr.z * pp.z);
                LP sacc = a, yv = LP(0);
#pragma unroll 2
                for (int k = e; k < e + n; ++k) {
                    const uint32_t tr = TM[k];
                    const int m = (int)DomTerm::m(tr);
                    const LP li = V[DomTerm::l(tr)] * inv(m);
                    sacc -= li * V[DomTerm::u(tr)];
                    if (diag) yv += li * Y[m];
                }
                e += n;
                V[t] = sacc;
                if (diag) {
                    singular = singular || !(lp_abs(sacc) > Mode::pivot_rel * lp_abs(a));
                    reinterpret_cast<LP*>(RF + rc)[3] = lp_rcp(sacc);
                    Y[rc] -= yv;
                }
            }
            __syncthreads();
        }
        for (int l = (int)H.nlev - 1; l >= 0; --l) {  // backward substitution
            const int p1 = LPV[l + 1];
            for (int p = LPV[l] + r0; p < p1; p += ts) {
                const uint32_t pv = PV[p];
                const int us = (int)(pv & 0xFFFFu), nu = (int)(pv >> 16);
                LP dl = Y[p];
                for (int k = 0; k < nu; ++k) dl -= V[us + k] * Y[TK[us + k].x >> 16];
                Y[p] = dl * inv(p);
            }
            __syncthreads();
        }
        for (int p = r0; p < nc; p += ts)  // the owned corrections, for the other domains
            if (CML[p] >> 31) GDL[CML[p] & 0x7FFFFFFFu] = Y[p];
        if (__syncthreads_or(singular) && r0 == 0) atomicOr(&sync->singular[slot], 1);
        if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
        const int any_bad = __ldcg(&sync->bad[slot]), any_nc = __ldcg(&sync->notconv[slot]);
        const int any_sing = __ldcg(&sync->singular[slot]);
        if (dm == 0 && r0 == 0) {  // free the slot used two iterations from now
            sync->notconv[(it + 2) & 3] = 0;
            sync->bad[(it + 2) & 3] = 0;
            sync->singular[(it + 2) & 3] = 0;
        }
        if (any_bad) {
            status = ILVES_MOL_NONFINITE;
            iters = it;
            break;
        }
        if (any_nc == 0) {
            status = ILVES_MOL_CONVERGED;
            iters = it;
            break;
        }
        if (it >= A.max_iter) break;
        if (any_sing) {
            status = ILVES_MOL_SINGULAR_PIVOT;
            iters = it;
            break;
        }
        // ---- lambda += delta of the owned constraints; the owned atoms move
        for (int p = r0; p < nc; p += ts)
            if (CML[p] >> 31) {
                const int cl = (int)(CML[p] & 0x7FFFFFFFu);
                GLAM[cl] = DF ? as_bits(df_add_f(as_df(GLAM[cl]), (float)Y[p])) : GLAM[cl] + to_hp(Y[p]);
            }
        update_owned(true);
        if (!(alive = grid_sync(&sync->barrier, nb, budget))) break;
    }
    if (!alive) {
        status = ILVES_MOL_WAIT_TIMEOUT;
        if (r0 == 0) atomicOr(&sync->timeout, 1);
    }
    for (int k = r0; k < no; k += ts) {
        const int64_t g = gid(AML[k]);
        for (int c = 0; c < 3; ++c)
            A.x_out[3 * g + c] = DF ? A.x_unc[3 * g + c] + df_join(as_df(X[c * na + k])) : X[c * na + k];
    }
    if (A.lambda_out)
        for (int p = r0; p < nc; p += ts)
            if (CML[p] >> 31) {
                const int cl = (int)(CML[p] & 0x7FFFFFFFu);
                A.lambda_out[__ldg(con_gid + cl)] = DF ? df_join(as_df(GLAM[cl])) : GLAM[cl];
            }
    if (dm == 0 && r0 == 0) {
        if (A.iterations_out) A.iterations_out[D.mol_id] = iters;
        if (A.status_out) A.status_out[D.mol_id] = status;
    }
}

// ------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------
constexpr int kStaticSlotSmem = 128;  // bytes: the pool-ticket words of the slots of a CTA
static_assert(kStaticSlotSmem >= (int)(kMaxSlotsPerCta * sizeof(unsigned)), "ticket words");
static_assert(kStaticSlotSmem >= (int)(kNarrowSlotsPerCta * sizeof(unsigned)), "ticket words");

struct SmallSched {
    const int32_t* cta_slot_ptr;
    const int32_t* cta_nwide;  // per CTA: its first slots are wide (96-thread teams)
    const int32_t* slot_ptr;
    const int32_t* slot_mol;
    const int32_t* slot_off;
    const int32_t* pool_mol;  // the wide class's pool, then the narrow class's
    uint32_t* pool_ctr;       // {next ticket, slots done} of the wide pool, then of the narrow pool
    int32_t pool_n, n_slots;                // wide class
    int32_t pool_n_narrow, n_slots_narrow;  // narrow class
};

// One class's pool: the molecules, their number, the ticket counters and the class's slots.
struct SlotPool {
    const int32_t* mol;
    uint32_t* ctr;
    int32_t n, n_slots;
};

template <class Team>
__device__ __forceinline__ int pool_ticket(const SlotPool& P, const Team& tm, unsigned* box) {
    if (tm.rank() == 0) *box = atomicAdd(P.ctr, 1u);
    tm.sync();
    const unsigned t = *box;
    tm.sync();  // every thread has read the box before the next ticket is written
    return t < (unsigned)P.n ? __ldg(P.mol + t) : -1;
}

// One slot of a CTA, run by a team of Team::kSize threads: the slot owns a fixed slice of
// the CTA's shared-memory arena, solves its queue
// of molecules one after the other, then draws molecules from its class's pool (one
// atomic ticket each) until the pool is empty; teams never wait for each other.  Each
// molecule's program blob is staged into the slice with asynchronous 16-byte copies, and
// the next queued molecule's program and atom inputs are prefetched into L2 while the
// current one is solved.  The last team of the class to finish resets the class's pool
// counters for the next launch.
template <class Mode, class Team>
__device__ __forceinline__ void run_slot(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob,
                                         const SmallSched& S, const SlotPool& P, const SolveArgs& A,
                                         uint8_t* arena, unsigned* box, int slot) {
    const Team tm;
    const int lane = tm.rank();
    uint8_t* slice = arena + S.slot_off[slot];
    const int q1 = S.slot_ptr[slot + 1];
    int q = S.slot_ptr[slot];
    int mol = q < q1 ? S.slot_mol[q] : (P.n > 0 ? pool_ticket(P, tm, box) : -1);
    while (mol >= 0) {
        const MolDesc D = desc[mol];
        const ProgLayout PL = prog_layout<uint16_t>(D.na, D.nc, D.ntask, D.nterm, D.nlevel, D.n_seg);
        const uint4* src = reinterpret_cast<const uint4*>(blob + D.blob_off);
        uint4* dst = reinterpret_cast<uint4*>(slice);
        const int n16 = (int)(PL.staged >> 4);
        for (int k = lane; k < n16; k += Team::kSize) cp_async16(dst + k, src + k);  // all in flight
        if (q + 1 < q1) {  // the next queued molecule's program and atom inputs into L2 meanwhile
            const MolDesc Dn = desc[S.slot_mol[q + 1]];
            const uint32_t nb = prog_layout<uint16_t>(Dn.na, Dn.nc, Dn.ntask, Dn.nterm, Dn.nlevel, Dn.n_seg).bytes;
            const uint8_t* pb = blob + Dn.blob_off;
            constexpr uint32_t kStep = 128u * Team::kSize;
            for (uint32_t o = 128u * lane; o < nb; o += kStep) prefetch_l2(pb + o);
            if (Dn.atom_base >= 0) {
                const uint8_t* xo = reinterpret_cast<const uint8_t*>(A.x_old + 3 * (int64_t)Dn.atom_base);
                const uint8_t* xu = reinterpret_cast<const uint8_t*>(A.x_unc + 3 * (int64_t)Dn.atom_base);
                const uint8_t* wm = reinterpret_cast<const uint8_t*>(A.inv_mass + Dn.atom_base);
                for (uint32_t o = 128u * lane; o < 24u * (uint32_t)Dn.na; o += kStep) {
                    prefetch_l2(xo + o);
                    prefetch_l2(xu + o);
                }
                for (uint32_t o = 128u * lane; o < 8u * (uint32_t)Dn.na; o += kStep) prefetch_l2(wm + o);
            }
        }
        cp_async_wait_all();
        tm.sync();
        solve_molecule<Mode, uint16_t, Team>(tm, D, slice, slice + PL.staged, A, blob + D.blob_off);
        tm.sync();
        ++q;
        mol = q < q1 ? S.slot_mol[q] : (P.n > 0 ? pool_ticket(P, tm, box) : -1);
    }
    if (P.n > 0 && lane == 0) {
        __threadfence();  // this team's last ticket is ordered before its "done"
        const unsigned done = atomicAdd(P.ctr + 1, 1u);
        if (done == (unsigned)P.n_slots - 1u) {  // every team of the class has drawn its last ticket
            __threadfence();
            atomicExch(P.ctr, 0u);
            atomicExch(P.ctr + 1, 0u);
        }
    }
}

// Persistent batched kernel.  In CTA c the first 3 nw warps (nw = cta_nwide[c]) form the
// 96-thread teams of the wide slots, each following warp is the one-warp team of a narrow
// slot (molecules small enough that three of them fit the shared memory of one wide
// molecule); a CTA's narrow slots follow its wide ones.  The pool-ticket word of a team is
// that of its first warp.
static_assert(kSlotThreads == 3 * 32, "a wide slot's team is three warps");
template <class Mode>
__global__ void __launch_bounds__(kSlotCtaThreads, 1)
k_solve_small(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob, SmallSched S,
              SolveArgs A) {
    extern __shared__ __align__(16) uint8_t arena[];
    __shared__ __align__(16) unsigned ticket_box[kStaticSlotSmem / sizeof(unsigned)];
    const int s0 = S.cta_slot_ptr[blockIdx.x], s1 = S.cta_slot_ptr[blockIdx.x + 1];
    const int nw = S.cta_nwide[blockIdx.x];
    const int warp = (int)(threadIdx.x / 32);
    if (warp < 3 * nw) {
        const SlotPool P{S.pool_mol, S.pool_ctr, S.pool_n, S.n_slots};
        run_slot<Mode, SlotTeam>(desc, blob, S, P, A, arena, ticket_box + 3 * (warp / 3), s0 + warp / 3);
    } else if (s0 + nw + (warp - 3 * nw) < s1) {
        const SlotPool P{S.pool_mol + S.pool_n, S.pool_ctr + 2, S.pool_n_narrow, S.n_slots_narrow};
        run_slot<Mode, NarrowTeam>(desc, blob, S, P, A, arena, ticket_box + warp, s0 + nw + (warp - 3 * nw));
    }
}

// Large molecules: one CTA per molecule, program and state in global memory.
template <class Mode>
__global__ void __launch_bounds__(512, 1)
k_solve_large(const MolDesc* __restrict__ desc, const uint8_t* __restrict__ blob, uint8_t* work,
              SolveArgs A) {
    const BlockTeam tm;
    const MolDesc D = desc[blockIdx.x];
    solve_molecule<Mode, uint32_t, BlockTeam>(tm, D, blob + D.blob_off, work + D.work_off, A, blob + D.blob_off);
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
    f(T->d_sync);
    f(T->d_work);
    for (auto& s : T->sched) {
        f(s.cta_slot_ptr);
        f(s.cta_nwide);
        f(s.slot_ptr);
        f(s.slot_mol);
        f(s.slot_off);
        f(s.pool_mol);
        f(s.pool_ctr);
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
    T->d_sync = nullptr;
    T->d_work = nullptr;
    T->side_stream = T->ev_fork = T->ev_join = nullptr;
}

template <class Mode>
static const void* small_kernel() {
    return (const void*)k_solve_small<Mode>;
}

// The batched kernel's dynamic shared-memory limit belongs to the kernel (per device), not
// to a topology: it is raised to the largest arena any topology launches it with, so
// topologies with different arenas (CTAs per SM) can alternate on one device.
constexpr int kMaxAttrDevices = 64;
static std::mutex g_attr_mutex;
static int g_small_smem[kMaxAttrDevices][3] = {};
static cudaError_t ensure_small_smem(int dev, int mode, const void* fn, int arena) {
    if (dev < 0 || dev >= kMaxAttrDevices) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, arena);
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (g_small_smem[dev][mode] >= arena) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, arena);
    if (e == cudaSuccess) g_small_smem[dev][mode] = arena;
    return e;
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
    // the batched kernel's dynamic arena; its static shared memory (one pool-ticket word
    // per slot) comes off the per-block limit
    const int arena = std::min(smem_optin - kStaticSlotSmem, smem_sm / ctas_per_sm - 1024) & ~15;
    // molecules whose slice does not fit an arena take the CTA-per-molecule path
    for (auto& M : T->mols)
        if (!M.large && footprint(M, ILVES_PREC_FP64) > (uint32_t)arena) M.large = true;
    // descriptors, program blobs, atom ids
    std::vector<int32_t> order;
    for (int32_t m = 0; m < T->n_mol; ++m)
        if (!T->mols[m].large) order.push_back(m);
    T->n_small = (int32_t)order.size();
    for (int32_t m = 0; m < T->n_mol; ++m)
        if (T->mols[m].large && !T->mols[m].parted) order.push_back(m);
    T->n_large = (int32_t)order.size() - T->n_small;
    T->parted_desc.clear();
    for (int32_t m = 0; m < T->n_mol; ++m)
        if (T->mols[m].parted && !T->mols[m].opm) {
            T->parted_desc.push_back((int32_t)order.size());
            order.push_back(m);
        }
    T->opm_desc.clear();
    for (int32_t m = 0; m < T->n_mol; ++m)
        if (T->mols[m].opm) {
            T->opm_desc.push_back((int32_t)order.size());
            order.push_back(m);
        }
    std::vector<int32_t> desc_index(T->n_mol);
    std::vector<MolDesc> desc(T->n_mol);
    T->desc_mol = order;
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
        D.n_seg = M.n_seg;
        D.n_sept = M.n_sept;
        D.n_cent = M.n_cent;
        D.pprog_bytes = M.pprog_bytes;
        D.opm = M.opm;
        D.work_off = 0;
        if (M.opm) {  // overlapping domains: positions (SoA), owned corrections, lambda
            D.work_off = woff;
            woff += (24 * (int64_t)na + 16 * (int64_t)D.nc + 255) & ~int64_t(255);
        } else if (M.large) {  // state, then (partitioned) 4 contribution values per separator task
            D.work_off = woff;
            const int64_t st = std::max(state_layout(na, D.nc, M.ntask, 8, false).bytes,
                                        state_layout(na, D.nc, M.ntask, 4, true).bytes);
            woff += (st + 4 * 8 * (int64_t)M.n_sept + 255) & ~int64_t(255);
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
    if (!T->parted_desc.empty() || !T->opm_desc.empty()) {
        T->sync_bytes = (int64_t)(T->parted_desc.size() + T->opm_desc.size()) * (int64_t)sizeof(PartSync);
        if ((e = cudaMalloc((void**)&T->d_sync, T->sync_bytes)) != cudaSuccess) return to_status(e);
    }
    // persistent schedules, one per precision mode
    for (int mode = 0; mode < 3; ++mode) {
        // auto: the largest slot count per CTA whose slices fit the arena (searched downwards)
        int warps = o.warps_per_cta > 0 ? o.warps_per_cta : kMaxSlotsPerCta;
        warps = std::max(1, std::min(kMaxSlotsPerCta, warps));
        HostSchedule HS;
        build_batched_schedule(T, mode, n_sm * ctas_per_sm, warps, arena, HS);
        for (auto& km : HS.slot_mol) km = desc_index[km];
        for (auto& km : HS.pool_mol) km = desc_index[km];
        DeviceSchedule& DS = T->sched[mode];
        DS.n_cta = HS.n_cta;
        DS.warps = HS.warps;
        DS.arena = HS.arena;
        DS.n_slots = HS.n_slots_wide;
        DS.pool_n = HS.pool_wide;
        DS.n_slots_narrow = (int32_t)HS.slot_off.size() - HS.n_slots_wide;
        DS.pool_n_narrow = (int32_t)HS.pool_mol.size() - HS.pool_wide;
        DS.block_threads = HS.block_threads;
        DS.launch_cta = 0;
        DS.launch_smem = 16;
        for (int32_t c = 0; c < HS.n_cta; ++c) {
            const int32_t s0 = HS.cta_slot_ptr[c], s1 = HS.cta_slot_ptr[c + 1];
            if (s1 > s0) DS.launch_cta = c + 1;
            int32_t used = 0;
            for (int32_t sl = s0; sl < s1; ++sl) used = std::max(used, HS.slot_off[sl] + HS.slot_bytes[sl]);
            DS.launch_smem = std::max(DS.launch_smem, (used + 15) & ~15);
        }
        if (!HS.pool_mol.empty()) {
            if ((e = upload(&DS.pool_mol, HS.pool_mol)) != cudaSuccess) return to_status(e);
            if ((e = upload(&DS.pool_ctr, std::vector<uint32_t>(4, 0u))) != cudaSuccess) return to_status(e);
        }
        if ((e = upload(&DS.cta_slot_ptr, HS.cta_slot_ptr)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.cta_nwide, HS.cta_nwide)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.slot_ptr, HS.slot_ptr)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.slot_mol, HS.slot_mol)) != cudaSuccess) return to_status(e);
        if ((e = upload(&DS.slot_off, HS.slot_off)) != cudaSuccess) return to_status(e);
    }
    if (T->n_large > 0 || !T->parted_desc.empty() || !T->opm_desc.empty()) {
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

// Enqueues every kernel of one solve on `stream`: the CTA-per-molecule kernel and the
// cooperative launches of partitioned molecules on the topology's side stream (fork /
// join through events), the warp-per-molecule kernel and the copy of unconstrained atoms
// on `stream`.  `work` holds the large molecules' state, `sync` their barrier areas.
template <class Mode>
static ilves_status launch_all(ilves_topology* T, const SolveArgs& A, cudaStream_t stream, uint8_t* work,
                               uint8_t* sync) {
    cudaError_t e;
    int launches = 0;
    const DeviceSchedule& DS = T->sched[Mode::id];
    if ((e = ensure_small_smem(T->device, Mode::id, small_kernel<Mode>(), DS.arena)) != cudaSuccess)
        return to_status(e);
    const bool side_work = T->n_large > 0 || !T->parted_desc.empty() || !T->opm_desc.empty();
    if (side_work) {
        cudaStream_t side = (cudaStream_t)T->side_stream;
        if ((e = cudaEventRecord((cudaEvent_t)T->ev_fork, stream)) != cudaSuccess) return to_status(e);
        if ((e = cudaStreamWaitEvent(side, (cudaEvent_t)T->ev_fork, 0)) != cudaSuccess) return to_status(e);
        if (T->n_large > 0) {
            k_solve_large<Mode><<<T->n_large, T->large_threads, 0, side>>>(T->d_desc + T->n_small, T->d_blob, work, A);
            if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
            ++launches;
        }
        if (!T->parted_desc.empty() || !T->opm_desc.empty()) {
            if ((e = cudaMemsetAsync(sync, 0, T->sync_bytes, side)) != cudaSuccess) return to_status(e);
        }
        {  // overlapping domains: one cooperative launch per molecule
            for (size_t k = 0; k < T->opm_desc.size(); ++k) {
                const int32_t di = T->opm_desc[k];
                const MolHost& MH = T->mols[T->desc_mol[di]];
                // the programs staged in shared memory when every domain still fits the SMs
                // with them, else read from global memory (state in shared memory either way)
                // sizes: mixed [0] / [2], float64 [1] / [3], float-float [4] / [5]
                const int qs = Mode::df ? 4 : (sizeof(typename Mode::LP) == 8 ? 1 : 0);
                const int qn = Mode::df ? 5 : 2 + qs;
                const int per_sm = (MH.n_dom + T->n_sm - 1) / std::max(1, T->n_sm);
                uint32_t staged = (int64_t)per_sm * (MH.dom_smem[qs] + 1024) <= 233472 && MH.dom_smem[qs] <= 232448;
                const int smem = staged ? MH.dom_smem[qs] : MH.dom_smem[qn];
                if ((e = cudaFuncSetAttribute(k_solve_opm<Mode>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
                    cudaSuccess)
                    return to_status(e);
                const MolDesc* dptr = T->d_desc + di;
                PartSync* sp = reinterpret_cast<PartSync*>(sync) + T->parted_desc.size() + k;
                SolveArgs Aa = A;
                uint32_t ph = (uint32_t)T->wait_test;
                void* args[] = {(void*)&dptr, (void*)&T->d_blob, (void*)&work, (void*)&sp,
                                (void*)&Aa,   (void*)&ph,        (void*)&staged};
                if ((e = cudaLaunchCooperativeKernel((const void*)k_solve_opm<Mode>, dim3(MH.n_dom), dim3(kPartThreads),
                                                     args, (size_t)smem, side)) != cudaSuccess)
                    return to_status(e);
                ++launches;
            }
        }
        if (!T->parted_desc.empty()) {
            for (size_t k = 0; k < T->parted_desc.size(); ++k) {
                const int32_t di = T->parted_desc[k];
                const MolHost& MH = T->mols[T->desc_mol[di]];
                const int n_parts = MH.n_seg - 1;
                // shared memory: the separator block if it fits, then the parts' copies if
                // every part gets a CTA of its own at that size
                // (with a staged copy of the contributions if that fits too)
                uint32_t sep_b = 0, sep_ct = 0;
                if (MH.sprog_bytes > 0) {
                    const uint32_t with_ct = sep_smem_bytes<Mode>(MH.n_sep, MH.n_sept, MH.sprog_bytes, true);
                    const uint32_t without = sep_smem_bytes<Mode>(MH.n_sep, MH.n_sept, MH.sprog_bytes, false);
                    if (with_ct <= kPartedSmemMax) {
                        sep_b = with_ct;
                        sep_ct = 1;
                    } else if (without <= kPartedSmemMax) {
                        sep_b = without;
                    }
                }
                const uint32_t need_part = part_smem_bytes<Mode>(MH.part_na, MH.part_np, MH.part_nt);
                // part programs in shared memory: 256-thread CTAs (their terms are laid out
                // thread by thread for kPartThreads threads)
                const uint32_t pp = MH.pprog_max > 0 && T->parted_threads == kPartThreads ? 1u : 0u;
                const uint32_t need_pp =
                    pp ? part_prog_smem_bytes<Mode>(MH.part_na, MH.part_np, MH.part_nt, MH.pprog_max) : 0u;
                if ((e = cudaFuncSetAttribute(k_solve_parted<Mode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)kPartedSmemMax)) != cudaSuccess)
                    return to_status(e);
                // configurations, best first: separator CTA of its own + part copies and
                // programs; the same without programs; CTA 0 with the separator block and the
                // part copies (with, then without programs); CTA 0 with the separator block only
                constexpr int kCands = 5;
                // the parts' values go through to global memory only if the separator phase
                // reads interior pivots' values (terms beyond the two contribution slots)
                const uint32_t wt = MH.sprog_bytes == 0 || MH.sep_interior > 0 ? 1u : 0u;
                const uint32_t ph = (uint32_t)T->wait_test;
                const PartedSmem cands[kCands] = {{sep_b, need_pp, n_parts, 1u, sep_ct, wt, ph},
                                                  {sep_b, need_part, n_parts, 0u, sep_ct, wt, ph},
                                                  {sep_b, need_pp, 0, 1u, sep_ct, wt, ph},
                                                  {sep_b, need_part, 0, 0u, sep_ct, wt, ph},
                                                  {sep_b, 0u, 0, 0u, sep_ct, wt, ph}};
                PartedSmem cfg = cands[kCands - 1];
                size_t dyn = sep_b;
                int max_grid = 1;
                for (const PartedSmem& c : cands) {
                    if (c.prog && !pp) continue;
                    const size_t d = c.sep_cta == 0 ? align16(c.sep_bytes) + c.part_bytes
                                                     : std::max<size_t>(c.sep_bytes, c.part_bytes);
                    if (d > kPartedSmemMax) continue;
                    int per_sm = 0;
                    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_parted<Mode>,
                                                                           T->parted_threads, d)) != cudaSuccess)
                        return to_status(e);
                    const int mg = std::max(1, per_sm * T->n_sm);
                    const int needed = c.sep_cta > 0 ? n_parts + 1 : (c.part_bytes > 0 ? n_parts : 1);
                    if (mg >= needed || &c == &cands[kCands - 1]) {
                        cfg = c;
                        dyn = d;
                        max_grid = mg;
                        break;
                    }
                }
                const MolDesc* dptr = T->d_desc + di;
                PartSync* sp = reinterpret_cast<PartSync*>(sync) + k;
                SolveArgs Aa = A;
                void* args[] = {(void*)&dptr, (void*)&T->d_blob, (void*)&work, (void*)&sp, (void*)&Aa, (void*)&cfg};
                const dim3 grid(cfg.sep_cta > 0 ? n_parts + 1 : std::min(n_parts, max_grid)), block(T->parted_threads);
                if ((e = cudaLaunchCooperativeKernel((const void*)k_solve_parted<Mode>, grid, block, args, dyn, side)) !=
                    cudaSuccess)
                    return to_status(e);
                ++launches;
            }
        }
        if ((e = cudaEventRecord((cudaEvent_t)T->ev_join, side)) != cudaSuccess) return to_status(e);
    }
    if (T->n_small > 0 && DS.launch_cta > 0) {
        SmallSched S{DS.cta_slot_ptr, DS.cta_nwide, DS.slot_ptr,     DS.slot_mol,       DS.slot_off,
                     DS.pool_mol,     DS.pool_ctr,  DS.pool_n,       DS.n_slots,        DS.pool_n_narrow,
                     DS.n_slots_narrow};
        k_solve_small<Mode><<<DS.launch_cta, DS.block_threads, DS.launch_smem, stream>>>(T->d_desc, T->d_blob, S, A);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
    }
    const int nf = (int)T->free_atoms.size();
    if (nf > 0 && A.x_out != A.x_unc) {
        k_copy_free<<<(nf + 255) / 256, 256, 0, stream>>>(T->d_free_atoms, nf, A.x_unc, A.x_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
        ++launches;
    }
    if (side_work) {
        if ((e = cudaStreamWaitEvent(stream, (cudaEvent_t)T->ev_join, 0)) != cudaSuccess) return to_status(e);
    }
    T->last_launches = launches;
    return ILVES_OK;
}

template <class Mode>
static ilves_status launch_mode(ilves_topology* T, const SolveArgs& A, cudaStream_t stream) {
    return launch_all<Mode>(T, A, stream, T->d_work, T->d_sync);
}

// ------------------------------------------------------------------------------------
// Allocation-free variant (see ilves_solve_static_scratch in ilves.h).  The state of
// molecules solved by a CTA or a cooperative group of CTAs (large and partitioned
// molecules, with the partitioned molecules' contribution slots) and the partitioned
// molecules' grid-barrier areas live in this file-scope device array instead of the
// topology's workspace; the solve clears the barrier areas with a memset on the side
// stream.  Host code must not pass the symbol itself to a kernel (in host code it names a
// host-side stand-in); its device address is looked up on every call, so a device reset
// between calls cannot leave a stale address behind.
// ------------------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.
static ilves_status static_scratch_address(uint8_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return ILVES_ERR_CUDA;
    *out = reinterpret_cast<uint8_t*>(p);
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
    o->partition_min_constraints = 0;
    o->part_constraints = 0;
    o->wait_test = 0;
    o->overlap = 0;
    o->narrow_atoms = 0;
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
        o.warps_per_cta > 16 || o.ctas_per_sm < 0 || o.ctas_per_sm > 4 || o.wait_test < 0 || o.wait_test > 64 ||
        o.overlap < 0 || o.overlap > 16 || o.narrow_atoms < -1 || o.narrow_atoms > 255)
        return ILVES_ERR_INVALID_ARG;
    ilves_topology* T = new ilves_topology();
    T->wait_test = o.wait_test;
    T->opts = o;
    T->tuning.chosen = o;
    // the planner sizes partitioned molecules for the device's SM count (all parts of a
    // cooperative launch must be resident at once); a host-only plan assumes 152 SMs
    if (o.device != -2) {
        int dev = o.device;
        if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = -1;
        int n_sm = 0;
        if (dev >= 0 && cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            T->n_sm = n_sm;
    }
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
    A.chord = (precision & ILVES_CHORD) ? 1 : 0;
    A.start_diag = (precision & ILVES_START_DIAG) ? 1 : 0;
    if (A.start_diag && lambda0) return ILVES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    T->last_launches = 0;
    switch (precision & ~(ILVES_CHORD | ILVES_START_DIAG)) {
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
    const int32_t prec_mode = precision & ~(ILVES_CHORD | ILVES_START_DIAG);
    if ((precision & ILVES_START_DIAG) && lambda0) return ILVES_ERR_INVALID_ARG;
    if (prec_mode < ILVES_PREC_FP64 || prec_mode > ILVES_PREC_MIXED_DF) return ILVES_ERR_INVALID_ARG;
    const uint64_t work_aligned = ((uint64_t)T->work_bytes + 255) & ~uint64_t(255);
    if (work_aligned + (uint64_t)T->sync_bytes > (uint64_t)kStaticScratchBytes) return ILVES_ERR_TOO_LARGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return ILVES_ERR_CUDA;
    if (dev != T->device) return ILVES_ERR_INVALID_ARG;
    uint8_t* scratch = nullptr;
    ilves_status st = static_scratch_address(&scratch);
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
    A.chord = (precision & ILVES_CHORD) ? 1 : 0;
    A.start_diag = (precision & ILVES_START_DIAG) ? 1 : 0;
    cudaStream_t s = (cudaStream_t)stream;
    T->last_launches = 0;
    uint8_t* sync = scratch + work_aligned;
    switch (prec_mode) {
        case ILVES_PREC_FP64: return launch_all<ModeFP64>(T, A, s, scratch, sync);
        case ILVES_PREC_MIXED: return launch_all<ModeMixed>(T, A, s, scratch, sync);
        default: return launch_all<ModeMixedDF>(T, A, s, scratch, sync);
    }
}

// ------------------------------------------------------------------------------------
// autotuning: candidate set-up options, each timed on the caller's inputs
// ------------------------------------------------------------------------------------
namespace {
struct TuneBuffers {
    double* x = nullptr;
    double* lam = nullptr;
    int32_t* it = nullptr;
    int32_t* st = nullptr;
    ~TuneBuffers() {
        cudaFree(x);
        cudaFree(lam);
        cudaFree(it);
        cudaFree(st);
    }
};

// Mean milliseconds of one ilves_solve over `reps` (after one untimed solve); < 0 if a solve
// failed or some molecule did not converge.
float time_solves(ilves_topology* T, const double* x_old, const double* x_unc, const double* inv_mass,
                  const double* d, double tol, int32_t precision, int32_t reps, cudaStream_t s, TuneBuffers& B,
                  std::vector<int32_t>& status_host) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.f;
    float ms = -1.f;
    const int32_t max_iter = (precision & ILVES_CHORD) ? 60 : 25;
    auto one = [&]() {
        return ilves_solve(T, x_old, x_unc, inv_mass, d, tol, max_iter, precision, nullptr, B.x, B.lam, B.it, B.st, s);
    };
    bool ok = one() == ILVES_OK && cudaStreamSynchronize(s) == cudaSuccess;
    if (ok) {
        cudaEventRecord(e0, s);
        for (int32_t r = 0; r < reps && ok; ++r) ok = one() == ILVES_OK;
        cudaEventRecord(e1, s);
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok) ms /= (float)reps;
    }
    status_host.assign(T->n_mol, 0);
    if (ok && T->n_mol > 0)
        ok = cudaMemcpy(status_host.data(), B.st, sizeof(int32_t) * T->n_mol, cudaMemcpyDeviceToHost) == cudaSuccess;
    for (int32_t v : status_host) ok = ok && v == ILVES_MOL_CONVERGED;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? ms : -1.f;
}

bool same_opts(const ilves_setup_opts& a, const ilves_setup_opts& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }
}  // namespace

extern "C" ilves_status ilves_autotune(ilves_topology* T, const double* x_old, const double* x_unc,
                                       const double* inv_mass, const double* d, double tol, int32_t precision,
                                       int32_t reps, void* stream, ilves_tuning* out) {
    if (!T || !T->on_device || reps < 1) return ILVES_ERR_INVALID_ARG;
    const int32_t mode = precision & ~(ILVES_CHORD | ILVES_START_DIAG);
    if (mode < ILVES_PREC_FP64 || mode > ILVES_PREC_MIXED_DF) return ILVES_ERR_INVALID_ARG;
    if (T->n_atoms > 0 && (!x_old || !x_unc || !inv_mass)) return ILVES_ERR_INVALID_ARG;
    if (T->n_c > 0 && !d) return ILVES_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != T->device) return ILVES_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    TuneBuffers buf;
    cudaError_t e;
    if (T->n_atoms > 0 && (e = cudaMalloc((void**)&buf.x, sizeof(double) * 3 * (size_t)T->n_atoms)) != cudaSuccess)
        return to_status(e);
    if (T->n_c > 0 && (e = cudaMalloc((void**)&buf.lam, sizeof(double) * (size_t)T->n_c)) != cudaSuccess)
        return to_status(e);
    if (T->n_mol > 0) {
        if ((e = cudaMalloc((void**)&buf.it, sizeof(int32_t) * T->n_mol)) != cudaSuccess) return to_status(e);
        if ((e = cudaMalloc((void**)&buf.st, sizeof(int32_t) * T->n_mol)) != cudaSuccess) return to_status(e);
    }
    std::vector<int32_t> stat;
    const ilves_setup_opts base = T->opts;
    const float before = time_solves(T, x_old, x_unc, inv_mass, d, tol, precision, reps, s, buf, stat);
    if (before < 0.f) return ILVES_ERR_CUDA;
    // candidates: one knob at a time away from the current options
    bool has_small = T->n_small > 0, has_parted = false;
    for (const auto& M : T->mols) has_parted = has_parted || M.parted;
    std::vector<ilves_setup_opts> cands;
    auto add = [&](ilves_setup_opts c) {
        for (const auto& x : cands)
            if (same_opts(x, c)) return;
        if (!same_opts(c, base)) cands.push_back(c);
    };
    if (has_small) {
        for (int32_t w : {8, 7, 6}) {
            ilves_setup_opts c = base;
            c.warps_per_cta = w;
            add(c);
        }
        {
            ilves_setup_opts c = base;
            c.ctas_per_sm = base.ctas_per_sm == 2 ? 1 : 2;
            add(c);
        }
        for (int32_t slack : {-1, 1, 3}) {
            ilves_setup_opts c = base;
            c.ordering = slack < 0 ? 0 : 2;
            c.degree_slack = slack < 0 ? 2 : slack;
            add(c);
        }
        for (int32_t na : {-1, 50, 60, 70, 100}) {  // the one-warp class: none, or up to na atoms
            ilves_setup_opts c = base;
            c.narrow_atoms = na;
            add(c);
        }
    }
    if (has_parted) {
        for (int32_t ov : {0, 2, 3, 4, 6}) {
            ilves_setup_opts c = base;
            c.overlap = ov;
            add(c);
        }
    }
    float best = before;
    ilves_topology* winner = nullptr;
    ilves_setup_opts best_opts = base;
    for (const ilves_setup_opts& c : cands) {
        ilves_topology* C = new ilves_topology();
        C->n_sm = T->n_sm;
        C->wait_test = c.wait_test;
        C->opts = c;
        ilves_status st = plan_topology(C, T->n_atoms, T->n_c, T->con_i.data(), T->con_j.data(), c);
        if (st == ILVES_OK) st = upload_topology(C, c);
        float ms = -1.f;
        if (st == ILVES_OK) ms = time_solves(C, x_old, x_unc, inv_mass, d, tol, precision, reps, s, buf, stat);
        if (st == ILVES_OK && ms >= 0.f && ms < best) {
            if (winner) ilves_destroy_topology(winner);
            winner = C;
            best = ms;
            best_opts = c;
        } else {
            ilves_destroy_topology(C);
        }
    }
    if (winner) {  // the topology takes the winner's plan; the old plan goes with the winner object
        std::swap(*T, *winner);
        ilves_destroy_topology(winner);
    }
    T->opts = best_opts;
    T->tuning.chosen = best_opts;
    T->tuning.candidates = (int32_t)cands.size() + 1;
    T->tuning.best_ms = best;
    T->tuning.before_ms = before;
    if (out) *out = T->tuning;
    return ILVES_OK;
}

extern "C" ilves_status ilves_topology_tuning(const ilves_topology* T, ilves_tuning* out) {
    if (!T || !out) return ILVES_ERR_INVALID_ARG;
    *out = T->tuning;
    return ILVES_OK;
}

extern "C" int64_t ilves_static_scratch_bytes(void) { return (int64_t)kStaticScratchBytes; }

extern "C" int64_t ilves_topology_device_bytes(const ilves_topology* T) {
    if (!T || !T->on_device) return 0;
    int64_t b = T->blob_bytes + (int64_t)T->n_mol * (int64_t)sizeof(MolDesc) + T->work_bytes + T->sync_bytes;
    b += 4 * (int64_t)T->n_atoms;                        // atom ids
    b += 4 * (int64_t)T->free_atoms.size();
    b += (int64_t)T->n_c * (4 + 4 + 16 + 16 + 32);      // atoms, neighbour table, warm-start workspace
    b += 4 * (int64_t)T->n_atoms;                        // warm-start atom weights
    for (const auto& sc : T->sched) b += 4 * (int64_t)(2 * sc.n_cta + 2 * T->n_small + 64);
    return b;
}

extern "C" int64_t ilves_topology_workspace_bytes(const ilves_topology* T) {
    return T ? ((T->work_bytes + 255) & ~int64_t(255)) + T->sync_bytes : 0;
}

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

extern "C" ilves_status ilves_topology_export_domains(const ilves_topology* T, int32_t mol, int32_t* n_dom,
                                                      int32_t* atom_bounds, int32_t* con_ptr, int32_t* con_gid,
                                                      int32_t* owned) {
    if (!T || mol < 0 || mol >= T->n_mol) return ILVES_ERR_INVALID_ARG;
    program_export_domains(T, mol, n_dom, atom_bounds, con_ptr, con_gid, owned);
    return ILVES_OK;
}

extern "C" ilves_status ilves_topology_export_molecule(const ilves_topology* T, int32_t mol, int32_t* pos_gid,
                                                       int32_t* level, int32_t* up_ptr, int32_t* up_idx) {
    if (!T || mol < 0 || mol >= T->n_mol || T->mols[mol].opm) return ILVES_ERR_INVALID_ARG;
    program_export(T, mol, pos_gid, level, up_ptr, up_idx);
    return ILVES_OK;
}

extern "C" ilves_status ilves_topology_export_layout(const ilves_topology* T, int32_t mol, int32_t* atom_gid,
                                                     int32_t* n_parts, int32_t* part_levels,
                                                     int32_t* part_prog_bytes, int32_t* sep_summary) {
    if (!T || mol < 0 || mol >= T->n_mol) return ILVES_ERR_INVALID_ARG;
    program_export_layout(T, mol, atom_gid, n_parts, part_levels, part_prog_bytes, sep_summary);
    return ILVES_OK;
}

extern "C" ilves_status ilves_topology_schedule(const ilves_topology* T, int32_t precision, int32_t n_cta,
                                                int32_t arena_bytes, int32_t* n_slots, int32_t* pool_n,
                                                int32_t* slot_cta, int32_t* slot_bytes, int32_t* slot_queue,
                                                int32_t* slot_team, int32_t* mol_slot, int32_t* mol_bytes,
                                                int32_t* mol_team, int32_t* class_info) {
    if (!T || precision < 0 || precision > 2 || n_cta < 1 || arena_bytes < 1) return ILVES_ERR_INVALID_ARG;
    HostSchedule HS;
    build_batched_schedule(const_cast<ilves_topology*>(T), precision, n_cta, kMaxSlotsPerCta, arena_bytes, HS);
    const int32_t ns = (int32_t)HS.slot_off.size();
    if (n_slots) *n_slots = ns;
    if (pool_n) *pool_n = (int32_t)HS.pool_mol.size();
    for (int32_t c = 0; c + 1 < (int32_t)HS.cta_slot_ptr.size(); ++c)
        for (int32_t s = HS.cta_slot_ptr[c]; s < HS.cta_slot_ptr[c + 1]; ++s) {
            if (slot_cta) slot_cta[s] = c;
            if (slot_bytes) slot_bytes[s] = HS.slot_bytes[s];
            if (slot_queue) slot_queue[s] = HS.slot_ptr[s + 1] - HS.slot_ptr[s];
            if (slot_team) slot_team[s] = HS.slot_team[s];
        }
    if (class_info) {
        class_info[0] = HS.n_slots_wide;
        class_info[1] = HS.pool_wide;
        class_info[2] = HS.block_threads;
        class_info[3] = HS.warps;
    }
    if (mol_slot || mol_bytes || mol_team) {
        for (int32_t m = 0; m < T->n_mol; ++m) {
            const bool warp = !T->mols[m].large;
            if (mol_slot) mol_slot[m] = warp ? -1 : -2;
            if (mol_bytes) mol_bytes[m] = warp ? (int32_t)footprint(T->mols[m], precision) : 0;
            if (mol_team) mol_team[m] = warp ? T->mols[m].team : 0;
        }
        if (mol_slot)
            for (int32_t s = 0; s < ns; ++s)
                for (int32_t q = HS.slot_ptr[s]; q < HS.slot_ptr[s + 1]; ++q) mol_slot[HS.slot_mol[q]] = s;
    }
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
