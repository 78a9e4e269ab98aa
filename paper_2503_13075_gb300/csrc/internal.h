// internal.h -- data layouts shared by the host planner (topology.cpp) and the
// CUDA kernels (solve.cu).  Not part of the public ABI.
//
// Every molecule is described by a "program": a compact, 16-byte aligned blob of
// 16-bit indices that a team of threads (one warp, or one CTA for large molecules)
// copies next to its numerical state and then interprets once per Newton iteration.
//
// Constraint numbering inside a molecule is the ELIMINATION POSITION p (0..nc-1):
// pivots are sorted by level, so the pivots of one level are contiguous.
//
// LU form: A = L U with L unit lower triangular and U upper triangular (diagonal
// d_j).  L is stored unscaled, Lt[q,j] = L[q,j] d_j, together with inv_j = 1 / d_j,
// so that every entry is computed by the same division-free expression:
//   DIAG j        d_j     = a_jj - sum_m Lt[j,m] inv_m U[m,j];   inv_j = 1 / d_j
//                 y_j     = sigma_j - sum_m Lt[j,m] inv_m y_m     (forward solve, fused)
//   U (j,q)       U[j,q]  = a_jq - sum_m Lt[j,m] inv_m U[m,q]    for q in N+(j)
//   L (q,j)       Lt[q,j] = a_qj - sum_m Lt[q,m] inv_m U[m,j]    for q in N+(j)
// where N+(j) are the later neighbours of j in the filled graph and m runs over
// earlier pivots adjacent to both row and column.  Task t writes value slot t.
// Within a level the DIAG tasks come first, then for each pivot its U row and its
// L column.  The backward solve is delta_j = inv_j (y_j - sum_{q in N+(j)} U[j,q] delta_q).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define ILVES_HD __host__ __device__ __forceinline__
#else
#define ILVES_HD inline
#endif

namespace ilves {

constexpr uint32_t kNoAtom32 = 0xFFFFFFFFu;

// Program words.  IdxT is uint16_t for molecules run by one warp (compact, staged in
// shared memory) and uint32_t for large molecules run by a whole CTA.
//   Task (large molecules): row, col of the target entry; atomsign = (shared atom << 1) |
//         (sign product < 0), the dummy atom for fill entries, unused for DIAG tasks;
//         tstart = first term.  Task t's terms are [tstart_t, tstart_{t+1}); a sentinel
//         task ends the list.
//   Task word (warp molecules): 32 bits, see TaskWord; no term pointer: in every level
//         thread r of the molecule's team (kSlotThreads threads) owns tasks t0 + r,
//         t0 + r + kSlotThreads, ..., and the terms are stored thread by thread (thread
//         r's terms of level 0, then of level 1, ...), starting at lane_term[r]; a thread
//         walks its terms with a running offset.
//   Term: l = slot of Lt[row, m], u = slot of U[m, col], m = the earlier pivot.
//   Piv:  diag = first slot of the pivot's U row (its L column follows), nup = |N+(pivot)|.
//   ConA: local atom ids (i, j) of the constraint at position p.
// inc[e] = p << 1 | (atom is the second atom of constraint p)
template <class IdxT> struct Task { IdxT row, col, atomsign, tstart; };
template <class IdxT> struct ConA { IdxT i, j; };
template <class IdxT> struct Piv { IdxT diag, nup; };

// Compact task word: row (8) | col (8) << 8 | shared atom (9) << 16 | negative sign
// product (1) << 25 | number of terms (6) << 26.
struct TaskWord {
    static constexpr uint32_t kMaxTerms = 63, kMaxAtom = 511;
    static ILVES_HD uint32_t row(uint32_t w) { return w & 0xFFu; }
    static ILVES_HD uint32_t col(uint32_t w) { return (w >> 8) & 0xFFu; }
    static ILVES_HD uint32_t atom(uint32_t w) { return (w >> 16) & 0x1FFu; }
    static ILVES_HD uint32_t neg(uint32_t w) { return (w >> 25) & 1u; }
    static ILVES_HD uint32_t nterm(uint32_t w) { return w >> 26; }
    static ILVES_HD uint32_t make(uint32_t row, uint32_t col, uint32_t atom, uint32_t neg, uint32_t nterm) {
        return row | (col << 8) | (atom << 16) | (neg << 25) | (nterm << 26);
    }
};

// Term words.  Warp-sized molecules (fewer than 256 constraints and 4096 slots) pack a
// term in 32 bits: l (12) | u (12) << 12 | m (8) << 24.  Large molecules use 4 x 32 bits.
struct TermWide { uint32_t l, u, m, pad; };
template <class IdxT> struct TermOf;
template <> struct TermOf<uint16_t> {
    using T = uint32_t;
    using TaskT = uint32_t;
    static ILVES_HD uint32_t l(T t) { return t & 0xFFFu; }
    static ILVES_HD uint32_t u(T t) { return (t >> 12) & 0xFFFu; }
    static ILVES_HD uint32_t m(T t) { return t >> 24; }
    static ILVES_HD T make(uint32_t l, uint32_t u, uint32_t m) { return l | (u << 12) | (m << 24); }
};
template <> struct TermOf<uint32_t> {
    using T = TermWide;
    using TaskT = Task<uint32_t>;
    static ILVES_HD uint32_t l(T t) { return t.l; }
    static ILVES_HD uint32_t u(T t) { return t.u; }
    static ILVES_HD uint32_t m(T t) { return t.m; }
    static ILVES_HD T make(uint32_t l, uint32_t u, uint32_t m) { return TermWide{l, u, m, 0u}; }
};
constexpr uint32_t kCompactMaxConstraints = 256, kCompactMaxSlots = 4096, kCompactMaxTerms = 65000;
// Threads of the team that solves one molecule of the batched kernel (whole warps; three
// warps cut the passes of wide levels at no cost in residency, which shared memory
// limits to about eight molecules per SM), the batched kernel's CTA size bound and its
// molecule slots per CTA.  Measured on the 4096-tree batch (mixed, kernel only): 32
// threads 224 us, 64 195 us, 96 185 us, 128 206 us.
#ifndef ILVES_SLOT_THREADS
#define ILVES_SLOT_THREADS 96
#endif
constexpr int kSlotThreads = ILVES_SLOT_THREADS;
constexpr int kSlotCtaThreads = 768;
constexpr int kMaxSlotsPerCta = kSlotCtaThreads / kSlotThreads;
// Narrow class: molecules of at most narrow_atoms atoms get one-warp teams, up to
// kNarrowSlotsPerCta per CTA beside its 96-thread teams.  Their slices are small, so an
// SM's shared memory holds about three times as many of them: batches of 20-50 and 50-100
// atoms (mixed) ran 1.54x and 1.28x faster that way than on 96-thread teams; on batches of
// mixed sizes (20-200 atoms) the gain depends on the precision mode, so the automatic
// choice keeps them on 96 threads and leaves the threshold to the autotuner.
constexpr int kNarrowThreads = 32;
constexpr int kNarrowSlotsPerCta = kSlotCtaThreads / kNarrowThreads;
constexpr int kDefaultNarrowAtoms = 100;

ILVES_HD uint32_t align16(uint32_t b) { return (b + 15u) & ~15u; }

// `staged` = bytes a warp copies into shared memory (everything but con_gid, which is
// read from the global copy of the blob); `bytes` = the whole blob.
// Partitioned molecules add the Schur-contribution tables (see SepInfo, Contrib).
struct ProgLayout {
    uint32_t seg, con_atoms, piv, lvl_task, lvl_piv, lane_term, inc_ptr, inc, atom_off, tasks, terms, sep_info,
        cptr, cent, pprog_off, pprog, staged, con_gid, bytes;
};

// Partitioned molecules: the separator block's entries receive the terms of interior
// pivots (the Schur complement contributions) from the parts that own those pivots.
// Part q computes, for each Contrib entry of its list, the partial sums over terms
// [e0, e1) of task `task` (all with the earlier pivot m inside part q):
//   sum L[row,m] inv_m U[m,col]   and, for a DIAG task, sum L[row,m] inv_m y_m
// into slot `slot` (0 or 1) of that task.  The separator phase then subtracts the
// `ngroups` slots and the remaining terms [b_start, end) itself.
struct SepInfo { uint32_t b_start, ngroups; };
struct Contrib { uint32_t task, slot, e0, e1; };

// Part programs (partitioned molecules): each part's factorisation and back substitution
// again, in 16-bit part-local indices, small enough to stage in the shared memory of the
// part's CTA.  Positions, task slots and atoms count from the part's first; a row or
// column that is a separator is coded 0x8000 | k, k indexing the part's separator table
// (global positions); a fill entry's atom is 0xFFFF.  Terms are stored thread by thread
// for a team of kPartThreads, like the warp programs.  Layout (16-byte aligned sections):
//   header    PartProgHeader
//   lvl_piv   uint16 x (nlev + 1)       local positions of each level
//   lvl_task  uint16 x (nlev + 1)       local task slots of each level
//   septab    int32  x nsep             global positions of the separators referenced
//   lane_term uint32 x kPartThreads     first term of each team thread
//   piv       uint32 x np               U-row slot | (number of U-row entries << 16)
//   aorder    uint16 x na               the part's atoms in update order (decreasing degree)
//   tasks     uint2  x nt               (row | col << 16, atom | neg << 16 | nterm << 24)
//   terms     uint2  x nterm            (l | u << 16, m)
//   contribs  uint2  x ncontrib         the part's Schur contributions (see Contrib):
//                                       (CT slot | DIAG << 31, first cterm | count << 16)
//   cterms    uint2  x ncterm           their terms, (l | u << 16, m)
// followed, in shared memory only, by a scratch section (not in the blob) that holds the
// separators' current and reference rows and solution values during a phase.
constexpr int kPartThreads = 256;
constexpr uint32_t kPartSep = 0x8000u, kPartNoAtom = 0xFFFFu;
struct PartProgHeader { uint32_t np, nt, na, nlev, nsep, nterm, ncontrib, ncterm; };
struct PartProgLayout {
    uint32_t lvl_piv, lvl_task, septab, lane_term, piv, aorder, tasks, terms, contribs, cterms, scratch, bytes;
};
constexpr uint32_t kPartSepScratch = 2u * 32u + 8u;  // per separator: two rows and a value (float64)
ILVES_HD PartProgLayout part_prog_layout(uint32_t np, uint32_t nt, uint32_t na, uint32_t nlev, uint32_t nsep,
                                         uint32_t nterm, uint32_t ncontrib, uint32_t ncterm) {
    PartProgLayout L;
    uint32_t o = (uint32_t)sizeof(PartProgHeader);
    L.lvl_piv = o;   o = align16(o + 2u * (nlev + 1));
    L.lvl_task = o;  o = align16(o + 2u * (nlev + 1));
    L.septab = o;    o = align16(o + 4u * nsep);
    L.lane_term = o; o = align16(o + 4u * (uint32_t)kPartThreads);
    L.piv = o;       o = align16(o + 4u * np);
    L.aorder = o;    o = align16(o + 2u * na);
    L.tasks = o;     o = align16(o + 8u * nt);
    L.terms = o;     o = align16(o + 8u * nterm);
    L.contribs = o;  o = align16(o + 8u * ncontrib);
    L.cterms = o;    o = align16(o + 8u * ncterm);
    L.scratch = o;   o = align16(o + kPartSepScratch * nsep);
    L.bytes = o;
    return L;
}

// Separator program (partitioned molecules): the separator block's factorisation in
// indices local to the block (positions from the first separator, task slots from the
// first separator task), staged in the shared memory of the CTA that solves the block.
// A term whose eliminated pivot is a separator is (l | u << 16, m); one whose pivot is an
// interior pivot (beyond the parts' contribution slots) is (0xFFFFFFFF, global term index).
//   header    SepProgHeader
//   lvl_piv   uint16 x (nlev + 1)
//   lvl_task  uint16 x (nlev + 1)
//   piv       uint32 x nsep             U-row slot | (number of U-row entries << 16)
//   tasks     uint2  x (nt + 1)         (row | col << 16, first term | ngroups << 30), sentinel
//   terms     uint2  x nterm
struct SepProgHeader { uint32_t nsep, nt, nlev, nterm; };
struct SepProgLayout { uint32_t lvl_piv, lvl_task, piv, tasks, terms, bytes; };
constexpr uint32_t kSepInterior = 0xFFFFFFFFu;
ILVES_HD SepProgLayout sep_prog_layout(uint32_t nsep, uint32_t nt, uint32_t nlev, uint32_t nterm) {
    SepProgLayout L;
    uint32_t o = (uint32_t)sizeof(SepProgHeader);
    L.lvl_piv = o;   o = align16(o + 2u * (nlev + 1));
    L.lvl_task = o;  o = align16(o + 2u * (nlev + 1));
    L.piv = o;       o = align16(o + 4u * nsep);
    L.tasks = o;     o = align16(o + 8u * (nt + 1));
    L.terms = o;     o = align16(o + 8u * nterm);
    L.bytes = o;
    return L;
}

// Overlapping domains (OPM, supplement Sec. 3): one connected system solved as a
// quasi-Newton iteration over domains.  Atoms are cut into contiguous parts; part d owns
// the constraints whose smaller atom it holds, and its domain adds the atoms within
// `overlap` edges of its atoms; the domain's system is A restricted to the constraints
// between domain atoms, factorised and solved by one CTA in shared memory, and only the
// owned constraints' corrections are kept.  Blob of an OPM molecule:
//   OpmBlobHeader, dom_off uint32 x (n_dom + 1) (byte offsets of the domain programs from
//   the blob start), con_gid int32 x nc (global id of each molecule-local constraint), then
//   the domain programs.  Domain program (indices local to the domain, 16-byte aligned
//   sections):
//   header    DomProgHeader
//   lvl_piv   uint16 x (nlev + 1)       positions of each level
//   lvl_task  uint16 x (nlev + 1)       task slots of each level
//   lane_term uint32 x kPartThreads     first term of each team thread
//   piv       uint32 x nc               U-row slot | (number of U-row entries << 16)
//   con       uint32 x nc               local atoms i | j << 16 of position p
//   con_ml    uint32 x nc               molecule-local constraint | (owned << 31)
//   atom_ml   int32  x na               molecule-local atom of each domain atom (owned atoms
//                                       first, in order, then the halo)
//   inc_ptr   uint16 x (na_own + 1)     incidence of the owned atoms
//   inc       uint16 x n_inc            position p << 1 | (atom is the second atom of p)
//   aorder    uint16 x na_own           owned atoms in update order (decreasing degree)
//   tasks     uint2  x nt               (row | col << 16, atom | neg << 16 | nterm << 24)
//   terms     uint32 x nterm            l | u << 11 | m << 22 (DomTerm), thread by thread
// so a domain has fewer than 2048 task slots and 1024 constraints.
struct DomTerm {
    static constexpr uint32_t kMaxSlots = 2048, kMaxCons = 1024;
    static ILVES_HD uint32_t l(uint32_t t) { return t & 0x7FFu; }
    static ILVES_HD uint32_t u(uint32_t t) { return (t >> 11) & 0x7FFu; }
    static ILVES_HD uint32_t m(uint32_t t) { return t >> 22; }
    static ILVES_HD uint32_t make(uint32_t l, uint32_t u, uint32_t m) { return l | (u << 11) | (m << 22); }
};
struct OpmBlobHeader { uint32_t n_dom, overlap, pad0, pad1; };
struct DomProgHeader { uint32_t na, na_own, nc, nt, nterm, nlev, n_inc, pad; };
struct DomProgLayout {
    uint32_t lvl_piv, lvl_task, lane_term, piv, con, con_ml, atom_ml, inc_ptr, inc, aorder, tasks, terms, bytes;
};
ILVES_HD DomProgLayout dom_prog_layout(uint32_t na, uint32_t na_own, uint32_t nc, uint32_t nt, uint32_t nterm,
                                       uint32_t nlev, uint32_t n_inc) {
    DomProgLayout L;
    uint32_t o = (uint32_t)sizeof(DomProgHeader);
    L.lvl_piv = o;   o = align16(o + 2u * (nlev + 1));
    L.lvl_task = o;  o = align16(o + 2u * (nlev + 1));
    L.lane_term = o; o = align16(o + 4u * (uint32_t)kPartThreads);
    L.piv = o;       o = align16(o + 4u * nc);
    L.con = o;       o = align16(o + 4u * nc);
    L.con_ml = o;    o = align16(o + 4u * nc);
    L.atom_ml = o;   o = align16(o + 4u * na);
    L.inc_ptr = o;   o = align16(o + 2u * (na_own + 1));
    L.inc = o;       o = align16(o + 2u * n_inc);
    L.aorder = o;    o = align16(o + 2u * na_own);
    L.tasks = o;     o = align16(o + 8u * nt);
    L.terms = o;     o = align16(o + 4u * nterm);
    L.bytes = o;
    return L;
}
// Shared-memory state of a domain behind its program (Mode sizes: hp = 8 bytes of the
// float64 class, lp = factor element size): X (SoA, 3 na float64), WL (na + 1, lp; the
// extra atom has zero weight), W (na_own float64), RHO (SoA, 3 nc float64), RHOF and RF
// (nc x 4 lp; .w = w_i + w_j and 1 / pivot), D2 (nc float64), Y (nc lp), V (nt lp).  With
// `disp` (float-float mode) X holds displacements x - x_unc, RHO only the low float parts
// of rho (the high parts are RHOF.xyz) and SK the differences x_unc,i - x_unc,j (SoA, 3 nc
// float-float pairs); the float64-class values are float-float pairs in the same 8 bytes.
struct DomStateLayout { uint32_t x, wl, w, rho, sk, rhof, rf, d2, y, v, bytes; };
ILVES_HD DomStateLayout dom_state_layout(uint32_t na, uint32_t na_own, uint32_t nc, uint32_t nt, uint32_t lp,
                                         bool disp = false) {
    DomStateLayout S;
    uint32_t o = 0;
    S.x = o;    o = align16(o + 24u * na);
    S.wl = o;   o = align16(o + lp * (na + 1));
    S.w = o;    o = align16(o + 8u * na_own);
    S.rho = o;  o = align16(o + (disp ? 12u : 24u) * nc);
    S.sk = o;   o = align16(o + (disp ? 24u * nc : 0u));
    S.rhof = o; o = align16(o + 4u * lp * nc);
    S.rf = o;   o = align16(o + 4u * lp * nc);
    S.d2 = o;   o = align16(o + 8u * nc);
    S.y = o;    o = align16(o + lp * nc);
    S.v = o;    o = align16(o + lp * nt);
    S.bytes = o;
    return S;
}

// Segment table (n_seg + 1 rows of {first position, first level-table entry, first atom}):
// one segment for an ordinary molecule; for a partitioned molecule one per part, then the
// separators (constraints between parts), whose atom range is empty.
struct SegRow { int32_t piv, lvl, atom; };

template <class IdxT>
ILVES_HD ProgLayout prog_layout(uint32_t na, uint32_t nc, uint32_t ntask, uint32_t nterm,
                                uint32_t nlevel, uint32_t n_seg = 1, uint32_t n_sept = 0, uint32_t n_cent = 0,
                                uint32_t pprog_bytes = 0) {
    ProgLayout L;
    const uint32_t ix = (uint32_t)sizeof(IdxT);
    const bool compact = ix == 2u;
    uint32_t o = 0;
    L.seg = o;       o = align16(o + 12u * (n_seg + 1));
    L.con_atoms = o; o = align16(o + 2u * ix * nc);
    L.piv = o;       o = align16(o + 2u * ix * nc);
    L.lvl_task = o;  o = align16(o + ix * (nlevel + 1));
    L.lvl_piv = o;   o = align16(o + ix * (nlevel + 1));
    L.lane_term = o; o = align16(o + (compact ? ix * (uint32_t)kSlotThreads : 0u));
    L.inc_ptr = o;   o = align16(o + ix * (na + 1));
    L.inc = o;       o = align16(o + ix * 2u * nc);
    L.atom_off = o;  o = align16(o + (compact ? ix * na : 0u));  // atom slot -> local atom
    L.tasks = o;     o = align16(o + (compact ? 4u * ntask : 4u * ix * (ntask + 1)));
    L.terms = o;     o = align16(o + (uint32_t)sizeof(typename TermOf<IdxT>::T) * nterm);
    const bool parted = n_seg > 1;
    L.sep_info = o;  o = align16(o + (parted ? 8u * n_sept : 0u));
    L.cptr = o;      o = align16(o + (parted ? 4u * n_seg : 0u));  // n_parts + 1 = n_seg entries
    L.cent = o;      o = align16(o + (parted ? 16u * n_cent : 0u));
    L.pprog_off = o; o = align16(o + (pprog_bytes ? 4u * (n_seg + 1) : 0u));  // parts, separators, end
    L.pprog = o;     o = align16(o + pprog_bytes);
    L.staged = o;
    L.con_gid = o;   o = align16(o + 4u * nc);
    L.bytes = o;
    return L;
}

// Numerical state of one molecule (after its program).  Float64-class values (float64,
// or float-float pairs of the same size) take 8 bytes; lp_bytes is the factor element
// size (4 for float32, 8 for float64); 3-vectors of the factor precision take 4
// elements and use the fourth: rhof[p].w holds w_i + w_j (the weight of a DIAG entry),
// rf[p].w holds 1 / pivot p of the current factor.  Atom arrays have na + 1 entries:
// the extra atom has zero weight and is what fill entries of the pattern point at.
// With `disp` (float-float mode) the state keeps displacements x - x_unc and the
// per-constraint differences s_k = x_unc,i - x_unc,j, and rho keeps only the low
// float parts of rho (the high parts are rhof.xyz).
// `stage` (= rf, up to the end) is free until the first violation pass: the warp path
// gathers x_old there (AoS, 24 B per atom) while it sets the molecule up; the region is
// extended when the arrays after rf are smaller than that.
struct StateLayout {
    uint32_t x, w, wl, rho, s, d2, lam, rhof, y, rf, vals, stage, bytes;
};

ILVES_HD StateLayout state_layout(uint32_t na, uint32_t nc, uint32_t ntask, uint32_t lp_bytes, bool disp) {
    StateLayout S;
    const uint32_t vp = 4u * lp_bytes;
    uint32_t o = 0;
    S.x = o;      o = align16(o + 24u * na);             // SoA: x[0..na), y[..], z[..]
    S.w = o;      o = align16(o + 8u * (na + 1));
    S.wl = o;     o = align16(o + lp_bytes * (na + 1));
    S.rho = o;    o = align16(o + (disp ? 12u : 24u) * nc);  // SoA
    S.s = o;      o = align16(o + (disp ? 24u * nc : 0u));
    S.d2 = o;     o = align16(o + 8u * nc);
    S.lam = o;    o = align16(o + 8u * nc);
    S.rhof = o;   o = align16(o + vp * nc);
    S.y = o;      o = align16(o + (lp_bytes > 4u ? lp_bytes : 4u) * nc);
    S.rf = o;     o = align16(o + vp * nc);
    S.vals = o;   o = align16(o + lp_bytes * ntask);
    S.stage = S.rf;
    const uint32_t stage_end = align16(S.stage + 24u * na);
    S.bytes = o > stage_end ? o : stage_end;
    return S;
}

// One molecule as the kernels see it (72 bytes).
struct MolDesc {
    int64_t blob_off;    // byte offset of the program blob in the blob buffer (16-B aligned)
    int64_t work_off;    // large path: byte offset of the numerical state in the workspace
    int32_t atom_base;   // first global atom if the molecule's atoms are contiguous, else -1
    int32_t gid_off;     // offset of this molecule's global atom ids in atom_gid[]
    int32_t mol_id;      // output index (molecules ordered by smallest atom)
    int32_t nterm;
    int32_t ntask;
    int32_t na, nc;
    int32_t nlevel;  // level-table entries - 1 (for one segment: its number of levels)
    int32_t n_seg;   // 1, or parts + 1 for a partitioned molecule
    int32_t n_sept;  // partitioned: tasks of the separator segment (they are the last ones)
    int32_t n_cent;  // partitioned: Schur contribution entries over all parts
    int32_t pprog_bytes;  // partitioned: bytes of the segment programs (parts, then separators)
    int32_t opm;          // overlapping domains: overlap depth (0 = not solved by domains)
};

}  // namespace ilves
