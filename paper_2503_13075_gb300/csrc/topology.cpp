// topology.cpp -- host-side setup of the ILVES constraint topology (no CUDA calls).
//
// Implements the initialisation the paper performs once per neighbour-list
// rebuild (supplement Sec. 3): constraint graph G -> connected components
// (molecules) -> line graph L(G), whose adjacency is the sparsity pattern of the
// Newton matrix A (supplement Sec. 2.3: a_ij = 0 unless bonds i and j share an
// atom) -> fill-reducing elimination order -> symbolic LU.  On top of that it
// compiles, per molecule, the level-scheduled task program the CUDA kernels
// interpret, and partitions the molecules over persistent CTAs.
//
// Elimination order.  The paper uses an approximate-minimum-degree order per
// partition (supplement Sec. 3).  Here the order is chosen for a GPU team that
// synchronises once per elimination-tree level: pivots are eliminated in rounds,
// each round taking a greedy independent set of the vertices whose current degree
// is at most (minimum degree + slack).  slack = 0 is a multiple-minimum-degree
// order; a larger slack admits a little more fill for far fewer levels (on a
// chain it becomes cyclic reduction).  The slack is chosen per molecule by a cost
// model of the kernel (level passes + work), see choose_order().
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <iterator>
#include <numeric>
#include <queue>
#include <vector>

#include "ilves.h"
#include "internal.h"
#include "topology_impl.h"

namespace ilves {

static int32_t uf_find(std::vector<int32_t>& p, int32_t a) {
    while (p[a] != a) {
        p[a] = p[p[a]];
        a = p[a];
    }
    return a;
}

// ------------------------------------------------------------------------------------
// elimination by rounds of independent low-degree vertices
// ------------------------------------------------------------------------------------
struct Elimination {
    std::vector<std::vector<int32_t>> nplus;  // neighbours at elimination time (local ids)
    std::vector<int32_t> order;               // elimination sequence
    int64_t n_fill = 0;
};

// dst := (dst U src) \ {skip}; both sorted
static void sorted_merge_into(std::vector<int32_t>& dst, const std::vector<int32_t>& src, int32_t skip,
                              std::vector<int32_t>& tmp) {
    tmp.clear();
    tmp.reserve(dst.size() + src.size());
    size_t i = 0, j = 0;
    while (i < dst.size() || j < src.size()) {
        int32_t v;
        if (j >= src.size() || (i < dst.size() && dst[i] < src[j])) {
            v = dst[i++];
        } else if (i >= dst.size() || src[j] < dst[i]) {
            v = src[j++];
        } else {
            v = dst[i++];
            ++j;
        }
        if (v != skip) tmp.push_back(v);
    }
    dst.swap(tmp);
}

// stage (optional): vertices of a higher stage become eligible only once every vertex of a
// lower stage is eliminated (used to eliminate the separators of a partition last).
static Elimination eliminate_rounds(int32_t n, std::vector<std::vector<int32_t>> H, int32_t slack,
                                    bool one_per_round, const std::vector<int8_t>* stage = nullptr) {
    Elimination E;
    E.nplus.assign(n, {});
    E.order.reserve(n);
    std::vector<int32_t> stamp(n, -1);
    std::vector<char> alive(n, 1);
    int32_t remaining = n, rnd = 0;
    std::vector<std::pair<int32_t, int32_t>> dv;
    std::vector<int32_t> chosen, tmp;
    int64_t added = 0;
    int8_t cur_stage = 0;
    std::vector<int32_t> left_in_stage(2, 0);
    if (stage)
        for (int32_t v = 0; v < n; ++v) ++left_in_stage[(*stage)[v]];
    while (remaining > 0) {
        if (stage && left_in_stage[cur_stage] == 0) ++cur_stage;
        dv.clear();
        for (int32_t v = 0; v < n; ++v)
            if (alive[v] && (!stage || (*stage)[v] == cur_stage)) dv.push_back({(int32_t)H[v].size(), v});
        std::sort(dv.begin(), dv.end());
        const int32_t mind = dv[0].first;
        chosen.clear();
        for (auto& pr : dv) {
            const int32_t dg = pr.first, v = pr.second;
            if (dg > mind + slack) break;
            if (stamp[v] == rnd) continue;
            chosen.push_back(v);
            stamp[v] = rnd;
            for (int32_t u : H[v]) stamp[u] = rnd;
            if (one_per_round) break;
        }
        for (int32_t v : chosen) {
            E.nplus[v] = H[v];
            for (int32_t x : H[v]) {
                auto& hx = H[x];
                hx.erase(std::lower_bound(hx.begin(), hx.end(), v));
                const size_t before = hx.size();
                sorted_merge_into(hx, H[v], x, tmp);
                added += (int64_t)(hx.size() - before);
            }
            H[v].clear();
            H[v].shrink_to_fit();
            alive[v] = 0;
            E.order.push_back(v);
            if (stage) --left_in_stage[(*stage)[v]];
        }
        remaining -= (int32_t)chosen.size();
        ++rnd;
    }
    E.n_fill = added / 2;
    return E;
}

// ------------------------------------------------------------------------------------
// per-molecule program
// ------------------------------------------------------------------------------------
struct Program {
    int32_t nlevel = 0;
    std::vector<int32_t> pos_con;            // local constraint id at each position
    std::vector<int32_t> level;              // per position
    std::vector<std::vector<int32_t>> up;    // N+(p) as sorted positions
    std::vector<int32_t> diag_task;          // per position: slot of its DIAG task
    std::vector<int32_t> ustart;             // per position: first slot of its U row (then L column)
    std::vector<TaskW> tasks;                // + sentinel
    std::vector<TermW> terms;
    std::vector<int32_t> lvl_task, lvl_piv;  // per segment: n_lev + 1 entries, concatenated
    // segments: parts of a partitioned molecule (then the separators), or one segment
    int32_t n_seg = 1;
    std::vector<int32_t> seg_piv, seg_lvl, seg_atom;  // n_seg + 1 each
    int64_t passes_factor = 0, passes_solve = 0;
    int64_t n_fill = 0;
    // partitioned: Schur contributions of the parts to the separator tasks
    int32_t sep_t0 = 0;                        // first task of the separator segment
    std::vector<SepInfo> sep_info;             // per separator task
    std::vector<int32_t> cptr;                 // per part: [cptr[q], cptr[q+1]) into cent
    std::vector<Contrib> cent;
    // partitioned: part programs (see PartProgHeader), empty if a part does not fit them
    std::vector<uint8_t> pprog;
    std::vector<uint32_t> pprog_off;  // per part, the separator program, its end
    uint32_t pprog_max = 0;           // largest part program (bytes)
    int32_t sep_interior = 0;         // separator-program terms on interior pivots
    // overlapping domains: the whole blob, and per domain its part bounds (atoms), constraints
    // (molecule-local, ascending) with owned flags, levels and program bytes
    std::vector<uint8_t> opm_blob;
    std::vector<int32_t> dom_bounds, dom_con_ptr, dom_cons, dom_levels, dom_bytes;
    std::vector<uint8_t> dom_owned;
};

// Part programs of a partitioned molecule (16-bit part-local encoding of the part's
// tasks, terms and pivots; see PartProgHeader); false if some part exceeds the
// encoding's ranges.
static bool build_part_programs(Program& P, int32_t na_dummy, const std::vector<int32_t>& ci,
                                const std::vector<int32_t>& cj) {
    std::vector<int32_t> deg(na_dummy, 0);
    for (size_t c = 0; c < ci.size(); ++c) {
        ++deg[ci[c]];
        ++deg[cj[c]];
    }
    const int32_t n_parts = P.n_seg - 1;
    const int32_t sep_p0 = P.seg_piv[n_parts];
    P.pprog.clear();
    P.pprog_off.assign(n_parts + 1, 0);
    P.pprog_max = 0;
    for (int32_t g = 0; g < n_parts; ++g) {
        const int32_t P0 = P.seg_piv[g], P1 = P.seg_piv[g + 1], np = P1 - P0;
        const int32_t lv0 = P.seg_lvl[g], nlev = P.seg_lvl[g + 1] - 1 - lv0;
        const int32_t T0 = P.lvl_task[lv0], T1 = P.lvl_task[lv0 + nlev], nt = T1 - T0;
        const int32_t A0 = P.seg_atom[g], A1 = P.seg_atom[g + 1];
        if (np >= (int32_t)kPartSep || nt >= 65536 || A1 - A0 >= (int32_t)kPartNoAtom) return false;
        std::vector<int32_t> septab;
        auto code = [&](int32_t pos, uint32_t& c) {
            if (pos >= P0 && pos < P1) {
                c = (uint32_t)(pos - P0);
                return true;
            }
            if (pos < sep_p0) return false;  // another part: not expected in this part's tasks
            auto it = std::lower_bound(septab.begin(), septab.end(), pos);
            c = kPartSep | (uint32_t)(it - septab.begin());
            return true;
        };
        for (int32_t t = T0; t < T1; ++t)
            for (int32_t pos : {(int32_t)P.tasks[t].row, (int32_t)P.tasks[t].col})
                if (pos >= sep_p0) septab.push_back(pos);
        std::sort(septab.begin(), septab.end());
        septab.erase(std::unique(septab.begin(), septab.end()), septab.end());
        if (septab.size() >= kPartSep) return false;
        // terms, thread by thread over the part's levels
        std::vector<uint32_t> lane_term(kPartThreads);
        std::vector<uint32_t> terms;
        for (int32_t r = 0; r < kPartThreads; ++r) {
            lane_term[r] = (uint32_t)(terms.size() / 2);
            for (int32_t l = 0; l < nlev; ++l)
                for (int32_t t = P.lvl_task[lv0 + l] + r; t < P.lvl_task[lv0 + l + 1]; t += kPartThreads)
                    for (uint32_t k = P.tasks[t].tstart; k < P.tasks[t + 1].tstart; ++k) {
                        const TermW& tr = P.terms[k];
                        const int32_t l_ = (int32_t)tr.l - T0, u_ = (int32_t)tr.u - T0, m_ = (int32_t)tr.m - P0;
                        if (l_ < 0 || l_ >= nt || u_ < 0 || u_ >= nt || m_ < 0 || m_ >= np) return false;
                        terms.push_back((uint32_t)l_ | ((uint32_t)u_ << 16));
                        terms.push_back((uint32_t)m_);
                    }
        }
        const uint32_t nterm = (uint32_t)(terms.size() / 2);
        // the part's Schur contributions: separator task slot in the contribution table,
        // DIAG flag, and their terms in part-local indices
        std::vector<uint32_t> contribs, cterms;
        for (int32_t c = P.cptr[g]; c < P.cptr[g + 1]; ++c) {
            const Contrib& E = P.cent[c];
            const TaskW& tk = P.tasks[E.task];
            const uint32_t ct = 4u * (E.task - (uint32_t)P.sep_t0) + E.slot;
            const uint32_t first = (uint32_t)(cterms.size() / 2), count = E.e1 - E.e0;
            if (ct >= 0x80000000u || first + count >= 65536u) return false;
            contribs.push_back(ct | (tk.row == tk.col ? 0x80000000u : 0u));
            contribs.push_back(first | (count << 16));
            for (uint32_t e = E.e0; e < E.e1; ++e) {
                const TermW& tr = P.terms[e];
                const int32_t l_ = (int32_t)tr.l - T0, u_ = (int32_t)tr.u - T0, m_ = (int32_t)tr.m - P0;
                if (l_ < 0 || l_ >= nt || u_ < 0 || u_ >= nt || m_ < 0 || m_ >= np) return false;
                cterms.push_back((uint32_t)l_ | ((uint32_t)u_ << 16));
                cterms.push_back((uint32_t)m_);
            }
        }
        const uint32_t ncontrib = (uint32_t)(contribs.size() / 2), ncterm = (uint32_t)(cterms.size() / 2);
        const PartProgLayout L =
            part_prog_layout(np, nt, A1 - A0, nlev, (uint32_t)septab.size(), nterm, ncontrib, ncterm);
        const size_t base = P.pprog.size();
        P.pprog_off[g] = (uint32_t)base;
        P.pprog.resize(base + L.scratch, 0);  // the scratch section exists in shared memory only
        uint8_t* d = P.pprog.data() + base;
        const PartProgHeader H{(uint32_t)np,    (uint32_t)nt, (uint32_t)(A1 - A0), (uint32_t)nlev,
                               (uint32_t)septab.size(), nterm, ncontrib, ncterm};
        std::memcpy(d, &H, sizeof(H));
        auto* lp = reinterpret_cast<uint16_t*>(d + L.lvl_piv);
        auto* lt = reinterpret_cast<uint16_t*>(d + L.lvl_task);
        for (int32_t l = 0; l <= nlev; ++l) {
            lp[l] = (uint16_t)(P.lvl_piv[lv0 + l] - P0);
            lt[l] = (uint16_t)(P.lvl_task[lv0 + l] - T0);
        }
        std::memcpy(d + L.septab, septab.data(), septab.size() * 4);
        std::memcpy(d + L.lane_term, lane_term.data(), lane_term.size() * 4);
        // update order: decreasing degree, so a warp's lanes run equal incidence loops
        std::vector<int32_t> ord(A1 - A0);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return deg[A0 + x] > deg[A0 + y]; });
        auto* ao = reinterpret_cast<uint16_t*>(d + L.aorder);
        for (int32_t k = 0; k < A1 - A0; ++k) ao[k] = (uint16_t)ord[k];
        auto* pv = reinterpret_cast<uint32_t*>(d + L.piv);
        for (int32_t p = P0; p < P1; ++p) {
            const int32_t us = P.ustart[p] - T0, nu = (int32_t)P.up[p].size();
            if (us < 0 || us + nu > nt) return false;
            pv[p - P0] = (uint32_t)us | ((uint32_t)nu << 16);
        }
        auto* tw = reinterpret_cast<uint32_t*>(d + L.tasks);
        for (int32_t t = T0; t < T1; ++t) {
            const TaskW& w = P.tasks[t];
            uint32_t rc, cc;
            if (!code((int32_t)w.row, rc) || !code((int32_t)w.col, cc)) return false;
            const uint32_t nterm_t = P.tasks[t + 1].tstart - w.tstart;
            if (nterm_t > 255u) return false;
            // the shared atom of an off-diagonal entry is an atom of the part's constraint
            const int32_t a = (int32_t)(w.atomsign >> 1);
            uint32_t ac = kPartNoAtom;
            if (w.row != w.col && a != na_dummy) {
                if (a < A0 || a >= A1) return false;
                ac = (uint32_t)(a - A0);
            }
            tw[2 * (t - T0)] = rc | (cc << 16);
            tw[2 * (t - T0) + 1] = ac | ((w.atomsign & 1u) << 16) | (nterm_t << 24);
        }
        std::memcpy(d + L.terms, terms.data(), terms.size() * 4);
        std::memcpy(d + L.contribs, contribs.data(), contribs.size() * 4);
        std::memcpy(d + L.cterms, cterms.data(), cterms.size() * 4);
        P.pprog_max = std::max(P.pprog_max, L.bytes);
        // keep each part program 16-byte aligned
        P.pprog.resize((P.pprog.size() + 15) & ~size_t(15), 0);
    }
    P.pprog_off[n_parts] = (uint32_t)P.pprog.size();
    return true;
}

// The separator block's program (see SepProgHeader), appended to the part programs;
// pprog_off[n_parts] .. pprog_off[n_parts + 1] delimits it.
static void build_sep_program(Program& P, int32_t nc) {
    const int32_t n_parts = P.n_seg - 1;
    const int32_t sep_p0 = P.seg_piv[n_parts], nsep = nc - sep_p0;
    const int32_t lv0 = P.seg_lvl[n_parts], nlev = P.seg_lvl[n_parts + 1] - 1 - lv0;
    const int32_t T0 = P.sep_t0, nt = (int32_t)P.tasks.size() - 1 - T0;
    P.pprog_off.resize(n_parts + 2);
    P.pprog_off[n_parts + 1] = P.pprog_off[n_parts] = (uint32_t)P.pprog.size();
    P.sep_interior = 0;
    if (nsep >= 65536 || nt >= 65536) return;  // no program: too large for shared memory anyway
    std::vector<uint32_t> tw(2 * (nt + 1)), terms;
    for (int32_t k = 0; k < nt; ++k) {
        const int32_t t = T0 + k;
        const SepInfo si = P.sep_info[k];
        tw[2 * k] = (P.tasks[t].row - (uint32_t)sep_p0) | ((P.tasks[t].col - (uint32_t)sep_p0) << 16);
        tw[2 * k + 1] = (uint32_t)(terms.size() / 2) | (si.ngroups << 30);
        for (uint32_t e = si.b_start; e < P.tasks[t + 1].tstart; ++e) {
            const TermW& tr = P.terms[e];
            if ((int32_t)tr.m >= sep_p0) {
                terms.push_back((tr.l - (uint32_t)T0) | ((tr.u - (uint32_t)T0) << 16));
                terms.push_back(tr.m - (uint32_t)sep_p0);
            } else {
                terms.push_back(kSepInterior);
                terms.push_back(e);
                ++P.sep_interior;
            }
        }
    }
    const uint32_t nterm = (uint32_t)(terms.size() / 2);
    tw[2 * nt] = 0u;
    tw[2 * nt + 1] = nterm;
    const SepProgLayout L = sep_prog_layout((uint32_t)nsep, (uint32_t)nt, (uint32_t)nlev, nterm);
    const size_t base = P.pprog.size();
    P.pprog.resize(base + L.bytes, 0);
    uint8_t* d = P.pprog.data() + base;
    const SepProgHeader H{(uint32_t)nsep, (uint32_t)nt, (uint32_t)nlev, nterm};
    std::memcpy(d, &H, sizeof(H));
    auto* lp = reinterpret_cast<uint16_t*>(d + L.lvl_piv);
    auto* lt = reinterpret_cast<uint16_t*>(d + L.lvl_task);
    for (int32_t l = 0; l <= nlev; ++l) {
        lp[l] = (uint16_t)(P.lvl_piv[lv0 + l] - sep_p0);
        lt[l] = (uint16_t)(P.lvl_task[lv0 + l] - T0);
    }
    auto* pv = reinterpret_cast<uint32_t*>(d + L.piv);
    for (int32_t p = sep_p0; p < nc; ++p)
        pv[p - sep_p0] = (uint32_t)(P.ustart[p] - T0) | ((uint32_t)P.up[p].size() << 16);
    std::memcpy(d + L.tasks, tw.data(), tw.size() * 4);
    std::memcpy(d + L.terms, terms.data(), terms.size() * 4);
    P.pprog_off[n_parts + 1] = (uint32_t)P.pprog.size();
}

// seg (optional): segment of every local constraint (a part, or n_seg - 1 for the
// separators); positions are ordered by segment, then level; levels count only
// dependencies inside the same segment (earlier segments are complete before a later
// segment starts).
static Program compile(int32_t nc, const Elimination& E, const std::vector<int32_t>& ci,
                       const std::vector<int32_t>& cj, int32_t team, int32_t na_dummy,
                       const std::vector<int32_t>* seg = nullptr, int32_t n_seg = 1,
                       const std::vector<int32_t>* seg_atom = nullptr) {
    Program P;
    P.n_fill = E.n_fill;
    P.n_seg = n_seg;
    auto sg = [&](int32_t v) { return seg ? (*seg)[v] : 0; };
    std::vector<int32_t> lev(nc, 0);
    for (int32_t v : E.order)
        for (int32_t x : E.nplus[v])
            if (sg(x) == sg(v)) lev[x] = std::max(lev[x], lev[v] + 1);
    std::vector<int32_t> seqidx(nc);
    for (int32_t i = 0; i < nc; ++i) seqidx[E.order[i]] = i;
    P.pos_con.resize(nc);
    std::iota(P.pos_con.begin(), P.pos_con.end(), 0);
    std::sort(P.pos_con.begin(), P.pos_con.end(), [&](int32_t a, int32_t b) {
        if (sg(a) != sg(b)) return sg(a) < sg(b);
        return lev[a] != lev[b] ? lev[a] < lev[b] : seqidx[a] < seqidx[b];
    });
    std::vector<int32_t> pos_of(nc);
    for (int32_t p = 0; p < nc; ++p) pos_of[P.pos_con[p]] = p;
    P.level.resize(nc);
    P.up.assign(nc, {});
    for (int32_t p = 0; p < nc; ++p) {
        const int32_t v = P.pos_con[p];
        P.level[p] = lev[v];
        for (int32_t x : E.nplus[v]) P.up[p].push_back(pos_of[x]);
        std::sort(P.up[p].begin(), P.up[p].end());
    }
    std::vector<std::vector<int32_t>> dn(nc);  // N-(p), ascending
    for (int32_t m = 0; m < nc; ++m)
        for (int32_t q : P.up[m]) dn[q].push_back(m);
    // segment boundaries and per-segment level boundaries (positions)
    P.seg_piv.assign(n_seg + 1, nc);
    for (int32_t p = nc - 1; p >= 0; --p) P.seg_piv[sg(P.pos_con[p])] = p;
    for (int32_t g = n_seg - 1; g >= 0; --g) P.seg_piv[g] = std::min(P.seg_piv[g], P.seg_piv[g + 1]);
    P.seg_lvl.assign(n_seg + 1, 0);
    P.lvl_piv.clear();
    std::vector<int32_t> seg_nlev(n_seg, 0);
    for (int32_t g = 0; g < n_seg; ++g) {
        const int32_t p0 = P.seg_piv[g], p1 = P.seg_piv[g + 1];
        const int32_t nl = p1 > p0 ? P.level[p1 - 1] + 1 : 0;
        seg_nlev[g] = nl;
        P.seg_lvl[g] = (int32_t)P.lvl_piv.size();
        std::vector<int32_t> starts(nl + 1, p1);
        for (int32_t p = p1 - 1; p >= p0; --p) starts[P.level[p]] = p;
        P.lvl_piv.insert(P.lvl_piv.end(), starts.begin(), starts.end());
    }
    P.seg_lvl[n_seg] = (int32_t)P.lvl_piv.size();
    P.nlevel = (int32_t)P.lvl_piv.size() - 1;  // one segment: its level count
    P.seg_atom.assign(n_seg + 1, 0);
    if (seg_atom) P.seg_atom = *seg_atom;
    // task slots: per segment and level, the DIAG tasks of its pivots, then per pivot its
    // U row and L column
    P.diag_task.resize(nc);
    P.ustart.resize(nc);
    P.lvl_task.assign(P.lvl_piv.size(), 0);
    int32_t t = 0;
    for (int32_t g = 0; g < n_seg; ++g) {
        const int32_t b = P.seg_lvl[g];
        for (int32_t l = 0; l < seg_nlev[g]; ++l) {
            P.lvl_task[b + l] = t;
            for (int32_t p = P.lvl_piv[b + l]; p < P.lvl_piv[b + l + 1]; ++p) P.diag_task[p] = t++;
            for (int32_t p = P.lvl_piv[b + l]; p < P.lvl_piv[b + l + 1]; ++p) {
                P.ustart[p] = t;
                t += 2 * (int32_t)P.up[p].size();
            }
        }
        P.lvl_task[b + seg_nlev[g]] = t;
    }
    auto kpos = [&](int32_t m, int32_t q) {
        const auto& u = P.up[m];
        return (int32_t)(std::lower_bound(u.begin(), u.end(), q) - u.begin());
    };
    auto slot_U = [&](int32_t m, int32_t q) { return P.ustart[m] + kpos(m, q); };
    auto slot_L = [&](int32_t q, int32_t m) { return P.ustart[m] + (int32_t)P.up[m].size() + kpos(m, q); };
    // shared atom and sign product s_a(atom) s_b(atom) of two constraints of the graph;
    // fill entries point at a dummy atom of zero weight (index na) so they assemble to 0
    auto atomsign = [&](int32_t pa, int32_t pb) -> uint32_t {
        const int32_t a = P.pos_con[pa], b = P.pos_con[pb];
        const uint32_t ai = ci[a], aj = cj[a], bi = ci[b], bj = cj[b];
        if (ai == bi) return ai << 1;         // (+1)(+1)
        if (aj == bj) return aj << 1;         // (-1)(-1)
        if (ai == bj) return (ai << 1) | 1u;  // (+1)(-1)
        if (aj == bi) return (aj << 1) | 1u;  // (-1)(+1)
        return (uint32_t)na_dummy << 1;       // fill entry
    };
    std::vector<int32_t> ms;
    auto common = [&](int32_t a, int32_t b) {
        ms.clear();
        std::set_intersection(dn[a].begin(), dn[a].end(), dn[b].begin(), dn[b].end(),
                              std::back_inserter(ms));
    };
    P.tasks.assign(t + 1, TaskW{0, 0, 0, 0});
    std::vector<std::vector<TermW>> tterms(t);
    for (int32_t p = 0; p < nc; ++p) {
        const int32_t td = P.diag_task[p];
        // DIAG: a_pp = 4 (w_i + w_j) r_p . rho_p; the kernels keep w_i + w_j next to rho_p
        P.tasks[td] = {(uint32_t)p, (uint32_t)p, (uint32_t)na_dummy << 1, 0u};
        for (int32_t m : dn[p]) tterms[td].push_back({(uint32_t)slot_L(p, m), (uint32_t)slot_U(m, p), (uint32_t)m, 0u});
        const int32_t nu = (int32_t)P.up[p].size();
        for (int32_t k = 0; k < nu; ++k) {
            const int32_t q = P.up[p][k];
            const int32_t tu = P.ustart[p] + k, tl = P.ustart[p] + nu + k;
            P.tasks[tu] = {(uint32_t)p, (uint32_t)q, atomsign(p, q), 0u};
            common(p, q);
            for (int32_t m : ms) tterms[tu].push_back({(uint32_t)slot_L(p, m), (uint32_t)slot_U(m, q), (uint32_t)m, 0u});
            P.tasks[tl] = {(uint32_t)q, (uint32_t)p, atomsign(q, p), 0u};
            for (int32_t m : ms) tterms[tl].push_back({(uint32_t)slot_L(q, m), (uint32_t)slot_U(m, p), (uint32_t)m, 0u});
        }
    }
    for (int32_t k = 0; k < t; ++k) {
        P.tasks[k].tstart = (uint32_t)P.terms.size();
        P.terms.insert(P.terms.end(), tterms[k].begin(), tterms[k].end());
    }
    P.tasks[t] = {0u, 0u, kNoAtom32, (uint32_t)P.terms.size()};  // sentinel
    if (n_seg > 1) {
        // Schur contributions: the terms of a separator task are in ascending pivot
        // position, so the interior pivots come first, grouped by part; the first two
        // groups are summed by their parts, the rest (and the separator pivots) by the
        // separator phase itself
        const int32_t sep_seg = n_seg - 1, sep_p0 = P.seg_piv[sep_seg];
        P.sep_t0 = P.lvl_task[P.seg_lvl[sep_seg]];
        std::vector<int32_t> seg_of(nc, sep_seg);
        for (int32_t g = 0; g < sep_seg; ++g)
            for (int32_t p = P.seg_piv[g]; p < P.seg_piv[g + 1]; ++p) seg_of[p] = g;
        std::vector<std::vector<Contrib>> per_part(sep_seg);
        P.sep_info.assign(t - P.sep_t0, SepInfo{0u, 0u});
        for (int32_t k = P.sep_t0; k < t; ++k) {
            const uint32_t e0 = P.tasks[k].tstart, e1 = P.tasks[k + 1].tstart;
            uint32_t e = e0, ng = 0;
            while (e < e1 && (int32_t)P.terms[e].m < sep_p0 && ng < 2) {
                const int32_t q = seg_of[P.terms[e].m];
                uint32_t f = e;
                while (f < e1 && (int32_t)P.terms[f].m < sep_p0 && seg_of[P.terms[f].m] == q) ++f;
                per_part[q].push_back(Contrib{(uint32_t)k, ng, e, f});
                ++ng;
                e = f;
            }
            P.sep_info[k - P.sep_t0] = SepInfo{e, ng};
        }
        P.cptr.assign(sep_seg + 1, 0);
        for (int32_t q = 0; q < sep_seg; ++q) {
            P.cptr[q] = (int32_t)P.cent.size();
            P.cent.insert(P.cent.end(), per_part[q].begin(), per_part[q].end());
        }
        P.cptr[sep_seg] = (int32_t)P.cent.size();
    }
    for (int32_t g = 0; g < n_seg; ++g) {
        const int32_t b = P.seg_lvl[g];
        for (int32_t l = 0; l < seg_nlev[g]; ++l) {
            P.passes_factor += (P.lvl_task[b + l + 1] - P.lvl_task[b + l] + team - 1) / team;
            P.passes_solve += (P.lvl_piv[b + l + 1] - P.lvl_piv[b + l] + team - 1) / team;
        }
    }
    return P;
}

// Greedy partition of a molecule's atoms (already in index order) into n_parts
// contiguous parts, after the paper's description (supplement Sec. 3): atoms are taken in
// order while the part is below target + offset; the last atom of a part is chosen among
// the sizes within maxDeviation of the target by cut edges (penalty cutPenalty per edge
// crossing the boundary) and distance to the target size.  O(|E|).
static std::vector<int32_t> partition_atoms(int32_t na, const std::vector<int32_t>& ci,
                                            const std::vector<int32_t>& cj, int32_t n_parts,
                                            double max_dev = 0.05, double cut_penalty = 10.0) {
    std::vector<std::vector<int32_t>> nb(na);
    for (size_t k = 0; k < ci.size(); ++k) {
        nb[ci[k]].push_back(cj[k]);
        nb[cj[k]].push_back(ci[k]);
    }
    std::vector<int32_t> bounds{0};
    int32_t a0 = 0;
    for (int32_t p = 0; p + 1 < n_parts && a0 < na; ++p) {
        const double target = (double)(na - a0) / (double)(n_parts - p);
        const int32_t lo = std::max(a0 + 1, (int32_t)std::floor(a0 + target * (1.0 - max_dev)));
        const int32_t hi = std::min(na - 1, (int32_t)std::ceil(a0 + target * (1.0 + max_dev)));
        // open = edges from [a0, e) to [e, na): sweep e upwards from a0
        int64_t open = 0;
        int32_t best_e = std::min(na - 1, std::max(lo, a0 + 1));
        double best = 1e300;
        for (int32_t e = a0 + 1; e <= hi; ++e) {
            const int32_t u = e - 1;  // atom u joins the part
            for (int32_t v : nb[u]) open += (v >= e) ? 1 : ((v >= a0 && v < u) ? -1 : 0);
            if (e < lo) continue;
            const double score = cut_penalty * (double)open + std::fabs((double)(e - a0) - target);
            if (score < best) {
                best = score;
                best_e = e;
            }
        }
        if (best_e <= a0) break;
        bounds.push_back(best_e);
        a0 = best_e;
    }
    bounds.push_back(na);
    return bounds;
}

// ------------------------------------------------------------------------------------
// overlapping domains (supplement Sec. 3, the Overlapping Partitioning Method)
// ------------------------------------------------------------------------------------
struct DomainPlan {
    std::vector<int32_t> atoms;  // molecule-local atoms: the part's own (in order), then the halo (ascending)
    int32_t na_own = 0;
    std::vector<int32_t> cons;   // molecule-local constraints between domain atoms, ascending
    std::vector<uint8_t> owned;  // per entry of cons: the part owns it (holds its smaller atom)
};

// Part d owns atoms [bounds[d], bounds[d + 1]) and the constraints whose smaller atom it
// owns; its domain adds every atom within `overlap` edges of its atoms (breadth-first over
// the constraint graph) and holds the constraints whose two atoms are domain atoms.
static std::vector<DomainPlan> opm_domains(int32_t na, const std::vector<int32_t>& ci, const std::vector<int32_t>& cj,
                                           const std::vector<int32_t>& bounds, int32_t overlap) {
    const int32_t nc = (int32_t)ci.size(), nd = (int32_t)bounds.size() - 1;
    std::vector<std::vector<int32_t>> inc(na);
    for (int32_t c = 0; c < nc; ++c) {
        inc[ci[c]].push_back(c);
        inc[cj[c]].push_back(c);
    }
    std::vector<int32_t> part_of(na), amark(na, -1), cmark(nc, -1);
    for (int32_t d = 0; d < nd; ++d)
        for (int32_t a = bounds[d]; a < bounds[d + 1]; ++a) part_of[a] = d;
    std::vector<DomainPlan> D(nd);
    std::vector<int32_t> frontier, next, halo;
    for (int32_t d = 0; d < nd; ++d) {
        DomainPlan& P = D[d];
        frontier.clear();
        halo.clear();
        for (int32_t a = bounds[d]; a < bounds[d + 1]; ++a) {
            amark[a] = d;
            P.atoms.push_back(a);
            frontier.push_back(a);
        }
        P.na_own = (int32_t)P.atoms.size();
        for (int32_t step = 0; step < overlap; ++step) {
            next.clear();
            for (int32_t a : frontier)
                for (int32_t c : inc[a]) {
                    const int32_t b = ci[c] == a ? cj[c] : ci[c];
                    if (amark[b] != d) {
                        amark[b] = d;
                        next.push_back(b);
                        halo.push_back(b);
                    }
                }
            frontier.swap(next);
        }
        std::sort(halo.begin(), halo.end());
        P.atoms.insert(P.atoms.end(), halo.begin(), halo.end());
        for (int32_t a : P.atoms)
            for (int32_t c : inc[a])
                if (cmark[c] != d && amark[ci[c]] == d && amark[cj[c]] == d) {
                    cmark[c] = d;
                    P.cons.push_back(c);
                }
        std::sort(P.cons.begin(), P.cons.end());
        for (int32_t c : P.cons) P.owned.push_back(part_of[std::min(ci[c], cj[c])] == d ? 1 : 0);
    }
    return D;
}

// One domain's program (see DomProgHeader) appended to `out` (16-byte aligned); false if the
// domain exceeds the 16-bit encoding.  loc: scratch of one entry per molecule atom, all -1.
static bool build_domain_program(const DomainPlan& P, const std::vector<int32_t>& ci, const std::vector<int32_t>& cj,
                                 std::vector<int32_t>& loc, std::vector<uint8_t>& out, int32_t& nlev, int32_t& ntask,
                                 int32_t& nterm, int64_t& n_fill, uint32_t smem[6]) {
    const int32_t na = (int32_t)P.atoms.size(), ne = (int32_t)P.cons.size(), no = P.na_own;
    if (na >= 0xFFFF || ne >= (int32_t)DomTerm::kMaxCons) return false;
    for (int32_t k = 0; k < na; ++k) loc[P.atoms[k]] = k;
    std::vector<int32_t> eci(ne), ecj(ne);
    std::vector<std::vector<int32_t>> ainc(na);
    for (int32_t e = 0; e < ne; ++e) {
        eci[e] = loc[ci[P.cons[e]]];
        ecj[e] = loc[cj[P.cons[e]]];
        ainc[eci[e]].push_back(e);
        ainc[ecj[e]].push_back(e);
    }
    for (int32_t a : P.atoms) loc[a] = -1;
    std::vector<std::vector<int32_t>> adj(ne);
    for (int32_t a = 0; a < na; ++a)
        for (int32_t x : ainc[a])
            for (int32_t y : ainc[a])
                if (x != y) adj[x].push_back(y);
    for (auto& v : adj) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    // elimination order: rounds of independent near-minimum-degree pivots, the slack giving
    // the fewest levels, then the fewest terms
    Program Q;
    int64_t best = -1;
    for (int32_t slack : {2, 3, 4, 6}) {
        Program C = compile(ne, eliminate_rounds(ne, adj, slack, false), eci, ecj, kPartThreads, na);
        const int64_t key = ((int64_t)C.nlevel << 40) + (int64_t)C.terms.size();
        if (best < 0 || key < best) {
            best = key;
            Q = std::move(C);
        }
    }
    const int32_t nt = (int32_t)Q.tasks.size() - 1;
    if (nt >= (int32_t)DomTerm::kMaxSlots || Q.terms.size() >= (size_t)UINT32_MAX) return false;
    for (int32_t t = 0; t < nt; ++t)
        if (Q.tasks[t + 1].tstart - Q.tasks[t].tstart > 255u) return false;
    std::vector<int32_t> pos_of(ne);
    for (int32_t p = 0; p < ne; ++p) pos_of[Q.pos_con[p]] = p;
    int32_t n_inc = 0;
    for (int32_t a = 0; a < no; ++a) n_inc += (int32_t)ainc[a].size();
    const DomProgLayout L = dom_prog_layout(na, no, ne, nt, (uint32_t)Q.terms.size(), Q.nlevel, n_inc);
    const size_t base = out.size();
    out.resize(base + L.bytes, 0);
    uint8_t* d = out.data() + base;
    const DomProgHeader H{(uint32_t)na, (uint32_t)no, (uint32_t)ne, (uint32_t)nt, (uint32_t)Q.terms.size(),
                          (uint32_t)Q.nlevel, (uint32_t)n_inc, 0u};
    std::memcpy(d, &H, sizeof(H));
    auto* lp = reinterpret_cast<uint16_t*>(d + L.lvl_piv);
    auto* lt = reinterpret_cast<uint16_t*>(d + L.lvl_task);
    for (int32_t l = 0; l <= Q.nlevel; ++l) {
        lp[l] = (uint16_t)Q.lvl_piv[l];
        lt[l] = (uint16_t)Q.lvl_task[l];
    }
    auto* lane = reinterpret_cast<uint32_t*>(d + L.lane_term);
    auto* tm = reinterpret_cast<uint32_t*>(d + L.terms);
    size_t o = 0;
    for (int32_t r = 0; r < kPartThreads; ++r) {
        lane[r] = (uint32_t)o;
        for (int32_t l = 0; l < Q.nlevel; ++l)
            for (int32_t t = Q.lvl_task[l] + r; t < Q.lvl_task[l + 1]; t += kPartThreads)
                for (uint32_t k = Q.tasks[t].tstart; k < Q.tasks[t + 1].tstart; ++k)
                    tm[o++] = DomTerm::make(Q.terms[k].l, Q.terms[k].u, Q.terms[k].m);
    }
    auto* pv = reinterpret_cast<uint32_t*>(d + L.piv);
    auto* con = reinterpret_cast<uint32_t*>(d + L.con);
    auto* cml = reinterpret_cast<uint32_t*>(d + L.con_ml);
    for (int32_t p = 0; p < ne; ++p) {
        const int32_t e = Q.pos_con[p];
        pv[p] = (uint32_t)Q.ustart[p] | ((uint32_t)Q.up[p].size() << 16);
        con[p] = (uint32_t)eci[e] | ((uint32_t)ecj[e] << 16);
        cml[p] = (uint32_t)P.cons[e] | (P.owned[e] ? 0x80000000u : 0u);
    }
    std::memcpy(d + L.atom_ml, P.atoms.data(), 4u * (size_t)na);
    auto* ip = reinterpret_cast<uint16_t*>(d + L.inc_ptr);
    auto* iv = reinterpret_cast<uint16_t*>(d + L.inc);
    int32_t k = 0;
    for (int32_t a = 0; a < no; ++a) {
        ip[a] = (uint16_t)k;
        for (int32_t e : ainc[a]) iv[k++] = (uint16_t)(((uint32_t)pos_of[e] << 1) | (ecj[e] == a ? 1u : 0u));
    }
    ip[no] = (uint16_t)k;
    std::vector<int32_t> ord(no);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return ainc[x].size() > ainc[y].size(); });
    auto* ao = reinterpret_cast<uint16_t*>(d + L.aorder);
    for (int32_t a = 0; a < no; ++a) ao[a] = (uint16_t)ord[a];
    auto* tw = reinterpret_cast<uint32_t*>(d + L.tasks);
    for (int32_t t = 0; t < nt; ++t) {
        const TaskW& w = Q.tasks[t];
        const uint32_t a = w.atomsign >> 1;
        const uint32_t ac = (w.row == w.col || a >= (uint32_t)na) ? 0xFFFFu : a;
        tw[2 * t] = w.row | (w.col << 16);
        tw[2 * t + 1] = ac | ((w.atomsign & 1u) << 16) | ((Q.tasks[t + 1].tstart - w.tstart) << 24);
    }
    nlev = Q.nlevel;
    ntask = nt;
    nterm = (int32_t)Q.terms.size();
    n_fill = Q.n_fill;
    smem[2] = dom_state_layout(na, no, ne, nt, 4).bytes;
    smem[3] = dom_state_layout(na, no, ne, nt, 8).bytes;
    smem[5] = dom_state_layout(na, no, ne, nt, 4, true).bytes;
    smem[0] = L.bytes + smem[2];
    smem[1] = L.bytes + smem[3];
    smem[4] = L.bytes + smem[5];
    return true;
}

// The OPM blob of molecule M (OpmBlobHeader, domain offsets, constraint ids, programs) with
// parts of about part_size constraints; false if a domain does not fit the encoding.
static bool build_opm(Program& P, MolHost& M, int32_t part_size, int32_t overlap, int32_t max_parts) {
    const int32_t na = (int32_t)M.atoms.size(), nc = (int32_t)M.cons.size();
    const int32_t n_parts = std::max(2, std::min(max_parts, (nc + part_size - 1) / part_size));
    P.dom_bounds = partition_atoms(na, M.ci, M.cj, n_parts);
    const std::vector<DomainPlan> doms = opm_domains(na, M.ci, M.cj, P.dom_bounds, overlap);
    const int32_t nd = (int32_t)doms.size();
    const uint32_t head = align16((uint32_t)sizeof(OpmBlobHeader) + 4u * (nd + 1));
    const uint32_t progs = align16(head + 4u * (uint32_t)nc);
    P.opm_blob.assign(progs, 0);
    std::vector<uint32_t> off(nd + 1, 0);
    std::vector<int32_t> loc(na, -1);
    P.dom_con_ptr.assign(1, 0);
    P.dom_cons.clear();
    P.dom_owned.clear();
    P.dom_levels.assign(nd, 0);
    P.dom_bytes.assign(nd, 0);
    for (int32_t& v : M.dom_smem) v = 0;
    M.nlevel = M.ntask = M.nterm = 0;
    M.n_fill = 0;
    for (int32_t d = 0; d < nd; ++d) {
        off[d] = (uint32_t)P.opm_blob.size();
        int32_t nl = 0, nt = 0, ntm = 0;
        int64_t fill = 0;
        uint32_t sm[6];
        if (!build_domain_program(doms[d], M.ci, M.cj, loc, P.opm_blob, nl, nt, ntm, fill, sm)) return false;
        P.dom_levels[d] = nl;
        P.dom_bytes[d] = (int32_t)(P.opm_blob.size() - off[d]);
        for (int q = 0; q < 6; ++q) M.dom_smem[q] = std::max<int32_t>(M.dom_smem[q], (int32_t)sm[q]);
        M.nlevel = std::max(M.nlevel, nl);
        M.ntask += nt;
        M.nterm += ntm;
        M.n_fill += fill;
        P.dom_cons.insert(P.dom_cons.end(), doms[d].cons.begin(), doms[d].cons.end());
        P.dom_owned.insert(P.dom_owned.end(), doms[d].owned.begin(), doms[d].owned.end());
        P.dom_con_ptr.push_back((int32_t)P.dom_cons.size());
    }
    off[nd] = (uint32_t)P.opm_blob.size();
    const OpmBlobHeader H{(uint32_t)nd, (uint32_t)overlap, 0u, 0u};
    std::memcpy(P.opm_blob.data(), &H, sizeof(H));
    std::memcpy(P.opm_blob.data() + sizeof(H), off.data(), 4u * (nd + 1));
    std::memcpy(P.opm_blob.data() + head, M.cons.data(), 4u * (size_t)nc);  // global constraint ids
    M.n_dom = nd;
    M.n_seg = nd;
    M.nlevel = std::max(M.nlevel, 1);
    return true;
}

// Kernel cost model (cycles per Newton iteration for one team), with the pass costs
// measured by clock counters in the batched kernel on GB300 (eight teams per SM): a
// factorisation level pass ~1390 cycles, a back-substitution level pass ~620; the work of
// tasks and terms is spread over the team's lanes.
static double program_cost(const Program& P, int32_t team) {
    const double work = (double)P.tasks.size() * 6.0 + (double)P.terms.size() * 4.0;
    return 1390.0 * (double)P.passes_factor + 620.0 * (double)P.passes_solve + work / team;
}

static Program choose_order(int32_t nc, int32_t na, const std::vector<std::vector<int32_t>>& adj,
                            const std::vector<int32_t>& ci, const std::vector<int32_t>& cj,
                            const ilves_setup_opts& o, int32_t team) {
    if (o.ordering == 1) return compile(nc, eliminate_rounds(nc, adj, 0, true), ci, cj, team, na);
    if (o.ordering == 2) return compile(nc, eliminate_rounds(nc, adj, o.degree_slack, false), ci, cj, team, na);
    Program best;
    double best_cost = 1e300;
    const bool big = nc > 4096;
    for (int32_t slack : {0, 1, 2, 3, 5}) {
        if (big && slack != 2) continue;  // large systems: one fixed order keeps setup fast
        Program P = compile(nc, eliminate_rounds(nc, adj, slack, false), ci, cj, team, na);
        const double c = program_cost(P, team);
        if (c < best_cost) {
            best_cost = c;
            best = std::move(P);
        }
    }
    return best;
}

// ------------------------------------------------------------------------------------
// blob writers (16-bit program for warp molecules, 32-bit for large molecules)
// ------------------------------------------------------------------------------------
template <class IdxT>
static ProgLayout layout_for(const MolHost& M) {
    return prog_layout<IdxT>((uint32_t)M.atoms.size(), (uint32_t)M.cons.size(), (uint32_t)M.ntask,
                             (uint32_t)M.nterm, (uint32_t)M.nlevel, (uint32_t)M.n_seg, (uint32_t)M.n_sept,
                             (uint32_t)M.n_cent, sizeof(IdxT) == 4 ? (uint32_t)M.pprog_bytes : 0u);
}

template <class IdxT>
static void write_blob(uint8_t* dst, const MolHost& M, const Program& P) {
    constexpr bool kCompact = sizeof(IdxT) == 2;
    const ProgLayout L = layout_for<IdxT>(M);
    std::memset(dst, 0, L.bytes);
    auto* seg = reinterpret_cast<SegRow*>(dst + L.seg);
    for (int32_t g = 0; g <= P.n_seg; ++g) seg[g] = SegRow{P.seg_piv[g], P.seg_lvl[g], P.seg_atom[g]};
    auto* con = reinterpret_cast<ConA<IdxT>*>(dst + L.con_atoms);
    auto* con_gid = reinterpret_cast<int32_t*>(dst + L.con_gid);
    auto* piv = reinterpret_cast<Piv<IdxT>*>(dst + L.piv);
    auto* lvl_task = reinterpret_cast<IdxT*>(dst + L.lvl_task);
    auto* lvl_piv = reinterpret_cast<IdxT*>(dst + L.lvl_piv);
    auto* inc_ptr = reinterpret_cast<IdxT*>(dst + L.inc_ptr);
    auto* inc = reinterpret_cast<IdxT*>(dst + L.inc);
    auto* terms = reinterpret_cast<typename TermOf<IdxT>::T*>(dst + L.terms);
    const int32_t nc = (int32_t)M.cons.size(), na = (int32_t)M.atoms.size();
    for (int32_t p = 0; p < nc; ++p) {
        const int32_t c = P.pos_con[p];
        con[p].i = (IdxT)M.ci[c];
        con[p].j = (IdxT)M.cj[c];
        con_gid[p] = M.cons[c];
        piv[p].diag = (IdxT)P.ustart[p];
        piv[p].nup = (IdxT)P.up[p].size();
    }
    for (size_t l = 0; l < P.lvl_piv.size(); ++l) {
        lvl_task[l] = (IdxT)P.lvl_task[l];
        lvl_piv[l] = (IdxT)P.lvl_piv[l];
    }
    std::vector<int32_t> cnt(na + 1, 0);
    for (int32_t p = 0; p < nc; ++p) {
        ++cnt[con[p].i + 1];
        ++cnt[con[p].j + 1];
    }
    for (int32_t a = 0; a < na; ++a) cnt[a + 1] += cnt[a];
    for (int32_t a = 0; a <= na; ++a) inc_ptr[a] = (IdxT)cnt[a];
    std::vector<int32_t> fillp(cnt.begin(), cnt.end() - 1);
    for (int32_t p = 0; p < nc; ++p) {
        inc[fillp[con[p].i]++] = (IdxT)((uint32_t)p << 1);
        inc[fillp[con[p].j]++] = (IdxT)(((uint32_t)p << 1) | 1u);
    }
    if constexpr (kCompact) {  // the local atom of each atom slot (ascending global order)
        auto* aslot = reinterpret_cast<IdxT*>(dst + L.atom_off);
        for (int32_t a = 0; a < na; ++a) aslot[M.aperm.empty() ? a : M.aperm[a]] = (IdxT)a;
    }
    auto term_of = [&](size_t k) { return TermOf<IdxT>::make(P.terms[k].l, P.terms[k].u, P.terms[k].m); };
    if constexpr (kCompact) {
        // task words; terms thread by thread (thread r of the molecule's team of M.team
        // threads owns t0 + r + M.team k of every level), each thread's terms in level order
        auto* tasks = reinterpret_cast<uint32_t*>(dst + L.tasks);
        auto* lane_term = reinterpret_cast<IdxT*>(dst + L.lane_term);
        const int32_t ntask = (int32_t)P.tasks.size() - 1;
        for (int32_t t = 0; t < ntask; ++t) {
            const TaskW& w = P.tasks[t];
            const uint32_t nt = P.tasks[t + 1].tstart - w.tstart;
            tasks[t] = TaskWord::make(w.row, w.col, w.atomsign >> 1, w.atomsign & 1u, nt);
        }
        size_t o = 0;
        const int32_t nl = (int32_t)P.lvl_task.size() - 1;
        const int32_t team = M.team;
        for (int32_t r = 0; r < team; ++r) {
            lane_term[r] = (IdxT)o;
            for (int32_t l = 0; l < nl; ++l) {
                const int32_t t0 = P.lvl_task[l], t1 = P.lvl_task[l + 1];
                for (int32_t t = t0 + r; t < t1; t += team)
                    for (uint32_t k = P.tasks[t].tstart; k < P.tasks[t + 1].tstart; ++k) terms[o++] = term_of(k);
            }
        }
    } else {
        auto* tasks = reinterpret_cast<Task<IdxT>*>(dst + L.tasks);
        const IdxT no_atom = (IdxT)~(IdxT)0;
        for (size_t t = 0; t < P.tasks.size(); ++t) {
            const TaskW& w = P.tasks[t];
            tasks[t].row = (IdxT)w.row;
            tasks[t].col = (IdxT)w.col;
            tasks[t].atomsign = w.atomsign == kNoAtom32 ? no_atom : (IdxT)w.atomsign;  // sentinel
            tasks[t].tstart = (IdxT)w.tstart;
        }
        for (size_t k = 0; k < P.terms.size(); ++k) terms[k] = term_of(k);
        if (P.n_seg > 1) {
            std::memcpy(dst + L.sep_info, P.sep_info.data(), P.sep_info.size() * sizeof(SepInfo));
            std::memcpy(dst + L.cptr, P.cptr.data(), P.cptr.size() * sizeof(int32_t));
            std::memcpy(dst + L.cent, P.cent.data(), P.cent.size() * sizeof(Contrib));
            if (M.pprog_bytes > 0) {
                std::memcpy(dst + L.pprog_off, P.pprog_off.data(), P.pprog_off.size() * sizeof(uint32_t));
                std::memcpy(dst + L.pprog, P.pprog.data(), P.pprog.size());
            }
        }
    }
}

// Batched molecules: relabel the local atoms in order of decreasing degree (number of
// constraints; ties keep their order), so that the lanes of a warp update atoms with equal
// incidence counts -- the position update's float64 loop then runs no longer than its
// atoms need.  The program's shared atoms follow the new labels; aperm maps them back.
static void relabel_atoms_by_degree(MolHost& M, Program& P) {
    const int32_t na = (int32_t)M.atoms.size(), nc = (int32_t)M.ci.size();
    std::vector<int32_t> deg(na, 0);
    for (int32_t c = 0; c < nc; ++c) {
        ++deg[M.ci[c]];
        ++deg[M.cj[c]];
    }
    M.aperm.resize(na);
    std::iota(M.aperm.begin(), M.aperm.end(), 0);
    std::stable_sort(M.aperm.begin(), M.aperm.end(), [&](int32_t a, int32_t b) { return deg[a] > deg[b]; });
    std::vector<int32_t> inv(na);
    for (int32_t a = 0; a < na; ++a) inv[M.aperm[a]] = a;
    for (int32_t c = 0; c < nc; ++c) {
        M.ci[c] = inv[M.ci[c]];
        M.cj[c] = inv[M.cj[c]];
    }
    for (TaskW& w : P.tasks) {
        const uint32_t a = w.atomsign >> 1;
        if (w.atomsign != kNoAtom32 && a < (uint32_t)na) w.atomsign = ((uint32_t)inv[a] << 1) | (w.atomsign & 1u);
    }
}

// true if a program fits the compact (warp) encoding: task words hold at most
// TaskWord::kMaxTerms terms, term and slot indices fit their fields
static bool fits_compact(const Program& P) {
    if (P.tasks.size() >= kCompactMaxSlots || P.terms.size() > kCompactMaxTerms) return false;
    for (size_t t = 0; t + 1 < P.tasks.size(); ++t)
        if (P.tasks[t + 1].tstart - P.tasks[t].tstart > TaskWord::kMaxTerms) return false;
    return true;
}

// ------------------------------------------------------------------------------------
// planning entry points (used by the C ABI in solve.cu)
// ------------------------------------------------------------------------------------
ilves_status plan_topology(ilves_topology* T, int32_t n_atoms, int32_t n_c, const int32_t* ai,
                           const int32_t* aj, const ilves_setup_opts& o) {
    T->n_atoms = n_atoms;
    T->n_c = n_c;
    for (int32_t k = 0; k < n_c; ++k) {
        if (ai[k] < 0 || ai[k] >= n_atoms || aj[k] < 0 || aj[k] >= n_atoms || ai[k] == aj[k])
            return ILVES_ERR_TOPOLOGY;
    }
    {
        std::vector<uint64_t> keys(n_c);
        for (int32_t k = 0; k < n_c; ++k) {
            const uint64_t a = (uint64_t)std::min(ai[k], aj[k]), b = (uint64_t)std::max(ai[k], aj[k]);
            keys[k] = (a << 32) | b;
        }
        std::sort(keys.begin(), keys.end());
        for (int32_t k = 1; k < n_c; ++k)
            if (keys[k] == keys[k - 1]) return ILVES_ERR_TOPOLOGY;
    }
    // connected components; the root of each is its smallest atom
    std::vector<int32_t> par(n_atoms);
    std::iota(par.begin(), par.end(), 0);
    for (int32_t k = 0; k < n_c; ++k) {
        const int32_t a = uf_find(par, ai[k]), b = uf_find(par, aj[k]);
        if (a != b) par[std::max(a, b)] = std::min(a, b);
    }
    std::vector<char> used(n_atoms, 0);
    for (int32_t k = 0; k < n_c; ++k) used[ai[k]] = used[aj[k]] = 1;
    std::vector<int32_t> mol_of_root(n_atoms, -1);
    int32_t n_mol = 0;
    for (int32_t a = 0; a < n_atoms; ++a) {
        if (!used[a]) {
            T->free_atoms.push_back(a);
            continue;
        }
        const int32_t r = uf_find(par, a);
        if (mol_of_root[r] < 0) mol_of_root[r] = n_mol++;
    }
    T->mols.assign(n_mol, MolHost{});
    for (int32_t a = 0; a < n_atoms; ++a)
        if (used[a]) T->mols[mol_of_root[uf_find(par, a)]].atoms.push_back(a);
    for (int32_t k = 0; k < n_c; ++k) T->mols[mol_of_root[uf_find(par, ai[k])]].cons.push_back(k);
    T->n_mol = n_mol;
    // neighbour table used by the learned warm start's features
    T->con_i.assign(ai, ai + n_c);
    T->con_j.assign(aj, aj + n_c);
    T->nbr.assign((size_t)n_c * 4, -1);
    T->nbr_atom.assign((size_t)n_c * 4, -1);
    {
        std::vector<int32_t> deg(n_atoms + 1, 0);
        for (int32_t k = 0; k < n_c; ++k) {
            ++deg[ai[k] + 1];
            ++deg[aj[k] + 1];
        }
        for (int32_t a = 0; a < n_atoms; ++a) deg[a + 1] += deg[a];
        std::vector<int32_t> inc_all(2 * (size_t)n_c), fillp(deg.begin(), deg.end() - 1);
        for (int32_t k = 0; k < n_c; ++k) {  // constraints at each atom, ascending ids
            inc_all[fillp[ai[k]]++] = k;
            inc_all[fillp[aj[k]]++] = k;
        }
        for (int32_t k = 0; k < n_c; ++k) {
            for (int side = 0; side < 2; ++side) {
                const int32_t a = side ? aj[k] : ai[k];
                int32_t slot = 2 * side;
                for (int32_t e = deg[a]; e < deg[a + 1] && slot < 2 * side + 2; ++e) {
                    if (inc_all[e] == k) continue;
                    T->nbr[(size_t)k * 4 + slot] = inc_all[e];
                    T->nbr_atom[(size_t)k * 4 + slot] = a;
                    ++slot;
                }
            }
        }
    }
    std::vector<int32_t> local(n_atoms, -1);
    const int32_t warp_limit = o.max_warp_constraints > 0 ? o.max_warp_constraints : 1024;
    T->progs.assign(n_mol, nullptr);
    // narrow class threshold.  Explicit (narrow_atoms > 0): every batched molecule of at
    // most that many atoms.  Default (0): kDefaultNarrowAtoms, but only for a batch made of
    // such molecules -- at least 90 % of the batched atoms, and more batched molecules than
    // the wide teams the GPU holds (eight per SM) -- where one-warp teams measured faster;
    // on batches of mixed sizes the gain depends on the precision mode (20-200 atoms with
    // one-warp teams up to 60 atoms: 6 % faster in mixed mode, 5 % slower in float64), so
    // there the autotuner decides; a lone molecule finishes sooner on 96 threads.
    int32_t narrow = o.narrow_atoms > 0 ? o.narrow_atoms : -1;
    if (o.narrow_atoms == 0) {
        int64_t batched = 0, small = 0, n_batched = 0;
        for (int32_t m = 0; m < n_mol; ++m) {
            const int64_t na = (int64_t)T->mols[m].atoms.size(), nc = (int64_t)T->mols[m].cons.size();
            if (nc > warp_limit || nc >= (int64_t)kCompactMaxConstraints || na > (int64_t)TaskWord::kMaxAtom) continue;
            batched += na;
            ++n_batched;
            if (na <= kDefaultNarrowAtoms) small += na;
        }
        const int64_t wide_teams = (int64_t)kMaxSlotsPerCta * (T->n_sm > 0 ? T->n_sm : 152);
        if (n_batched > wide_teams && small * 10 >= batched * 9) narrow = kDefaultNarrowAtoms;
    }
    std::vector<std::vector<int32_t>> inc, adj;
    for (int32_t m = 0; m < n_mol; ++m) {
        MolHost& M = T->mols[m];
        const int32_t na = (int32_t)M.atoms.size(), nc = (int32_t)M.cons.size();
        for (int32_t a = 0; a < na; ++a) local[M.atoms[a]] = a;
        M.ci.resize(nc);
        M.cj.resize(nc);
        inc.assign(na, {});
        for (int32_t c = 0; c < nc; ++c) {
            const int32_t k = M.cons[c];
            M.ci[c] = local[ai[k]];
            M.cj[c] = local[aj[k]];
            inc[M.ci[c]].push_back(c);
            inc[M.cj[c]].push_back(c);
        }
        adj.assign(nc, {});
        for (int32_t a = 0; a < na; ++a)
            for (int32_t x : inc[a])
                for (int32_t y : inc[a])
                    if (x != y) adj[x].push_back(y);
        for (auto& v : adj) {
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
        }
        M.large = nc > warp_limit || nc >= (int32_t)kCompactMaxConstraints || na > (int32_t)TaskWord::kMaxAtom;
        const int32_t part_min = o.partition_min_constraints > 0 ? o.partition_min_constraints : 4096;
        if (nc >= part_min && o.overlap > 0) {
            // overlapping domains: parts of ~part_size constraints, each domain widened by
            // `overlap` edges; all domains run at once (cooperative launch), so their number
            // and shared memory must fit the device: at most three per SM, each domain's
            // float64-mode state within an SM's share (a domain's program is staged in shared
            // memory too when that also fits, else read from global memory)
            M.large = M.parted = true;
            M.opm = o.overlap;
            Program* P = new Program();
            const int32_t n_sm = T->n_sm > 0 ? T->n_sm : 152;
            int32_t part_size = o.part_constraints > 0 ? o.part_constraints : 256;
            bool ok = false;
            for (int attempt = 0; attempt < 16 && !ok; ++attempt) {
                const int32_t max_parts = o.part_constraints > 0 ? 8192 : 3 * n_sm;
                if (!build_opm(*P, M, part_size, o.overlap, max_parts)) {
                    part_size = std::max(16, part_size * 3 / 4);  // a domain outgrew the encoding
                    continue;
                }
                if (o.part_constraints > 0) {
                    ok = true;
                    break;
                }
                const int32_t per_sm = (M.n_dom + n_sm - 1) / n_sm;
                ok = per_sm <= 3 && (int64_t)per_sm * (M.dom_smem[3] + 1024) <= 233472 &&
                     M.dom_smem[3] <= 232448;
                if (!ok) part_size = part_size * 5 / 4;
            }
            if (ok) {
                M.passes = 0;
                T->progs[m] = P;
                continue;
            }
            // no domain plan fits the device (halos too large for co-resident domains):
            // the molecule takes the Schur-complement path below
            delete P;
            M.opm = 0;
            M.n_dom = 0;
            for (int32_t& v : M.dom_smem) v = 0;
        }
        if (nc >= part_min) {
            // partitioned: parts of ~part_size constraints eliminated first, separators last
            M.large = M.parted = true;
            // automatic part size: about 256 constraints, but never more parts (plus the
            // separator CTA) than three CTAs per SM can keep resident, since the parts of a
            // cooperative launch run at once with their programs in shared memory
            int32_t part_size = o.part_constraints > 0 ? o.part_constraints : 256;
            if (o.part_constraints <= 0) {
                const int32_t max_parts = 3 * (T->n_sm > 0 ? T->n_sm : 152) - 1;
                part_size = std::max(part_size, (nc + max_parts - 1) / max_parts);
            }
            const int32_t n_parts = std::max(2, std::min(8192, (nc + part_size - 1) / part_size));
            std::vector<int32_t> bounds = partition_atoms(na, M.ci, M.cj, n_parts);
            const int32_t np = (int32_t)bounds.size() - 1;
            std::vector<int32_t> part_of(na);
            for (int32_t q = 0; q < np; ++q)
                for (int32_t a = bounds[q]; a < bounds[q + 1]; ++a) part_of[a] = q;
            std::vector<int32_t> seg(nc);
            std::vector<int8_t> stage(nc);
            for (int32_t c = 0; c < nc; ++c) {
                const bool inner = part_of[M.ci[c]] == part_of[M.cj[c]];
                seg[c] = inner ? part_of[M.ci[c]] : np;
                stage[c] = inner ? 0 : 1;
            }
            std::vector<int32_t> seg_atom(bounds);
            seg_atom.push_back(na);  // the separator segment owns no atoms
            // elimination order: rounds of independent pivots of near-minimum degree; the
            // degree slack is tuned per molecule for the fewest levels in the deepest part
            // (every level of a part costs a CTA barrier and a dependent chain, twice per
            // iteration), then the fewest terms
            Program* P = nullptr;
            int64_t best_key = 0;
            for (int32_t slack : {2, 3, 4, 6}) {
                Program C = compile(nc, eliminate_rounds(nc, adj, slack, false, &stage), M.ci, M.cj, 256, na, &seg,
                                    np + 1, &seg_atom);
                int32_t deepest = 0;
                for (int32_t q = 0; q < np; ++q) deepest = std::max(deepest, C.seg_lvl[q + 1] - 1 - C.seg_lvl[q]);
                const int64_t key = ((int64_t)deepest << 40) + (int64_t)C.terms.size();
                if (!P || key < best_key) {
                    delete P;
                    P = new Program(std::move(C));
                    best_key = key;
                }
            }
            M.n_seg = np + 1;
            M.n_sept = (int32_t)P->sep_info.size();
            M.n_sep = nc - P->seg_piv[np];
            for (int32_t q = 0; q < np; ++q) {
                M.part_na = std::max(M.part_na, P->seg_atom[q + 1] - P->seg_atom[q]);
                M.part_np = std::max(M.part_np, P->seg_piv[q + 1] - P->seg_piv[q]);
                M.part_nt = std::max(M.part_nt, P->lvl_task[P->seg_lvl[q + 1] - 1] - P->lvl_task[P->seg_lvl[q]]);
            }
            M.n_cent = (int32_t)P->cent.size();
            // segment programs: the parts' (all or none), then the separator block's
            if (!build_part_programs(*P, na, M.ci, M.cj)) {
                P->pprog.clear();
                P->pprog_off.assign(np + 1, 0u);
                P->pprog_max = 0;
            }
            build_sep_program(*P, nc);
            M.pprog_bytes = (int32_t)P->pprog.size();
            M.pprog_max = (int32_t)P->pprog_max;
            M.sprog_bytes = (int32_t)(P->pprog_off[np + 1] - P->pprog_off[np]);
            M.sep_interior = P->sep_interior;
            M.nlevel = P->nlevel;
            M.ntask = (int32_t)P->tasks.size() - 1;
            M.nterm = (int32_t)P->terms.size();
            M.n_fill = P->n_fill;
            M.passes = P->passes_factor + P->passes_solve;
            T->progs[m] = P;
            continue;
        }
        M.team = (!M.large && na <= narrow) ? kNarrowThreads : kSlotThreads;
        Program* P = new Program(choose_order(nc, na, adj, M.ci, M.cj, o, M.large ? 1024 : M.team));
        if (!M.large && !fits_compact(*P)) {
            M.large = true;
            M.team = kSlotThreads;
            *P = choose_order(nc, na, adj, M.ci, M.cj, o, 1024);
        }
        if (!M.large) relabel_atoms_by_degree(M, *P);
        M.nlevel = P->nlevel;
        M.ntask = (int32_t)P->tasks.size() - 1;
        M.nterm = (int32_t)P->terms.size();
        M.n_fill = P->n_fill;
        M.passes = P->passes_factor + P->passes_solve;
        T->progs[m] = P;
    }
    return ILVES_OK;
}

int64_t program_blob_bytes(const ilves_topology* T, int32_t m) {
    const MolHost& M = T->mols[m];
    if (M.opm) return (int64_t)T->progs[m]->opm_blob.size();
    return M.large ? layout_for<uint32_t>(M).bytes : layout_for<uint16_t>(M).bytes;
}

void program_write_blob(const ilves_topology* T, int32_t m, uint8_t* dst) {
    const MolHost& M = T->mols[m];
    if (M.opm)
        std::memcpy(dst, T->progs[m]->opm_blob.data(), T->progs[m]->opm_blob.size());
    else if (M.large)
        write_blob<uint32_t>(dst, M, *T->progs[m]);
    else
        write_blob<uint16_t>(dst, M, *T->progs[m]);
}

void program_export(const ilves_topology* T, int32_t m, int32_t* pos_gid, int32_t* level,
                    int32_t* up_ptr, int32_t* up_idx) {
    const MolHost& M = T->mols[m];
    const Program& P = *T->progs[m];
    const int32_t nc = (int32_t)M.cons.size();
    int32_t e = 0;
    for (int32_t p = 0; p < nc; ++p) {
        if (pos_gid) pos_gid[p] = M.cons[P.pos_con[p]];
        if (level) level[p] = P.level[p];
        if (up_ptr) up_ptr[p] = e;
        for (int32_t q : P.up[p]) {
            if (up_idx) up_idx[e] = q;
            ++e;
        }
    }
    if (up_ptr) up_ptr[nc] = e;
}

void program_export_layout(const ilves_topology* T, int32_t m, int32_t* atom_gid, int32_t* n_parts,
                           int32_t* part_levels, int32_t* part_prog_bytes, int32_t* sep_summary) {
    const MolHost& M = T->mols[m];
    const Program& P = *T->progs[m];
    const int32_t na = (int32_t)M.atoms.size();
    if (atom_gid)
        for (int32_t a = 0; a < na; ++a) atom_gid[a] = M.atoms[M.aperm.empty() ? a : M.aperm[a]];
    if (M.opm) {  // overlapping domains: the domains' levels and program bytes
        const int32_t nd = (int32_t)P.dom_levels.size();
        if (n_parts) *n_parts = nd;
        int32_t mx = 0;
        for (int32_t d = 0; d < nd; ++d) {
            if (part_levels) part_levels[d] = P.dom_levels[d];
            if (part_prog_bytes) part_prog_bytes[d] = P.dom_bytes[d];
            mx = std::max(mx, P.dom_bytes[d]);
        }
        if (sep_summary) {  // no separator block: the domains' shared memory instead
            sep_summary[0] = 0;
            sep_summary[1] = M.dom_smem[0];
            sep_summary[2] = M.dom_smem[3];
            sep_summary[3] = mx;
        }
        return;
    }
    const int32_t np = M.parted ? P.n_seg - 1 : 0;
    if (n_parts) *n_parts = np;
    const bool have_parts = M.parted && P.pprog_max > 0;
    for (int32_t q = 0; q < np; ++q) {
        if (part_levels) part_levels[q] = P.seg_lvl[q + 1] - 1 - P.seg_lvl[q];
        if (part_prog_bytes) part_prog_bytes[q] = have_parts ? (int32_t)(P.pprog_off[q + 1] - P.pprog_off[q]) : 0;
    }
    if (sep_summary) {
        sep_summary[0] = M.parted ? P.seg_lvl[np + 1] - 1 - P.seg_lvl[np] : 0;
        sep_summary[1] = M.parted ? M.sprog_bytes : 0;
        sep_summary[2] = M.parted ? M.sep_interior : 0;
        sep_summary[3] = M.parted ? M.pprog_max : 0;
    }
}

void program_export_domains(const ilves_topology* T, int32_t m, int32_t* n_dom, int32_t* atom_bounds,
                            int32_t* con_ptr, int32_t* con_gid, int32_t* owned) {
    const MolHost& M = T->mols[m];
    const Program& P = *T->progs[m];
    const int32_t nd = M.opm ? (int32_t)P.dom_levels.size() : 0;
    if (n_dom) *n_dom = nd;
    if (!M.opm) return;
    for (int32_t d = 0; d <= nd; ++d) {
        if (atom_bounds) atom_bounds[d] = P.dom_bounds[d];
        if (con_ptr) con_ptr[d] = P.dom_con_ptr[d];
    }
    for (size_t k = 0; k < P.dom_cons.size(); ++k) {
        if (con_gid) con_gid[k] = M.cons[P.dom_cons[k]];
        if (owned) owned[k] = P.dom_owned[k];
    }
}

void free_programs(ilves_topology* T) {
    for (Program* P : T->progs) delete P;
    T->progs.clear();
}

// bytes of one molecule's shared-memory slice for a precision mode
uint32_t footprint(const MolHost& M, int mode) {
    const uint32_t lp = mode == ILVES_PREC_FP64 ? 8u : 4u;
    const ProgLayout L = layout_for<uint16_t>(M);
    const StateLayout S = state_layout((uint32_t)M.atoms.size(), (uint32_t)M.cons.size(), (uint32_t)M.ntask,
                                       lp, mode == ILVES_PREC_MIXED_DF);
    return L.staged + S.bytes;
}

// Slot schedule of the batched kernel.  Molecules of each class (96-thread teams, and the
// narrow class of one-warp teams) are sorted by shared-memory footprint (largest first).
// The smallest ones of a class, holding about kPoolShare of its estimated cost, form the
// class's pool, which every slot of the class draws from at run time once its own queue
// is done; they fill the gaps of the static queues, so slots finish within about one small
// molecule of each other.  The rest is cut into G consecutive queues: a queue takes
// molecules while its estimated cost stays under the per-queue target, and molecules that
// find no queue go to the front of the pool.  Each queue's slot gets a fixed slice sized
// for its first (largest) molecule.  The first k CTAs hold x wide and y narrow slots (96 x
// + 32 y threads at most kSlotCtaThreads), the others only wide slots (as many as the
// options allow): the slots of each class are dealt to the CTAs that take them in snake
// order, so every CTA mixes large and small slices, and (x, y, k) is the triple of least
// estimated time (the slower class's cost over its slots) whose slices fit the arena.
// Slots never wait for each other.
constexpr double kPoolShare = 0.10, kQueueSlack = 1.05;

// estimated cost of one molecule for the schedule (level passes and work of its team)
double schedule_cost(const MolHost& M) {
    return 90.0 * (double)M.passes + (6.0 * M.ntask + 4.0 * M.nterm + 60.0 * M.cons.size()) / 32.0;
}

// Time a one-warp team takes per unit of schedule cost (the cost of its 32-lane program),
// relative to a 96-thread team: calibrated on the 20-200-atom batch (mixed), where 1.2-1.4
// balanced the two classes' end times and gave the fastest launches (1.8 left the one-warp
// slots idle for the last ~25 % of the launch).
constexpr double kNarrowTeamTime = 1.3;

namespace {
struct ClassPlan {
    std::vector<int32_t> sorted;  // the class's molecules, largest footprint first
    std::vector<uint32_t> fp;     // footprint per molecule id
    std::vector<double> cost;     // schedule cost per molecule id
    size_t cut = 0;               // sorted[cut..) is the pool part
    double head_cost = 0.0, total = 0.0;
};
struct ClassSlots {
    std::vector<std::vector<int32_t>> queue;  // per slot
    std::vector<uint32_t> slice;              // per slot
    std::vector<int32_t> pool;
};

ClassPlan class_plan(const ilves_topology* T, int mode, const std::vector<int32_t>& mols) {
    ClassPlan C;
    C.fp.assign(T->n_mol, 0u);
    C.cost.assign(T->n_mol, 0.0);
    for (int32_t m : mols) {
        C.sorted.push_back(m);
        C.fp[m] = footprint(T->mols[m], mode);
        C.cost[m] = schedule_cost(T->mols[m]);
        C.total += C.cost[m];
    }
    std::sort(C.sorted.begin(), C.sorted.end(), [&](int32_t a, int32_t b) {
        return C.fp[a] != C.fp[b] ? C.fp[a] > C.fp[b] : a < b;
    });
    // pool: the longest suffix whose cost stays within kPoolShare of the total
    C.cut = C.sorted.size();
    double pool_cost = 0.0;
    while (C.cut > 0 && pool_cost + C.cost[C.sorted[C.cut - 1]] <= kPoolShare * C.total)
        pool_cost += C.cost[C.sorted[--C.cut]];
    C.head_cost = C.total - pool_cost;
    return C;
}

// The slots of one class for G queues: every non-empty queue, plus pool-only slots (at most
// one per pool molecule), in queue order (largest slices first).
ClassSlots class_slots(const ClassPlan& C, int64_t G) {
    ClassSlots S;
    if (G <= 0 || C.sorted.empty()) return S;
    const double target = C.head_cost / (double)G * kQueueSlack;
    std::vector<std::vector<int32_t>> groups(G);
    int64_t g = 0;
    double acc = 0.0;
    bool full = false;  // every queue closed: the rest joins the pool (it stays the smallest)
    for (size_t k = 0; k < C.cut; ++k) {
        const int32_t m = C.sorted[k];
        if (!full && !groups[g].empty() && acc + C.cost[m] > target) {
            if (g + 1 < G) {
                ++g;
                acc = 0.0;
            } else {
                full = true;
            }
        }
        if (full) {
            S.pool.push_back(m);
            continue;
        }
        groups[g].push_back(m);
        acc += C.cost[m];
    }
    for (size_t k = C.cut; k < C.sorted.size(); ++k) S.pool.push_back(C.sorted[k]);
    const uint32_t pool_fp = S.pool.empty() ? 0u : C.fp[S.pool.front()];
    for (int64_t gi = 0, po = 0; gi < G; ++gi) {
        if (!groups[gi].empty()) {
            S.slice.push_back(C.fp[groups[gi].front()]);
            S.queue.push_back(std::move(groups[gi]));
        } else if (po < (int64_t)S.pool.size()) {
            S.slice.push_back(pool_fp);
            S.queue.emplace_back();
            ++po;
        }
    }
    return S;
}

// n slots dealt to CTAs [0, cap.size()) in snake order (largest slices first, so every CTA
// mixes large and small ones), skipping CTAs that hold cap[c] slots already; false if the
// capacities do not hold them all
bool deal(size_t n, const std::vector<int32_t>& cap, std::vector<std::vector<int32_t>>& out) {
    const int64_t nc = (int64_t)cap.size();
    int64_t room = 0;
    for (int32_t c : cap) room += c;
    if ((int64_t)n > room) return false;
    int64_t p = 0;
    for (size_t si = 0; si < n; ++si) {
        for (;; ++p) {
            const int64_t r = p / nc, k = p % nc, c = (r % 2 == 0) ? k : nc - 1 - k;
            if ((int32_t)out[c].size() < cap[c]) {
                out[c].push_back((int32_t)si);
                ++p;
                break;
            }
        }
    }
    return true;
}
}  // namespace

void build_batched_schedule(ilves_topology* T, int mode, int32_t n_cta, int32_t warps, int32_t arena,
                            HostSchedule& S) {
    std::vector<int32_t> wide, narrow;
    for (int32_t m = 0; m < T->n_mol; ++m) {
        const MolHost& M = T->mols[m];
        if (M.large) continue;
        (M.team == kNarrowThreads ? narrow : wide).push_back(m);
    }
    const ClassPlan CW = class_plan(T, mode, wide), CN = class_plan(T, mode, narrow);
    // candidates: CTAs [0, k) hold x wide and y narrow slots, CTAs [k, n_cta) xmax wide
    // slots only (k = n_cta: every CTA alike); least estimated time first
    struct Cand { int32_t x, y, k; double t; };
    std::vector<Cand> cands;
    const int32_t xmax = wide.empty() ? 0 : std::max(1, std::min(kMaxSlotsPerCta, warps));
    auto est = [&](int64_t w_slots, int64_t n_slots) {
        const double tw = CW.total > 0.0 ? CW.total / (double)std::max<int64_t>(1, w_slots) : 0.0;
        const double tn = CN.total > 0.0 ? CN.total * kNarrowTeamTime / (double)std::max<int64_t>(1, n_slots) : 0.0;
        return std::max(tw, tn);
    };
    if (narrow.empty()) {
        for (int32_t x = 1; x <= xmax; ++x) cands.push_back({x, 0, n_cta, est((int64_t)n_cta * x, 0)});
    } else {
        for (int32_t x = wide.empty() ? 0 : 1; x <= (wide.empty() ? 0 : xmax); ++x) {
            const int32_t ymax = std::min(kNarrowSlotsPerCta, (kSlotCtaThreads - kSlotThreads * x) / kNarrowThreads);
            for (int32_t y = 1; y <= ymax; ++y) {
                const int32_t k0 = (wide.empty() || x == xmax) ? n_cta : 1;
                Cand best{x, y, n_cta, 1e300};
                for (int32_t k = k0; k <= n_cta; ++k) {
                    const double t = est((int64_t)k * x + (int64_t)(n_cta - k) * xmax, (int64_t)k * y);
                    if (t < best.t) best = {x, y, k, t};
                }
                cands.push_back(best);
                if (best.k != n_cta)  // every CTA alike, in case the best split does not fit
                    cands.push_back({x, y, n_cta, est((int64_t)n_cta * x, (int64_t)n_cta * y)});
            }
        }
    }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) {
        if (a.t != b.t) return a.t < b.t;
        return a.x + a.y > b.x + b.y;
    });
    ClassSlots SW, SN;
    std::vector<std::vector<int32_t>> cw(n_cta), cn(n_cta);  // slot indices per CTA
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        const Cand& c = cands[ci];
        std::vector<int32_t> capw(n_cta), capn(n_cta);
        int64_t nw = 0, nn = 0;
        for (int32_t q = 0; q < n_cta; ++q) {
            capw[q] = q < c.k ? c.x : xmax;
            capn[q] = q < c.k ? c.y : 0;
            nw += capw[q];
            nn += capn[q];
        }
        SW = class_slots(CW, nw);
        SN = class_slots(CN, nn);
        for (auto& v : cw) v.clear();
        for (auto& v : cn) v.clear();
        std::vector<int32_t> capk(capn.begin(), capn.begin() + std::max<int32_t>(1, c.k));
        std::vector<std::vector<int32_t>> cnk(capk.size());
        bool fits = deal(SW.slice.size(), capw, cw) && deal(SN.slice.size(), capk, cnk);
        for (size_t q = 0; q < cnk.size(); ++q) cn[q] = cnk[q];
        for (int32_t q = 0; q < n_cta && fits; ++q) {
            uint64_t used = 0;
            for (int32_t si : cw[q]) used += SW.slice[si];
            for (int32_t si : cn[q]) used += SN.slice[si];
            fits = used <= (uint64_t)arena;
        }
        if (fits || ci + 1 == cands.size()) break;
    }
    S = HostSchedule{};
    S.arena = arena;
    S.cta_slot_ptr.assign(1, 0);
    S.slot_ptr.assign(1, 0);
    S.pool_mol = SW.pool;
    S.pool_mol.insert(S.pool_mol.end(), SN.pool.begin(), SN.pool.end());
    S.pool_wide = (int32_t)SW.pool.size();
    int32_t used_cta = 0;
    for (int32_t k = 0; k < n_cta; ++k)
        if (!cw[k].empty() || !cn[k].empty()) used_cta = k + 1;
    for (int32_t k = 0; k < used_cta; ++k) {  // the slot-owning CTAs are a prefix (snake order)
        uint32_t off = 0;
        auto put = [&](const ClassSlots& CS, int32_t si, int32_t team) {
            S.slot_off.push_back((int32_t)off);
            S.slot_bytes.push_back((int32_t)CS.slice[si]);
            S.slot_team.push_back(team);
            off += CS.slice[si];
            S.slot_mol.insert(S.slot_mol.end(), CS.queue[si].begin(), CS.queue[si].end());
            S.slot_ptr.push_back((int32_t)S.slot_mol.size());
        };
        for (int32_t si : cw[k]) put(SW, si, kSlotThreads);
        for (int32_t si : cn[k]) put(SN, si, kNarrowThreads);
        S.cta_slot_ptr.push_back((int32_t)S.slot_off.size());
        S.cta_nwide.push_back((int32_t)cw[k].size());
        S.warps = std::max<int32_t>(S.warps, (int32_t)(cw[k].size() + cn[k].size()));
        S.block_threads =
            std::max<int32_t>(S.block_threads, (int32_t)(kSlotThreads * cw[k].size() + kNarrowThreads * cn[k].size()));
        S.n_slots_wide += (int32_t)cw[k].size();
    }
    S.n_cta = used_cta;
}

}  // namespace ilves
