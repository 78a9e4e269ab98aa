// topology_impl.h -- host-side structures of an ilves_topology (not public ABI).
#pragma once
#include <stdint.h>

#include <vector>

#include "ilves.h"
#include "internal.h"

namespace ilves {

struct TaskW { uint32_t row, col, atomsign, tstart; };
struct TermW { uint32_t l, u, m, pad; };

struct MolHost {
    std::vector<int32_t> atoms;      // global atom ids, ascending
    std::vector<int32_t> cons;       // global constraint ids, ascending (local constraint id order)
    std::vector<int32_t> ci, cj;     // per local constraint: local atom ids
    // batched (compact) molecules: local atom a is atoms[aperm[a]] (local atoms ordered by
    // degree, so a warp's lanes update atoms with the same number of constraints; the
    // kernels reach the inputs and outputs through the atom slots, in the order of atoms);
    // empty = identity
    std::vector<int32_t> aperm;
    bool large = false;
    bool parted = false;  // partitioned: solved by a cooperative multi-CTA launch
    // batched molecules: threads of the team the program is laid out for (kSlotThreads, or
    // kNarrowThreads for the narrow class)
    int32_t team = kSlotThreads;
    int32_t n_seg = 1;
    int32_t nlevel = 0, ntask = 0, nterm = 0, n_fill = 0;
    int32_t n_sept = 0, n_cent = 0;  // partitioned: separator tasks, Schur contribution entries
    int32_t n_sep = 0;               // partitioned: separator constraints
    int32_t part_na = 0, part_np = 0, part_nt = 0;  // partitioned: largest part (atoms, pivots, tasks)
    int32_t pprog_bytes = 0;         // partitioned: bytes of the segment programs
    int32_t pprog_max = 0;           // partitioned: largest part program (bytes; 0 = none)
    int32_t sprog_bytes = 0;         // partitioned: bytes of the separator program (0 = none)
    int32_t sep_interior = 0;        // partitioned: separator terms on interior pivots (read from global)
    int32_t opm = 0;                 // overlapping domains: overlap depth (0 = not solved by domains)
    int32_t n_dom = 0;               // overlapping domains: number of domains (CTAs)
    // overlapping domains: largest shared memory of a domain, program staged + state
    // (float32 / float64 factor), then state only (program read from global memory), then
    // staged and state only in the float-float mode
    int32_t dom_smem[6] = {0, 0, 0, 0, 0, 0};
    int64_t passes = 0;
};

struct Program;  // topology.cpp

// Slot schedule of the batched kernel: CTA c owns slots [cta_slot_ptr[c],
// cta_slot_ptr[c + 1]), the first cta_nwide[c] of them run by 96-thread teams (warps
// 0 .. 3 cta_nwide[c] - 1), the others by one-warp teams (the narrow class, the warps after
// them).  Slot s owns the shared-memory slice at slot_off[s] and solves slot_mol[slot_ptr[s]
// .. slot_ptr[s + 1]) in order, then takes molecules from its class's pool (pool_mol: the
// wide class's pool_wide molecules, then the narrow class's; one atomic ticket each) until
// it is empty.  Pool molecules are the smallest of their class and fit every slice of it.
struct HostSchedule {
    int32_t n_cta = 0, warps = 0, arena = 0;
    std::vector<int32_t> cta_slot_ptr, cta_nwide, slot_ptr, slot_mol, slot_off, slot_bytes, slot_team, pool_mol;
    int32_t n_slots_wide = 0, pool_wide = 0, block_threads = 0;
};

struct DeviceSchedule {
    int32_t n_cta = 0, warps = 0, arena = 0;
    int32_t n_slots = 0, pool_n = 0;                // wide class
    int32_t n_slots_narrow = 0, pool_n_narrow = 0;  // narrow class (its pool follows the wide pool)
    int32_t block_threads = 0;                      // threads per launched CTA
    // launch shape: only the CTAs that own slots (a prefix: slots are dealt from CTA 0), each
    // with the shared memory of its slices -- a topology of a few molecules then occupies a
    // few SMs, and solves of several topologies on different streams run side by side
    int32_t launch_cta = 0, launch_smem = 0;
    int32_t* cta_slot_ptr = nullptr;
    int32_t* cta_nwide = nullptr;
    int32_t* slot_ptr = nullptr;
    int32_t* slot_mol = nullptr;  // index into the small-molecule descriptor array
    int32_t* slot_off = nullptr;
    int32_t* pool_mol = nullptr;
    uint32_t* pool_ctr = nullptr;  // {next ticket, slots done} of the wide, then of the narrow
                                   // pool; zero between launches
};

}  // namespace ilves

struct ilves_topology {
    int32_t n_atoms = 0, n_c = 0, n_mol = 0;
    std::vector<ilves::MolHost> mols;
    std::vector<ilves::Program*> progs;  // owned
    std::vector<int32_t> free_atoms;
    // per global constraint: atoms, and up to 4 line-graph neighbours (2 sharing atom_i,
    // then 2 sharing atom_j; -1 = none) with the global id of the shared atom
    std::vector<int32_t> con_i, con_j, nbr, nbr_atom;
    // device side
    int32_t device = -1;
    bool on_device = false;
    int32_t n_sm = 0;
    ilves::MolDesc* d_desc = nullptr;        // all molecules (small first, then large)
    int32_t n_small = 0, n_large = 0;
    uint8_t* d_blob = nullptr;
    int64_t blob_bytes = 0;
    int32_t* d_atom_gid = nullptr;
    int32_t* d_free_atoms = nullptr;
    int32_t* d_con_i = nullptr;
    int32_t* d_con_j = nullptr;
    int32_t* d_nbr = nullptr;       // n_c x 4
    int32_t* d_nbr_atom = nullptr;  // n_c x 4
    float* d_ws_con = nullptr;      // warm-start workspace: n_c x 8 floats (s, sigma0/d^2, rho, d)
    float* d_ws_atom = nullptr;     // n_atoms floats (inverse masses)
    uint8_t* d_work = nullptr;               // large-molecule numerical state
    int64_t work_bytes = 0;
    ilves::DeviceSchedule sched[3];          // per precision mode
    void* side_stream = nullptr;             // cudaStream_t for the large-molecule kernel
    void* ev_fork = nullptr;
    void* ev_join = nullptr;
    int32_t large_threads = 512;
    std::vector<int32_t> parted_desc;        // descriptor indices of partitioned molecules
    uint8_t* d_sync = nullptr;               // per partitioned molecule: barrier counter + flags
    int64_t sync_bytes = 0;
    std::vector<int32_t> desc_mol;           // molecule id of each descriptor
    int32_t parted_threads = 256;
    int32_t parted_max_ctas = 0;
    int32_t last_launches = 0;
    int32_t wait_test = 0;                   // testing: phantom CTAs the partitioned grid barriers wait for
    std::vector<int32_t> opm_desc;           // descriptor indices of molecules solved by overlapping domains
    ilves_setup_opts opts{};                 // the options the topology was planned with
    ilves_tuning tuning{};                   // the last ilves_autotune (candidates == 0: none)
};

namespace ilves {
ilves_status plan_topology(ilves_topology* T, int32_t n_atoms, int32_t n_c, const int32_t* ai,
                           const int32_t* aj, const ilves_setup_opts& o);
uint32_t footprint(const MolHost& M, int mode);
double schedule_cost(const MolHost& M);
void build_batched_schedule(ilves_topology* T, int mode, int32_t n_cta, int32_t warps, int32_t arena,
                            HostSchedule& S);
int64_t program_blob_bytes(const ilves_topology* T, int32_t m);
void program_write_blob(const ilves_topology* T, int32_t m, uint8_t* dst);
void program_export(const ilves_topology* T, int32_t m, int32_t* pos_gid, int32_t* level,
                    int32_t* up_ptr, int32_t* up_idx);
void program_export_layout(const ilves_topology* T, int32_t m, int32_t* atom_gid, int32_t* n_parts,
                           int32_t* part_levels, int32_t* part_prog_bytes, int32_t* sep_summary);
void free_programs(ilves_topology* T);
void program_export_domains(const ilves_topology* T, int32_t m, int32_t* n_dom, int32_t* atom_bounds,
                            int32_t* con_ptr, int32_t* con_gid, int32_t* owned);
}  // namespace ilves
