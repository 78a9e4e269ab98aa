/*
 * ilves.h -- C ABI of the GB300 (sm_103a) ILVES-M constraint solver.
 *
 * The library solves, for every molecule (connected component of the constraint
 * graph) of a batch, the per-time-step constraint equations of constrained
 * leap-frog / Verlet molecular dynamics (paper, supplement Sec. 2.3):
 *
 *   find lambda such that  sigma_k(x(lambda)) = |x_i - x_j|^2 - d_k^2 = 0  for all k,
 *   x(lambda) = x_unc - M^-1 G(x_old)^T lambda,
 *
 * with Newton's method (ILVES-M, supplement Sec. 2.3, Newton equations for the
 * constraint equation; supplement Sec. 3):
 *
 *   A(x(lambda_l), x_old) delta_l = sigma(x(lambda_l)),  lambda_{l+1} = lambda_l + delta_l,
 *   A(x, y) = G(x) M^-1 G(y)^T   (supplement Sec. 2.3, definition of A),
 *
 * factorising A with a sparse LU in a fill-reducing elimination order computed
 * once per topology (supplement Sec. 3), until max_k |sigma_k| / d_k^2 <= tol
 * (supplement Sec. 4, stopping rule) or max_iter linear solves.
 *
 * Conventions
 *  - sigma = -2 g with the paper's g_i = (d_i^2 - |q_a - q_b|^2) / 2 (supplement
 *    Sec. 2.2), and h^2 is absorbed into lambda: the paper's multipliers are
 *    lambda_paper = -2 lambda / h^2.  Positions do not depend on the convention.
 *  - x_unc = q_k + h v_{k-1/2} + h^2 M^-1 f_ext(t_k) is the unconstrained update
 *    (supplement Sec. 2.3, Eq. for phi_k); x_old = q_k.
 *  - Atom arrays are (n_atoms, 3) row-major float64 (x, y, z per atom); constraint
 *    arrays have n_constraints entries in the caller's constraint order.
 *  - Molecules are the connected components of the constraint graph, numbered in
 *    increasing order of their smallest atom index.  Atoms in no constraint are
 *    copied from x_unc to x_out unchanged.
 *  - "iterations" of a molecule is the number of linear solves performed.  The
 *    convergence test precedes each solve, so a feasible x_unc needs 0.
 *
 * Memory and errors
 *  - ilves_setup_topology takes HOST arrays and owns every device buffer it
 *    allocates (pattern, schedule, workspace) until ilves_destroy_topology.
 *  - ilves_solve takes DEVICE pointers owned by the caller, allocates nothing and
 *    is stream-ordered on `stream` (a cudaStream_t; NULL = legacy default stream).
 *    It returns after enqueueing the work; results are valid once the stream
 *    reaches that point.
 *  - Return values report argument and launch failures only.  Numerical
 *    failures are reported per molecule in mol_status_out.
 *  - Functions are not thread-safe on the same topology object, and the solves of one
 *    topology must be ordered on one stream (large molecules use the topology's workspace);
 *    solves of different topologies may run concurrently on different streams.
 */
#ifndef ILVES_H
#define ILVES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ilves_topology ilves_topology; /* opaque */

typedef enum {
    ILVES_OK = 0,
    ILVES_ERR_INVALID_ARG = 1, /* NULL pointer, negative size, unknown option */
    ILVES_ERR_TOPOLOGY = 2,    /* index out of range, i == j, duplicate constraint */
    ILVES_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    ILVES_ERR_OOM = 4,         /* device allocation failed during setup */
    ILVES_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    ILVES_ERR_TOO_LARGE = 6    /* the scratch a call needs exceeds the library's static maximum */
} ilves_status;

/* Per-molecule outcome written to mol_status_out. */
typedef enum {
    ILVES_MOL_CONVERGED = 0,      /* max |sigma| / d^2 <= tol */
    ILVES_MOL_MAX_ITER = 1,       /* tolerance not reached in max_iter solves */
    ILVES_MOL_SINGULAR_PIVOT = 2, /* a pivot of the LU vanished (|u_jj| tiny) */
    ILVES_MOL_NONFINITE = 3,      /* a violation became NaN or Inf */
    ILVES_MOL_WAIT_TIMEOUT = 4    /* partitioned solve: a bounded wait for other CTAs gave up;
                                     the molecule's outputs are not valid */
} ilves_mol_status;

/* Arithmetic of a solve.
 *  FP64:     every step in float64 (the plain reference configuration).
 *  MIXED:    Jacobian assembly, LU factorisation and triangular solves in float32;
 *            violations, multiplier accumulation and position updates in float64.
 *            The outer Newton loop acts as iterative refinement.
 *  MIXED_DF: as MIXED, but the float64-class steps run in float-float arithmetic
 *            (unevaluated sums of two float32 words, about 48 significant bits) on
 *            the float32 units, on displacements x - x_unc whose magnitude keeps the
 *            absolute rounding error far below the tolerance.  Inputs and outputs
 *            stay float64. */
typedef enum { ILVES_PREC_FP64 = 0, ILVES_PREC_MIXED = 1, ILVES_PREC_MIXED_DF = 2 } ilves_precision;

/* Method flag, OR-ed into the precision argument of ilves_solve:
 *  ILVES_CHORD selects ILVES-F (supplement Sec. 3, simplified Newton / chord method):
 *  the symmetric matrix A(x_old, x_old) is factorised once per solve and reused by every
 *  iteration, which then only substitutes forward and backward.  Convergence is linear,
 *  so it needs more iterations than ILVES-M (the default, a fresh Newton matrix per
 *  iteration) to reach the same tolerance. */
#define ILVES_CHORD 256

/* Start flag, OR-ed into the precision argument of ilves_solve: the solve computes the
 * diagonal (Jacobi) starting multipliers itself, in its set-up pass, instead of reading
 * lambda0 (which must then be NULL):
 *   lambda0_k = sigma_k(x_unc) / (4 (w_i + w_j) (s_k . r_k)),  s = x_unc,i - x_unc,j,
 *   r = x_old,i - x_old,j,
 * i.e. one Newton step (Sec. 2.3) on the diagonal of A(x_unc, x_old) alone, in float32
 * arithmetic on coordinates rounded to float32; 0 where that quotient is not finite.  The
 * values are the ones ilves_warm_start computes without a network, so the two routes
 * give identical solves; the flag saves that separate pass over the inputs.  The paper
 * starts from lambda0 = 0 (Sec. 2.3); the guess is this library's addition. */
#define ILVES_START_DIAG 512

typedef struct {
    int32_t ordering;        /* 0 = autotuned (default); 1 = minimum degree, one pivot per step;
                                2 = rounds of independent low-degree pivots with `degree_slack` */
    int32_t degree_slack;    /* ordering 2: admit pivots up to min degree + slack per round */
    int32_t warps_per_cta;   /* 0 = autotuned; else 1..8 molecule slots (96-thread teams) per persistent CTA
                                of the 96-thread-team class */
    int32_t ctas_per_sm;     /* 0 = autotuned; else 1..4 */
    int32_t device;          /* CUDA device ordinal the topology lives on (-1 = current device,
                                -2 = plan on the host only: no CUDA call, ilves_solve refused) */
    int32_t max_warp_constraints; /* molecules larger than this use the multi-warp path (0 = auto) */
    int32_t partition_min_constraints; /* molecules with at least this many constraints are
                                          partitioned over many CTAs (0 = 4096) */
    int32_t part_constraints;      /* target constraints per part of a partitioned molecule (0 = 256) */
    int32_t wait_test;             /* testing only (0 in normal use): the grid barriers of partitioned
                                      solves also wait for this many CTAs that do not exist, so every
                                      bounded wait runs out and the molecule reports
                                      ILVES_MOL_WAIT_TIMEOUT; the kernel then returns normally */
    int32_t overlap;               /* partitioned molecules: 0 = exact Newton with a Schur complement
                                      over the separator constraints (default); I > 0 = overlapping
                                      domains (supplement Sec. 3, Overlapping Partitioning Method):
                                      each part's domain adds the atoms within I edges, every domain
                                      solves its own system and keeps its owned constraints'
                                      corrections (quasi-Newton, same root); 1..16.  A molecule whose
                                      domains cannot all be resident at once keeps the Schur path. */
    int32_t narrow_atoms;          /* batched molecules of at most this many atoms are solved by
                                      one-warp teams (up to 24 per persistent CTA, beside its
                                      96-thread teams) instead of 96-thread teams: three small
                                      molecules then share the shared memory and the warps of one
                                      large one; the planner puts them on as many CTAs as balance the
                                      two classes.  0 = automatic (100 atoms when such molecules hold
                                      at least 90 % of the batched atoms and outnumber the 96-thread
                                      teams the GPU holds, else none; ilves_autotune tries other
                                      thresholds), -1 = none, else 1..255 */
} ilves_setup_opts;

/* Fills `opts` with the defaults. */
void ilves_default_opts(ilves_setup_opts* opts);

/* Outcome of ilves_autotune: the set-up options the topology now runs with (`chosen`), how
 * many configurations were timed, and the mean time of one solve (ms, CUDA events) in the
 * chosen configuration and in the one the topology had before tuning. */
typedef struct {
    ilves_setup_opts chosen;
    int32_t candidates;   /* 0: the topology was never tuned */
    float best_ms;
    float before_ms;
} ilves_tuning;

/*
 * Builds the solver's view of a constraint topology (supplement Sec. 3,
 * initialisation): connected components (molecules), the line graph L(G) whose
 * adjacency is the pattern of A, a fill-reducing elimination order per molecule,
 * the symbolic LU pattern with its level schedule, the atom -> constraint
 * incidence, and a work partition of molecules over persistent CTAs.  Everything
 * is uploaded once to the device and reused by every ilves_solve.
 *
 *  n_atoms, n_constraints: sizes (>= 0).
 *  atom_i, atom_j: HOST int32 arrays of n_constraints atom indices, 0 <= i,j < n_atoms,
 *                  i != j, no two constraints on the same unordered pair.
 *  opts: may be NULL (defaults).
 *  out: receives the new topology; *out is NULL on error.
 * Errors: ILVES_ERR_INVALID_ARG, ILVES_ERR_TOPOLOGY, ILVES_ERR_OOM, ILVES_ERR_CUDA.
 */
ilves_status ilves_setup_topology(int32_t n_atoms, int32_t n_constraints, const int32_t* atom_i,
                                  const int32_t* atom_j, const ilves_setup_opts* opts,
                                  ilves_topology** out);

/*
 * One constraint solve for every molecule of the topology (the per-step hot path).
 *
 *  x_old     DEVICE float64 (n_atoms, 3): reference positions q_k (defines G(x_old)).
 *  x_unc     DEVICE float64 (n_atoms, 3): unconstrained update.
 *  inv_mass  DEVICE float64 (n_atoms): 1 / m_a >= 0 (0 = anchored atom).
 *  d         DEVICE float64 (n_constraints): target distances d_k > 0.
 *  tol       relative tolerance on |sigma_k| / d_k^2 (e.g. 1e-12).
 *  max_iter  maximum number of linear solves per molecule (>= 0).
 *  precision one of ilves_precision, optionally OR-ed with ILVES_CHORD and ILVES_START_DIAG.
 *  lambda0   DEVICE float32 (n_constraints) initial multipliers, or NULL for zero (NULL
 *            with ILVES_START_DIAG).
 *  x_out     DEVICE float64 (n_atoms, 3): constrained positions (may alias x_unc).
 *  lambda_out DEVICE float64 (n_constraints): multipliers, or NULL.
 *  iterations_out DEVICE int32 (n_molecules): linear solves per molecule, or NULL.
 *  mol_status_out DEVICE int32 (n_molecules): ilves_mol_status per molecule, or NULL.
 *  stream    cudaStream_t to enqueue on.
 * Every array argument may instead be page-locked HOST memory allocated or registered
 * through CUDA (cudaHostAlloc, cudaMallocHost, cudaHostRegister), whose host address is
 * also its device address: the kernels then read the inputs and write the outputs in
 * place over the host link, overlapped with the solve, with no staging copies (the
 * caller synchronises the stream before reading the outputs).  Pageable host memory is
 * not supported.  The caller owns every buffer; none is retained after the call.
 * The call enqueues only kernel launches, an asynchronous memset and event fork/join
 * between the stream and the topology's side stream, so it can be captured into a CUDA
 * graph (stream capture) after one ordinary call has set the kernels' attributes; each
 * replay solves the inputs then in the captured buffers.
 * Errors: ILVES_ERR_INVALID_ARG (NULL required pointer, bad precision, max_iter < 0,
 *         lambda0 given with ILVES_START_DIAG),
 *         ILVES_ERR_CUDA (launch failure).  Allocates nothing.
 */
ilves_status ilves_solve(ilves_topology* topo, const double* x_old, const double* x_unc,
                         const double* inv_mass, const double* d, double tol, int32_t max_iter,
                         int32_t precision, const float* lambda0, double* x_out,
                         double* lambda_out, int32_t* iterations_out, int32_t* mol_status_out,
                         void* stream);

/*
 * Allocation-free variant of ilves_solve.  The paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory when they solve: for
 * example an MD engine that reserves the device memory pool for its own buffers after
 * start-up, or code that must not call cudaMalloc / cudaFree because those may
 * synchronise the device in the middle of an asynchronous time-stepping pipeline.
 *
 * Semantics, arguments and results are those of ilves_solve.  The difference: the solver
 * state of every molecule that a whole CTA or a cooperative group of CTAs solves (molecules
 * too large for one warp team, partitioned molecules with their Schur contribution slots,
 * and molecules solved by overlapping domains with their positions, corrections and
 * multipliers), and the grid-barrier areas of those solves, live in one file-scope
 * device array of ilves_static_scratch_bytes() bytes (16 MiB) instead of the topology's
 * workspace.  Every GPU that loads the library holds that array until exit.
 *  - The call allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *    It clears the barrier area itself, with an asynchronous memset on the topology's
 *    side stream (a memset, not an allocation).
 *  - ilves_setup_topology still reserves the topology's own workspace (counted by
 *    ilves_topology_device_bytes); this entry point leaves it unused.
 *  - The topology must have been set up on the CURRENT device.  Every call looks up the
 *    array's device address on that device (cudaGetSymbolAddress); the first call on a
 *    device may also load the library's device code, so make it before any stream capture.
 *  - Returns ILVES_ERR_TOO_LARGE, without launching anything, when the topology's
 *    state and barrier areas (ilves_topology_workspace_bytes) exceed the static maximum.
 *  - All calls share the one array.  Each call writes every state location before it
 *    reads it and clears the barrier area, so results do not depend on what an earlier
 *    call left there; but calls that overlap on the GPU (other streams, other threads, or
 *    ilves_solve_static_scratch on two topologies at once) race on the array: serialise them.
 */
ilves_status ilves_solve_static_scratch(ilves_topology* topo, const double* x_old, const double* x_unc,
                                        const double* inv_mass, const double* d, double tol,
                                        int32_t max_iter, int32_t precision, const float* lambda0,
                                        double* x_out, double* lambda_out, int32_t* iterations_out,
                                        int32_t* mol_status_out, void* stream);

/*
 * Measured autotuning of a set-up topology (no counterpart in the paper: the paper tunes
 * nothing at run time).  Re-plans the topology under candidate set-up options, one knob at
 * a time from its current options -- the batched kernel's molecule slots per CTA
 * (warps_per_cta 8, 7, 6), CTAs per SM (1, 2), the elimination order (per-molecule cost
 * model, or rounds with degree slack 1 or 3), the one-warp team class (narrow_atoms -1, 50,
 * 60, 70, 100), and for molecules above the partition
 * threshold the exact Schur complement (overlap 0) or overlapping domains of depth 2, 3, 4
 * or 6 -- times `reps` solves of each on the given inputs (CUDA events on `stream`, after
 * one untimed solve), and keeps the fastest configuration whose solves all converge.  The
 * topology keeps its identity; its programs, schedules and workspace are replaced.
 * Results of the tuned topology meet the same tolerances; they may differ in rounding
 * (another elimination order) and in iteration counts (overlapping domains).
 *  Inputs as for ilves_solve (DEVICE or page-locked host buffers); precision as for
 *  ilves_solve (the mode to tune for);
 *  reps >= 1; out: HOST, may be NULL.
 * Synchronous (it synchronises `stream`); allocates device memory for its own outputs and the
 * candidate topologies, so call it at set-up, not inside a time step or a stream capture.
 * Errors: ILVES_ERR_INVALID_ARG, ILVES_ERR_OOM, ILVES_ERR_CUDA.
 */
ilves_status ilves_autotune(ilves_topology* topo, const double* x_old, const double* x_unc, const double* inv_mass,
                            const double* d, double tol, int32_t precision, int32_t reps, void* stream,
                            ilves_tuning* out);

/* The topology's last tuning (out->candidates == 0 if ilves_autotune never ran on it; the
 * chosen options are then the set-up options). */
ilves_status ilves_topology_tuning(const ilves_topology* topo, ilves_tuning* out);

/* Device memory (bytes) a set-up topology holds: programs, schedules, workspaces. */
int64_t ilves_topology_device_bytes(const ilves_topology* topo);

/* Size in bytes of the static scratch array used by ilves_solve_static_scratch. */
int64_t ilves_static_scratch_bytes(void);

/* Bytes of large-molecule solver state a topology needs (its workspace, or the part of
 * the static scratch array ilves_solve_static_scratch would use). */
int64_t ilves_topology_workspace_bytes(const ilves_topology* topo);

/* ---------------------------------------------------------------------------------
 * Learned warm start.  The paper starts Newton from lambda_0 = 0 (supplement Sec. 2.3);
 * these entry points add a small network that predicts lambda_0 from local geometry.
 * The Newton loop of ilves_solve is unchanged and still decides convergence.
 *
 * Features (16 per constraint k with atoms i, j; s = x_unc,i - x_unc,j,
 * rho = x_old,i - x_old,j, W = w_i + w_j), float32:
 *   f0 = (s.s - d^2)/d^2, f1 = s.rho/d^2 - 1, f2 = (w_i - w_j)/W, f3 = |s - rho|^2/d^2,
 *   and for 4 neighbour slots (line-graph neighbours sharing atom i: slots 0-1, sharing
 *   atom j: slots 2-3, ascending constraint id, missing -> zeros), neighbour l sharing a:
 *   (s_l.s_l - d_l^2)/d_l^2,  s_k(a) s_l(a) s.rho_l/(d d_l),  w_a/W.
 * Target: y = lambda * scale, scale = 4 W s.rho / d^2; lambda_0 = y / scale.
 * Network: 16 -> 128 -> ReLU -> 128 -> ReLU -> 1; bfloat16 inputs and W1, W2 (first
 * hidden layer rounded to bfloat16), float32 accumulation, biases and output layer.
 * Parameters (float32, ILVES_MLP_PARAMS values): W1 [128][16] (out x in), b1[128],
 * W2 [128][128], b2[128], w3[128], b3.
 * ------------------------------------------------------------------------------- */
#define ILVES_MLP_FEATURES 16
#define ILVES_MLP_HIDDEN 128
#define ILVES_MLP_PARAMS 18817

typedef struct ilves_mlp ilves_mlp; /* opaque: parameters, Adam state, activation buffers */

/* Number of float32 parameters (ILVES_MLP_PARAMS). */
int64_t ilves_mlp_param_count(void);

/* Synchronises and reports how many tensor-core waits of this network's kernels gave up
 * (bounded waits; the affected launch stops early, frees its tensor memory and leaves
 * its outputs incomplete).  ILVES_OK if none, ILVES_ERR_TIMEOUT otherwise. */
ilves_status ilves_mlp_check(const ilves_mlp* mlp, int32_t* waits_given_up);

/* Testing only: with on != 0 the network's forward kernels first wait on a tensor-core
 * completion barrier that nothing signals (before any MMA is issued), so the bounded wait
 * runs out, the kernel frees its tensor memory and returns, and ilves_mlp_check reports
 * ILVES_ERR_TIMEOUT.  on = 0 restores normal operation. */
ilves_status ilves_mlp_set_wait_test(ilves_mlp* mlp, int32_t on);

/* Creates a network on the current device with He-uniform weights drawn from `seed` and
 * activation buffers for up to max_batch training rows (allocates device memory). */
ilves_status ilves_mlp_create(int32_t max_batch, uint64_t seed, ilves_mlp** out);
void ilves_mlp_destroy(ilves_mlp* mlp);

/* Copies the float32 parameters from / to HOST memory (synchronous; setting resets Adam). */
ilves_status ilves_mlp_set_params(ilves_mlp* mlp, const float* host_params);
ilves_status ilves_mlp_get_params(const ilves_mlp* mlp, float* host_params);

/* Features (DEVICE float32, n_constraints x 16) and target scales (n_constraints, may be
 * NULL) of every constraint of the topology.  Inputs as for ilves_solve. */
ilves_status ilves_mlp_features(const ilves_topology* topo, const double* x_old, const double* x_unc,
                                const double* inv_mass, const double* d, float* features, float* scale,
                                void* stream);

/* Inference on n feature rows (DEVICE, row-major n x 16, 16-byte aligned): y (n
 * floats).  Runs on the tensor cores (tcgen05); ILVES_ERR_INVALID_ARG if features is
 * not 16-byte aligned. */
ilves_status ilves_mlp_forward(const ilves_mlp* mlp, const float* features, int32_t n, float* y, void* stream);

/* One fused kernel computing features, the network and lambda_0 = y / scale for every
 * constraint (DEVICE float32 lambda0, n_constraints), ready for ilves_solve's lambda0.
 * mlp == NULL gives the diagonal (Jacobi) guess lambda_0 = sigma_0 / A_kk at x_unc. */
ilves_status ilves_warm_start(const ilves_mlp* mlp, const ilves_topology* topo, const double* x_old,
                              const double* x_unc, const double* inv_mass, const double* d, float* lambda0,
                              void* stream);

/* Mean-squared-error gradient (DEVICE float32, ILVES_MLP_PARAMS values, may be NULL)
 * and loss (DEVICE float, may be NULL) on n <= max_batch rows (features 16-byte
 * aligned); parameters unchanged. */
ilves_status ilves_mlp_gradient(ilves_mlp* mlp, const float* features, const float* target, int32_t n,
                                float* grad, float* loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on n <= max_batch
 * rows; the loss before the step goes to loss (DEVICE float, may be NULL). */
ilves_status ilves_mlp_train_step(ilves_mlp* mlp, const float* features, const float* target, int32_t n,
                                  float lr, float* loss, void* stream);

/* Sizes of a topology (any pointer may be NULL):
 *  n_molecules, nnz_factor (entries of L+U including fill, summed over molecules),
 *  max_levels (largest level count of any molecule), n_fill (fill entries),
 *  n_large (molecules on the multi-warp path). */
ilves_status ilves_topology_info(const ilves_topology* topo, int32_t* n_molecules,
                                 int64_t* nnz_factor, int32_t* max_levels, int64_t* n_fill,
                                 int32_t* n_large);

/* Copies per-molecule sizes to HOST arrays of n_molecules entries (any may be NULL):
 * atoms, constraints, levels of the factorisation, and the 0-based global index of
 * the molecule's first (smallest) atom. */
ilves_status ilves_topology_molecules(const ilves_topology* topo, int32_t* atoms,
                                      int32_t* constraints, int32_t* levels, int32_t* first_atom);

/* Symbolic structure of molecule `mol` (HOST arrays; any may be NULL), for checking the
 * planner: pos_gid[p] = global constraint id eliminated at position p (nc entries);
 * level[p] = its level; N+(p) (later neighbours in the filled graph, as positions) is
 * up_idx[up_ptr[p] .. up_ptr[p+1]) with up_ptr of nc+1 entries and up_idx of
 * up_ptr[nc] entries (call once with up_idx = NULL to size it). */
ilves_status ilves_topology_export_molecule(const ilves_topology* topo, int32_t mol, int32_t* pos_gid,
                                            int32_t* level, int32_t* up_ptr, int32_t* up_idx);

/* Overlapping domains of molecule `mol` (supplement Sec. 3, Overlapping Partitioning
 * Method; HOST outputs, any may be NULL; call once with the arrays NULL to size them):
 *  n_dom: number of domains (0 if the molecule is not solved by overlapping domains);
 *  atom_bounds (n_dom + 1): domain d's part owns the molecule's atoms [atom_bounds[d],
 *    atom_bounds[d + 1]) in increasing global order (molecule-local indices);
 *  con_ptr (n_dom + 1): domain d's constraints are con_gid[con_ptr[d] .. con_ptr[d + 1]);
 *  con_gid: global constraint ids of each domain's constraints, increasing;
 *  owned: 1 where the domain owns the constraint (its part holds the constraint's atom of
 *    smaller index), else 0.
 * Errors: ILVES_ERR_INVALID_ARG (NULL topology, mol out of range). */
ilves_status ilves_topology_export_domains(const ilves_topology* topo, int32_t mol, int32_t* n_dom,
                                           int32_t* atom_bounds, int32_t* con_ptr, int32_t* con_gid,
                                           int32_t* owned);

/* Data layout of molecule `mol` as the kernels see it (HOST outputs, any may be NULL), for
 * checking the planner:
 *  atom_gid[a] (n_atoms of the molecule entries): global atom of local atom a -- batched
 *    molecules order their local atoms by decreasing number of constraints;
 *  n_parts: parts of a partitioned molecule (0 otherwise; domains of a molecule solved by
 *    overlapping domains); per part (n_parts entries): part_levels (elimination levels of
 *    the part or domain) and part_prog_bytes (bytes of its shared-memory program; 0 when the
 *    parts run from the global program);
 *  sep_summary[4]: the separator block's levels, its program's bytes, the number of its
 *    terms on interior pivots (read from the parts' global state), and the largest part
 *    program with its scratch area (bytes); for overlapping domains: 0, the largest
 *    domain's shared memory with its program staged (float32 factor), its float64-mode
 *    state alone (bytes), and the largest domain program (bytes).
 * No counterpart in the paper: introspection of this library's planner. */
ilves_status ilves_topology_export_layout(const ilves_topology* topo, int32_t mol, int32_t* atom_gid,
                                          int32_t* n_parts, int32_t* part_levels, int32_t* part_prog_bytes,
                                          int32_t* sep_summary);

/* Host-side plan of the batched kernel's slot schedule for one precision mode
 * (ILVES_PREC_*), as it would be built for a grid of n_cta CTAs with arena_bytes of
 * shared memory each; no device is needed (introspection and tests).  Outputs (any may
 * be NULL): n_slots, pool_n (molecules drawn at run time from the pools); per slot (HOST
 * arrays of n_slots entries; call once with them NULL to size them): slot_cta (CTA of the
 * slot), slot_bytes (its shared-memory slice), slot_queue (number of statically queued
 * molecules), slot_team (threads of its team: 96, or 32 for the narrow class; a CTA's
 * 96-thread slots come first); per molecule (n_molecules entries): mol_slot (slot whose
 * queue holds it, -1 for its class's pool, -2 for molecules off the batched path),
 * mol_bytes (its shared-memory footprint in this mode, 0 off the batched path) and
 * mol_team (threads of the team that solves it, 0 off the batched path); class_info[4]:
 * the 96-thread slots, the 96-thread class's pool molecules, the threads per CTA of the
 * launch and the most slots of one CTA.  No counterpart in the paper: the schedule is this
 * library's batching of independent molecules. */
ilves_status ilves_topology_schedule(const ilves_topology* topo, int32_t precision, int32_t n_cta,
                                     int32_t arena_bytes, int32_t* n_slots, int32_t* pool_n,
                                     int32_t* slot_cta, int32_t* slot_bytes, int32_t* slot_queue,
                                     int32_t* slot_team, int32_t* mol_slot, int32_t* mol_bytes,
                                     int32_t* mol_team, int32_t* class_info);

/* Measures the float64 FMA rate of the current device (GFLOP/s, 2 flops per FMA) with
 * a kernel of eight independent FMA chains per thread over every SM, timed with CUDA events
 * on `stream` (synchronous; allocates and frees a small device buffer).  No counterpart in
 * the paper: the mixed mode keeps violations, multiplier sums and position updates in
 * float64 (supplement Sec. 2.3 quantities), and this rate is their ceiling beside HBM.
 *  iters: FMAs per chain (e.g. 4096).  gflops: HOST output.
 * Errors: ILVES_ERR_INVALID_ARG (NULL gflops, iters < 1), ILVES_ERR_OOM, ILVES_ERR_CUDA. */
ilves_status ilves_measure_fp64_fma(int32_t iters, double* gflops, void* stream);

/* Releases every device and host buffer of the topology (NULL is ignored). */
void ilves_destroy_topology(ilves_topology* topo);

/* Static string naming a status code. */
const char* ilves_status_string(int32_t status);

/* Number of kernel launches the most recent ilves_solve on this topology enqueued. */
int32_t ilves_last_launch_count(const ilves_topology* topo);

#ifdef __cplusplus
}
#endif
#endif /* ILVES_H */
