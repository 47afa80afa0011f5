/*
 * spg.h -- C ABI of libspg: low-energy states of clustered Ising / Potts
 * models on quasi-2D grids by boundary-MPS contraction of the PEPS of their
 * Boltzmann distribution and a merging branch-and-bound (beam) search,
 * following arXiv:2502.02317 (SpinGlassPEPS.jl).
 *
 * Conventions (all entry points):
 *   - return 0 (SPG_OK) on success, a negative SPG_E* code on failure; the
 *     message of the last failure on a context is spg_last_error(ctx);
 *   - every input array is a HOST pointer and is copied during the call;
 *     the caller keeps ownership;
 *   - handles (spg_ctx, spg_problem, spg_result) are owned by the library and
 *     released with the matching *_destroy, which accept NULL;
 *   - energies are exact int64 integers in units of 2^-energy_shift;
 *   - no C++ exception crosses this boundary.
 *
 * The library runs on one CUDA device, on the stream given to spg_create
 * (or a stream it creates).  Solves are enqueued on that stream: spg_solve
 * returns once the work is enqueued; spg_result_get / spg_result_info wait
 * for it.
 */
#ifndef SPG_H
#define SPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPG_OK 0
#define SPG_EINVAL (-1)       /* bad argument, size or structure           */
#define SPG_EINEXACT (-2)     /* J or h not on the 2^-energy_shift grid    */
#define SPG_ENOMEM (-3)       /* host or device allocation failed          */
#define SPG_ECUDA (-4)        /* a CUDA call failed                        */
#define SPG_ETIMEOUT (-5)     /* a bounded device wait ran out             */
#define SPG_ENUMERIC (-6)     /* NaN/Inf or an energy consistency failure  */
#define SPG_EUNSUPPORTED (-7) /* valid input outside the built limits      */

#define SPG_SQUARE 0 /* grid edges: 4-neighbour (square lattice)            */
#define SPG_KING 1   /* grid edges: 8-neighbour (king's graph)              */

#define SPG_FP64 0  /* every contraction, SVD and marginal in FP64          */
#define SPG_MIXED 1 /* FP32 contractions, FP64 marginal normalisation       */

/* SPG_MIXED solves, log Z and marginals run the FP64 path instead when
 * beta times the largest summed span (max - min) of one site's weight
 * tables (local, left, up, anti-diagonal) exceeds this: the product of a
 * site's weight factors may then fall below FP32's normal range (e^-87)
 * for states that matter, whose conditionals would come out as zero.
 * spg_info.precision_used reports it.  (Measured: beta = 4 on Gaussian
 * Chimera cells spans e^-91 .. e^-142, beta = 1 about e^-35.) */
#define SPG_FP32_WEIGHT_SPAN 80.0

/* Built limits (SPG_EUNSUPPORTED beyond them). */
#define SPG_MAX_STATES 256    /* states of one cluster (2^8 spins)          */
#define SPG_MAX_PROJ 16       /* distinct rows/columns of a pairwise table  */
#define SPG_MAX_CHI 64        /* boundary-MPS bond dimension                */
#define SPG_MAX_COLS 128      /* grid columns                               */
#define SPG_MAX_BEAM 4096     /* max_states                                 */

typedef struct spg_ctx spg_ctx;
typedef struct spg_problem spg_problem;
typedef struct spg_result spg_result;

/* Solver parameters (Sec. 3.1 of the paper: MpsParameters(bond_dim,
 * num_sweeps), SearchParameters(max_states, cut_off_prob), MpsContractor(...;
 * beta)).  spg_params_default fills the defaults listed per field. */
typedef struct {
  double beta;         /* inverse temperature, > 0 (default 1)               */
  int32_t chi;         /* boundary-MPS bond dimension (default 16)           */
  int32_t num_sweeps;  /* variational sweeps after each zipper (default 0)   */
  int32_t beam;        /* max_states: partial states kept (default 256)      */
  int32_t precision;   /* SPG_FP64 or SPG_MIXED (default SPG_FP64)           */
  double cut_off_prob; /* drop children with p < c * max p (default 0: off)  */
  int32_t svd_iters;   /* subspace iterations of a large truncation; -1 (the
                          default): 6 in SPG_FP64, 2 in SPG_MIXED (FP32
                          accuracy does not improve beyond 2)                */
  int32_t warm_start;  /* 1: start the variational compression of every
                          boundary row from the network attached with
                          spg_set_warm_start instead of the SVD zipper (which
                          stays the fallback for rows the network does not
                          cover); needs num_sweeps >= 1 (default 0: off)    */
  uint64_t seed;       /* seed of the truncation's start block (default 0)   */
  int32_t merge;       /* 1: merge branches equal on the boundary of the
                          explored region (merge_branches; default 1)        */
  int32_t fp64_rows;   /* SPG_MIXED: the truncations of the boundary MPSs of
                          rows 1 .. fp64_rows (the final rows of the bottom-up
                          sweep; also row 0, which only spg_log_partition
                          builds, when fp64_rows >= 1) run in FP64 on the
                          FP32 zipper matrices: the left-canonical QR of the
                          MPS below, the QRs and the Jacobi SVD; results are
                          rounded back to FP32.  0: none; -1 (the default):
                          every row of problems with at most
                          SPG_FP64_ROWS_AUTO_SITES sites, none above.
                          Ignored in SPG_FP64.                              */
  int32_t check_fp64;  /* SPG_MIXED, 1: after the search, compare the
                          log-conditionals of every returned state along its
                          path (teacher-forced, site by site) with those from
                          plain FP64 boundary MPSs; the largest difference is
                          the result's max_logmarg_err.  Costs a plain FP64
                          boundary phase per solve (default 0: off).        */
  int32_t droplet_hamming; /* droplets (below): a candidate excitation is
                              kept when it differs from the state and from
                              every droplet kept so far in more than this
                              many Potts variables (default 0)              */
  double droplet_energy;   /* droplets (SingleLayerDroplets, Sec. 2 and 3.1):
                              energy cutoff of the low-energy excitations
                              collected in the merges, in the units of J
                              (multiplied by 2^energy_shift and rounded
                              down); < 0 (the default -1): no droplets      */
  int32_t group_max;       /* spg_solve_batch: most items solved in lockstep
                              as one group (spg_solve_group); 0: automatic
                              (one per SM, within half the free device
                              memory), 1: every item on its own            */
  int32_t reserved;        /* must be 0                                      */
} spg_params;

/* Droplets kept per partial configuration (SPG_EUNSUPPORTED-free: a state
 * whose list would grow beyond this keeps its first SPG_MAX_DROPLETS in the
 * acceptance order and the result's info reports droplet_overflow). */
#define SPG_MAX_DROPLETS 16

/* fp64_rows = -1 truncates every row in FP64 on problems of at most this
 * many sites: there the truncations are often near-exact (chi close to the
 * cut's rank), the discarded directions sit at the FP32 noise floor and an
 * FP32 truncation rotates noise into the kept ones; FP64 rows cost little
 * on such lattices and much on large ones, where truncation error
 * dominates. */
#define SPG_FP64_ROWS_AUTO_SITES 64

/* Per-result diagnostics. */
typedef struct {
  int32_t n_states;        /* states returned                               */
  int32_t near_ties;       /* prune steps whose cut fell within 1e-9 in log p */
  int32_t degenerate_cuts; /* truncations whose cut fell in a degenerate gap */
  int32_t error_flags;     /* device-side checks that failed (0 = none)     */
  double ms_boundary;      /* device time of the boundary-MPS phase (GPU
                              global timer at the phase's ends)              */
  double ms_search;        /* device time of the search phase (same timer)   */
  double candidates;       /* sum over sites of (live beam x states)         */
  double boundary_lognorm; /* log-norm of the last boundary MPS built        */
  int64_t kernel_launches; /* CUDA kernels this solve enqueued              */
  int32_t jacobi_sweeps_max; /* most sweeps one small Jacobi SVD needed (cap 60) */
  int32_t fp64_rows;       /* boundary rows truncated in FP64 (SPG_MIXED)    */
  int32_t precision_used;  /* SPG_FP64 when an SPG_MIXED solve ran the FP64
                              path because its weights exceed FP32's range
                              (see SPG_FP32_WEIGHT_SPAN), else as asked     */
  int32_t droplet_overflow; /* droplet candidates not considered or not kept
                              because a list was full (0: the droplets are
                              those of an unbounded list)                   */
  double max_logmarg_err;  /* check_fp64: max over returned states and sites
                              of |log p_mixed - log p_FP64| / max(1,
                              |log p_FP64|) of the state's own conditional;
                              0 in SPG_FP64; NaN when not checked           */
  int32_t group_size;      /* instances of the lockstep group the solve ran
                              in (1: alone); kernel_launches and the phase
                              times are the group's                          */
  int32_t reserved;
} spg_info;

/* Library version, major*10000 + minor*100 + patch. */
int spg_version(void);

/* Defaults for every field of *p.  Returns SPG_EINVAL if p is NULL. */
int spg_params_default(spg_params* p);

/* Lattice transformations (Sec. 3.1: the instance solved on every rotation
 * and reflection of its grid).  Transformation k in 0..7 of an R x C grid of
 * clusters: bit 4 transposes (i, j) -> (j, i) (the grid becomes C x R), then
 * bit 1 reverses the rows and bit 2 the columns of the resulting grid; k = 0
 * is the identity.  Writes site_map[s] (R*C entries, caller-owned) = the
 * row-major site of the transformed grid that holds original site s, and the
 * transformed grid's shape (either pointer may be NULL).  Host only, no
 * device needed.  SPG_EINVAL for rows, cols < 1, k outside 0..7 or a NULL
 * site_map. */
int spg_lattice_site_map(int32_t rows, int32_t cols, int32_t k, int32_t* site_map, int32_t* new_rows,
                         int32_t* new_cols);

/* Clustered Hamiltonian on the host: the paper's
 * potts_hamiltonian(ising_graph(inst); spectrum = full_spectrum,
 * cluster_assignment_rule) (Sec. 2, Eq. 1 and 2; Sec. 3.1 and 3.1.1:
 * Sparsity, the large clusters of Pegasus and Zephyr).  Host only, no device
 * and no context.  The spins of each grid cell form one Potts variable with
 * 2^k states, k <= SPG_MAX_HAMILTONIAN_SPINS (more than the solver's
 * SPG_MAX_STATES: spg_problem_ising takes clusters of up to 8 spins); state
 * x = sum_q b_q 2^q over the cluster's spins in ascending index, s = 2b - 1.
 *   local table   E_s[x]: fields and couplings inside cluster s (int64, units
 *                 of 2^-energy_shift);
 *   edge k        one per pair of neighbouring clusters (m < n, row-major;
 *                 edges in ascending (m, n)) with a coupling between them:
 *                 reduced table R[Dm][Dn] (row-major) and projectors Pm[x]
 *                 (d_m states), Pn[y] (d_n states) with
 *                 E_e[x, y] = R[Pm[x]][Pn[y]]; Pm numbers the distinct rows of
 *                 E_e in order of first occurrence (x ascending), Pn the
 *                 columns.  E_e is never formed: it is built over the
 *                 configurations of the spins its couplers touch (at most
 *                 SPG_MAX_HAMILTONIAN_COUPLED per side).
 * Inputs as spg_problem_ising (copied; J, h on the 2^-energy_shift grid, h
 * may be NULL).  Returns SPG_EINVAL (sizes, NULL arrays, clusters or
 * couplings off the grid, couplings between non-neighbouring clusters),
 * SPG_EINEXACT, SPG_EUNSUPPORTED (a cluster or an edge side beyond the
 * limits), SPG_ENOMEM.  The accessors copy into caller arrays, which may be
 * NULL to query sizes first. */
#define SPG_MAX_HAMILTONIAN_SPINS 24
#define SPG_MAX_HAMILTONIAN_COUPLED 12
typedef struct spg_hamiltonian spg_hamiltonian;
int spg_potts_hamiltonian(int32_t n_spins, int32_t n_edges, const int32_t* ei, const int32_t* ej, const double* J,
                          const double* h, const int32_t* cluster_of_spin, int32_t grid_rows, int32_t grid_cols,
                          const int32_t* cluster_row, const int32_t* cluster_col, int32_t energy_shift,
                          int32_t node_type, spg_hamiltonian** out);
/* Number of sites (grid cells) and of edges. */
int spg_hamiltonian_size(const spg_hamiltonian* H, int32_t* n_sites, int32_t* n_edges);
/* States of site s (2^k) and, if E is not NULL, its local table E[states]. */
int spg_hamiltonian_local(const spg_hamiltonian* H, int32_t site, int64_t* n_states, int64_t* E);
/* Edge k: its sites m < n, reduced sizes Dm, Dn and, where not NULL, R
 * [Dm*Dn], Pm [states of m], Pn [states of n]. */
int spg_hamiltonian_edge(const spg_hamiltonian* H, int32_t k, int32_t* m, int32_t* n, int32_t* Dm, int32_t* Dn,
                         int64_t* R, int32_t* Pm, int32_t* Pn);
/* Joint projections of site s = (i, j) for its PEPS tensor (Sec. 2, Fig. 1(c);
 * Sec. 3.1 Sparsity): the classes of equal table rows of a state over a set
 * of its edges, numbered in order of first occurrence (x ascending), one
 * class when the set has no edge:
 *   SPG_CLASS_L: edges to (i, j-1) and (i-1, j-1)   SPG_CLASS_U: (i-1, j)
 *   SPG_CLASS_R: edges to (i, j+1) and (i-1, j+1)   SPG_CLASS_G: (i+1, j+1)
 *   SPG_CLASS_D: edges to (i+1, j-1), (i+1, j) and (i+1, j+1).
 * They are found over the configurations of the spins those edges couple
 * (at most 20, and at most 2^24 key entries: configurations x the edges'
 * row lengths; SPG_EUNSUPPORTED beyond).  Writes the class count and, where
 * not NULL, P[states of s] and reps[class count] (the first state of each
 * class). */
#define SPG_CLASS_L 0
#define SPG_CLASS_U 1
#define SPG_CLASS_R 2
#define SPG_CLASS_D 3
#define SPG_CLASS_G 4
int spg_hamiltonian_classes(const spg_hamiltonian* H, int32_t site, int32_t which, int32_t* n_classes, int32_t* P,
                            int32_t* reps);
/* Class weights of site s at inverse temperature beta: C[h][v][r][d] = sum
 * over the states x with (P_L, P_U, P_R, P_D)(x) = (h, v, r, d) of
 * exp(-beta 2^-energy_shift (E_s[x] - min E_s)) (row-major, NL*NU*NR*ND
 * doubles).  With the Boltzmann factors of the reduced tables this is the
 * whole site tensor: W[l, r, u, d] = sum_{h, v} b_left[l][h] b_up[u][v]
 * C[h][v][r][d] (times the anti-diagonal factor on king's graphs), so no
 * tensor over the 2^k states is formed.  SPG_EINVAL for beta <= 0. */
int spg_hamiltonian_class_weights(const spg_hamiltonian* H, int32_t site, double beta, double* C);
/* The PEPS site tensor of site s = (i, j) at inverse temperature beta (Sec. 2,
 * Fig. 1(b)-(c); the row MPO of the boundary-MPS contraction), assembled from
 * the class weights C and the Boltzmann factors of the reduced tables
 * between class representatives (first states), never from a tensor over the
 * states:
 *   W[(a, g)][(a', g')][u][d] = b_ad[a][u] [g' = P_G(u)]
 *       sum_{h, v} b_left[(a, g)][h] b_up[u][v] C[h][v][a'][d]
 * with a the P_R class of (i, j-1), g the P_G class of (i-1, j-1) (left bond
 * a * G_in + g), a' this site's P_R class and g' the P_G class of (i-1, j)
 * (right bond a' * G_out + g'), u the P_D class of (i-1, j), d this site's
 * P_D class; b_left the factors of the edges to (i, j-1) and (i-1, j-1),
 * b_up of the edge to (i-1, j), b_ad of the edge (i-1, j)-(i, j-1), and
 * P_G(u) the P_G class of the states of class u.  Every weight is shifted by
 * its table's minimum (exp(-beta 2^-shift (E - min E))), so log Z = log of
 * the contracted network - beta 2^-shift (sum of the local tables' and the
 * edges' minima).  A missing neighbour or edge contributes dimension 1 and
 * factors 1.  Writes dims = {DL, DR, DU, ND} and, where not NULL, W
 * (row-major [DL][DR][DU][ND] doubles).  SPG_EINVAL for beta <= 0;
 * SPG_EUNSUPPORTED when the sums exceed 4e9 multiply-adds
 * (DL DU NR ND NL NU). */
int spg_hamiltonian_site_tensor(const spg_hamiltonian* H, int32_t site, double beta, int32_t* dims, double* W);
void spg_hamiltonian_destroy(spg_hamiltonian* H);

/* Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * (may be NULL: the library creates and owns a non-blocking stream).  The
 * context owns its device workspace, grown on demand and reused. */
int spg_create(spg_ctx** out, int device, void* cuda_stream);
/* Releases the context.  Problems, results and networks made through it
 * (including the results of spg_solve_batch) may be destroyed before or
 * after it, in any order: a context destroyed while such handles are alive
 * is released with the last of them (no call other than their destroy may
 * use them after spg_destroy). */
void spg_destroy(spg_ctx* ctx);
const char* spg_last_error(const spg_ctx* ctx);

/* Ising form (Eq. 2): E(s) = sum_e J_e s_ei s_ej + sum_i h_i s_i, s = +-1.
 *   n_spins, n_edges        : sizes; spins are 0 .. n_spins-1
 *   ei, ej, J               : [n_edges] couplings (ei != ej)
 *   h                       : [n_spins] fields, or NULL for h = 0
 *   cluster_of_spin         : [n_spins] cluster id 0 .. n_clusters-1
 *   grid_rows, grid_cols    : the grid; n_clusters = grid_rows * grid_cols
 *   cluster_row, cluster_col: [n_clusters] grid cell of each cluster (one
 *                             cluster per cell)
 *   energy_shift            : J and h must be multiples of 2^-energy_shift
 *                             (else SPG_EINEXACT); energies are integers in
 *                             that unit
 *   node_type               : SPG_SQUARE or SPG_KING; a coupling between
 *                             clusters that are not grid neighbours of that
 *                             type is SPG_EINVAL
 * A cluster's state is x = sum_k b_k 2^k over its spins in ascending index,
 * with s = 2 b - 1 (Sec. 2: clusters become Potts variables).
 * King's graphs (Sec. 2, Fig. 1(b)): diagonal couplings are carried by the
 * PEPS through joint projections of each cluster onto its edges (the
 * boundary-MPS physical index of a cluster is its projection onto all three
 * edges below it; the row MPO's bond pairs the left cluster's projection with
 * the up-left cluster's down-right projection, up to 16 x 16).  A joint
 * projection with more than 16 classes is SPG_EUNSUPPORTED.  Variational
 * sweeps (num_sweeps > 0) contract such sites one up index at a time. */
int spg_problem_ising(spg_ctx* ctx, int32_t n_spins, int32_t n_edges, const int32_t* ei,
                      const int32_t* ej, const double* J, const double* h,
                      const int32_t* cluster_of_spin, int32_t grid_rows, int32_t grid_cols,
                      const int32_t* cluster_row, const int32_t* cluster_col,
                      int32_t energy_shift, int32_t node_type, spg_problem** out);

/* New couplings and fields for an Ising problem (same spins, edge list and
 * clusters as at creation; J [n_edges], h [n_spins] or NULL): the tables
 * are recomputed and written in place of the old ones, so solves captured
 * for this problem replay with the new values (a stream of instances of one
 * structure runs from captured graphs).  Waits for the work already
 * enqueued on the context and its batch workers.  SPG_EUNSUPPORTED (problem
 * unchanged) when the new values change the tables' structure (their
 * distinct rows and columns), SPG_EINEXACT as spg_problem_ising. */
int spg_problem_update_ising(spg_problem* prob, const double* J, const double* h);

/* Potts form (Eq. 1): sites are the grid cells in row-major order.
 *   d        : [rows*cols] states per site
 *   local_E  : concatenated local tables, site by site (sum d entries)
 *   em, en   : [n_edges] grid-neighbour site pairs
 *   pair_E   : concatenated d_em x d_en row-major tables (one per edge;
 *              tables on the same pair are added)
 * All energies are int64 in units of 2^-energy_shift. */
int spg_problem_potts(spg_ctx* ctx, int32_t grid_rows, int32_t grid_cols, const int32_t* d,
                      const int64_t* local_E, int32_t n_edges, const int32_t* em,
                      const int32_t* en, const int64_t* pair_E, int32_t energy_shift,
                      int32_t node_type, spg_problem** out);
void spg_problem_destroy(spg_problem* prob);

/* Grid and per-site sizes of a problem (any pointer may be NULL). */
int spg_problem_shape(const spg_problem* prob, int32_t* rows, int32_t* cols, int32_t* d_per_site);

/* Low-energy spectrum (Sec. 2 and Sec. 3.1 low_energy_spectrum): boundary
 * MPSs bottom-up (zipper + SVD truncation to chi, num_sweeps variational
 * sweeps), then the branch-and-bound search in row-major order keeping
 * `beam` partial states, merging those equal on the boundary of the explored
 * region.  Enqueued on the context's stream; *out is valid at once, its
 * contents after spg_result_get.  The solve is a fixed sequence of kernels
 * for a given (problem, params, workspace): from its second occurrence on a
 * context it is captured into one CUDA graph and replayed (the context keeps
 * the 8 most recent). */
int spg_solve(spg_ctx* ctx, const spg_problem* prob, const spg_params* prm, spg_result** out);

/* Lockstep group: n problems of one structure (same lattice, cluster sizes,
 * projections and energy scale; only the energy values differ) solved with
 * the same parameters as ONE launch sequence, every kernel covering all n
 * instances (each instance's tables, copied from its problem at the call,
 * and workspace sit at a fixed stride in one device block).  A group costs
 * the kernel launches of one solve and its one-CTA kernels (QR, Jacobi)
 * occupy n SMs at once; each result equals that of spg_solve on its problem.
 * Captured into one CUDA graph from the second call with the same first
 * problem, n and parameters, like spg_solve.  n in 1..SPG_MAX_GROUP.
 * SPG_EINVAL when a problem's structure differs from probs[0]'s (or its
 * weights need the FP64 path while probs[0]'s do not, see
 * SPG_FP32_WEIGHT_SPAN); SPG_EUNSUPPORTED with warm_start or check_fp64. */
#define SPG_MAX_GROUP 255
int spg_solve_group(spg_ctx* ctx, int32_t n, const spg_problem* const* probs, const spg_params* prm,
                    spg_result** out);

/* Batching: solve n independent problems concurrently (instances of uneven
 * size, each with its own parameters prms[i]); every problem is solved
 * exactly as by spg_solve.  Items of one structure with equal parameters
 * (see spg_solve_group) are solved in lockstep groups of up to
 * prms[i].group_max (0: automatic); the groups, and the items that fit no
 * group, run on up to 32 worker streams owned by the context (each with its
 * own workspace), enqueued from as many host threads, so that their chains
 * of dependent kernels overlap on the GPU.  The streams only overlap when the process has as many hardware work
 * queues: loading the library sets CUDA_DEVICE_MAX_CONNECTIONS=32 unless it
 * is already set, which takes effect if the process creates its CUDA
 * context afterwards (with CUDA's default of 8 queues, more than 8 solves
 * in flight share queues and serialise).  out: n result handles, each
 * waited for by spg_result_get.  Returns
 * once everything is enqueued; work enqueued later on the context's stream
 * runs after the batch.  On failure no handle is returned. */
int spg_solve_batch(spg_ctx* ctx, int32_t n, const spg_problem* const* probs, const spg_params* prms,
                    spg_result** out);

/* The 8 lattice transformations solved as one batch (Sec. 3.1: the
 * example solves the instance on every rotation and reflection of its grid
 * and keeps the best): transformation k of spg_lattice_site_map applied to
 * the problem as it was given (Ising form: the clusters' grid positions
 * move, spins and couplings stay; Potts form: sites move with their local
 * tables, every pairwise table stays on its renumbered edge), the 8
 * problems solved concurrently as by spg_solve_batch with the same
 * parameters, and the result of the first lowest best energy (ties to the
 * lowest k) returned with its states on the ORIGINAL sites, in that
 * lattice's order (energy, then its own lexicographic order).  best_k
 * (may be NULL): the chosen k; best_per_lattice (may be NULL, 8 entries):
 * every lattice's best energy.  Synchronous.  SPG_EUNSUPPORTED when a
 * transposed grid exceeds SPG_MAX_COLS. */
int spg_solve_lattice8(spg_ctx* ctx, const spg_problem* prob, const spg_params* prm, spg_result** out,
                       int32_t* best_k, int64_t* best_per_lattice);

/* Copy the final states out (waits for the solve).  States are sorted by
 * (energy ascending, state lexicographically ascending).
 *   states         : [n_states x n_sites] cluster states, or NULL
 *   energies_fixed : [n_states] int64 energies, or NULL
 *   energies       : [n_states] the same as double (exact below 2^53), or NULL
 *   log_probs      : [n_states] log of the estimated probability, or NULL
 *   max_logmarg_err: the result's log-marginal error against plain FP64
 *                    (spg_info.max_logmarg_err), or NULL
 * Call first with all arrays NULL to read n_states and n_sites. */
int spg_result_get(spg_result* res, int32_t* n_states, int32_t* n_sites, uint16_t* states,
                   int64_t* energies_fixed, double* energies, double* log_probs, double* max_logmarg_err);
int spg_result_info(spg_result* res, spg_info* info);
/* Droplets of the best returned state (unpack_droplets, Sec. 3.1): the
 * low-energy excitations collected in the merges (params.droplet_energy >=
 * 0 and merge = 1), as full configurations with their exact energies,
 * sorted by (energy, state).  n (<= SPG_MAX_DROPLETS), energies [n] int64,
 * states [n x n_sites]; any pointer may be NULL.  Reading: a partial
 * configuration that loses a merge agrees with the winner on every fixed
 * variable next to the unexplored region, so it is an excitation of the
 * winner, dE = E_loser - E_winner, valid for all the winner's descendants;
 * a winner keeps its parent's droplets and accepts, in (dE, state) order,
 * each loser of its merge class and each loser with one of its own droplets
 * applied, when dE <= droplet_energy and it differs from the winner and from
 * every droplet kept so far in more than droplet_hamming variables. */
int spg_result_droplets(spg_result* res, int32_t* n, int64_t* energies, uint16_t* states);

/* Diversity of a set of solutions (Fig. 3 (c), (f)): how many solutions lie
 * within approximation ratio a_r of the best energy and differ pairwise in
 * more than N/2 variables.  Host only.  vars [n x N] (row-major int32: the
 * spins of each solution, or its Potts states; the caller decodes cluster
 * states into spins for a count over spins), energies [n] (int64), e_best:
 * the best energy considered (not necessarily in the set).  Readings: the
 * printed ratio E - E_best < a_r 2 E_best, which no negative E_best meets,
 * is taken as E - E_best < 2 a_r |E_best| (strict); the pairwise condition
 * by first fit: the solutions within the ratio in ascending (energy,
 * lexicographic vars, index) order, each counted when it differs in more than N/2
 * variables (2 d > N) from every one counted before it (the rule of the
 * droplets' Hamming cutoff).  Writes the count and, where not NULL, the
 * counted solutions' indices in counting order (chosen [n]).  SPG_EINVAL for
 * n < 0, N < 1, a_r < 0 or NULL arrays with n > 0. */
int spg_diversity(int32_t n, int32_t N, const int32_t* vars, const int64_t* energies, int64_t e_best, double a_r,
                  int32_t* count, int32_t* chosen);
void spg_result_destroy(spg_result* res);

/* Teacher-forced conditional marginals (Sec. 2, Fig. 1(d)): for each of the
 * n_prefix prefixes (prefixes[k*site .. k*site+site-1] = states of sites
 * 0 .. site-1), log p(x_site | prefix) for every state x of `site`, written
 * to log_marg[k*d_site + x].  Uses the same boundary MPSs (built down to
 * the site's row, in the state a solve leaves them) and environment kernels
 * as spg_solve.  Synchronous. */
int spg_debug_marginals(spg_ctx* ctx, const spg_problem* prob, const spg_params* prm,
                        int32_t site, int32_t n_prefix, const uint16_t* prefixes,
                        double* log_marg);

/* log Z of the problem at prm->beta from the boundary MPSs contracted down
 * to the top row (Sec. 2: approximate contraction of the PEPS).  Exact when
 * no truncation happens.  Synchronous. */
int spg_log_partition(spg_ctx* ctx, const spg_problem* prob, const spg_params* prm,
                      double* log_z);

/* Truncated SVD of one zipper matrix (the SVDTruncate step, Sec. 3.1; the
 * same kernels the zipper uses): for M (m x n, row-major, FP64) return the
 * keep largest singular triplets
 *   V     : n x keep row-major, column k = k-th right singular vector
 *   US    : m x keep row-major, column k = sigma_k times the k-th left one
 *   sigma : keep values, descending
 * All four are DEVICE pointers owned by the caller.  n <= 128 is exact
 * (Jacobi on the QR of M); larger n uses `iters` rounds of subspace
 * iteration on a block of min(n, max(2 keep, keep + 8), 128) columns.
 * Limits: 1 <= m, n <= 16384, 1 <= keep <= min(64, m, n), 0 <= iters <= 64
 * (vectors of 2048 or more entries are orthonormalised by a multi-CTA tall
 * QR).
 * Workspace comes from the context (allocated on first use).  Enqueued on
 * the context's stream; returns after the stream has finished the work. */
int spg_truncate(spg_ctx* ctx, const double* M, int32_t m, int32_t n, int32_t keep, int32_t iters,
                 double* V, double* US, double* sigma);

/* spg_tc_product -- the product step of the FP32 truncated SVD on the
 * tensor cores (Sec. 2 and Sec. 3.1 SVDTruncate: the subspace iteration of
 * the truncation multiplies the zipper matrix M, and its transpose, by the
 * current block of vectors).  All pointers are device pointers:
 *   M    [m x n] row-major FP32 (the zipper matrix)
 *   Bt   [s x K] row-major FP32, K = n when trans == 0, K = m when trans == 1
 *   out  trans == 0: [s x m], out[j][i] = sum_k M[i][k] Bt[j][k]
 *        trans == 1: [s x n], out[j][i] = sum_k M[k][i] Bt[j][k]
 * Each FP32 operand is split into a TF32 high part and its FP32 remainder;
 * three tcgen05 products (hi*hi + hi*lo + lo*hi) accumulate in FP32, which
 * keeps FP32-level accuracy.  This is the path the mixed-precision solve
 * takes for large zipper matrices; it is exported for parity tests and for
 * callers that run their own truncations.  Limits (those of that path): s a
 * multiple of 16 in 16..128, m >= 256, n >= 256, m * n * s >= 2^22, else
 * SPG_EUNSUPPORTED.  Workspace comes from the context; enqueued on the
 * context's stream; returns after the stream has finished the work
 * (SPG_ECUDA with an error flag set if a bounded wait in the kernel gave up). */
int spg_tc_product(spg_ctx* ctx, const float* M, int32_t m, int32_t n, const float* Bt, int32_t s, int32_t trans,
                   float* out);

/* spg_truncate_static -- the truncation of spg_truncate for callers that
 * cannot allocate device memory.  The paper has no counterpart: it is an
 * interface addition of this library.
 *
 * Who needs it: code whose device memory is all owned by its own pool
 * allocator (a framework's caching allocator or an arena reserved at
 * start-up, which leaves nothing to allocate and may forbid raw cudaMalloc),
 * latency-critical loops that cannot pay the device synchronisation an
 * allocation may cause, and plug-ins that may not grow their host's device
 * footprint after initialisation.  This entry point calls no cudaMalloc,
 * cudaFree or other allocating routine; it needs no spg_ctx.
 *
 * Scratch: one fixed array of SPG_TRUNC_STATIC_SCRATCH_BYTES compiled into
 * the library; every GPU on which the library is loaded holds it until the
 * process exits.  Hence the limits m, n <= SPG_TRUNC_STATIC_MAX_DIM and
 * keep <= SPG_TRUNC_STATIC_MAX_KEEP; a larger call returns
 * SPG_EUNSUPPORTED without touching the device.  All calls share the array
 * and it keeps the last call's contents: calls whose work overlaps on the
 * GPU (two streams, or two host threads) race and give wrong results, so
 * serialise them.  The first call on a device (that device current) looks
 * up the array's device address once and caches it; make that first call
 * before any stream capture.
 *
 * Arguments as spg_truncate (M, V, US, sigma are DEVICE pointers owned by
 * the caller), on the current device; cuda_stream is a cudaStream_t (NULL:
 * the legacy default stream).  Returns after the stream has finished the
 * work (it waits for the stream), so a stream that is being captured is
 * rejected with SPG_EINVAL before anything is enqueued on it.  SPG_EINVAL
 * for NULL pointers or inconsistent sizes, SPG_ECUDA if a CUDA call fails. */
#define SPG_TRUNC_STATIC_MAX_DIM 256
#define SPG_TRUNC_STATIC_MAX_KEEP 32
#define SPG_TRUNC_STATIC_SCRATCH_BYTES 1181696 /* 147712 doubles, 1.13 MiB */
int spg_truncate_static(const double* M, int32_t m, int32_t n, int32_t keep, int32_t iters, double* V,
                        double* US, double* sigma, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned warm start of the variational compression.  The paper compresses
 * every boundary MPS by num_sweeps variational sweeps started from the SVD
 * zipper (Sec. 3.1, MpsParameters(bond_dim, num_sweeps)).  The warm start
 * predicts the starting MPS of row r from the couplings near that row with a
 * small MLP trained on the boundary MPSs this library itself produces; the
 * sweeps then refine it.  The paper has no learned part: these calls are
 * an addition of this library, and the zipper remains the default.
 * ------------------------------------------------------------------------ */

/* Inputs of the network for the sites of boundary row `row` of an Ising
 * problem (clusters of <= 8 spins): out[j*SPG_WS_FEATURES + f], host array
 * of cols * SPG_WS_FEATURES floats owned by the caller.  For every cluster
 * (i, k) with i in row .. row+2 and k in j-2 .. j+2 (zeros outside the
 * grid), i outer, SPG_WS_PER_CLUSTER numbers: the couplings between the
 * cluster's spin positions q1 < q2 (28 slots in lexicographic order; the
 * position of a spin is its rank in the cluster, the order of the state
 * encoding), the fields of the 8 positions, and per position the summed
 * couplings to the cluster below (8) and to the cluster on the right (8).
 * Then j == 0, j == cols-1, j == 1, j == cols-2, min(rows - row, 8) / 8,
 * then zeros.  Host only.  SPG_EUNSUPPORTED for Potts problems. */
#define SPG_WS_FEATURES 800
#define SPG_WS_PER_CLUSTER 52
int spg_warm_features(const spg_problem* prob, int32_t row, float* out);

/* The boundary MPS B_row that the method builds (the zipper, then
 * prm->num_sweeps sweeps, at prm's precision), written to the DEVICE array
 * out: cols sites, each padded to [16][chi][chi] (entry (s, a, a') at
 * (s*chi + a)*chi + a', zeros beyond the site's dims), double in SPG_FP64
 * and float in SPG_MIXED.  fix_signs = 1 negates every left-bond row of
 * site j >= 1 whose largest-magnitude entry (first on ties, entries in
 * (s, a') order) is negative, together with the matching column of site
 * j-1, from the last site down (the same MPS in the sign gauge of the
 * zipper's SVDs).  dims (host, may be NULL): cols x {p, chi_l, chi_r}.
 * 1 <= row < rows; row = 0 exports every row 1 .. rows-1, each as it is
 * finished, to out [rows-1][cols][16][chi][chi] (row r at index r-1) with
 * dims [rows-1][cols][3].  Synchronous. */
int spg_boundary_export(spg_ctx* ctx, const spg_problem* prob, const spg_params* prm, int32_t row,
                        int32_t fix_signs, void* out, int32_t* dims);

/* A three-layer perceptron y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with
 * its training state, on the context's device and stream.  Parameters are
 * one flat FP32 array [W1 (hidden x in) | b1 | W2 (hidden x hidden) | b2 |
 * W3 (out x hidden) | b3], row-major, initialised from seed with
 * uniform(+-1/sqrt(fan_in)) weights and zero biases.  Limits: n_in <= 4096,
 * n_hidden <= 1024, n_out <= 65536. */
typedef struct spg_mlp spg_mlp;
int spg_mlp_create(spg_ctx* ctx, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, spg_mlp** out);
void spg_mlp_destroy(spg_mlp* mlp);
/* Number of parameters; copy them out to / in from host arrays (either may
 * be NULL; a set resets the Adam moments and refreshes the BF16 copy). */
int64_t spg_mlp_num_params(const spg_mlp* mlp);
int spg_mlp_params(spg_mlp* mlp, float* get_host, const float* set_host);
/* Forward pass of n samples: X [n x n_in] -> Y [n x n_out], DEVICE arrays
 * owned by the caller.  bf16 = 1: weights and layer inputs rounded to
 * BF16, products accumulated in FP32 (inference); 0: FP32.  Synchronous. */
int spg_mlp_forward(spg_mlp* mlp, const float* X, int32_t n, float* Y, int32_t bf16);
/* Loss 0.5/n * sum (Y - T)^2 over n samples (X [n x n_in], T [n x n_out],
 * DEVICE) and its gradient, in the flat parameter layout, to grad_host
 * (host array of spg_mlp_num_params floats, may be NULL).  FP32. */
int spg_mlp_loss_grad(spg_mlp* mlp, const float* X, const float* T, int32_t n, double* loss, float* grad_host);
/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr)
 * on minibatches of `batch` samples drawn with replacement from the n
 * samples (X, T as in spg_mlp_loss_grad) by a counter-based hash of
 * (seed, step, slot).  *loss (may be NULL) = the mean minibatch loss of the
 * last min(steps, 50) steps.  FP32.  Synchronous. */
int spg_mlp_train(spg_mlp* mlp, const float* X, const float* T, int64_t n, int32_t batch, int32_t steps, double lr,
                  uint64_t seed, double* loss);

/* Attach a network (n_in = SPG_WS_FEATURES, n_out = 16 * chi * chi) for
 * solves with params.warm_start = 1 on this context (NULL detaches).  The
 * context does not own it; keep it alive while such solves run.  Rows whose
 * sites the network does not cover (another chi, a Potts problem) fall
 * back to the SVD zipper. */
int spg_set_warm_start(spg_ctx* ctx, spg_mlp* mlp);

/* Sweeps to fidelity: build the boundary MPSs of rows rows-1 .. row+1 as a
 * solve does, then start row `row` from the SVD zipper (init = 0) or from
 * the attached network (init = 1) and run n_sweeps single variational
 * sweeps, writing after sweep k (1-based) log_overlap[k-1] =
 * log <phi_k | W psi> with psi = B_{row+1} and phi_k normalised.  init = 2
 * runs both on the same B_{row+1}: the zipper's trace to log_overlap[0 ..
 * n_sweeps), the network's to log_overlap[n_sweeps .. 2 n_sweeps).  The
 * sweeps maximise this overlap, so F_k / F_best = exp(2 (log_overlap[k-1]
 * - best)) is the fidelity relative to the best compression reached.
 * Synchronous. */
int spg_sweep_trace(spg_ctx* ctx, const spg_problem* prob, const spg_params* prm, int32_t row, int32_t init,
                    int32_t n_sweeps, double* log_overlap);

/* Failure detection (no counterpart in the paper).  Every wait inside the
 * library's kernels is bounded: on a timeout the kernel records the event,
 * finishes its copies in flight, releases its tensor memory and returns, and
 * the call or result reports SPG_ETIMEOUT.
 *
 * spg_check_bounded_wait runs that failure path on purpose: one kernel
 * waits `polls` polls on an mbarrier that nothing completes.  Returns
 * SPG_ETIMEOUT (the expected outcome, message in spg_last_error), after
 * which the context stays usable; any other code means the bounded wait
 * did not report its timeout.
 *
 * spg_inject_alloc_failure(after): test hook, process-wide; the (after+1)-th
 * device workspace or problem-table allocation from now on fails as if the
 * device were out of memory (the call returns SPG_ENOMEM); after < 0 turns
 * the hook off.  Host only. */
int spg_check_bounded_wait(spg_ctx* ctx, int64_t polls);
int spg_inject_alloc_failure(int32_t after);

/* Measured ALU peak of the current device (measurement aid, no counterpart
 * in the paper): the fused multiply-add throughput of all SMs, kind 0 FP32,
 * kind 1 FP64, in TFLOP/s (2 flops per FMA), timed with CUDA events on
 * cuda_stream (NULL: the legacy default stream).  Synchronous. */
int spg_peak_probe_stream(void* cuda_stream, int32_t kind, double* tflops);

/* Per-kernel device timing (tracing aid).  spg_profile(ctx, 1) starts
 * recording one CUDA event before every kernel the library launches;
 * spg_profile_report waits for the context's stream and writes a JSON object
 * {"kernel name": [launches, total_ms, algorithmic_flops], ...} (times
 * between consecutive
 * events on the stream; the last kernel of the window is closed by an event
 * recorded in the report call) into json_out (NUL-terminated, truncated to
 * cap bytes), then clears the record.  spg_profile(ctx, 0) stops recording.
 * Recording adds one event per launch; timed runs keep it off. */
int spg_profile(spg_ctx* ctx, int enable);
int spg_profile_report(spg_ctx* ctx, char* json_out, size_t cap);

/* Autotuner of tile shapes (the paper has no counterpart: its package leaves
 * kernel tiling to its tensor libraries).  Three kernels come in variants
 * that differ only in how outputs are spread over threads and blocks and
 * compute every output by the same operations, so that results do not
 * depend on the variant, bit for bit:
 *   k_gemm      (SIMT products of the truncations and sweeps): 1, 2, 4 or 8
 *               outputs per thread along each tile edge (variants 0..3);
 *   k_xgemm     (the sweeps' per-state products): 1, 2 or 4 states per
 *               block (variants 0..2; FP64 up to 2);
 *   k_marginals (mixed mode): the boundary-MPS site staged in shared memory
 *               (variant 0, when it fits) or read through the L1 cache
 *               (variant 1, more warps per SM).
 * Process-wide mode (all contexts and devices):
 *   SPG_TUNE_OFF        the built-in choice everywhere;
 *   SPG_TUNE_ON         (default) the first launch of a shape (kernel, sizes,
 *                       strides, instances of the group, device) on a stream
 *                       that is not being captured runs every valid variant
 *                       three times on the real operands, timed with CUDA
 *                       events on that stream (the host waits for the stream
 *                       there), and keeps the fastest for that launch and all
 *                       later ones of the shape, graph captures included; a
 *                       shape first met inside a capture or while
 *                       spg_profile records keeps the built-in choice until
 *                       an uncaptured launch times it;
 *   SPG_TUNE_FORCE + k  variant k of every tuned kernel (the last valid one
 *                       at or below k), nothing timed: for tests.
 * A solve's first, uncaptured run is where its shapes are timed, so a first
 * solve takes longer with SPG_TUNE_ON.  Graphs already captured keep the
 * variants they were captured with.
 * spg_autotune_set: sets the mode (SPG_EINVAL outside 0 .. SPG_TUNE_FORCE+3),
 *   returns the previous one in *previous (may be NULL).
 * spg_autotune_clear: forgets every timed shape (SPG_EINVAL while another
 *   host thread is timing one).
 * spg_autotune_report: the number of timed shapes and, into text_out
 *   (NUL-terminated, truncated to cap bytes; may be NULL), one line per shape:
 *   "<kernel> dev <d> group <n> shape <sizes...> -> <variant> us <t0> <t1> ..."
 *   (best time of each variant in microseconds, -1 for one that could not
 *   run the shape).  Host only; never fails. */
#define SPG_TUNE_OFF 0
#define SPG_TUNE_ON 1
#define SPG_TUNE_FORCE 2
int spg_autotune_set(int32_t mode, int32_t* previous);
int spg_autotune_clear(void);
int spg_autotune_report(int32_t* n_shapes, char* text_out, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* SPG_H */
