/*
 * octofmm.h -- C ABI of the GB300 fast-multipole self-gravity solve.
 *
 * The solve is the gravity half of Octo-Tiger (arXiv 2412.15518): a fast
 * multipole method on an adaptive octree whose every node holds an 8x8x8
 * sub-grid of cells (Sec. 4.3.2), conserving linear momentum and, through a
 * correction term, angular momentum (Sec. 4.3.1), with cell-to-cell
 * interactions taken from a fixed stencil (Sec. 5.5).  The paper states the
 * method in prose only; the operations below are the reading documented with
 * each entry point:
 *
 *   * a leaf cell is a point mass m = rho h^3 at its centre (h = cell side);
 *     phi(x) = -G sum_b m_b / |x - x_b| in free space, self pair excluded;
 *   * moments up to order 3 about each cell's centre of mass;
 *   * two level-L cells at integer offset d are "near" iff |d| <= 1/theta;
 *     a non-near pair interacts at level L iff L = 0 or the parents are near
 *     (multipole-to-local, order 3, plus the angular-momentum correction);
 *     near pairs of two leaf cells interact exactly, near pairs with one
 *     leaf cell interact by multipole at level L, near pairs of two interior
 *     cells descend one level;
 *   * exact degree-3 local-to-local shifts down the tree, then at each leaf
 *     cell phi = L0 + near terms, g = -L1 + a_c + near terms.
 *
 * Conventions for every call:
 *   * return 0 (OT_OK) or a negative OT_ERR_* code; nothing is thrown, no
 *     call traps the GPU; ot_error_string() names each code;
 *   * device buffers are owned by the caller (for instance torch tensors),
 *     must live on the tree's device, hold float64, be 8-byte aligned and
 *     contiguous in the layouts stated below;
 *   * the library owns the tree workspace (moments, expansions, tables,
 *     work lists, CUDA graphs); it allocates device memory only in
 *     ot_build_tree and when a solve first meets a new (theta, precision)
 *     plan; a solve with a known plan allocates nothing;
 *   * work is enqueued asynchronously on the caller's CUDA stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream); the
 *     caller synchronises before reading outputs;
 *   * leaf order is the caller's order; cell (i, j, k) of a leaf's 8^3
 *     sub-grid is at index i + 8 j + 64 k (x fastest);
 *   * calls on one tree must not overlap in time (one stream at a time).
 */
#ifndef OCTOFMM_H
#define OCTOFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OT_OK 0
#define OT_ERR_INVALID_ARG -1    /* bad size, option or theta out of range        */
#define OT_ERR_INVALID_TREE -2   /* leaf out of range, duplicate, overlap, holes  */
#define OT_ERR_NOT_BALANCED -3   /* adjacent leaves differ by more than one level */
#define OT_ERR_BAD_POINTER -4    /* NULL, or not device memory where required     */
#define OT_ERR_BAD_ALIGNMENT -5  /* buffer not 8-byte aligned                     */
#define OT_ERR_CUDA -6           /* a CUDA runtime call failed                    */
#define OT_ERR_TIMEOUT -7        /* a bounded device wait gave up                 */
#define OT_ERR_DEVICE_STATUS -8  /* a kernel latched an error in the status word  */

/* Bits of the device status word (ot_tree_stats.device_status). */
#define OT_STATUS_BAD_INDEX 1    /* a tree lookup a validated tree cannot produce  */
#define OT_STATUS_BAD_ITEM 2     /* reserved: a work item longer than a kernel
                                    stages (no kernel of this version latches it) */
#define OT_STATUS_BAD_DENSITY 4  /* a hydro face state with density <= 0 or NaN    */
#define OT_ERR_NO_MEMORY -9      /* host or device allocation failed              */
#define OT_ERR_WRONG_DEVICE -10  /* buffer on another device than the tree        */
#define OT_ERR_TOO_LARGE -11     /* problem exceeds a fixed-size scratch buffer   */

#define OT_PRECISION_FP64 0      /* every step in FP64                           */
#define OT_PRECISION_FP32_BULK 1 /* the FP32-bulk form: every pair's monopole part
                                    (m_B D^(n)(R), the terms that involve the
                                    source only through its mass, including the
                                    exact near pairs and every leaf-leaf pair),
                                    the angular-momentum correction's sums, the
                                    upward and downward passes and every moment
                                    and expansion sum in FP64; the contractions
                                    of the source's quadrupole and octupole with
                                    the derivative tensors in FP32, summed over
                                    at most 64 pairs and then added to the FP64
                                    sums.  Error vs FP64 <= 1e-6 (relative to
                                    the field's maximum)                       */
#define OT_PRECISION_FP32_WIDE 2 /* a wider FP32 share than the FP32-bulk form:
                                    every per-pair multipole term in FP32 (the
                                    monopole parts, the correction's per-pair
                                    contractions and the far leaf-leaf pairs
                                    too), FP64 exact near pairs, masses, centres
                                    of mass, every moment and expansion sum and
                                    the correction's mass ratio; the products of
                                    the M2M and L2L shifts in FP32, each widened
                                    exactly into an FP64 sum.  Error vs FP64
                                    <= 1e-6 (relative to the field's maximum);
                                    conservation of momentum and angular
                                    momentum to FP32 rounding only            */

typedef struct ot_tree ot_tree; /* opaque, library-owned */

/* Octree description (Sec. 4.3.2).  leaves: host int32 [n_leaf][4] =
 * (L, ix, iy, iz), 0 <= ix, iy, iz < 2^L, 0 <= L <= 15; a level-L node covers
 * origin + [ix, ix+1) * size / 2^L per axis and holds 8^3 cells of side
 * size / (8 * 2^L).  The leaves must tile the cube exactly (a complete octree)
 * and be 2:1 balanced across faces, edges and corners. */
typedef struct {
    double origin[3];
    double size;
    int32_t n_leaf;
    const int32_t* leaves;
} ot_tree_desc;

/* Solve options.  theta: opening parameter of the near test |d| <= 1/theta,
 * 0.3 <= theta <= 1 (default 0.5).  G: gravitational constant (default 1).
 * precision: OT_PRECISION_*.  am_correction: 1 adds the angular-momentum
 * correction (Sec. 4.3.1), 0 leaves it out.  self_term: 1 adds each leaf
 * cell's own uniform-cube self potential -G rho h^2 C at its centre
 * (C = 3 (ln(2 + sqrt 3) - pi/6)); 0 excludes the self pair entirely. */
typedef struct {
    double theta;
    double G;
    int32_t precision;
    int32_t am_correction;
    int32_t self_term;
    int32_t reserved;
} ot_solve_opts;

#define OT_MAX_LEVELS 16

/* Counts of a tree and of its current plan (theta, precision). */
typedef struct {
    int32_t n_levels;                          /* Lmax + 1                          */
    int32_t n_leaf;
    int64_t n_nodes[OT_MAX_LEVELS];            /* nodes per level                   */
    int64_t n_leaf_nodes[OT_MAX_LEVELS];       /* leaf nodes per level              */
    int64_t n_m2l;                             /* directed far multipole pairs      */
    int64_t n_p2p;                             /* directed exact near leaf pairs    */
    int64_t n_seam;                            /* directed near leaf/interior pairs */
    int64_t n_lattice;                         /* far pairs of two leaf cells       */
    int64_t n_m2p;                             /* pairs: interior source, leaf target */
    int64_t n_p2m;                             /* pairs: leaf source, interior target */
    int64_t n_mm;                              /* pairs: two interior cells         */
    double flops_am;                           /* algorithmic flops of one interaction
                                                  launch with the correction (fma = 2) */
    double flops_noam;                         /* the same without the correction    */
    double flops_near;                         /* part of either kept in FP64 by the
                                                  wide FP32 form (exact near pairs)  */
    int64_t n_work_items;                      /* items of the persistent launch    */
    int32_t tuned_chunk;                       /* stencil entries per work item     */
    int32_t tuned_ctas_per_sm;                 /* persistent CTAs per SM            */
    int32_t tuned_warps_per_cta;
    int32_t tuned_lattice_ctas_per_sm;         /* wide FP32 form: persistent CTAs per
                                                  SM of each lattice kernel (0: one
                                                  CTA per leaf node)                 */
    int32_t device_status;                     /* latched device errors, 0 = none;
                                                  reading it clears it.  Bits: 1 a
                                                  tree lookup a valid tree cannot
                                                  produce, 2 reserved (a work item
                                                  longer than a kernel stages; no
                                                  kernel of this version stages a
                                                  bounded number), 4 a hydro state
                                                  with a density <= 0 (or NaN)      */
    int64_t workspace_bytes;                   /* device memory held by the tree    */
    double flops_bulk64;                       /* FP32-bulk form, one interaction
                                                  launch with the correction: FP64
                                                  flops (monopole parts, correction
                                                  sums, every leaf-leaf pair)        */
    double flops_bulk32;                       /* ... and its FP32 flops (source
                                                  quadrupole/octupole contractions) */
    double flops_adjoint;                      /* FP64 flops of one reverse sweep of
                                                  the interactions (with the
                                                  correction), counted like flops_am */
    double flops_tangent;                      /* FP64 flops of the tangent solve's
                                                  interactions (dual numbers: value
                                                  and tangent, with the correction) */
} ot_tree_stats;

/* Builds the octree, its level tables, neighbour tables, stencils and work
 * lists (host), and uploads them to `device`.  Defining passage: Sec. 4.3.2
 * (an adaptive octree whose every node holds an 8x8x8 sub-grid of cells) and
 * Sec. 5.5 (a fixed stencil of cell-to-cell interactions instead of
 * interaction lists; structure-of-arrays data).  device = -1 validates and
 * counts on the host only (no CUDA call; solves then fail with
 * OT_ERR_INVALID_ARG).  On success *out owns the workspace until
 * ot_destroy_tree. */
int ot_build_tree(const ot_tree_desc* desc, int device, ot_tree** out);

/* Upward pass: leaf moments (m = rho h^3 at the cell centre) and exact M2M
 * to every interior cell's centre of mass.  Defining passage: Sec. 4.3.2
 * (the FMM approximates distant cells through the tree: the multipole
 * moments of every tree cell).  rho: device float64 [n_leaf][512].  The
 * moments stay in the tree workspace; ot_get_moments reads them.  FP64. */
int ot_compute_moments(ot_tree* tree, const double* rho, void* stream);

/* Full solve: moments, every cell-to-cell interaction of every level in one
 * persistent launch, L2L shifts and evaluation.  Defining passage: Sec. 2
 * (FMM self-gravity), Sec. 4.3.1 (linear momentum conserved, angular
 * momentum through the correction term), Sec. 4.3.2 (octree of 8^3
 * sub-grids) and Sec. 5.5 (stencil, structure of arrays).  rho: device float64
 * [n_leaf][512]; phi: device float64 [n_leaf][512]; g: device float64
 * [n_leaf][3][512] (component-major per leaf).  opts may be NULL
 * (defaults).  The first solve of a plan captures a CUDA graph that later
 * solves with the same buffers replay. */
int ot_solve_gravity(ot_tree* tree, const double* rho, double* phi, double* g,
                     const ot_solve_opts* opts, void* stream);

/* Same as ot_solve_gravity with HOST buffers, all on `stream`; the outputs
 * are valid after the stream is synchronised.  Page-locked (pinned) buffers,
 * which the device can address, are read and written by the solve's own
 * kernels across the host link (no staging copies; a CUDA graph per buffer
 * set, as for device buffers); pageable buffers are copied in to and out of
 * device staging buffers around the solve.  Buffers must be 8-byte aligned. */
int ot_solve_gravity_host(ot_tree* tree, const double* rho_host, double* phi_host,
                          double* g_host, const ot_solve_opts* opts, void* stream);

/* Adjoint of the solve: drho = dJ/drho for J = sum_c (w1_c phi_c + w2_c . g_c),
 * the exact derivative of the discrete solve (through the centres of mass
 * and the correction's mass ratio), FP64 only (OT_PRECISION_FP64).  The paper
 * differentiates nothing; this is the reverse sweep of the solve that
 * ot_solve_gravity defines (each step of Sec. 4.3 transposed).  w1:
 * device float64 [n_leaf][512]; w2: device float64 [n_leaf][3][512]; drho:
 * device float64 [n_leaf][512] (overwritten).  Runs the forward solve itself
 * (its outputs go to internal buffers) and then the reverse sweep.  The
 * first call allocates the adjoint workspace (43 doubles per cell). */
int ot_gravity_backward(ot_tree* tree, const double* rho, const double* w1, const double* w2,
                        double* drho, const ot_solve_opts* opts, void* stream);

/* Tangent of the solve: the time derivative of the potential and of the
 * acceleration, phi_dot = (d phi / d rho) . rho_dot and g_dot likewise, for
 * densities changing at rho_dot (Sec. 2: the FMM includes the time
 * derivative of the potential, which energy conservation in the rotating
 * frame needs, Sec. 4.3.1; in the paper's code rho_dot comes from the
 * hydrodynamics).  The exact derivative of the discrete solve (through the
 * centres of mass and the correction's mass ratio), FP64 only.  rho,
 * rho_dot: device float64 [n_leaf][512]; phi_dot: device float64
 * [n_leaf][512]; g_dot: device float64 [n_leaf][3][512]; phi, g: the solve
 * itself in the same layouts, or NULL to skip.  The first call allocates the
 * tangent workspace (67 doubles per cell). */
int ot_solve_gravity_tangent(ot_tree* tree, const double* rho, const double* rho_dot, double* phi,
                             double* g, double* phi_dot, double* g_dot, const ot_solve_opts* opts,
                             void* stream);

/* PPM reconstruction of the hydro solver's 26 directional cell values, the
 * second workload on the same tree (Sec. 2: the finite-volume hydrodynamics
 * computes the values at all 26 spatial directions of a grid cell with the
 * piecewise parabolic method).  For each of the 13 lines through a cell (the
 * 26 neighbour offsets up to sign), 1-D PPM (Colella & Woodward 1984) on the
 * cell averages along the line: fourth-order boundary values held between the
 * neighbouring averages, then the parabola constraints.  Cells outside the
 * domain continue the averages by clamping each index into the grid.  The
 * tree's leaves must all be at one level (OT_ERR_INVALID_ARG otherwise).
 * u: device float64 [n_leaf][n_fields][512] cell averages (1 <= n_fields <=
 * 64); out: device float64 [n_leaf][n_fields][26][512], direction index of
 * offset o in {-1,0,1}^3 = (ox+1) + 3 (oy+1) + 9 (oz+1), minus 1 above 13.
 * FP64, written so that the limiter's decisions match a plain FP64
 * evaluation of the same formulas (no fused multiply-adds). */
int ot_ppm_reconstruct(ot_tree* tree, const double* u, int n_fields, double* out, void* stream);

/* Right-hand side of the hydro solver, dU/dt of the conserved fields
 * U = (rho, s_x, s_y, s_z, E) of an ideal gas with adiabatic index gamma
 * (Sec. 2: finite-volume hydrodynamics with PPM values at all 26 directions
 * of a cell; Sec. 4.3.1: mass, momentum and energy conserved across refinement
 * jumps by matching the fluxes there; Sec. 4.3.1: the hydro solver runs
 * beside the gravity solve in every Runge-Kutta stage).  Every leaf sees 3
 * ghost layers at its own level (the same-level cells; across a refinement
 * jump the mean of the 8 finer cells or the coarser cell's average; indices
 * clamped into the domain); PPM (Colella & Woodward 1984) gives the states
 * at the centre, edge midpoints and corners of each face; the face flux is
 * the 2-D Simpson rule (weights (1, 4, 1) x (1, 4, 1) / 36) of the local
 * Lax-Friedrichs (Rusanov) flux F* = (F(U_L) + F(U_R)) / 2 - a (U_R - U_L) / 2,
 * a the larger of |v_a| + sqrt(max(gamma p / rho, 0)) of the two states,
 * p = (gamma - 1) (E - s.s / (2 rho)); a face on the domain boundary takes
 * the inside state on both sides (transmissive); a face next to a finer
 * region takes the mean of the 4 finer faces' fluxes (flux matching);
 * dU/dt = sum over axes of (F_low - F_high) / h + (0, rho g, s.g).
 * OT_ERR_INVALID_ARG for gamma <= 1 or not finite.  A face state whose
 * density is not positive (a non-physical state) is latched in the device
 * status word (bit 4), which ot_tree_info reports as OT_ERR_DEVICE_STATUS;
 * the rates are then not finite.  u: device float64
 * [n_leaf][5][512]; g: device float64 [n_leaf][3][512] (e.g. the gravity
 * solve's output) or NULL for no gravity; dudt: device float64
 * [n_leaf][5][512].  The first call allocates the workspace (the PPM values
 * of the cells and their primitive variables, the PPM values of the ghost
 * cells next to the faces, and the face fluxes: about 311 doubles per
 * cell).  FP64, written so that every
 * operation matches a plain FP64 evaluation of the same formulas (no fused
 * multiply-adds). */
int ot_hydro_rhs(ot_tree* tree, const double* u, const double* g, double gamma, double* dudt, void* stream);

/* One time step of the coupled hydro-gravity system, on the device (Sec.
 * 4.3.1: a third-order Runge-Kutta scheme whose every stage runs the hydro
 * solver and the FMM gravity solve; the paper names GPU-resident data as the
 * next step, Sec. 5.5 and Sec. 8).  The scheme is the strong-stability-
 * preserving third-order method of Shu & Osher (1988): U1 = U0 + dt L(U0),
 * U2 = 3/4 U0 + 1/4 (U1 + dt L(U1)), U3 = 1/3 U0 + 2/3 (U2 + dt L(U2)),
 * each combination in that order, where L is ot_hydro_rhs with, when
 * gravity is 1, the acceleration of one ot_solve_gravity of the stage's own
 * density U[:, 0] (opts: that solve's options, NULL for the defaults;
 * gravity 0: no gravity, opts unused).  u: device float64 [n_leaf][5][512],
 * U^n in, U^(n+1) out.  dt: finite.  OT_ERR_INVALID_ARG for a bad gamma, dt,
 * gravity flag or solve option.  The first call allocates 20 doubles per
 * cell besides ot_hydro_rhs's workspace; the gravity solves replay one CUDA
 * graph. */
int ot_hydro_rk3_step(ot_tree* tree, double* u, double dt, double gamma, int gravity,
                      const ot_solve_opts* opts, void* stream);

/* Chooses the persistent launch's stencil-chunk length and the CTAs per SM
 * of the general kernel (and, wide FP32 form, of the lattice kernels) for
 * this plan: every candidate is timed as the whole solve graph it would run,
 * on `stream` (synchronised), and the fastest is kept.  rho/phi/g as in
 * ot_solve_gravity (phi and g hold the solve's result afterwards). */
int ot_autotune(ot_tree* tree, const double* rho, double* phi, double* g,
                const ot_solve_opts* opts, void* stream);

/* Device time in milliseconds of the interaction phase and of the whole
 * solve in the most recent ot_solve_gravity(_host) on this tree, from CUDA
 * events recorded inside the solve's CUDA graph.  The interaction phase runs
 * from the end of the leaf-moment kernel to the end of the last interaction
 * kernel; the M2M kernels of the interior levels run inside it, concurrently
 * with the leaf-leaf interactions.  Waits for those events.  Either pointer
 * may be NULL. */
int ot_last_solve_times(ot_tree* tree, float* interact_ms, float* solve_ms);

/* Counts of the tree and of the current plan; synchronises the tree's last
 * stream to read the device status word, and clears the word after reading
 * it (an error is reported once; returns OT_ERR_DEVICE_STATUS then, with
 * the counts and device_status filled in). */
int ot_tree_info(ot_tree* tree, ot_tree_stats* stats);

/* Allocation-free solve for callers that cannot allocate device memory:
 * plug-ins whose host application owns all device memory and only hands
 * them buffers, and real-time loops that forbid allocation after start-up
 * (ot_build_tree allocates the tree workspace, so those callers cannot use
 * ot_solve_gravity).  The paper has no counterpart; it is the same solve as
 * ot_solve_gravity (same kernels, same results to rounding) for small trees,
 * without a tree handle: every piece of scratch (node tables, moments,
 * expansions, stencil tables, work items) lives in one fixed 4 MiB device
 * array inside the library, held by every GPU that loads it until the
 * process exits.  desc: host leaf list as for ot_build_tree, at most 9 nodes
 * (the root leaf alone, or the root and its 8 leaf children: 4,096 cells);
 * rho, phi, g: device buffers on the CURRENT device, layouts as for
 * ot_solve_gravity; opts checked as for ot_solve_gravity, and 0.5 <= theta
 * <= 1.  Larger trees return OT_ERR_TOO_LARGE.  No device memory is allocated
 * (host-side planning uses the heap, and the tables are uploaded from it
 * with cudaMemcpyAsync before the call returns).  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array and
 * each call clears what must start at zero; calls that overlap on the GPU
 * race, so issue them on one stream or synchronise between them.  Errors that
 * a kernel latches in the device status word (a plan error) are not reported
 * by this entry point: it has no handle to report them through. */
int ot_solve_gravity_static(const ot_tree_desc* desc, const double* rho, double* phi, double* g,
                            const ot_solve_opts* opts, void* stream);

/* Reads the moments of every cell of level `level` (Sec. 4.3.2: the
 * multipole moments of the tree cells, as ot_compute_moments or the last
 * solve left them) in physical units: out, device float64
 * [n_nodes(level)][20][512] -- per node of the level (in the tree's
 * breadth-first order of that level) and per component, the 512 cells in
 * i + 8 j + 64 k order; components m, X (centre of mass, 3), M2 (about X,
 * packed xx xy xz yy yz zz, 6), M3 (about X, packed xxx xxy xxz xyy xyz xzz
 * yyy yyz yzz zzz, 10).  node_xyz: optional host int32 [n_nodes(level)][3],
 * the nodes' coordinates at that level (NULL to skip).  Asynchronous on
 * `stream` (one conversion kernel); returns OT_ERR_INVALID_ARG for a level
 * outside the tree. */
int ot_get_moments(ot_tree* tree, int level, double* out, int32_t* node_xyz, void* stream);

/* Sets the persistent launch's shape without the autotuner (for instance the
 * shape an earlier ot_autotune chose, read back by ot_tree_info): chunk =
 * stencil entries per work item (1 <= chunk <= 4096), ctas_per_sm = CTAs of
 * the general kernel per SM (1..16), lattice_ctas_per_sm = persistent CTAs
 * per SM of the wide FP32 form's lattice kernels (0 = one per leaf node,
 * 1..16).  The general kernels of every form take items of any length.
 * Rebuilds the work items (host) and re-uploads them; the next solve
 * captures a new graph. */
int ot_set_launch_shape(ot_tree* tree, int chunk, int ctas_per_sm, int lattice_ctas_per_sm);

/* Measures the CUDA-core arithmetic peaks of `device` with throughput
 * microkernels (independent FMA chains on every SM, timed with CUDA events
 * on an internal stream, best of `reps` launches): FP64 FMA, FP32 FMA and
 * the paired FP32 FMA (two per instruction), in TFLOP/s (an FMA counts 2).
 * Any output pointer may be NULL.  Allocates and frees a small device
 * buffer; synchronises the device. */
int ot_alu_peaks(int device, int reps, double* fp64_tflops, double* fp32_tflops,
                 double* fp32x2_tflops);

/* Releases the workspace; NULL is ignored. */
void ot_destroy_tree(ot_tree* tree);

/* Static string for an OT_* code. */
const char* ot_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* OCTOFMM_H */
