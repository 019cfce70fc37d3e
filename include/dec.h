/*
 * dec.h - C ABI of the GB300 DEC steady-conduction library (libdec_gb300).
 *
 * The library computes, on one GPU, the data-parallel hot path of the
 * discrete exterior calculus (DEC) method for 3D elliptic boundary value
 * problems of arXiv 2104.05999 ("Parallelized DEC for three-dimensional
 * elliptic problems"), with steady heat conduction as the proxy problem:
 *
 *   dec_mesh_upload      cells and incidence: the edge list of the
 *                        tetrahedral complex, i.e. the sparsity of d0
 *                        (Sec. 2.1, cell complexes and coboundary d)
 *   dec_hodge_assemble   diagonal Hodge star *1 on edges from the
 *                        circumcentric dual, times conductivity, zeroed on
 *                        dual faces that a penny crack cuts (Sec. 2.1, 2.5)
 *   dec_laplacian_build  node Laplacian L = d0^T *1 d0 with Dirichlet rows
 *                        and zero-flux (natural) boundaries (Sec. 2.3,
 *                        Eq. 11-13) plus a sparse-approximate-inverse
 *                        preconditioner (Sec. 2.3, ParaSails family)
 *   dec_solve            preconditioned conjugate gradients to a relative
 *                        residual (Sec. 2.3, Sec. 3.1)
 *   dec_k_eff            effective conductivity: heat flux through the
 *                        Dirichlet face x = 0 (Sec. 2.5)
 *
 * Conventions for every entry point:
 *   - Return value: a dec_status; DEC_OK (0) on success.  No call aborts.
 *     dec_last_error() returns a text for the last failure of a context.
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the context's GPU; copies use unified
 *     addressing.  Input buffers are copied: the caller keeps ownership and
 *     may free or reuse them when the call returns.  Output buffers are
 *     allocated by the caller and written before the call returns.
 *   - All GPU work is ordered on the stream given to dec_create.  A call
 *     returns once its outputs are valid; host-side scalars it returns are
 *     synchronised.
 *   - Calls must come in order: mesh_upload, hodge_assemble,
 *     laplacian_build, solve, k_eff.  A call made before its predecessor
 *     returns DEC_ERR_STATE.  A new mesh_upload invalidates everything after
 *     it; a new hodge_assemble invalidates the Laplacian and the solution.
 *   - Device memory is owned by the context and reused across calls while
 *     sizes allow; dec_destroy frees it.
 *   - Index types: node ids are int32 (n < 2^31 - 1), counts are int64.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef DEC_GB300_H
#define DEC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dec_ctx dec_ctx;

typedef enum {
  DEC_OK = 0,
  DEC_ERR_ARG = 1,          /* invalid argument (NULL, size, enum value)    */
  DEC_ERR_MESH = 2,         /* node id out of range, inverted or flat tet   */
  DEC_ERR_CUDA = 3,         /* a CUDA runtime call failed (text has it)     */
  DEC_ERR_BREAKDOWN = 4,    /* CG breakdown: p^T L p <= 0 or not finite     */
  DEC_NOT_CONVERGED = 5,    /* max_iter reached before rtol                 */
  DEC_ERR_TIMEOUT = 6,      /* a bounded device-side wait ran out           */
  DEC_ERR_STATE = 7,        /* entry point called out of order              */
  DEC_ERR_LIMIT = 8         /* a size exceeds a documented limit            */
} dec_status;

/* node tags (node_tag argument of dec_mesh_upload) */
enum { DEC_NODE_FREE = 0, DEC_NODE_DIRICHLET = 1, DEC_NODE_NEUMANN = 2 };
/* preconditioners (dec_laplacian_build) */
enum {
  DEC_PRECOND_JACOBI = 0,       /* 1 / L_ii, per instance                     */
  DEC_PRECOND_FSAI = 1,         /* FSAI factor per instance (value set)       */
  DEC_PRECOND_FSAI_SHARED = 2   /* prepares the batched solve
                                   (DEC_MODE_MIXED_BATCHED): Dirichlet sets
                                   share the FSAI factor of their common L;
                                   crack states and conductivity fields get
                                   one FP32-built BF16 factor each (rows
                                   longer than 12 keep the factor of the
                                   uncracked operator, resp. of field 0)      */
};
/* solve modes (dec_solve) */
enum {
  DEC_MODE_FP64 = 0,   /* PCG in FP64 (matrix, preconditioner, vectors)       */
  DEC_MODE_MIXED = 1,  /* PCG with FP32 vectors and L and a BF16 FSAI factor
                          (FP32 Jacobi) inside FP64 defect correction: the
                          FP32 update is added to an FP64 solution x and the
                          FP32 residual replaced by r = b - L x in FP64 each
                          time it has dropped by 1e-2, keeping the search
                          direction; convergence is decided in FP64.  Runs
                          as one persistent cooperative kernel per instance
                          up to 400,000 nodes, as one kernel per phase
                          above                                            */
  DEC_MODE_MIXED_PHASED = 2, /* the same solve as DEC_MODE_MIXED, run as one
                                kernel per phase (CUDA graphs) instead    */
  DEC_MODE_MIXED_BATCHED = 3  /* the mixed solve of all instances (crack
                                states or Dirichlet sets, at most 64) in
                                one persistent launch over a sparse matrix -
                                multiple vector product, with per-instance
                                convergence masks; needs
                                DEC_PRECOND_FSAI_SHARED                    */
};

/* Local edge slots of a tet: slot s joins local vertices LOCAL[s] =
 * (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).  t2e[t*6+s] is that edge's id. */

/* Create a context on CUDA device `device`, ordering its work on `stream`
 * (a cudaStream_t of that device).  With stream = NULL the context creates a
 * private non-blocking stream; device inputs must then be complete when a
 * call is made.  *ctx receives the handle. */
dec_status dec_create(dec_ctx** ctx, int device, void* stream);

/* Free every device buffer of the context and the context itself.
 * Accepts NULL. */
dec_status dec_destroy(dec_ctx* ctx);

/* Text of the last error of `ctx` (or of the last failed dec_create when
 * ctx is NULL).  Valid until the next call on the context. */
const char* dec_last_error(const dec_ctx* ctx);

/* Upload a tetrahedral mesh and build its edge list (the incidence d0 of
 * Sec. 2.1) on the GPU.
 *   xyz      [n_nodes*3] f64, host or device: node coordinates x, y, z.
 *   tets     [n_tets*4] int32, host or device: node ids of each tet,
 *            positively oriented ((x1-x0).((x2-x0)x(x3-x0)) > 0).
 *   node_tag [n_nodes] uint8, host or device: DEC_NODE_* per node.
 * Edges come out unique with i < j, sorted by (i, j).  Errors:
 * DEC_ERR_ARG for NULL pointers, n_nodes < 4 or >= 2^31 - 1, n_tets < 1 or
 * 6*n_tets >= 2^32; DEC_ERR_MESH when a node id is out of range, a tet is
 * not positively oriented, or a tag is not 0, 1 or 2. */
dec_status dec_mesh_upload(dec_ctx* ctx, const double* xyz, int64_t n_nodes,
                           const int32_t* tets, int64_t n_tets,
                           const uint8_t* node_tag);

/* Assemble the diagonal Hodge star *1 on edges (Sec. 2.1: ratio of the
 * circumcentric dual face area to the edge length, signed pieces), with
 * each tet's share scaled by its conductivity, and the crack state of
 * every edge (Sec. 2.5: a cracked dual face gets conductivity 0).
 *   k        [n_tets] f64 host or device, or NULL for k = 1.  Must be
 *            finite and > 0.
 *   discs    [n_discs*7] f64 host or device (cx, cy, cz, nx, ny, nz, r),
 *            unit normals, r > 0; NULL with n_discs = 0 for no cracks.
 *   scales   [n_scales] f64 host or device, increasing radius factors of
 *            the crack states of one disc population, or NULL (one state,
 *            factor 1).  n_scales <= 255.
 * An edge is cut in state b when a disc with radius scales[b]*r meets a
 * sub-triangle (midpoint, face circumcentre, tet circumcentre) of its dual
 * face; the whole edge then gets *1 = 0 in that state.
 * Errors: DEC_ERR_STATE without a mesh, DEC_ERR_ARG for bad k, discs or
 * scales. */
dec_status dec_hodge_assemble(dec_ctx* ctx, const double* k,
                              const double* discs, int64_t n_discs,
                              const double* scales, int32_t n_scales);

/* Several conductivity fields on one mesh (Sec. 1: the same mesh serves
 * many material fields; Sec. 2.1: conductivity lives on the dual 2-cells):
 * assemble one Hodge star *1 per field, each as dec_hodge_assemble does for
 * that field (bit for bit), with one common set of cracks.  The fields then
 * are the instances of dec_laplacian_build (n_sets must be 1), dec_solve
 * (every mode; DEC_MODE_MIXED_BATCHED solves all fields in one launch, with
 * one FSAI factor per field) and dec_k_eff.
 *   k         [n_fields*n_tets] f64 host or device: field f's conductivity of
 *             tet t at k[f*n_tets + t]; finite and > 0.
 *   n_fields  1..64.
 *   discs, n_discs   as for dec_hodge_assemble (one crack state).
 * dec_get_hodge reports field 0.  dec_crack_evolve needs a single field.
 * Errors: DEC_ERR_STATE without a mesh, DEC_ERR_ARG for bad k or discs,
 * DEC_ERR_LIMIT for more than 64 fields. */
dec_status dec_hodge_assemble_fields(dec_ctx* ctx, const double* k, int32_t n_fields,
                                     const double* discs, int64_t n_discs);

/* geometry precisions (dec_set_geom_precision) */
enum {
  DEC_GEOM_FP64 = 0,    /* every tet's geometry in FP64 (the default)          */
  DEC_GEOM_MIXED = 1    /* FP32 for well-shaped tets, FP64 for the others      */
};

/* Choose the arithmetic of the per-tet geometry (Sec. 2.1: circumcentres and
 * the dual-face pieces over edge lengths) for the following
 * dec_hodge_assemble and dec_hodge_assemble_fields calls of the context.
 * DEC_GEOM_MIXED computes a tet in FP32 when L^3 <= 16 |6 V| (L its longest
 * edge from its first vertex, V its volume; a regular tet has
 * L^3 / |6 V| = 2.8, a Kuhn tet 5.2), in FP64 otherwise.  Crack decisions
 * are those of the FP64 geometry: the FP32 circumcentre only serves as a
 * filter with an error bound, and any tet that a disc may cut has its
 * circumcentre formed again in FP64 for the exact test.  The FP32 pieces
 * carry relative errors of order 1e-6, so *1, T and k_eff move by about
 * that much against the FP64 geometry (DEC_GEOM_FP64 keeps agreement with
 * the FP64 definition to 1e-12).  dec_get_geom_fp64_tets gives the number
 * of tets the last assembly computed in FP64 (all of them with
 * DEC_GEOM_FP64).
 * Errors: DEC_ERR_ARG (NULL context or pointer, unknown precision). */
dec_status dec_set_geom_precision(dec_ctx* ctx, int32_t precision);
dec_status dec_get_geom_fp64_tets(const dec_ctx* ctx, int64_t* n_tets);

/* Build the node Laplacian and the right-hand sides (Sec. 2.3, Eq. 11-13),
 * node form: L_ij = -*1_ij, L_ii = sum_j *1_ij; Dirichlet columns move to
 * the right-hand side (b_i = sum_{j in D} *1_ij T0_j), Dirichlet rows
 * become identity rows with b_i = 0 (the unknown is T - T0 on Dirichlet
 * nodes, i.e. 0); a free row whose weights are all zero becomes an
 * identity row too.  Then set up the preconditioner.
 *   T0       [n_sets*n_nodes] f64 host or device: Dirichlet values (only
 *            entries at Dirichlet nodes are read).
 *   n_sets   number of Dirichlet value sets (right-hand sides), >= 1.
 *            With n_scales > 1 in dec_hodge_assemble, or several fields in
 *            dec_hodge_assemble_fields, n_sets must be 1: the instances are
 *            then the crack states or the fields.
 *   precond  DEC_PRECOND_JACOBI or DEC_PRECOND_FSAI (factored sparse
 *            approximate inverse on the pattern of lower(L): G^T G ~ L^-1).
 * Errors: DEC_ERR_STATE, DEC_ERR_ARG, DEC_ERR_LIMIT when an FSAI row has
 * more than 32 lower-pattern entries (a node with more than 31 neighbours of
 * smaller id). */
dec_status dec_laplacian_build(dec_ctx* ctx, const double* T0, int32_t n_sets,
                               int32_t precond);

/* Solve L u = b for every instance by PCG from u = 0 until
 * ||b - L u||_2 <= rtol ||b||_2 (FP64 true residual), then form the
 * temperature T = u + T0 on Dirichlet nodes.
 *   rtol      relative residual, > 0 (e.g. 1e-10).
 *   max_iter  cap on (inner) CG iterations per instance, >= 1.
 *   mode      DEC_MODE_FP64 or DEC_MODE_MIXED.
 *   T_out     [B*n_nodes] f64 host or device, or NULL to keep T on the GPU
 *             only (k_eff still works).  B = number of instances.
 *   iters     [B] int32 host, or NULL: CG iterations used per instance.
 *   relres    [B] f64 host, or NULL: final FP64 relative residuals.
 * Errors: DEC_ERR_STATE, DEC_ERR_ARG, DEC_ERR_BREAKDOWN, DEC_NOT_CONVERGED
 * (outputs are still written with the last iterate). */
dec_status dec_solve(dec_ctx* ctx, double rtol, int32_t max_iter, int32_t mode,
                     double* T_out, int32_t* iters, double* relres);

/* Effective conductivity per instance (Sec. 2.5) from the last solve, in
 * FP64 with the unmodified *1 (cut edges 0):
 *   q_in   [B] host: sum over Dirichlet nodes on x = 0 of sum_j *1_ij (T_i - T_j)
 *   q_out  [B] host or NULL: same over x = 1 with (T_j - T_i)
 *   energy [B] host or NULL: sum over edges of *1_e (T_i - T_j)^2
 * For T0 = 1 on x = 0 and 0 on x = 1 in the unit cube, k_eff = q_in. */
dec_status dec_k_eff(dec_ctx* ctx, double* q_in, double* q_out, double* energy);

/* Launch shape the last DEC_MODE_MIXED_BATCHED solve of this context used,
 * as picked by its autotuner: the first batched solve of a problem size
 * (nodes, matrix entries) at each instance stride (8, 16, 32, 64) times a
 * few iterations of every variant and keeps the fastest for the context's
 * later solves of that size.
 *   gather_entries  host: 1000 * K / 8 (K = matrix entries per chunk of a
 *                   warp's structure staged in shared memory; Dirichlet
 *                   sets of 8 or 16 instances only) + 100 * (gathers into
 *                   shared memory by cp.async) + 10 * (next entries'
 *                   structure loaded while the gathers are in flight) +
 *                   gathers per round trip, + 500 when only the FSAI halves
 *                   are staged (the SpMM as variant 12): one of 2, 4, 12,
 *                   114, 106, 1004, 2004, 2002, 2512.
 * All variants give bit-identical results.  DEC_ERR_STATE before the first
 * batched solve.  (No counterpart in the paper: a launch-shape choice.) */
dec_status dec_get_batch_variant(dec_ctx* ctx, int32_t* gather_entries);

/* Launch shapes of the single-instance SELL kernels (the L product of
 * DEC_MODE_FP64 and of the per-phase mixed modes, and the two FSAI halves),
 * as picked by their autotuner: the first such solve of a problem size
 * (nodes, matrix entries) in a precision times a few launches of every
 * shape on the context's scratch vectors and keeps the fastest.
 *   precision  0: FP64 (DEC_MODE_FP64), 1: FP32 / BF16 (mixed modes).
 *   l_shape    host: 100 * (resident blocks per SM) + (matrix entries per
 *              round trip): one of 408, 808, 412, 804; 0 before any solve.
 *   g_shape    host: 14 (slices staged in shared memory) or 8 (round trips
 *              of 8 entries); 0 before any solve with FSAI.
 * Every shape gives bit-identical results.  (No counterpart in the paper:
 * a launch-shape choice.) */
dec_status dec_get_sell_variant(const dec_ctx* ctx, int32_t precision, int32_t* l_shape,
                                int32_t* g_shape);

/* Make the following single-instance solves use the given shapes (codes of
 * dec_get_sell_variant; 0: the autotuner's choice, tuned again at the next
 * solve).  Errors: DEC_ERR_ARG for an unknown code. */
dec_status dec_set_sell_variant(dec_ctx* ctx, int32_t l_shape, int32_t g_shape);

/* Make the following batched solves of the context use one variant (a code
 * of dec_get_batch_variant) instead of the autotuner's choice; 0 returns to
 * the autotuner.  A solve whose batch the variant does not fit (a staged
 * variant with crack states or fields, or more than 16 instances) fails
 * with DEC_ERR_ARG.  Errors: DEC_ERR_ARG for an unknown code.  (No
 * counterpart in the paper: used to compare launch shapes.) */
dec_status dec_set_batch_variant(dec_ctx* ctx, int32_t variant);

/* Device time in ms of the persistent kernel launch of the last successful
 * DEC_MODE_MIXED_BATCHED solve (the launch that solved every instance, not
 * the autotuner's trial launches), measured by CUDA events recorded on the
 * context's stream around that launch.  DEC_ERR_STATE before the first
 * batched solve.  (No counterpart in the paper: a measurement aid.) */
dec_status dec_get_batch_kernel_ms(dec_ctx* ctx, double* ms);

/* Where the last batched solve spent a full FP32 iteration, in ms per
 * iteration (device time read at the grid barriers by one thread of block
 * 0, averaged over the iterations that ran all five phases): ms5[0] the
 * sparse matrix - multiple vector product and p.q, [1] the x and r updates
 * and r.r, [2] the lower FSAI half t = G r, [3] the upper half z = G^T t and
 * r.z, [4] the p update.  DEC_ERR_STATE before the first batched solve.
 * (No counterpart in the paper: a measurement aid.) */
dec_status dec_get_batch_phase_ms(dec_ctx* ctx, double* ms5);

/* crack rules (dec_crack_evolve) */
enum {
  DEC_CRACK_MAX_FLUX = 0,   /* the face with the largest flux cracks (Sec. 3.3)   */
  DEC_CRACK_ORDER = 1,      /* faces crack in a caller-drawn order (Sec. 3.4)     */
  DEC_CRACK_REBUILD = 16    /* or-ed into a rule: rebuild L, b and the
                               preconditioner and solve from zero at every
                               step, instead of updating the changed rows and
                               starting from the previous solution            */
};

/* Crack growth (Sec. 2.5; deterministic cracking Sec. 3.3, stochastic
 * cracking Sec. 3.4).  Starting from the current state (after
 * dec_laplacian_build with one Dirichlet set, no crack states and
 * DEC_PRECOND_JACOBI or DEC_PRECOND_FSAI), solve, then repeat: crack one
 * dual face (its edge's *1 becomes 0 for L, b, the preconditioner and
 * k_eff), solve again, record k_eff.  A crack changes a few values of the
 * system only (Sec. 2.3): each step recomputes rows i and j of L and b (as a
 * full build would), the FSAI rows whose lower-pattern block holds i or j
 * (or the two Jacobi entries), and starts PCG from the previous solution;
 * with DEC_CRACK_REBUILD or-ed into the rule it rebuilds L and the
 * preconditioner and solves from zero instead.  The stopping rule is the
 * same either way: ||b - L u|| <= rtol ||b||.  Candidates are the edges that still conduct (*1 > 0, not cut):
 * in the node form every dual face lies between two dual cells.
 *   rule      DEC_CRACK_MAX_FLUX: the candidate with the largest
 *             |*1_e (T_i - T_j)| in the current solution (the flux 2-form on
 *             its dual face; the smallest edge id wins a tie);
 *             DEC_CRACK_ORDER: edge order[s] at step s.
 *   max_steps at most this many cracks.
 *   order     [max_steps] int32 edge ids (dec_get_edges numbering), host or
 *             device; only read for DEC_CRACK_ORDER, else may be NULL.
 *   rtol, max_iter, mode   as for dec_solve (FP64, MIXED or MIXED_PHASED).
 *   k_stop    stop after the step whose k_eff <= k_stop * k_eff(uncracked)
 *             (e.g. 1e-9: the domain no longer conducts).
 *   cracked   [max_steps] int32 host: edge cracked at each step.
 *   k_eff     [max_steps] f64 host: q_in (as dec_k_eff) after each step.
 *   steps     host: number of steps done (fewer than max_steps when k_stop
 *             is reached or no candidate is left).
 * The cracks stay in the context (dec_get_hodge shows them as cut in state
 * 0; dec_k_eff reports the last state).  Errors: DEC_ERR_STATE, DEC_ERR_ARG
 * (also for an order entry that is not a conducting, uncut edge; the steps
 * before it are kept), and the errors of dec_solve (the crack of the step
 * whose solve failed stays in the context; *steps counts completed steps). */
dec_status dec_crack_evolve(dec_ctx* ctx, int32_t rule, int32_t max_steps,
                            const int32_t* order, double rtol, int32_t max_iter, int32_t mode,
                            double k_stop, int32_t* cracked, double* k_eff, int32_t* steps);

/* Stochastic cracking of several Monte-Carlo paths at once (Sec. 3.4: the
 * damage at which the domain stops conducting, over many random orders).
 * Starting from the current state (as for dec_crack_evolve: one Dirichlet
 * set, no crack states, one conductivity field), path b cracks the edges
 * orders[b][0], orders[b][1], ... one per step, each in its own copy of *1;
 * after every step all paths are solved together by the batched mixed
 * solve (one instance per path, one FSAI factor per path, every solve
 * started from the previous solutions) and k_eff is recorded.  A path stops
 * after the step whose k_eff <= k_stop * its uncracked k_eff.
 *   n_paths   2..64.
 *   orders    [n_paths*max_steps] int32 edge ids, host or device.
 *   rtol, max_iter   as for dec_solve.
 *   k_eff     [n_paths*max_steps] f64 host: q_in of path b after step s at
 *             k_eff[b*max_steps + s] (entries past a path's last step are
 *             not written).
 *   steps     [n_paths] int32 host: steps done per path.
 * Afterwards the context holds the paths as instances (dec_k_eff reports
 * each path's last state; dec_solve with DEC_MODE_MIXED_BATCHED solves them
 * again).  Errors: DEC_ERR_STATE, DEC_ERR_ARG (also for an order entry that
 * is not a conducting, uncut edge of its path; the steps before it are
 * kept), and the errors of dec_solve. */
dec_status dec_crack_paths(dec_ctx* ctx, int32_t n_paths, int32_t max_steps,
                           const int32_t* orders, double rtol, int32_t max_iter,
                           double k_stop, double* k_eff, int32_t* steps);

/* ---- the paper's own tet-centred form ---- */

/* Solve the mixed system of Sec. 2.3 (Eq. 11-13) with one potential per tet
 * and one flux per triangular face, the flux block eliminated as the
 * paper's Schur-complement solve does: the flux block (1/kappa) *2 is
 * diagonal (*2_f = signed circumcentric dual edge length / face area), so
 * the potentials alpha solve the two-point operator
 *   sum over the faces f of T of w_f (alpha_T - alpha_T'),  w_f = kappa / *2_f,
 * where a face whose three nodes are Dirichlet ties alpha_T to the mean T0
 * of those nodes and any other boundary face carries the prescribed outward
 * flux (Eq. 13; none: zero flux).  Sec. 3.1's limiter raises *2 entries
 * below `limiter` to it.  Cracked faces (Sec. 2.5) get w_f = 0.  FP64 PCG
 * from alpha = 0 to ||b - S alpha|| <= rtol ||b||, preconditioned by an
 * FSAI factor (the sparse approximate inverse family of the paper's
 * solver; pattern: each tet's lower neighbours and itself).
 *   T0            [n_nodes] f64 host or device: node values (read on
 *                 Dirichlet nodes).
 *   kappa         conductivity, > 0.  limiter: <= 0 for none (e.g. 1e-8).
 *   cracked_faces [n_cracked] int32 host or device face ids
 *                 (dec_tet_get_faces numbering), or NULL.
 *   face_flux     [n_faces] f64 host or device outward flux through each
 *                 face (read on non-Dirichlet boundary faces), or NULL.
 *   alpha         [n_tets] f64 host or device, or NULL: potential per tet
 *                 (at its circumcentre).
 *   q2            [2] f64 host, or NULL: heat entering through the Dirichlet
 *                 faces on x = 0 and leaving through those on x = 1.
 *   iters, relres, n_limited   host outputs, or NULL.
 * A tet whose faces all carry w = 0 gets alpha = 0; a group of tets cut off
 * from every Dirichlet face keeps alpha = 0 (its block is singular with a
 * zero right-hand side unless face fluxes enter it).  Needs an uploaded
 * mesh only (independent of the node-form calls).  Errors: DEC_ERR_STATE,
 * DEC_ERR_ARG (also a cracked face id out of range), DEC_ERR_BREAKDOWN,
 * DEC_NOT_CONVERGED (outputs still written), DEC_ERR_TIMEOUT. */
dec_status dec_tet_solve(dec_ctx* ctx, const double* T0, double kappa, double limiter,
                         const int32_t* cracked_faces, int64_t n_cracked,
                         const double* face_flux, double rtol, int32_t max_iter, double* alpha,
                         double* q2, int32_t* iters, double* relres, int64_t* n_limited);

/* Faces of the uploaded mesh: the sorted node triples (i < j < k) in
 * lexicographic order, and the face opposite local vertex v of tet t at
 * t2f[t*4 + v].  n_faces host; faces [n_faces*3] and t2f [n_tets*4] int32
 * host or device, either may be NULL. */
dec_status dec_tet_get_faces(dec_ctx* ctx, int64_t* n_faces, int32_t* faces, int32_t* t2f);

/* Flux vector at each tet's barycentre from the last dec_tet_solve
 * (Whitney 2-form interpolation of the face fluxes, the paper's vector
 * output): v = sum_i phi_i (b - x_i) / (3 V), phi_i the outward flux through
 * the face opposite vertex i.  v [n_tets*3] f64 host or device.
 * DEC_ERR_STATE without a solution. */
dec_status dec_tet_whitney(dec_ctx* ctx, double* v);

/* CG iterations summed over the steps of the last dec_crack_evolve or
 * dec_crack_paths call (over all paths; the first solve before any crack
 * not counted). */
dec_status dec_get_crack_iterations(const dec_ctx* ctx, int64_t* iters);

/* ---- sizes and intermediate results (parity checks, debugging) ---- */

/* n_nodes, n_tets, n_edges, nnz of L (with the diagonal), instances B. */
dec_status dec_get_sizes(const dec_ctx* ctx, int64_t* n_nodes, int64_t* n_tets,
                         int64_t* n_edges, int64_t* nnz, int32_t* n_instances);

/* Edge list E [n_edges*2] int32 (i < j, sorted) and tet->edge map
 * t2e [n_tets*6] int32; either may be NULL.  Host or device buffers. */
dec_status dec_get_edges(dec_ctx* ctx, int32_t* E, int32_t* t2e);

/* Hodge star *1 of the uncracked mesh w [n_edges] f64, and the first crack
 * state per edge first_cut [n_edges] uint8 (n_scales, or 1 without scales,
 * when never cut); either may be NULL.  Host or device buffers. */
dec_status dec_get_hodge(dec_ctx* ctx, double* w, uint8_t* first_cut);

/* CSR of L: rowptr [n_nodes+1] int32, col [nnz] int32, columns sorted,
 * diagonal included.  val [nnz] f64 and b [n_nodes] f64 of instance
 * `inst` (after DEC_PRECOND_FSAI_SHARED, val is the common operator of
 * Dirichlet sets, or the uncracked operator for crack states; b is still
 * per instance).  Any pointer may be
 * NULL.  Host or device buffers. */
dec_status dec_get_csr(dec_ctx* ctx, int32_t inst, int32_t* rowptr,
                       int32_t* col, double* val, double* b);

/* FSAI factor in L's CSR layout, g [nnz] f64: entries with col <= row hold
 * G[row][col], entries with col > row hold G[col][row] (the transpose).
 * Jacobi: the diagonal holds 1/L_ii and off-diagonals 0.  Host or device. */
dec_status dec_get_precond(dec_ctx* ctx, double* g);

/* ---- measurement ---- */

/* kernels that dec_time_kernel can time */
enum {
  DEC_KERNEL_SPMV_F64 = 0,   /* q = L p, FP64 values and vectors, fused p.q   */
  DEC_KERNEL_SPMV_F32 = 1,   /* same with FP32 values and vectors             */
  DEC_KERNEL_FSAI_F64 = 2,   /* z = G^T (G r), FP64 factor (two launches)     */
  DEC_KERNEL_FSAI_BF16 = 3   /* same with the BF16 factor and FP32 vectors    */
};

/* Launch one solver kernel `reps` times on instance 0's matrix after a
 * successful dec_laplacian_build, each launch timed alone with CUDA events
 * on the context's stream and preceded, outside the timed interval, by a
 * write of `flush_bytes` bytes of device memory (pass more than the L2 size
 * to time the kernel with a cold cache).  *avg_ms receives the mean launch
 * duration.  The launch configuration is the one dec_solve uses.  Allocates
 * a flush buffer of `flush_bytes` owned by the context.  Overwrites the
 * solver's scratch vectors (a later dec_k_eff is unaffected).
 * Errors: DEC_ERR_STATE, DEC_ERR_ARG for an unknown kernel or reps < 1. */
dec_status dec_time_kernel(dec_ctx* ctx, int32_t kernel, int32_t reps,
                           int64_t flush_bytes, double* avg_ms);

/* Number of CUDA kernels the context has launched since dec_create,
 * counting every kernel node of each replayed CUDA graph. */
dec_status dec_get_launch_count(const dec_ctx* ctx, int64_t* count);

/* ---- testing aid (no counterpart in the paper) ---- */

/* Run the failure path of the persistent solves without any endless wait.
 * The persistent kernels (DEC_MODE_MIXED up to 400,000 nodes and
 * DEC_MODE_MIXED_BATCHED) separate their phases by grid barriers that poll a
 * counter at most 2^24 times (32-256 ns apart) before the kernel records a
 * failure, every block leaves at its next barrier and the call returns
 * DEC_ERR_TIMEOUT.  With this switch on, later persistent launches of the
 * context use
 *   spin_limit       polls per barrier wait instead of 2^24 (0: unchanged),
 *   withhold_block   1: the last block of the grid returns before its first
 *                    barrier, so the other blocks' wait runs out after
 *                    spin_limit polls; 0: every block takes part.
 * Every wait stays bounded; the context remains usable, and the next solve
 * after dec_set_barrier_test(ctx, 0, 0) starts from scratch.
 * Errors: DEC_ERR_ARG (NULL context, spin_limit < 0 or >= 2^32,
 * withhold_block not 0 or 1). */
dec_status dec_set_barrier_test(dec_ctx* ctx, int64_t spin_limit, int32_t withhold_block);

/* ---- an entry point that allocates no device memory ---- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that must not let a library allocate device memory: code that runs inside
 * a framework owning every device allocation through its own pool, under a
 * fixed device-memory budget, or where a cudaMalloc would synchronise the
 * device at a bad moment.  It computes the same three sums as dec_k_eff for
 * one instance, from arrays the caller already holds, and needs no context:
 *   q_in   = sum over edges (i,j) of w_e (T_i - T_j) signed by which end is a
 *            Dirichlet node on x = 0 (outflow of those nodes),
 *   q_out  = the same for Dirichlet nodes on x = 1 (inflow),
 *   energy = sum over edges of w_e (T_i - T_j)^2.
 *   device    CUDA device of the arrays; stream: cudaStream_t or NULL.
 *   E         [n_edges*2] int32 device: edges (i, j).
 *   w         [n_edges] f64 device: *1 of each edge (0 where cut).
 *   T         [n_nodes] f64 device: temperatures (Dirichlet values included).
 *   xyz       [n_nodes*3] f64 device; node_tag [n_nodes] uint8 device.
 *   out3      [3] f64 host or device: q_in, q_out, energy.
 * Its only scratch (per-block partial sums and an arrival counter) is a
 * fixed 768 KiB array inside the library's device image, present on every
 * GPU that loads the library until the process exits; n_edges may therefore
 * not exceed 67,108,864 (DEC_ERR_LIMIT beyond).  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) once.  Every
 * call clears the counter
 * and reuses the same array, so calls that overlap on the GPU (other
 * streams, other host threads, on the same device) race: serialise them.
 * The call returns after out3 is written.  No cudaMalloc or cudaFree is
 * made.  Errors: DEC_ERR_ARG (NULL pointer, n_edges < 1, bad device),
 * DEC_ERR_LIMIT, DEC_ERR_CUDA. */
dec_status dec_k_eff_edges_noalloc(int device, void* stream, const int32_t* E,
                                   int64_t n_edges, const double* w, const double* T,
                                   const double* xyz, const uint8_t* node_tag,
                                   double* out3);

#ifdef __cplusplus
}
#endif
#endif /* DEC_GB300_H */
