/*
 * al.h -- C ABI of the B300 actuator-line transfer operators.
 *
 * One coupling step of the two-way actuator-line method of arXiv 2609.39443
 * (Sec. 3.2, Algorithm 1 steps 1-5 and 7-8) on a uniform Cartesian fluid
 * grid:
 *   1. actuator points P_a and their velocities are given (Eqs.
 *      almKinematicCoupling, almActuatorPoint);
 *   2. the fluid velocity is sampled at P_a (Eq. almPreliminaryVelocity),
 *      the upstream sampling point P_s is built (Eq. almSamplingPoint) and
 *      the velocity (and, for free-surface flow, the volume fraction and
 *      mixture density rho = alpha rho1 + (1-alpha) rho2, Sec. 2.1) is
 *      sampled there (Eq. almRelativeVelocity);
 *   3. the Morison line force is evaluated and under-relaxed (Eqs.
 *      almLineForce, almForceRelaxation) and returned per CV as F_i = f_i L_i;
 *   4. the equal and opposite reaction is projected onto the grid with the
 *      truncated 2-D Gaussian, nearest-segment interpolation and per-node
 *      normalisation (Eqs. almProjectionPoint, almGaussian,
 *      almMomentumSource), so that sum_j S_j V = -sum_i F_i (Sec. 3.2.4).
 *
 * All functions return an int status: AL_OK (0) or a negative AL_ERR_*.
 * No function exits the process, throws, or traps the device.  Argument
 * errors are detected on the host before anything is enqueued.  Device-side
 * anomalies (points outside the grid, zero weights, ...) are counted in the
 * caller's status array and never stop the step.
 *
 * Memory: the caller owns every field, point and output buffer (device
 * memory, passed as plain pointers).  The library owns only its scratch
 * (per-point state, geometry, weights, bin masks), allocated by
 * al_create_grid / al_load_beams and freed by al_destroy.
 *
 * Streams: a `stream` argument is a cudaStream_t passed as void*; NULL is
 * the legacy default stream.  al_sample_drag_spread is asynchronous and
 * stream-ordered; it performs no allocation and no host synchronisation.
 */
#ifndef AL_H
#define AL_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define AL_OK              0
#define AL_ERR_ARG        -1   /* null pointer, bad size, inconsistent descriptor */
#define AL_ERR_CUDA       -2   /* a CUDA runtime call failed (message via al_last_cuda_error) */
#define AL_ERR_OOM        -3   /* device allocation failed */
#define AL_ERR_STATE      -4   /* call out of order (e.g. step before al_load_beams) */
#define AL_ERR_TIMEOUT    -5   /* a bounded wait ran out */
#define AL_ERR_CAPACITY   -6   /* request larger than a fixed capacity */

/* ---- enumerations ------------------------------------------------------ */
#define AL_FP32 0              /* fields, points, S and F stored as float  */
#define AL_FP64 1              /* ... stored as double                     */

#define AL_SAMPLE_TRILINEAR 0  /* trilinear interpolation of cell values   */
#define AL_SAMPLE_CELL      1  /* value of the single containing cell (the paper's operator) */
#define AL_SAMPLE_GAUSS     2  /* kernel-weighted volume average: sum_j g_j U_j / sum_j g_j over the
                                  cells whose centre lies within 3 eps of the point, g_j =
                                  exp(-(|C_j - p| / eps)^2) with the line's projection width eps
                                  (Eq. almGaussian; the smooth sampler proposed in Sec. 6); cells
                                  outside the grid do not enter; no centre within 3 eps: the
                                  containing cell */

#define AL_PROJ_NEAREST     0  /* al_beam_desc.proj_mode: the closest segment of each line */
#define AL_PROJ_INTEGRATED  1  /* ... every segment within 3 eps, integrated 3-D Gaussian */

#define AL_REFLECT_X_LO 1      /* al_beam_desc.wall_reflect bits: faces that reflect the kernel */
#define AL_REFLECT_X_HI 2
#define AL_REFLECT_Y_LO 4
#define AL_REFLECT_Y_HI 8
#define AL_REFLECT_Z_LO 16
#define AL_REFLECT_Z_HI 32

#define AL_DRAG_DISCRETE 0     /* Eq. almLineForce: |U_r| (C_dn U_n + C_dt U_t)        */
#define AL_DRAG_SPLIT    1     /* Eq. fext_drag: C_dn |U_n| U_n + C_dt |U_t| U_t        */

/* ---- device status counters (int[AL_STATUS_N], caller-owned, device) --- */
#define AL_ST_PA_OUTSIDE     0 /* actuator point outside the grid: no load this step   */
#define AL_ST_PS_OUTSIDE     1 /* sampling point outside the grid: no load (Sec. 3.2.5) */
#define AL_ST_FALLBACK       2 /* |u0_n| < tau: fallback upstream direction used       */
#define AL_ST_FALLBACK_ZERO  3 /* fallback direction parallel to the tangent: P_s = P_a */
#define AL_ST_ZERO_WEIGHT    4 /* node with w_k = 0: load deposited in its cell        */
#define AL_ST_DEPOSIT_LOST   5 /* zero-weight node outside the grid: load lost         */
#define AL_ST_REFINED        6 /* geometric decisions re-taken in FP64 (near ties)     */
#define AL_ST_IRREGULAR      7 /* lines projected by exhaustive segment search         */
#define AL_ST_SUPPORT        8 /* (cell, line) pairs within 3 eps: kernel-cell updates   */
#define AL_ST_REPLAYED       9 /* bricks that replayed recorded pairs instead of gathering them */
#define AL_ST_COLUMN        10 /* bricks whose both passes took the column march (AL_OPT_COLUMN) */
#define AL_ST_GUARD         15 /* bit flags of index guards in the column-march set-up that skipped an
                                  access (never expected to be set; tests require zero) */
#define AL_STATUS_N         16

/* ---- descriptors ------------------------------------------------------- */
typedef struct al_grid_s *al_grid;    /* opaque instance handle */

/* Uniform Cartesian grid.  Cell (i,j,k) has centre
 * origin + ((i+1/2) dx, (j+1/2) dx, (k+1/2) dx), volume dx^3, and linear
 * index i + nx*(j + ny*k) (x fastest) in every field array. */
typedef struct {
    int nx, ny, nz;            /* cells per axis, each >= 1 */
    double dx;                 /* cell size (m), > 0 */
    double origin[3];          /* grid corner (m) */
    int precision;             /* AL_FP32 or AL_FP64 */
    int has_alpha;             /* 1: a volume-fraction field is sampled and rho = alpha rho1 + (1-alpha) rho2 */
    double rho1, rho2;         /* phase densities (kg/m^3) */
    double rho_const;          /* density when has_alpha = 0 */
} al_grid_desc;

/* Actuator lines (one per beam).  Line l owns points line_off[l] ..
 * line_off[l+1]-1, ordered root to tip.  All arrays are HOST memory, read
 * during the call and copied; the caller may free them afterwards. */
typedef struct {
    int n_lines;               /* >= 0 */
    const int *line_off;       /* [n_lines + 1], non-decreasing, line_off[0] = 0 */
    const double *d;           /* [n_lines] drag reference length (m) */
    const double *cdn, *cdt;   /* [n_lines] normal / tangential drag coefficients */
    const double *eps;         /* [n_lines] Gaussian width (m), > 0; cut-off at 3 eps */
    const double *ell_s;       /* [n_lines] sampling distance (m), >= 0 */
    const double *alpha_f;     /* [n_lines] relaxation factor in (0, 1] */
    const double *cv_len;      /* [n_points] CV length L_i (m), the Delta s_i of Eq. almMomentumSource */
    double n_p[3];             /* sampling-plane normal: unit vector or 0 (no projection) */
    double g_up[3];            /* global upstream direction for the fallback */
    double tau;                /* fallback threshold on |u0_n| (m/s) */
    int sample_mode;           /* AL_SAMPLE_* (both samples use the same operator) */
    int drag_mode;             /* AL_DRAG_* */
    int tangents_given;        /* 1: al_step_in.tangent is used instead of the centreline tangent */
    /* Morison inertia (Eq. fext_addedmass; not part of the paper's model, which
     * has C_Mn = C_Mt = 0): per-line added-mass coefficients, both NULL for a
     * drag-only closure.  With them, f* gains rho A (C_Mt a_t + C_Mn a_n + a_f)
     * with A = pi d^2 / 4, a_f = (U - U_prev)/dt sampled at P_s with the same
     * operator, and a = a_f - a_b (the fluid's acceleration relative to the
     * beam) split along the tangent. */
    const double *cm_n, *cm_t; /* [n_lines] or NULL */
    /* Projection (Sec. 3.2.4): AL_PROJ_NEAREST is the paper's (each cell takes
     * the closest segment of each line, Eq. almProjectionPoint);
     * AL_PROJ_INTEGRATED is the variant Sec. 6 proposes: every segment whose
     * closest point lies within 3 eps adds the integral of the 3-D Gaussian
     * exp(-|x|^2/eps^2) / (pi^(3/2) eps^3) along it, the load per length
     * interpolated linearly between its nodes (closed forms in erf and exp of
     * the tangential coordinate; its integral across an infinite line is the
     * 2-D kernel of Eq. almGaussian).  It takes the segment weights pass and
     * records for every line; status[AL_ST_SUPPORT] then counts (cell,
     * segment) pairs. */
    int proj_mode;
    /* Kernel reflected at grid faces (the one-sided or reflected kernel that
     * Sec. 6 proposes, read as a mirror); 0 keeps the paper's truncated
     * kernel.  Bit 2a (2a + 1) of this AL_REFLECT_* mask makes the low (high)
     * face of axis a = x, y, z reflect.  The kernel is then also evaluated at
     * ghost cells up to ceil(3 eps / h) + 1 layers beyond such a face, and each
     * ghost's share goes to the grid cell it mirrors: kernel mass that falls
     * outside the domain comes back next to the wall instead of being spread
     * over the node's whole support by the normalisation.
     * Requirements (AL_ERR_ARG otherwise):
     *   - AL_PROJ_NEAREST;
     *   - ceil(3 eps / h) + 1 <= n on every reflecting axis.
     * The nodes must lie inside the grid box.  The brick weights pass and the
     * gather without records are used, whatever the options say.
     * status[AL_ST_SUPPORT] counts ghost pairs too. */
    int wall_reflect;
} al_beam_desc;

/* Inputs of one step: DEVICE pointers, element type per grid precision,
 * SoA (component c of the vector field is the array [c]).  Unused optional
 * pointers are NULL. */
typedef struct {
    const void *U[3];          /* [N_c] fluid velocity */
    const void *alpha;         /* [N_c] volume fraction (required iff has_alpha) */
    const void *P[3];          /* [N_p] actuator points (m) */
    const void *Pdot[3];       /* [N_p] actuator-point velocities (m/s) */
    const void *P_spread[3];   /* [N_p] optional positions for the projection (Algorithm 1,
                                  step 7: positions after the beam update); NULL: P */
    const void *tangent[3];    /* [N_p] optional tangents (used iff tangents_given) */
    /* inertia term only (al_beam_desc.cm_n set), otherwise ignored: */
    const void *U_prev[3];     /* [N_c] fluid velocity dt earlier; NULL: a_f = 0 */
    const void *Pddot[3];      /* [N_p] actuator-point accelerations (m/s^2); NULL: a_b = 0 */
    double dt;                 /* time between U_prev and U (s), > 0 when U_prev is given */
} al_step_in;

/* Outputs of one step: DEVICE pointers. */
typedef struct {
    void *S[3];                /* [N_c] momentum source (N/m^3), every cell overwritten */
    void *F[3];                /* [N_p] per-CV line load on the beam F_i = f_i L_i (N) */
    double *totals;            /* [6] or NULL: sum F (3), sum S V (3), FP64 */
    int *status;               /* [AL_STATUS_N] or NULL: counters, ADDED to (zero them first) */
} al_step_out;

/* ---- single-instance API ----------------------------------------------- */

/* Create an instance on the current CUDA device.  Validates the grid
 * descriptor (AL_ERR_ARG) and allocates the per-grid scratch. */
int al_create_grid(const al_grid_desc *desc, al_grid *out);

/* Copy the line table and per-line coefficients to the device, allocate the
 * per-point scratch and reset the relaxation state (the next step is
 * un-relaxed, f = f*).  May be called again to replace the lines.
 * Synchronous with respect to the host. */
int al_load_beams(al_grid g, const al_beam_desc *beams);

/* One coupling step (sampling, line force, relaxation, projection) on
 * `stream`.  S and F are fully overwritten; totals (if given) are
 * overwritten; status counters (if given) are incremented.  Updates the
 * instance's relaxation state f_prev.  Consecutive steps of one instance
 * must be ordered (same stream or explicit dependencies). */
int al_sample_drag_spread(al_grid g, const al_step_in *in, const al_step_out *out, void *stream);

/* Free everything the instance owns.  Synchronises the device first. */
int al_destroy(al_grid g);

/* Relaxation state export / import (checkpoint, eviction): f_prev as
 * 3 x N_p values of the grid precision in DEVICE memory, plus whether a
 * previous force exists.  Stream-ordered on `stream`. */
int al_get_state(al_grid g, void *f_prev_dev, int *has_prev, void *stream);
int al_set_state(al_grid g, const void *f_prev_dev, int has_prev, void *stream);

/* Phase timing (tracing).  When enabled, each step records CUDA events on
 * its stream at the phase boundaries below; al_trace_last waits for the
 * last step's final event and returns the elapsed milliseconds of each
 * phase.  Off by default; enabling creates AL_TRACE_N + 1 events. */
#define AL_PH_POINTS    0      /* sampling, line force, segment geometry, line certificates */
#define AL_PH_MASK      1      /* brick masks */
#define AL_PH_WEIGHTS   2      /* nodal weights w_k */
#define AL_PH_NORMALISE 3      /* f^_k = F_k / w_k */
#define AL_PH_SPREAD    4      /* momentum source S (every cell), zero-weight deposits */
#define AL_PH_TOTALS    5      /* FP64 totals */
#define AL_TRACE_N      6
int al_trace_enable(al_grid g, int on);
int al_trace_last(al_grid g, float *ms /* [AL_TRACE_N] */);

/* Execution options of an instance (results agree within the parity
 * tolerances whichever is chosen; the autotuner picks them per workload).
 * AL_OPT_WEIGHTS selects how the nodal weights w_k (Sec. 3.2.4) are summed:
 *   AL_WEIGHTS_BRICK (default): cell-centric over the projection bricks, every
 *     (cell, line) pair once, as exact fixed-point integers (deterministic);
 *   AL_WEIGHTS_SEGMENT: segment-centric (one warp per segment over the cells
 *     between its bisector planes, compensated FP32) for lines with a walk
 *     certificate, the brick pass for the others.
 * Takes effect at the next step; AL_ERR_ARG for an unknown option or value. */
#define AL_OPT_WEIGHTS      1
#define AL_WEIGHTS_BRICK    0
#define AL_WEIGHTS_SEGMENT  1
/* AL_OPT_BRICK_Z: height in cells (4, 8 or 16; default 8) of the 16 x 16 x h
 * bricks the projection tiles the grid into (the bins of the line masks and
 * the shared-memory tiles of both brick passes). */
#define AL_OPT_BRICK_Z      2
/* AL_OPT_SPREAD_CTAS (batches only, al_batch_set_option): persistent CTAs per
 * SM of the batched brick passes, 0 = as many as fit. */
#define AL_OPT_SPREAD_CTAS  3
/* AL_OPT_SPREAD selects the projection of Eq. almMomentumSource:
 *   AL_SPREAD_GATHER (default): cell-centric pass per brick, every cell of S
 *     written once by one thread, its sources summed in line order, or, when
 *     records are replayed (AL_OPT_RECORD) or the integrated projection is
 *     chosen, as exact fixed-point integers, whose sum does not depend on
 *     the order (bitwise reproducible either way);
 *   AL_SPREAD_SCATTER: for comparison, lines with a walk certificate add
 *     their sources segment by segment with float atomics (summation order,
 *     hence the last bits, vary run to run); the other lines and the
 *     zero-weight deposits go through the gather first.  Single instances
 *     only (a batch always gathers). */
#define AL_OPT_SPREAD       4
#define AL_SPREAD_GATHER    0
#define AL_SPREAD_SCATTER   1
/* AL_OPT_RECORD (default 1; 0: off; 2: no records, but the gather sums in
 * the fixed point a replay uses, which gives the replay's bits, for checks):
 * with AL_WEIGHTS_SEGMENT and the gather, the
 * segment pass records every (cell, segment) pair it finds inside the 3 eps
 * support (cell, node, the two node weights), in a region per brick sized
 * from the previous step's counts, and the gather replays the records of
 * its brick instead of recomputing those pairs.  A brick whose pairs did not
 * fit its region (the first step, a beam that moved into it) is recomputed,
 * with the same bits.  The record arena (16 bytes per pair in FP32, 24 in
 * FP64, sized from the lines' length and kernel width) is held only while
 * records can be used: al_load_beams, al_set_option (AL_OPT_WEIGHTS,
 * AL_OPT_RECORD) and al_autotune allocate it when the options turn records
 * on (segment weights with AL_OPT_RECORD = 1, or AL_PROJ_INTEGRATED with
 * AL_OPT_RECORD = 1) and free it when they turn them off, synchronising the
 * device; set these options before adding the instance to a batch. */
#define AL_OPT_RECORD       5
/* AL_OPT_COLUMN (default 1; 0: off): the column march of FP32 instances
 * with the nearest-segment projection, no reflecting face and the gather.
 * A line whose segments all climb (D_z / |D| >= 0.8 in cell units) and
 * whose bisector signs are certified monotone over a brick's candidate
 * segments (k_lines) takes it; a brick whose candidate lines all take it
 * computes both passes by marching each column up the brick: the closest
 * segment of a cell only moves up the line as z grows, one bisector test
 * per cell instead of a search, with the same exact near-tie decisions as
 * the brick passes.  Other bricks take the brick passes for both passes
 * (the weights option then applies to their other lines).  The results
 * agree within the parity tolerances either way. */
#define AL_OPT_COLUMN       6
/* AL_OPT_OWN_X0 / AL_OPT_OWN_X1 (defaults 0 and -1 = nx): the instance owns
 * the cells with x index in [x0, x1) of its grid, one slab of a
 * decomposition of a larger grid along x (al_slab_plan); x0 a multiple of 16
 * (a brick column), x1 too or nx.  The weights pass adds only the owned
 * cells' contributions (partial sums, exchanged between slabs with
 * al_weights_get / al_weights_set between al_step_begin and al_step_end),
 * and the spread writes only the owned cells of S (the others are left as
 * they are).  A slab takes the brick weights, the gather and no records
 * whatever the other options say; it refuses a reflecting face, the
 * integrated projection (AL_ERR_STATE at the step) and batches. */
#define AL_OPT_OWN_X0       7
#define AL_OPT_OWN_X1       8
int al_set_option(al_grid g, int option, int value);

/* One coupling step with the fields and results in host memory (Algorithm 1
 * steps 1-5 and 7-8 with the transfers a coupled solver makes every step):
 * on `stream`, copy each input of host_in into the same field of dev_in
 * (U, alpha, P, Pdot, and P_spread, tangent, U_prev, Pddot where dev_in has
 * them; host_in's pointers: pinned host memory, the same layout and sizes),
 * run the step of al_sample_drag_spread on dev_in / dev_out, and copy S and
 * F of dev_out into host_out's S and F (pinned host memory; a NULL host
 * field is not copied).  totals and status stay where dev_out puts them.
 * The step of a call waits for the step of the previous al_step_host call
 * on the same instance, whatever its stream: a caller that alternates two
 * streams and two sets of device buffers overlaps the copies of one step
 * with the step and the copies of the other, with the steps in call order.
 * A buffer set must not be reused before the call that last used it has
 * completed on its stream (same stream: ordered).  Returns AL_ERR_ARG for
 * a NULL descriptor and the errors of al_sample_drag_spread; allocates no
 * device memory (one event, created at the first call). */
int al_step_host(al_grid g, const al_step_in *host_in, const al_step_out *host_out, const al_step_in *dev_in,
                 const al_step_out *dev_out, void *stream);

/* Kernels this instance's al_sample_drag_spread calls have launched so far
 * (cumulative, counted on the host as they are enqueued; the autotuner's
 * trial steps count too).  Returns AL_ERR_ARG for a NULL argument. */
int al_launches(al_grid g, long long *n);

/* Autotuner: runs the caller's step (same in/out as al_sample_drag_spread)
 * under every combination of AL_OPT_WEIGHTS (with AL_WEIGHTS_SEGMENT: with
 * and without AL_OPT_RECORD), AL_OPT_BRICK_Z and, for instances that can take
 * it, AL_OPT_COLUMN on and off: one warm-up step, then `trials` steps each
 * timed alone with CUDA events on `stream` after a write of twice the L2
 * (the cold cache a coupled solver leaves between calls); a combination's
 * time is its fastest step, and the fastest combination is kept.  The
 * relaxation state and the status counters are restored afterwards; S, F
 * and totals hold the last trial's outputs.  *choice (optional) = 10000 *
 * column march + 1000 * records + 100 * weights mode + brick height.
 * Synchronises the stream; allocates a temporary copy of the relaxation
 * state and the L2-sized buffer (when that allocation fails, the steps are
 * timed without it). */
int al_autotune(al_grid g, const al_step_in *in, const al_step_out *out, int trials, void *stream, int *choice);

/* Sizes of an instance: cells and points. */
int al_sizes(al_grid g, long long *n_cells, long long *n_points, int *n_lines);

/* Device bytes the library holds for the instance.  It holds at most three
 * allocations: per-grid scratch (al_create_grid), per-point scratch and line
 * table (al_load_beams) and the record arena while records are on
 * (AL_OPT_RECORD); each is counted rounded up to whole 2 MiB pages, the unit
 * the driver commits.  The caller's fields, points and outputs are not
 * included.  An admission controller adds them to this figure to bound what
 * a resident instance takes. */
int al_footprint(al_grid g, unsigned long long *bytes);

/* Quasi-static reconstruction of the beam side (the structural check of the
 * wave-flume case, Sec. 7): each node's load F_k (per-CV line force, e.g.
 * the F of the last al_sample_drag_spread) acts as a static point load on a
 * linear Euler-Bernoulli cantilever per line, clamped at the line's first
 * node and straight along the unit vector `axis` in its rest positions P0.
 * With stations a_k = (P0_k - P0_root).axis and only the load normal to the
 * axis bending the beam,
 *   P_out_i = P0_i + sum_k F_perp,k g(a_i, a_k) / EI_l,
 *   g(x, a) = x^2 (3a - x) / 6 (x <= a),  a^2 (3x - a) / 6 (x >= a).
 * Feeding P_out back as the next step's positions closes a coupled step on
 * the GPU (quasi-static structure, no beam dynamics).
 * P0, F, P_out: DEVICE SoA in the grid's precision, n_points each (P_out may
 * not alias P0 or F).  EI: HOST [n_lines] bending stiffness (N m^2), > 0,
 * copied to the grid's device buffer.  axis: host, unit length.
 * Stream-ordered on `stream`; AL_ERR_ARG for a bad argument, AL_ERR_STATE
 * before al_load_beams. */
int al_beam_quasistatic(al_grid g, const double *EI, const double axis[3], const void *const P0[3],
                        const void *const F[3], void *const P_out[3], void *stream);

/* ---- batched form ------------------------------------------------------ */
/* Many independent instances advanced together: every phase of the step is
 * one launch over the work items of all instances (points, lines, bricks),
 * each item mapped to its instance through a device work list, and the
 * projection runs as a persistent kernel over the bricks of every instance.
 * With graphs on, the launch sequence is captured once into a CUDA graph and
 * replayed.  Results are bitwise those of al_sample_drag_spread on each
 * instance alone. */
typedef struct al_batch_s *al_batch;

int al_batch_create(al_batch *out);
/* Register an instance with the device buffers of its steps; the buffers and
 * the instance must stay valid while the batch is used.  All instances of a
 * batch share one precision.  The step descriptors are copied. */
int al_batch_add(al_batch b, al_grid g, const al_step_in *in, const al_step_out *out);
/* Reserve n_slots slots of the given precision (before commit); slots beyond
 * the added instances start empty and are bound later with al_batch_assign. */
int al_batch_reserve(al_batch b, int n_slots, int precision);
/* Freeze the batch: upload the work list (synchronous).  use_graph: capture
 * the step into a CUDA graph on the first al_batch_run.  spread_ctas_per_sm:
 * persistent grid of the projection (0: occupancy maximum). */
int al_batch_commit(al_batch b, int use_graph, int spread_ctas_per_sm);
/* One coupling step of every instance, stream-ordered on `stream`. */
int al_batch_run(al_batch b, void *stream);
/* One coupling step of the n_idx instances idx[0..n_idx) (distinct indices
 * in add order), without a graph: the selection's work list is copied from a
 * ring of 8 pinned slots allocated at commit, so a call waits only when the
 * slot it reuses is still being read by a step 8 calls back.  Instances with
 * steps in flight on other streams must not be selected again until those
 * steps complete (steps of one instance are ordered). */
int al_batch_run_subset(al_batch b, const int *idx, int n_idx, void *stream);
/* Bind (g non-NULL) or clear (g NULL) one slot of a committed batch without a
 * graph; the slot's descriptor is copied on `stream`, so later runs on that
 * stream see it.  The previous binding must not have steps in flight. */
int al_batch_assign(al_batch b, int slot, al_grid g, const al_step_in *in, const al_step_out *out, void *stream);
int al_batch_destroy(al_batch b);

/* Batch execution options after commit: AL_OPT_BRICK_Z (the brick height of
 * every instance inside the batch; each instance keeps its own for
 * al_sample_drag_spread) and AL_OPT_SPREAD_CTAS.  Rebuilds the device work
 * lists (synchronises the device) and drops a captured graph. */
int al_batch_set_option(al_batch b, int option, int value);

/* Batch autotuner: times al_batch_run under every brick height and
 * persistent grid size (`trials` runs each after a warm-up) and keeps the
 * fastest; every instance's relaxation state and status counters are
 * restored.  *choice (optional) = 10 * brick height + CTAs per SM (0 = as
 * many as fit).  Every slot must be bound. */
int al_batch_autotune(al_batch b, int trials, void *stream, int *choice);

/* Kernels the batch's al_batch_run / al_batch_run_subset calls have
 * launched so far (cumulative, counted on the host: an enqueue counts its
 * kernels, a graph replay the kernels captured in the graph; the batch
 * autotuner's trial runs count too).  Returns AL_ERR_ARG for a NULL argument. */
int al_batch_launches(al_batch b, long long *n);

/* ---- the step in two phases (decomposition along x, Sec. 3.2.5) ------- */
/* al_step_begin runs a step up to the nodal weights (Algorithm 1 steps 1-3:
 * points, line geometry, bins and the weights pass); al_step_end runs the
 * rest (normalisation, spread and totals).  Together they equal
 * al_sample_drag_spread (same in / out).  Between them the nodal weights of
 * the brick pass, w_k / (eta0 V) as unsigned fixed-point integers in units
 * of 2^-wshift of their line (one unsigned long long per point, a line's
 * shift being a function of its geometry only), can be read and replaced:
 * the slabs of a decomposition sum their partial weights there (an exact,
 * order-free integer all-reduce) before each ends its step.  al_weights_get
 * / _set copy them to / from a DEVICE array of N_p (stream-ordered);
 * AL_ERR_STATE unless the instance takes the brick weights (a slab always
 * does). */
int al_step_begin(al_grid g, const al_step_in *in, const al_step_out *out, void *stream);
int al_step_end(al_grid g, const al_step_in *in, const al_step_out *out, void *stream);
int al_weights_get(al_grid g, void *dst, void *stream);
int al_weights_set(al_grid g, const void *src, void *stream);

/* Slab plan of rank `rank` of `n_ranks` for a grid split along x (host only,
 * no device work): the owned cells [x0, x1) are whole brick columns dealt
 * evenly; the local grid [lx0, lx1) adds a halo of `halo` cells each side
 * (clipped to the grid), with halo = ceil((ell_s + 3 eps + L) / h) + 2
 * rounded up to a multiple of 16, the largest over the lines (ell_s the
 * sampling distance, L the longest segment): every point whose segments come
 * within 3 eps of an owned cell samples inside the local grid.  A line is
 * taken (whole) when its points' x range widened by 3 eps + L + h meets the
 * owned cells; `lines` (optional, n_lines entries) receives their indices in
 * increasing order, and owner (optional, N_p entries) the rank whose owned
 * cells contain each point's x (clamped to the grid).  P_host: HOST, 3 x N_p
 * doubles, the positions the projection uses.  AL_ERR_ARG for a bad
 * descriptor or rank. */
typedef struct {
    int x0, x1;          /* owned cells along x, global indices */
    int lx0, lx1;        /* the local grid's cells along x, global indices */
    int halo;            /* halo width in cells */
    int n_lines;         /* lines the rank takes */
} al_slab;
int al_slab_plan(const al_grid_desc *grid, const al_beam_desc *beams, const double *P_host, int n_ranks, int rank,
                 al_slab *out, int *lines, int *owner);

/* ---- serving: continuous batching of coupling-step requests ------------ */
/* Many simulations send coupling-step requests (the actuator-point positions
 * of their next step, Algorithm 1 step 1) as they arrive; the server keeps
 * each admitted simulation resident (its instance bound to a slot of one
 * batch, with the caller's device fields and outputs) and advances every
 * resident simulation that has a queued request and no step in flight in
 * one batched launch sequence, a wave; waves alternate between two streams
 * of the server's own, so one forms and launches while the previous one
 * runs.  A simulation's requests run in submission order, one at a time, and
 * a served step gives the bits of the same step run in a batch.  Per wave
 * the requests' positions travel in one host-to-device copy and the line
 * forces in one device-to-host copy (packed in pinned staging buffers). */
typedef struct al_server_s *al_server;
typedef struct {
    unsigned long long hbm_budget; /* device bytes the resident simulations may hold: for each, the
                                      library's (al_footprint of its instance) plus what the caller
                                      declares for its own buffers at admission */
    int max_sims;                  /* slots: simulations resident at a time, >= 1 */
    int max_wave;                  /* simulations advanced by one wave, 1 .. max_sims */
    int max_points;                /* points one wave carries at most (sizes the staging buffers);
                                      no simulation may have more */
    int precision;                 /* AL_FP32 or AL_FP64, shared by every simulation */
} al_server_desc;
int al_server_create(const al_server_desc *desc, al_server *out);
/* Admit a simulation: creates its instance (al_create_grid, al_load_beams)
 * and binds it to a free slot.  in / out are its DEVICE buffers as for
 * al_sample_drag_spread (caller-owned, valid until al_server_release;
 * in->P is overwritten by each request's positions); caller_bytes is what
 * those buffers take.  AL_ERR_CAPACITY, with nothing kept, when no slot is
 * free, N_p > max_points, or footprint + caller_bytes would pass the
 * budget.  Synchronous. *sim receives the slot. */
int al_server_admit(al_server s, const al_grid_desc *grid, const al_beam_desc *beams, const al_step_in *in,
                    const al_step_out *out, unsigned long long caller_bytes, int *sim);
/* Queue one coupling step of simulation sim: P_host (HOST, 3 x N_p SoA in the
 * precision, read when the step is launched) and F_host (HOST, 3 x N_p,
 * written when the step is retired by a poll); tag identifies it in
 * al_server_poll.  Both buffers stay valid until then. */
int al_server_submit(al_server s, int sim, const void *P_host, void *F_host, long long tag);
/* Progress: retire the waves that completed (their forces unpacked into the
 * requests' F_host), then launch a wave on each free stream.  Writes up to
 * max_done tags of completed requests (the rest are reported by later
 * polls).  wait != 0: if nothing has completed, wait for the oldest wave in
 * flight, polling its event for at most the server's wait limit; when the
 * limit runs out, AL_ERR_TIMEOUT (*n_done = 0, the wave still in flight and
 * retired by a later poll). */
int al_server_poll(al_server s, long long *done_tags, int max_done, int *n_done, int wait);
/* Evict: waits (within the wait limit; AL_ERR_TIMEOUT otherwise, the
 * simulation still resident) for the simulation's step in flight, unbinds
 * and destroys its instance, frees its slot and budget share.  AL_ERR_STATE
 * while requests are still queued. */
int al_server_release(al_server s, int sim);
/* The limit of the waits of al_server_poll and al_server_release, in seconds
 * (0 <= seconds <= 1e6; 10 at creation).  AL_ERR_ARG outside that range. */
int al_server_set_timeout(al_server s, double seconds);
/* Device bytes held by the resident simulations (as counted at admission)
 * and how many are resident (optional). */
int al_server_footprint(al_server s, unsigned long long *bytes, int *resident);
/* Waves launched so far and the steps they carried (mean wave = steps / waves). */
int al_server_stats(al_server s, long long *waves, long long *steps);
int al_server_destroy(al_server s);

/* ---- line forces without device allocation ----------------------------- */
/* The paper has no counterpart of this entry point.  It exists for callers
 * that cannot allocate device memory where they need the line forces: code
 * running under an allocator that forbids device allocation after start-up
 * (a fixed, pre-reserved pool; a real-time loop that cannot take an
 * allocation's latency or its possible implicit synchronisation), or a
 * plug-in whose host application owns all device memory and hands it only
 * buffers.  It computes F = f L for every actuator point with the point
 * evaluation of al_sample_drag_spread (sampling, upstream direction, Morison
 * drag, and the inertia term when beams->cm_n / cm_t are given, with
 * in->U_prev, in->Pddot and in->dt as in al_step_in; F[3] overwritten),
 * relaxed against f_prev (device, 3 arrays of N_p) when f_prev is non-NULL
 * and un-relaxed (f = f*) when it is NULL, without an al_grid and without
 * allocating: no cudaMalloc, no cudaFree, nothing else that allocates device
 * memory.  All buffers are the caller's (DEVICE pointers as in al_step_in;
 * P_spread and the projection are not used, so proj_mode and wall_reflect
 * are only checked).  The descriptors are checked by the rules of
 * al_create_grid and al_load_beams (AL_ERR_ARG); AL_SAMPLE_GAUSS is not
 * offered here (AL_ERR_ARG): it needs an al_grid.  A line set without points
 * (n_lines = 0, line_off may then be NULL) returns AL_OK after zeroing the
 * shared counters (when status is NULL).
 * The host arrays of `beams` are copied into one fixed __device__ array of
 * about 1 MiB (1,065,472 bytes) held by every GPU that loads the library until the process
 * exits; lines beyond AL_NOALLOC_MAX_LINES or points beyond
 * AL_NOALLOC_MAX_POINTS are rejected with AL_ERR_CAPACITY.  The first call
 * on each device looks up that array's device address (once, with the
 * device current).  Every call shares the array and it keeps the last call's
 * contents: calls whose work overlaps on the GPU (unordered streams) race,
 * so order them.  status (device int[AL_STATUS_N], optional) is added to as
 * in al_sample_drag_spread; when NULL, counters in the shared array are used
 * (zeroed by the call).  Stream-ordered on `stream`; a CUDA failure returns
 * AL_ERR_CUDA with its text in al_last_cuda_error. */
#define AL_NOALLOC_MAX_POINTS 65536
#define AL_NOALLOC_MAX_LINES  4096
int al_line_forces_noalloc(const al_grid_desc *grid, const al_beam_desc *beams, const al_step_in *in,
                           const void *const f_prev[3], void *const F[3], int *status, void *stream);

/* Human-readable text of a status code (static storage). */
const char *al_error_string(int code);

/* Text of the last CUDA error seen by this thread (static per thread). */
const char *al_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AL_H */
