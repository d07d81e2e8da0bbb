/*
 * ade_sph.h -- C ABI of the GB300 SPH advection-dispersion library (libade_sph.so).
 *
 * The library evaluates, on one GPU, the SPH form of the Lagrangian advection-dispersion
 * equation of Klapp et al., "Consistent SPH simulations of the anisotropic dispersion of a
 * contaminant plume" (arXiv 2108.09488):
 *   Sec. 2.1, Eq. 1-3   dC/dt = div(D grad C) - C div v, dx/dt = v, with the dispersion tensor
 *                       D_ij = (aT|v| + Dm) delta_ij + (aL - aT) v_i v_j / |v|;
 *   Sec. 2.2, Eq. 4-5   its SPH pair sum over the neighbours within the kernel support;
 *   Sec. 2.3, Eq. 7     the Wendland kernels (C4 of the paper, support h; C2, support 2h);
 *   Sec. 2.4, Eq. 8-10  the predictor-corrector update and the time-step rule.
 * Neighbours come from a cell-linked list rebuilt every step by a stable radix sort of the
 * particles by cell key.
 *
 * Conventions for every entry point:
 *   - All functions are extern "C", take plain pointers and sizes and never throw.
 *   - Pointers named *_dev are device pointers; *_host are host pointers.  The caller owns every
 *     buffer it passes (particle state, workspace, outputs).  The library owns only the opaque
 *     context and its CUDA graph.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device work is enqueued on
 *     it; only calls that return host values (ade_get_stats, ade_count_pairs, ade_step_timed,
 *     ade_closed_form_error, and ade_run when asked for stats) wait.
 *   - Return value: ADE_OK (0) or a negative ADE_ERR_* code; ade_last_error() gives the message
 *     of the last failure on the calling thread.  A context stays usable after ADE_ERR_NUMERIC.
 *   - Positions are fixed-point: coordinate u in [0, L) is the uint32 word round(u/L * 2^32)
 *     mod 2^32, stored axis-major ([dim][n]).  The difference of two words read as int32 is
 *     the minimum-image separation in the periodic box (Sec. 3 uses periodic borders).
 *   - Particle arrays are in the caller's particle order; the sorted order is internal.
 */
#ifndef ADE_SPH_H
#define ADE_SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADE_OK 0
#define ADE_ERR_ARG (-1)      /* invalid argument or unsupported configuration */
#define ADE_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define ADE_ERR_NUMERIC (-3)  /* a NaN or Inf concentration was produced */
#define ADE_ERR_TIMEOUT (-4)  /* a bounded device wait gave up (reserved: no kernel of this
                                 * version waits on another block) */
#define ADE_ERR_CAPACITY (-5) /* workspace or a static limit too small */
#define ADE_ERR_STATE (-6)    /* call out of order (e.g. no particles bound) */

#define ADE_WENDLAND_C2 0 /* W = B (1-q)^4 (1+4q), q = r/(2h): support 2h */
#define ADE_WENDLAND_C4 1 /* Eq. 7: W = B (1-q)^6 (1+6q+35q^2/3), q = r/h: support h */

#define ADE_FLAG_DIRECT 1u /* interaction kernel: direct walk over global memory (default) */
#define ADE_FLAG_TILED 2u  /* interaction kernel: shared-memory tiles where the grid allows */
#define ADE_FLAG_BRANCHED 4u /* interaction kernel: direct walk branching on the support test */
#define ADE_FLAG_TRIMMED 8u  /* with DIRECT or BRANCHED (or alone = DIRECT): each particle visits only
                                the stencil cells within (1 + 2^-12) H of itself; the skipped
                                candidates contribute exactly 0, so results are bitwise unchanged
                                (square or cubic boxes; other boxes walk the full stencil) */
#define ADE_FLAG_PAIRED 16u  /* with DIRECT or BRANCHED (alone = DIRECT), optionally TRIMMED: that
                                direct walk with two adjacent sorted particles per thread, which
                                share one candidate stream (the union of their stencil ranges) and
                                evaluate both terms with packed FP32x2 instructions; candidates
                                outside a particle's own range contribute exactly 0, so results are
                                bitwise those of the one-particle walk.  Not in velocity-field
                                mode. */

#define ADE_DT_LAMBDA_MAX 0 /* dt = coef h^2 / lambda_max(D) */
#define ADE_DT_TRACE 1      /* Eq. 10: dt = coef h^2 / (D_xx + D_yy [+ D_zz]) */

typedef struct ade_ctx ade_ctx;

/* Problem parameters (Sec. 2-3).  Passed by pointer, copied into the context. */
typedef struct ade_params {
    int dim;           /* 2 or 3 */
    int kernel;        /* ADE_WENDLAND_C2 or ADE_WENDLAND_C4 */
    double box[3];     /* periodic box side per axis (box[2] ignored in 2D) */
    double h;          /* smoothing length; support radius 2h (C2) or h (C4) */
    double alpha_L;    /* longitudinal dispersivity (Eq. 3) */
    double alpha_T;    /* transverse dispersivity (Eq. 3) */
    double D_m;        /* molecular diffusion (Eq. 3) */
    double v[3];       /* uniform flow velocity (Sec. 3: constant in space and time) */
    double mass;       /* particle mass m_b (uniform) */
    double rho;        /* particle density rho_b (uniform; rhobar_ab = rho) */
    double gamma;      /* Gamma of Eq. 5; <= 0 selects dim + 2 (4 in 2D as printed) */
    double dt;         /* time step; <= 0 selects the rule in dt_rule */
    int dt_rule;       /* ADE_DT_LAMBDA_MAX or ADE_DT_TRACE */
    double dt_coef;    /* coefficient of the rule; <= 0 selects 0.1 (Eq. 10) */
    int cell_subdiv;   /* cells per support radius along each axis, 1..6; 0 = automatic */
    unsigned flags;    /* 0 (library's choice), ADE_FLAG_DIRECT, ADE_FLAG_TILED, ADE_FLAG_BRANCHED,
                          or ADE_FLAG_TRIMMED alone or with DIRECT or BRANCHED */
    double vmax;       /* 0: uniform velocity v.  > 0: velocity-field mode -- each particle carries
                          its own constant velocity (ade_set_velocity_field), |v_a| <= vmax; v is
                          then unused, the dt rules take |v| = vmax, and the cell grid is sized for
                          H + dt vmax (see ade_set_velocity_field). */
    double tau;        /* 0: Eq. 1 (Fick).  > 0: Cattaneo's form, Eq. 14 (Sec. 5), with relaxation
                          time tau: tau d2C/dt2 + dC/dt = R(C), advanced as dC/dt = Q,
                          tau dQ/dt = R - Q by the midpoint rule of Eq. 8-9 (see ade_set_flux); the
                          dt rules are capped at tau.  Uniform velocity, single plume only. */
} ade_params;

/* FP64 diagnostics of the current state. */
typedef struct ade_stats {
    double mass;      /* sum_a m_a C_a */
    double c_min;     /* min_a C_a (negative values are reported, never clipped) */
    double c_max;     /* max_a C_a */
    double t;         /* simulated time */
    long long step;   /* steps taken */
    long long pairs;  /* ordered in-support pairs per rate evaluation (last counted) */
    int status;       /* 0, or ADE_ERR_NUMERIC if a NaN/Inf was produced */
} ade_stats;

/* Derived configuration of a context. */
typedef struct ade_info {
    double support;   /* support radius H */
    double dt;        /* time step in use */
    double D[9];      /* dispersion tensor (dim x dim, row-major, Eq. 3) */
    int nc[3];        /* cells per axis */
    int ncells;       /* total cells */
    int cell_subdiv;  /* cells per support radius in use */
    int stencil_rows; /* rows of cells visited per particle */
    int sort_passes;  /* radix-sort passes per cell build */
    int variant;      /* interaction kernel: 0 direct walk (branch-free), 1 shared-memory tiles,
                         2 direct walk branching on the support test, 3 and 4 the two direct
                         walks with per-particle trimmed rows */
    int tile[3];      /* target cells per tile (tiled variant) */
    int tile_capacity;/* staged particles per tile (tiled variant) */
    size_t workspace_bytes;
    double skin;      /* velocity-field mode: cell-grid margin dt vmax (+ rounding) added to H */
} ade_info;

/* Device workspace needed for n particles with parameters p (bytes, 256-byte aligned). */
int ade_workspace_bytes(const ade_params *p, int n, size_t *bytes);

/* Create a context bound to the caller's particle state and workspace.
 *   xq_dev [dim][n] uint32 fixed-point positions, C_dev [n] float concentrations: updated in
 *   place by ade_step / ade_run.  workspace_dev: at least ade_workspace_bytes(p, n) bytes,
 *   256-byte aligned.  All three must stay valid until ade_destroy.  No device work is issued. */
int ade_init_particles(ade_ctx **out, const ade_params *p, int n, uint32_t *xq_dev,
                       float *C_dev, void *workspace_dev, size_t workspace_bytes);

/* Configuration in use (support radius, dt, D, grid).  Host only. */
int ade_get_info(const ade_ctx *ctx, ade_info *info_host);

/* Cell-linked list of the current positions: cell keys, stable radix sort by key (ties keep the
 * caller's particle order), sorted particle copy and the cell start table. */
int ade_build_cells(ade_ctx *ctx, void *stream);

/* Copy the last cell build out: perm_dev [n] (caller index at each sorted position) and
 * cell_start_dev [ncells + 1] (cell c holds sorted positions cell_start[c] .. cell_start[c+1]-1).
 * Either pointer may be NULL. */
int ade_get_cells(ade_ctx *ctx, uint32_t *perm_dev, uint32_t *cell_start_dev, void *stream);

/* Eq. 4 at the current state for every particle: builds the cell list, then writes dC/dt into
 * dCdt_dev [n] (caller order). */
int ade_dispersion_rate(ade_ctx *ctx, float *dCdt_dev, void *stream);

/* Number of ordered in-support pairs (b != a, |x_ab| < H) of the current state, the unit of the
 * interaction count: builds the cell list and runs one counting evaluation; waits for the stream. */
int ade_count_pairs(ade_ctx *ctx, long long *pairs_host, void *stream);

/* nsteps predictor-corrector steps (Eq. 8-9), each: cell build, rate at level l with the fused
 * predictor, rate at level l+1/2 with the fused corrector (which writes one partial of sum C,
 * min C and max C per warp), and the fold of those partials into the step's FP64 statistics. */
int ade_step(ade_ctx *ctx, int nsteps, void *stream);

/* As ade_step, replaying captured CUDA graphs: one graph of 32 steps per whole multiple of 32
 * (no launch gap between those steps) and a graph of one step for the rest (each captured on the
 * first call that needs it, outside any capture of the caller's).  With stats_host non-NULL it
 * waits for the stream and fills in the last step's statistics (those of the state it wrote; with
 * nsteps = 0, those of the current state as ade_get_stats); with NULL it only enqueues. */
int ade_run(ade_ctx *ctx, int nsteps, ade_stats *stats_host, void *stream);

/* One step (as ade_step) bracketed by CUDA events on `stream`; waits for it and returns the device
 * time of each phase in phase_ms_host[4] = {cell build, predictor rate, corrector rate, fold of
 * the statistics} (milliseconds).  Used for per-kernel roofline measurements. */
int ade_step_timed(ade_ctx *ctx, double *phase_ms_host, void *stream);

/* Kernel launches one step enqueues: the cell build (count, one scan launch over tiles of 4096
 * cells, placement, ordering), the velocity-field gather in velocity-field mode, the two rate
 * launches and the statistics fold. */
int ade_launches_per_step(const ade_ctx *ctx, int *launches);

/* FP64 mass, min and max of the current concentrations (recomputed from C, so a caller's own
 * writes to C count); waits for the stream. */
int ade_get_stats(ade_ctx *ctx, ade_stats *stats_host, void *stream);

/* Error of the current state against the closed form of Sec. 3 (Eq. 12-13 in 2D, the same
 * Gaussian with covariance w^2 I + 2 t D in 3D), centre x0 + v t, summed over image shells
 * |n_i| <= nimg, evaluated in FP64 on the device.  out_host[4] = {L2 = sqrt(sum_a V_a
 * (C_a - C_an)^2) with V_a = m/rho, Linf = max |C_a - C_an|, RMSE of C/C0, max |C_an|}.
 * Waits for the stream. */
int ade_closed_form_error(ade_ctx *ctx, const double *x0_host, double w, double C0,
                          int nimg, double *out_host, void *stream);

/* Autotuner for a context created with cell_subdiv = 0 and flags = 0: times the cell build plus
 * two evaluations of Eq. 4 (the work of a step) for every cell subdivision (1..6 cells per
 * support radius) and every interaction variant (branch-free or branched direct walk, each with
 * full or trimmed rows, the paired branch-free walk with full or trimmed rows, and shared-memory
 * tiles), then re-times the three fastest in three interleaved rounds and keeps the fastest;
 * results change only in summation order (not at all between the full, trimmed and paired
 * walks).  The particle state is not modified; waits; best_ms_host (the time of a build plus two
 * evaluations) may be NULL. */
int ade_autotune(ade_ctx *ctx, double *best_ms_host, void *stream);

/* Change alpha_L, alpha_T and D_m (Eq. 3) of a context, keeping its time step, grid and state. */
int ade_set_dispersivity(ade_ctx *ctx, double alpha_L, double alpha_T, double D_m);

/* ---- Velocity-field mode (heterogeneous flow) -----------------------------------------------
 * For a context created with vmax > 0.  Each particle a moves with its own constant velocity v_a
 * (dx_a/dt = v_a, Eq. 1) and carries its own tensor D_a (Eq. 3); the rate of Eq. 4 then has both
 * terms: the dispersive sum with the per-component harmonic mean of Eq. 5,
 * K_ij = 4 D_ij,a D_ij,b / (D_ij,a + D_ij,b) (0 where both are 0), and the convective sum
 * C_a (m/rho) (v_a - v_b) . grad_a W_ab.  Relative positions change during a step, so the cell
 * list built at the start of a step is sized for H + dt vmax (every pair within H at the half step
 * is found), while the support test uses H.  Interaction kernel: direct walk (no tiles); the
 * adjoint, the closed-form error and batches are for the uniform case and return ADE_ERR_STATE /
 * ADE_ERR_ARG here.
 *   v_dev [dim][n] float (axis-major, caller order, device): copied into the workspace, so the
 *   caller may free it on return.  Checks max_a |v_a| <= vmax and that every component is finite
 *   (ADE_ERR_ARG otherwise; the context then has no field).  Waits for the stream.  Until a field
 *   is set, rate, pair-count and step calls return ADE_ERR_STATE. */
int ade_set_velocity_field(ade_ctx *ctx, const float *v_dev, void *stream);

/* ---- Cattaneo form (Eq. 14) ---------------------------------------------------------------------
 * For a context created with tau > 0 the state is (x, C, Q), Q = dC/dt the relaxing flux; a step
 * is C^{l+1/2} = C^l + dt/2 Q^l, Q^{l+1/2} = Q^l + dt/2 (R(C^l) - Q^l)/tau, then
 * C^{l+1} = C^l + dt Q^{l+1/2}, Q^{l+1} = Q^l + dt (R(C^{l+1/2}) - Q^{l+1/2})/tau, with positions as
 * in Eq. 8-9.  The flux lives in the workspace (caller order).  ade_set_flux sets it from
 * Q_dev [n] (device, caller order, copied) or, with Q_dev NULL, to R(C) at the current state (the
 * Fickian flux: the parabolic solution's initial rate, and sum Q = 0 so sum m C is conserved).
 * Steps return ADE_ERR_STATE until a flux is set.  ade_get_flux copies it to Q_dev [n].  Neither
 * waits. */
int ade_set_flux(ade_ctx *ctx, const float *Q_dev, void *stream);
int ade_get_flux(ade_ctx *ctx, float *Q_dev, void *stream);

/* ---- Checkpoint and resume ---------------------------------------------------------------------
 * No counterpart in the paper (its runs are single jobs); long runs on shared machines need to stop
 * and continue.  A snapshot of a single-plume context is one host buffer: a header (format magic
 * and version, dim, n, mode, step, simulated time, dt and the parameters), the state -- xq [dim][n],
 * C [n], the Cattaneo flux Q [n] when tau > 0, the velocity field v [dim][n] when vmax > 0 -- and a
 * CRC-32 (IEEE 802.3 polynomial) of all of it.  The caller owns the buffer (pageable or pinned host
 * memory of at least ade_checkpoint_bytes bytes) and writes it wherever it likes.
 * ade_checkpoint_save copies the state out and waits for the stream.  ade_checkpoint_load checks the
 * magic, size, checksum and that n, mode, parameters and dt equal the context's (ADE_ERR_ARG
 * otherwise, before any device copy), then copies the state in, restores step and time, and waits;
 * stepping on from a restored context gives the same bits as the original run. */
int ade_checkpoint_bytes(const ade_ctx *ctx, size_t *bytes);
int ade_checkpoint_save(ade_ctx *ctx, void *host_buf, size_t bytes, void *stream);
int ade_checkpoint_load(ade_ctx *ctx, const void *host_buf, size_t bytes, void *stream);

/* ---- Adjoint (dispersivity inversion) ---------------------------------------------------------
 * The paper has no adjoint; it is derived from Eq. 3-5 and Eq. 8-9 for the uniform-velocity case.
 * With the rate r = L(theta) C linear in C, theta = (alpha_L, alpha_T, D_m), L symmetric and the
 * same at every step (uniform drift), one step is C^{l+1} = S C^l, S = I + dt L + dt^2 L^2 / 2.
 * For J = 1/2 sum_a (C_a^N - C*_a)^2 with dt fixed:
 *   dJ/dC^0 = S^N (C^N - C*)  and  dJ/dtheta_k = sum_l lambda^{l+1} . (dS/dtheta_k) C^l,
 *   lambda^N = C^N - C*, lambda^l = S lambda^{l+1}.
 * The forward run starts from the context's current state (which is not modified), uses one cell
 * list built at the current positions, and keeps C every ckpt_every steps; segments are recomputed
 * on the way back.  Pair arithmetic is FP32; J and the dot products are FP64. */

/* Device workspace of ade_adjoint for nsteps steps with checkpoints every ckpt_every steps. */
int ade_adjoint_workspace_bytes(const ade_ctx *ctx, int nsteps, int ckpt_every, size_t *bytes);

/* C_target_dev [n] (caller order): the target field C*.  Outputs: dJdC0_dev [n] (caller order, may
 * be NULL), dJdtheta_host[3] = dJ/d(alpha_L, alpha_T, D_m) (may be NULL), J_host (may be NULL),
 * C_final_dev [n] = C^N (caller order, may be NULL).  Waits for the stream. */
int ade_adjoint(ade_ctx *ctx, const float *C_target_dev, int nsteps, int ckpt_every,
                void *adjoint_workspace_dev, size_t adjoint_workspace_bytes, float *dJdC0_dev,
                double *dJdtheta_host, double *J_host, float *C_final_dev, void *stream);

/* ---- Batched plumes -------------------------------------------------------------------------
 * Many independent plumes (the convergence ladder and dispersivity sweep of Sec. 3-4 run side by
 * side) stepped together: one cell build over all plumes (global cell keys offset per plume) and
 * two persistent rate launches per step that take (plume, particle range) work items from an
 * atomic counter, largest estimated cost first.  Each particle is evaluated by the same code as in
 * a single-plume context, so a plume's results are bit-identical to ade_step on a context with the
 * same parameters and cell subdivision (ade_batch_get_plume_info reports it).
 * Layout: plume p owns caller particles [off_p, off_p + n_p), off_p = n_0 + ... + n_{p-1};
 * xq_dev holds the plumes' [dim][n_p] position blocks back to back (plume p's block starts at
 * element dim * off_p) and C_dev the concentrations back to back.  All plumes share dim, kernel and
 * a cubic box side per plume; each has its own h, dispersivities, velocity and time step. */
typedef struct ade_batch ade_batch;

/* Workspace for a batch (bytes, 256-byte aligned); sized for every cell subdivision the autotuner
 * may choose. */
int ade_batch_workspace_bytes(int nplumes, const ade_params *p, const int *n, size_t *bytes);

/* Create a batch bound to the caller's state and workspace; uploads the per-plume constants and
 * the work list on `stream` and waits for that upload. */
int ade_batch_init(ade_batch **out, int nplumes, const ade_params *p, const int *n, uint32_t *xq_dev,
                   float *C_dev, void *workspace_dev, size_t workspace_bytes, void *stream);

/* nsteps predictor-corrector steps (Eq. 8-9) of every plume, each with its own time step. */
int ade_batch_step(ade_batch *b, int nsteps, void *stream);

/* As ade_batch_step, replaying one captured CUDA graph per step; only enqueues. */
int ade_batch_run(ade_batch *b, int nsteps, void *stream);

/* FP64 per-plume mass, min and max (stats_host[nplumes]); waits for the stream. */
int ade_batch_stats(ade_batch *b, ade_stats *stats_host, void *stream);

/* Total ordered in-support pairs over all plumes (support decided in FP64); waits. */
int ade_batch_count_pairs(ade_batch *b, long long *pairs_host, void *stream);

/* Per-plume configuration: support, dt, D, grid and cell subdivision in use; tile[0..2] report the
 * batch's work-item size, persistent grid size and number of work items. */
int ade_batch_get_plume_info(const ade_batch *b, int plume, ade_info *info_host);

/* Autotuner: times the cell build plus one evaluation of every plume for each cell-subdivision
 * policy (per-plume cost model, or 1..6 cells per support radius), work-item size (64..1024
 * particles), persistent grid size (4, 8, 16 blocks per SM) and walk (one particle per thread, or
 * the paired walk: two adjacent particles per thread, same sums), keeps the fastest and re-plans.
 * Leaves the particle state unchanged; waits; best_ms_host (may be NULL) gets the best time. */
int ade_batch_autotune(ade_batch *b, double *best_ms_host, void *stream);

/* The batch's configuration -- cell-subdivision policy (0 = per-plume cost model, 1..6 cells per
 * support radius), work-item size in particles, persistent grid in blocks and walk (1: paired) --
 * as chosen by ade_batch_autotune, and its application to another batch of the same plumes so that
 * both run the same kernels (no counterpart in the paper).  set: subdiv_mode in [0, 6], tile_size
 * in [32, 4096], grid_blocks in [1, 65536], paired 0 or 1; re-plans the work list and uploads it on
 * `stream` (waits); ADE_ERR_ARG outside those ranges, the batch unchanged.  Host pointers may not
 * be NULL. */
int ade_batch_get_config(const ade_batch *b, int *subdiv_mode_host, int *tile_size_host, int *grid_blocks_host,
                         int *paired_host);
int ade_batch_set_config(ade_batch *b, int subdiv_mode, int tile_size, int grid_blocks, int paired, void *stream);

/* One batched step bracketed by CUDA events; waits; phase_ms_host[4] = {cell build, predictor,
 * corrector, 0} in milliseconds. */
int ade_batch_step_timed(ade_batch *b, double *phase_ms_host, void *stream);

/* Kernel launches one batched step enqueues. */
int ade_batch_launches_per_step(const ade_batch *b, int *launches);

void ade_batch_destroy(ade_batch *b);

/* ---- Parameter sweep (many dispersivity sets on one plume) -------------------------------------
 * P parameter sets theta_k = (alpha_L, alpha_T, D_m)_k (Eq. 3) evolved side by side on one particle
 * set with one uniform velocity and one time step, each with its own concentration field: the
 * forward runs of a dispersivity sweep or inversion.  The cell list, the positions and each pair's
 * geometry are shared; with a uniform v the pair factor of Eq. 5 is affine in u = (vhat . e)^2,
 * Dcal = a_k u + b_k with a_k = 2 Gamma (aL - aT)|v| and b_k = 2 (Gamma - d)(aT|v| + Dm) - 2 (aL - aT)|v|,
 * so a set costs a few operations per pair on top of the shared geometry.  Up to 8 sets per rate
 * launch.  dt = p->dt if positive, else the smallest value of the dt rule over the sets.
 *   theta_host [ntheta][3]; xq_dev [dim][n] (shared positions, updated in place); C_dev [ntheta][n]
 *   (set k's field at C_dev + k n, caller order, updated in place).  1 <= ntheta <= 64.
 * Positions, C and the workspace must stay valid until ade_sweep_destroy.  Velocity-field mode is
 * not available here (ADE_ERR_ARG). */
typedef struct ade_sweep ade_sweep;
int ade_sweep_workspace_bytes(const ade_params *p, int n, int ntheta, size_t *bytes);
int ade_sweep_init(ade_sweep **out, const ade_params *p, int n, int ntheta, const double *theta_host,
                   uint32_t *xq_dev, float *C_dev, void *workspace_dev, size_t workspace_bytes);
/* Support, common dt, grid; tile[0] = rate launches per evaluation (groups of sets). */
int ade_sweep_get_info(const ade_sweep *sw, ade_info *info_host);
/* Eq. 4 for every set at the current state: dCdt_dev [ntheta][n], caller order. */
int ade_sweep_rate(ade_sweep *sw, float *dCdt_dev, void *stream);
/* Ordered in-support pairs of the shared geometry (each set evaluates them all); waits. */
int ade_sweep_count_pairs(ade_sweep *sw, long long *pairs_host, void *stream);
/* nsteps predictor-corrector steps (Eq. 8-9) of every set; ade_sweep_run replays a captured graph. */
int ade_sweep_step(ade_sweep *sw, int nsteps, void *stream);
int ade_sweep_run(ade_sweep *sw, int nsteps, void *stream);
/* One step bracketed by events; waits; phase_ms_host[4] = {cell build, predictors, correctors, 0}. */
int ade_sweep_step_timed(ade_sweep *sw, double *phase_ms_host, void *stream);
int ade_sweep_launches_per_step(const ade_sweep *sw, int *launches);
/* FP64 mass, min and max per set (stats_host[ntheta]); waits. */
int ade_sweep_stats(ade_sweep *sw, ade_stats *stats_host, void *stream);
void ade_sweep_destroy(ade_sweep *sw);

/* Cell build that allocates nothing (no counterpart in the paper: it is a service for callers).
 * Some callers cannot call cudaMalloc or give the library a workspace -- plug-ins handed only
 * their input and output buffers, code whose device memory belongs to another allocator, loops
 * that cannot accept cudaMalloc's implicit synchronisation.  This call performs the same work as
 * ade_build_cells (cell keys, one-digit counting sort, per-cell order by caller index, sorted
 * copy), with its scratch in one static device array of the library (about 16 MiB, reserved on
 * every GPU that loads the library until the process exits).
 *   dim 2 or 3; n particles (0 <= n <= ADE_NOALLOC_MAX_PARTICLES); xq_dev [dim][n] fixed-point
 *   positions and C_dev [n] (inputs); nc_host [dim] cells per axis, product <= ADE_NOALLOC_MAX_CELLS.
 *   Outputs: perm_dev [n] caller index at each sorted position, cell_start_dev [ncells + 1],
 *   sorted_dev [n] 16-byte records {x, y, z (0 in 2D), C bits} in sorted order.
 *   Alignment: sorted_dev 16 bytes; xq_dev, C_dev, perm_dev and cell_start_dev 4 bytes.  A
 *   misaligned pointer returns ADE_ERR_ARG before any GPU work.
 * Larger sizes return ADE_ERR_CAPACITY without touching the GPU.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is cached per device together with the driver's ID
 * of the context it was taken in; a call made in another context (after cudaDeviceReset, or after
 * another library replaced the primary context) looks it up again, so make such a call outside
 * stream capture too.  All calls share the array and it keeps the last call's
 * contents (the per-cell counters are cleared by every call): calls that overlap on the GPU race,
 * so order them on one stream.  Work is enqueued on `stream`; the call does not wait. */
#define ADE_NOALLOC_MAX_PARTICLES 1048576
#define ADE_NOALLOC_MAX_CELLS 1048576
int ade_build_cells_noalloc(int dim, int n, const uint32_t *xq_dev, const float *C_dev,
                            const int *nc_host, uint32_t *perm_dev, uint32_t *cell_start_dev,
                            void *sorted_dev, void *stream);

/* Measured issue rates of the FP32 fused multiply-add pipe and of the reciprocal-square-root unit
 * on the current device (operations per second, best of three timed launches after a warm-up
 * launch on `stream`; about 10 ms of work in all).  The interaction kernels' ALU roof is stated in
 * FP32-pipe instructions and MUFU operations per pair; this turns those counts into time on the
 * device at hand.  Allocates (and frees) one small device buffer; waits for the stream. */
int ade_alu_peaks(double *ffma_per_s_host, double *rsqrt_per_s_host, void *stream);

/* Release the context (not the caller's buffers). */
void ade_destroy(ade_ctx *ctx);

/* Message of the last failure on the calling thread ("" if none). */
const char *ade_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADE_SPH_H */
