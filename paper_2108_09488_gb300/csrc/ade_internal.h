// ade_internal.h -- types shared by the host entry points and the kernels of libade_sph.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/ade_sph.h"

namespace ade {

constexpr int kMaxSubdiv = 6;                                   // cells per support radius
constexpr int kMaxRows = (2 * kMaxSubdiv + 1) * (2 * kMaxSubdiv + 1);
constexpr int kRateThreads = 128;                              // direct variant
constexpr int kTileThreads = 256;                              // tiled variant
constexpr int kMaxCellBits = 24;                                // ncells <= 2^24
constexpr int kScanTileCells = 2048;                            // cells per scan block (cells.cu)
constexpr int kGraphSteps = 32;                                 // steps captured in ade_run's long graph

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel launched by
// launch_pdl may have its CTAs scheduled while the kernel before it on the stream is still
// running; it calls pdl_wait() before its first access to memory that earlier work on the stream
// writes or reads (the wait returns once those grids have completed and their writes are visible;
// without a programmatic predecessor it returns at once), then pdl_trigger(), which lets the next
// kernel's CTAs be scheduled once every CTA of this grid has started.  The cell-build kernels and
// the statistics fold start with both calls, so each launch gap overlaps the tail of the previous
// kernel and no data dependency changes.  The rate kernels only wait: when their grid fits in one
// wave an early trigger would park the next launch's CTAs, waiting, beside them for the whole
// launch (measured up to 15 us slower per step at 512^2); the implicit trigger at completion
// still hides the launch gap.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// One row of the neighbour-cell stencil: cells (cx - w .. cx + w, cy + dy, cz + dz).
struct StencilRow {
    signed char dy, dz, w, pad;
};

// Everything the interaction kernel needs, passed by value (kernel parameter space).
// Lengths are in fixed-point units of the x axis (L_x / 2^32).
struct RateParams {
    int n;
    int ncx, ncy, ncz;
    int nrows;
    StencilRow rows[kMaxRows];
    float H2;        // support radius squared
    float invH;      // 1 / support radius
    float sy, sz;    // L_y / L_x, L_z / L_x (1 for a cubic box)
    // Pair factor of Eq. 5 for the uniform tensor of Eq. 3 (K = 2D): Dcal = a (vhat . e)^2 + b with
    // e = x_ab / r, a = 2 Gamma (alpha_L - alpha_T)|v|, b = 2 (Gamma - dim) d_T - 2 (alpha_L - alpha_T)|v|,
    // d_T = alpha_T |v| + D_m.  The walks evaluate t = (uw . x_ab) / r with uw = sqrt(|a|) vhat and
    // Dcal' = t^2 + ub, ub = sign(a) b, so Dcal = sign(a) Dcal'; the sign is folded into upf.
    float uw[3];
    float ub;
    float upf;       // sign(a) * pf
    float pf;        // 1/2 (m / rho) * kernel prefactor of W'(r)/r
    float dt;        // step length used by the epilogue
    uint32_t inc[3]; // fixed-point position increment used by the epilogue
    uint32_t back[3];// evaluation position minus cell-build position (0, or the half-step drift)
    int variant;     // 0 = direct walk (branch-free), 1 = shared-memory tiles, 2 = direct walk
                     // branching on the support test, 3 / 4 = 0 / 2 with per-particle trimmed rows,
                     // 5 / 6 / 7 / 8 = 0 / 3 / 2 / 4 with two targets per thread (packed FP32x2)
    int k;           // halo width in cells (cells per support radius)
    int tx, ty, tz;  // target cells per tile
    int ntx, nty, ntz;  // tiles per axis
    int cap;         // staged-particle capacity of a tile
    double u[3];     // FP64 length of one fixed-point unit per axis (L_i / 2^32)
    double H2d;      // FP64 support radius squared (pair counting decides support in FP64)
    int goff;        // batched plumes: first particle (caller and sorted order) of this plume
    int coff;        // batched plumes: first cell of this plume in the global cell table
    int m1;               // -1: the multiplier of the walks' separations (see sep in rate_common.cuh)
    const uint4 *pencil;  // trimmed walks: per pencil (cy, cz) the transverse bounding box
                          // {min y, max y, min z, max z} of its particles at the cell build
};

// Velocity-field mode: per-particle velocities (Eq. 1) and tensors (Eq. 3).
struct FieldParams {
    double aL, aT, Dm;       // Eq. 3 coefficients (the per-particle D is formed in FP64)
    float gamma;             // Gamma of Eq. 5
    float pconv;             // (m / rho) kc L_x / 2^32: convective prefactor (x_ab in x-axis units)
    double vscale[3];        // dt / L_i * 2^32: fixed-point drift per unit velocity over one step
};

// Per-particle field records of velocity-field mode (workspace).  v is constant in time, so the
// records are formed once per field (or dispersivity change) in the caller's order and only
// permuted into the cell-sorted order after each cell build:
//   2D: V = {vx, vy, 0, 0},          DA = {Dxx, Dxy, Dyy, lo(Dxy)}
//   3D: V = {vx, vy, vz, lo(Dxz)},   DA = {Dxx, Dxy, Dxz, lo(Dxy)}, DB = {Dyy, Dyz, Dzz, lo(Dyz)}
//   Inc = {hx, hy, hz, c}: fixed-point half-step drift h_i = round(v_i dt/2 / L_i 2^32) and the
//   full-step drift round(v_i dt / L_i 2^32) = 2 h_i + c_i, c_i in {-1, 0, 1} packed as 2-bit
//   fields (c_i + 1) << 2i.
struct FieldWork {
    float4 *Vc, *DAc, *DBc;  // [n] caller order (DBc: 3D only)
    uint4 *IncC;             // [n] caller order
    float4 *V, *DA, *DB;     // [n] cell-sorted order
    uint4 *Inc;              // [n] cell-sorted order
    unsigned *vmax_bits;     // max |v_a| as FP32 bits (ade_set_velocity_field)
};

// Parameter sweep (sweep.cu): one group of up to kSweepGroup parameter sets per launch.
constexpr int kSweepGroup = 8;
constexpr int kSweepMax = 64;     // parameter sets per sweep
struct SweepParams {
    float vh[3];                  // unit vector of the uniform velocity (x axis when v = 0)
    float a[kSweepGroup];         // Dcal = a u + b per set of the group, u = (vhat . e)^2
    float b[kSweepGroup];
    int g0;                       // first set of the group
    int nt;                       // sets in the group: 1, 2, 4 or 8
    int P4;                       // stride of the interleaved sorted concentrations
};

struct SweepOut {
    float *rate;                  // EPI_RATE: [P][n] caller order (may be NULL)
    float *Cout;                  // EPI_PREDICT: sorted half-step concentrations [n][P4]
    uint4 *Pout;                  // EPI_PREDICT: sorted half-step positions (group 0 writes)
    float *C;                     // EPI_CORRECT: caller concentrations [P][n], updated in place
    uint32_t *xq;                 // EPI_CORRECT: caller positions (group 0 writes)
    int *status;                  // EPI_CORRECT: set to 1 on a non-finite C
    unsigned long long *pairs;    // pair counter (counting launch)
};

// One work item of the batched rate kernel: `count` sorted particles of plume `plume` starting
// at plume-local sorted index `start`.
struct BatchTile {
    int plume, start, count, pad;
};

// Outputs of the fused epilogues.
struct EpiOut {
    float *rate;              // EPI_RATE: dC/dt in caller order
    uint4 *Pout;              // EPI_PREDICT: sorted half-step state
    uint32_t *xq;             // EPI_CORRECT: caller state, updated in place
    float *C;                 // EPI_CORRECT
    float4 *wpart;            // EPI_CORRECT: per-warp {sum C as FP32 hi + lo, min C, max C}
    int *status;              // EPI_CORRECT: set to 1 on a non-finite C
    unsigned long long *pairs; // optional in-support pair counter
    float *Q;                 // Eq. 14 (NULL: Eq. 1): flux dC/dt in caller order, updated by the corrector
    float *Qh;                // Eq. 14: sorted half-step flux (predictor writes, corrector reads)
    float tau_inv;            // Eq. 14: 1 / tau
};

enum Epilogue { EPI_RATE = 0, EPI_PREDICT = 1, EPI_CORRECT = 2 };

// Device buffers carved out of the caller's workspace.
struct Work {
    uint32_t *keys;        // [n] cell key per caller particle
    uint32_t *rank;        // [n] provisional rank inside the cell
    uint32_t *count;       // [ncells] particles per cell
    uint32_t *block_sums;  // [scan blocks]
    uint32_t *perm_tmp;    // [n] provisional cell-sorted permutation
    uint32_t *perm;        // [n] caller index at each sorted position
    uint32_t *cell_start;  // [ncells + 1]
    uint4 *P0;             // [n] sorted {x, y, z, C} at level l
    uint4 *P1;             // [n] sorted state at level l + 1/2
    uint4 *pencil = nullptr;  // [ncy * ncz] transverse bounding boxes of the pencils (NULL: not built)
    uint32_t *tile_sums = nullptr;             // [tiles of 4096 cells, 128 B apart] totals for the one-pass scan
                                               // (k_count adds, k_place clears; null: multi-launch scan)
    double *partials;      // per-block reduction partials (state statistics)
    float4 *wpart;         // per-warp partials of the corrector (EpiOut::wpart)
    double *stats;         // {sum C, min C, max C, -, closed-form slots}
    double *cf_partials;   // closed-form error partials
    int *status;           // non-finite flag
    unsigned long long *pairs;
};

// NVTX range for the duration of a host call (visible in Nsight timelines; no cost without a tool).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Records msg as the calling thread's last error (read by ade_last_error) and returns code.
int report_error(int code, const char *msg);

// Pair-factor constants Kc[6], c0 of a uniform dispersion tensor D (dim x dim, Eq. 5, K = 2D).
void pair_coeffs(int dim, double gamma, const double *D, float *Kc, float *c0);
// The interaction walks' form of the same factor for the tensor of Eq. 3 (RateParams uw, ub, upf;
// pf must be set first).
void rate_pair_consts(int dim, double gamma, const double *v, double alpha_L, double alpha_T, double D_m,
                      RateParams *rp);

// Launchers (cells.cu, rate.cu, reduce.cu).  All return cudaGetLastError() of the launches.
int scan_blocks(int m);
// Kernel launches of one launch_build_cells (the scan takes one launch with look-back flags, else
// two, or three on large grids).
int tile_blocks(int m);          // tiles of the one-pass scan
size_t tile_sums_bytes(int m);   // their totals (one 128-byte line each)
int cell_build_launches(int n, int ncells, bool onepass);
// count_zero: w.count[0, ncells) is known to be zero (every build leaves it zero), so the memset
// that otherwise starts the build is skipped.
cudaError_t launch_build_cells(int dim, const uint32_t *xq, const float *C, int n, const int *nc,
                               int ncells, const Work &w, cudaStream_t s, bool count_zero = false);
// Batched plumes: keys are coff_p + local key; plume_of[i] gives the plume of caller particle i.
cudaError_t launch_build_cells_batch(int dim, const uint32_t *xq, const float *C, int n, int ncells,
                                     const RateParams *descs, const uint16_t *plume_of,
                                     const Work &w, cudaStream_t s);
// paired: the persistent kernel's threads take two adjacent sorted particles (the paired walk).
cudaError_t launch_rate_batch(int dim, int kernel, int epi, const uint4 *Pe, const uint32_t *cell_start,
                              const uint32_t *perm, const RateParams *descs, const BatchTile *tiles,
                              int ntiles, unsigned *queue, int grid, const EpiOut &out, cudaStream_t s,
                              bool paired = false);
cudaError_t launch_batch_stats(const float *C, const int *offsets, int nplumes, double *stats,
                               cudaStream_t s);
cudaError_t launch_rate(int dim, int kernel, bool iso, int epi, const uint4 *Pe, const uint4 *Pc,
                        const uint32_t *cell_start, const uint32_t *perm, const RateParams &prm,
                        const EpiOut &out, cudaStream_t s);
// Fixed-order fold of the corrector's m per-warp partials into stats[0..2] = {sum C (FP64),
// min C, max C}: one thread-block cluster of up to kFoldMaxCtas CTAs (reduce.cu).
constexpr int kFoldMaxCtas = 8;
cudaError_t launch_fold_warp_partials(const float4 *wpart, int m, double *stats, cudaStream_t s);
cudaError_t launch_closed_form_error(int dim, const uint32_t *xq, const float *C, int n,
                                     const double *box, const double *center, const double *Sinv,
                                     double amp, double C0, double vol, int nimg,
                                     double *partials, int nblocks, double *out, cudaStream_t s);

cudaError_t launch_state_stats(const float *C, int n, double *partials, double *stats, cudaStream_t s);

// Velocity-field mode (rate_field.cu).
// Caller-order records from v [dim][n] (vx, vy, vz into Vc; v_dev may be NULL to re-form the
// tensors from the velocities already in Vc), and max |v| into fw.vmax_bits when v_dev is given.
cudaError_t launch_field_records(int dim, const float *v_dev, int n, const FieldParams &fp, const FieldWork &fw,
                                 cudaStream_t s);
// Sorted records: V[i] = Vc[perm[i]] (and DA, DB).
cudaError_t launch_field_permute(int dim, const uint32_t *perm, int n, const FieldWork &fw, cudaStream_t s);
// Paired walks (variants 5-8; rate_pair.cu), called by launch_rate.
cudaError_t launch_rate_pair(int dim, int kernel, int epi, bool iso, const uint4 *Pe, const uint4 *Pc,
                             const uint32_t *cs, const uint32_t *perm, const RateParams &prm, const EpiOut &out,
                             cudaStream_t s);
cudaError_t launch_rate_field(int dim, int kernel, int epi, const uint4 *Pe, const uint32_t *cell_start,
                              const uint32_t *perm, const FieldWork &fw, const RateParams &prm,
                              const FieldParams &fp, const EpiOut &out, cudaStream_t s);

// Parameter sweep (sweep.cu).
cudaError_t launch_sweep_gather(const uint32_t *perm, const float *C, int n, int P, int P4, float *Cs,
                                cudaStream_t s);
cudaError_t launch_rate_sweep(int dim, int kernel, int epi, bool count, const uint4 *Pe, const float *Ce,
                              const uint32_t *cell_start, const uint32_t *perm, const RateParams &prm,
                              const SweepParams &sp, const SweepOut &out, cudaStream_t s);

int rate_blocks(int n);
int rate_launch_blocks(int dim, const RateParams &prm, bool iso);
// Warps of one uniform-velocity rate launch (= per-warp partials its corrector writes).
int rate_launch_warps(int dim, const RateParams &prm, bool iso);
size_t tiled_smem_bytes(int dim, const RateParams &prm);
int closed_form_blocks(int n);

}  // namespace ade

struct ade_ctx {
    ade_params p;
    int n;
    int dim;
    int nc[3];
    int ncells;
    int subdiv;
    int ncells_cap;       // workspace capacity in cells (every grid the autotuner may pick)
    int partials_cap;     // workspace capacity in reduction partials
    int wpart_cap;        // workspace capacity in per-warp corrector partials
    bool count_clean;     // w.count[0, ncells_cap) is zero (cleared once; every cell build leaves it so)
    uint32_t *xq;
    float *C;
    void *ws;
    size_t ws_bytes;
    ade::Work w;
    double H;
    double dt;
    double D[9];
    ade::RateParams rp;   // rate constants (dt/inc set per use)
    uint32_t inc[3];
    uint32_t inc_half[3];
    bool iso;
    double t;
    long long step;
    long long pairs;
    cudaGraph_t graph;             // one step (ade_run)
    cudaGraphExec_t graph_exec;
    cudaGraph_t graph_multi;       // kGraphSteps steps (ade_run)
    cudaGraphExec_t graph_exec_multi;
    cudaStream_t cap_stream;
    bool status_cleared;
    cudaEvent_t ev[5];    // per-phase timing events (created on first timed step)
    bool ev_ready;
    // velocity-field mode (p.vmax > 0)
    bool field;
    bool field_set;       // a valid field has been copied in
    bool field_dirty;     // tensors must be re-formed (dispersivities changed)
    // Cattaneo form (Eq. 14, p.tau > 0)
    bool catt;
    bool flux_set;        // Q holds a flux (ade_set_flux)
    float *Q;             // [n] caller order
    float *Qh;            // [n] sorted half-step flux
    double Hgrid;         // radius the cell grid is built for: H, or H + skin in field mode
    double skin;
    ade::FieldParams fp;  // constants (scales set per use)
    ade::FieldWork fw;
};
