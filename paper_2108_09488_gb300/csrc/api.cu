// api.cu -- extern "C" entry points of libade_sph.so (declared in include/ade_sph.h).
//
// Host-side set-up in FP64: the dispersion tensor (Eq. 3), the time step (Eq. 10 or the
// largest-eigenvalue rule), the cell grid and neighbour stencil, the kernel constants of Eq. 4-5
// and Eq. 7, and the fixed-point drift per (half) step.  Device work is enqueued on the caller's
// stream; a step is a cell build followed by two fused rate launches and a reduction.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ade_internal.h"

#include <algorithm>
#include <vector>

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define ADE_CK(call)                                                                            \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(ADE_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwo32 = 4294967296.0;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Eq. 3: D_ij = (aT |v| + Dm) delta_ij + (aL - aT) v_i v_j / |v| (second term 0 when v = 0).
void dispersion_tensor(int dim, const double *v, double aL, double aT, double Dm, double *D)
{
    double vv = 0.0;
    for (int i = 0; i < dim; ++i) vv += v[i] * v[i];
    const double vabs = sqrt(vv);
    for (int i = 0; i < 9; ++i) D[i] = 0.0;
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
            double d = (i == j) ? aT * vabs + Dm : 0.0;
            if (vabs > 0.0) d += (aL - aT) * v[i] * v[j] / vabs;
            D[i * dim + j] = d;
        }
}

// Largest eigenvalue of a symmetric dim x dim matrix by cyclic Jacobi rotations.
double lambda_max(int dim, const double *Din)
{
    double a[3][3] = {{0}};
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) a[i][j] = Din[i * dim + j];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < dim; ++p)
            for (int q = p + 1; q < dim; ++q) off += a[p][q] * a[p][q];
        if (off < 1e-300) break;
        for (int p = 0; p < dim; ++p)
            for (int q = p + 1; q < dim; ++q) {
                if (a[p][q] == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < dim; ++k) {
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < dim; ++k) {
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
            }
    }
    double m = a[0][0];
    for (int i = 1; i < dim; ++i) m = fmax(m, a[i][i]);
    return m;
}

// Time step: p->dt when positive, else coef h^2 / den with den = lambda_max(D) or tr D (Eq. 10).
// In velocity-field mode D varies per particle; den is then the largest value the rule takes over
// |v| <= vmax: lambda_max = max(aL, aT) vmax + Dm, tr D = (aL + (dim - 1) aT) vmax + dim Dm.
int time_step(const ade_params *p, const double *D, double *dt_out)
{
    double dt = p->dt;
    if (!(dt > 0.0)) {
        const double coef = p->dt_coef > 0.0 ? p->dt_coef : 0.1;
        double den;
        if (p->vmax > 0.0) {
            if (p->dt_rule == ADE_DT_TRACE)
                den = (p->alpha_L + (p->dim - 1) * p->alpha_T) * p->vmax + p->dim * p->D_m;
            else
                den = fmax(p->alpha_L, p->alpha_T) * p->vmax + p->D_m;
        } else if (p->dt_rule == ADE_DT_TRACE) {
            den = 0.0;
            for (int i = 0; i < p->dim; ++i) den += D[i * p->dim + i];
        } else {
            den = lambda_max(p->dim, D);
        }
        if (!(den > 0.0)) return fail(ADE_ERR_ARG, "dispersion tensor is zero: give dt explicitly");
        dt = coef * p->h * p->h / den;
        // Eq. 14: the flux relaxes with rate 1/tau; the explicit midpoint rule needs dt <= ~2 tau
        if (p->tau > 0.0) dt = fmin(dt, p->tau);
    }
    *dt_out = dt;
    return ADE_OK;
}

// Neighbour-cell stencil for cells of side s[] and support H: every row (dy, dz) whose cells can
// hold a point within H (1 + 2^-12) of a point in the centre cell, with the x half-width w of that
// row.  Two cells offset by o are at least sum_i (max(|o_i| - 1, 0) s_i)^2 apart (squared).  The
// margin puts every particle of a cell outside a row beyond H by far more than the FP32 rounding
// of a pair's distance, so a walk that visits such a particle (the paired walk does) adds an
// exactly zero term.
int build_rows(int dim, int k, const double *s, double H, ade::StencilRow *rows)
{
    int nr = 0;
    const int kz = dim == 3 ? k : 0;
    const double Hm = H * (1.0 + 1.0 / 4096.0);
    const double H2 = Hm * Hm;
    for (int dz = -kz; dz <= kz; ++dz)
        for (int dy = -k; dy <= k; ++dy) {
            double ey = fmax(fabs((double)dy) - 1.0, 0.0) * s[1];
            double ez = dim == 3 ? fmax(fabs((double)dz) - 1.0, 0.0) * s[2] : 0.0;
            double e2 = ey * ey + ez * ez;
            if (e2 >= H2) continue;
            int w = k;
            while (w > 0) {
                double ex = fmax((double)w - 1.0, 0.0) * s[0];
                if (ex * ex + e2 < H2) break;
                --w;
            }
            rows[nr].dy = (signed char)dy;
            rows[nr].dz = (signed char)dz;
            rows[nr].w = (signed char)w;
            rows[nr].pad = 0;
            ++nr;
        }
    return nr;
}

struct Grid {
    int nc[3];
    int ncells;
    int subdiv;
    int nrows;
    ade::StencilRow rows[ade::kMaxRows];
};

// Grid with `k` cells per support radius: nc_i = floor(L_i k / H), so each cell is at least H/k
// wide and a particle's neighbours lie within k cells along every axis.  Needs nc_i >= 2k+1 so
// the stencil never wraps onto itself.
bool make_grid(const ade_params &p, double H, int k, Grid *g)
{
    double ncells = 1.0;
    double s[3] = {1, 1, 1};
    for (int i = 0; i < 3; ++i) g->nc[i] = 1;
    for (int i = 0; i < p.dim; ++i) {
        double c = floor(p.box[i] * k / H);
        if (c < 2 * k + 1 || c > 65535.0) return false;
        g->nc[i] = (int)c;
        s[i] = p.box[i] / c;
        ncells *= c;
    }
    if (ncells > (double)(1u << ade::kMaxCellBits)) return false;
    g->ncells = (int)ncells;
    g->subdiv = k;
    g->nrows = build_rows(p.dim, k, s, H, g->rows);
    return true;
}

// Cost model for the automatic choice: candidates visited per particle plus a per-row overhead.
double grid_cost(const Grid &g, int n)
{
    double ppc = (double)n / g.ncells;
    double cand = 0.0;
    for (int r = 0; r < g.nrows; ++r) cand += (2 * g.rows[r].w + 1) * ppc;
    return cand + 4.0 * g.nrows;
}

int choose_grid(const ade_params &p, double H, int n, Grid *g)
{
    if (p.cell_subdiv > 0) {
        if (p.cell_subdiv > ade::kMaxSubdiv || !make_grid(p, H, p.cell_subdiv, g))
            return fail(ADE_ERR_ARG, "cell_subdiv=%d does not fit the box (need >= 2k+1 cells per axis, <= 2^24 cells)",
                        p.cell_subdiv);
        return ADE_OK;
    }
    bool found = false;
    double best = 0.0;
    for (int k = 1; k <= ade::kMaxSubdiv; ++k) {
        Grid t;
        if (!make_grid(p, H, k, &t)) continue;
        double c = grid_cost(t, n);
        if (!found || c < best) {
            *g = t;
            best = c;
            found = true;
        }
    }
    if (!found) return fail(ADE_ERR_ARG, "box too small for the support radius (need >= 3 cells per axis)");
    return ADE_OK;
}

int validate(const ade_params *p, int n)
{
    if (!p) return fail(ADE_ERR_ARG, "params is NULL");
    if (p->dim != 2 && p->dim != 3) return fail(ADE_ERR_ARG, "dim must be 2 or 3 (got %d)", p->dim);
    if (p->kernel != ADE_WENDLAND_C2 && p->kernel != ADE_WENDLAND_C4)
        return fail(ADE_ERR_ARG, "unknown kernel %d", p->kernel);
    if (n < 0 || n > (1 << 28)) return fail(ADE_ERR_ARG, "n=%d out of range [0, 2^28]", n);
    for (int i = 0; i < p->dim; ++i)
        if (!(p->box[i] > 0.0) || !isfinite(p->box[i])) return fail(ADE_ERR_ARG, "box[%d] must be > 0", i);
    if (!(p->h > 0.0) || !isfinite(p->h)) return fail(ADE_ERR_ARG, "h must be > 0");
    if (!(p->alpha_L >= 0.0) || !(p->alpha_T >= 0.0) || !(p->D_m >= 0.0) || !isfinite(p->alpha_L) ||
        !isfinite(p->alpha_T) || !isfinite(p->D_m))
        return fail(ADE_ERR_ARG, "alpha_L, alpha_T, D_m must be finite and >= 0");
    if (!(p->mass > 0.0) || !(p->rho > 0.0)) return fail(ADE_ERR_ARG, "mass and rho must be > 0");
    for (int i = 0; i < p->dim; ++i)
        if (!isfinite(p->v[i])) return fail(ADE_ERR_ARG, "v must be finite");
    if (!isfinite(p->dt) || !isfinite(p->gamma)) return fail(ADE_ERR_ARG, "dt and gamma must be finite");
    if (p->dt_rule != ADE_DT_LAMBDA_MAX && p->dt_rule != ADE_DT_TRACE) return fail(ADE_ERR_ARG, "unknown dt_rule");
    if (p->cell_subdiv < 0 || p->cell_subdiv > ade::kMaxSubdiv) return fail(ADE_ERR_ARG, "cell_subdiv must be 0..6");
    // the paired walks: PAIRED with DIRECT or BRANCHED (not both), optionally TRIMMED
    const unsigned pf = p->flags & ~(ADE_FLAG_DIRECT | ADE_FLAG_TRIMMED);
    const unsigned pb = p->flags & ~(ADE_FLAG_BRANCHED | ADE_FLAG_TRIMMED);
    const bool paired_ok = pf == ADE_FLAG_PAIRED || pb == ADE_FLAG_PAIRED;
    if (p->flags != 0u && p->flags != ADE_FLAG_DIRECT && p->flags != ADE_FLAG_TILED &&
        p->flags != ADE_FLAG_BRANCHED && p->flags != ADE_FLAG_TRIMMED &&
        p->flags != (ADE_FLAG_TRIMMED | ADE_FLAG_DIRECT) && p->flags != (ADE_FLAG_TRIMMED | ADE_FLAG_BRANCHED) &&
        !paired_ok)
        return fail(ADE_ERR_ARG, "unknown or conflicting flags");
    if (!(p->vmax >= 0.0) || !isfinite(p->vmax)) return fail(ADE_ERR_ARG, "vmax must be finite and >= 0");
    if (p->vmax > 0.0 && p->flags != 0u && p->flags != ADE_FLAG_DIRECT)
        return fail(ADE_ERR_ARG, "velocity-field mode uses the direct walk: flags must be 0 or ADE_FLAG_DIRECT");
    if (!(p->tau >= 0.0) || !isfinite(p->tau)) return fail(ADE_ERR_ARG, "tau must be finite and >= 0");
    if (p->tau > 0.0 && p->vmax > 0.0)
        return fail(ADE_ERR_ARG, "the Cattaneo form (tau > 0) is available with a uniform velocity only");
    const double H = p->kernel == ADE_WENDLAND_C2 ? 2.0 * p->h : p->h;
    for (int i = 0; i < p->dim; ++i)
        if (!(H < 0.5 * p->box[i])) return fail(ADE_ERR_ARG, "support radius must be < box/2 (minimum image)");
    return ADE_OK;
}

// Tiles of the shared-memory variant (opt-in with ADE_FLAG_TILED): about 8 targets per thread, halo staged in <= ~100 KB,
// and T + 2k < nc along every axis so that the halo holds each cell once and every staged
// particle lies within half a box of the tile centre.
void choose_tiles(int dim, int n, const Grid &g, bool iso, unsigned flags, ade::RateParams *rp)
{
    rp->variant = 0;
    rp->k = g.subdiv;
    rp->tx = rp->ty = rp->tz = 1;
    rp->ntx = rp->nty = rp->ntz = 1;
    rp->cap = 0;
    if (!iso || !(flags & ADE_FLAG_TILED) || n == 0) return;
    const int k = g.subdiv;
    const double ppc = (double)n / g.ncells;
    const double want = 8.0 * ade::kTileThreads;
    int t[3] = {1, 1, 1};
    if (dim == 2) {
        int T = (int)lround(sqrt(want / fmax(ppc, 1e-3)));
        T = T < 1 ? 1 : (T > 64 ? 64 : T);
        t[0] = t[1] = T;
    } else {
        t[1] = t[2] = 2;
        int T = (int)lround(want / fmax(ppc, 1e-3) / 4.0);
        t[0] = T < 1 ? 1 : (T > 32 ? 32 : T);
    }
    for (int i = 0; i < dim; ++i)
        while (t[i] > 1 && t[i] + 2 * k >= g.nc[i]) --t[i];
    for (int i = 0; i < dim; ++i)
        if (t[i] + 2 * k >= g.nc[i]) return;  // the grid is too small for a halo: direct walk
    for (;;) {
        double halo = 1.0;
        for (int i = 0; i < dim; ++i) halo *= t[i] + 2 * k;
        rp->tx = t[0];
        rp->ty = t[1];
        rp->tz = dim == 3 ? t[2] : 1;
        rp->cap = (int)ceil(halo * ppc * 1.25) + 64;
        if (ade::tiled_smem_bytes(dim, *rp) <= 100 * 1024) break;
        int big = 0;
        for (int i = 1; i < dim; ++i)
            if (t[i] > t[big]) big = i;
        if (t[big] == 1) return;
        --t[big];
    }
    rp->ntx = (g.nc[0] + rp->tx - 1) / rp->tx;
    rp->nty = (g.nc[1] + rp->ty - 1) / rp->ty;
    rp->ntz = dim == 3 ? (g.nc[2] + rp->tz - 1) / rp->tz : 1;
    rp->variant = 1;
}

struct Layout {
    size_t keys, rank, count, block_sums, perm_tmp, perm, cell_start, P0, P1, partials, wpart, stats,
        cf_partials, status, pairs, pencil, tile_sums, fVc, fDAc, fDBc, fIncC, fV, fDA, fDB, fInc,
        fbits, Q, Qh, total;
};

// field_dim: 0 for a uniform velocity, else dim (velocity-field buffers are added at the end).
// nw_partials: per-warp corrector partials of the widest rate launch.  npencils: pencil boxes of
// the trimmed walks (0: none).
Layout layout(int n, int ncells, int nb_partials, int nw_partials, int field_dim = 0, bool catt = false,
              int npencils = 0)
{
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes > 0 ? bytes : 1);
        return o;
    };
    L.keys = take((size_t)n * 4);
    L.rank = take((size_t)n * 4);
    L.count = take((size_t)ncells * 4);
    L.block_sums = take((size_t)ade::scan_blocks(ncells) * 4);
    L.perm_tmp = take((size_t)n * 4);
    L.perm = take((size_t)n * 4);
    L.cell_start = take(((size_t)ncells + 1) * 4);
    L.P0 = take((size_t)n * 16);
    L.P1 = take((size_t)n * 16);
    L.partials = take((size_t)3 * (nb_partials > 0 ? nb_partials : 1) * 8);
    L.wpart = take((size_t)(nw_partials > 0 ? nw_partials : 1) * 16);
    L.stats = take(8 * 8);
    L.cf_partials = take((size_t)3 * (nb_partials > 0 ? nb_partials : 1) * 8);
    L.status = take(64);
    L.pairs = take(64);
    L.pencil = npencils > 0 ? take((size_t)npencils * 16) : 0;
    L.tile_sums = take(ade::tile_sums_bytes(ncells));
    L.fVc = L.fDAc = L.fDBc = L.fIncC = L.fV = L.fDA = L.fDB = L.fInc = L.fbits = 0;
    if (field_dim) {
        const size_t rec = (size_t)n * 16, rec3 = field_dim == 3 ? (size_t)n * 16 : 16;
        L.fVc = take(rec);
        L.fDAc = take(rec);
        L.fDBc = take(rec3);
        L.fIncC = take(rec);
        L.fV = take(rec);
        L.fDA = take(rec);
        L.fDB = take(rec3);
        L.fInc = take(rec);
        L.fbits = take(64);
    }
    L.Q = L.Qh = 0;
    if (catt) {
        L.Q = take((size_t)n * 4);
        L.Qh = take((size_t)n * 4);
    }
    L.total = off;
    return L;
}

struct Derived {
    double H;
    double dt;
    double D[9];     // Eq. 3 for the uniform velocity p->v
    double skin;     // velocity-field mode: relative drift allowance of the cell grid
    double Hgrid;    // radius the grid and stencil are built for: H + skin
    Grid g;
    int nb_partials;
    int nw_partials;
    int ncells_cap;
    int pencils_cap;     // pencils (ncy * ncz) of the largest grid the context may use
    ade::RateParams tiles;
    Layout L;
};

int derive(const ade_params *p, int n, Derived *d)
{
    int rc = validate(p, n);
    if (rc) return rc;
    d->H = p->kernel == ADE_WENDLAND_C2 ? 2.0 * p->h : p->h;
    dispersion_tensor(p->dim, p->v, p->alpha_L, p->alpha_T, p->D_m, d->D);
    rc = time_step(p, d->D, &d->dt);
    if (rc) return rc;
    d->skin = 0.0;
    if (p->vmax > 0.0) {
        // relative drift up to the half step, |v_a - v_b| dt / 2 <= vmax dt, plus the rounding of
        // two fixed-point increments per axis
        double umax = 0.0;
        for (int i = 0; i < p->dim; ++i) umax = fmax(umax, p->box[i] / kTwo32);
        d->skin = p->vmax * d->dt + 4.0 * umax;
    }
    d->Hgrid = d->H + d->skin;
    rc = choose_grid(*p, d->Hgrid, n, &d->g);
    if (rc) return rc;
    // tiles are for the uniform-velocity kernel in a cubic box
    const bool iso = p->box[1] == p->box[0] && (p->dim == 2 || p->box[2] == p->box[0]) && !(p->vmax > 0.0);
    memset(&d->tiles, 0, sizeof(d->tiles));
    d->tiles.n = n;
    choose_tiles(p->dim, n, d->g, iso, p->flags, &d->tiles);
    int nbr = ade::rate_blocks(n), nbc = ade::closed_form_blocks(n);
    int nbt = ade::rate_launch_blocks(p->dim, d->tiles, iso);
    d->nb_partials = nbr > nbc ? nbr : nbc;
    if (nbt > d->nb_partials) d->nb_partials = nbt;
    d->nw_partials = std::max(nbr * (ade::kRateThreads / 32), ade::rate_launch_warps(p->dim, d->tiles, iso));
    int ncells_cap = d->g.ncells;
    int pencils_cap = d->g.ncells / d->g.nc[0];
    if (p->cell_subdiv == 0 && p->flags == 0u) {
        // automatic grid: size the workspace for every configuration the autotuner may pick
        for (int k = 1; k <= ade::kMaxSubdiv; ++k) {
            Grid g;
            if (!make_grid(*p, d->Hgrid, k, &g)) continue;
            ncells_cap = std::max(ncells_cap, g.ncells);
            pencils_cap = std::max(pencils_cap, g.ncells / g.nc[0]);
            ade::RateParams t;
            memset(&t, 0, sizeof(t));
            t.n = n;
            choose_tiles(p->dim, n, g, iso, ADE_FLAG_TILED, &t);
            d->nb_partials = std::max(d->nb_partials, ade::rate_launch_blocks(p->dim, t, iso));
            d->nw_partials = std::max(d->nw_partials, ade::rate_launch_warps(p->dim, t, iso));
        }
    }
    d->ncells_cap = ncells_cap;
    // pencil boxes serve the trimmed walks of the uniform-velocity kernels
    d->pencils_cap = p->vmax > 0.0 ? 0 : pencils_cap;
    d->L = layout(n, ncells_cap, d->nb_partials, d->nw_partials, p->vmax > 0.0 ? p->dim : 0, p->tau > 0.0,
                  d->pencils_cap);
    return ADE_OK;
}

uint32_t fixed_increment(double v, double dt, double L)
{
    double q = nearbyint(v * dt / L * kTwo32);
    long long w = (long long)fmod(q, kTwo32);
    return (uint32_t)w;
}

// Velocity-field mode needs a field before any evaluation.
int need_field(const ade_ctx *c)
{
    if (c->field && !c->field_set) return fail(ADE_ERR_STATE, "velocity-field mode: call ade_set_velocity_field first");
    return ADE_OK;
}

// Steps of the Cattaneo form need the flux Q = dC/dt of the current state.
int need_flux(const ade_ctx *c)
{
    if (c->catt && !c->flux_set) return fail(ADE_ERR_STATE, "Cattaneo form (tau > 0): call ade_set_flux first");
    return ADE_OK;
}

// Re-form the caller-order tensor records after a dispersivity change (not inside a capture:
// ade_run calls this before capturing).
int refresh_field(ade_ctx *c, cudaStream_t s)
{
    if (c->field && c->field_set && c->field_dirty) {
        ADE_CK(ade::launch_field_records(c->dim, nullptr, c->n, c->fp, c->fw, s));
        c->field_dirty = false;
    }
    return ADE_OK;
}

// The cell counts arrive uninitialised: clear the whole capacity once (before any graph capture);
// from then on every cell build leaves them zero.
int clean_counts(ade_ctx *c, cudaStream_t s)
{
    if (!c->count_clean) {
        ADE_CK(cudaMemsetAsync(c->w.count, 0, (size_t)c->ncells_cap * sizeof(uint32_t), s));
        // the one-pass scan's flags and {ticket, epoch}: from then on each scan leaves them valid
        ADE_CK(cudaMemsetAsync(c->w.tile_sums, 0, ade::tile_sums_bytes(c->ncells_cap), s));
        c->count_clean = true;
    }
    return ADE_OK;
}

// Enqueue one cell build; in velocity-field mode followed by the permutation of the v and D
// records into the sorted order.
int enqueue_cells(ade_ctx *c, cudaStream_t s)
{
    int rc = need_field(c);
    if (rc) return rc;
    rc = refresh_field(c, s);
    if (rc) return rc;
    rc = clean_counts(c, s);
    if (rc) return rc;
    cudaError_t e = ade::launch_build_cells(c->dim, c->xq, c->C, c->n, c->nc, c->ncells, c->w, s, true);
    if (e != cudaSuccess) {
        c->count_clean = false;   // a build that did not run to the end may leave counts behind
        return fail(ADE_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    if (c->field) ADE_CK(ade::launch_field_permute(c->dim, c->w.perm, c->n, c->fw, s));
    return ADE_OK;
}

ade::EpiOut epi_none()
{
    ade::EpiOut o;
    memset(&o, 0, sizeof(o));
    return o;
}

enum Phase { AT_BUILD = 0, PREDICTOR = 1, CORRECTOR = 2 };

// One rate evaluation on the last cell build.  AT_BUILD: the state of the build (rate or pair
// count).  PREDICTOR: C^{l+1/2} = C^l + dt/2 r^l, x^{l+1/2} = x^l + dt/2 v.  CORRECTOR:
// C^{l+1} = C^l + dt r^{l+1/2}, x^{l+1} = x^l + dt v, evaluated at the half-step state P1.
int enqueue_eval(ade_ctx *c, Phase ph, ade::EpiOut out, cudaStream_t s)
{
    const int epi = ph == PREDICTOR ? ade::EPI_PREDICT : (ph == CORRECTOR ? ade::EPI_CORRECT : ade::EPI_RATE);
    const uint4 *Pe = ph == CORRECTOR ? c->w.P1 : c->w.P0;
    ade::RateParams rp = c->rp;
    rp.dt = ph == PREDICTOR ? (float)(0.5 * c->dt) : (ph == CORRECTOR ? (float)c->dt : 0.f);
    for (int i = 0; i < 3; ++i) {
        rp.inc[i] = ph == PREDICTOR ? c->inc_half[i] : (ph == CORRECTOR ? c->inc[i] : 0u);
        rp.back[i] = ph == CORRECTOR ? c->inc_half[i] : 0u;
    }
    if (c->catt && ph != AT_BUILD) {
        out.Q = c->Q;
        out.Qh = c->Qh;
        out.tau_inv = (float)(1.0 / c->p.tau);
    }
    if (c->field) {
        ADE_CK(ade::launch_rate_field(c->dim, c->p.kernel, epi, Pe, c->w.cell_start, c->w.perm, c->fw, rp, c->fp,
                                      out, s));
        return ADE_OK;
    }
    ADE_CK(ade::launch_rate(c->dim, c->p.kernel, c->iso, epi, Pe, c->w.P0, c->w.cell_start, c->w.perm, rp,
                            out, s));
    return ADE_OK;
}

ade::EpiOut epi_corrector(ade_ctx *c)
{
    ade::EpiOut out = epi_none();
    out.xq = c->xq;
    out.C = c->C;
    out.wpart = c->w.wpart;
    out.status = c->w.status;
    return out;
}

// FP64 {sum C, min C, max C} of the state the corrector just wrote, folded from its per-warp
// partials into w.stats (the step's diagnostics of Eq. 9).
int enqueue_fold(ade_ctx *c, cudaStream_t s)
{
    const int m = c->field ? ade::rate_blocks(c->n) * (ade::kRateThreads / 32)
                           : ade::rate_launch_warps(c->dim, c->rp, c->iso);
    if (m > c->wpart_cap) return fail(ADE_ERR_CAPACITY, "corrector partials exceed the workspace");
    ADE_CK(ade::launch_fold_warp_partials(c->w.wpart, m, c->w.stats, s));
    return ADE_OK;
}

// Enqueue one predictor-corrector step (Eq. 8-9) and the fold of its diagnostics.
int enqueue_step(ade_ctx *c, cudaStream_t s)
{
    int rc = enqueue_cells(c, s);
    if (rc) return rc;
    if (c->n == 0) return ADE_OK;
    ade::EpiOut out = epi_none();
    out.Pout = c->w.P1;
    rc = enqueue_eval(c, PREDICTOR, out, s);
    if (rc) return rc;
    rc = enqueue_eval(c, CORRECTOR, epi_corrector(c), s);
    if (rc) return rc;
    return enqueue_fold(c, s);
}

// The workspace arrives uninitialised: clear the status word once, before the first step (and
// the cell counts, so that a step captured into a graph holds no memset).
int clear_status_once(ade_ctx *c, cudaStream_t s)
{
    if (!c->status_cleared) {
        ADE_CK(cudaMemsetAsync(c->w.status, 0, sizeof(int), s));
        c->status_cleared = true;
    }
    return clean_counts(c, s);
}

// kc of W'(r)/r = kc f(q) for support H: Wendland C2 (support 2h, f = (1-q)^3) kc = -20 B / H^2;
// Wendland C4 (Eq. 7, support h, f = (1-q)^5 (1+5q)) kc = -(56/3) B / H^2; B the normalisation.
double kernel_kc(int kernel, int dm, double H)
{
    if (kernel == ADE_WENDLAND_C2) {
        const double B = dm == 2 ? 7.0 / (kPi * H * H) : 21.0 / (2.0 * kPi * H * H * H);
        return -20.0 * B / (H * H);
    }
    const double B = dm == 2 ? 9.0 / (kPi * H * H) : 495.0 / (32.0 * kPi * H * H * H);
    return -(56.0 / 3.0) * B / (H * H);
}

// Velocity-field constants: Eq. 3 coefficients for the per-particle tensors, Gamma, the convective
// prefactor (m/rho) kc L_x/2^32 (x_ab in fixed-point units of the x axis) and the fixed-point
// drift per unit velocity over one step, dt / L_i 2^32.
void field_constants(ade_ctx *c)
{
    const ade_params &p = c->p;
    ade::FieldParams &fp = c->fp;
    memset(&fp, 0, sizeof(fp));
    fp.aL = p.alpha_L;
    fp.aT = p.alpha_T;
    fp.Dm = p.D_m;
    fp.gamma = (float)(p.gamma > 0.0 ? p.gamma : p.dim + 2.0);
    fp.pconv = (float)((p.mass / p.rho) * kernel_kc(p.kernel, p.dim, c->H) * (p.box[0] / kTwo32));
    for (int i = 0; i < 3; ++i) fp.vscale[i] = i < p.dim ? c->dt / p.box[i] * kTwo32 : 0.0;
}

// Per-plume constants: Eq. 3 (D), the time step (Eq. 10 or the largest-eigenvalue rule), the
// fixed-point drift per step and half step, and the interaction constants of Eq. 4-5 / Eq. 7 in
// fixed-point units of the x axis.
int plume_constants(const ade_params *p, int n, const Derived &d, double *D, double *dt_out,
                    uint32_t *inc, uint32_t *inc_half, ade::RateParams *rp_out, bool *iso)
{
    // Eq. 3 and the time step (from derive)
    for (int i = 0; i < 9; ++i) D[i] = d.D[i];
    const double dt = d.dt;
    *dt_out = dt;
    for (int i = 0; i < 3; ++i) {
        double L = i < p->dim ? p->box[i] : 1.0;
        double vi = i < p->dim ? p->v[i] : 0.0;
        inc[i] = fixed_increment(vi, dt, L);
        inc_half[i] = fixed_increment(vi, 0.5 * dt, L);
    }

    // Rate constants, lengths in fixed-point units of the x axis.
    ade::RateParams &rp = *rp_out;
    memset(&rp, 0, sizeof(rp));
    rp.n = n;
    rp.ncx = d.g.nc[0];
    rp.ncy = d.g.nc[1];
    rp.ncz = d.g.nc[2];
    rp.nrows = d.g.nrows;
    for (int r = 0; r < d.g.nrows; ++r) rp.rows[r] = d.g.rows[r];
    const double u = p->box[0] / kTwo32;
    const double Hu = d.H / u;
    rp.H2 = (float)(Hu * Hu);
    for (int i = 0; i < 3; ++i) rp.u[i] = (i < p->dim ? p->box[i] : 1.0) / kTwo32;
    rp.H2d = d.H * d.H;
    rp.invH = (float)(1.0 / Hu);
    rp.sy = (float)(p->box[1] / p->box[0]);
    rp.sz = p->dim == 3 ? (float)(p->box[2] / p->box[0]) : 1.0f;
    *iso = p->box[1] == p->box[0] && (p->dim == 2 || p->box[2] == p->box[0]);
    const double gamma = p->gamma > 0.0 ? p->gamma : p->dim + 2.0;
    const int dm = p->dim;
    rp.pf = (float)(0.5 * (p->mass / p->rho) * kernel_kc(p->kernel, dm, d.H));
    ade::rate_pair_consts(dm, gamma, p->v, p->alpha_L, p->alpha_T, p->D_m, &rp);
    rp.m1 = -1;
    rp.variant = d.tiles.variant == 1 ? 1 : ((p->flags & ADE_FLAG_BRANCHED) ? 2 : 0);
    if (rp.variant != 1 && (p->flags & ADE_FLAG_TRIMMED)) rp.variant = rp.variant == 2 ? 4 : 3;  // trimmed rows
    if (p->flags & ADE_FLAG_PAIRED)                                                           // paired walks
        rp.variant = (p->flags & ADE_FLAG_BRANCHED) ? ((p->flags & ADE_FLAG_TRIMMED) ? 8 : 7)
                                                    : ((p->flags & ADE_FLAG_TRIMMED) ? 6 : 5);
    rp.k = d.tiles.k;
    rp.tx = d.tiles.tx;
    rp.ty = d.tiles.ty;
    rp.tz = d.tiles.tz;
    rp.ntx = d.tiles.ntx;
    rp.nty = d.tiles.nty;
    rp.ntz = d.tiles.ntz;
    rp.cap = d.tiles.cap;
    return ADE_OK;
}

template <typename T>
T *at(void *base, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

}  // namespace

// Pair-factor constants for a uniform tensor D (Eq. 5 with K = 2D):
// Gamma x^T K x / r^2 - tr K = x^T Gamma (K - K_last I) x / r^2 + (Gamma K_last - tr K).
void ade::pair_coeffs(int dm, double gamma, const double *D, float *Kc, float *c0)
{
    auto K = [&](int i, int j) { return 2.0 * D[i * dm + j]; };  // harmonic mean of equal D
    const double Klast = K(dm - 1, dm - 1);
    double trK = 0.0;
    for (int i = 0; i < dm; ++i) trK += K(i, i);
    Kc[0] = (float)(gamma * (K(0, 0) - Klast));
    Kc[1] = dm == 3 ? (float)(gamma * (K(1, 1) - Klast)) : 0.0f;
    Kc[2] = 0.0f;
    Kc[3] = (float)(2.0 * gamma * K(0, 1));
    Kc[4] = dm == 3 ? (float)(2.0 * gamma * K(0, 2)) : 0.0f;
    Kc[5] = dm == 3 ? (float)(2.0 * gamma * K(1, 2)) : 0.0f;
    *c0 = (float)(gamma * Klast - trK);
}

// Eq. 3 gives D = d_T I + (d_L - d_T) vhat vhat^T with d_T = alpha_T |v| + D_m, d_L = alpha_L |v| + D_m;
// with K = 2D, Eq. 5's Gamma e^T K e - tr K = a (vhat . e)^2 + b, a = 2 Gamma (d_L - d_T),
// b = 2 (Gamma - dim) d_T - 2 (d_L - d_T).  The walks use uw = sqrt|a| vhat, ub = sign(a) b and
// upf = sign(a) pf (v = 0: vhat is the x axis and a = 0).
void ade::rate_pair_consts(int dm, double gamma, const double *v, double alpha_L, double alpha_T, double D_m,
                           RateParams *rp)
{
    double sp = 0.0;
    for (int i = 0; i < dm; ++i) sp += v[i] * v[i];
    sp = sqrt(sp);
    const double dT = alpha_T * sp + D_m, dLT = (alpha_L - alpha_T) * sp;
    const double a = 2.0 * gamma * dLT;
    const double b = 2.0 * (gamma - dm) * dT - 2.0 * dLT;
    const double sa = a < 0.0 ? -1.0 : 1.0;
    const double ra = sqrt(fabs(a));
    for (int i = 0; i < 3; ++i) {
        const double vh = sp > 0.0 ? (i < dm ? v[i] / sp : 0.0) : (i == 0 ? 1.0 : 0.0);
        rp->uw[i] = (float)(ra * vh);
    }
    rp->ub = (float)(sa * b);
    rp->upf = (float)(sa * (double)rp->pf);
}

int ade::report_error(int code, const char *msg) { return fail(code, "%s", msg); }

extern "C" {

const char *ade_last_error(void) { return g_err; }

int ade_workspace_bytes(const ade_params *p, int n, size_t *bytes)
{
    if (!bytes) return fail(ADE_ERR_ARG, "bytes is NULL");
    Derived d;
    int rc = derive(p, n, &d);
    if (rc) return rc;
    *bytes = d.L.total;
    return ADE_OK;
}

int ade_init_particles(ade_ctx **out, const ade_params *p, int n, uint32_t *xq_dev, float *C_dev,
                       void *workspace_dev, size_t workspace_bytes)
{
    if (!out) return fail(ADE_ERR_ARG, "out is NULL");
    *out = nullptr;
    Derived d;
    int rc = derive(p, n, &d);
    if (rc) return rc;
    if (n > 0 && (!xq_dev || !C_dev)) return fail(ADE_ERR_ARG, "xq_dev and C_dev must be non-NULL");
    if (!workspace_dev) return fail(ADE_ERR_ARG, "workspace_dev is NULL");
    if (((uintptr_t)workspace_dev & 255u) != 0u) return fail(ADE_ERR_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < d.L.total)
        return fail(ADE_ERR_CAPACITY, "workspace too small: %zu < %zu bytes", workspace_bytes, d.L.total);

    ade_ctx *c = new (std::nothrow) ade_ctx;
    if (!c) return fail(ADE_ERR_CAPACITY, "out of host memory");
    memset(c, 0, sizeof(*c));
    c->p = *p;
    c->n = n;
    c->dim = p->dim;
    for (int i = 0; i < 3; ++i) c->nc[i] = d.g.nc[i];
    c->ncells = d.g.ncells;
    c->subdiv = d.g.subdiv;
    c->ncells_cap = d.ncells_cap;
    c->partials_cap = d.nb_partials;
    c->wpart_cap = d.nw_partials;
    c->xq = xq_dev;
    c->C = C_dev;
    c->ws = workspace_dev;
    c->ws_bytes = workspace_bytes;
    c->H = d.H;
    c->w.keys = at<uint32_t>(workspace_dev, d.L.keys);
    c->w.rank = at<uint32_t>(workspace_dev, d.L.rank);
    c->w.count = at<uint32_t>(workspace_dev, d.L.count);
    c->w.block_sums = at<uint32_t>(workspace_dev, d.L.block_sums);
    c->w.perm_tmp = at<uint32_t>(workspace_dev, d.L.perm_tmp);
    c->w.perm = at<uint32_t>(workspace_dev, d.L.perm);
    c->w.cell_start = at<uint32_t>(workspace_dev, d.L.cell_start);
    c->w.P0 = at<uint4>(workspace_dev, d.L.P0);
    c->w.P1 = at<uint4>(workspace_dev, d.L.P1);
    c->w.partials = at<double>(workspace_dev, d.L.partials);
    c->w.wpart = at<float4>(workspace_dev, d.L.wpart);
    c->w.stats = at<double>(workspace_dev, d.L.stats);
    c->w.cf_partials = at<double>(workspace_dev, d.L.cf_partials);
    c->w.status = at<int>(workspace_dev, d.L.status);
    c->w.pairs = at<unsigned long long>(workspace_dev, d.L.pairs);
    c->w.pencil = d.pencils_cap > 0 ? at<uint4>(workspace_dev, d.L.pencil) : nullptr;
    c->w.tile_sums = at<uint32_t>(workspace_dev, d.L.tile_sums);

    rc = plume_constants(p, n, d, c->D, &c->dt, c->inc, c->inc_half, &c->rp, &c->iso);
    if (rc) {
        delete c;
        return rc;
    }
    c->rp.pencil = c->w.pencil;
    c->Hgrid = d.Hgrid;
    c->skin = d.skin;
    c->field = p->vmax > 0.0;
    if (c->field) {
        c->iso = false;
        c->fw.Vc = at<float4>(workspace_dev, d.L.fVc);
        c->fw.DAc = at<float4>(workspace_dev, d.L.fDAc);
        c->fw.DBc = at<float4>(workspace_dev, d.L.fDBc);
        c->fw.IncC = at<uint4>(workspace_dev, d.L.fIncC);
        c->fw.Inc = at<uint4>(workspace_dev, d.L.fInc);
        c->fw.V = at<float4>(workspace_dev, d.L.fV);
        c->fw.DA = at<float4>(workspace_dev, d.L.fDA);
        c->fw.DB = at<float4>(workspace_dev, d.L.fDB);
        c->fw.vmax_bits = at<unsigned>(workspace_dev, d.L.fbits);
        field_constants(c);
        c->field_set = n == 0;
    }
    c->catt = p->tau > 0.0;
    if (c->catt) {
        c->Q = at<float>(workspace_dev, d.L.Q);
        c->Qh = at<float>(workspace_dev, d.L.Qh);
        c->flux_set = n == 0;
    }
    *out = c;
    return ADE_OK;
}

}  // extern "C"

namespace {

// Forget the captured step graphs (the configuration they were captured with has changed).
void drop_graphs(ade_ctx *c)
{
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->graph_exec_multi) cudaGraphExecDestroy(c->graph_exec_multi);
    if (c->graph_multi) cudaGraphDestroy(c->graph_multi);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_exec_multi = nullptr;
    c->graph_multi = nullptr;
}

// Capture `steps` consecutive steps into one graph.
int capture_steps(ade_ctx *c, int steps, cudaGraph_t *graph, cudaGraphExec_t *exec)
{
    if (!c->cap_stream) ADE_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    ADE_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = ADE_OK;
    for (int k = 0; k < steps && rc == ADE_OK; ++k) rc = enqueue_step(c, c->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    ADE_CK(e);
    cudaError_t ei = cudaGraphInstantiate(exec, g, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(g);
        *exec = nullptr;
        return fail(ADE_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    }
    *graph = g;
    return ADE_OK;
}

// Switch a context to cell subdivision k and kernel variant (tiled or direct); the workspace
// layout is fixed at init, so only the grid, the stencil and the tile fields change.
int apply_config(ade_ctx *c, int k, int variant)
{
    const bool tiled = variant == 1;
    Grid g;
    if (!make_grid(c->p, c->Hgrid, k, &g)) return fail(ADE_ERR_ARG, "subdivision %d does not fit", k);
    if (g.ncells > c->ncells_cap) return fail(ADE_ERR_CAPACITY, "grid exceeds the workspace");
    ade::RateParams t;
    memset(&t, 0, sizeof(t));
    t.n = c->n;
    choose_tiles(c->dim, c->n, g, c->iso, tiled ? ADE_FLAG_TILED : ADE_FLAG_DIRECT, &t);
    if (tiled && t.variant != 1) return fail(ADE_ERR_ARG, "tiles do not fit this grid");
    if (ade::rate_launch_blocks(c->dim, t, c->iso) > c->partials_cap ||
        ade::rate_launch_warps(c->dim, t, c->iso) > c->wpart_cap)
        return fail(ADE_ERR_CAPACITY, "tiles exceed the workspace");
    for (int i = 0; i < 3; ++i) c->nc[i] = g.nc[i];
    c->ncells = g.ncells;
    c->subdiv = g.subdiv;
    ade::RateParams &rp = c->rp;
    rp.ncx = g.nc[0];
    rp.ncy = g.nc[1];
    rp.ncz = g.nc[2];
    rp.nrows = g.nrows;
    for (int r = 0; r < g.nrows; ++r) rp.rows[r] = g.rows[r];
    rp.variant = tiled ? 1 : variant;
    rp.k = t.k;
    rp.tx = t.tx;
    rp.ty = t.ty;
    rp.tz = t.tz;
    rp.ntx = t.ntx;
    rp.nty = t.nty;
    rp.ntz = t.ntz;
    rp.cap = t.cap;
    drop_graphs(c);
    return ADE_OK;
}

}  // namespace

extern "C" {

int ade_autotune(ade_ctx *c, double *best_ms_host, void *stream)
{
    ade::NvtxRange nvtx_("ade_autotune");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (c->p.cell_subdiv != 0 || c->p.flags != 0u)
        return fail(ADE_ERR_STATE, "autotuning needs cell_subdiv = 0 and flags = 0");
    if (c->n == 0) {
        if (best_ms_host) *best_ms_host = 0.0;
        return ADE_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    ADE_CK(cudaEventCreate(&e0));
    ADE_CK(cudaEventCreate(&e1));
    int rc = ADE_OK;
    // one timed cell build + two rate evaluations (the work of a step) of configuration
    // (k, variant); false if it does not fit
    auto time_once = [&](int k, int variant, double *ms) -> bool {
        if (apply_config(c, k, variant) != ADE_OK) return false;
        cudaError_t e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) rc = enqueue_cells(c, s);
        if (rc == ADE_OK && e == cudaSuccess) rc = enqueue_eval(c, AT_BUILD, epi_none(), s);
        if (rc == ADE_OK && e == cudaSuccess) rc = enqueue_eval(c, AT_BUILD, epi_none(), s);
        if (rc != ADE_OK) return false;
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float f = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(ADE_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
            return false;
        }
        *ms = f;
        return true;
    };
    // Pass 1: every configuration, best of two back-to-back evaluations.  Pass 2: the three
    // fastest again, interleaved over three rounds (so slow drifts of the clock or the power state
    // over the sweep do not favour whichever configuration ran first), best of all their times.
    struct Cand {
        double ms;
        int k, variant;
    };
    Cand top[3] = {{1e30, c->subdiv, c->rp.variant}, {1e30, 0, -1}, {1e30, 0, -1}};
    for (int k = 1; rc == ADE_OK && k <= ade::kMaxSubdiv; ++k)
        for (int variant = 0; rc == ADE_OK && variant < 9; ++variant) {
            if (c->field && variant != 0) continue;  // one interaction kernel in velocity-field mode
            double ms = 1e30, t = 0.0;
            for (int rep = 0; rep < 2; ++rep)
                if (time_once(k, variant, &t)) ms = std::min(ms, t);
            if (rc != ADE_OK || ms >= top[2].ms) continue;
            Cand cnd{ms, k, variant};
            for (int q = 0; q < 3; ++q)
                if (cnd.ms < top[q].ms) std::swap(cnd, top[q]);
        }
    for (int round = 0; rc == ADE_OK && round < 3; ++round)
        for (int q = 0; rc == ADE_OK && q < 3; ++q) {
            double t = 0.0;
            if (top[q].variant >= 0 && top[q].ms < 1e30 && time_once(top[q].k, top[q].variant, &t))
                top[q].ms = std::min(top[q].ms, t);
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    int b = 0;
    for (int q = 1; q < 3; ++q)
        if (top[q].variant >= 0 && top[q].ms < top[b].ms) b = q;
    rc = apply_config(c, top[b].k, top[b].variant);
    if (rc) return rc;
    if (best_ms_host) *best_ms_host = top[b].ms;
    return ADE_OK;
}

int ade_set_velocity_field(ade_ctx *c, const float *v_dev, void *stream)
{
    ade::NvtxRange nvtx_("ade_set_velocity_field");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (!c->field) return fail(ADE_ERR_STATE, "context was created with vmax = 0 (uniform velocity)");
    if (c->n > 0 && !v_dev) return fail(ADE_ERR_ARG, "v_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    c->field_set = false;
    if (c->n == 0) {
        c->field_set = true;
        return ADE_OK;
    }
    ADE_CK(ade::launch_field_records(c->dim, v_dev, c->n, c->fp, c->fw, s));
    unsigned bits = 0;
    ADE_CK(cudaMemcpyAsync(&bits, c->fw.vmax_bits, sizeof(bits), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    float smax;
    memcpy(&smax, &bits, sizeof(smax));
    if (!((double)smax <= c->p.vmax))
        return fail(ADE_ERR_ARG, "velocity field: max |v| = %g exceeds vmax = %g (or is not finite)", (double)smax,
                    c->p.vmax);
    c->field_set = true;
    c->field_dirty = false;
    return ADE_OK;
}

int ade_set_flux(ade_ctx *c, const float *Q_dev, void *stream)
{
    ade::NvtxRange nvtx_("ade_set_flux");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (!c->catt) return fail(ADE_ERR_STATE, "context was created with tau = 0 (Eq. 1 has no flux variable)");
    cudaStream_t s = (cudaStream_t)stream;
    c->flux_set = false;
    if (c->n > 0) {
        if (Q_dev) {
            ADE_CK(cudaMemcpyAsync(c->Q, Q_dev, (size_t)c->n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        } else {
            // Q^0 = R(C^0): the flux of Eq. 1 at the current state
            int rc = enqueue_cells(c, s);
            if (rc) return rc;
            ade::EpiOut out = epi_none();
            out.rate = c->Q;
            rc = enqueue_eval(c, AT_BUILD, out, s);
            if (rc) return rc;
        }
    }
    c->flux_set = true;
    return ADE_OK;
}

int ade_get_flux(ade_ctx *c, float *Q_dev, void *stream)
{
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (!c->catt) return fail(ADE_ERR_STATE, "context was created with tau = 0 (Eq. 1 has no flux variable)");
    if (c->n > 0 && !Q_dev) return fail(ADE_ERR_ARG, "Q_dev is NULL");
    if (c->n > 0)
        ADE_CK(cudaMemcpyAsync(Q_dev, c->Q, (size_t)c->n * sizeof(float), cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
    return ADE_OK;
}

int ade_set_dispersivity(ade_ctx *c, double alpha_L, double alpha_T, double D_m)
{
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (!(alpha_L >= 0.0) || !(alpha_T >= 0.0) || !(D_m >= 0.0) || !isfinite(alpha_L) ||
        !isfinite(alpha_T) || !isfinite(D_m))
        return fail(ADE_ERR_ARG, "alpha_L, alpha_T, D_m must be finite and >= 0");
    c->p.alpha_L = alpha_L;
    c->p.alpha_T = alpha_T;
    c->p.D_m = D_m;
    dispersion_tensor(c->dim, c->p.v, alpha_L, alpha_T, D_m, c->D);
    const double gamma = c->p.gamma > 0.0 ? c->p.gamma : c->dim + 2.0;
    ade::rate_pair_consts(c->dim, gamma, c->p.v, alpha_L, alpha_T, D_m, &c->rp);
    if (c->field) {
        c->fp.aL = alpha_L;
        c->fp.aT = alpha_T;
        c->fp.Dm = D_m;
        c->field_dirty = true;   // tensors re-formed on the caller's stream before the next use
    }
    drop_graphs(c);
    return ADE_OK;
}

int ade_get_info(const ade_ctx *c, ade_info *info)
{
    if (!c || !info) return fail(ADE_ERR_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->support = c->H;
    info->dt = c->dt;
    for (int i = 0; i < 9; ++i) info->D[i] = c->D[i];
    for (int i = 0; i < 3; ++i) info->nc[i] = c->nc[i];
    info->ncells = c->ncells;
    info->cell_subdiv = c->subdiv;
    info->stencil_rows = c->rp.nrows;
    info->sort_passes = 1;
    info->variant = c->rp.variant;
    info->tile[0] = c->rp.tx;
    info->tile[1] = c->rp.ty;
    info->tile[2] = c->rp.tz;
    info->tile_capacity = c->rp.cap;
    info->workspace_bytes = c->ws_bytes;
    info->skin = c->skin;
    return ADE_OK;
}

int ade_build_cells(ade_ctx *c, void *stream)
{
    ade::NvtxRange nvtx_("ade_build_cells");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    return enqueue_cells(c, (cudaStream_t)stream);
}

int ade_get_cells(ade_ctx *c, uint32_t *perm_dev, uint32_t *cell_start_dev, void *stream)
{
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (perm_dev && c->n > 0)
        ADE_CK(cudaMemcpyAsync(perm_dev, c->w.perm, (size_t)c->n * 4, cudaMemcpyDeviceToDevice, s));
    if (cell_start_dev)
        ADE_CK(cudaMemcpyAsync(cell_start_dev, c->w.cell_start, ((size_t)c->ncells + 1) * 4,
                               cudaMemcpyDeviceToDevice, s));
    return ADE_OK;
}

int ade_dispersion_rate(ade_ctx *c, float *dCdt_dev, void *stream)
{
    ade::NvtxRange nvtx_("ade_dispersion_rate");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (c->n > 0 && !dCdt_dev) return fail(ADE_ERR_ARG, "dCdt_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = enqueue_cells(c, s);
    if (rc || c->n == 0) return rc;
    ade::EpiOut out = epi_none();
    out.rate = dCdt_dev;
    return enqueue_eval(c, AT_BUILD, out, s);
}

int ade_count_pairs(ade_ctx *c, long long *pairs_host, void *stream)
{
    ade::NvtxRange nvtx_("ade_count_pairs");
    if (!c || !pairs_host) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    *pairs_host = 0;
    int rc = enqueue_cells(c, s);
    if (rc || c->n == 0) return rc;
    ADE_CK(cudaMemsetAsync(c->w.pairs, 0, 8, s));
    ade::EpiOut out = epi_none();
    out.pairs = c->w.pairs;
    rc = enqueue_eval(c, AT_BUILD, out, s);
    if (rc) return rc;
    unsigned long long v = 0;
    ADE_CK(cudaMemcpyAsync(&v, c->w.pairs, 8, cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    c->pairs = (long long)v;
    *pairs_host = (long long)v;
    return ADE_OK;
}

int ade_step(ade_ctx *c, int nsteps, void *stream)
{
    ade::NvtxRange nvtx_("ade_step");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(ADE_ERR_ARG, "nsteps must be >= 0");
    if (need_field(c) || need_flux(c)) return ADE_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = clear_status_once(c, s);
    if (rc0) return rc0;
    for (int k = 0; k < nsteps; ++k) {
        int rc = enqueue_step(c, s);
        if (rc) return rc;
    }
    c->step += nsteps;
    c->t += nsteps * c->dt;
    return ADE_OK;
}

// Copies {sum C, min C, max C} from w.stats and the status word out (waits for the stream).
static int read_stats(ade_ctx *c, ade_stats *st, cudaStream_t s)
{
    double h[3];
    int status = 0;
    ADE_CK(cudaMemcpyAsync(h, c->w.stats, sizeof(h), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaMemcpyAsync(&status, c->w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    st->mass = h[0] * c->p.mass;
    st->c_min = h[1];
    st->c_max = h[2];
    st->t = c->t;
    st->step = c->step;
    st->pairs = c->pairs;
    st->status = status ? ADE_ERR_NUMERIC : ADE_OK;
    return status ? fail(ADE_ERR_NUMERIC, "non-finite concentration produced") : ADE_OK;
}

int ade_get_stats(ade_ctx *c, ade_stats *st, void *stream)
{
    if (!c || !st) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = clear_status_once(c, s);
    if (rc0) return rc0;
    ADE_CK(ade::launch_state_stats(c->C, c->n, c->w.partials, c->w.stats, s));
    return read_stats(c, st, s);
}

int ade_run(ade_ctx *c, int nsteps, ade_stats *st, void *stream)
{
    ade::NvtxRange nvtx_("ade_run");
    if (!c) return fail(ADE_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(ADE_ERR_ARG, "nsteps must be >= 0");
    if (need_field(c) || need_flux(c)) return ADE_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int rc0 = clear_status_once(c, s);
    if (rc0) return rc0;
    rc0 = refresh_field(c, s);
    if (rc0) return rc0;
    // whole multiples of kGraphSteps replay one graph of kGraphSteps steps (no launch gap between
    // them), the rest a graph of one step
    const int nmulti = nsteps / ade::kGraphSteps, nsingle = nsteps % ade::kGraphSteps;
    if (nmulti > 0 && !c->graph_exec_multi) {
        int rc = capture_steps(c, ade::kGraphSteps, &c->graph_multi, &c->graph_exec_multi);
        if (rc) return rc;
    }
    if (nsingle > 0 && !c->graph_exec) {
        int rc = capture_steps(c, 1, &c->graph, &c->graph_exec);
        if (rc) return rc;
    }
    for (int k = 0; k < nmulti; ++k) ADE_CK(cudaGraphLaunch(c->graph_exec_multi, s));
    for (int k = 0; k < nsingle; ++k) ADE_CK(cudaGraphLaunch(c->graph_exec, s));
    c->step += nsteps;
    c->t += nsteps * c->dt;
    if (!st) return ADE_OK;
    // the last step folded the diagnostics of the state it wrote (the current state)
    if (nsteps > 0 && c->n > 0) return read_stats(c, st, s);
    return ade_get_stats(c, st, stream);
}

int ade_step_timed(ade_ctx *c, double *phase_ms, void *stream)
{
    ade::NvtxRange nvtx_("ade_step_timed");
    if (!c || !phase_ms) return fail(ADE_ERR_ARG, "NULL argument");
    if (need_field(c) || need_flux(c)) return ADE_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = clear_status_once(c, s);
    if (rc) return rc;
    if (!c->ev_ready) {
        for (int k = 0; k < 5; ++k) ADE_CK(cudaEventCreate(&c->ev[k]));
        c->ev_ready = true;
    }
    ADE_CK(cudaEventRecord(c->ev[0], s));
    rc = enqueue_cells(c, s);
    if (rc) return rc;
    ADE_CK(cudaEventRecord(c->ev[1], s));
    if (c->n > 0) {
        ade::EpiOut out = epi_none();
        out.Pout = c->w.P1;
        rc = enqueue_eval(c, PREDICTOR, out, s);
        if (rc) return rc;
        ADE_CK(cudaEventRecord(c->ev[2], s));
        rc = enqueue_eval(c, CORRECTOR, epi_corrector(c), s);
        if (rc) return rc;
        ADE_CK(cudaEventRecord(c->ev[3], s));
        rc = enqueue_fold(c, s);
        if (rc) return rc;
    } else {
        ADE_CK(cudaEventRecord(c->ev[2], s));
        ADE_CK(cudaEventRecord(c->ev[3], s));
    }
    ADE_CK(cudaEventRecord(c->ev[4], s));
    ADE_CK(cudaEventSynchronize(c->ev[4]));
    for (int k = 0; k < 4; ++k) {
        float ms = 0.f;
        ADE_CK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        phase_ms[k] = ms;
    }
    c->step += 1;
    c->t += c->dt;
    return ADE_OK;
}

int ade_launches_per_step(const ade_ctx *c, int *launches)
{
    if (!c || !launches) return fail(ADE_ERR_ARG, "NULL argument");
    // the cell build (count, 2 or 3 scan launches, place, order), [velocity-field gather,]
    // predictor, corrector, fold of the corrector's partials
    *launches = ade::cell_build_launches(c->n, c->ncells, c->w.tile_sums != nullptr) + (c->n > 0 ? 3 + (c->field ? 1 : 0) : 0);
    return ADE_OK;
}

int ade_closed_form_error(ade_ctx *c, const double *x0, double w, double C0, int nimg, double *outh,
                          void *stream)
{
    ade::NvtxRange nvtx_("ade_closed_form_error");
    if (!c || !x0 || !outh) return fail(ADE_ERR_ARG, "NULL argument");
    if (!(w > 0.0) || nimg < 0 || nimg > 8) return fail(ADE_ERR_ARG, "need w > 0 and 0 <= nimg <= 8");
    if (c->field) return fail(ADE_ERR_STATE, "the closed form of Eq. 12-13 is for a uniform velocity");
    cudaStream_t s = (cudaStream_t)stream;
    const int dm = c->dim;
    double center[3] = {0, 0, 0}, box[3] = {1, 1, 1};
    for (int i = 0; i < dm; ++i) {
        box[i] = c->p.box[i];
        double u = x0[i] + c->p.v[i] * c->t;
        center[i] = u - box[i] * floor(u / box[i]);
    }
    // S = w^2 I + 2 t D, its inverse and determinant (2x2 or 3x3 by cofactors)
    double S[3][3] = {{0}};
    for (int i = 0; i < dm; ++i)
        for (int j = 0; j < dm; ++j) S[i][j] = 2.0 * c->t * c->D[i * dm + j] + (i == j ? w * w : 0.0);
    if (dm == 2) S[2][2] = 1.0;
    double c00 = S[1][1] * S[2][2] - S[1][2] * S[2][1];
    double c01 = S[1][2] * S[2][0] - S[1][0] * S[2][2];
    double c02 = S[1][0] * S[2][1] - S[1][1] * S[2][0];
    double det = S[0][0] * c00 + S[0][1] * c01 + S[0][2] * c02;
    double inv[9];
    inv[0] = c00 / det;
    inv[1] = (S[0][2] * S[2][1] - S[0][1] * S[2][2]) / det;
    inv[2] = (S[0][1] * S[1][2] - S[0][2] * S[1][1]) / det;
    inv[3] = c01 / det;
    inv[4] = (S[0][0] * S[2][2] - S[0][2] * S[2][0]) / det;
    inv[5] = (S[0][2] * S[1][0] - S[0][0] * S[1][2]) / det;
    inv[6] = c02 / det;
    inv[7] = (S[0][1] * S[2][0] - S[0][0] * S[2][1]) / det;
    inv[8] = (S[0][0] * S[1][1] - S[0][1] * S[1][0]) / det;
    const double amp = C0 * pow(w, dm) / sqrt(det);
    const int nb = ade::closed_form_blocks(c->n);
    ADE_CK(ade::launch_closed_form_error(dm, c->xq, c->C, c->n, box, center, inv, amp, C0, 0.0, nimg,
                                         c->w.cf_partials, nb, c->w.stats + 4, s));
    double h[3];
    ADE_CK(cudaMemcpyAsync(h, c->w.stats + 4, sizeof(h), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    const double V = c->p.mass / c->p.rho;
    outh[0] = sqrt(V * h[0]);
    outh[1] = c->n > 0 ? h[1] : 0.0;
    outh[2] = c->n > 0 ? sqrt(h[0] / c->n) / C0 : 0.0;
    outh[3] = c->n > 0 ? h[2] : 0.0;
    return ADE_OK;
}

void ade_destroy(ade_ctx *c)
{
    if (!c) return;
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ev_ready)
        for (int k = 0; k < 5; ++k) cudaEventDestroy(c->ev[k]);
    delete c;
}

}  // extern "C"

// =============================================================================================
// Batched plumes: many independent plumes stepped together (one cell build, two persistent rate
// launches per step for the whole batch).
// =============================================================================================

struct ade_batch {
    int P = 0, dim = 0, kernel = 0, N = 0;
    std::vector<ade_params> params;
    std::vector<int> n, offsets;          // caller offsets (offsets[P] = N)
    std::vector<int> subdiv_choice;       // per-plume cell subdivision in use
    std::vector<ade::RateParams> pred, corr;  // per-plume constants for the two evaluations
    std::vector<double> dt, D;            // per-plume time step and tensor (9 each)
    std::vector<int> ncells;
    int NC = 0, NC_max = 0;
    int tile_size = ade::kRateThreads, grid = 0, sms = 0;
    int subdiv_mode = 0;                  // 0 = per-plume cost model, 1..6 forced where valid
    bool paired = false;                  // the rate kernel's threads take two particles (paired walk)
    std::vector<ade::BatchTile> tiles;
    uint32_t *xq = nullptr;
    float *C = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    ade::Work w;
    ade::RateParams *d_pred = nullptr, *d_corr = nullptr;
    ade::BatchTile *d_tiles = nullptr;
    unsigned *queue = nullptr;
    uint16_t *plume_of = nullptr;
    int *d_offsets = nullptr;
    double *d_stats = nullptr;
    int max_tiles = 0;
    long long step = 0;
    bool status_cleared = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

struct BatchLayout {
    size_t keys, rank, count, block_sums, tile_sums, perm_tmp, perm, cell_start, P0, P1, pred, corr, tiles,
        queue, plume_of, offsets, stats, status, pairs, total;
};

BatchLayout batch_layout(int P, int N, int NC_max, int max_tiles)
{
    BatchLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes > 0 ? bytes : 1);
        return o;
    };
    L.keys = take((size_t)N * 4);
    L.rank = take((size_t)N * 4);
    L.count = take((size_t)NC_max * 4);
    L.block_sums = take((size_t)ade::scan_blocks(NC_max) * 4);
    L.tile_sums = take(ade::tile_sums_bytes(NC_max));
    L.perm_tmp = take((size_t)N * 4);
    L.perm = take((size_t)N * 4);
    L.cell_start = take(((size_t)NC_max + 1) * 4);
    L.P0 = take((size_t)N * 16);
    L.P1 = take((size_t)N * 16);
    L.pred = take((size_t)P * sizeof(ade::RateParams));
    L.corr = take((size_t)P * sizeof(ade::RateParams));
    L.tiles = take((size_t)max_tiles * sizeof(ade::BatchTile));
    L.queue = take(64);
    L.plume_of = take((size_t)N * 2);
    L.offsets = take(((size_t)P + 1) * 4);
    L.stats = take((size_t)P * 3 * 8);
    L.status = take(64);
    L.pairs = take(64);
    L.total = off;
    return L;
}

constexpr int kMinTile = 32;

int batch_validate(int P, const ade_params *p, const int *n)
{
    if (P < 1 || P > 65535) return fail(ADE_ERR_ARG, "nplumes must be in 1..65535");
    if (!p || !n) return fail(ADE_ERR_ARG, "NULL argument");
    long long N = 0;
    for (int i = 0; i < P; ++i) {
        int rc = validate(p + i, n[i]);
        if (rc) return rc;
        if (p[i].dim != p[0].dim || p[i].kernel != p[0].kernel)
            return fail(ADE_ERR_ARG, "all plumes of a batch need the same dim and kernel");
        if (!(p[i].box[1] == p[i].box[0] && (p[i].dim == 2 || p[i].box[2] == p[i].box[0])))
            return fail(ADE_ERR_ARG, "batched plumes need a cubic box (equal sides)");
        if (p[i].vmax > 0.0) return fail(ADE_ERR_ARG, "batched plumes have a uniform velocity (vmax must be 0)");
        if (p[i].tau > 0.0) return fail(ADE_ERR_ARG, "batched plumes follow Eq. 1 (tau must be 0)");
        N += n[i];
    }
    if (N > (1ll << 28)) return fail(ADE_ERR_ARG, "total particles exceed 2^28");
    return ADE_OK;
}

// Worst-case total cells over every subdivision a plume may be given.
int batch_max_cells(int P, const ade_params *p, const int *n, long long *nc_max)
{
    long long tot = 0;
    for (int i = 0; i < P; ++i) {
        const double H = p[i].kernel == ADE_WENDLAND_C2 ? 2.0 * p[i].h : p[i].h;
        long long m = 0;
        for (int k = 1; k <= ade::kMaxSubdiv; ++k) {
            Grid g;
            if (make_grid(p[i], H, k, &g)) m = std::max<long long>(m, g.ncells);
        }
        if (m == 0) return fail(ADE_ERR_ARG, "plume %d: box too small for the support radius", i);
        tot += m;
    }
    if (tot > (1ll << ade::kMaxCellBits)) return fail(ADE_ERR_ARG, "batch exceeds 2^24 cells");
    *nc_max = tot;
    return ADE_OK;
}

int batch_max_tiles(int P, const int *n)
{
    long long t = 0;
    for (int i = 0; i < P; ++i) t += (n[i] + kMinTile - 1) / kMinTile;
    return (int)t;
}

// Plan the batch for the current subdivision mode and tile size: per-plume constants, global
// cell offsets and the work list, ordered by decreasing estimated cost (candidates per item).
int batch_plan(ade_batch *b)
{
    b->NC = 0;
    std::vector<std::pair<double, ade::BatchTile>> items;
    for (int i = 0; i < b->P; ++i) {
        ade_params pp = b->params[i];
        if (b->subdiv_mode > 0) {
            const double H = pp.kernel == ADE_WENDLAND_C2 ? 2.0 * pp.h : pp.h;
            Grid g;
            if (make_grid(pp, H, b->subdiv_mode, &g)) pp.cell_subdiv = b->subdiv_mode;
        }
        pp.flags = ADE_FLAG_DIRECT;
        Derived d;
        int rc = derive(&pp, b->n[i], &d);
        if (rc) return rc;
        ade::RateParams rp;
        bool iso = true;
        uint32_t inc[3], inc_half[3];
        rc = plume_constants(&pp, b->n[i], d, &b->D[9 * i], &b->dt[i], inc, inc_half, &rp, &iso);
        if (rc) return rc;
        rp.goff = b->offsets[i];
        rp.coff = b->NC;
        b->ncells[i] = d.g.ncells;
        b->subdiv_choice[i] = d.g.subdiv;
        b->NC += d.g.ncells;
        ade::RateParams pr = rp, co = rp;
        pr.dt = (float)(0.5 * b->dt[i]);
        co.dt = (float)b->dt[i];
        for (int a = 0; a < 3; ++a) {
            pr.inc[a] = inc_half[a];
            pr.back[a] = 0u;
            co.inc[a] = inc[a];
            co.back[a] = inc_half[a];
        }
        b->pred[i] = pr;
        b->corr[i] = co;
        // work items and their estimated cost: candidates per particle x particles
        const double ppc = (double)b->n[i] / d.g.ncells;
        double cand = 0.0;
        for (int r = 0; r < d.g.nrows; ++r) cand += (2 * d.g.rows[r].w + 1) * ppc;
        for (int s0 = 0; s0 < b->n[i]; s0 += b->tile_size) {
            ade::BatchTile t;
            t.plume = i;
            t.start = s0;
            t.count = std::min(b->tile_size, b->n[i] - s0);
            t.pad = 0;
            items.push_back({(cand + 4.0 * d.g.nrows) * t.count, t});
        }
    }
    if (b->NC > b->NC_max) return fail(ADE_ERR_CAPACITY, "batch cell table exceeds the workspace");
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, ade::BatchTile> &x, const std::pair<double, ade::BatchTile> &y) {
                         return x.first > y.first;
                     });
    if ((int)items.size() > b->max_tiles) return fail(ADE_ERR_CAPACITY, "too many work items");
    b->tiles.clear();
    for (auto &it : items) b->tiles.push_back(it.second);
    return ADE_OK;
}

int batch_upload(ade_batch *b, cudaStream_t s)
{
    ADE_CK(cudaMemcpyAsync(b->d_pred, b->pred.data(), b->P * sizeof(ade::RateParams), cudaMemcpyHostToDevice, s));
    ADE_CK(cudaMemcpyAsync(b->d_corr, b->corr.data(), b->P * sizeof(ade::RateParams), cudaMemcpyHostToDevice, s));
    if (!b->tiles.empty())
        ADE_CK(cudaMemcpyAsync(b->d_tiles, b->tiles.data(), b->tiles.size() * sizeof(ade::BatchTile),
                               cudaMemcpyHostToDevice, s));
    ADE_CK(cudaStreamSynchronize(s));   // the host vectors may change before the next call
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return ADE_OK;
}

int batch_cells(ade_batch *b, cudaStream_t s)
{
    ADE_CK(ade::launch_build_cells_batch(b->dim, b->xq, b->C, b->N, b->NC, b->d_pred, b->plume_of, b->w, s));
    return ADE_OK;
}

int batch_enqueue_step(ade_batch *b, cudaStream_t s)
{
    int rc = batch_cells(b, s);
    if (rc) return rc;
    ade::EpiOut out = epi_none();
    out.Pout = b->w.P1;
    ADE_CK(ade::launch_rate_batch(b->dim, b->kernel, ade::EPI_PREDICT, b->w.P0, b->w.cell_start, b->w.perm,
                                  b->d_pred, b->d_tiles, (int)b->tiles.size(), b->queue, b->grid, out, s, b->paired));
    out = epi_none();
    out.xq = b->xq;
    out.C = b->C;
    out.status = b->w.status;
    ADE_CK(ade::launch_rate_batch(b->dim, b->kernel, ade::EPI_CORRECT, b->w.P1, b->w.cell_start, b->w.perm,
                                  b->d_corr, b->d_tiles, (int)b->tiles.size(), b->queue, b->grid, out, s, b->paired));
    return ADE_OK;
}

int batch_clear_status_once(ade_batch *b, cudaStream_t s)
{
    if (!b->status_cleared) {
        ADE_CK(cudaMemsetAsync(b->w.status, 0, sizeof(int), s));
        b->status_cleared = true;
    }
    return ADE_OK;
}

}  // namespace

extern "C" {

int ade_batch_workspace_bytes(int nplumes, const ade_params *p, const int *n, size_t *bytes)
{
    if (!bytes) return fail(ADE_ERR_ARG, "bytes is NULL");
    int rc = batch_validate(nplumes, p, n);
    if (rc) return rc;
    long long ncm = 0;
    rc = batch_max_cells(nplumes, p, n, &ncm);
    if (rc) return rc;
    long long N = 0;
    for (int i = 0; i < nplumes; ++i) N += n[i];
    *bytes = batch_layout(nplumes, (int)N, (int)ncm, batch_max_tiles(nplumes, n)).total;
    return ADE_OK;
}

int ade_batch_init(ade_batch **out, int nplumes, const ade_params *p, const int *n, uint32_t *xq_dev,
                   float *C_dev, void *workspace_dev, size_t workspace_bytes, void *stream)
{
    if (!out) return fail(ADE_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = batch_validate(nplumes, p, n);
    if (rc) return rc;
    long long ncm = 0;
    rc = batch_max_cells(nplumes, p, n, &ncm);
    if (rc) return rc;
    ade_batch *b = new (std::nothrow) ade_batch;
    if (!b) return fail(ADE_ERR_CAPACITY, "out of host memory");
    b->P = nplumes;
    b->dim = p[0].dim;
    b->kernel = p[0].kernel;
    b->params.assign(p, p + nplumes);
    b->n.assign(n, n + nplumes);
    b->offsets.assign(nplumes + 1, 0);
    for (int i = 0; i < nplumes; ++i) b->offsets[i + 1] = b->offsets[i] + n[i];
    b->N = b->offsets[nplumes];
    b->NC_max = (int)ncm;
    b->max_tiles = batch_max_tiles(nplumes, n);
    b->subdiv_choice.assign(nplumes, 0);
    b->ncells.assign(nplumes, 0);
    b->pred.resize(nplumes);
    b->corr.resize(nplumes);
    b->dt.assign(nplumes, 0.0);
    b->D.assign(9 * (size_t)nplumes, 0.0);
    const BatchLayout L = batch_layout(nplumes, b->N, b->NC_max, b->max_tiles);
    if (b->N > 0 && (!xq_dev || !C_dev)) {
        delete b;
        return fail(ADE_ERR_ARG, "xq_dev and C_dev must be non-NULL");
    }
    if (!workspace_dev || ((uintptr_t)workspace_dev & 255u) != 0u) {
        delete b;
        return fail(ADE_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
    }
    if (workspace_bytes < L.total) {
        delete b;
        return fail(ADE_ERR_CAPACITY, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
    }
    b->xq = xq_dev;
    b->C = C_dev;
    b->ws = workspace_dev;
    b->ws_bytes = workspace_bytes;
    memset(&b->w, 0, sizeof(b->w));
    b->w.keys = at<uint32_t>(workspace_dev, L.keys);
    b->w.rank = at<uint32_t>(workspace_dev, L.rank);
    b->w.count = at<uint32_t>(workspace_dev, L.count);
    b->w.block_sums = at<uint32_t>(workspace_dev, L.block_sums);
    b->w.perm_tmp = at<uint32_t>(workspace_dev, L.perm_tmp);
    b->w.perm = at<uint32_t>(workspace_dev, L.perm);
    b->w.cell_start = at<uint32_t>(workspace_dev, L.cell_start);
    b->w.tile_sums = at<uint32_t>(workspace_dev, L.tile_sums);   // cleared with the counts every build
    b->w.P0 = at<uint4>(workspace_dev, L.P0);
    b->w.P1 = at<uint4>(workspace_dev, L.P1);
    b->w.status = at<int>(workspace_dev, L.status);
    b->w.pairs = at<unsigned long long>(workspace_dev, L.pairs);
    b->d_pred = at<ade::RateParams>(workspace_dev, L.pred);
    b->d_corr = at<ade::RateParams>(workspace_dev, L.corr);
    b->d_tiles = at<ade::BatchTile>(workspace_dev, L.tiles);
    b->queue = at<unsigned>(workspace_dev, L.queue);
    b->plume_of = at<uint16_t>(workspace_dev, L.plume_of);
    b->d_offsets = at<int>(workspace_dev, L.offsets);
    b->d_stats = at<double>(workspace_dev, L.stats);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete b;
        return fail(ADE_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    }
    b->grid = b->sms * 8;
    rc = batch_plan(b);
    if (rc) {
        delete b;
        return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint16_t> pid((size_t)b->N);
    for (int i = 0; i < nplumes; ++i)
        std::fill(pid.begin() + b->offsets[i], pid.begin() + b->offsets[i + 1], (uint16_t)i);
    e = cudaSuccess;
    if (b->N > 0) e = cudaMemcpyAsync(b->plume_of, pid.data(), pid.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_offsets, b->offsets.data(), b->offsets.size() * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        delete b;
        return fail(ADE_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }
    rc = batch_upload(b, s);
    if (rc) {
        delete b;
        return rc;
    }
    *out = b;
    return ADE_OK;
}

int ade_batch_step(ade_batch *b, int nsteps, void *stream)
{
    ade::NvtxRange nvtx_("ade_batch_step");
    if (!b || nsteps < 0) return fail(ADE_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = batch_clear_status_once(b, s);
    for (int k = 0; rc == ADE_OK && k < nsteps; ++k) rc = batch_enqueue_step(b, s);
    if (rc) return rc;
    b->step += nsteps;
    return ADE_OK;
}

int ade_batch_run(ade_batch *b, int nsteps, void *stream)
{
    ade::NvtxRange nvtx_("ade_batch_run");
    if (!b || nsteps < 0) return fail(ADE_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = batch_clear_status_once(b, s);
    if (rc) return rc;
    if (!b->graph_exec && nsteps > 0) {
        if (!b->cap_stream) ADE_CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        ADE_CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = batch_enqueue_step(b, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        ADE_CK(e);
        cudaError_t ei = cudaGraphInstantiate(&b->graph_exec, g, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(g);
            b->graph_exec = nullptr;
            return fail(ADE_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
        }
        b->graph = g;
    }
    for (int k = 0; k < nsteps; ++k) ADE_CK(cudaGraphLaunch(b->graph_exec, s));
    b->step += nsteps;
    return ADE_OK;
}

int ade_batch_stats(ade_batch *b, ade_stats *st, void *stream)
{
    if (!b || !st) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = batch_clear_status_once(b, s);
    if (rc) return rc;
    ADE_CK(ade::launch_batch_stats(b->C, b->d_offsets, b->P, b->d_stats, s));
    std::vector<double> h(3 * (size_t)b->P);
    int status = 0;
    ADE_CK(cudaMemcpyAsync(h.data(), b->d_stats, h.size() * 8, cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaMemcpyAsync(&status, b->w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    for (int i = 0; i < b->P; ++i) {
        st[i].mass = h[3 * i] * b->params[i].mass;
        st[i].c_min = b->n[i] > 0 ? h[3 * i + 1] : 0.0;
        st[i].c_max = b->n[i] > 0 ? h[3 * i + 2] : 0.0;
        st[i].t = b->step * b->dt[i];
        st[i].step = b->step;
        st[i].pairs = 0;
        st[i].status = status ? ADE_ERR_NUMERIC : ADE_OK;
    }
    return status ? fail(ADE_ERR_NUMERIC, "non-finite concentration produced") : ADE_OK;
}

int ade_batch_count_pairs(ade_batch *b, long long *pairs_host, void *stream)
{
    if (!b || !pairs_host) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = batch_cells(b, s);
    if (rc) return rc;
    ADE_CK(cudaMemsetAsync(b->w.pairs, 0, 8, s));
    ade::EpiOut out = epi_none();
    out.pairs = b->w.pairs;
    ADE_CK(ade::launch_rate_batch(b->dim, b->kernel, ade::EPI_RATE, b->w.P0, b->w.cell_start, b->w.perm,
                                  b->d_pred, b->d_tiles, (int)b->tiles.size(), b->queue, b->grid, out, s, b->paired));
    unsigned long long v = 0;
    ADE_CK(cudaMemcpyAsync(&v, b->w.pairs, 8, cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    *pairs_host = (long long)v;
    return ADE_OK;
}

int ade_batch_get_config(const ade_batch *b, int *subdiv_mode, int *tile_size, int *grid_blocks, int *paired)
{
    if (!b || !subdiv_mode || !tile_size || !grid_blocks || !paired) return fail(ADE_ERR_ARG, "NULL argument");
    *subdiv_mode = b->subdiv_mode;
    *tile_size = b->tile_size;
    *grid_blocks = b->grid;
    *paired = b->paired ? 1 : 0;
    return ADE_OK;
}

int ade_batch_set_config(ade_batch *b, int subdiv_mode, int tile_size, int grid_blocks, int paired, void *stream)
{
    if (!b) return fail(ADE_ERR_ARG, "batch is NULL");
    if (subdiv_mode < 0 || subdiv_mode > ade::kMaxSubdiv || tile_size < kMinTile || tile_size > 4096 ||
        grid_blocks < 1 || grid_blocks > 65536 || (paired != 0 && paired != 1))
        return fail(ADE_ERR_ARG, "configuration out of range");
    const int m0 = b->subdiv_mode, t0 = b->tile_size, g0 = b->grid;
    const bool p0 = b->paired;
    b->subdiv_mode = subdiv_mode;
    b->tile_size = tile_size;
    b->grid = grid_blocks;
    b->paired = paired != 0;
    int rc = batch_plan(b);
    if (rc) {
        b->subdiv_mode = m0;
        b->tile_size = t0;
        b->grid = g0;
        b->paired = p0;
        batch_plan(b);
        return rc;
    }
    return batch_upload(b, (cudaStream_t)stream);
}

int ade_batch_get_plume_info(const ade_batch *b, int plume, ade_info *info)
{
    if (!b || !info || plume < 0 || plume >= b->P) return fail(ADE_ERR_ARG, "bad argument");
    memset(info, 0, sizeof(*info));
    const ade::RateParams &rp = b->pred[plume];
    const ade_params &p = b->params[plume];
    info->support = p.kernel == ADE_WENDLAND_C2 ? 2.0 * p.h : p.h;
    info->dt = b->dt[plume];
    for (int i = 0; i < 9; ++i) info->D[i] = b->D[9 * plume + i];
    info->nc[0] = rp.ncx;
    info->nc[1] = rp.ncy;
    info->nc[2] = rp.ncz;
    info->ncells = b->ncells[plume];
    info->cell_subdiv = b->subdiv_choice[plume];
    info->stencil_rows = rp.nrows;
    info->sort_passes = 1;
    info->variant = 0;
    info->tile[0] = b->tile_size;
    info->tile[1] = b->grid;
    info->tile[2] = (int)b->tiles.size();
    info->workspace_bytes = b->ws_bytes;
    return ADE_OK;
}

int ade_batch_autotune(ade_batch *b, double *best_ms_host, void *stream)
{
    ade::NvtxRange nvtx_("ade_batch_autotune");
    if (!b) return fail(ADE_ERR_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    ADE_CK(cudaEventCreate(&e0));
    ADE_CK(cudaEventCreate(&e1));
    // one candidate: cell build + one evaluation of every plume (no output), best of two
    auto time_cfg = [&](double *ms) -> int {
        int rc = batch_plan(b);
        if (rc) return rc;
        rc = batch_upload(b, s);
        if (rc) return rc;
        double best = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            ADE_CK(cudaEventRecord(e0, s));
            rc = batch_cells(b, s);
            if (rc) return rc;
            ade::EpiOut out = epi_none();
            ADE_CK(ade::launch_rate_batch(b->dim, b->kernel, ade::EPI_RATE, b->w.P0, b->w.cell_start,
                                          b->w.perm, b->d_pred, b->d_tiles, (int)b->tiles.size(), b->queue,
                                          b->grid, out, s, b->paired));
            ADE_CK(cudaEventRecord(e1, s));
            ADE_CK(cudaEventSynchronize(e1));
            float f = 0.f;
            ADE_CK(cudaEventElapsedTime(&f, e0, e1));
            best = std::min(best, (double)f);
        }
        *ms = best;
        return ADE_OK;
    };
    int rc = ADE_OK;
    double best = 1e30, ms = 0.0;
    int best_mode = b->subdiv_mode, best_tile = b->tile_size, best_grid = b->grid;
    for (int mode = 0; rc == ADE_OK && mode <= ade::kMaxSubdiv; ++mode) {
        b->subdiv_mode = mode;
        rc = time_cfg(&ms);
        if (rc == ADE_OK && ms < best) {
            best = ms;
            best_mode = mode;
        }
    }
    b->subdiv_mode = best_mode;
    const int tile_sizes[] = {64, 128, 256, 512, 1024};
    for (int ti = 0; rc == ADE_OK && ti < 5; ++ti) {
        b->tile_size = tile_sizes[ti];
        rc = time_cfg(&ms);
        if (rc == ADE_OK && ms < best) {
            best = ms;
            best_tile = tile_sizes[ti];
        }
    }
    b->tile_size = best_tile;
    const int per_sm[] = {4, 8, 16};
    for (int gi = 0; rc == ADE_OK && gi < 3; ++gi) {
        b->grid = b->sms * per_sm[gi];
        rc = time_cfg(&ms);
        if (rc == ADE_OK && ms < best) {
            best = ms;
            best_grid = b->grid;
        }
    }
    b->grid = best_grid;
    // the walk: one particle per thread, or two adjacent particles (paired walk)
    bool best_paired = b->paired;
    for (int pw = 0; rc == ADE_OK && pw < 2; ++pw) {
        b->paired = pw == 1;
        rc = time_cfg(&ms);
        if (rc == ADE_OK && ms < best) {
            best = ms;
            best_paired = b->paired;
        }
    }
    b->paired = best_paired;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = batch_plan(b);
    if (rc) return rc;
    rc = batch_upload(b, s);
    if (rc) return rc;
    if (best_ms_host) *best_ms_host = best;
    return ADE_OK;
}

int ade_batch_step_timed(ade_batch *b, double *phase_ms, void *stream)
{
    ade::NvtxRange nvtx_("ade_batch_step_timed");
    if (!b || !phase_ms) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = batch_clear_status_once(b, s);
    if (rc) return rc;
    cudaEvent_t ev[4];
    for (int k = 0; k < 4; ++k) ADE_CK(cudaEventCreate(&ev[k]));
    ADE_CK(cudaEventRecord(ev[0], s));
    rc = batch_cells(b, s);
    if (rc) return rc;
    ADE_CK(cudaEventRecord(ev[1], s));
    ade::EpiOut out = epi_none();
    out.Pout = b->w.P1;
    ADE_CK(ade::launch_rate_batch(b->dim, b->kernel, ade::EPI_PREDICT, b->w.P0, b->w.cell_start, b->w.perm,
                                  b->d_pred, b->d_tiles, (int)b->tiles.size(), b->queue, b->grid, out, s, b->paired));
    ADE_CK(cudaEventRecord(ev[2], s));
    out = epi_none();
    out.xq = b->xq;
    out.C = b->C;
    out.status = b->w.status;
    ADE_CK(ade::launch_rate_batch(b->dim, b->kernel, ade::EPI_CORRECT, b->w.P1, b->w.cell_start, b->w.perm,
                                  b->d_corr, b->d_tiles, (int)b->tiles.size(), b->queue, b->grid, out, s, b->paired));
    ADE_CK(cudaEventRecord(ev[3], s));
    ADE_CK(cudaEventSynchronize(ev[3]));
    for (int k = 0; k < 3; ++k) {
        float ms = 0.f;
        ADE_CK(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
        phase_ms[k] = ms;
    }
    phase_ms[3] = 0.0;
    for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
    b->step += 1;
    return ADE_OK;
}

int ade_batch_launches_per_step(const ade_batch *b, int *launches)
{
    if (!b || !launches) return fail(ADE_ERR_ARG, "NULL argument");
    *launches = b->w.tile_sums ? 6 : 8;  // count, the scan (one launch, else three), place, order, predictor, corrector
    return ADE_OK;
}

void ade_batch_destroy(ade_batch *b)
{
    if (!b) return;
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

}  // extern "C"

// =============================================================================================
// Parameter sweep: one plume, P dispersivity sets sharing particles, velocity and time step.
// =============================================================================================

struct ade_sweep {
    ade_params p;                      // geometry and velocity (dispersivities of set 0)
    int n = 0, dim = 0, P = 0, P4 = 0;
    int nc[3] = {1, 1, 1};
    int ncells = 0;
    uint32_t *xq = nullptr;
    float *C = nullptr;                // caller concentrations [P][n]
    ade::Work w;
    float *Cs0 = nullptr, *Cs1 = nullptr;   // sorted, interleaved [n][P4] at l and l + 1/2
    double *pstats = nullptr;               // {sum, min, max} per set
    ade::RateParams rp;
    std::vector<ade::SweepParams> groups;
    std::vector<double> theta;              // [P][3]
    double dt = 0.0, t = 0.0;
    long long step = 0, pairs = 0;
    uint32_t inc[3], inc_half[3];
    bool status_cleared = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev[4];
    bool ev_ready = false;
};

namespace {

struct SweepLayout {
    Derived d;
    size_t Cs0, Cs1, pstats, total;
};

// Common parameters and workspace of a sweep.  theta may be NULL (workspace size only: the layout
// does not depend on the dispersivities or the time step).
int sweep_layout(const ade_params *p, int n, int P, const double *theta, ade_params *pp_out, SweepLayout *L)
{
    if (!p) return fail(ADE_ERR_ARG, "params is NULL");
    if (P < 1 || P > ade::kSweepMax) return fail(ADE_ERR_ARG, "ntheta must be in 1..%d", ade::kSweepMax);
    if (p->vmax > 0.0) return fail(ADE_ERR_ARG, "a sweep has a uniform velocity (vmax must be 0)");
    if (p->tau > 0.0) return fail(ADE_ERR_ARG, "a sweep follows Eq. 1 (tau must be 0)");
    if (p->flags != 0u && p->flags != ADE_FLAG_DIRECT) return fail(ADE_ERR_ARG, "a sweep uses the direct walk");
    ade_params pp = *p;
    pp.flags = ADE_FLAG_DIRECT;
    if (theta) {
        for (int k = 0; k < P; ++k)
            for (int j = 0; j < 3; ++j)
                if (!(theta[3 * k + j] >= 0.0) || !isfinite(theta[3 * k + j]))
                    return fail(ADE_ERR_ARG, "theta[%d] must be finite and >= 0", k);
        if (!(p->dt > 0.0)) {
            // one time step for all sets: the smallest the rule gives over the sets (a set with a
            // zero tensor does not disperse and sets no limit)
            double dtmin = 0.0;
            bool any = false;
            for (int k = 0; k < P; ++k) {
                ade_params q = pp;
                q.alpha_L = theta[3 * k];
                q.alpha_T = theta[3 * k + 1];
                q.D_m = theta[3 * k + 2];
                double D[9], dtk = 0.0, dmax = 0.0;
                dispersion_tensor(q.dim == 3 ? 3 : 2, q.v, q.alpha_L, q.alpha_T, q.D_m, D);
                for (int i = 0; i < 9; ++i) dmax = fmax(dmax, fabs(D[i]));
                if (!(dmax > 0.0)) continue;
                int rc = time_step(&q, D, &dtk);
                if (rc) return rc;
                dtmin = any ? std::min(dtmin, dtk) : dtk;
                any = true;
            }
            if (!any) return fail(ADE_ERR_ARG, "every set has a zero dispersion tensor: give dt explicitly");
            pp.dt = dtmin;
        }
        pp.alpha_L = theta[0];
        pp.alpha_T = theta[1];
        pp.D_m = theta[2];
    } else if (!(pp.dt > 0.0)) {
        pp.dt = 1.0;
    }
    int rc = derive(&pp, n, &L->d);
    if (rc) return rc;
    const int P4 = (P + 3) & ~3;
    size_t off = L->d.L.total;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes > 0 ? bytes : 1);
        return o;
    };
    L->Cs0 = take((size_t)n * P4 * 4);
    L->Cs1 = take((size_t)n * P4 * 4);
    L->pstats = take((size_t)3 * P * 8);
    L->total = off;
    if (pp_out) *pp_out = pp;
    return ADE_OK;
}

int sweep_cells(ade_sweep *sw, cudaStream_t s)
{
    ADE_CK(ade::launch_build_cells(sw->dim, sw->xq, sw->C, sw->n, sw->nc, sw->ncells, sw->w, s));
    ADE_CK(ade::launch_sweep_gather(sw->w.perm, sw->C, sw->n, sw->P, sw->P4, sw->Cs0, s));
    return ADE_OK;
}

// The evaluations of every group: predictors (all groups), or correctors (all groups).
int sweep_evals(ade_sweep *sw, int ph, cudaStream_t s)
{
    ade::RateParams rp = sw->rp;
    ade::SweepOut out;
    memset(&out, 0, sizeof(out));
    const uint4 *Pe = sw->w.P0;
    const float *Ce = sw->Cs0;
    int epi = ade::EPI_PREDICT;
    if (ph == 1) {
        rp.dt = (float)(0.5 * sw->dt);
        for (int i = 0; i < 3; ++i) {
            rp.inc[i] = sw->inc_half[i];
            rp.back[i] = 0u;
        }
        out.Cout = sw->Cs1;
        out.Pout = sw->w.P1;
    } else {
        epi = ade::EPI_CORRECT;
        Pe = sw->w.P1;
        Ce = sw->Cs1;
        rp.dt = (float)sw->dt;
        for (int i = 0; i < 3; ++i) {
            rp.inc[i] = sw->inc[i];
            rp.back[i] = sw->inc_half[i];
        }
        out.C = sw->C;
        out.xq = sw->xq;
        out.status = sw->w.status;
    }
    for (const ade::SweepParams &g : sw->groups)
        ADE_CK(ade::launch_rate_sweep(sw->dim, sw->p.kernel, epi, false, Pe, Ce, sw->w.cell_start, sw->w.perm, rp,
                                      g, out, s));
    return ADE_OK;
}

int sweep_step(ade_sweep *sw, cudaStream_t s)
{
    int rc = sweep_cells(sw, s);
    if (rc || sw->n == 0) return rc;
    rc = sweep_evals(sw, 1, s);
    if (rc) return rc;
    return sweep_evals(sw, 2, s);
}

int sweep_clear_status_once(ade_sweep *sw, cudaStream_t s)
{
    if (!sw->status_cleared) {
        ADE_CK(cudaMemsetAsync(sw->w.status, 0, sizeof(int), s));
        sw->status_cleared = true;
    }
    return ADE_OK;
}

}  // namespace

extern "C" {

int ade_sweep_workspace_bytes(const ade_params *p, int n, int ntheta, size_t *bytes)
{
    if (!bytes) return fail(ADE_ERR_ARG, "bytes is NULL");
    SweepLayout L;
    int rc = sweep_layout(p, n, ntheta, nullptr, nullptr, &L);
    if (rc) return rc;
    *bytes = L.total;
    return ADE_OK;
}

int ade_sweep_init(ade_sweep **out, const ade_params *p, int n, int ntheta, const double *theta_host,
                   uint32_t *xq_dev, float *C_dev, void *workspace_dev, size_t workspace_bytes)
{
    if (!out) return fail(ADE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!theta_host) return fail(ADE_ERR_ARG, "theta_host is NULL");
    ade_params pp;
    SweepLayout L;
    int rc = sweep_layout(p, n, ntheta, theta_host, &pp, &L);
    if (rc) return rc;
    if (n > 0 && (!xq_dev || !C_dev)) return fail(ADE_ERR_ARG, "xq_dev and C_dev must be non-NULL");
    if (!workspace_dev || ((uintptr_t)workspace_dev & 255u) != 0u)
        return fail(ADE_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
    if (workspace_bytes < L.total)
        return fail(ADE_ERR_CAPACITY, "workspace too small: %zu < %zu bytes", workspace_bytes, L.total);
    ade_sweep *sw = new (std::nothrow) ade_sweep;
    if (!sw) return fail(ADE_ERR_CAPACITY, "out of host memory");
    sw->p = pp;
    sw->n = n;
    sw->dim = pp.dim;
    sw->P = ntheta;
    sw->P4 = (ntheta + 3) & ~3;
    for (int i = 0; i < 3; ++i) sw->nc[i] = L.d.g.nc[i];
    sw->ncells = L.d.g.ncells;
    sw->xq = xq_dev;
    sw->C = C_dev;
    const Layout &W = L.d.L;
    sw->w.keys = at<uint32_t>(workspace_dev, W.keys);
    sw->w.rank = at<uint32_t>(workspace_dev, W.rank);
    sw->w.count = at<uint32_t>(workspace_dev, W.count);
    sw->w.block_sums = at<uint32_t>(workspace_dev, W.block_sums);
    sw->w.perm_tmp = at<uint32_t>(workspace_dev, W.perm_tmp);
    sw->w.perm = at<uint32_t>(workspace_dev, W.perm);
    sw->w.cell_start = at<uint32_t>(workspace_dev, W.cell_start);
    sw->w.tile_sums = at<uint32_t>(workspace_dev, W.tile_sums);   // cleared with the counts every build
    sw->w.P0 = at<uint4>(workspace_dev, W.P0);
    sw->w.P1 = at<uint4>(workspace_dev, W.P1);
    sw->w.partials = at<double>(workspace_dev, W.partials);
    sw->w.wpart = at<float4>(workspace_dev, W.wpart);
    sw->w.stats = at<double>(workspace_dev, W.stats);
    sw->w.cf_partials = at<double>(workspace_dev, W.cf_partials);
    sw->w.status = at<int>(workspace_dev, W.status);
    sw->w.pairs = at<unsigned long long>(workspace_dev, W.pairs);
    sw->Cs0 = at<float>(workspace_dev, L.Cs0);
    sw->Cs1 = at<float>(workspace_dev, L.Cs1);
    sw->pstats = at<double>(workspace_dev, L.pstats);
    double D[9];
    bool iso = false;
    rc = plume_constants(&pp, n, L.d, D, &sw->dt, sw->inc, sw->inc_half, &sw->rp, &iso);
    if (rc) {
        delete sw;
        return rc;
    }
    sw->rp.variant = 0;
    sw->theta.assign(theta_host, theta_host + 3 * ntheta);
    // Dcal = a u + b per set (uniform v, K = 2D)
    const int dm = pp.dim;
    double vabs = 0.0;
    for (int i = 0; i < dm; ++i) vabs += pp.v[i] * pp.v[i];
    vabs = sqrt(vabs);
    const double gamma = pp.gamma > 0.0 ? pp.gamma : dm + 2.0;
    ade::SweepParams base;
    memset(&base, 0, sizeof(base));
    for (int i = 0; i < 3; ++i) base.vh[i] = vabs > 0.0 ? (float)(i < dm ? pp.v[i] / vabs : 0.0) : (i == 0 ? 1.f : 0.f);
    base.P4 = sw->P4;
    for (int g0 = 0; g0 < ntheta;) {
        int nt = ade::kSweepGroup;
        while (nt > ntheta - g0) nt >>= 1;
        ade::SweepParams g = base;
        g.g0 = g0;
        g.nt = nt;
        for (int k = 0; k < nt; ++k) {
            const double aL = theta_host[3 * (g0 + k)], aT = theta_host[3 * (g0 + k) + 1],
                         Dm = theta_host[3 * (g0 + k) + 2];
            g.a[k] = (float)(2.0 * gamma * (aL - aT) * vabs);
            g.b[k] = (float)(2.0 * (gamma - dm) * (aT * vabs + Dm) - 2.0 * (aL - aT) * vabs);
        }
        sw->groups.push_back(g);
        g0 += nt;
    }
    *out = sw;
    return ADE_OK;
}

int ade_sweep_get_info(const ade_sweep *sw, ade_info *info)
{
    if (!sw || !info) return fail(ADE_ERR_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->support = sw->p.kernel == ADE_WENDLAND_C2 ? 2.0 * sw->p.h : sw->p.h;
    info->dt = sw->dt;
    for (int i = 0; i < 3; ++i) info->nc[i] = sw->nc[i];
    info->ncells = sw->ncells;
    info->cell_subdiv = sw->rp.k;
    info->stencil_rows = sw->rp.nrows;
    info->sort_passes = 1;
    info->tile[0] = (int)sw->groups.size();   // launches per evaluation
    return ADE_OK;
}

int ade_sweep_rate(ade_sweep *sw, float *dCdt_dev, void *stream)
{
    ade::NvtxRange nvtx_("ade_sweep_rate");
    if (!sw) return fail(ADE_ERR_ARG, "sweep is NULL");
    if (sw->n > 0 && !dCdt_dev) return fail(ADE_ERR_ARG, "dCdt_dev is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = sweep_cells(sw, s);
    if (rc || sw->n == 0) return rc;
    ade::SweepOut out;
    memset(&out, 0, sizeof(out));
    out.rate = dCdt_dev;
    for (const ade::SweepParams &g : sw->groups)
        ADE_CK(ade::launch_rate_sweep(sw->dim, sw->p.kernel, ade::EPI_RATE, false, sw->w.P0, sw->Cs0,
                                      sw->w.cell_start, sw->w.perm, sw->rp, g, out, s));
    return ADE_OK;
}

int ade_sweep_count_pairs(ade_sweep *sw, long long *pairs_host, void *stream)
{
    if (!sw || !pairs_host) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    *pairs_host = 0;
    int rc = sweep_cells(sw, s);
    if (rc || sw->n == 0) return rc;
    ADE_CK(cudaMemsetAsync(sw->w.pairs, 0, 8, s));
    ade::SweepOut out;
    memset(&out, 0, sizeof(out));
    out.pairs = sw->w.pairs;
    ADE_CK(ade::launch_rate_sweep(sw->dim, sw->p.kernel, ade::EPI_RATE, true, sw->w.P0, sw->Cs0, sw->w.cell_start,
                                  sw->w.perm, sw->rp, sw->groups[0], out, s));
    unsigned long long v = 0;
    ADE_CK(cudaMemcpyAsync(&v, sw->w.pairs, 8, cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    sw->pairs = (long long)v;
    *pairs_host = (long long)v;
    return ADE_OK;
}

int ade_sweep_step(ade_sweep *sw, int nsteps, void *stream)
{
    ade::NvtxRange nvtx_("ade_sweep_step");
    if (!sw) return fail(ADE_ERR_ARG, "sweep is NULL");
    if (nsteps < 0) return fail(ADE_ERR_ARG, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = sweep_clear_status_once(sw, s);
    if (rc) return rc;
    for (int k = 0; k < nsteps; ++k) {
        rc = sweep_step(sw, s);
        if (rc) return rc;
    }
    sw->step += nsteps;
    sw->t += nsteps * sw->dt;
    return ADE_OK;
}

int ade_sweep_run(ade_sweep *sw, int nsteps, void *stream)
{
    ade::NvtxRange nvtx_("ade_sweep_run");
    if (!sw) return fail(ADE_ERR_ARG, "sweep is NULL");
    if (nsteps < 0) return fail(ADE_ERR_ARG, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = sweep_clear_status_once(sw, s);
    if (rc) return rc;
    if (!sw->graph_exec && nsteps > 0) {
        if (!sw->cap_stream) ADE_CK(cudaStreamCreateWithFlags(&sw->cap_stream, cudaStreamNonBlocking));
        ADE_CK(cudaStreamBeginCapture(sw->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = sweep_step(sw, sw->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(sw->cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        ADE_CK(e);
        cudaError_t ei = cudaGraphInstantiate(&sw->graph_exec, g, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(g);
            sw->graph_exec = nullptr;
            return fail(ADE_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
        }
        sw->graph = g;
    }
    for (int k = 0; k < nsteps; ++k) ADE_CK(cudaGraphLaunch(sw->graph_exec, s));
    sw->step += nsteps;
    sw->t += nsteps * sw->dt;
    return ADE_OK;
}

int ade_sweep_step_timed(ade_sweep *sw, double *phase_ms, void *stream)
{
    ade::NvtxRange nvtx_("ade_sweep_step_timed");
    if (!sw || !phase_ms) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = sweep_clear_status_once(sw, s);
    if (rc) return rc;
    if (!sw->ev_ready) {
        for (int k = 0; k < 4; ++k) ADE_CK(cudaEventCreate(&sw->ev[k]));
        sw->ev_ready = true;
    }
    ADE_CK(cudaEventRecord(sw->ev[0], s));
    rc = sweep_cells(sw, s);
    if (rc) return rc;
    ADE_CK(cudaEventRecord(sw->ev[1], s));
    if (sw->n > 0) {
        rc = sweep_evals(sw, 1, s);
        if (rc) return rc;
    }
    ADE_CK(cudaEventRecord(sw->ev[2], s));
    if (sw->n > 0) {
        rc = sweep_evals(sw, 2, s);
        if (rc) return rc;
    }
    ADE_CK(cudaEventRecord(sw->ev[3], s));
    ADE_CK(cudaEventSynchronize(sw->ev[3]));
    for (int k = 0; k < 3; ++k) {
        float ms = 0.f;
        ADE_CK(cudaEventElapsedTime(&ms, sw->ev[k], sw->ev[k + 1]));
        phase_ms[k] = ms;
    }
    phase_ms[3] = 0.0;
    sw->step += 1;
    sw->t += sw->dt;
    return ADE_OK;
}

int ade_sweep_launches_per_step(const ade_sweep *sw, int *launches)
{
    if (!sw || !launches) return fail(ADE_ERR_ARG, "NULL argument");
    // the cell build (count, 2 or 3 scan launches, place, order), gather; one predictor and one
    // corrector per group
    *launches = ade::cell_build_launches(sw->n, sw->ncells, sw->w.tile_sums != nullptr) + (sw->n > 0 ? 1 + 2 * (int)sw->groups.size() : 0);
    return ADE_OK;
}

int ade_sweep_stats(ade_sweep *sw, ade_stats *st, void *stream)
{
    if (!sw || !st) return fail(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = sweep_clear_status_once(sw, s);
    if (rc) return rc;
    for (int k = 0; k < sw->P; ++k)
        ADE_CK(ade::launch_state_stats(sw->C + (size_t)k * sw->n, sw->n, sw->w.partials, sw->pstats + 3 * k, s));
    std::vector<double> h(3 * (size_t)sw->P);
    int status = 0;
    ADE_CK(cudaMemcpyAsync(h.data(), sw->pstats, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaMemcpyAsync(&status, sw->w.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    ADE_CK(cudaStreamSynchronize(s));
    for (int k = 0; k < sw->P; ++k) {
        st[k].mass = h[3 * k] * sw->p.mass;
        st[k].c_min = h[3 * k + 1];
        st[k].c_max = h[3 * k + 2];
        st[k].t = sw->t;
        st[k].step = sw->step;
        st[k].pairs = sw->pairs;
        st[k].status = status ? ADE_ERR_NUMERIC : ADE_OK;
    }
    return status ? fail(ADE_ERR_NUMERIC, "non-finite concentration produced") : ADE_OK;
}

void ade_sweep_destroy(ade_sweep *sw)
{
    if (!sw) return;
    if (sw->graph_exec) cudaGraphExecDestroy(sw->graph_exec);
    if (sw->graph) cudaGraphDestroy(sw->graph);
    if (sw->cap_stream) cudaStreamDestroy(sw->cap_stream);
    if (sw->ev_ready)
        for (int k = 0; k < 4; ++k) cudaEventDestroy(sw->ev[k]);
    delete sw;
}

}  // extern "C"
