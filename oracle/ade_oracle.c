/*
 * ade_oracle.c -- plain FP64 CPU oracle for the SPH advection-dispersion path.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU-baseline
 * leg of the benchmark are the only callers.  The GPU library never links, loads or
 * calls this file, and this file includes nothing from the GPU library.
 *
 * Source: Klapp, Sigalotti, Alvarado-Rodriguez, Rendon, "Consistent SPH simulations
 * of the anisotropic dispersion of a contaminant plume" (arXiv 2108.09488).
 *   Sec. 2.1, Eq. 1-3  Lagrangian ADE and the dispersion tensor
 *   Sec. 2.2, Eq. 4-5  SPH rate dC/dt (dispersive pair sum + convective term)
 *   Sec. 2.3, Eq. 7    Wendland C4 kernel (its h is the support radius)
 *   Sec. 2.4, Eq. 8-9  predictor-corrector update
 *   Sec. 3,   Eq. 12-13 closed-form advected anisotropic Gaussian
 *
 * Everything is written for clarity, not speed: one particle at a time, FP64,
 * no blocking and no reordering beyond what the equations state.  OpenMP only
 * splits the outer loop over particles; each particle's sum runs sequentially.
 *
 * Readings taken where the paper is silent or garbled (each one is repeated at the
 * function that uses it):
 *   - support radius H: Wendland C2 has support 2h; Wendland C4 has support h (Eq. 7);
 *   - the pair sum runs over b != a with |x_ab| < H, minimum-image distance in the
 *     periodic box (Sec. 3); pairs at zero distance are skipped (Eq. 5 is 0/0 there);
 *   - harmonic mean 4 D_a D_b / (D_a + D_b) is taken as 0 when D_a + D_b == 0;
 *   - Gamma = m + 2 (4 in 2D as printed after Eq. 5, 5 in 3D);
 *   - Eq. 8's position line is read as the midpoint x^{l+1/2} = x^l + dt/2 v and the
 *     rate at level l is evaluated fresh each step (two evaluations per step);
 *   - Eq. 12's denominator is read as 8 t^2 C2 + 4 w^2 t C3 + 2 w^4 (= 2 C4^2) and its
 *     centre as x0 + v t, summed over periodic images.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORC_WENDLAND_C2 = 0, ORC_WENDLAND_C4 = 1 };

/* ------------------------------------------------------------------------- */
/* Eq. 3: D_ij = (aT |v| + Dm) delta_ij + (aL - aT) v_i v_j / |v|.            */
/* At |v| = 0 the second term is taken as 0 (the limit of v_i v_j/|v|).      */
/* D is dim x dim, row-major.                                                */
/* ------------------------------------------------------------------------- */
void orc_dispersion_tensor(int dim, const double *v, double aL, double aT, double Dm,
                           double *D)
{
    double s = 0.0;
    for (int i = 0; i < dim; ++i) s += v[i] * v[i];
    double vabs = sqrt(s);
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
            double d = (i == j) ? (aT * vabs + Dm) : 0.0;
            if (vabs > 0.0) d += (aL - aT) * (v[i] * v[j]) / vabs;
            D[i * dim + j] = d;
        }
}

/* ------------------------------------------------------------------------- */
/* Kernels, written for the support radius H and q = r/H.                    */
/*   Wendland C4 (Eq. 7): W = B (1-q)^6 (1 + 6q + 35 q^2/3),                 */
/*     B = 9/(pi H^2) in 2D (as printed), 495/(32 pi H^3) in 3D.             */
/*   Wendland C2 (support 2h): W = B (1-q)^4 (1 + 4q),                       */
/*     B = 7/(pi H^2) in 2D, 21/(2 pi H^3) in 3D.                            */
/* The 3D and C2 normalisations are those of the Wendland family (Dehnen and */
/* Aly 2012, cited with Eq. 7); the tests integrate W to 1 by quadrature.    */
/* ------------------------------------------------------------------------- */
static double kernel_norm(int kind, int dim, double H)
{
    if (kind == ORC_WENDLAND_C4)
        return dim == 2 ? 9.0 / (M_PI * H * H) : 495.0 / (32.0 * M_PI * H * H * H);
    return dim == 2 ? 7.0 / (M_PI * H * H) : 21.0 / (2.0 * M_PI * H * H * H);
}

double orc_kernel_w(int kind, int dim, double H, double r)
{
    double q = r / H;
    if (q >= 1.0) return 0.0;
    double B = kernel_norm(kind, dim, H);
    double omq = 1.0 - q;
    if (kind == ORC_WENDLAND_C4)
        return B * pow(omq, 6) * (1.0 + 6.0 * q + 35.0 * q * q / 3.0);
    return B * pow(omq, 4) * (1.0 + 4.0 * q);
}

/* dW/dr, by the product rule on the expressions above:
 *   C4: dW/dq = B[-6(1-q)^5 (1 + 6q + 35q^2/3) + (1-q)^6 (6 + 70q/3)]
 *   C2: dW/dq = B[-4(1-q)^3 (1 + 4q) + 4 (1-q)^4]
 * and dW/dr = dW/dq / H.                                                    */
double orc_kernel_dwdr(int kind, int dim, double H, double r)
{
    double q = r / H;
    if (q >= 1.0) return 0.0;
    double B = kernel_norm(kind, dim, H);
    double omq = 1.0 - q;
    double dWdq;
    if (kind == ORC_WENDLAND_C4)
        dWdq = B * (-6.0 * pow(omq, 5) * (1.0 + 6.0 * q + 35.0 * q * q / 3.0) +
                    pow(omq, 6) * (6.0 + 70.0 * q / 3.0));
    else
        dWdq = B * (-4.0 * pow(omq, 3) * (1.0 + 4.0 * q) + 4.0 * pow(omq, 4));
    return dWdq / H;
}

/* ------------------------------------------------------------------------- */
/* Periodic minimum image (Sec. 3: periodic borders of the square).          */
/* ------------------------------------------------------------------------- */
static void min_image(int dim, const double *xa, const double *xb, const double *box,
                      double *xab)
{
    for (int i = 0; i < dim; ++i) {
        double d = xa[i] - xb[i];
        d -= box[i] * nearbyint(d / box[i]);
        xab[i] = d;
    }
}

/* ------------------------------------------------------------------------- */
/* One ordered pair (a, b) of Eq. 4, split into its two sums.                */
/*   disp = 1/2 (m_b / rhobar_ab) Dcal_ab (C_a - C_b) x_ab . grad_a W_ab / r^2 */
/*   conv = C_a (m_b / rhobar_ab) sum_i (v_i,a - v_i,b) dW_ab/dx_i,a          */
/* with Eq. 5: Dcal_ab = sum_ij [4 D_ij,a D_ij,b / (D_ij,a + D_ij,b)]         */
/*                           [Gamma x_i x_j / r^2 - delta_ij]                */
/* and grad_a W_ab = (dW/dr) x_ab / r.  rhobar_ab = (rho_a + rho_b)/2.        */
/* ------------------------------------------------------------------------- */
void orc_pair_term(int dim, const double *xab, const double *Da, const double *Db,
                   double Ca, double Cb, const double *va, const double *vb, double mb,
                   double rhoa, double rhob, int kind, double H, double gamma,
                   double *disp, double *conv)
{
    double r2 = 0.0;
    for (int i = 0; i < dim; ++i) r2 += xab[i] * xab[i];
    double r = sqrt(r2);
    double dWdr = orc_kernel_dwdr(kind, dim, H, r);
    double rhobar = 0.5 * (rhoa + rhob);

    double Dcal = 0.0;
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
            double den = Da[i * dim + j] + Db[i * dim + j];
            double K = (den != 0.0) ? 4.0 * Da[i * dim + j] * Db[i * dim + j] / den : 0.0;
            Dcal += K * (gamma * xab[i] * xab[j] / r2 - (i == j ? 1.0 : 0.0));
        }

    double gradW[3];
    double xdotgrad = 0.0;
    for (int i = 0; i < dim; ++i) {
        gradW[i] = dWdr * xab[i] / r;
        xdotgrad += xab[i] * gradW[i];
    }
    *disp = 0.5 * (mb / rhobar) * Dcal * (Ca - Cb) * xdotgrad / r2;

    double dv = 0.0;
    for (int i = 0; i < dim; ++i) dv += (va[i] - vb[i]) * gradW[i];
    *conv = Ca * (mb / rhobar) * dv;
}

/* ------------------------------------------------------------------------- */
/* Neighbour lists in CSR form: ptr[n+1], idx[ptr[n]].                      */
/* Neighbours of a are all b != a with minimum-image distance 0 < r < H.     */
/* Brute force: every pair is examined.                                      */
/* Cell list: the classic head/next linked list of cells of side >= H, with  */
/* the 3^dim surrounding cells visited under periodic wrap.  Used only when  */
/* every axis has at least 3 cells; otherwise brute force is used.  Within   */
/* each particle's list the neighbours are sorted by index, so both methods   */
/* return identical lists.                                                   */
/* Returns the number of neighbours, or -1 if cap is too small.              */
/* ------------------------------------------------------------------------- */
static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static int in_support(int dim, const double *x, int a, int b, const double *box, double H)
{
    double xab[3];
    min_image(dim, x + (size_t)a * dim, x + (size_t)b * dim, box, xab);
    double r2 = 0.0;
    for (int i = 0; i < dim; ++i) r2 += xab[i] * xab[i];
    return r2 > 0.0 && r2 < H * H;
}

long long orc_neighbours_brute(int dim, int n, const double *x, const double *box, double H,
                               long long *ptr, int *idx, long long cap)
{
    long long k = 0;
    for (int a = 0; a < n; ++a) {
        ptr[a] = k;
        for (int b = 0; b < n; ++b) {
            if (b == a || !in_support(dim, x, a, b, box, H)) continue;
            if (k >= cap) return -1;
            idx[k++] = b;
        }
    }
    ptr[n] = k;
    return k;
}

typedef struct {
    int dim, nc[3], ncells;
    int *head, *next;
} cell_list;

static int cells_usable(int dim, const double *box, double H, int *nc)
{
    for (int i = 0; i < 3; ++i) nc[i] = 1;
    for (int i = 0; i < dim; ++i) {
        nc[i] = (int)floor(box[i] / H);
        if (nc[i] < 3) return 0;
    }
    return 1;
}

static int cell_of(int dim, const double *xa, const double *box, const int *nc, int *c)
{
    for (int i = 0; i < dim; ++i) {
        double u = xa[i] / box[i];
        u -= floor(u);
        int ci = (int)floor(u * nc[i]);
        if (ci >= nc[i]) ci = nc[i] - 1;
        if (ci < 0) ci = 0;
        c[i] = ci;
    }
    for (int i = dim; i < 3; ++i) c[i] = 0;
    return (c[2] * nc[1] + c[1]) * nc[0] + c[0];
}

static int build_cell_list(int dim, int n, const double *x, const double *box, double H,
                           cell_list *cl)
{
    cl->dim = dim;
    if (!cells_usable(dim, box, H, cl->nc)) return 0;
    cl->ncells = cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->head = (int *)malloc(sizeof(int) * (size_t)cl->ncells);
    cl->next = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < cl->ncells; ++c) cl->head[c] = -1;
    for (int a = n - 1; a >= 0; --a) {
        int ci[3];
        int c = cell_of(dim, x + (size_t)a * dim, box, cl->nc, ci);
        cl->next[a] = cl->head[c];
        cl->head[c] = a;
    }
    return 1;
}

static void free_cell_list(cell_list *cl)
{
    free(cl->head);
    free(cl->next);
}

/* Collect the neighbours of particle a from the cell list into buf (unsorted). */
static int cell_neighbours(const cell_list *cl, const double *x, const double *box, double H,
                           int a, int *buf)
{
    int dim = cl->dim, ca[3], cnt = 0;
    cell_of(dim, x + (size_t)a * dim, box, cl->nc, ca);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) { lo[i] = -1; hi[i] = 1; }
    for (int dz = lo[2]; dz <= hi[2]; ++dz)
        for (int dy = lo[1]; dy <= hi[1]; ++dy)
            for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                int cx = (ca[0] + dx + cl->nc[0]) % cl->nc[0];
                int cy = (ca[1] + dy + cl->nc[1]) % cl->nc[1];
                int cz = (ca[2] + dz + cl->nc[2]) % cl->nc[2];
                int c = (cz * cl->nc[1] + cy) * cl->nc[0] + cx;
                for (int b = cl->head[c]; b >= 0; b = cl->next[b])
                    if (b != a && in_support(dim, x, a, b, box, H)) buf[cnt++] = b;
            }
    return cnt;
}

long long orc_neighbours_cells(int dim, int n, const double *x, const double *box, double H,
                               long long *ptr, int *idx, long long cap)
{
    cell_list cl;
    if (!build_cell_list(dim, n, x, box, H, &cl))
        return orc_neighbours_brute(dim, n, x, box, H, ptr, idx, cap);
    int *buf = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    long long k = 0;
    for (int a = 0; a < n; ++a) {
        ptr[a] = k;
        int cnt = cell_neighbours(&cl, x, box, H, a, buf);
        qsort(buf, (size_t)cnt, sizeof(int), cmp_int);
        if (k + cnt > cap) { k = -1; break; }
        memcpy(idx + k, buf, sizeof(int) * (size_t)cnt);
        k += cnt;
    }
    if (k >= 0) ptr[n] = k;
    free(buf);
    free_cell_list(&cl);
    return k;
}

/* ------------------------------------------------------------------------- */
/* Eq. 4 for every particle.  Per-particle D_a comes from v_a by Eq. 3.      */
/* x, v: [n][dim]; C, m, rho: [n].  The dispersive and convective sums are   */
/* returned separately (either output may be NULL).  Neighbours come from the */
/* cell list (or brute force when use_brute != 0 or the box has < 3 cells).  */
/* With sel != NULL only the nsel particles sel[0..nsel) are evaluated and   */
/* output k belongs to particle sel[k].                                      */
/* Returns the number of ordered in-support pairs of the evaluated particles. */
/* ------------------------------------------------------------------------- */
long long orc_rate_sel(int dim, int n, const double *x, const double *v, const double *C,
                       const double *m, const double *rho, const double *box, int kind, double H,
                       double gamma, double aL, double aT, double Dm, int use_brute, int nsel,
                       const int *sel, double *rate, double *rate_disp, double *rate_conv)
{
    if (!sel) nsel = n;
    double *D = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 9);
    for (int a = 0; a < n; ++a)
        orc_dispersion_tensor(dim, v + (size_t)a * dim, aL, aT, Dm, D + (size_t)a * 9);

    cell_list cl;
    int have_cells = !use_brute && build_cell_list(dim, n, x, box, H, &cl);
    long long npairs = 0;

#pragma omp parallel reduction(+ : npairs)
    {
        int *buf = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 256)
        for (int k_out = 0; k_out < nsel; ++k_out) {
            const int a = sel ? sel[k_out] : k_out;
            int cnt;
            if (have_cells) {
                cnt = cell_neighbours(&cl, x, box, H, a, buf);
                qsort(buf, (size_t)cnt, sizeof(int), cmp_int);
            } else {
                cnt = 0;
                for (int b = 0; b < n; ++b)
                    if (b != a && in_support(dim, x, a, b, box, H)) buf[cnt++] = b;
            }
            double sd = 0.0, sc = 0.0;
            for (int k = 0; k < cnt; ++k) {
                int b = buf[k];
                double xab[3], pd, pc;
                min_image(dim, x + (size_t)a * dim, x + (size_t)b * dim, box, xab);
                orc_pair_term(dim, xab, D + (size_t)a * 9, D + (size_t)b * 9, C[a], C[b],
                              v + (size_t)a * dim, v + (size_t)b * dim, m[b], rho[a], rho[b],
                              kind, H, gamma, &pd, &pc);
                sd += pd;
                sc += pc;
            }
            if (rate) rate[k_out] = sd + sc;
            if (rate_disp) rate_disp[k_out] = sd;
            if (rate_conv) rate_conv[k_out] = sc;
            npairs += cnt;
        }
        free(buf);
    }
    if (have_cells) free_cell_list(&cl);
    free(D);
    return npairs;
}

long long orc_rate(int dim, int n, const double *x, const double *v, const double *C,
                   const double *m, const double *rho, const double *box, int kind, double H,
                   double gamma, double aL, double aT, double Dm, int use_brute,
                   double *rate, double *rate_disp, double *rate_conv)
{
    return orc_rate_sel(dim, n, x, v, C, m, rho, box, kind, H, gamma, aL, aT, Dm, use_brute, n,
                        NULL, rate, rate_disp, rate_conv);
}

/* ------------------------------------------------------------------------- */
/* Eq. 8-9: one predictor-corrector step, in place on x and C.               */
/*   r^l       = R(x^l, C^l)                                                 */
/*   C^{l+1/2} = C^l + dt/2 r^l,   x^{l+1/2} = x^l + dt/2 v                  */
/*   r^{l+1/2} = R(x^{l+1/2}, C^{l+1/2})                                     */
/*   C^{l+1}   = C^l + dt r^{l+1/2}, x^{l+1} = x^l + dt v   (v constant)      */
/* Positions are wrapped into [0, box).                                      */
/* ------------------------------------------------------------------------- */
static double wrap(double u, double L)
{
    u -= L * floor(u / L);
    if (u >= L) u -= L;
    return u;
}

long long orc_step(int dim, int n, double *x, const double *v, double *C, const double *m,
                   const double *rho, const double *box, int kind, double H, double gamma,
                   double aL, double aT, double Dm, double dt, int use_brute)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(sizeof(double) * nn);
    double *Ch = (double *)malloc(sizeof(double) * nn);
    double *xh = (double *)malloc(sizeof(double) * nn * dim);
    long long pairs = orc_rate(dim, n, x, v, C, m, rho, box, kind, H, gamma, aL, aT, Dm,
                               use_brute, r, NULL, NULL);
    for (int a = 0; a < n; ++a) {
        Ch[a] = C[a] + 0.5 * dt * r[a];
        for (int i = 0; i < dim; ++i)
            xh[(size_t)a * dim + i] = wrap(x[(size_t)a * dim + i] + 0.5 * dt * v[(size_t)a * dim + i], box[i]);
    }
    pairs += orc_rate(dim, n, xh, v, Ch, m, rho, box, kind, H, gamma, aL, aT, Dm, use_brute, r,
                      NULL, NULL);
    for (int a = 0; a < n; ++a) {
        C[a] = C[a] + dt * r[a];
        for (int i = 0; i < dim; ++i)
            x[(size_t)a * dim + i] = wrap(x[(size_t)a * dim + i] + dt * v[(size_t)a * dim + i], box[i]);
    }
    free(r);
    free(Ch);
    free(xh);
    return pairs;
}

/* ------------------------------------------------------------------------- */
/* Eq. 14 (Sec. 5): Cattaneo's hyperbolic form                               */
/*   tau d2C/dt2 + dC/dt = R(C),  R = the right-hand side of Eq. 1 (Eq. 4).  */
/* Written as the first-order system dC/dt = Q, tau dQ/dt = R(C) - Q and     */
/* advanced by the midpoint rule of Eq. 8-9 applied to (C, Q):               */
/*   C^{l+1/2} = C^l + dt/2 Q^l,   Q^{l+1/2} = Q^l + dt/2 (R(C^l) - Q^l)/tau  */
/*   C^{l+1}   = C^l + dt Q^{l+1/2},                                        */
/*   Q^{l+1}   = Q^l + dt (R(C^{l+1/2}) - Q^{l+1/2})/tau                     */
/* with R evaluated at x^l and x^{l+1/2} as in orc_step.  In place on x, C,   */
/* Q.  Returns the in-support pairs of the two evaluations.                  */
/* ------------------------------------------------------------------------- */
long long orc_step_cattaneo(int dim, int n, double *x, const double *v, double *C, double *Q,
                            const double *m, const double *rho, const double *box, int kind,
                            double H, double gamma, double aL, double aT, double Dm, double dt,
                            double tau, int use_brute)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *r = (double *)malloc(sizeof(double) * nn);
    double *Ch = (double *)malloc(sizeof(double) * nn);
    double *Qh = (double *)malloc(sizeof(double) * nn);
    double *xh = (double *)malloc(sizeof(double) * nn * dim);
    long long pairs = orc_rate(dim, n, x, v, C, m, rho, box, kind, H, gamma, aL, aT, Dm,
                               use_brute, r, NULL, NULL);
    for (int a = 0; a < n; ++a) {
        Ch[a] = C[a] + 0.5 * dt * Q[a];
        Qh[a] = Q[a] + 0.5 * dt * (r[a] - Q[a]) / tau;
        for (int i = 0; i < dim; ++i)
            xh[(size_t)a * dim + i] = wrap(x[(size_t)a * dim + i] + 0.5 * dt * v[(size_t)a * dim + i], box[i]);
    }
    pairs += orc_rate(dim, n, xh, v, Ch, m, rho, box, kind, H, gamma, aL, aT, Dm, use_brute, r,
                      NULL, NULL);
    for (int a = 0; a < n; ++a) {
        C[a] = C[a] + dt * Qh[a];
        Q[a] = Q[a] + dt * (r[a] - Qh[a]) / tau;
        for (int i = 0; i < dim; ++i)
            x[(size_t)a * dim + i] = wrap(x[(size_t)a * dim + i] + dt * v[(size_t)a * dim + i], box[i]);
    }
    free(r);
    free(Ch);
    free(Qh);
    free(xh);
    return pairs;
}

/* ------------------------------------------------------------------------- */
/* Cell list on fixed-point positions (integer only, so the result is exact). */
/* A position u in [0, L) is stored as xq = round(u / L * 2^32) mod 2^32.     */
/* Cell index along an axis with nc cells: (xq * nc) >> 32.                  */
/* Linear key: (cz * ncy + cy) * ncx + cx.  xq is [dim][n] (one row per axis). */
/* ------------------------------------------------------------------------- */
void orc_cell_keys(int dim, int n, const uint32_t *xq, const int *nc, uint32_t *key)
{
    for (int a = 0; a < n; ++a) {
        uint32_t c[3] = {0, 0, 0};
        for (int i = 0; i < dim; ++i)
            c[i] = (uint32_t)(((uint64_t)xq[(size_t)i * n + a] * (uint64_t)nc[i]) >> 32);
        uint32_t ny = dim >= 2 ? (uint32_t)nc[1] : 1u;
        key[a] = (c[2] * ny + c[1]) * (uint32_t)nc[0] + c[0];
    }
}

/* Stable counting sort of particles by key (ties keep ascending index).
 * perm[k] = index of the particle at sorted position k.
 * cell_start[c] = number of particles with key < c, for c = 0..ncells
 * (so cell c holds sorted positions cell_start[c] .. cell_start[c+1]-1).     */
int orc_sort_cells(int n, const uint32_t *key, int ncells, uint32_t *perm, uint32_t *cell_start)
{
    for (int a = 0; a < n; ++a)
        if (key[a] >= (uint32_t)ncells) return -1;
    uint32_t *cnt = (uint32_t *)calloc((size_t)ncells + 1, sizeof(uint32_t));
    for (int a = 0; a < n; ++a) cnt[key[a]]++;
    uint32_t acc = 0;
    for (int c = 0; c < ncells; ++c) {
        cell_start[c] = acc;
        acc += cnt[c];
    }
    cell_start[ncells] = acc;
    for (int c = 0; c < ncells; ++c) cnt[c] = cell_start[c];
    for (int a = 0; a < n; ++a) perm[cnt[key[a]]++] = (uint32_t)a;
    free(cnt);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Closed form, Eq. 12-13 (2D) and its 3D counterpart, with periodic images. */
/* 2D, as printed with the denominator read as 2 C4^2:                        */
/*   C/C0 = w^2/C4 exp{[-X^2 A1 - Y^2 A2 + 4 X Y A3] / (8t^2 C2 + 4w^2 t C3 + 2w^4)} */
/*   A1 = 2tDyy + w^2, A2 = 2tDxx + w^2, A3 = tDxy, C2 = DxxDyy - Dxy^2,       */
/*   C3 = Dxx + Dyy, C4 = sqrt(4t^2 C2 + 2tw^2 C3 + w^4),                     */
/* with (X, Y) = x - x0 - v t.  3D: the same Gaussian written with            */
/*   S = w^2 I + 2 t D:  C/C0 = w^3/sqrt(det S) exp(-1/2 X^T S^{-1} X).       */
/* The plume centre x0 + v t is wrapped into the box and every image shift    */
/* n L with |n_i| <= nimg is summed.  x: [n][dim]; D: dim x dim row-major.    */
/* ------------------------------------------------------------------------- */
static double gauss2d_eq12(double X, double Y, const double *D, double w, double t)
{
    double Dxx = D[0], Dxy = D[1], Dyy = D[3];
    double w2 = w * w;
    double A1 = 2.0 * t * Dyy + w2;
    double A2 = 2.0 * t * Dxx + w2;
    double A3 = t * Dxy;
    double C2 = Dxx * Dyy - Dxy * Dxy;
    double C3 = Dxx + Dyy;
    double C4 = sqrt(4.0 * t * t * C2 + 2.0 * t * w2 * C3 + w2 * w2);
    double num = -X * X * A1 - Y * Y * A2 + 4.0 * X * Y * A3;
    double den = 8.0 * t * t * C2 + 4.0 * w2 * t * C3 + 2.0 * w2 * w2;
    return w2 / C4 * exp(num / den);
}

static double gauss3d(const double *X, const double *D, double w, double t)
{
    double S[9];
    for (int i = 0; i < 9; ++i) S[i] = 2.0 * t * D[i];
    for (int i = 0; i < 3; ++i) S[i * 4] += w * w;
    /* inverse by cofactors */
    double c00 = S[4] * S[8] - S[5] * S[7];
    double c01 = -(S[3] * S[8] - S[5] * S[6]);
    double c02 = S[3] * S[7] - S[4] * S[6];
    double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
    double inv[9];
    inv[0] = c00 / det;
    inv[1] = -(S[1] * S[8] - S[2] * S[7]) / det;
    inv[2] = (S[1] * S[5] - S[2] * S[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (S[0] * S[8] - S[2] * S[6]) / det;
    inv[5] = -(S[0] * S[5] - S[2] * S[3]) / det;
    inv[6] = c02 / det;
    inv[7] = -(S[0] * S[7] - S[1] * S[6]) / det;
    inv[8] = (S[0] * S[4] - S[1] * S[3]) / det;
    double quad = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) quad += X[i] * inv[i * 3 + j] * X[j];
    return w * w * w / sqrt(det) * exp(-0.5 * quad);
}

void orc_closed_form(int dim, int n, const double *x, const double *box, const double *x0,
                     const double *v, const double *D, double w, double C0, double t, int nimg,
                     double *C)
{
    double c[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) c[i] = wrap(x0[i] + v[i] * t, box[i]);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < n; ++a) {
        double X0[3] = {0, 0, 0};
        min_image(dim, x + (size_t)a * dim, c, box, X0);
        double s = 0.0;
        int lz = dim == 3 ? nimg : 0;
        for (int iz = -lz; iz <= lz; ++iz)
            for (int iy = -nimg; iy <= nimg; ++iy)
                for (int ix = -nimg; ix <= nimg; ++ix) {
                    double X[3] = {X0[0] + ix * box[0], X0[1] + iy * box[1],
                                   dim == 3 ? X0[2] + iz * box[2] : 0.0};
                    s += dim == 2 ? gauss2d_eq12(X[0], X[1], D, w, t) : gauss3d(X, D, w, t);
                }
        C[a] = C0 * s;
    }
}

/* ------------------------------------------------------------------------- */
/* Host threads used by the OpenMP loops (for timing on one core or all).    */
/* ------------------------------------------------------------------------- */
#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
