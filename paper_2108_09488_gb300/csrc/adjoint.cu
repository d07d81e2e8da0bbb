// adjoint.cu -- gradients of a concentration misfit with respect to the dispersivities, the molecular
// diffusion and the initial concentrations: the hand-written adjoint of the SPH step.
//
// The paper has no adjoint; this is derived from Eq. 3-5 and Eq. 8-9.  For a uniform velocity and
// uniform m / rho (the configured workloads):
//   * the rate is linear in C, r = L(theta) C, with (L u)_a = sum_b w_ab (u_a - u_b) and symmetric
//     weights w_ab = w_ba (the pair factor of Eq. 5 is even in x_ab), so L is symmetric;
//   * D of Eq. 3 is linear in theta = (alpha_L, alpha_T, D_m):  D = alpha_L B_L + alpha_T B_T + D_m I
//     with B_L = v v^T/|v| and B_T = |v| I - v v^T/|v|; for equal D_a = D_b the harmonic mean of
//     Eq. 5 is 2D, so L = alpha_L L_L + alpha_T L_T + D_m L_m with L_k the operator for D = B_k;
//   * the relative particle positions do not change (uniform drift), so L is the same at every
//     step and one predictor-corrector step (Eq. 8-9) is C^{l+1} = S C^l, S = I + dt L + dt^2 L^2 / 2.
// For J = 1/2 |C^N - C*|^2 and a fixed dt:
//   lambda^N = C^N - C*,  lambda^l = S^T lambda^{l+1} = S lambda^{l+1},  dJ/dC^0 = lambda^0,
//   dJ/dtheta_k = sum_l lambda^{l+1} . (dS/dtheta_k) C^l
//               = sum_l [ dt p.(L_k u) + dt^2/2 ( p.(L_k L u) + (L p).(L_k u) ) ],  u = C^l, p = lambda^{l+1}.
// Forward states are kept as checkpoints every `ckpt_every` steps and recomputed segment by segment
// on the way back.  All operators use one cell list built at the initial positions (the geometry
// is frozen, which is exact for a uniform drift), so forward and adjoint apply the same L.
// Pair arithmetic is FP32 with compensated row sums (as in rate.cu); dot products and J are FP64.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "ade_internal.h"

namespace {

constexpr int kT = 256;

// Up to three pair-factor sets (operators) and the weights of their combination.
struct ApplyCoef {
    float Kc[3][6];
    float c0[3];
    float theta[3];
};

__device__ __forceinline__ void nadd(float &sum, float &comp, float x)
{
    float t = sum + x;
    if (fabsf(sum) >= fabsf(x))
        comp += (sum - t) + x;
    else
        comp += (x - t) + sum;
    sum = t;
}

template <int KERNEL>
__device__ __forceinline__ float shape_f(float omq)
{
    if (KERNEL == ADE_WENDLAND_C2) return omq * omq * omq;
    float o2 = omq * omq;
    return o2 * o2 * omq * fmaf(-5.f, omq, 6.f);
}

template <int DIM>
__device__ __forceinline__ float dcal_k(float dx, float dy, float dz, float rinv2, const float *Kc, float c0)
{
    float Q;
    if (DIM == 2) {
        Q = dx * fmaf(Kc[0], dx, Kc[3] * dy);
    } else {
        float qx = fmaf(Kc[0], dx, fmaf(Kc[3], dy, Kc[4] * dz));
        float qy = fmaf(Kc[1], dy, Kc[5] * dz);
        Q = fmaf(dx, qx, dy * qy);
    }
    return fmaf(Q, rinv2, c0);
}

// out_k[i] = (L_k v)_i for sorted particle i, k < NOUT; with NOUT == 3 and comb != NULL also
// comb[i] = sum_k theta_k out_k[i]; with NOUT == 1 and axpy != NULL also axpy[i] = base[i] + alpha
// (L v)_i.  Same candidate walk and summation order as the rate kernel's direct variant.
template <int DIM, int KERNEL, int NOUT>
__global__ __launch_bounds__(kT) void k_apply(const uint4 *__restrict__ P, const uint32_t *__restrict__ cs,
                                              const float *__restrict__ v, const ade::RateParams prm,
                                              const ApplyCoef co, float *__restrict__ out0,
                                              float *__restrict__ out1, float *__restrict__ out2,
                                              float *__restrict__ comb, const float *__restrict__ base,
                                              float alpha, float *__restrict__ axpy)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= prm.n) return;
    const uint4 pa = __ldg(P + i);
    const float va = __ldg(v + i);
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz;
    const int cx = (int)__umulhi(pa.x, (uint32_t)ncx);
    const int cy = (int)__umulhi(pa.y, (uint32_t)ncy);
    const int cz = DIM == 3 ? (int)__umulhi(pa.z, (uint32_t)ncz) : 0;
    float acc[NOUT], cmp[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) acc[k] = cmp[k] = 0.f;
    for (int ri = 0; ri < prm.nrows; ++ri) {
        const ade::StencilRow row = prm.rows[ri];
        int yy = cy + row.dy;
        yy += (yy < 0) ? ncy : 0;
        yy -= (yy >= ncy) ? ncy : 0;
        int zz = 0;
        if (DIM == 3) {
            zz = cz + row.dz;
            zz += (zz < 0) ? ncz : 0;
            zz -= (zz >= ncz) ? ncz : 0;
        }
        const int basec = (zz * ncy + yy) * ncx;
        const int lo = cx - row.w, hi = cx + row.w + 1;
        int r0[2], r1[2];
        if (lo < 0) {
            r0[0] = __ldg(cs + basec + lo + ncx);
            r1[0] = __ldg(cs + basec + ncx);
            r0[1] = __ldg(cs + basec);
            r1[1] = __ldg(cs + basec + hi);
        } else if (hi > ncx) {
            r0[0] = __ldg(cs + basec + lo);
            r1[0] = __ldg(cs + basec + ncx);
            r0[1] = __ldg(cs + basec);
            r1[1] = __ldg(cs + basec + hi - ncx);
        } else {
            r0[0] = __ldg(cs + basec + lo);
            r1[0] = __ldg(cs + basec + hi);
            r0[1] = r1[1] = 0;
        }
        float rs[NOUT];
#pragma unroll
        for (int k = 0; k < NOUT; ++k) rs[k] = 0.f;
        for (int piece = 0; piece < 2; ++piece)
            for (int j = r0[piece]; j < r1[piece]; ++j) {
                const uint4 pb = __ldg(P + j);
                float dx = (float)(int)(pa.x - pb.x);
                float dy = (float)(int)(pa.y - pb.y) * prm.sy;
                float dz = DIM == 3 ? (float)(int)(pa.z - pb.z) * prm.sz : 0.f;
                float r2 = fmaf(dx, dx, dy * dy);
                if (DIM == 3) r2 = fmaf(dz, dz, r2);
                if (r2 < prm.H2 && r2 > 0.f) {
                    const float rinv = rsqrtf(r2);
                    const float f = shape_f<KERNEL>(fmaf(-(r2 * rinv), prm.invH, 1.f));
                    const float dv = va - __ldg(v + j);
                    const float ri2 = rinv * rinv;
#pragma unroll
                    for (int k = 0; k < NOUT; ++k)
                        rs[k] = fmaf(f * dcal_k<DIM>(dx, dy, dz, ri2, co.Kc[k], co.c0[k]), dv, rs[k]);
                }
            }
#pragma unroll
        for (int k = 0; k < NOUT; ++k) nadd(acc[k], cmp[k], rs[k]);
    }
    float r[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) r[k] = prm.pf * (acc[k] + cmp[k]);
    out0[i] = r[0];
    if (NOUT == 3) {
        out1[i] = r[1 % NOUT];
        out2[i] = r[2 % NOUT];
        if (comb) comb[i] = fmaf(co.theta[0], r[0], fmaf(co.theta[1], r[1 % NOUT], co.theta[2] * r[2 % NOUT]));
    } else if (axpy) {
        axpy[i] = fmaf(alpha, r[0], __ldg(base + i));
    }
}

__global__ void k_axpy(float *out, const float *x, float alpha, const float *y, int n)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n) out[i] = fmaf(alpha, y[i], x[i]);
}

__global__ void k_gather(float *out, const float *in, const uint32_t *perm, int n)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n) out[i] = in[perm[i]];
}

__global__ void k_scatter(float *out, const float *in, const uint32_t *perm, int n)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n) out[perm[i]] = in[i];
}

__global__ void k_sorted_C(float *out, const uint4 *P, int n)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i < n) out[i] = __uint_as_float(P[i].w);
}

// ND FP64 dot products x_d . y_d, d < ND; per-block partials, the last block folds them in a fixed
// order into out[0..ND) and resets the counter.
constexpr int kMaxDots = 9;
struct DotArgs {
    const float *x[kMaxDots];
    const float *y[kMaxDots];
};

template <int ND>
__global__ __launch_bounds__(kT) void k_dots(DotArgs a, int n, double *partials, unsigned *done,
                                             double *out)
{
    __shared__ double sh[ND][kT / 32];
    __shared__ bool last;
    const int i = blockIdx.x * kT + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        double v = i < n ? (double)a.x[d][i] * (double)a.y[d][i] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[d][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < ND) {
        double s = 0.0;
        for (int w = 0; w < kT / 32; ++w) s += sh[threadIdx.x][w];
        partials[(size_t)blockIdx.x * ND + threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < ND) {
            double s = 0.0;
            for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partials + (size_t)b * ND + threadIdx.x);
            out[threadIdx.x] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) *done = 0u;
    }
}

int blocks(int n) { return (n + kT - 1) / kT; }

// Adjoint workspace layout (floats in units of n, then doubles).
struct AdjLayout {
    size_t ckpt, seg, a, h, p, b, hp, lam, r3, la3, tgt, tmp, dots, partials, J, done, total;
    int nck;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

AdjLayout adj_layout(int n, int nsteps, int ck)
{
    AdjLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al256(bytes > 0 ? bytes : 1);
        return o;
    };
    const size_t fv = (size_t)n * 4;
    L.nck = (nsteps + ck - 1) / ck;
    L.ckpt = take(fv * (L.nck + 1));
    L.seg = take(fv * ck);
    L.a = take(fv);
    L.h = take(fv);
    L.p = take(fv);
    L.b = take(fv);
    L.hp = take(fv);
    L.lam = take(fv);
    L.r3 = take(fv * 3);
    L.la3 = take(fv * 3);
    L.tgt = take(fv);
    L.tmp = take(fv);
    L.dots = take((size_t)nsteps * kMaxDots * 8);
    L.partials = take((size_t)blocks(n) * kMaxDots * 8);
    L.J = take(64);
    L.done = take(64);
    L.total = off;
    return L;
}

#define ADJ_CK(call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            char m_[256];                                                                          \
            snprintf(m_, sizeof(m_), "%s: %s", #call, cudaGetErrorString(e_));                     \
            return ade::report_error(ADE_ERR_CUDA, m_);                                            \
        }                                                                                          \
    } while (0)

struct Adj {
    ade_ctx *c;
    cudaStream_t s;
    ApplyCoef op;     // the operator L(theta) in slot 0
    ApplyCoef basis;  // L_L, L_T, L_m in slots 0..2, theta as combination weights
    int n;
};

template <int DIM, int KERNEL>
cudaError_t apply_t(const Adj &A, const float *v, int multi, float *o0, float *o1, float *o2, float *comb,
                    const float *base, float alpha, float *axpy)
{
    const int nb = blocks(A.n);
    const ade::Work &w = A.c->w;
    if (multi)
        k_apply<DIM, KERNEL, 3><<<nb, kT, 0, A.s>>>(w.P0, w.cell_start, v, A.c->rp, A.basis, o0, o1, o2, comb,
                                                    nullptr, 0.f, nullptr);
    else
        k_apply<DIM, KERNEL, 1><<<nb, kT, 0, A.s>>>(w.P0, w.cell_start, v, A.c->rp, A.op, o0, nullptr, nullptr,
                                                    nullptr, base, alpha, axpy);
    return cudaGetLastError();
}

cudaError_t apply(const Adj &A, const float *v, int multi, float *o0, float *o1, float *o2, float *comb,
                  const float *base, float alpha, float *axpy)
{
    const int dim = A.c->dim, kern = A.c->p.kernel;
    if (dim == 2)
        return kern == ADE_WENDLAND_C2 ? apply_t<2, ADE_WENDLAND_C2>(A, v, multi, o0, o1, o2, comb, base, alpha, axpy)
                                       : apply_t<2, ADE_WENDLAND_C4>(A, v, multi, o0, o1, o2, comb, base, alpha, axpy);
    return kern == ADE_WENDLAND_C2 ? apply_t<3, ADE_WENDLAND_C2>(A, v, multi, o0, o1, o2, comb, base, alpha, axpy)
                                   : apply_t<3, ADE_WENDLAND_C4>(A, v, multi, o0, o1, o2, comb, base, alpha, axpy);
}

// One forward step C_out = S C_in: a = L u, h = u + dt/2 a, C_out = u + dt L h.
cudaError_t fwd_step(const Adj &A, const float *u, float *a, float *h, float *out, float dt)
{
    cudaError_t e = apply(A, u, 0, a, nullptr, nullptr, nullptr, u, 0.5f * dt, h);
    if (e != cudaSuccess) return e;
    return apply(A, h, 0, a, nullptr, nullptr, nullptr, u, dt, out);
}

}  // namespace

extern "C" int ade_adjoint_workspace_bytes(const ade_ctx *c, int nsteps, int ckpt_every, size_t *bytes)
{
    if (!c || !bytes || nsteps < 1 || ckpt_every < 1) return ade::report_error(ADE_ERR_ARG, "bad argument");
    *bytes = adj_layout(c->n, nsteps, ckpt_every).total;
    return ADE_OK;
}

extern "C" int ade_adjoint(ade_ctx *c, const float *C_target_dev, int nsteps, int ckpt_every, void *aws,
                           size_t aws_bytes, float *dJdC0_dev, double *dJdtheta_host, double *J_host,
                           float *C_final_dev, void *stream)
{
    ade::NvtxRange nvtx_("ade_adjoint");
    if (!c || !C_target_dev || nsteps < 1 || ckpt_every < 1 || !aws)
        return ade::report_error(ADE_ERR_ARG, "bad argument");
    if (c->field) return ade::report_error(ADE_ERR_STATE, "the adjoint is for a uniform velocity (vmax = 0)");
    if (c->catt) return ade::report_error(ADE_ERR_STATE, "the adjoint is for Eq. 1 (tau = 0)");
    const AdjLayout L = adj_layout(c->n, nsteps, ckpt_every);
    if (aws_bytes < L.total || ((uintptr_t)aws & 255u)) return ade::report_error(ADE_ERR_CAPACITY, "adjoint workspace too small or misaligned");
    const int n = c->n;
    if (n == 0) {
        if (dJdtheta_host) dJdtheta_host[0] = dJdtheta_host[1] = dJdtheta_host[2] = 0.0;
        if (J_host) *J_host = 0.0;
        return ADE_OK;
    }
    Adj A;
    A.c = c;
    A.s = (cudaStream_t)stream;
    A.n = n;
    memset(&A.op, 0, sizeof(A.op));
    memset(&A.basis, 0, sizeof(A.basis));
    const double gamma = c->p.gamma > 0.0 ? c->p.gamma : c->dim + 2.0;
    ade::pair_coeffs(c->dim, gamma, c->D, A.op.Kc[0], &A.op.c0[0]);
    const double theta[3] = {c->p.alpha_L, c->p.alpha_T, c->p.D_m};
    double vabs2 = 0.0;
    for (int i = 0; i < c->dim; ++i) vabs2 += c->p.v[i] * c->p.v[i];
    const double vabs = sqrt(vabs2);
    for (int k = 0; k < 3; ++k) {
        // B_L = v v^T / |v|, B_T = |v| I - v v^T / |v|, B_m = I (the theta-derivatives of Eq. 3)
        double B[9] = {0};
        for (int i = 0; i < c->dim; ++i)
            for (int j = 0; j < c->dim; ++j) {
                const double vv = vabs > 0.0 ? c->p.v[i] * c->p.v[j] / vabs : 0.0;
                const double I = i == j ? 1.0 : 0.0;
                B[i * c->dim + j] = k == 0 ? vv : (k == 1 ? vabs * I - vv : I);
            }
        ade::pair_coeffs(c->dim, gamma, B, A.basis.Kc[k], &A.basis.c0[k]);
        A.basis.theta[k] = (float)theta[k];
    }
    char *base = static_cast<char *>(aws);
    float *ckpt = reinterpret_cast<float *>(base + L.ckpt);
    float *seg = reinterpret_cast<float *>(base + L.seg);
    float *a = reinterpret_cast<float *>(base + L.a);
    float *h = reinterpret_cast<float *>(base + L.h);
    float *p = reinterpret_cast<float *>(base + L.p);
    float *bb = reinterpret_cast<float *>(base + L.b);
    float *hp = reinterpret_cast<float *>(base + L.hp);
    float *lam = reinterpret_cast<float *>(base + L.lam);
    float *r3 = reinterpret_cast<float *>(base + L.r3);
    float *la3 = reinterpret_cast<float *>(base + L.la3);
    float *tgt = reinterpret_cast<float *>(base + L.tgt);
    float *tmp = reinterpret_cast<float *>(base + L.tmp);
    double *dots = reinterpret_cast<double *>(base + L.dots);
    double *partials = reinterpret_cast<double *>(base + L.partials);
    double *Jd = reinterpret_cast<double *>(base + L.J);
    unsigned *done = reinterpret_cast<unsigned *>(base + L.done);
    const float dt = (float)c->dt;
    const int nb = blocks(n);
    cudaStream_t s = A.s;

    // frozen geometry: one cell list at the current positions (counts and tile totals cleared first)
    cudaError_t e = ade::launch_build_cells(c->dim, c->xq, c->C, n, c->nc, c->ncells, c->w, s);
    if (e != cudaSuccess) return ade::report_error(ADE_ERR_CUDA, cudaGetErrorString(e));
    ADJ_CK(cudaMemsetAsync(done, 0, sizeof(unsigned), s));
    k_sorted_C<<<nb, kT, 0, s>>>(ckpt, c->w.P0, n);
    k_gather<<<nb, kT, 0, s>>>(tgt, C_target_dev, c->w.perm, n);
    // forward with checkpoints every ckpt_every steps
    for (int l = 0; l < nsteps; ++l) {
        const float *u = (l % ckpt_every == 0) ? ckpt + (size_t)(l / ckpt_every) * n : tmp;
        float *out = ((l + 1) % ckpt_every == 0 || l + 1 == nsteps) ? ckpt + (size_t)((l + ckpt_every) / ckpt_every) * n : tmp;
        if (u == tmp && out == tmp) {
            ADJ_CK(fwd_step(A, tmp, a, h, lam, dt));
            ADJ_CK(cudaMemcpyAsync(tmp, lam, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        } else {
            ADJ_CK(fwd_step(A, u, a, h, out, dt));
        }
    }
    // C^N sits in checkpoint slot nck (the last step always writes a slot)
    const float *CN = ckpt + (size_t)L.nck * n;
    if (C_final_dev) k_scatter<<<nb, kT, 0, s>>>(C_final_dev, CN, c->w.perm, n);
    // lambda^N = C^N - C*, J = 1/2 |lambda^N|^2
    k_axpy<<<nb, kT, 0, s>>>(p, CN, -1.0f, tgt, n);
    {
        DotArgs da;
        memset(&da, 0, sizeof(da));
        da.x[0] = p;
        da.y[0] = p;
        k_dots<1><<<nb, kT, 0, s>>>(da, n, partials, done, Jd);
        ADJ_CK(cudaGetLastError());
    }
    // backward, segment by segment
    float *r[3] = {r3, r3 + n, r3 + 2 * (size_t)n};
    float *la[3] = {la3, la3 + n, la3 + 2 * (size_t)n};
    for (int sgi = L.nck - 1; sgi >= 0; --sgi) {
        const int l0 = sgi * ckpt_every;
        const int l1 = l0 + ckpt_every < nsteps ? l0 + ckpt_every : nsteps;
        ADJ_CK(cudaMemcpyAsync(seg, ckpt + (size_t)sgi * n, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        for (int l = l0; l + 1 < l1; ++l)
            ADJ_CK(fwd_step(A, seg + (size_t)(l - l0) * n, a, h, seg + (size_t)(l + 1 - l0) * n, dt));
        for (int l = l1 - 1; l >= l0; --l) {
            const float *u = seg + (size_t)(l - l0) * n;
            // r_k = L_k u and a = L u;  la_k = L_k a
            ADJ_CK(apply(A, u, 1, r[0], r[1], r[2], a, nullptr, 0.f, nullptr));
            ADJ_CK(apply(A, a, 1, la[0], la[1], la[2], nullptr, nullptr, 0.f, nullptr));
            // b = L p, hp = p + dt/2 b
            ADJ_CK(apply(A, p, 0, bb, nullptr, nullptr, nullptr, p, 0.5f * dt, hp));
            DotArgs da;
            for (int k = 0; k < 3; ++k) {
                da.x[k] = p;
                da.y[k] = r[k];
                da.x[3 + k] = p;
                da.y[3 + k] = la[k];
                da.x[6 + k] = bb;
                da.y[6 + k] = r[k];
            }
            k_dots<9><<<nb, kT, 0, s>>>(da, n, partials, done, dots + (size_t)l * kMaxDots);
            ADJ_CK(cudaGetLastError());
            // lambda^l = p + dt L hp
            ADJ_CK(apply(A, hp, 0, bb, nullptr, nullptr, nullptr, p, dt, lam));
            ADJ_CK(cudaMemcpyAsync(p, lam, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        }
    }
    if (dJdC0_dev) k_scatter<<<nb, kT, 0, s>>>(dJdC0_dev, p, c->w.perm, n);
    ADJ_CK(cudaGetLastError());
    std::vector<double> hd((size_t)nsteps * kMaxDots);
    double Jh = 0.0;
    ADJ_CK(cudaMemcpyAsync(hd.data(), dots, hd.size() * 8, cudaMemcpyDeviceToHost, s));
    ADJ_CK(cudaMemcpyAsync(&Jh, Jd, 8, cudaMemcpyDeviceToHost, s));
    ADJ_CK(cudaStreamSynchronize(s));
    if (J_host) *J_host = 0.5 * Jh;
    if (dJdtheta_host) {
        const double dtd = (double)dt;
        for (int k = 0; k < 3; ++k) {
            double g = 0.0;
            for (int l = 0; l < nsteps; ++l) {
                const double *d = hd.data() + (size_t)l * kMaxDots;
                g += dtd * d[k] + 0.5 * dtd * dtd * (d[3 + k] + d[6 + k]);
            }
            dJdtheta_host[k] = g;
        }
    }
    return ADE_OK;
}
