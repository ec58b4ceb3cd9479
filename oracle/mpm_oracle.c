/*
 * mpm_oracle.c -- plain FP64 CPU reference for the batched differentiable MPM path.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's CPU
 * baseline; never by the product library.  Single-threaded, one environment at a
 * time, dense grid, particles in input order, no blocking or fusion.
 *
 * Paper: arXiv 2412.12089 ("Stabilizing RL in Differentiable Multiphysics
 * Simulation").  The MLS-MPM transfer scheme follows the published MLS-MPM method
 * the paper builds on (App. D.3: "CPIC steps 2--4"): quadratic B-spline weights,
 * D^-1 = 4/dx^2, affine momentum A = m C - dt V (4/dx^2) tau.  Constitutive laws are
 * App. D.3's von Mises elastoplastic and weakly-compressible fluid models; the
 * softened contact is App. D.3's s = min(exp(-alpha d), 1) with a linear blend of
 * pre- and post-projection grid velocity.  The reverse pass is the exact discrete
 * adjoint (Sec. 4.1) with per-control-step checkpoints and forward recomputation.
 */
#include "mpm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ 3x3 algebra */

static void m3_zero(double* A) { memset(A, 0, 9 * sizeof(double)); }
static void m3_eye(double* A) { m3_zero(A); A[0] = A[4] = A[8] = 1.0; }

static void m3_mul(const double* A, const double* B, double* O) /* O = A B */
{
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = acc;
        }
    memcpy(O, T, sizeof T);
}

static void m3_mul_bt(const double* A, const double* B, double* O) /* O = A B^T */
{
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += A[3 * i + k] * B[3 * j + k];
            T[3 * i + j] = acc;
        }
    memcpy(O, T, sizeof T);
}

static void m3_mul_at(const double* A, const double* B, double* O) /* O = A^T B */
{
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += A[3 * k + i] * B[3 * k + j];
            T[3 * i + j] = acc;
        }
    memcpy(O, T, sizeof T);
}

static double m3_det(const double* A)
{
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* O = A^{-T} (cofactor matrix / det). */
static void m3_inv_t(const double* A, double* O)
{
    double cof[9];
    cof[0] = A[4] * A[8] - A[5] * A[7];
    cof[1] = -(A[3] * A[8] - A[5] * A[6]);
    cof[2] = A[3] * A[7] - A[4] * A[6];
    cof[3] = -(A[1] * A[8] - A[2] * A[7]);
    cof[4] = A[0] * A[8] - A[2] * A[6];
    cof[5] = -(A[0] * A[7] - A[1] * A[6]);
    cof[6] = A[1] * A[5] - A[2] * A[4];
    cof[7] = -(A[0] * A[5] - A[2] * A[3]);
    cof[8] = A[0] * A[4] - A[1] * A[3];
    double det = A[0] * cof[0] + A[1] * cof[1] + A[2] * cof[2];
    for (int i = 0; i < 9; i++) O[i] = cof[i] / det;
}

static double v3_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------ SVD */

/*
 * F = U diag(sig) V^T by one-sided (Hestenes) Jacobi on the columns of B = F V,
 * iterated to convergence.  Convention: det U = det V = +1, |sig| sorted in
 * descending order, a reflection carried by the sign of sig[2].
 */
void orc_svd3(const double* F, double* U, double* sig, double* V)
{
    double B[9];
    memcpy(B, F, sizeof B);
    m3_eye(V);
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int r = 0; r < 3; r++) {
            int p = P[r][0], q = P[r][1];
            double a = 0, b = 0, g = 0;
            for (int k = 0; k < 3; k++) {
                a += B[3 * k + p] * B[3 * k + p];
                b += B[3 * k + q] * B[3 * k + q];
                g += B[3 * k + p] * B[3 * k + q];
            }
            if (g == 0.0 || fabs(g) <= 1e-300) continue;
            double rel = fabs(g) / sqrt(a * b);
            if (rel > off) off = rel;
            if (rel < 1e-17) continue;
            double zeta = (b - a) / (2.0 * g);
            double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
            for (int k = 0; k < 3; k++) {
                double bp = B[3 * k + p], bq = B[3 * k + q];
                B[3 * k + p] = c * bp - s * bq;
                B[3 * k + q] = s * bp + c * bq;
                double vp = V[3 * k + p], vq = V[3 * k + q];
                V[3 * k + p] = c * vp - s * vq;
                V[3 * k + q] = s * vp + c * vq;
            }
        }
        if (off < 1e-15) break;
    }
    double nrm[3];
    for (int j = 0; j < 3; j++)
        nrm[j] = sqrt(B[j] * B[j] + B[3 + j] * B[3 + j] + B[6 + j] * B[6 + j]);
    /* sort columns by descending norm (a column swap negates det V; fixed below) */
    int idx[3] = {0, 1, 2};
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++)
            if (nrm[idx[j]] > nrm[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    double Bs[9], Vs[9];
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) {
            Bs[3 * k + j] = B[3 * k + idx[j]];
            Vs[3 * k + j] = V[3 * k + idx[j]];
        }
    double ns[3] = {nrm[idx[0]], nrm[idx[1]], nrm[idx[2]]};
    if (m3_det(Vs) < 0) {
        for (int k = 0; k < 3; k++) { Vs[3 * k + 2] = -Vs[3 * k + 2]; Bs[3 * k + 2] = -Bs[3 * k + 2]; }
    }
    /* U columns: normalised B columns; complete an orthonormal frame if degenerate */
    double scale = ns[0] > 0 ? ns[0] : 1.0;
    double u0[3], u1[3], u2[3];
    if (ns[0] > 1e-300) {
        for (int k = 0; k < 3; k++) u0[k] = Bs[3 * k] / ns[0];
    } else {
        u0[0] = 1; u0[1] = 0; u0[2] = 0;
    }
    if (ns[1] > 1e-13 * scale) {
        for (int k = 0; k < 3; k++) u1[k] = Bs[3 * k + 1] / ns[1];
    } else {
        /* any unit vector orthogonal to u0 */
        double e[3] = {0, 0, 0};
        int m = fabs(u0[0]) < 0.6 ? 0 : (fabs(u0[1]) < 0.6 ? 1 : 2);
        e[m] = 1.0;
        double d = v3_dot(e, u0);
        for (int k = 0; k < 3; k++) u1[k] = e[k] - d * u0[k];
        double l = sqrt(v3_dot(u1, u1));
        for (int k = 0; k < 3; k++) u1[k] /= l;
    }
    /* u2: from B when well-conditioned, else the cross product; sign gives det U = +1 */
    double cr[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2],
                    u0[0] * u1[1] - u0[1] * u1[0]};
    double s2;
    if (ns[2] > 1e-13 * scale) {
        double b2[3] = {Bs[2], Bs[5], Bs[8]};
        s2 = v3_dot(b2, cr); /* = +-ns[2] up to rounding: sign carries det F */
        s2 = (s2 >= 0 ? ns[2] : -ns[2]);
    } else {
        double b2[3] = {Bs[2], Bs[5], Bs[8]};
        s2 = v3_dot(b2, cr);
    }
    for (int k = 0; k < 3; k++) u2[k] = cr[k];
    for (int k = 0; k < 3; k++) {
        U[3 * k + 0] = u0[k];
        U[3 * k + 1] = u1[k];
        U[3 * k + 2] = u2[k];
    }
    memcpy(V, Vs, sizeof Vs);
    sig[0] = ns[0];
    sig[1] = ns[1];
    sig[2] = s2;
}

/* ------------------------------------------------------------------ materials */

#define SIG_MIN 1e-4 /* singular values are clamped here before the log (Hencky strain) */

/* Hencky strain eps_i = log(max(sig_i, SIG_MIN)). */
static double hencky_eps(double s) { return log(s > SIG_MIN ? s : SIG_MIN); }

/*
 * Kirchhoff stress tau = P F^T.
 *  NEOHOOKEAN: tau = mu (F F^T - I) + lam log(J) I.
 *  MUSCLE    : neo-Hookean + a_g * act_stress * (F e_z)(F e_z)^T.
 *  VONMISES  : App. D.3 elastic law read as Kirchhoff stress,
 *              tau = U (2 mu eps + lam tr(eps) I) U^T,  eps = log Sigma.
 *  FLUID     : App. D.3 P = lam J (J - 1) F^{-T} with lam := bulk modulus, so
 *              tau = bulk J (J - 1) I, plus a Newtonian term visc J (C + C^T).
 */
void orc_tau(const orc_spec* s, const double* F, const double* C, double a_g, double* tau)
{
    switch (s->material) {
    case ORC_NEOHOOKEAN:
    case ORC_MUSCLE: {
        m3_mul_bt(F, F, tau);
        double J = m3_det(F);
        double lj = s->lam * log(J);
        for (int i = 0; i < 9; i++) tau[i] *= s->mu;
        for (int i = 0; i < 3; i++) tau[4 * i] += -s->mu + lj;
        if (s->material == ORC_MUSCLE && a_g != 0.0) {
            double f[3] = {F[2], F[5], F[8]};
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) tau[3 * i + j] += a_g * s->act_stress * f[i] * f[j];
        }
        break;
    }
    case ORC_VONMISES: {
        double U[9], sg[3], V[9];
        orc_svd3(F, U, sg, V);
        double e[3] = {hencky_eps(sg[0]), hencky_eps(sg[1]), hencky_eps(sg[2])};
        double tr = e[0] + e[1] + e[2];
        double t[3];
        for (int i = 0; i < 3; i++) t[i] = 2.0 * s->mu * e[i] + s->lam * tr;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += U[3 * i + k] * t[k] * U[3 * j + k];
                tau[3 * i + j] = acc;
            }
        break;
    }
    case ORC_FLUID: {
        double J = m3_det(F);
        double p = s->bulk * J * (J - 1.0);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                tau[3 * i + j] = (i == j ? p : 0.0) + s->visc * J * (C[3 * i + j] + C[3 * j + i]);
        break;
    }
    default:
        m3_zero(tau);
    }
}

/*
 * Adjoint of rotated-frame isotropic maps.  For G(F) = U diag(g(sig)) V^T the
 * derivative in the rotated frame dF^ = U^T dF V is: diagonal dG^_ii = sum_k
 * dg_i/dsig_k dF^_kk; each off-diagonal pair (i,j) mixes (dF^_ij, dF^_ji) with
 * A = (g_i - g_j)/(sig_i - sig_j) on the symmetric part and
 * B = (g_i + g_j)/(sig_i + sig_j) on the antisymmetric part.  A takes its limit
 * dg_i/dsig_i - dg_i/dsig_j when sig_i ~ sig_j (always the case at F = I).
 */
static void iso_vjp(const double* U, const double* sg, const double* V, const double* g,
                    const double Jg[3][3], const double* Gb, double* Fb_acc)
{
    double M[9], T[9], K[9];
    m3_mul_at(U, Gb, T);
    m3_mul(T, V, M); /* M = U^T Gb V */
    m3_zero(K);
    for (int k = 0; k < 3; k++) {
        double acc = 0;
        for (int i = 0; i < 3; i++) acc += Jg[i][k] * M[4 * i];
        K[4 * k] = acc;
    }
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; r++) {
        int i = P[r][0], j = P[r][1];
        double ds = sg[i] - sg[j];
        double A;
        if (fabs(ds) < 1e-6 * fmax(1.0, fabs(sg[i])))
            A = Jg[i][i] - Jg[i][j];
        else
            A = (g[i] - g[j]) / ds;
        double ss = sg[i] + sg[j];
        if (fabs(ss) < 1e-12) ss = (ss >= 0 ? 1e-12 : -1e-12);
        double B = (g[i] + g[j]) / ss;
        double sym = 0.5 * (M[3 * i + j] + M[3 * j + i]);
        double asy = 0.5 * (M[3 * i + j] - M[3 * j + i]);
        K[3 * i + j] = A * sym + B * asy;
        K[3 * j + i] = A * sym - B * asy;
    }
    double UK[9], R[9];
    m3_mul(U, K, UK);
    m3_mul_bt(UK, V, R); /* U K V^T */
    for (int i = 0; i < 9; i++) Fb_acc[i] += R[i];
}

/*
 * Adjoint of the Hencky stress tau = U diag(t(sig)) U^T.  With x = omega_U,ij
 * solved from dF^ (x (sig_j^2 - sig_i^2) = sig_j dF^_ij + sig_i dF^_ji), the
 * off-diagonal rotated stress is dtau^_ij = Q_ij (sig_j dF^_ij + sig_i dF^_ji) with
 * Q_ij = (t_j - t_i)/(sig_j^2 - sig_i^2), whose limit at sig_i = sig_j is mu/sig^2.
 */
static void hencky_tau_vjp(const orc_spec* s, const double* F, const double* taub, double* Fb)
{
    double U[9], sg[3], V[9];
    orc_svd3(F, U, sg, V);
    double e[3], t[3];
    for (int i = 0; i < 3; i++) e[i] = hencky_eps(sg[i]);
    double tr = e[0] + e[1] + e[2];
    for (int i = 0; i < 3; i++) t[i] = 2.0 * s->mu * e[i] + s->lam * tr;
    double M[9], T[9], K[9];
    m3_mul_at(U, taub, T);
    m3_mul(T, U, M); /* M = U^T taub U */
    m3_zero(K);
    for (int k = 0; k < 3; k++) {
        double de = sg[k] > SIG_MIN ? 1.0 / sg[k] : 0.0; /* d eps_k / d sig_k */
        double acc = 0;
        for (int i = 0; i < 3; i++) acc += M[4 * i] * ((i == k ? 2.0 * s->mu : 0.0) + s->lam) * de;
        K[4 * k] = acc;
    }
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; r++) {
        int i = P[r][0], j = P[r][1];
        double Q;
        double dsq = sg[j] * sg[j] - sg[i] * sg[i];
        if (fabs(sg[j] - sg[i]) < 1e-6 * fmax(1.0, fabs(sg[i]))) {
            double sm = 0.5 * (fabs(sg[i]) + fabs(sg[j]));
            if (sm < SIG_MIN) sm = SIG_MIN;
            Q = s->mu / (sm * sm);
        } else if (fabs(dsq) < 1e-300) {
            Q = 0.0;
        } else {
            Q = (t[j] - t[i]) / dsq;
        }
        double sym = M[3 * i + j] + M[3 * j + i];
        K[3 * i + j] += Q * sg[j] * sym;
        K[3 * j + i] += Q * sg[i] * sym;
    }
    double UK[9], R[9];
    m3_mul(U, K, UK);
    m3_mul_bt(UK, V, R);
    for (int i = 0; i < 9; i++) Fb[i] += R[i];
}

void orc_tau_vjp(const orc_spec* s, const double* F, const double* C, double a_g,
                 const double* taub, double* Fb, double* Cb, double* agb)
{
    switch (s->material) {
    case ORC_NEOHOOKEAN:
    case ORC_MUSCLE: {
        /* Fb += mu (taub + taub^T) F + lam tr(taub) F^{-T} */
        double Ts[9], R[9], Fit[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) Ts[3 * i + j] = taub[3 * i + j] + taub[3 * j + i];
        m3_mul(Ts, F, R);
        m3_inv_t(F, Fit);
        double tr = taub[0] + taub[4] + taub[8];
        for (int i = 0; i < 9; i++) Fb[i] += s->mu * R[i] + s->lam * tr * Fit[i];
        if (s->material == ORC_MUSCLE && a_g != 0.0) {
            double f[3] = {F[2], F[5], F[8]};
            double fb[3] = {0, 0, 0};
            double quad = 0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    fb[i] += a_g * s->act_stress * Ts[3 * i + j] * f[j];
                    quad += f[i] * taub[3 * i + j] * f[j];
                }
            for (int i = 0; i < 3; i++) Fb[3 * i + 2] += fb[i];
            if (agb) *agb += s->act_stress * quad;
        } else if (s->material == ORC_MUSCLE && agb) {
            double f[3] = {F[2], F[5], F[8]};
            double quad = 0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) quad += f[i] * taub[3 * i + j] * f[j];
            *agb += s->act_stress * quad;
        }
        break;
    }
    case ORC_VONMISES:
        hencky_tau_vjp(s, F, taub, Fb);
        break;
    case ORC_FLUID: {
        double J = m3_det(F);
        double tr = taub[0] + taub[4] + taub[8];
        double cc = 0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) cc += taub[3 * i + j] * (C[3 * i + j] + C[3 * j + i]);
        double Jb = s->bulk * (2.0 * J - 1.0) * tr + s->visc * cc;
        double Fit[9];
        m3_inv_t(F, Fit);
        for (int i = 0; i < 9; i++) Fb[i] += Jb * J * Fit[i];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) Cb[3 * i + j] += s->visc * J * (taub[3 * i + j] + taub[3 * j + i]);
        break;
    }
    default:
        break;
    }
}

/*
 * Plastic projection (applied in G2P after the F update).
 *  VONMISES: App. D.3 return mapping: eps^ = eps - tr(eps)/3, dgam = |eps^| - c_y sig_y/(2 mu);
 *            if dgam > 0, F <- U exp(eps - dgam eps^/|eps^|) V^T.
 *  FLUID   : F <- J^{1/3} I.
 *  others  : identity.
 */
void orc_project(const orc_spec* s, const double* Ft, double* Fo)
{
    if (s->material == ORC_VONMISES) {
        double U[9], sg[3], V[9];
        orc_svd3(Ft, U, sg, V);
        double e[3];
        for (int i = 0; i < 3; i++) e[i] = hencky_eps(sg[i]);
        double tr3 = (e[0] + e[1] + e[2]) / 3.0;
        double eh[3] = {e[0] - tr3, e[1] - tr3, e[2] - tr3};
        double nh = sqrt(v3_dot(eh, eh));
        double dg = nh - s->c_y * s->yield_stress / (2.0 * s->mu);
        if (dg <= 0.0) {
            memcpy(Fo, Ft, 9 * sizeof(double));
            return;
        }
        double g[3];
        for (int i = 0; i < 3; i++) g[i] = exp(e[i] - dg * eh[i] / nh);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += U[3 * i + k] * g[k] * V[3 * j + k];
                Fo[3 * i + j] = acc;
            }
    } else if (s->material == ORC_FLUID) {
        double J = m3_det(Ft);
        double c = cbrt(J);
        m3_zero(Fo);
        Fo[0] = Fo[4] = Fo[8] = c;
    } else {
        memcpy(Fo, Ft, 9 * sizeof(double));
    }
}

void orc_project_vjp(const orc_spec* s, const double* Ft, const double* Fob, double* Ftb)
{
    if (s->material == ORC_VONMISES) {
        double U[9], sg[3], V[9];
        orc_svd3(Ft, U, sg, V);
        double e[3];
        for (int i = 0; i < 3; i++) e[i] = hencky_eps(sg[i]);
        double tr3 = (e[0] + e[1] + e[2]) / 3.0;
        double eh[3] = {e[0] - tr3, e[1] - tr3, e[2] - tr3};
        double nh = sqrt(v3_dot(eh, eh));
        double cyl = s->c_y * s->yield_stress / (2.0 * s->mu);
        double dg = nh - cyl;
        if (dg <= 0.0) {
            memcpy(Ftb, Fob, 9 * sizeof(double));
            return;
        }
        /* new log-strain: e_new = tr(e)/3 + cyl * n, n = eh/|eh|; g = exp(e_new) */
        double nv[3] = {eh[0] / nh, eh[1] / nh, eh[2] / nh};
        double g[3];
        for (int i = 0; i < 3; i++) g[i] = exp(tr3 + cyl * nv[i]);
        /* dg_i/dsig_k = g_i (1/3 + cyl (delta_ik - n_i n_k - 1/3)/|eh|) deps_k/dsig_k */
        double Jg[3][3];
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
                double de = sg[k] > SIG_MIN ? 1.0 / sg[k] : 0.0;
                double dn = ((i == k ? 1.0 : 0.0) - nv[i] * nv[k] - 1.0 / 3.0) / nh;
                Jg[i][k] = g[i] * (1.0 / 3.0 + cyl * dn) * de;
            }
        memset(Ftb, 0, 9 * sizeof(double));
        iso_vjp(U, sg, V, g, Jg, Fob, Ftb);
    } else if (s->material == ORC_FLUID) {
        double J = m3_det(Ft);
        double tr = Fob[0] + Fob[4] + Fob[8];
        double Fit[9];
        m3_inv_t(Ft, Fit);
        double c = tr * cbrt(J) / 3.0; /* d(J^{1/3})/dJ * J = J^{1/3}/3 */
        for (int i = 0; i < 9; i++) Ftb[i] = c * Fit[i];
    } else {
        memcpy(Ftb, Fob, 9 * sizeof(double));
    }
}

/* ------------------------------------------------------------------ colliders */

/* Box SDF in its own frame: distance d, gradient n, Hessian H. */
static void sdf_box(const double* p, const double* h, double* d, double* n, double* H)
{
    double q[3], sgn[3];
    for (int k = 0; k < 3; k++) {
        sgn[k] = p[k] >= 0 ? 1.0 : -1.0;
        q[k] = fabs(p[k]) - h[k];
    }
    m3_zero(H);
    if (q[0] > 0 || q[1] > 0 || q[2] > 0) {
        double m[3];
        for (int k = 0; k < 3; k++) m[k] = q[k] > 0 ? q[k] : 0.0;
        double l = sqrt(v3_dot(m, m));
        *d = l;
        for (int k = 0; k < 3; k++) n[k] = sgn[k] * m[k] / l;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                H[3 * i + j] = ((i == j && q[i] > 0) ? 1.0 : 0.0) / l - n[i] * n[j] / l;
    } else {
        int ks = 0;
        for (int k = 1; k < 3; k++)
            if (q[k] > q[ks]) ks = k;
        *d = q[ks];
        n[0] = n[1] = n[2] = 0;
        n[ks] = sgn[ks];
    }
}

/* Capsule along the body x axis: radius dims[0], half-length dims[1]. */
static void sdf_capsule(const double* p, const double* dims, double* d, double* n, double* H)
{
    double R = dims[0], hl = dims[1];
    double cx = p[0] < -hl ? -hl : (p[0] > hl ? hl : p[0]);
    double e[3] = {p[0] - cx, p[1], p[2]};
    double l = sqrt(v3_dot(e, e));
    m3_zero(H);
    if (l < 1e-12) {
        *d = -R;
        n[0] = 0; n[1] = 0; n[2] = 1;
        return;
    }
    *d = l - R;
    for (int k = 0; k < 3; k++) n[k] = e[k] / l;
    double px = (fabs(p[0]) < hl) ? 0.0 : 1.0; /* projector P = diag(px, 1, 1) */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double Pij = (i == j) ? (i == 0 ? px : 1.0) : 0.0;
            H[3 * i + j] = (Pij - n[i] * n[j]) / l;
        }
}

/* Open-top container: inner cavity [-a,a]^2 x [-az, inf), wall thickness w, as the union
 * of five boxes.  The walls reach down through the floor and overlap each other at the
 * vertical edges, so the solid has no internal faces (on a shared face two boxes would
 * report the same zero distance with opposite normals). */
static void sdf_container(const double* p, const double* dims, double* d, double* n, double* H)
{
    double a = dims[0], w = dims[1], az = dims[2];
    double zc = -0.5 * w, hz = az + 0.5 * w; /* walls span z in [-az - w, az] */
    double cen[5][3] = {{0, 0, -az - 0.5 * w},
                        {a + 0.5 * w, 0, zc},
                        {-(a + 0.5 * w), 0, zc},
                        {0, a + 0.5 * w, zc},
                        {0, -(a + 0.5 * w), zc}};
    double hal[5][3] = {{a + w, a + w, 0.5 * w},
                        {0.5 * w, a + w, hz},
                        {0.5 * w, a + w, hz},
                        {a + w, 0.5 * w, hz},
                        {a + w, 0.5 * w, hz}};
    double best = INFINITY;
    for (int k = 0; k < 5; k++) {
        double pl[3] = {p[0] - cen[k][0], p[1] - cen[k][1], p[2] - cen[k][2]};
        double dk, nk[3], Hk[9];
        sdf_box(pl, hal[k], &dk, nk, Hk);
        if (dk < best) {
            best = dk;
            memcpy(n, nk, sizeof nk);
            memcpy(H, Hk, sizeof Hk);
        }
    }
    *d = best;
}

/*
 * Collider at world point xw for pose q = (c, theta) and pose velocity u = (v_c, omega):
 * signed distance d (> 0 outside), outward normal n = grad d, Hessian H (world frame),
 * and the rigid body's velocity vb at xw.
 */
/* One rigid body of shape `kind` at pose q (4 entries), pose velocity u. */
static void collider_body(const orc_spec* s, int kind, const double* xw, const double* q, const double* u,
                          double* d, double* n, double* H, double* vb)
{
    double ct = cos(q[3]), st = sin(q[3]);
    double r[3] = {xw[0] - q[0], xw[1] - q[1], xw[2] - q[2]};
    double p[3] = {ct * r[0] + st * r[1], -st * r[0] + ct * r[1], r[2]}; /* R(-theta) r */
    double nb[3], Hb[9];
    switch (kind) {
    case ORC_COLL_CAPSULE: sdf_capsule(p, s->coll_dims, d, nb, Hb); break;
    case ORC_COLL_BOX: sdf_box(p, s->coll_dims, d, nb, Hb); break;
    case ORC_COLL_CONTAINER: sdf_container(p, s->coll_dims, d, nb, Hb); break;
    default:
        *d = INFINITY;
        nb[0] = nb[1] = 0; nb[2] = 1;
        m3_zero(Hb);
    }
    double R[9] = {ct, -st, 0, st, ct, 0, 0, 0, 1};
    for (int i = 0; i < 3; i++) n[i] = R[3 * i] * nb[0] + R[3 * i + 1] * nb[1] + R[3 * i + 2] * nb[2];
    double T[9];
    m3_mul(R, Hb, T);
    m3_mul_bt(T, R, H);
    vb[0] = u[0] - u[3] * r[1];
    vb[1] = u[1] + u[3] * r[0];
    vb[2] = u[2];
}

int orc_pose_len(const orc_spec* s)
{
    return s->coll_kind == ORC_COLL_CAPSULES ? 4 * s->n_caps : 4;
}

/* The collider at xw: a single body, or for ORC_COLL_CAPSULES the union of the capsules,
 * i.e. the capsule nearest to xw (smallest signed distance; the first on a tie), whose index
 * is returned in *which (0 for single bodies). */
static void collider_pick(const orc_spec* s, const double* xw, const double* q, const double* u, double* d,
                          double* n, double* H, double* vb, int* which)
{
    *which = 0;
    if (s->coll_kind != ORC_COLL_CAPSULES) {
        collider_body(s, s->coll_kind, xw, q, u, d, n, H, vb);
        return;
    }
    collider_body(s, ORC_COLL_CAPSULE, xw, q, u, d, n, H, vb);
    for (int j = 1; j < s->n_caps; j++) {
        double dj, nj[3], Hj[9], vj[3];
        collider_body(s, ORC_COLL_CAPSULE, xw, q + 4 * j, u + 4 * j, &dj, nj, Hj, vj);
        if (dj < *d) {
            *d = dj;
            memcpy(n, nj, sizeof nj);
            memcpy(H, Hj, sizeof Hj);
            memcpy(vb, vj, sizeof vj);
            *which = j;
        }
    }
}

void orc_collider(const orc_spec* s, const double* xw, const double* q, const double* u,
                  double* d, double* n, double* H, double* vb)
{
    int which;
    collider_pick(s, xw, q, u, d, n, H, vb, &which);
}

/* dd/dtheta and dn/dtheta at xw (world frame) for the body `kind` at pose q. */
static void collider_dtheta(const orc_spec* s, int kind, const double* xw, const double* q, double* dd_dth,
                            double* dn_dth)
{
    double ct = cos(q[3]), st = sin(q[3]);
    double r[3] = {xw[0] - q[0], xw[1] - q[1], xw[2] - q[2]};
    double p[3] = {ct * r[0] + st * r[1], -st * r[0] + ct * r[1], r[2]};
    double nb[3], Hb[9], d;
    switch (kind) {
    case ORC_COLL_CAPSULE: sdf_capsule(p, s->coll_dims, &d, nb, Hb); break;
    case ORC_COLL_BOX: sdf_box(p, s->coll_dims, &d, nb, Hb); break;
    case ORC_COLL_CONTAINER: sdf_container(p, s->coll_dims, &d, nb, Hb); break;
    default:
        *dd_dth = 0; dn_dth[0] = dn_dth[1] = dn_dth[2] = 0;
        return;
    }
    double tb[3] = {p[1], -p[0], 0.0}; /* dp/dtheta for p = R(-theta) r */
    *dd_dth = v3_dot(nb, tb);
    double hb[3];
    for (int i = 0; i < 3; i++) hb[i] = Hb[3 * i] * tb[0] + Hb[3 * i + 1] * tb[1] + Hb[3 * i + 2] * tb[2];
    /* dn/dtheta = R (K nb + Hb tb), K = generator of rotation about z */
    double kb[3] = {-nb[1] + hb[0], nb[0] + hb[1], hb[2]};
    dn_dth[0] = ct * kb[0] - st * kb[1];
    dn_dth[1] = st * kb[0] + ct * kb[1];
    dn_dth[2] = kb[2];
}

/* ------------------------------------------------------------------ B-spline weights */

/* Quadratic B-spline weights at the three nodes base+0..2 for fx = X - base in [0.5, 1.5),
 * and their derivatives with respect to fx. */
void orc_weights(double fx, double* w, double* dw)
{
    w[0] = 0.5 * (1.5 - fx) * (1.5 - fx);
    w[1] = 0.75 - (fx - 1.0) * (fx - 1.0);
    w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);
    dw[0] = fx - 1.5;
    dw[1] = -2.0 * (fx - 1.0);
    dw[2] = fx - 0.5;
}

/* Cell base per axis, clamped into [0, G-3]; sets *oob when clamping. */
static void particle_base(const orc_spec* s, const double* x, int* base, double* fx, int* oob)
{
    double G = (double)s->G;
    for (int k = 0; k < 3; k++) {
        double X = x[k] * G;
        double fb = floor(X - 0.5);
        int b;
        if (!(fb == fb) || fb < 0.0) { b = 0; *oob = 1; }
        else if (fb > (double)(s->G - 3)) { b = s->G - 3; *oob = 1; }
        else b = (int)fb;
        base[k] = b;
        fx[k] = X - b;
    }
}

static double group_act(const orc_spec* s, const int* group, int p, const double* act)
{
    if (s->material != ORC_MUSCLE || !group || !act) return 0.0;
    int g = group[p];
    if (g < 0 || g >= s->n_groups) return 0.0;
    return act[s->n_coll_act + g];
}

/* ------------------------------------------------------------------ forward stages */

int orc_p2g(const orc_spec* s, int n, const double* x, const double* v, const double* C,
            const double* F, const int* group, const double* act, double* g)
{
    int G = s->G, status = 0;
    double dx = 1.0 / G, Dinv = 4.0 * G * G; /* D^-1 = 4/dx^2 */
    for (int p = 0; p < n; p++) {
        int base[3], oob = 0;
        double fx[3], w[3][3], dw[3][3];
        particle_base(s, x + 3 * p, base, fx, &oob);
        if (oob) status |= ORC_ST_DOMAIN;
        for (int k = 0; k < 3; k++) orc_weights(fx[k], w[k], dw[k]);
        double tau[9], A[9];
        orc_tau(s, F + 9 * p, C + 9 * p, group_act(s, group, p, act), tau);
        for (int i = 0; i < 9; i++) A[i] = s->p_mass * C[9 * p + i] - s->dt * s->p_vol * Dinv * tau[i];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][b] * w[2][c];
                    int ix = base[0] + a, iy = base[1] + b, iz = base[2] + c;
                    double r[3] = {ix * dx - x[3 * p], iy * dx - x[3 * p + 1], iz * dx - x[3 * p + 2]};
                    double* gn = g + 4 * (((long)iz * G + iy) * G + ix);
                    gn[0] += wt * s->p_mass;
                    for (int i = 0; i < 3; i++)
                        gn[1 + i] += wt * (s->p_mass * v[3 * p + i] + A[3 * i] * r[0] + A[3 * i + 1] * r[1] +
                                           A[3 * i + 2] * r[2]);
                }
    }
    return status;
}

/* Node update (forward).  Returns the final velocity in vo. */
static void node_update(const orc_spec* s, int ix, int iy, int iz, const double* gn, const double* q,
                        const double* u, double* vo)
{
    int G = s->G, b = s->bound;
    double dx = 1.0 / G;
    double v[3];
    for (int i = 0; i < 3; i++) v[i] = gn[1 + i] / gn[0] + s->dt * s->gravity[i];
    if (s->coll_kind != ORC_COLL_NONE) {
        double xw[3] = {ix * dx, iy * dx, iz * dx}, d, nn[3], H[9], vb[3];
        int which;
        collider_pick(s, xw, q, u, &d, nn, H, vb, &which);
        double sc = d > 0 ? exp(-s->alpha * d) : 1.0;
        double vr[3] = {v[0] - vb[0], v[1] - vb[1], v[2] - vb[2]};
        double vn = v3_dot(vr, nn);
        double vr2[3];
        if (vn < 0) {
            double vt[3] = {vr[0] - vn * nn[0], vr[1] - vn * nn[1], vr[2] - vn * nn[2]};
            double L = sqrt(v3_dot(vt, vt));
            double f = L > 0 ? 1.0 + s->coll_mu * vn / L : 0.0;
            if (f < 0) f = 0;
            for (int i = 0; i < 3; i++) vr2[i] = f * vt[i];
        } else {
            memcpy(vr2, vr, sizeof vr);
        }
        for (int i = 0; i < 3; i++) v[i] = v[i] + sc * (vr2[i] + vb[i] - v[i]);
    }
    if (iz < b && v[2] < 0) {
        if (s->ground_mu > 0) {
            double L = sqrt(v[0] * v[0] + v[1] * v[1]);
            double f = L > 0 ? 1.0 + s->ground_mu * v[2] / L : 0.0;
            if (f < 0) f = 0;
            v[0] *= f;
            v[1] *= f;
        }
        v[2] = 0;
    }
    int idx[3] = {ix, iy, iz};
    for (int k = 0; k < 2; k++)
        if ((idx[k] < b && v[k] < 0) || (idx[k] >= G - b && v[k] > 0)) v[k] = 0;
    if (iz >= G - b && v[2] > 0) v[2] = 0;
    memcpy(vo, v, sizeof v);
}

void orc_grid_update(const orc_spec* s, const double* g, const double* q, const double* u, double* gv)
{
    int G = s->G;
    for (int iz = 0; iz < G; iz++)
        for (int iy = 0; iy < G; iy++)
            for (int ix = 0; ix < G; ix++) {
                long id = ((long)iz * G + iy) * G + ix;
                const double* gn = g + 4 * id;
                if (gn[0] > 0) {
                    node_update(s, ix, iy, iz, gn, q, u, gv + 3 * id);
                } else {
                    gv[3 * id] = gv[3 * id + 1] = gv[3 * id + 2] = 0.0;
                }
            }
}

int orc_g2p(const orc_spec* s, int n, double* x, double* v, double* C, double* F, const double* gv)
{
    int G = s->G, status = 0;
    double dx = 1.0 / G, Dinv = 4.0 * G * G;
    for (int p = 0; p < n; p++) {
        int base[3], oob = 0;
        double fx[3], w[3][3], dw[3][3];
        particle_base(s, x + 3 * p, base, fx, &oob);
        if (oob) status |= ORC_ST_DOMAIN;
        for (int k = 0; k < 3; k++) orc_weights(fx[k], w[k], dw[k]);
        double vn[3] = {0, 0, 0}, Cn[9] = {0};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][b] * w[2][c];
                    int ix = base[0] + a, iy = base[1] + b, iz = base[2] + c;
                    double r[3] = {ix * dx - x[3 * p], iy * dx - x[3 * p + 1], iz * dx - x[3 * p + 2]};
                    const double* gvn = gv + 3 * (((long)iz * G + iy) * G + ix);
                    for (int i = 0; i < 3; i++) {
                        vn[i] += wt * gvn[i];
                        for (int j = 0; j < 3; j++) Cn[3 * i + j] += Dinv * wt * gvn[i] * r[j];
                    }
                }
        double Ft[9], Fup[9];
        m3_eye(Fup);
        for (int i = 0; i < 9; i++) Fup[i] += s->dt * Cn[i];
        m3_mul(Fup, F + 9 * p, Ft);
        orc_project(s, Ft, F + 9 * p);
        for (int i = 0; i < 3; i++) {
            v[3 * p + i] = vn[i];
            x[3 * p + i] += s->dt * vn[i];
        }
        memcpy(C + 9 * p, Cn, sizeof Cn);
        double J = m3_det(F + 9 * p);
        if (!(J > 0)) status |= ORC_ST_INVERTED;
        for (int i = 0; i < 3; i++)
            if (!isfinite(x[3 * p + i])) status |= ORC_ST_NAN;
    }
    return status;
}

int orc_substep(const orc_spec* s, int n, double* x, double* v, double* C, double* F, const int* group,
                const double* q, const double* u, const double* act)
{
    long NN = (long)s->G * s->G * s->G;
    double* g = (double*)calloc(4 * NN, sizeof(double));
    double* gv = (double*)calloc(3 * NN, sizeof(double));
    int st = orc_p2g(s, n, x, v, C, F, group, act, g);
    orc_grid_update(s, g, q, u, gv);
    st |= orc_g2p(s, n, x, v, C, F, gv);
    free(g);
    free(gv);
    return st;
}

/* ------------------------------------------------------------------ adjoint stages */

/*
 * Adjoint of node_update.  vob: adjoint of the node's final velocity.  Outputs the
 * adjoints of the node's (m, p) in gnb (accumulated), and accumulates dL/dq into qb
 * and dL/du into ub through the collider terms.
 */
static void node_update_adj(const orc_spec* s, int ix, int iy, int iz, const double* gn,
                            const double* q, const double* u, const double* vob, double* gnb,
                            double* qb, double* ub)
{
    int G = s->G, b = s->bound;
    double dx = 1.0 / G;
    /* ---- recompute the forward trace ---- */
    double v0[3], v1[3];
    for (int i = 0; i < 3; i++) {
        v0[i] = gn[1 + i] / gn[0];
        v1[i] = v0[i] + s->dt * s->gravity[i];
    }
    double v2[3];
    memcpy(v2, v1, sizeof v1);
    double xw[3] = {ix * dx, iy * dx, iz * dx}, d = 0, nn[3] = {0, 0, 1}, H[9], vb[3] = {0, 0, 0};
    double sc = 0, vr[3], vn = 0, vt[3] = {0, 0, 0}, L = 0, f = 0, vr2[3];
    int branch = 0; /* 0: separating, 1: friction f>0, 2: stopped */
    int which = 0;  /* body whose pose the contact depends on */
    if (s->coll_kind != ORC_COLL_NONE) {
        collider_pick(s, xw, q, u, &d, nn, H, vb, &which);
        sc = d > 0 ? exp(-s->alpha * d) : 1.0;
        for (int i = 0; i < 3; i++) vr[i] = v1[i] - vb[i];
        vn = v3_dot(vr, nn);
        if (vn < 0) {
            for (int i = 0; i < 3; i++) vt[i] = vr[i] - vn * nn[i];
            L = sqrt(v3_dot(vt, vt));
            f = L > 0 ? 1.0 + s->coll_mu * vn / L : 0.0;
            if (f > 0) {
                branch = 1;
                for (int i = 0; i < 3; i++) vr2[i] = f * vt[i];
            } else {
                branch = 2;
                vr2[0] = vr2[1] = vr2[2] = 0;
            }
        } else {
            memcpy(vr2, vr, sizeof vr);
        }
        for (int i = 0; i < 3; i++) v2[i] = v1[i] + sc * (vr2[i] + vb[i] - v1[i]);
    }
    double v3v[3];
    memcpy(v3v, v2, sizeof v2);
    int ground = 0;
    double gL = 0, gf = 0;
    if (iz < b && v2[2] < 0) {
        ground = 1;
        if (s->ground_mu > 0) {
            gL = sqrt(v2[0] * v2[0] + v2[1] * v2[1]);
            gf = gL > 0 ? 1.0 + s->ground_mu * v2[2] / gL : 0.0;
            if (gf < 0) gf = 0;
            v3v[0] *= gf;
            v3v[1] *= gf;
        }
        v3v[2] = 0;
    }
    int idx[3] = {ix, iy, iz};
    int zero[3] = {0, 0, 0};
    for (int k = 0; k < 2; k++)
        if ((idx[k] < b && v3v[k] < 0) || (idx[k] >= G - b && v3v[k] > 0)) zero[k] = 1;
    if (iz >= G - b && v3v[2] > 0) zero[2] = 1;

    /* ---- reverse ---- */
    double v3b[3];
    for (int k = 0; k < 3; k++) v3b[k] = zero[k] ? 0.0 : vob[k];
    double v2b[3];
    if (ground) {
        if (s->ground_mu > 0) {
            if (gL > 0 && gf > 0) {
                double dot = v3b[0] * v2[0] + v3b[1] * v2[1];
                /* gf = 1 + mu vz / L: dgf/dvxy = -mu vz vxy / L^3, dgf/dvz = mu / L */
                v2b[0] = gf * v3b[0] + dot * (-s->ground_mu * v2[2] * v2[0] / (gL * gL * gL));
                v2b[1] = gf * v3b[1] + dot * (-s->ground_mu * v2[2] * v2[1] / (gL * gL * gL));
                v2b[2] = dot * s->ground_mu / gL;
            } else {
                v2b[0] = v2b[1] = v2b[2] = 0.0;
            }
        } else {
            v2b[0] = v3b[0];
            v2b[1] = v3b[1];
            v2b[2] = 0.0;
        }
    } else {
        memcpy(v2b, v3b, sizeof v3b);
    }
    double v1b[3];
    if (s->coll_kind != ORC_COLL_NONE) {
        /* v2 = v1 + sc (vr2 + vb - v1) */
        double scb = 0;
        for (int i = 0; i < 3; i++) {
            v1b[i] = (1.0 - sc) * v2b[i];
            scb += v2b[i] * (vr2[i] + vb[i] - v1[i]);
        }
        double vr2b[3] = {sc * v2b[0], sc * v2b[1], sc * v2b[2]};
        double vbb[3] = {vr2b[0], vr2b[1], vr2b[2]};
        double vrb[3] = {0, 0, 0}, nb[3] = {0, 0, 0};
        if (branch == 0) {
            for (int i = 0; i < 3; i++) vrb[i] = vr2b[i];
        } else if (branch == 1) {
            /* vr2 = f vt, f = 1 + mu vn / L */
            double dot = v3_dot(vr2b, vt);
            double vtb[3];
            for (int i = 0; i < 3; i++) vtb[i] = f * vr2b[i] - dot * s->coll_mu * vn * vt[i] / (L * L * L);
            double vnb = dot * s->coll_mu / L;
            /* vt = vr - vn n */
            for (int i = 0; i < 3; i++) {
                vrb[i] += vtb[i];
                nb[i] += -vn * vtb[i];
            }
            vnb += -v3_dot(vtb, nn);
            /* vn = vr . n */
            for (int i = 0; i < 3; i++) {
                vrb[i] += vnb * nn[i];
                nb[i] += vnb * vr[i];
            }
        }
        /* vr = v1 - vb */
        for (int i = 0; i < 3; i++) {
            v1b[i] += vrb[i];
            vbb[i] -= vrb[i];
        }
        double db = d > 0 ? scb * (-s->alpha * sc) : 0.0;
        /* pose adjoints: dd/dc = -n, dn/dc = -H, dvb/dc via omega, and theta terms */
        double dd_dth, dn_dth[3];
        const double* qj = q + 4 * which;
        const double* uj = u + 4 * which;
        double* qbj = qb + 4 * which;
        double* ubj = ub + 4 * which;
        collider_dtheta(s, s->coll_kind == ORC_COLL_CAPSULES ? ORC_COLL_CAPSULE : s->coll_kind, xw, qj, &dd_dth,
                        dn_dth);
        double r[3] = {xw[0] - qj[0], xw[1] - qj[1], xw[2] - qj[2]};
        for (int i = 0; i < 3; i++) {
            double Hn = H[3 * i] * nb[0] + H[3 * i + 1] * nb[1] + H[3 * i + 2] * nb[2];
            qbj[i] += -nn[i] * db - Hn;
        }
        qbj[0] += -uj[3] * vbb[1];
        qbj[1] += uj[3] * vbb[0];
        qbj[3] += dd_dth * db + v3_dot(dn_dth, nb);
        ubj[0] += vbb[0];
        ubj[1] += vbb[1];
        ubj[2] += vbb[2];
        ubj[3] += -r[1] * vbb[0] + r[0] * vbb[1];
    } else {
        memcpy(v1b, v2b, sizeof v2b);
    }
    /* v0 = p/m */
    double m = gn[0];
    double dot = v3_dot(v1b, v0);
    gnb[0] += -dot / m;
    for (int i = 0; i < 3; i++) gnb[1 + i] += v1b[i] / m;
}

int orc_substep_adj(const orc_spec* s, int n, const double* x, const double* v, const double* C,
                    const double* F, const int* group, const double* q, const double* u,
                    const double* act, double* xb, double* vb, double* Cb, double* Fb, double* qb,
                    double* ub, double* actb)
{
    int G = s->G, status = 0;
    long NN = (long)G * G * G;
    double dx = 1.0 / G, Dinv = 4.0 * G * G;
    /* forward recomputation of this substep's grid */
    double* g = (double*)calloc(4 * NN, sizeof(double));
    double* gv = (double*)calloc(3 * NN, sizeof(double));
    double* gvb = (double*)calloc(3 * NN, sizeof(double));
    double* gb = (double*)calloc(4 * NN, sizeof(double));
    status |= orc_p2g(s, n, x, v, C, F, group, act, g);
    orc_grid_update(s, g, q, u, gv);

    /* ---- G2P adjoint: particle adjoints in (xb, Fb) partial, grid velocity adjoint ---- */
    double* xbp = (double*)calloc(3 * (size_t)n, sizeof(double));
    double* Fbp = (double*)calloc(9 * (size_t)n, sizeof(double));
    for (int p = 0; p < n; p++) {
        int base[3], oob = 0;
        double fx[3], w[3][3], dw[3][3];
        particle_base(s, x + 3 * p, base, fx, &oob);
        for (int k = 0; k < 3; k++) orc_weights(fx[k], w[k], dw[k]);
        /* recompute v', C' */
        double vn[3] = {0, 0, 0}, Cn[9] = {0};
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][bb] * w[2][c];
                    int ix = base[0] + a, iy = base[1] + bb, iz = base[2] + c;
                    double r[3] = {ix * dx - x[3 * p], iy * dx - x[3 * p + 1], iz * dx - x[3 * p + 2]};
                    const double* gvn = gv + 3 * (((long)iz * G + iy) * G + ix);
                    for (int i = 0; i < 3; i++) {
                        vn[i] += wt * gvn[i];
                        for (int j = 0; j < 3; j++) Cn[3 * i + j] += Dinv * wt * gvn[i] * r[j];
                    }
                }
        double Fup[9], Ft[9];
        m3_eye(Fup);
        for (int i = 0; i < 9; i++) Fup[i] += s->dt * Cn[i];
        m3_mul(Fup, F + 9 * p, Ft);
        /* F' = Proj(Ft) */
        double Ftb[9];
        orc_project_vjp(s, Ft, Fb + 9 * p, Ftb);
        /* Ft = (I + dt C') F */
        double Cnb[9], T[9];
        m3_mul_bt(Ftb, F + 9 * p, T); /* Ftb F^T */
        for (int i = 0; i < 9; i++) Cnb[i] = Cb[9 * p + i] + s->dt * T[i];
        m3_mul_at(Fup, Ftb, T); /* (I + dt C')^T Ftb */
        for (int i = 0; i < 9; i++) Fbp[9 * p + i] = T[i];
        /* x' = x + dt v' */
        double vnb[3];
        for (int i = 0; i < 3; i++) {
            vnb[i] = vb[3 * p + i] + s->dt * xb[3 * p + i];
            xbp[3 * p + i] = xb[3 * p + i];
        }
        /* v' = sum w v_i ; C' = Dinv sum w v_i r^T */
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][bb] * w[2][c];
                    double gw[3] = {dw[0][a] * w[1][bb] * w[2][c] * G, w[0][a] * dw[1][bb] * w[2][c] * G,
                                    w[0][a] * w[1][bb] * dw[2][c] * G};
                    int ix = base[0] + a, iy = base[1] + bb, iz = base[2] + c;
                    double r[3] = {ix * dx - x[3 * p], iy * dx - x[3 * p + 1], iz * dx - x[3 * p + 2]};
                    long id = ((long)iz * G + iy) * G + ix;
                    const double* gvn = gv + 3 * id;
                    double Cr[3], CTv[3];
                    for (int i = 0; i < 3; i++) {
                        Cr[i] = Cnb[3 * i] * r[0] + Cnb[3 * i + 1] * r[1] + Cnb[3 * i + 2] * r[2];
                        CTv[i] = Cnb[i] * gvn[0] + Cnb[3 + i] * gvn[1] + Cnb[6 + i] * gvn[2];
                    }
                    for (int i = 0; i < 3; i++) gvb[3 * id + i] += wt * vnb[i] + Dinv * wt * Cr[i];
                    double sdw = v3_dot(vnb, gvn) + Dinv * v3_dot(gvn, Cr);
                    for (int k = 0; k < 3; k++) xbp[3 * p + k] += sdw * gw[k] - Dinv * wt * CTv[k];
                }
    }

    /* ---- grid adjoint ---- */
    for (int iz = 0; iz < G; iz++)
        for (int iy = 0; iy < G; iy++)
            for (int ix = 0; ix < G; ix++) {
                long id = ((long)iz * G + iy) * G + ix;
                if (g[4 * id] > 0) node_update_adj(s, ix, iy, iz, g + 4 * id, q, u, gvb + 3 * id, gb + 4 * id, qb, ub);
            }

    /* ---- P2G adjoint: gather grid (m, p) adjoints ---- */
    for (int p = 0; p < n; p++) {
        int base[3], oob = 0;
        double fx[3], w[3][3], dw[3][3];
        particle_base(s, x + 3 * p, base, fx, &oob);
        for (int k = 0; k < 3; k++) orc_weights(fx[k], w[k], dw[k]);
        double a_g = group_act(s, group, p, act);
        double tau[9], A[9];
        orc_tau(s, F + 9 * p, C + 9 * p, a_g, tau);
        for (int i = 0; i < 9; i++) A[i] = s->p_mass * C[9 * p + i] - s->dt * s->p_vol * Dinv * tau[i];
        double Ab[9] = {0}, vbn[3] = {0, 0, 0}, xbn[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][bb] * w[2][c];
                    double gw[3] = {dw[0][a] * w[1][bb] * w[2][c] * G, w[0][a] * dw[1][bb] * w[2][c] * G,
                                    w[0][a] * w[1][bb] * dw[2][c] * G};
                    int ix = base[0] + a, iy = base[1] + bb, iz = base[2] + c;
                    double r[3] = {ix * dx - x[3 * p], iy * dx - x[3 * p + 1], iz * dx - x[3 * p + 2]};
                    const double* gbn = gb + 4 * (((long)iz * G + iy) * G + ix);
                    double qv[3];
                    for (int i = 0; i < 3; i++)
                        qv[i] = s->p_mass * v[3 * p + i] + A[3 * i] * r[0] + A[3 * i + 1] * r[1] + A[3 * i + 2] * r[2];
                    double pb[3] = {gbn[1], gbn[2], gbn[3]};
                    double coef = gbn[0] * s->p_mass + v3_dot(pb, qv);
                    for (int i = 0; i < 3; i++) {
                        vbn[i] += s->p_mass * wt * pb[i];
                        for (int j = 0; j < 3; j++) Ab[3 * i + j] += wt * pb[i] * r[j];
                    }
                    for (int k = 0; k < 3; k++) {
                        double ATp = A[k] * pb[0] + A[3 + k] * pb[1] + A[6 + k] * pb[2];
                        xbn[k] += coef * gw[k] - wt * ATp;
                    }
                }
        /* A = m C - dt V Dinv tau */
        double taub[9], Cbn[9], Fbn[9];
        for (int i = 0; i < 9; i++) {
            Cbn[i] = s->p_mass * Ab[i];
            taub[i] = -s->dt * s->p_vol * Dinv * Ab[i];
            Fbn[i] = Fbp[9 * p + i];
        }
        double agb = 0;
        orc_tau_vjp(s, F + 9 * p, C + 9 * p, a_g, taub, Fbn, Cbn, &agb);
        if (s->material == ORC_MUSCLE && group && actb) {
            int gi = group[p];
            if (gi >= 0 && gi < s->n_groups) actb[s->n_coll_act + gi] += agb;
        }
        for (int i = 0; i < 3; i++) {
            xb[3 * p + i] = xbp[3 * p + i] + xbn[i];
            vb[3 * p + i] = vbn[i];
        }
        memcpy(Cb + 9 * p, Cbn, sizeof Cbn);
        memcpy(Fb + 9 * p, Fbn, sizeof Fbn);
    }
    free(g);
    free(gv);
    free(gvb);
    free(gb);
    free(xbp);
    free(Fbp);
    return status;
}

/* ------------------------------------------------------------------ rewards */

/*
 * Per-control-step reward from the end state (App. E task definitions), on the
 * subsample x' = particles 0..n_sub-1:
 *  FLAT  (RollingFlat): d = mean(z')/h_flat, R_d = (1/(1+d))^2 * (d > 0.33 ? 1 : 2),
 *        R_flat = -Var(z'); r = R_d + R_flat.   rparam[0] = h_flat.
 *  REACH (FluidMove R_d): d = |c - p*|^2 with c the collider position, R_d =
 *        (1/(1+d))^2 * (d > 0.02 ? 1 : 2).       rparam[0..2] = p*.
 *  JUMP  (SoftJumper): r = mean(v'_x) + k_up (mean(z') - h0) - k_a sum a^2.
 *        rparam = (h0, k_up, k_a).
 */
double orc_reward(const orc_spec* s, int n, const double* x, const double* v, const double* q,
                  const double* a)
{
    int ns = s->n_sub < n ? s->n_sub : n;
    switch (s->reward_kind) {
    case ORC_REWARD_FLAT: {
        double mz = 0;
        for (int p = 0; p < ns; p++) mz += x[3 * p + 2];
        mz /= ns;
        double var = 0;
        for (int p = 0; p < ns; p++) var += (x[3 * p + 2] - mz) * (x[3 * p + 2] - mz);
        var /= ns;
        double d = mz / s->rparam[0];
        double Rd = 1.0 / ((1.0 + d) * (1.0 + d)) * (d > 0.33 ? 1.0 : 2.0);
        return Rd - var;
    }
    case ORC_REWARD_REACH: {
        double d = 0;
        for (int i = 0; i < 3; i++) d += (q[i] - s->rparam[i]) * (q[i] - s->rparam[i]);
        return 1.0 / ((1.0 + d) * (1.0 + d)) * (d > 0.02 ? 1.0 : 2.0);
    }
    case ORC_REWARD_JUMP: {
        double mv = 0, mz = 0;
        for (int p = 0; p < ns; p++) {
            mv += v[3 * p];
            mz += x[3 * p + 2];
        }
        mv /= ns;
        mz /= ns;
        int A = s->n_coll_act + s->n_groups;
        double aa = 0;
        for (int j = 0; j < A; j++) aa += a[j] * a[j];
        return mv + s->rparam[1] * (mz - s->rparam[0]) - s->rparam[2] * aa;
    }
    default:
        return 0.0;
    }
}

void orc_reward_adj(const orc_spec* s, int n, const double* x, const double* v, const double* q,
                    const double* a, double rb, double* xb, double* vb, double* qb, double* ab)
{
    (void)v; /* every reward is linear in v: its adjoint does not depend on v's value */
    int ns = s->n_sub < n ? s->n_sub : n;
    switch (s->reward_kind) {
    case ORC_REWARD_FLAT: {
        double mz = 0;
        for (int p = 0; p < ns; p++) mz += x[3 * p + 2];
        mz /= ns;
        double d = mz / s->rparam[0];
        double fac = d > 0.33 ? 1.0 : 2.0;
        double dRd = -2.0 * fac / ((1.0 + d) * (1.0 + d) * (1.0 + d));
        for (int p = 0; p < ns; p++) {
            /* d mz / dz_p = 1/ns ; d var / dz_p = 2 (z_p - mz) / ns */
            xb[3 * p + 2] += rb * (dRd / (s->rparam[0] * ns) - 2.0 * (x[3 * p + 2] - mz) / ns);
        }
        break;
    }
    case ORC_REWARD_REACH: {
        double d = 0;
        for (int i = 0; i < 3; i++) d += (q[i] - s->rparam[i]) * (q[i] - s->rparam[i]);
        double fac = d > 0.02 ? 1.0 : 2.0;
        double dRd = -2.0 * fac / ((1.0 + d) * (1.0 + d) * (1.0 + d));
        for (int i = 0; i < 3; i++) qb[i] += rb * dRd * 2.0 * (q[i] - s->rparam[i]);
        break;
    }
    case ORC_REWARD_JUMP: {
        for (int p = 0; p < ns; p++) {
            vb[3 * p] += rb / ns;
            xb[3 * p + 2] += rb * s->rparam[1] / ns;
        }
        int A = s->n_coll_act + s->n_groups;
        for (int j = 0; j < A; j++) ab[j] += rb * (-2.0 * s->rparam[2] * a[j]);
        break;
    }
    default:
        break;
    }
}

/* ------------------------------------------------------------------ observations */

/*
 * Observation of a state (App. E task tables of the MPM tasks): the subsampled particle
 * positions x' (particles 0..ns-1, ns = min(n_sub, n)), their mean (the CoM of the subsample
 * for uniform density), then 4 pose entries holding the pose components the actions drive
 * (in action order, zeros past n_coll_act), then 3 entries holding the reach target p*
 * (reward REACH, else zeros).  obs[orc_obs_dim(s, n)] = 3 ns + 10.
 */
int orc_obs_dim(const orc_spec* s, int n)
{
    int ns = s->n_sub < n ? s->n_sub : n;
    return 3 * ns + 10;
}

void orc_observe(const orc_spec* s, int n, const double* x, const double* q, double* obs)
{
    int ns = s->n_sub < n ? s->n_sub : n;
    double m[3] = {0, 0, 0};
    for (int p = 0; p < ns; p++)
        for (int k = 0; k < 3; k++) {
            obs[3 * p + k] = x[3 * p + k];
            m[k] += x[3 * p + k];
        }
    double* tail = obs + 3 * ns;
    for (int k = 0; k < 3; k++) tail[k] = ns ? m[k] / ns : 0.0;
    for (int j = 0; j < 4; j++)
        tail[3 + j] = s->coll_kind == ORC_COLL_CAPSULES ? q[j] : (j < s->n_coll_act ? q[s->act_map[j]] : 0.0);
    for (int k = 0; k < 3; k++) tail[7 + k] = s->reward_kind == ORC_REWARD_REACH ? s->rparam[k] : 0.0;
}

/* Adjoint of orc_observe for an observation adjoint ob: adds to xb and the pose adjoint qb. */
static void observe_adj(const orc_spec* s, int n, const double* ob, double* xb, double* qb)
{
    int ns = s->n_sub < n ? s->n_sub : n;
    const double* tail = ob + 3 * ns;
    for (int p = 0; p < ns; p++)
        for (int k = 0; k < 3; k++) xb[3 * p + k] += ob[3 * p + k] + tail[k] / ns;
    if (s->coll_kind == ORC_COLL_CAPSULES) {
        for (int j = 0; j < 4; j++) qb[j] += tail[3 + j];
    } else {
        for (int j = 0; j < s->n_coll_act; j++) qb[s->act_map[j]] += tail[3 + j];
    }
}

/* ------------------------------------------------------------------ rollouts */

/* Pose velocity over a control step: the step's relative pose change per unit time. */
static void pose_velocity(const orc_spec* s, const double* a, double* u)
{
    double h = s->S * s->dt;
    int pl = orc_pose_len(s);
    for (int i = 0; i < pl; i++) u[i] = 0.0;
    if (s->coll_kind == ORC_COLL_CAPSULES) {
        for (int j = 0; j < pl; j++) u[j] = s->act_scale[j % 4] * a[j] / h;
    } else {
        for (int j = 0; j < s->n_coll_act; j++) u[s->act_map[j]] += s->act_scale[j] * a[j] / h;
    }
}

int orc_rollout(const orc_spec* s, int n, double* x, double* v, double* C, double* F, const int* group,
                double* q, const double* actions, int T, double* rewards)
{
    int A = s->n_coll_act + s->n_groups, status = 0;
    for (int t = 0; t < T; t++) {
        const double* a = actions + (size_t)t * A;
        const int pl = orc_pose_len(s);
        double u[ORC_MAX_POSE], qk[ORC_MAX_POSE];
        pose_velocity(s, a, u);
        for (int k = 0; k < s->S; k++) {
            for (int i = 0; i < pl; i++) qk[i] = q[i] + k * s->dt * u[i];
            status |= orc_substep(s, n, x, v, C, F, group, qk, u, a);
        }
        for (int i = 0; i < pl; i++) q[i] += s->S * s->dt * u[i];
        if (rewards) rewards[t] = orc_reward(s, n, x, v, q, a);
    }
    return status;
}

int orc_rollout_adj(const orc_spec* s, int n, const double* x0, const double* v0, const double* C0,
                    const double* F0, const int* group, const double* q0, const double* actions, int T,
                    const double* xbT, const double* vbT, const double* CbT, const double* FbT,
                    const double* rbar, double* act_grad, double* xb0, double* vb0, double* Cb0,
                    double* Fb0, double* qb0)
{
    return orc_rollout_adj_obs(s, n, x0, v0, C0, F0, group, q0, actions, T, xbT, vbT, CbT, FbT, rbar, NULL,
                               act_grad, xb0, vb0, Cb0, Fb0, qb0);
}

/* As orc_rollout_adj, with the adjoints of the observations (orc_observe) of the states at
 * every control-step boundary: obs_adj[(T + 1) * orc_obs_dim], row t for the state before
 * step t, row T for the final state (NULL: none). */
int orc_rollout_adj_obs(const orc_spec* s, int n, const double* x0, const double* v0, const double* C0,
                        const double* F0, const int* group, const double* q0, const double* actions, int T,
                        const double* xbT, const double* vbT, const double* CbT, const double* FbT,
                        const double* rbar, const double* obs_adj, double* act_grad, double* xb0, double* vb0,
                        double* Cb0, double* Fb0, double* qb0)
{
    const int od = orc_obs_dim(s, n);
    int A = s->n_coll_act + s->n_groups, S = s->S, status = 0;
    size_t sx = 3 * (size_t)n, sm = 9 * (size_t)n, blk = 2 * sx + 2 * sm;
    /* checkpoints of (x, v, C, F) and pose at every control-step boundary */
    double* ck = (double*)malloc(blk * (T + 1) * sizeof(double));
    const int pl = orc_pose_len(s);
    double* qs = (double*)malloc((size_t)pl * (T + 1) * sizeof(double));
    double* ring = (double*)malloc(blk * S * sizeof(double));
    memcpy(ck, x0, sx * sizeof(double));
    memcpy(ck + sx, v0, sx * sizeof(double));
    memcpy(ck + 2 * sx, C0, sm * sizeof(double));
    memcpy(ck + 2 * sx + sm, F0, sm * sizeof(double));
    memcpy(qs, q0, pl * sizeof(double));
    for (int t = 0; t < T; t++) {
        double* cur = ck + blk * (t + 1);
        memcpy(cur, ck + blk * t, blk * sizeof(double));
        memcpy(qs + pl * (t + 1), qs + pl * t, pl * sizeof(double));
        status |= orc_rollout(s, n, cur, cur + sx, cur + 2 * sx, cur + 2 * sx + sm, group, qs + pl * (t + 1),
                              actions + (size_t)t * A, 1, NULL);
    }
    /* adjoint state */
    for (size_t i = 0; i < sx; i++) {
        xb0[i] = xbT ? xbT[i] : 0.0;
        vb0[i] = vbT ? vbT[i] : 0.0;
    }
    for (size_t i = 0; i < sm; i++) {
        Cb0[i] = CbT ? CbT[i] : 0.0;
        Fb0[i] = FbT ? FbT[i] : 0.0;
    }
    double qb[ORC_MAX_POSE];
    for (int i = 0; i < ORC_MAX_POSE; i++) qb[i] = 0.0;
    for (int t = T - 1; t >= 0; t--) {
        const double* a = actions + (size_t)t * A;
        double* ag = act_grad + (size_t)t * A;
        for (int j = 0; j < A; j++) ag[j] = 0.0;
        double* end = ck + blk * (t + 1);
        /* reward of step t, from the end state and end pose */
        if (rbar && rbar[t] != 0.0)
            orc_reward_adj(s, n, end, end + sx, qs + pl * (t + 1), a, rbar[t], xb0, vb0, qb, ag);
        /* observation of the end state */
        if (obs_adj) observe_adj(s, n, obs_adj + (size_t)(t + 1) * od, xb0, qb);
        /* recompute substep states s_0..s_{S-1} of step t */
        double u[ORC_MAX_POSE];
        pose_velocity(s, a, u);
        memcpy(ring, ck + blk * t, blk * sizeof(double));
        for (int k = 0; k + 1 < S; k++) {
            double* nx = ring + blk * (k + 1);
            memcpy(nx, ring + blk * k, blk * sizeof(double));
            double qk[ORC_MAX_POSE];
            for (int i = 0; i < pl; i++) qk[i] = qs[pl * t + i] + k * s->dt * u[i];
            orc_substep(s, n, nx, nx + sx, nx + 2 * sx, nx + 2 * sx + sm, group, qk, u, a);
        }
        /* q_{t+1} = q_t + h u: dL/du += h qb_{t+1}; dL/dq_t = qb_{t+1} + sum_k dL/dq_k */
        double h = S * s->dt;
        double ub[ORC_MAX_POSE];
        for (int i = 0; i < pl; i++) ub[i] = h * qb[i];
        for (int k = S - 1; k >= 0; k--) {
            double* st = ring + blk * k;
            double qk[ORC_MAX_POSE], qkb[ORC_MAX_POSE];
            for (int i = 0; i < pl; i++) {
                qk[i] = qs[pl * t + i] + k * s->dt * u[i];
                qkb[i] = 0.0;
            }
            orc_substep_adj(s, n, st, st + sx, st + 2 * sx, st + 2 * sx + sm, group, qk, u, a, xb0, vb0, Cb0,
                            Fb0, qkb, ub, ag);
            /* q_k = q_t + k dt u */
            for (int i = 0; i < pl; i++) {
                qb[i] += qkb[i];
                ub[i] += k * s->dt * qkb[i];
            }
        }
        /* u[map[j]] += act_scale[j] a[j] / h (capsules: u[j] = act_scale[j % 4] a[j] / h) */
        if (s->coll_kind == ORC_COLL_CAPSULES) {
            for (int j = 0; j < pl; j++) ag[j] += ub[j] * s->act_scale[j % 4] / h;
        } else {
            for (int j = 0; j < s->n_coll_act; j++) ag[j] += ub[s->act_map[j]] * s->act_scale[j] / h;
        }
    }
    if (obs_adj) observe_adj(s, n, obs_adj, xb0, qb); /* observation of the initial state */
    memcpy(qb0, qb, pl * sizeof(double));
    free(ck);
    free(qs);
    free(ring);
    return status;
}

/* ------------------------------------------------------------------ binning mirror */

/* Built with -ffp-contract=off: x*G and the subtraction of 0.5 round separately. */
void orc_bin_keys_f32(int n, const float* x, int G, unsigned* keys)
{
    int TG = G / 4;
    for (int p = 0; p < n; p++) {
        int b[3];
        for (int k = 0; k < 3; k++) {
            volatile float X = x[3 * p + k] * (float)G;
            volatile float Y = X - 0.5f;
            int bi = (int)floorf(Y);
            if (bi < 0) bi = 0;
            if (bi > G - 3) bi = G - 3;
            b[k] = bi;
        }
        unsigned tile = (unsigned)(((b[2] >> 2) * TG + (b[1] >> 2)) * TG + (b[0] >> 2));
        unsigned cell = (unsigned)((b[2] & 3) * 16 + (b[1] & 3) * 4 + (b[0] & 3));
        keys[p] = tile * 64u + cell;
    }
}

/* Stable counting sort of keys (in original order among equal keys). */
void orc_stable_sort_u32(int n, const unsigned* keys, unsigned* perm)
{
    unsigned kmax = 0;
    for (int p = 0; p < n; p++)
        if (keys[p] > kmax) kmax = keys[p];
    unsigned* cnt = (unsigned*)calloc((size_t)kmax + 2, sizeof(unsigned));
    for (int p = 0; p < n; p++) cnt[keys[p] + 1]++;
    for (unsigned k = 0; k <= kmax; k++) cnt[k + 1] += cnt[k];
    for (int p = 0; p < n; p++) perm[cnt[keys[p]]++] = (unsigned)p;
    free(cnt);
}
