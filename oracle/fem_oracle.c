/*
 * fem_oracle.c -- FP64 reference of the tetrahedral FEM environment (see fem_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY; never linked into the product library.
 *
 * Written step by step from App. D.2 (stable neo-Hookean energy of tetrahedral elements,
 * forces from the energy gradient, semi-implicit Euler) and App. E (SoftJumper: damping,
 * activations, reward), with the readings listed in fem_oracle.h.  The reverse mode is
 * derived by hand from the same steps in reverse order.
 */
#include "fem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ 3x3 helpers */

static void mat_mul(const double* A, const double* B, double* C) /* C = A B */
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat_mul_bt(const double* A, const double* B, double* C) /* C = A B^T */
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * j + k];
            C[3 * i + j] = s;
        }
}

static double det3(const double* A)
{
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static void cross(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Cofactor matrix dJ/dF: its rows are the cross products of F's other two rows. */
static void cofactor(const double* F, double* cof)
{
    cross(F + 3, F + 6, cof);
    cross(F + 6, F, cof + 3);
    cross(F, F + 3, cof + 6);
}

static int inv3(const double* A, double* Ai)
{
    double d = det3(A);
    if (d == 0.0) return -1;
    double cof[9];
    cofactor(A, cof);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Ai[3 * i + j] = cof[3 * j + i] / d; /* adj(A) = cof^T */
    return 0;
}

static double ddot9(const double* A, const double* B)
{
    double s = 0.0;
    for (int i = 0; i < 9; i++) s += A[i] * B[i];
    return s;
}

/* Edge matrix of element e: column c = p[tet[c+1]] - p[tet[0]]. */
static void edges(const int* tet, const double* p, double* D)
{
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < 3; c++) D[3 * i + c] = p[3 * tet[c + 1] + i] - p[3 * tet[0] + i];
}

/* ------------------------------------------------------------------ material (App. D.2) */

static double alpha_of(const fem_spec* s)
{
    return s->alpha != 0.0 ? s->alpha : 1.0 + 0.75 * s->mu / s->lam;
}

double fem_psi(const fem_spec* s, const double* F, double a)
{
    double Ic = ddot9(F, F), J = det3(F), al = alpha_of(s);
    return 0.5 * s->mu * (Ic - 3.0) + 0.5 * s->lam * (J - al - a) * (J - al - a) - 0.5 * s->mu * log(Ic + 1.0);
}

void fem_stress(const fem_spec* s, const double* F, double a, double* P)
{
    double Ic = ddot9(F, F), J = det3(F), al = alpha_of(s), cof[9];
    cofactor(F, cof);
    double c1 = s->mu * (1.0 - 1.0 / (Ic + 1.0)), c2 = s->lam * (J - al - a);
    for (int i = 0; i < 9; i++) P[i] = c1 * F[i] + c2 * cof[i];
}

void fem_stress_vjp(const fem_spec* s, const double* F, double a, const double* Pb, double* Fb, double* ab)
{
    /* Psi's Hessian is symmetric, so Fb = dP[Pb]:
     *   mu (1 - 1/(Ic+1)) Pb + 2 mu (F:Pb)/(Ic+1)^2 F + lam (cof:Pb) cof + lam (J - alpha - a) dcof[Pb],
     * with dcof[D] rows D1 x F2 + F1 x D2, D2 x F0 + F2 x D0, D0 x F1 + F0 x D1.  dP/da = -lam cof. */
    double Ic = ddot9(F, F), J = det3(F), al = alpha_of(s), cof[9];
    cofactor(F, cof);
    double c1 = s->mu * (1.0 - 1.0 / (Ic + 1.0));
    double c3 = 2.0 * s->mu * ddot9(F, Pb) / ((Ic + 1.0) * (Ic + 1.0));
    double cp = ddot9(cof, Pb);
    double c4 = s->lam * cp, c5 = s->lam * (J - al - a);
    double dc[9], t1[3], t2[3];
    cross(Pb + 3, F + 6, t1);
    cross(F + 3, Pb + 6, t2);
    for (int k = 0; k < 3; k++) dc[k] = t1[k] + t2[k];
    cross(Pb + 6, F, t1);
    cross(F + 6, Pb, t2);
    for (int k = 0; k < 3; k++) dc[3 + k] = t1[k] + t2[k];
    cross(Pb, F + 3, t1);
    cross(F, Pb + 3, t2);
    for (int k = 0; k < 3; k++) dc[6 + k] = t1[k] + t2[k];
    for (int i = 0; i < 9; i++) Fb[i] = c1 * Pb[i] + c3 * F[i] + c4 * cof[i] + c5 * dc[i];
    if (ab) *ab = -s->lam * cp;
}

/* ------------------------------------------------------------------ mesh */

int fem_rest(const fem_spec* s, const int* tets, const double* rest_x, double rho, double* dminv, double* vol,
             double* inv_mass)
{
    double* m = calloc((size_t)s->n_v, sizeof(double));
    int bad = 0;
    for (int e = 0; e < s->n_t; e++) {
        double Dm[9];
        edges(tets + 4 * e, rest_x, Dm);
        double d = det3(Dm);
        if (d == 0.0 || inv3(Dm, dminv + 9 * e)) {
            bad = 1;
            continue;
        }
        vol[e] = fabs(d) / 6.0;
        for (int c = 0; c < 4; c++) m[tets[4 * e + c]] += 0.25 * rho * vol[e];
    }
    for (int i = 0; i < s->n_v; i++) inv_mass[i] = m[i] > 0.0 ? 1.0 / m[i] : 0.0;
    free(m);
    return bad ? -1 : 0;
}

double fem_energy(const fem_spec* s, const int* tets, const double* dminv, const double* vol, const double* x,
                  const double* a_elem)
{
    double E = 0.0;
    for (int e = 0; e < s->n_t; e++) {
        double Ds[9], F[9];
        edges(tets + 4 * e, x, Ds);
        mat_mul(Ds, dminv + 9 * e, F);
        E += vol[e] * fem_psi(s, F, a_elem ? a_elem[e] : 0.0);
    }
    return E;
}

/* Forces of element e with total stress Pt: H = -V0 Pt Dm^-T, f_{c+1} += H[:, c], f_0 -= sum. */
static void scatter_force(const int* tet, double V0, const double* Pt, const double* Dmi, double* f)
{
    double H[9];
    mat_mul_bt(Pt, Dmi, H); /* Pt (Dm^-1)^T */
    for (int c = 0; c < 3; c++)
        for (int i = 0; i < 3; i++) {
            double h = -V0 * H[3 * i + c];
            f[3 * tet[c + 1] + i] += h;
            f[3 * tet[0] + i] -= h;
        }
}

void fem_forces(const fem_spec* s, const int* tets, const double* dminv, const double* vol, const double* x,
                const double* v, const double* a_elem, double* f)
{
    memset(f, 0, sizeof(double) * 3 * (size_t)s->n_v);
    for (int e = 0; e < s->n_t; e++) {
        const int* tet = tets + 4 * e;
        double Ds[9], Vs[9], F[9], Fd[9], P[9];
        edges(tet, x, Ds);
        edges(tet, v, Vs);
        mat_mul(Ds, dminv + 9 * e, F);
        mat_mul(Vs, dminv + 9 * e, Fd); /* dF/dt */
        fem_stress(s, F, a_elem ? a_elem[e] : 0.0, P);
        for (int i = 0; i < 9; i++) P[i] += s->k_damp * Fd[i];
        scatter_force(tet, vol[e], P, dminv + 9 * e, f);
    }
}

/* ------------------------------------------------------------------ substep */

static int elem_status(const fem_spec* s, const int* tets, const double* dminv, const double* x)
{
    int st = 0;
    for (int e = 0; e < s->n_t; e++) {
        double Ds[9], F[9];
        edges(tets + 4 * e, x, Ds);
        mat_mul(Ds, dminv + 9 * e, F);
        double J = det3(F);
        if (!(J > 0.0)) st |= FEM_ST_INVERTED;
        if (!isfinite(J)) st |= FEM_ST_NAN;
    }
    return st;
}

int fem_substep(const fem_spec* s, const int* tets, const double* dminv, const double* vol, const double* inv_mass,
                double* x, double* v, const double* a_elem)
{
    int n = s->n_v;
    double* f = malloc(sizeof(double) * 3 * (size_t)n);
    int st = elem_status(s, tets, dminv, x);
    fem_forces(s, tets, dminv, vol, x, v, a_elem, f);
    for (int i = 0; i < n; i++) {
        double w[3];
        for (int k = 0; k < 3; k++) w[k] = v[3 * i + k] + s->dt * (inv_mass[i] * f[3 * i + k] + s->gravity[k]);
        if (x[3 * i + 2] <= s->ground_z && w[2] < 0.0) {
            double L = sqrt(w[0] * w[0] + w[1] * w[1]);
            double g = L > 0.0 ? fmax(0.0, 1.0 + s->ground_mu * w[2] / L) : 0.0;
            w[0] *= g;
            w[1] *= g;
            w[2] = 0.0;
        }
        for (int k = 0; k < 3; k++) {
            v[3 * i + k] = w[k];
            x[3 * i + k] += s->dt * w[k];
            if (!isfinite(x[3 * i + k])) st |= FEM_ST_NAN;
        }
    }
    free(f);
    return st;
}

/* Reverse of fem_substep from the substep's start state (x, v): xb, vb hold the adjoint of
 * the end state on entry and of the start state on return; ab_elem[e] += adjoint of a_e. */
static void fem_substep_adj(const fem_spec* s, const int* tets, const double* dminv, const double* vol,
                            const double* inv_mass, const double* x, const double* v, const double* a_elem,
                            double* xb, double* vb, double* ab_elem)
{
    int n = s->n_v;
    double* f = malloc(sizeof(double) * 3 * (size_t)n);
    double* fb = malloc(sizeof(double) * 3 * (size_t)n);
    fem_forces(s, tets, dminv, vol, x, v, a_elem, f);
    for (int i = 0; i < n; i++) {
        double w[3], out_b[3], wb[3];
        for (int k = 0; k < 3; k++) w[k] = v[3 * i + k] + s->dt * (inv_mass[i] * f[3 * i + k] + s->gravity[k]);
        /* x' = x + dt v': x-bar passes through, v'-bar gains dt x'-bar */
        for (int k = 0; k < 3; k++) out_b[k] = vb[3 * i + k] + s->dt * xb[3 * i + k];
        if (x[3 * i + 2] <= s->ground_z && w[2] < 0.0) {
            double L = sqrt(w[0] * w[0] + w[1] * w[1]);
            double g = L > 0.0 ? fmax(0.0, 1.0 + s->ground_mu * w[2] / L) : 0.0;
            /* out = (g w_x, g w_y, 0) with g = 1 + mu w_z / L where positive */
            if (L > 0.0 && g > 0.0) {
                double dot = out_b[0] * w[0] + out_b[1] * w[1];
                double iL3 = 1.0 / (L * L * L);
                wb[0] = g * out_b[0] - dot * s->ground_mu * w[2] * w[0] * iL3;
                wb[1] = g * out_b[1] - dot * s->ground_mu * w[2] * w[1] * iL3;
                wb[2] = dot * s->ground_mu / L;
            } else {
                wb[0] = wb[1] = wb[2] = 0.0;
            }
        } else {
            for (int k = 0; k < 3; k++) wb[k] = out_b[k];
        }
        /* w = v + dt (f / m + g) */
        for (int k = 0; k < 3; k++) {
            vb[3 * i + k] = wb[k];
            fb[3 * i + k] = s->dt * inv_mass[i] * wb[k];
        }
    }
    /* forces: per element, H-bar columns f-bar_{c+1} - f-bar_0, Pt-bar = -V0 H-bar Dm^-1 */
    for (int e = 0; e < s->n_t; e++) {
        const int* tet = tets + 4 * e;
        const double* Dmi = dminv + 9 * e;
        double Hb[9], Ptb[9], Ds[9], F[9], Fb[9], Fdb[9], Dsb[9], Vsb[9], ab = 0.0;
        for (int i = 0; i < 3; i++)
            for (int c = 0; c < 3; c++) Hb[3 * i + c] = fb[3 * tet[c + 1] + i] - fb[3 * tet[0] + i];
        mat_mul(Hb, Dmi, Ptb);
        for (int i = 0; i < 9; i++) Ptb[i] *= -vol[e];
        edges(tet, x, Ds);
        mat_mul(Ds, Dmi, F);
        fem_stress_vjp(s, F, a_elem ? a_elem[e] : 0.0, Ptb, Fb, &ab);
        if (ab_elem) ab_elem[e] += ab;
        for (int i = 0; i < 9; i++) Fdb[i] = s->k_damp * Ptb[i];
        mat_mul_bt(Fb, Dmi, Dsb);  /* F = Ds Dm^-1 */
        mat_mul_bt(Fdb, Dmi, Vsb); /* dF/dt = Vs Dm^-1 */
        for (int c = 0; c < 3; c++)
            for (int i = 0; i < 3; i++) {
                xb[3 * tet[c + 1] + i] += Dsb[3 * i + c];
                xb[3 * tet[0] + i] -= Dsb[3 * i + c];
                vb[3 * tet[c + 1] + i] += Vsb[3 * i + c];
                vb[3 * tet[0] + i] -= Vsb[3 * i + c];
            }
    }
    free(f);
    free(fb);
}

/* ------------------------------------------------------------------ control steps */

static void elem_acts(const fem_spec* s, const int* group, const double* a, double* a_elem)
{
    for (int e = 0; e < s->n_t; e++) a_elem[e] = s->act_scale * a[group[e]];
}

static double reward(const fem_spec* s, const double* x, const double* v, const double* a)
{
    if (s->reward_kind != FEM_REWARD_JUMP) return 0.0;
    int ns = s->n_sub < s->n_v ? s->n_sub : s->n_v;
    double vx = 0.0, z = 0.0, aa = 0.0;
    for (int i = 0; i < ns; i++) {
        vx += v[3 * i];
        z += x[3 * i + 2];
    }
    for (int j = 0; j < s->n_act; j++) aa += a[j] * a[j];
    return vx / ns + s->rparam[1] * (z / ns - s->rparam[0]) - s->rparam[2] * aa;
}

int fem_rollout(const fem_spec* s, const int* tets, const int* group, const double* dminv, const double* vol,
                const double* inv_mass, double* x, double* v, const double* actions, int T, double* rewards)
{
    double* ae = malloc(sizeof(double) * (size_t)(s->n_t > 0 ? s->n_t : 1));
    int st = 0;
    for (int t = 0; t < T; t++) {
        const double* a = actions + (size_t)t * s->n_act;
        elem_acts(s, group, a, ae);
        for (int k = 0; k < s->S; k++) st |= fem_substep(s, tets, dminv, vol, inv_mass, x, v, ae);
        if (rewards) rewards[t] = reward(s, x, v, a);
    }
    free(ae);
    return st;
}

int fem_rollout_adj(const fem_spec* s, const int* tets, const int* group, const double* dminv, const double* vol,
                    const double* inv_mass, const double* x0, const double* v0, const double* actions, int T,
                    const double* xbT, const double* vbT, const double* rbar, double* ag, double* xb0, double* vb0)
{
    int n3 = 3 * s->n_v, S = s->S, st = 0;
    size_t blk = (size_t)n3;
    /* checkpoints at control-step starts */
    double* ck = malloc(sizeof(double) * 2 * blk * (size_t)(T + 1));
    double* ring = malloc(sizeof(double) * 2 * blk * (size_t)(S + 1));
    double* ae = malloc(sizeof(double) * (size_t)(s->n_t > 0 ? s->n_t : 1));
    double* abe = malloc(sizeof(double) * (size_t)(s->n_t > 0 ? s->n_t : 1));
    memcpy(ck, x0, sizeof(double) * blk);
    memcpy(ck + blk, v0, sizeof(double) * blk);
    for (int t = 0; t < T; t++) {
        double* c0 = ck + 2 * blk * (size_t)t;
        double* c1 = c0 + 2 * blk;
        memcpy(c1, c0, sizeof(double) * 2 * blk);
        elem_acts(s, group, actions + (size_t)t * s->n_act, ae);
        for (int k = 0; k < S; k++) st |= fem_substep(s, tets, dminv, vol, inv_mass, c1, c1 + blk, ae);
    }
    for (int i = 0; i < n3; i++) {
        xb0[i] = xbT ? xbT[i] : 0.0;
        vb0[i] = vbT ? vbT[i] : 0.0;
    }
    memset(ag, 0, sizeof(double) * (size_t)T * s->n_act);
    for (int t = T - 1; t >= 0; t--) {
        const double* a = actions + (size_t)t * s->n_act;
        double* agt = ag + (size_t)t * s->n_act;
        /* reward of step t on its end state */
        if (rbar && s->reward_kind == FEM_REWARD_JUMP && rbar[t] != 0.0) {
            int ns = s->n_sub < s->n_v ? s->n_sub : s->n_v;
            for (int i = 0; i < ns; i++) {
                vb0[3 * i] += rbar[t] / ns;
                xb0[3 * i + 2] += rbar[t] * s->rparam[1] / ns;
            }
            for (int j = 0; j < s->n_act; j++) agt[j] += rbar[t] * (-2.0 * s->rparam[2] * a[j]);
        }
        /* recompute the step's substep states */
        elem_acts(s, group, a, ae);
        memcpy(ring, ck + 2 * blk * (size_t)t, sizeof(double) * 2 * blk);
        for (int k = 0; k < S - 1; k++) {
            double* r0 = ring + 2 * blk * (size_t)k;
            double* r1 = r0 + 2 * blk;
            memcpy(r1, r0, sizeof(double) * 2 * blk);
            fem_substep(s, tets, dminv, vol, inv_mass, r1, r1 + blk, ae);
        }
        memset(abe, 0, sizeof(double) * (size_t)s->n_t);
        for (int k = S - 1; k >= 0; k--) {
            double* r = ring + 2 * blk * (size_t)k;
            fem_substep_adj(s, tets, dminv, vol, inv_mass, r, r + blk, ae, xb0, vb0, abe);
        }
        for (int e = 0; e < s->n_t; e++) agt[group[e]] += s->act_scale * abe[e];
    }
    free(ck);
    free(ring);
    free(ae);
    free(abe);
    return st;
}
