/*
 * fem_oracle.h -- plain FP64 CPU reference of one tetrahedral-FEM environment.
 *
 * TEST INFRASTRUCTURE ONLY.  Like mpm_oracle.h, this oracle exists so that tests, the
 * package's smoke check and the CPU-baseline leg of the benchmark can check the CUDA path
 * against an obviously-correct implementation.  The product library never links, loads or
 * calls it, and it shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (arXiv 2412.12089, App. D.2 "Finite element method", and the SoftJumper
 * task of App. E):
 *   - tetrahedral elements with deformation gradient F = Ds Dm^-1 (Ds, Dm: edge matrices of
 *     the deformed and rest tetrahedron), rest volume V0 = |det Dm| / 6;
 *   - the stable neo-Hookean energy density of App. D.2,
 *       Psi = mu/2 (I_C - 3) + lam/2 (J - alpha - a)^2 - mu/2 log(I_C + 1),
 *     I_C = tr(F^T F), J = det F, with the per-element activation a entering the volume
 *     term (reading: an activation shifts the element's rest volume ratio) and, unless set,
 *     alpha = 1 + 3 mu / (4 lam), the value that makes F = I stress free;
 *   - a viscous damping stress k_damp dF/dt (reading of App. E's k_damp);
 *   - elastic + damping forces f = -dE/dx with E = sum_e V0 Psi, lumped vertex masses
 *     (rho V0 / 4 from each element), gravity, and a semi-implicit Euler substep
 *     v' = v + dt (f / m + g), x' = x + dt v';
 *   - the ground z = ground_z: a vertex at or below it with v'_z < 0 has v'_z set to 0 and
 *     its tangential velocity scaled by max(0, 1 + mu_g v'_z / |v'_t|) (Coulomb, the same
 *     projection as the MPM grid's ground);
 *   - control steps of S substeps with activations a_e = act_scale * action[group(e)]
 *     held over the step, and App. E's SoftJumper reward
 *       r = mean(v'_x) + c1 (mean(x'_z) - h0) - c2 sum_j action_j^2
 *     over the vertices with index < n_sub (rparam = (h0, c1, c2)).
 * The reverse mode is the exact discrete adjoint of the same FP64 algorithm, with
 * checkpoints at control steps and the substeps recomputed in reverse (Sec. 4.1).
 *
 * Conventions: x[n_v*3], v[n_v*3] vertex-major; 3x3 matrices row-major (M[3i+j] = M_ij);
 * tets[n_t*4] vertex indices; group[n_t] action index of each element.
 */
#ifndef FEM_ORACLE_H
#define FEM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { FEM_REWARD_NONE = 0, FEM_REWARD_JUMP = 3 };
enum { FEM_ST_NAN = 2, FEM_ST_INVERTED = 4 };

typedef struct {
    int n_v, n_t;       /* vertices, tetrahedra */
    int S;              /* substeps per control step */
    int n_act;          /* action entries (activation groups) */
    int reward_kind;    /* FEM_REWARD_* */
    int n_sub;          /* reward subsample: vertices 0..n_sub-1 */
    double dt;
    double gravity[3];
    double mu, lam, alpha;
    double k_damp;
    double act_scale;   /* activation per unit action */
    double ground_z, ground_mu;
    double rparam[4];
} fem_spec;

/* Rest quantities of a mesh: Dm^-1 per element (9), rest volume per element, inverse lumped
 * mass per vertex.  Returns 0, or -1 for a degenerate element. */
int fem_rest(const fem_spec* s, const int* tets, const double* rest_x, double rho, double* dminv, double* vol,
             double* inv_mass);

/* Energy density, first Piola-Kirchhoff stress P = dPsi/dF, and the adjoint of P: for an
 * adjoint Pb of P, Fb = (d^2 Psi / dF^2) : Pb and ab = (dP/da) : Pb. */
double fem_psi(const fem_spec* s, const double* F, double a);
void   fem_stress(const fem_spec* s, const double* F, double a, double* P);
void   fem_stress_vjp(const fem_spec* s, const double* F, double a, const double* Pb, double* Fb, double* ab);

/* Total elastic energy sum_e V0 Psi(F_e, a_e). */
double fem_energy(const fem_spec* s, const int* tets, const double* dminv, const double* vol, const double* x,
                  const double* a_elem);

/* Elastic + damping forces at (x, v) with per-element activations a_elem. */
void fem_forces(const fem_spec* s, const int* tets, const double* dminv, const double* vol, const double* x,
                const double* v, const double* a_elem, double* f);

/* One substep in place; status bits FEM_ST_*. */
int fem_substep(const fem_spec* s, const int* tets, const double* dminv, const double* vol, const double* inv_mass,
                double* x, double* v, const double* a_elem);

/* T control steps; actions[T*n_act]; rewards[T] or NULL.  x, v updated in place. */
int fem_rollout(const fem_spec* s, const int* tets, const int* group, const double* dminv, const double* vol,
                const double* inv_mass, double* x, double* v, const double* actions, int T, double* rewards);

/* Reverse mode of fem_rollout from (x0, v0): adjoints xbT, vbT of the final state (or NULL)
 * and rbar[T] of the rewards (or NULL).  Outputs: ag[T*n_act], xb0, vb0. */
int fem_rollout_adj(const fem_spec* s, const int* tets, const int* group, const double* dminv, const double* vol,
                    const double* inv_mass, const double* x0, const double* v0, const double* actions, int T,
                    const double* xbT, const double* vbT, const double* rbar, double* ag, double* xb0, double* vb0);

#ifdef __cplusplus
}
#endif
#endif
