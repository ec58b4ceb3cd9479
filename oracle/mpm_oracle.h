/*
 * mpm_oracle.h -- plain FP64 CPU reference of one batched-MPM environment.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that tests, the package's
 * smoke check and the CPU-baseline leg of the benchmark can check and time the
 * CUDA path against an obviously-correct implementation.  The product library
 * never links, loads or calls it, and it shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (arXiv 2412.12089, App. D.3 "Material point method"):
 *   one MLS-MPM substep = P2G scatter (APIC affine momentum + Kirchhoff stress
 *   impulse, quadratic B-splines) -> grid momentum update (gravity, softened
 *   SDF collider of App. D.3's last paragraph, domain walls) -> G2P gather
 *   (velocity, APIC C, advection, F update, plastic projection).
 *   Materials: the von Mises elastoplastic law and weakly compressible fluid of
 *   App. D.3 (Eqs. for P(F), delta-gamma, the projection), a compressible
 *   neo-Hookean solid and a neo-Hookean solid with an active fibre stress.
 *   The reverse mode is the exact discrete adjoint of the same FP64 algorithm,
 *   hand-derived (the paper differentiates its simulator by the discrete
 *   adjoint method, Sec. 4.1), with gradient checkpointing at control-step
 *   boundaries and recomputation of the substeps in reverse (Sec. 4.1).
 *
 * Conventions: state arrays are particle-major, x[n*3], v[n*3], C[n*9],
 * F[n*9] (3x3 row-major, M[3*i+j] = M_ij).  Particle order is input order.
 * The domain is [0,1]^3, z up, dx = 1/G.  The collider pose is
 * q = (c_x, c_y, c_z, theta) with theta a yaw angle about +z.
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_NEOHOOKEAN = 0, ORC_VONMISES = 1, ORC_FLUID = 2, ORC_MUSCLE = 3 };
enum { ORC_COLL_NONE = 0, ORC_COLL_CAPSULE = 1, ORC_COLL_BOX = 2, ORC_COLL_CONTAINER = 3, ORC_COLL_CAPSULES = 4 };
enum { ORC_MAX_CAPS = 8, ORC_MAX_POSE = 4 * ORC_MAX_CAPS };
enum { ORC_REWARD_NONE = 0, ORC_REWARD_FLAT = 1, ORC_REWARD_REACH = 2, ORC_REWARD_JUMP = 3 };
enum { ORC_ST_DOMAIN = 1, ORC_ST_NAN = 2, ORC_ST_INVERTED = 4 };

typedef struct {
    int G;              /* grid nodes per axis, dx = 1/G */
    int S;              /* substeps per control step; h = S*dt */
    int bound;          /* wall thickness b in nodes */
    int material;       /* ORC_NEOHOOKEAN .. ORC_MUSCLE */
    int coll_kind;      /* ORC_COLL_* */
    int n_coll_act;     /* leading action entries that drive the collider */
    int act_map[4];     /* pose component (0..3) driven by action j */
    int n_groups;       /* muscle actuator groups (actions after the collider's) */
    int reward_kind;    /* ORC_REWARD_* */
    int n_sub;          /* reward subsample: particles 0..n_sub-1 */
    double dt;
    double gravity[3];
    double p_mass, p_vol;
    double mu, lam;             /* Lame parameters */
    double yield_stress, c_y;   /* von Mises: delta-gamma threshold c_y*sigma_y/(2 mu) */
    double bulk, visc;          /* fluid: bulk modulus (lambda of App. D.3), viscosity */
    double act_stress;          /* muscle fibre stress scale */
    double coll_dims[4];        /* capsule: (radius, half-length); box: half extents;
                                   container: (inner half-width, wall, inner half-height) */
    double coll_mu;             /* collider friction mu_b */
    double alpha;               /* contact softness: s = min(exp(-alpha d), 1) */
    double act_scale[4];        /* pose change per unit action per control step */
    double ground_mu;           /* friction of the bottom wall (0: free slip) */
    double rparam[4];           /* reward parameters */
    int n_caps;                 /* ORC_COLL_CAPSULES: capsules (1..8), all of coll_dims; the
                                   pose vector holds 4 entries per capsule, capsule j's four
                                   actions (4j..4j+3) move its (c, theta) by act_scale[0..3] */
    double cap_offset[3];       /* initial position of capsule j: pose0 + j * cap_offset */
} orc_spec;

/* ---- building blocks (exported for the pin tests) ---- */
void   orc_svd3(const double* F, double* U, double* sig, double* V);
void   orc_tau(const orc_spec* s, const double* F, const double* C, double a_g, double* tau);
void   orc_tau_vjp(const orc_spec* s, const double* F, const double* C, double a_g,
                   const double* taub, double* Fb, double* Cb, double* agb);
void   orc_project(const orc_spec* s, const double* Ft, double* Fo);
void   orc_project_vjp(const orc_spec* s, const double* Ft, const double* Fob, double* Ftb);
void   orc_collider(const orc_spec* s, const double* xw, const double* q, const double* u,
                    double* d, double* n, double* H, double* vb);
/* Entries of the pose vector: 4, or 4 per capsule for ORC_COLL_CAPSULES. */
int    orc_pose_len(const orc_spec* s);
void   orc_weights(double fx, double* w, double* dw);

/* P2G into a dense grid g[G^3*4] = (m, p_x, p_y, p_z) per node, node index
 * (iz*G + iy)*G + ix.  The grid is accumulated into (zero it first). */
int    orc_p2g(const orc_spec* s, int n, const double* x, const double* v, const double* C,
               const double* F, const int* group, const double* act, double* g);
/* Grid update: from (m, p) to velocities gv[G^3*3] at pose q (this substep) and
 * pose velocity u. */
void   orc_grid_update(const orc_spec* s, const double* g, const double* q, const double* u,
                       double* gv);
/* G2P: new x, v, C, F from grid velocities (in place). */
int    orc_g2p(const orc_spec* s, int n, double* x, double* v, double* C, double* F,
               const double* gv);

/* One substep in place; returns status bits. */
int    orc_substep(const orc_spec* s, int n, double* x, double* v, double* C, double* F,
                   const int* group, const double* q, const double* u, const double* act);
/* Adjoint of one substep.  (x,v,C,F) is the state at the substep's start.  On entry
 * (xb,vb,Cb,Fb) hold the adjoint of the state at its end; on return the adjoint of the
 * state at its start.  qb, ub (4 each) and actb (A) are accumulated: qb receives
 * dL/dq for the pose used in this substep, ub dL/du through the body velocity. */
int    orc_substep_adj(const orc_spec* s, int n, const double* x, const double* v,
                       const double* C, const double* F, const int* group, const double* q,
                       const double* u, const double* act, double* xb, double* vb,
                       double* Cb, double* Fb, double* qb, double* ub, double* actb);

/* Reward of one control step from its end state, end pose q and action a. */
double orc_reward(const orc_spec* s, int n, const double* x, const double* v,
                  const double* q, const double* a);
/* Accumulates rb * d(reward)/d(x, v, q, a). */
void   orc_reward_adj(const orc_spec* s, int n, const double* x, const double* v,
                      const double* q, const double* a, double rb, double* xb, double* vb,
                      double* qb, double* ab);

/* T control steps of S substeps from (x,v,C,F,q) in place; actions[T*A] with
 * A = n_coll_act + n_groups; rewards[T]. */
int    orc_rollout(const orc_spec* s, int n, double* x, double* v, double* C, double* F,
                   const int* group, double* q, const double* actions, int T, double* rewards);
/* Forward + reverse of orc_rollout.  Checkpoints the state at every control-step
 * boundary and recomputes each step's substeps in reverse.  xbT..FbT: adjoint of the
 * final state (NULL = 0); rbar[T] (NULL = 0).  Outputs: act_grad[T*A]; xb0..Fb0 the
 * adjoint of the initial state; qb0 (4) of the initial pose.  The state arrays are left
 * at the initial state. */
int    orc_rollout_adj(const orc_spec* s, int n, const double* x0, const double* v0,
                       const double* C0, const double* F0, const int* group, const double* q0,
                       const double* actions, int T, const double* xbT, const double* vbT,
                       const double* CbT, const double* FbT, const double* rbar,
                       double* act_grad, double* xb0, double* vb0, double* Cb0, double* Fb0,
                       double* qb0);

/* Observation of a state (App. E task tables): x' of the subsample (particles 0..ns-1),
 * their mean, 4 entries of the action-driven pose components (action order, zero padded)
 * and 3 of the reach target (REACH, else zeros); orc_obs_dim = 3 ns + 10. */
int    orc_obs_dim(const orc_spec* s, int n);
void   orc_observe(const orc_spec* s, int n, const double* x, const double* q, double* obs);
/* orc_rollout_adj plus observation adjoints obs_adj[(T + 1) * orc_obs_dim] (row t: the
 * state before step t; row T: the final state), or NULL. */
int    orc_rollout_adj_obs(const orc_spec* s, int n, const double* x0, const double* v0,
                           const double* C0, const double* F0, const int* group, const double* q0,
                           const double* actions, int T, const double* xbT, const double* vbT,
                           const double* CbT, const double* FbT, const double* rbar,
                           const double* obs_adj, double* act_grad, double* xb0, double* vb0,
                           double* Cb0, double* Fb0, double* qb0);

/* Binning mirror in FP32 (compiled without FMA contraction): per particle, the cell
 * base = floor(x*G - 0.5) per axis as the GPU path computes it, the tile-major key
 * ((tile index)*64 + cell-in-tile) with 4^3-cell tiles, and a stable counting sort. */
void   orc_bin_keys_f32(int n, const float* x, int G, unsigned* keys);
void   orc_stable_sort_u32(int n, const unsigned* keys, unsigned* perm);

#ifdef __cplusplus
}
#endif
#endif
