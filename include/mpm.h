/*
 * mpm.h -- C ABI of the batched, differentiable MLS-MPM library for GB300 (sm_103a).
 *
 * The library runs the data-parallel hot path of the parallel differentiable
 * multiphysics simulator of arXiv 2412.12089 ("Stabilizing Reinforcement Learning in
 * Differentiable Multiphysics Simulation"): many independent MPM environments of
 * uneven size advance together, one control step (S substeps) per call, forward and in
 * reverse mode, so a first-order policy learner can back-propagate through them.
 *
 *  - One substep is the MLS-MPM P2G -> grid update -> G2P sequence of App. D.3 (the
 *    paper's "CPIC steps 2-4" of MLS-MPM), with the von Mises elastoplastic law and
 *    weakly compressible fluid of App. D.3, a compressible neo-Hookean solid, a
 *    neo-Hookean muscle with an active fibre stress, and App. D.3's softened contact
 *    s = min(exp(-alpha d), 1) against a kinematic collider moved by the actions.
 *  - env.step(a_t) -> (s_{t+1}, r_t) is the paper's transition (Alg. 1); rewards follow
 *    the task definitions of App. E.
 *  - Gradients are the exact discrete adjoint of the FP32 forward pass (Sec. 4.1), with
 *    checkpoints at control-step boundaries and the substeps recomputed in reverse
 *    (Sec. 4.1, gradient checkpointing).  mpm_backward reverses every recorded step;
 *    mpm_backward_begin/_step/_end reverse them one at a time, for consumers whose actions
 *    depend on observations (mpm_observe).
 *  - Environments may also be tetrahedral FEM meshes (App. D.2's stable neo-Hookean
 *    elements, MPM_MAT_FEM), batched, recorded, reversed and served alongside the MPM ones,
 *    and the collider may be a union of independently driven capsules (MPM_COLL_CAPSULES).
 *  - A continuous-batching server (mpm_server_create / mpm_submit / mpm_poll) admits
 *    rollout requests as memory frees up and runs them together.
 *
 * General conventions
 *  - Every call returns an mpm_status; no C++ exception crosses the ABI.  On failure
 *    mpm_last_error() describes the cause.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *    that take a stream are stream-ordered: they enqueue work and return.
 *  - Array arguments are plain pointers.  Unless stated otherwise they may point to
 *    device memory or to host memory (the library copies with cudaMemcpyDefault); the
 *    caller owns them and the library never frees them.  Device memory the library
 *    allocates itself (particle arena, grids, checkpoint tape) belongs to the context
 *    and is released by mpm_destroy.
 *  - Particle arrays cover all environments back to back, in environment order, each
 *    environment's particles in the caller's order: x[P][3], v[P][3], C[P][3][3],
 *    F[P][3][3] (row-major 3x3), P = sum of n_particles.  The library reorders particles
 *    internally (per-cell binning) and always returns arrays in the caller's order.
 *  - The domain is [0,1]^3 with z up; grid spacing dx = 1/grid_res.
 *  - Units are SI.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPM_OK = 0,
    MPM_ERR_INVALID_ARG = 1, /* bad pointer, size or spec field */
    MPM_ERR_OOM = 2,         /* device allocation failed */
    MPM_ERR_CUDA = 3,        /* a CUDA call failed; see mpm_last_error */
    MPM_ERR_NUMERIC = 4,     /* NaN/Inf or an inverted deformation gradient was flagged */
    MPM_ERR_DOMAIN = 5,      /* a particle left the grid (its cell index was clamped) */
    MPM_ERR_TIMEOUT = 6,     /* a bounded wait gave up */
    MPM_NOT_READY = 7,       /* mpm_poll: the request has not finished */
    MPM_ERR_BUDGET = 8,      /* a request can never fit the server's memory budget */
    MPM_ERR_STATE = 9        /* call not valid in the current state (e.g. tape full) */
} mpm_status;

/* Materials (App. D.3).  NEOHOOKEAN: tau = mu (F F^T - I) + lam log(J) I.
 * VONMISES: tau = U (2 mu eps + lam tr(eps) I) U^T, eps = log Sigma, with the von Mises
 * return mapping (threshold c_y * yield_stress / (2 mu); the paper prints c_y = 2).
 * FLUID: tau = bulk J (J - 1) I + visc J (C + C^T); projection F <- J^(1/3) I.
 * MUSCLE: neo-Hookean plus a_g * act_stress * (F e_z)(F e_z)^T for particles in actuator
 * group g (a_g = the group's action). */
enum { MPM_MAT_NEOHOOKEAN = 0, MPM_MAT_VONMISES = 1, MPM_MAT_FLUID = 2, MPM_MAT_MUSCLE = 3,
       MPM_MAT_FEM = 4 /* tetrahedral FEM (App. D.2): the particles are the mesh's vertices */ };

/* Kinematic collider shapes, in the body frame (body pose q = (c_x, c_y, c_z, theta),
 * theta = yaw about +z).  CAPSULE: axis along body x, coll_dims = (radius, half-length).
 * BOX: coll_dims = half extents.  CONTAINER: open-top box, coll_dims = (inner half-width,
 * wall thickness, inner half-height), origin at the cavity centre. */
enum { MPM_COLL_NONE = 0, MPM_COLL_CAPSULE = 1, MPM_COLL_BOX = 2, MPM_COLL_CONTAINER = 3,
       MPM_COLL_CAPSULES = 4 /* union of n_caps capsules of coll_dims, each driven on its own */ };

/* Per-control-step rewards (App. E), on the subsample of the first n_sub particles (in
 * the caller's order).  FLAT: RollingFlat R_d + R_flat, rparam[0] = h_flat.
 * REACH: FluidMove R_d of the collider position to rparam[0..2].
 * JUMP: SoftJumper mean(v_x) + rparam[1] (mean(z) - rparam[0]) - rparam[2] sum(a^2). */
enum { MPM_REWARD_NONE = 0, MPM_REWARD_FLAT = 1, MPM_REWARD_REACH = 2, MPM_REWARD_JUMP = 3 };

typedef struct {
    int32_t n_particles;  /* >= 1, <= 1,048,575 */
    int32_t grid_res;     /* G: multiple of 4, 8..128 */
    int32_t substeps;     /* S >= 1: substeps per control step, h = S * dt */
    int32_t bound;        /* wall thickness in nodes (separating slip walls), >= 0 */
    int32_t material;     /* MPM_MAT_* */
    int32_t collider;     /* MPM_COLL_* */
    int32_t n_coll_act;   /* 0..4 leading action entries that move the collider (4 * n_caps for
                             MPM_COLL_CAPSULES) */
    int32_t act_map[4];   /* pose component (0..3) that action j moves */
    int32_t n_groups;     /* muscle actuator groups; their actions follow the collider's */
    int32_t reward;       /* MPM_REWARD_* */
    int32_t n_sub;        /* reward subsample size */
    float dt;
    float gravity[3];
    float E, nu, rho, p_vol; /* Young's modulus, Poisson ratio, density, particle volume */
    float yield_stress, c_y;
    float bulk, visc, act_stress;
    float coll_dims[4];
    float coll_mu;        /* collider friction mu_b */
    float alpha;          /* contact softness, s = min(exp(-alpha d), 1) */
    float act_scale[4];   /* pose change per unit action per control step */
    float ground_mu;      /* Coulomb friction of the bottom wall (0 = free slip) */
    float rparam[4];
    float pose0[4];       /* initial collider pose */
    int32_t n_caps;       /* MPM_COLL_CAPSULES: 1..8 capsules.  Capsule j starts at pose0 + j *
                             cap_offset (same angle); its actions are 4j..4j+3 (dx, dy, dz,
                             dtheta per control step, scaled by act_scale[0..3]), so n_coll_act
                             = 4 * n_caps and act_map is not used.  Pose inputs and outputs of
                             this API stay 4-wide: poses set capsule 0 (the others follow the
                             offsets), reads return capsule 0, pose gradients sum over capsules
                             (the gradient with respect to pose0).  The union's contact at a
                             node is the nearest capsule's. */
    float cap_offset[3];
    /*
     * MPM_MAT_FEM (App. D.2 and App. E's SoftJumper): the n_particles particles are the vertices
     * of a tetrahedral mesh, simulated by the stable neo-Hookean energy
     *   Psi = mu/2 (I_C - 3) + lam/2 (J - alpha - a)^2 - mu/2 log(I_C + 1),
     * alpha = 1 + 3 mu / (4 lam), (mu, lam) from (E, nu), with a per-element activation
     * a = act_stress * action[fem_group[e]] (n_groups actions), a damping stress k_damp dF/dt,
     * lumped masses rho V0 / 4, gravity, a semi-implicit Euler substep, and the ground z =
     * ground_z (a vertex at or below it moving down stops, with Coulomb friction ground_mu).
     * No grid is used (grid_res only sizes an unused minimum arena; 8 is enough), the collider
     * must be MPM_COLL_NONE, n_particles <= 1024, n_tets <= 1024.  C and F of the state are not used (get_state
     * returns C = 0, F = I).  The mesh arrays are host memory, read during mpm_create (and
     * mpm_submit), not kept.
     */
    int32_t n_tets;
    const int32_t* fem_tets;   /* [n_tets][4] vertex indices */
    const float* fem_rest;     /* [n_particles][3] rest positions */
    const int32_t* fem_group;  /* [n_tets] action index of each element (< n_groups), or NULL */
    float k_damp;
    float ground_z;
} mpm_env_spec;

typedef struct {
    int32_t max_steps;      /* checkpoint tape capacity in control steps (0 = forward only) */
    int32_t per_env_launch; /* 1: launch every stage once per environment (baseline path) */
    int32_t use_graphs;     /* 1: replay control steps as captured CUDA graphs */
    int32_t chunk;          /* particles per CTA work item, 0 = default */
    int32_t device;         /* CUDA device ordinal */
    float grid_tape_fraction; /* share of the device's free memory (after the arena) that the
                                 grid tape may take: recorded steps keep every substep's grid
                                 so the reverse pass need not rebuild it; 0 = 0.5, < 0 = none */
    float keep_fraction;      /* share of the device's free memory after the grid tape (less
                                 this context's staging buffers) that kept substep states may
                                 take: each recorded step writes its substep states there (step
                                 t in slot t mod n, n = the whole steps that fit, at most
                                 max_steps), and the reverse pass of the last n recorded steps
                                 reads them instead of recomputing them from the step's
                                 checkpoint; needs the grid tape; 0 = 0.8, < 0 = none.  Callers
                                 built against the header without this field must zero it. */
} mpm_options;

typedef struct mpm_ctx mpm_ctx;

/*
 * Create a batch of n_envs environments.  Allocates (and owns) the particle arena, one
 * dense grid per environment, the checkpoint tape for opt->max_steps recorded control
 * steps with its recompute ring, and scratch.  The state starts at rest at the origin
 * with collider poses pose0; call mpm_set_state before stepping.
 * Errors: INVALID_ARG for an unusable spec (field named in mpm_last_error), OOM, CUDA.
 * Passage: App. F (the parallel environments of a task share one physics scene and are
 *   stepped together); the spec's fields are App. D.3's material, grid and contact
 *   parameters and App. E's task constants.
 */
mpm_status mpm_create(const mpm_env_spec* specs, int n_envs, const mpm_options* opt, mpm_ctx** out);
/* Release the context and every device buffer it owns (NULL is ignored).
 * Passage: none in the paper (resource management of the C ABI). */
void mpm_destroy(mpm_ctx* ctx);

/* Sizes of a context: environments, particles P, the action width A_max (the largest
 * n_coll_act + n_groups of the batch), control steps recorded since the last reset, and the
 * device bytes held (arena, grids, tape, scratch).  0 for a NULL context.
 * Passage: none in the paper (queries of the C ABI). */
int32_t mpm_n_envs(const mpm_ctx* ctx);
int64_t mpm_n_particles(const mpm_ctx* ctx);
int32_t mpm_action_dim(const mpm_ctx* ctx);
int32_t mpm_tape_length(const mpm_ctx* ctx);
int64_t mpm_device_bytes(const mpm_ctx* ctx);
/* Recorded control steps whose substep states the context keeps (mpm_options.keep_fraction):
 * the reverse pass skips the recompute of the last this many.  0 for a NULL context.
 * Passage: Sec. 4.1 (checkpoints at control-step boundaries, substeps recomputed in reverse);
 *   keeping them instead, where memory allows, is this library's trade of memory for time. */
int32_t mpm_kept_steps(const mpm_ctx* ctx);
/* Text of the last failure of a call on this context ("" if none); owned by the context,
 * valid until its next call.
 * Passage: none in the paper (error reporting of the C ABI). */
const char* mpm_last_error(const mpm_ctx* ctx);

/*
 * Set the particle state (x, v, C, F: layouts above; group: [P] actuator group per
 * particle, -1 = passive, NULL = all passive) and collider poses (pose: [n_envs][4],
 * NULL = keep).  Resets the checkpoint tape.  Any pointer may be host or device memory.
 * Passage: App. D.3 (the MPM particle state: position, velocity, APIC affine matrix C and
 *   deformation gradient F) and Sec. 3 (the environment state s_t an episode starts from).
 */
mpm_status mpm_set_state(mpm_ctx* ctx, const float* x, const float* v, const float* C, const float* F,
                         const int32_t* group, const float* pose, void* stream);
/* Copy the current state out, in the caller's particle order (any pointer may be NULL).
 * Passage: App. D.3 (the particle state) and Sec. 3 (the next state s_{t+1} of a step). */
mpm_status mpm_get_state(mpm_ctx* ctx, float* x, float* v, float* C, float* F, float* pose,
                         void* stream);

#define MPM_STEP_RECORD 1u /* checkpoint the step's start state for mpm_backward */

/*
 * Advance every environment by one control step (S substeps).
 * actions: [n_envs][A_max]; env e reads its first n_coll_act + n_groups entries.  The
 *   collider moves with constant pose velocity act_scale * a / h over the step.
 * reward:  [n_envs] output, or NULL.
 * flags:   MPM_STEP_RECORD to append the step to the tape (STATE if the tape is full);
 *   without it the tape is reset.
 * Passage: Alg. 1 and Sec. 3 (the transition env.step(a_t) -> s_{t+1}, r_t); each substep
 *   is App. D.3's MLS-MPM pass, the rewards are App. E's.
 */
mpm_status mpm_step(mpm_ctx* ctx, const float* actions, float* reward, uint32_t flags, void* stream);

/*
 * Reverse mode over the T = mpm_tape_length recorded steps (Sec. 4.1): each step's
 * substeps are recomputed from its checkpoint, then reversed.
 *  xb, vb, Cb, Fb: adjoint of the current (final) state, [P][3] / [P][3][3], or NULL (0).
 *  reward_adj:     [T][n_envs] adjoint of the rewards returned by the recorded steps, or NULL.
 *  action_grad:    [T][n_envs][A_max] output (entries past an env's action dim are 0).
 *  xb0..Fb0:       adjoint of the state at the start of the tape, or NULL.
 *  pose_grad0:     [n_envs][4] adjoint of the collider pose at the start, or NULL.
 * The tape is kept, so mpm_backward may be called again with other adjoints.
 * Passage: Sec. 4.1 (analytic first-order gradients through the simulator, with gradient
 *   checkpointing at control-step boundaries).
 */
mpm_status mpm_backward(mpm_ctx* ctx, const float* xb, const float* vb, const float* Cb, const float* Fb,
                        const float* reward_adj, float* action_grad, float* xb0, float* vb0, float* Cb0,
                        float* Fb0, float* pose_grad0, void* stream);

/*
 * The same reverse pass one recorded step at a time, for gradient consumers whose actions
 * depend on observations (a closed-loop policy a_t = pi(o_t), Sec. 4 and App. B): the adjoint
 * of step t's action is needed before the adjoint of o_t, which goes into the next (earlier)
 * step.
 *  mpm_backward_begin: xb..Fb as for mpm_backward.  Observation adjoints set earlier with
 *    mpm_set_obs_adjoint are dropped.  MPM_ERR_STATE without recorded steps or while a
 *    step-wise pass is open.
 *  mpm_backward_step: reverses the latest recorded step t not yet reversed (T - 1 first).
 *    reward_adj: [n_envs] adjoint of r_t, or NULL (0).  obs_adj: [n_envs][mpm_obs_dim]
 *    adjoint of the observation of step t's end state (row t + 1 of mpm_set_obs_adjoint's
 *    layout), or NULL (0).  action_grad: [n_envs][A_max] output, the total adjoint of a_t
 *    (everything after it included), or NULL.  step: t, or NULL.  MPM_ERR_STATE when no pass
 *    is open or every step is reversed.
 *  mpm_backward_end: after all T steps.  obs_adj: [n_envs][mpm_obs_dim] adjoint of the
 *    observation of the state at the start of the tape, or NULL.  xb0..pose_grad0 as for
 *    mpm_backward.  Closes the pass.
 * Pointers are device or host; each call copies its inputs before it returns.  mpm_step,
 * mpm_set_state and mpm_reset_tape abandon an open pass; mpm_backward refuses to run during
 * one.  With the same adjoints the results equal mpm_backward's.
 * Passage: Sec. 4.1 and Alg. 1 (the actor's first-order gradient through a closed-loop
 *   rollout).
 */
mpm_status mpm_backward_begin(mpm_ctx* ctx, const float* xb, const float* vb, const float* Cb, const float* Fb,
                              void* stream);
mpm_status mpm_backward_step(mpm_ctx* ctx, const float* reward_adj, const float* obs_adj, float* action_grad,
                             int32_t* step, void* stream);
mpm_status mpm_backward_end(mpm_ctx* ctx, const float* obs_adj, float* xb0, float* vb0, float* Cb0, float* Fb0,
                            float* pose_grad0, void* stream);

/* Forget the recorded steps; the current state stays.
 * Passage: Sec. 4.1 (the checkpoint tape of a rollout). */
mpm_status mpm_reset_tape(mpm_ctx* ctx);

/* Status word masks, per environment. */
#define MPM_FLAG_DOMAIN 0x1u  /* a particle left the grid (its stencil was clamped) */
#define MPM_FLAG_NAN 0x2u     /* NaN or Inf in the state */
#define MPM_FLAG_INVERTED 0x4u /* J = det F <= 0 */
#define MPM_FLAG_WAIT 0x8u    /* a bounded wait on an asynchronous copy gave up; that chunk's work was skipped */

/*
 * Synchronise and read the per-environment status words (an OR of the MPM_FLAG_* masks),
 * accumulated since the last call, which clears them.
 * flags: [n_envs] host array or NULL.  Returns TIMEOUT (MPM_FLAG_WAIT), NUMERIC (MPM_FLAG_NAN
 * or MPM_FLAG_INVERTED) or DOMAIN (MPM_FLAG_DOMAIN) if a mask is set, in that order.
 * Passage: none in the paper (failure reporting of the C ABI).
 */
mpm_status mpm_check_status(mpm_ctx* ctx, int32_t* flags);

/*
 * Per-cell binning as the hot path uses it, exposed for bit-exact checks.  x: device
 * [n][3] positions.  keys[i] = tile-major cell key of particle i: with the cell base
 * b = clamp(floor(x * G - 0.5), 0, G - 3) per axis (x*G and -0.5 each rounded to
 * nearest), key = ((bz/4 * G/4 + by/4) * G/4 + bx/4) * 64 + (bz%4)*16 + (by%4)*4 + bx%4.
 * perm: the stable sort of keys (perm[j] = index of the j-th smallest key, ties in index
 * order).  keys, perm: device [n].  Uses a device scratch it allocates and frees.
 * Passage: App. D.3 (MLS-MPM's quadratic B-spline stencil of the cell base); the sort is
 *   the binning scheme of this library, with no counterpart in the paper.
 */
mpm_status mpm_bin(const float* x, int32_t n, int32_t grid_res, uint32_t* keys, uint32_t* perm, void* stream);

/*
 * mpm_bin without any allocation.  Passage: none; the paper has no counterpart (a systems
 * entry point).
 * Same arguments, keys and perm as mpm_bin, bit for bit, but the sort scratch is a fixed
 * file-scope device array sized for mpm_bin_static_max() = 262144 particles (4 MiB + 64 KiB),
 * so it calls no cudaMalloc, cudaFree or allocating library routine.  It is for external
 * callers that cannot allocate device memory: a loop that keeps other streams busy, where a
 * cudaFree would synchronise the whole device and stall them, and a process that has
 * committed the device's memory to resident work, where a cudaMalloc can fail in the middle
 * of a run.  (This library's own server keeps a sort scratch of its own and does not call it.)
 *   n > mpm_bin_static_max(): MPM_ERR_INVALID_ARG, nothing launched.  Other argument errors
 *   as mpm_bin.  The work is enqueued on `stream` and the call returns without waiting.
 *   A CUDA error already pending on the calling thread when the call starts: MPM_ERR_CUDA,
 *   nothing launched, the pending error left in place for its owner.  A failed launch of
 *   this call: MPM_ERR_CUDA, and that error is consumed.
 *   The first call on a device, with that device current, looks up the array's device
 *   address (cudaGetSymbolAddress) and keeps it for the process; make that first call
 *   before any stream capture.  cudaDeviceReset on that device unloads the array and makes
 *   the kept address stale: do not call mpm_bin_static on a device after resetting it.
 *   Every call shares the one array: calls whose work overlaps on the GPU (other streams,
 *   unordered threads) race and give wrong keys and perm.  Nothing in the array needs to
 *   start at zero, so stale contents of an earlier call do not matter.
 */
mpm_status mpm_bin_static(const float* x, int32_t n, int32_t grid_res, uint32_t* keys, uint32_t* perm, void* stream);
int32_t mpm_bin_static_max(void);

/*
 * Task observation of every environment's current state, as App. E's task tables define it
 * for the MPM tasks: the positions x' of the subsampled particles (the caller's particles
 * 0..ns-1, ns = min(n_sub, n)), their mean (the CoM of the subsample), the pose components
 * the actions drive (action order) and the reach target p* (REACH reward).
 *   obs: device [n_envs][mpm_obs_dim(ctx)], one row per env laid out as
 *        [x' (3 * ns_max, zero padded past ns)][mean (3)][pose (4, zero padded)][p* (3)],
 *        ns_max = the largest ns of the batch, so mpm_obs_dim = 3 * ns_max + 10.
 *   Stream-ordered; the context's live state is read, nothing changed.
 * Passage: App. E (the observation spaces of the MPM tasks).
 */
int32_t mpm_obs_dim(const mpm_ctx* ctx);
mpm_status mpm_observe(mpm_ctx* ctx, float* obs, void* stream);
/*
 * Adjoints of the observations of the recorded states, for the next mpm_backward (which
 * consumes them): obs_adj, device or host, [T + 1][n_envs][mpm_obs_dim] with T the tape
 * length (row t: the state before recorded step t; row T: the current state).  Copied
 * before the call returns.  NULL forgets adjoints set earlier.  MPM_ERR_STATE without a
 * tape (max_steps = 0).
 * Passage: Sec. 4.1 and App. E (gradients through the observations a policy reads).
 */
mpm_status mpm_set_obs_adjoint(mpm_ctx* ctx, const float* obs_adj, void* stream);

/*
 * Autotuner for the scatter kernels (P2G and its adjoint's scatter half; the batching
 * scheme these shapes belong to has no counterpart in the paper).  On the context's
 * current state, times P2G of every material present with each scatter shape the kernels
 * are built for, `trials` timed launches each after one warm-up, and keeps the fastest per
 * material for every later step (captured graphs are dropped and captured again).  The
 * choices are also kept for the process, per (material, grid resolution, particles per cell
 * rounded to a power of two) and, for the grid kernels, as one CTA count: every context and
 * server group built later starts from them.  The
 * shapes, named by the cell capacity of their per-CTA counting sort: 512 and 1024 cells for
 * 256-particle CTAs of four warps, 256 cells for 64-particle CTAs of one warp.  It then tunes the grid kernels
 * and G2P (mpm_autotune_config).  The state is not changed.  Call it after mpm_set_state,
 * between steps.
 *   box_out: [4] host, chosen capacity by material (MPM_MAT_*), 0 for absent materials;
 *   ms_out:  [4][3] host, fastest trial's P2G time (ms) per material with 512, 1024 and 256 cells;
 *   either may be NULL.  trials in [1, 1000], else MPM_ERR_INVALID_ARG.  Synchronises.
 * Passage: none in the paper (launch-shape tuning of this library).
 */
mpm_status mpm_autotune(mpm_ctx* ctx, int32_t trials, int32_t* box_out, float* ms_out);
/*
 * The rest of what mpm_autotune chose, after the scatter shape and with the same trials (each
 * trial writes only the grids and, for G2P, the first block of the checkpoint tape's substep
 * ring, which is scratch between reverse passes; without a tape G2P keeps the default):
 *   grid_blocks: CTAs of the persistent grid-update kernel, the fastest grid update of 304,
 *     608, 1216 and 2432 CTAs (2, 4, 8, 16 per SM); the grid adjoint launches as many, or
 *     as many as fit on the device at once if fewer; grid_ms: [4] their fastest trials'
 *     times (ms);
 *   g2p_stage: [4] by material, 1 if G2P stages each chunk's x and H in shared memory by
 *     bulk copies, 0 if it loads them directly (-1 for absent materials); g2p_ms: [4][2]
 *     fastest trial's G2P time (ms) without and with the staging.
 * Before any mpm_autotune: the defaults (1216 CTAs, staging on) and zero times.  Any output
 * may be NULL.
 * Passage: none in the paper (launch-shape tuning of this library).
 */
mpm_status mpm_autotune_config(const mpm_ctx* ctx, int32_t* grid_blocks, float* grid_ms, int32_t* g2p_stage,
                               float* g2p_ms);

/* ------------------------------------------------------------------ instrumentation */

/* Kernel classes for mpm_time_kernel. */
enum { MPM_K_P2G = 1, MPM_K_GRID = 2, MPM_K_G2P = 3, MPM_K_G2P_ADJ = 4, MPM_K_GRID_ADJ = 5, MPM_K_P2G_ADJ = 6,
       MPM_K_BIN = 7, MPM_K_OTHER = 8 };

/* Number of CUDA kernels this context has launched (a replayed graph counts its kernels).
 * Passage: none in the paper (instrumentation). */
int64_t mpm_kernel_launches(const mpm_ctx* ctx);
/* Time every launch of one kernel class (MPM_K_*), or of every class (-1), with CUDA events
 * recorded on the launching stream; 0 = off.  While on, the context launches its kernels
 * directly instead of replaying graphs.  Passage: none in the paper (instrumentation). */
mpm_status mpm_time_kernel(mpm_ctx* ctx, int32_t kernel_class);
/* Synchronise and return the summed duration (ms) and count of the timed launches since the
 * last call, which resets them.  One class timed: total_ms[0], launches[0].  All classes
 * timed: total_ms[k], launches[k] for k = 0..MPM_K_OTHER (arrays of MPM_K_OTHER + 1).
 * Passage: none in the paper (instrumentation). */
mpm_status mpm_kernel_time(mpm_ctx* ctx, double* total_ms, int64_t* launches);
/* Synchronise and return the number of active 4^3 grid tiles of the last substep.
 * Passage: none in the paper (instrumentation). */
int32_t mpm_last_active_tiles(mpm_ctx* ctx);

/* ------------------------------------------------------------------ serving */

typedef struct mpm_server mpm_server;

typedef struct {
    double mem_fraction;   /* admission budget as a fraction of device memory, e.g. 0.8 */
    int32_t max_resident;  /* maximum environments resident at once (slots) */
    int32_t device;
    int32_t chunk;         /* particles per CTA work item, 0 = default */
} mpm_server_options;

typedef struct {
    mpm_env_spec spec;
    const float* x;        /* host [n][3] ... as in mpm_set_state */
    const float* v;
    const float* C;
    const float* F;
    const int32_t* group;  /* host [n] or NULL */
    int32_t horizon;       /* control steps, >= 1 */
    const float* actions;  /* host [horizon][A], A = n_coll_act + n_groups */
    int32_t want_grad;     /* 1: also run the reverse pass after the rollout */
    const float* reward_adj; /* host [horizon] adjoint of the rewards (NULL = all ones) */
} mpm_request;

typedef struct {
    int32_t status;          /* mpm_status of the request */
    int32_t horizon, action_dim, n_particles;
    const float* rewards;    /* [horizon] */
    const float* action_grad;/* [horizon][action_dim], NULL without want_grad */
    const float* x_final;    /* [n][3], the caller's particle order */
    double submit_ms, admit_ms, finish_ms; /* host clock, ms since server creation */
} mpm_result;

/*
 * A continuous-batching server: requests are admitted while resident environments are
 * running, as slots and memory free up (admission by memory budget), and all resident
 * environments advance together, one control step per tick, forward and reverse on two
 * streams.  Results stay library-owned until mpm_release.
 * Passage: none in the paper, which runs a fixed batch of parallel environments (App. F);
 *   request serving is a systems layer of this library.  Each request's rollout is the
 *   transition of Alg. 1 repeated, its gradient the reverse pass of Sec. 4.1.
 */
mpm_status mpm_server_create(const mpm_server_options* opt, mpm_server** out);
/* Stop the server and free everything it holds, outstanding results included.
 * Passage: none in the paper (systems call). */
void mpm_server_destroy(mpm_server* srv);
/* Copies the request's host arrays; returns at once with a ticket.  BUDGET if the
 * request alone can never fit the budget.
 * Passage: none in the paper (systems call); the request is one rollout of Alg. 1's
 *   env.step over its horizon, with Sec. 4.1's reverse pass when want_grad is set. */
mpm_status mpm_submit(mpm_server* srv, const mpm_request* req, uint64_t* ticket);
/* Non-blocking: NOT_READY, or OK with *out filled.
 * Passage: none in the paper (systems call). */
mpm_status mpm_poll(mpm_server* srv, uint64_t ticket, mpm_result* out);
/* Block until the ticket finishes or timeout_ms passes (TIMEOUT).
 * Passage: none in the paper (systems call). */
mpm_status mpm_wait(mpm_server* srv, uint64_t ticket, double timeout_ms, mpm_result* out);
/* Free a finished ticket's result buffers.  Passage: none in the paper (systems call). */
mpm_status mpm_release(mpm_server* srv, uint64_t ticket);
/* Text of the server's last failure.  Passage: none in the paper (systems call). */
const char* mpm_server_last_error(const mpm_server* srv);

#ifdef __cplusplus
}
#endif
#endif
