// mpm_types.h -- device-visible descriptors of the environment arena.
//
// Every kernel runs over a list of work items that may span many environments; each
// item names its environment, whose descriptor gives its parameters and the addresses of
// its buffers.  The buffers of one environment:
//   slots   n_slots state blocks, block s at slots + s*block: 24 float components of
//           n_pad particles each (x0..2, v0..2, C00..C22, H00..H22 with H = F - I), then n_pad u32 meta
//           words (caller particle id in bits 0..19, actuator group + 1 in bits 20..31)
//   ring    S-1 blocks of the same layout: substep states recomputed in reverse mode
//   keep    keep_n slots of S-1 blocks each: the substep states of the last keep_n recorded
//           control steps, written by the forward pass (step t in slot t mod keep_n), so the
//           reverse pass reads them instead of recomputing (none when keep_n == 0)
//   adj     two 24-component adjoint blocks (no meta)
//   perm    per slot, the binning permutation computed at that slot's step start
//   grid_*  G^3 float4 nodes each, node (ix, iy, iz) at (iz*G + iy)*G + ix
//   tile    (G/4)^3 activity flags, one per 4^3-node tile
//   pose    per slot, kPose floats: collider pose (c, theta) per body; act per slot, the step's actions
//   acc     per-env accumulators of the reverse pass
//   ctr     per-env step counters (EnvCtr)
#pragma once
#include <stdint.h>

namespace mpm {

constexpr int kComp = 24;  // float components of a particle state
constexpr int kMaxAct = 256;

struct EnvCtr {
  int live;   // slot holding the current state
  int next;   // slot the running control step writes
  int base;   // slot of the first recorded step's start state
  int rev;    // reverse pass: index t of the step being reversed
  int par;    // reverse pass: adj[par] holds the running adjoint
  int status; // status bits (1 domain, 2 NaN, 4 inverted)
  int t;      // control steps taken since the state was set
  int pad;
};

// Pose vector: 4 entries (c, theta) per rigid body; the multi-capsule collider has up to
// kMaxCaps bodies.  Every slot stores kPose floats.
constexpr int kMaxCaps = 8;
constexpr int kPose = 4 * kMaxCaps;

// Accumulator layout (floats) inside EnvDesc::acc.
enum {
  ACC_U = 0,                 // pose velocity of the running step (kPose)
  ACC_QB = kPose,            // adjoint of the pose at the running step's boundary (kPose)
  ACC_QKB = 2 * kPose,       // sum over substeps of dL/dq_k (kPose)
  ACC_KQKB = 3 * kPose,      // sum over substeps of k dt dL/dq_k (kPose)
  ACC_UB = 4 * kPose,        // dL/du through the body velocity (kPose)
  ACC_RSTAT = 5 * kPose,     // reward statistics of the running step (4)
  ACC_VSUM = 5 * kPose + 4,  // reverse pass: two sums (by substep parity) over the env's particles
                             // of the particle-velocity adjoint v-bar + dt x-bar; their mean is the
                             // reference subtracted before the G2P^T scatter and restored node by
                             // node (2 x 4)
  ACC_ACT = 5 * kPose + 12,  // dL/d(action) accumulated in the reverse step (A)
};

struct EnvDesc {
  // geometry and integration
  int n, n_pad, G, S, bound;
  int n_slots;
  int material, coll_kind, n_coll_act, n_groups, reward_kind, n_sub, A;
  int act_map[4];
  float dt, dx, inv_dx, p_mass, p_vol;
  float gravity[3];
  float mu, lam, cyl, bulk, visc, act_stress;
  float coll_dims[4], coll_mu, alpha, act_scale[4], ground_mu;
  int n_caps;           // multi-capsule collider: capsules (pose entries 4 * n_caps), else 0
  float cap_offset[3];  // initial position of capsule j: pose0 + j * cap_offset
  float rparam[4];
  // material FEM: elements (vertex indices, Dm^-1 row-major, rest volume, action index),
  // inverse lumped vertex masses, and the law's constants
  const int4* fem_tet;
  const float* fem_dminv;
  const float* fem_vol;
  const int* fem_group;
  const float* fem_inv_mass;
  // incidence lists (CSR): vertex i's element corners (4 el + c) at vinc[vinc_off[i] ..
  // vinc_off[i+1]), action group g's elements at ginc[ginc_off[g] .. ginc_off[g+1]), in
  // increasing order, so the sums over them are deterministic
  const int* fem_vinc_off;
  const int* fem_vinc;
  const int* fem_ginc_off;
  const int* fem_ginc;
  int n_tets;
  float k_damp, ground_z, fem_alpha;
  // buffers
  float* slots;
  long long block;  // floats per state block = 25 * n_pad
  float* ring;
  float* adj0;
  float* adj1;
  unsigned* perm;
  float4* grid_mp;
  float4* grid_v;
  float4* grid_vb;
  float4* grid_mpb;
  unsigned* tile;
  float* pose;
  float* act;
  float* acc;
  EnvCtr* ctr;
  // Optional per-environment horizon arrays (a served request carries its whole rollout on
  // the device); NULL = the batch-wide buffers passed to the launch.
  const float* act_env;   // [T][A] actions
  float* rew_env;         // [T] rewards
  const float* rbar_env;  // [T] reward adjoints
  float* agrad_env;       // [T][A] action gradients
  long long poff;     // offset of this env's particles in the batch's global index space
  unsigned key_env;   // environment index placed in the high bits of the binning key
  int keep_n;         // recorded control steps whose substep states are kept (0: none)
  float* keep;        // keep_n * (S - 1) blocks, or NULL
};

constexpr int kMatFem = 4;  // material id of tetrahedral-FEM environments

// Pose entries of an environment: 4 per rigid body.
__host__ __device__ inline int pose_len(const EnvDesc& e) { return e.coll_kind == 4 ? 4 * e.n_caps : 4; }

struct WorkItem {
  int env;
  int start;
  int count;
  int pad;
};

// Which state block a launch reads or writes.
enum : int {
  REF_LIVE = 0,  // ctr.live
  REF_NEXT = 1,  // ctr.next
  REF_REV = 2,   // ctr.base + ctr.rev (start of the step being reversed)
  REF_RING = 3,  // ring block k-1 for substep index k >= 1
  REF_REVEND = 4, // ctr.base + ctr.rev + 1 (end of the step being reversed)
  REF_FWDK = 5,   // the state after k substeps of the control step being recorded: ctr.live
                  // (k = 0), ctr.next (k = S), else keep slot (t mod keep_n) block k-1 with
                  // t = live - base, or ctr.next in place when no states are kept
  REF_REVK = 6    // the state after k substeps of the step being reversed: the step's start
                  // (k = 0) and end (k = S) checkpoints, else its kept block when the step is
                  // among the last keep_n recorded, or ring block k-1 (recomputed)
};

struct StateRef {
  int kind;
  int k;  // substep index (REF_RING)
};

constexpr unsigned kIdMask = (1u << 20) - 1u;

}  // namespace mpm
