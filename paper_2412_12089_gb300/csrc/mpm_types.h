// mpm_types.h -- device-visible descriptors of the environment arena.
//
// Every kernel runs over a list of work items that may span many environments; each
// item names its environment, whose descriptor gives its parameters and the addresses of
// its buffers.  The buffers of one environment:
//   slots   n_slots state blocks, block s at slots + s*block: 24 float components of
//           n_pad particles each (x0..2, v0..2, C00..C22, H00..H22 with H = F - I), then n_pad u32 meta
//           words (caller particle id in bits 0..19, actuator group + 1 in bits 20..31)
//   ring    S-1 blocks of the same layout: substep states recomputed in reverse mode
//   adj     two 24-component adjoint blocks (no meta)
//   perm    per slot, the binning permutation computed at that slot's step start
//   grid_*  G^3 float4 nodes each, node (ix, iy, iz) at (iz*G + iy)*G + ix
//   tile    (G/4)^3 activity flags, one per 4^3-node tile
//   pose    per slot, collider pose (c, theta); act per slot, the step's actions
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

// Accumulator layout (floats) inside EnvDesc::acc.
enum {
  ACC_U = 0,      // pose velocity of the running step (4)
  ACC_QB = 4,     // adjoint of the pose at the running step's boundary (4)
  ACC_QKB = 8,    // sum over substeps of dL/dq_k (4)
  ACC_KQKB = 12,  // sum over substeps of k dt dL/dq_k (4)
  ACC_UB = 16,    // dL/du through the body velocity (4)
  ACC_RSTAT = 20, // reward statistics of the running step (4)
  ACC_VSUM = 24,  // reverse pass: two sums (by substep parity) over the env's particles of
                  // the particle-velocity adjoint v-bar + dt x-bar; their mean is the reference
                  // subtracted before the G2P^T scatter and restored node by node (2 x 4)
  ACC_ACT = 32,   // dL/d(action) accumulated in the reverse step (A)
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
  float rparam[4];
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
  int pad_;
};

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
  REF_REVEND = 4 // ctr.base + ctr.rev + 1 (end of the step being reversed)
};

struct StateRef {
  int kind;
  int k;  // substep index (REF_RING)
};

constexpr unsigned kIdMask = (1u << 20) - 1u;

}  // namespace mpm
