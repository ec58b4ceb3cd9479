// kernels.h -- host-side launchers of the batched MPM kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>

#include "mpm_types.h"

namespace mpm {

// Kernel classes (for launch counting and per-class event timing).
enum KernelClass {
  KC_P2G = 1, KC_GRID = 2, KC_G2P = 3, KC_G2P_ADJ = 4, KC_GRID_ADJ = 5, KC_P2G_ADJ = 6, KC_BIN = 7, KC_OTHER = 8
};

// Every launcher below adds the number of kernels it enqueued to this counter.
long long kernel_launch_count();
void count_launches(int n);

// Optional timing hook: when set, launchers of class kc record start/stop events around the
// launch on its stream (direct launches only; no effect inside graph capture).
struct TimingHook {
  int kc = 0;  // class to time, -1 = every class
  void (*before)(void* user, int kc, cudaStream_t st) = nullptr;
  void (*after)(void* user, int kc, cudaStream_t st) = nullptr;
  void* user = nullptr;
};
void set_timing_hook(const TimingHook* h);

struct Launch {
  const EnvDesc* envs;   // device array
  const WorkItem* items; // device array of particle work items
  int material = 0;      // material of every item in [item_offset, item_offset + n_items)
  int n_items;
  int item_offset;       // first item (per-environment launches)
  uint2* active;         // active-tile list (env, tile)
  int* active_n;         // its length (device)
  int grid_blocks;       // CTAs of the persistent grid update (the grid adjoint caps it at one resident wave)
  int env0, n_env;       // environment range of the per-env kernels
  cudaStream_t stream;
  int sc_box = 512;      // scatter shape by the cell capacity of its counting sort: 512 or 1024
                         // (256-particle CTAs of four warps) or 256 (64-particle CTAs of one warp)
  int wait_polls = -1;   // polls of G2P's first wait on its staged copies (< 0: the full limit)
  int g2p_stage = 1;     // G2P stages a chunk's x and H by bulk copies (when read in place)
};

constexpr int kGridBlockChoices[4] = {152 * 2, 152 * 4, 152 * 8, 152 * 16};  // persistent grid CTAs

constexpr int kNScatterBoxes = 3;
constexpr int kScatterBoxes[kNScatterBoxes] = {512, 1024, 256};  // shapes the scatter kernels are built for

enum GridMode { GRID_FWD = 0, GRID_KEEP = 1 };

// Grid tape: recorded forward steps keep every substep's grid, (m, p) of the 64 nodes of
// each active tile in active-list order plus the list entries, in one pool; the reverse pass
// restores them instead of re-running P2G.  slot[t * S + k] = (first tile, tiles) of
// substep k of recorded step t, tiles = -1 when the pool was full (P2G rebuilds that grid).
struct GridTape {
  float4* mp;                  // pool, 64 nodes per tile
  uint2* list;                 // pool, the tiles' active-list entries
  int2* slot;                  // [T * S]
  unsigned long long* cursor;  // tiles taken by the recorded steps so far
  long long cap;               // pool tiles
  int T, S;
};

// skip_kept: in the reverse pass, skip every CTA when the tape kept substep k of the step
// being reversed; NULL = run.
void launch_p2g(const Launch& L, StateRef src, bool use_perm, int k, const GridTape* skip_kept = nullptr);
// record: also copy the active tiles' (m, p) into the tape slot of (recorded step, k), which
// launch_tape_alloc reserved.
void launch_grid(const Launch& L, int k, GridMode mode, bool rev, const GridTape* record = nullptr);
// Reserve the pool range of substep k of the recorded step (the active list's length).
void launch_tape_alloc(const Launch& L, const GridTape& tape, int k);
// Write substep k of the step being reversed back into the dense grids and make its tiles
// the active list (nothing when the slot was not kept).
void launch_restore(const Launch& L, const GridTape& tape, int k);
void launch_g2p(const Launch& L, StateRef src, StateRef dst, bool use_perm, int k);

void launch_step_begin(const Launch& L, const float* act_in, int a_max, bool record);
void launch_reward_end(const Launch& L, float* reward_out, bool record);

// nxt: the substep's end state (v', C' written by the forward G2P)
void launch_g2p_adj(const Launch& L, StateRef src, StateRef nxt, bool use_perm, int k);
void launch_grid_adj(const Launch& L, int k);
void launch_p2g_adj(const Launch& L, StateRef src, bool use_perm, int k);
// Reverse pass bookkeeping.  bwd_init sets the step index to T; each rev_begin decrements
// it, so one captured reverse-step graph serves every step.  rbar: [T][n_tot] reward
// adjoints (or NULL); act_grad: [T][n_tot][a_max] output.
void launch_bwd_init(const Launch& L, int T);
void launch_rev_begin(const Launch& L);
void launch_reward_adj(const Launch& L, const float* rbar, int n_tot);
void launch_adj_ref(const Launch& L);
void launch_rev_end(const Launch& L, float* act_grad, int n_tot, int a_max);

// Task observations (App. E): per env row [x' of caller particles 0..ns-1 (3 nsub_max,
// zero padded)][their mean 3][action-driven pose components 4][reach target 3].
struct ObsAdj {
  const float* adj;  // [T + 1][n_tot][dim] adjoints of the observations at the step boundaries
  const int* on;     // device flag: inject only when set
  int dim, nsub_max, n_tot;
};
void launch_observe(const Launch& L, float* obs, int dim, int nsub_max);
// which = 0: the end state of the step being reversed (row rev + 1); 1: the state before it
// (row rev; used once after the last reverse step, for the initial state).
void launch_obs_adj(const Launch& L, const ObsAdj& o, int which);

// State I/O: caller order (AoS) <-> arena blocks.
void launch_set_state(const Launch& L, const float* x, const float* v, const float* C, const float* F,
                      const int* group);
void launch_get_state(const Launch& L, StateRef src, float* x, float* v, float* C, float* F);
// The caller's pose ([n_envs][4], indexed by global env) <-> the slot pose vectors:
// POSE_SET buf -> slot 0 (capsule j offset by j * cap_offset), POSE_KEEP slot -> slot 0,
// POSE_GET slot body 0 -> buf, POSE_GRAD pose adjoint (summed over capsules) -> buf.
enum PoseIo { POSE_SET = 0, POSE_KEEP = 1, POSE_GET = 2, POSE_GRAD = 3 };
void launch_pose_io(const Launch& L, PoseIo mode, float* buf, int slot);
void launch_adj_in(const Launch& L, const float* xb, const float* vb, const float* Cb, const float* Fb);
void launch_adj_out(const Launch& L, StateRef src, float* xb, float* vb, float* Cb, float* Fb);

// Tetrahedral-FEM environments (material FEM): one CTA per environment listed in `list`
// (device, n entries) runs the whole control step (forward) or its reverse.  nv_max: the
// largest vertex count of the listed environments; act_max, nt_max: their largest action and
// element counts.
void launch_fem_forward(const Launch& L, const int* list, int n, int nv_max, int nt_max);
void launch_fem_reverse(const Launch& L, const int* list, int n, int nv_max, int act_max, int nt_max);

// Counts one kernel launch of class kc and records the timing hook's events around it (for
// launchers outside kernels.cu).
struct LaunchScope {
  int kc;
  cudaStream_t st;
  LaunchScope(int k, cudaStream_t s);
  ~LaunchScope();
};

// Binning: keys of the live state, LSD radix sort, per-env permutations.
struct SortScratch {
  unsigned* keys[2];
  unsigned* vals[2];
  unsigned* hist;
  long long cap;
  int max_blocks;
};
// Sort the live state of the launch's environments (global indices [poff0, poff0+n_total))
// and store each environment's permutation in perm[live].
void bin_envs(const Launch& L, long long poff0, long long n_total, int cell_bits, int key_bits, SortScratch& s);
// Stable LSD radix sort of (keys, vals) on the low key_bits bits; returns the buffer index
// (0 or 1) holding the result.
// hist: radix_hist_entries(n) counters of scratch.
int radix_sort(unsigned** keys, unsigned** vals, long long n, int key_bits, unsigned* hist, cudaStream_t st);
long long radix_hist_entries(long long n);
void launch_bin_keys_plain(const float* x, int n, int G, unsigned* keys, unsigned* vals, cudaStream_t st);

}  // namespace mpm
