// engine.h -- internal step machinery shared by the batch context and the server.
//
// A Group is a set of environments advanced together: every stage of a control step is one
// launch (one per material present) over all of the group's particle work items.  The
// batch context (runtime.cu) owns one group; the server (server.cu) keeps one group for
// environments running forward and one for environments running their reverse pass.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"
#include "mpm.h"
#include "mpm_types.h"

namespace mpm {

constexpr int kChunk = 256;  // particles per work item (CTA)
// Largest FEM mesh: the step kernels hold its vertices and per-element corner terms in shared memory.
constexpr int kFemMaxVerts = 1024;
constexpr int kFemMaxElems = 1024;

const char* check_spec(const mpm_env_spec& s);

// Byte offsets of one environment's buffers inside one allocation.
struct EnvLayout {
  int n_slots = 2;
  bool tape = false;
  bool own = false;  // accumulators, counters and horizon arrays live in the allocation
  int T = 0;         // horizon arrays (own only)
  long long n_pad = 0;
  size_t slots = 0, ring = 0, adj = 0, perm = 0, grid = 0, tile = 0, pose = 0, act = 0;
  size_t acc = 0, ctr = 0, act_env = 0, rew_env = 0, rbar_env = 0, agrad_env = 0, xout = 0;
  size_t fem = 0;  // material FEM: element data and inverse masses
  size_t total = 0;
};

EnvLayout env_layout(const mpm_env_spec& s, int n_slots, bool tape, bool own, int T);
// Parameters and buffer addresses of one environment; acc/ctr are taken from the layout when
// it owns them, else from the given pointers.
// The slot pose vector (kPose floats) of a fresh environment: pose0, and for the capsule union
// capsule j at pose0 + j * cap_offset.
void initial_pose(const mpm_env_spec& s, float* q);
void env_fill(EnvDesc& d, const mpm_env_spec& s, const EnvLayout& L, char* base, float* acc, EnvCtr* ctr);
// Material FEM: the element records, Dm^-1 and rest volumes (from the spec's rest positions,
// in double), groups and inverse lumped masses, copied into the environment's buffers
// (synchronous).  Nothing for other materials; cudaErrorInvalidValue for a degenerate element.
cudaError_t fem_upload(const mpm_env_spec& s, const EnvDesc& d);

struct MatGroup {
  int material;
  int item0;               // first item of the material in the group's item list
  std::vector<int> n_gt;   // [k] = items of the material whose env runs more than k substeps
  int sc_box = 512;        // shared-box capacity of its scatter kernels (autotuned)
  int g2p_stage = 1;       // G2P stages x and H by bulk copies (autotuned)
};

struct Group {
  std::vector<EnvDesc> desc;
  std::vector<mpm_env_spec> spec;
  int n_envs = 0, S_max = 1, A_max = 1, cell_bits = 0, key_bits = 0;  // S_max: over MPM envs (0: none)
  long long P = 0, tiles = 0;
  std::vector<WorkItem> items, items_env;
  std::vector<MatGroup> mats;
  int wait_polls = -1;     // G2P's first bounded wait (test-only MPM_TEST_G2P_WAIT_POLLS; < 0: full)
  int grid_blocks = 152 * 8;  // CTAs of the persistent grid update (autotuned); the grid adjoint caps it
  std::vector<int> env_item0, env_nitems;
  // FEM environments (their step kernels run one CTA per environment) and their extents
  std::vector<int> fem_envs;
  int* d_fem = nullptr;
  size_t fem_cap = 0;
  int fem_nv_max = 0, fem_act_max = 0, fem_nt_max = 0;
  EnvDesc* d_desc = nullptr;
  size_t desc_cap = 0;
  WorkItem* d_items = nullptr;
  WorkItem* d_items_env = nullptr;
  size_t items_cap = 0;
  uint2* active = nullptr;
  int* active_n = nullptr;
  long long active_cap = 0;
  SortScratch sort{};
  long long hist_cap = 0;
  // Grid tape: recorded forward steps keep every substep's grid so the reverse pass restores
  // it instead of re-running P2G (recompute and adjoint substeps alike).  The owner sets
  // want_tape, tape_T (recorded steps) and tape_budget (bytes) before group_build.
  bool want_tape = false;
  int tape_T = 0;
  double tape_budget = 0.0;
  GridTape tape{nullptr, nullptr, nullptr, nullptr, 0, 0, 0};  // tape.cap == 0: no tape
  size_t tape_mp_cap = 0, tape_list_cap = 0, tape_slot_cap = 0, tape_cursor_cap = 0;
  // Kept substep states: with a grid tape, the forward pass of a recorded step writes its
  // substep states to slot (t mod keep_n) of every environment's keep buffer instead of
  // running in place, so the reverse pass of the last keep_n recorded steps skips their
  // recompute.
  // The owner sets keep_frac (share of the memory free after the tape, less keep_reserve
  // bytes it allocates later; 0: none); group_build sizes keep_n (at most tape_T;
  // MPM_KEEP_STEPS caps it, for tests).
  double keep_frac = 0.0, keep_reserve = 0.0;
  int keep_n = 0;
  float* keep = nullptr;
  size_t keep_cap = 0;  // floats
  void release();
};

// (Re)build the group's work lists and device scratch for these environments (their
// descriptors' key_env and poff are assigned here).  Keeps scratch that is large enough.
cudaError_t group_build(Group& g, const std::vector<EnvDesc>& descs, const std::vector<mpm_env_spec>& specs);

Launch group_launch(const Group& g, cudaStream_t st);
Launch env_launch(const Group& g, int e, cudaStream_t st);

// One forward control step of every environment of the group (batched launches, or one
// launch per stage per environment when per_env).
void enqueue_forward(Group& g, cudaStream_t st, bool record, const float* act_in, int a_max, float* rew,
                     bool per_env);
// Autotuner, on the group's live state (binned first), `trials` timed launches of each
// choice after one warm-up, keeping the choice with the fastest trial:
//   - per material, P2G with every scatter shape the kernels are built for;
//   - the persistent grid kernels' CTA count (kGridBlockChoices);
//   - per material, G2P with and without the bulk-copy staging of x and H.
// Every trial writes only the grids (cleared again) and the first ring block (G2P, contexts
// with a tape only), so the state is unchanged.  Times (the fastest trial of each choice):
// p2g[m][b] of material group m with shape b, grid[c] with CTA choice c, g2p[m][s] of
// material group m without (s = 0) and with staging.
struct TuneTimes {
  std::vector<std::vector<float>> p2g, g2p;
  std::vector<float> grid;
};
cudaError_t autotune_scatter(Group& g, cudaStream_t st, int trials, TuneTimes* t);
// One reverse control step of every environment (step index from the device counters).
// obs: adjoints of the task observations at the step boundaries, or NULL.
// kept: the step is among the last g.keep_n recorded, whose substep states the forward pass
// kept (every environment of the group is at the same step): no recompute.
void enqueue_reverse(Group& g, cudaStream_t st, const float* rbar, float* agrad, int n_tot, int a_max, bool per_env,
                     const ObsAdj* obs = nullptr, bool kept = false);

}  // namespace mpm
