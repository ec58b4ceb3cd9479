// runtime.cu -- batch context of the MPM library: arena, control-step orchestration,
// checkpoint tape and reverse pass, CUDA-graph replay, and the C ABI of include/mpm.h.
//
// A control step (the paper's env.step, Alg. 1) = bin the live state, then S substeps of
// P2G -> grid -> G2P for all environments (one launch per stage), then rewards.  With
// MPM_STEP_RECORD the step's start state stays in the tape; the reverse pass restores
// each checkpoint, recomputes the step's substeps into a ring and runs the adjoint
// kernels backwards (Sec. 4.1, gradient checkpointing).  Every per-step quantity the
// kernels need comes from device-resident counters, so a captured control-step graph
// (and a reverse-step graph) is replayed unchanged at every step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mpm.h"
#include "kernels.h"
#include "mpm_types.h"

using namespace mpm;

namespace {

constexpr int kChunkDefault = 256;  // particles per work item (CTA)

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int bits_for(unsigned long long v) {  // bits needed to hold values 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0ull) ++b;
  return b;
}

}  // namespace

struct mpm_ctx {
  int device = 0;
  int n_envs = 0;
  long long P = 0;
  int A_max = 1;
  int T_cap = 0;
  int n_slots = 2;
  int S_max = 1;
  int chunk = kChunkDefault;
  bool per_env = false;
  bool use_graphs = false;
  std::vector<mpm_env_spec> specs;
  std::vector<EnvDesc> desc;
  EnvDesc* d_desc = nullptr;
  std::vector<WorkItem> items;            // grouped by material, then by substep count descending
  WorkItem* d_items = nullptr;
  struct MatGroup {
    int material;
    int item0;               // first item of the group
    std::vector<int> n_gt;   // [k] = items of the group whose env has S > k
  };
  std::vector<MatGroup> groups;
  std::vector<int> env_item0, env_nitems; // per-env item ranges (per-env launches)
  std::vector<WorkItem> items_env_order;  // items grouped by env (per-env launches)
  WorkItem* d_items_env = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  uint2* active = nullptr;
  int* active_n = nullptr;
  long long active_cap = 0;
  SortScratch sort{};
  int cell_bits = 0, key_bits = 0;
  float* act_in = nullptr;   // [n_envs][A_max]
  float* rew = nullptr;      // [n_envs]
  float* rbar = nullptr;     // [T_cap][n_envs]
  float* agrad = nullptr;    // [T_cap][n_envs][A_max]
  float* io = nullptr;       // [P][24] staging
  float* posebuf = nullptr;  // [n_envs][4]
  size_t acc_stride = 0;
  float* acc_all = nullptr;
  EnvCtr* ctr_all = nullptr;
  int h_live = 0, h_base = 0;  // host mirrors of the device counters (identical in all envs)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t g_fwd[2] = {nullptr, nullptr};
  cudaGraphExec_t g_rev = nullptr;
  long long g_fwd_kernels[2] = {0, 0};
  long long g_rev_kernels = 0;
  long long launches = 0;        // kernels this context launched (graph replays included)
  int time_kc = 0;               // kernel class timed with events (0 = none, -1 = all)
  std::vector<cudaEvent_t> ev;   // start/stop pairs of timed launches
  std::vector<int> ev_class;     // class of each pair
  int cur_class = 0;
  size_t ev_used = 0;
  std::string err;
  size_t total_bytes = 0;
};

struct mpm_server;  // defined in server.cu

namespace {

mpm_status fail(mpm_ctx* c, mpm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                            \
  } while (0)

const char* check_spec(const mpm_env_spec& s) {
  if (s.n_particles < 1 || s.n_particles > (int)kIdMask) return "n_particles";
  if (s.grid_res < 8 || s.grid_res > 128 || s.grid_res % 4) return "grid_res";
  if (s.substeps < 1 || s.substeps > 4096) return "substeps";
  if (s.bound < 0 || 2 * s.bound >= s.grid_res) return "bound";
  if (s.material < 0 || s.material > 3) return "material";
  if (s.collider < 0 || s.collider > 3) return "collider";
  if (s.n_coll_act < 0 || s.n_coll_act > 4) return "n_coll_act";
  for (int j = 0; j < s.n_coll_act; ++j)
    if (s.act_map[j] < 0 || s.act_map[j] > 3) return "act_map";
  if (s.n_groups < 0 || s.n_groups > 4094) return "n_groups";
  if (s.n_coll_act + s.n_groups > kMaxAct) return "action dim";
  if (s.reward < 0 || s.reward > 3) return "reward";
  if (s.reward != 0 && s.n_sub < 1) return "n_sub";
  if (!(s.dt > 0.f) || !(s.p_vol > 0.f) || !(s.rho > 0.f)) return "dt/p_vol/rho";
  if (s.reward == 1 && !(s.rparam[0] != 0.f)) return "rparam (h_flat)";
  if ((s.material == 0 || s.material == 1 || s.material == 3) && !(s.E > 0.f && s.nu >= 0.f && s.nu < 0.5f))
    return "E/nu";
  return nullptr;
}

Launch make_launch(mpm_ctx* c, cudaStream_t st) {
  Launch L;
  L.envs = c->d_desc;
  L.items = c->d_items;
  L.n_items = (int)c->items.size();
  L.item_offset = 0;
  L.active = c->active;
  L.active_n = c->active_n;
  L.grid_blocks = 152 * 8;
  L.env0 = 0;
  L.n_env = c->n_envs;
  L.stream = st;
  return L;
}

Launch env_launch(mpm_ctx* c, int e, cudaStream_t st) {
  Launch L = make_launch(c, st);
  L.items = c->d_items_env;
  L.item_offset = c->env_item0[e];
  L.n_items = c->env_nitems[e];
  L.env0 = e;
  L.n_env = 1;
  const int G = c->specs[e].grid_res;
  L.grid_blocks = std::max(1, std::min(152 * 8, (G / 4) * (G / 4) * (G / 4) / 8));
  return L;
}

// ---------------------------------------------------------------- step bodies

// Launch of one material group's items whose env runs more than k substeps.
Launch group_launch(mpm_ctx* c, const Launch& L, const mpm_ctx::MatGroup& g, int k) {
  Launch Lg = L;
  Lg.material = g.material;
  Lg.item_offset = g.item0;
  Lg.n_items = g.n_gt[std::min(k, c->S_max)];
  return Lg;
}

// All substeps of a forward control step, every material group.
void enqueue_substeps_fwd(mpm_ctx* c, Launch L) {
  for (int k = 0; k < c->S_max; ++k) {
    cudaMemsetAsync(c->active_n, 0, sizeof(int), L.stream);
    const StateRef src{k == 0 ? REF_LIVE : REF_NEXT, k};
    const StateRef dst{REF_NEXT, k};
    for (auto& g : c->groups) launch_p2g(group_launch(c, L, g, k), src, k == 0, k);
    launch_grid(L, k, GRID_FWD, false);
    for (auto& g : c->groups) launch_g2p(group_launch(c, L, g, k), src, dst, k == 0, k);
  }
}

void enqueue_forward(mpm_ctx* c, cudaStream_t st, bool record) {
  if (!c->per_env) {
    Launch L = make_launch(c, st);
    launch_step_begin(L, c->act_in, c->A_max, record);
    bin_envs(L, 0, c->P, c->cell_bits, c->key_bits, c->sort);
    enqueue_substeps_fwd(c, L);
    launch_reward_end(L, c->rew, record);
  } else {
    // baseline path: every stage launched once per environment
    for (int e = 0; e < c->n_envs; ++e) {
      Launch L = env_launch(c, e, st);
      L.material = c->specs[e].material;
      launch_step_begin(L, c->act_in, c->A_max, record);
      bin_envs(L, c->desc[e].poff, c->specs[e].n_particles, c->cell_bits, c->cell_bits, c->sort);
      for (int k = 0; k < c->specs[e].substeps; ++k) {
        cudaMemsetAsync(c->active_n, 0, sizeof(int), st);
        const StateRef src{k == 0 ? REF_LIVE : REF_NEXT, k};
        const StateRef dst{REF_NEXT, k};
        launch_p2g(L, src, k == 0, k);
        launch_grid(L, k, GRID_FWD, false);
        launch_g2p(L, src, dst, k == 0, k);
      }
      launch_reward_end(L, c->rew, record);
    }
  }
}

// One reverse control step (the step index comes from the device counters).  groups: the
// material groups to launch (per-environment launches pass a single group).
void enqueue_reverse_step(mpm_ctx* c, Launch L, int S, const std::vector<mpm_ctx::MatGroup>& groups, bool have_rbar) {
  launch_rev_begin(L);
  if (have_rbar) launch_reward_adj(L, c->rbar, c->n_envs);
  launch_adj_ref(L);
  auto gl = [&](const mpm_ctx::MatGroup& g, int k) {
    Launch Lg = L;
    Lg.material = g.material;
    Lg.item_offset = g.item0;
    Lg.n_items = g.n_gt[std::min(k, (int)g.n_gt.size() - 1)];
    return Lg;
  };
  // recompute substep states 1..S-1 into the ring (envs with S > k + 1)
  for (int k = 0; k + 1 < S; ++k) {
    cudaMemsetAsync(c->active_n, 0, sizeof(int), L.stream);
    const StateRef src{k == 0 ? REF_REV : REF_RING, k};
    const StateRef dst{REF_RING, k + 1};
    for (auto& g : groups) {
      Launch Lg = gl(g, k);
      Lg.n_items = g.n_gt[std::min(k + 1, (int)g.n_gt.size() - 1)];
      launch_p2g(Lg, src, k == 0, k);
    }
    launch_grid(L, k, GRID_FWD, true);
    for (auto& g : groups) {
      Launch Lg = gl(g, k);
      Lg.n_items = g.n_gt[std::min(k + 1, (int)g.n_gt.size() - 1)];
      launch_g2p(Lg, src, dst, k == 0, k);
    }
  }
  // adjoint substeps, last to first (envs with S > k)
  for (int k = S - 1; k >= 0; --k) {
    cudaMemsetAsync(c->active_n, 0, sizeof(int), L.stream);
    const StateRef src{k == 0 ? REF_REV : REF_RING, k};
    for (auto& g : groups) launch_p2g(gl(g, k), src, k == 0, k);
    launch_grid(L, k, GRID_KEEP, true);
    // the end state of substep k is ring block k+1 for envs with S > k+1 (a prefix of the
    // group) and the step's end checkpoint for envs whose last substep is k
    for (auto& g : groups) {
      Launch Lg = gl(g, k);
      const int n_ring = g.n_gt[std::min(k + 1, (int)g.n_gt.size() - 1)];
      if (n_ring > 0) {
        Launch La = Lg;
        La.n_items = n_ring;
        launch_g2p_adj(La, src, StateRef{REF_RING, k + 1}, k == 0, k);
      }
      if (Lg.n_items > n_ring) {
        Launch Lb = Lg;
        Lb.item_offset += n_ring;
        Lb.n_items -= n_ring;
        launch_g2p_adj(Lb, src, StateRef{REF_REVEND, 0}, k == 0, k);
      }
    }
    launch_grid_adj(L, k);
    for (auto& g : groups) launch_p2g_adj(gl(g, k), src, k == 0, k);
  }
  launch_rev_end(L, c->agrad, c->n_envs, c->A_max);
}

// Event timing of one kernel class (direct launches).
void ev_before(void* user, int kc, cudaStream_t st) {
  mpm_ctx* c = (mpm_ctx*)user;
  if (c->ev_used + 2 > c->ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      c->ev.push_back(e);
    }
  }
  if (c->ev_class.size() < c->ev.size() / 2) c->ev_class.resize(c->ev.size() / 2);
  c->ev_class[c->ev_used / 2] = kc;
  cudaEventRecord(c->ev[c->ev_used], st);
}
void ev_after(void* user, int kc, cudaStream_t st) {
  (void)kc;
  mpm_ctx* c = (mpm_ctx*)user;
  cudaEventRecord(c->ev[c->ev_used + 1], st);
  c->ev_used += 2;
}

// Launch-counting scope; installs the timing hook while direct launches are enqueued.
struct Enqueue {
  mpm_ctx* c;
  long long start;
  explicit Enqueue(mpm_ctx* ctx) : c(ctx), start(kernel_launch_count()) {
    if (c->time_kc) {
      TimingHook h;
      h.kc = c->time_kc;
      h.before = ev_before;
      h.after = ev_after;
      h.user = c;
      set_timing_hook(&h);
    }
  }
  ~Enqueue() {
    if (c->time_kc) set_timing_hook(nullptr);
    c->launches += kernel_launch_count() - start;
  }
};

mpm_status run_graph_or_direct(mpm_ctx* ctx, cudaGraphExec_t* slot, long long* slot_kernels, cudaStream_t st,
                               void (*body)(mpm_ctx*, cudaStream_t, void*), void* arg) {
  if (!ctx->use_graphs || ctx->per_env || ctx->time_kc) {
    Enqueue q(ctx);
    body(ctx, st, arg);
    CK(cudaGetLastError());
    return MPM_OK;
  }
  if (!*slot) {
    cudaGraph_t g;
    const long long before = kernel_launch_count();
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    body(ctx, ctx->cap_stream, arg);
    CK(cudaStreamEndCapture(ctx->cap_stream, &g));
    CK(cudaGraphInstantiate(slot, g, 0));
    cudaGraphDestroy(g);
    *slot_kernels = kernel_launch_count() - before;
  }
  CK(cudaGraphLaunch(*slot, st));
  ctx->launches += *slot_kernels;
  return MPM_OK;
}

void body_fwd(mpm_ctx* c, cudaStream_t st, void* arg) { enqueue_forward(c, st, *(bool*)arg); }

void body_rev(mpm_ctx* c, cudaStream_t st, void* arg) {
  Launch L = make_launch(c, st);
  enqueue_reverse_step(c, L, c->S_max, c->groups, *(bool*)arg);
}

}  // namespace

// ================================================================== C ABI

extern "C" {

const char* mpm_last_error(const mpm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
int32_t mpm_n_envs(const mpm_ctx* ctx) { return ctx ? ctx->n_envs : 0; }
int64_t mpm_n_particles(const mpm_ctx* ctx) { return ctx ? ctx->P : 0; }
int32_t mpm_action_dim(const mpm_ctx* ctx) { return ctx ? ctx->A_max : 0; }
int32_t mpm_tape_length(const mpm_ctx* ctx) { return ctx ? ctx->h_live - ctx->h_base : 0; }
int64_t mpm_device_bytes(const mpm_ctx* ctx) { return ctx ? (int64_t)ctx->total_bytes : 0; }

mpm_status mpm_create(const mpm_env_spec* specs, int n_envs, const mpm_options* opt, mpm_ctx** out) {
  if (!out) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  mpm_ctx* ctx = new mpm_ctx();
  auto bail = [&](mpm_status s) {
    *out = ctx;  // hand back the context so mpm_last_error works; caller destroys it
    return s;
  };
  if (!specs || n_envs < 1 || n_envs > (1 << 16)) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "n_envs"));
  mpm_options o{};
  if (opt) o = *opt;
  if (o.max_steps < 0 || o.max_steps > 100000) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "max_steps"));
  ctx->device = o.device;
  ctx->T_cap = o.max_steps;
  ctx->n_slots = std::max(o.max_steps + 1, 2);
  ctx->per_env = o.per_env_launch != 0;
  ctx->use_graphs = o.use_graphs != 0;
  ctx->chunk = kChunkDefault;
  if (o.chunk != 0 && o.chunk != kChunkDefault) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "chunk (only 256 is built)"));
  ctx->n_envs = n_envs;
  ctx->specs.assign(specs, specs + n_envs);
  for (int e = 0; e < n_envs; ++e) {
    const char* bad = check_spec(specs[e]);
    if (bad) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "env %d: invalid %s", e, bad));
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return bail(fail(ctx, MPM_ERR_CUDA, "cudaSetDevice(%d)", ctx->device));

  // ---- sizes
  int A_max = 1, S_max = 1, G_max = 8;
  long long P = 0;
  for (auto& s : ctx->specs) {
    A_max = std::max(A_max, s.n_coll_act + s.n_groups);
    S_max = std::max(S_max, s.substeps);
    G_max = std::max(G_max, s.grid_res);
    P += s.n_particles;
  }
  ctx->A_max = A_max;
  ctx->S_max = S_max;
  ctx->P = P;
  const unsigned long long max_cell = (unsigned long long)(G_max / 4) * (G_max / 4) * (G_max / 4) * 64ull - 1ull;
  ctx->cell_bits = bits_for(max_cell);
  ctx->key_bits = ctx->cell_bits + bits_for((unsigned long long)(n_envs - 1));
  if (ctx->key_bits > 32) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "too many environments for a 32-bit binning key"));
  const bool tape = ctx->T_cap > 0;
  ctx->acc_stride = (size_t)ACC_ACT + A_max;

  // ---- per-env layout inside one arena
  ctx->desc.resize(n_envs);
  std::vector<size_t> off_slots(n_envs), off_ring(n_envs), off_adj(n_envs), off_perm(n_envs), off_grid(n_envs),
      off_tile(n_envs), off_pose(n_envs), off_act(n_envs);
  size_t cur = 0;
  long long poff = 0;
  long long tiles_total = 0;
  for (int e = 0; e < n_envs; ++e) {
    const auto& s = ctx->specs[e];
    const long long n_pad = ((long long)s.n_particles + 31) / 32 * 32;
    const long long block = 25 * n_pad;
    const long long G3 = (long long)s.grid_res * s.grid_res * s.grid_res;
    const long long TG3 = (long long)(s.grid_res / 4) * (s.grid_res / 4) * (s.grid_res / 4);
    tiles_total += TG3;
    off_slots[e] = cur; cur = align256(cur + (size_t)ctx->n_slots * block * 4);
    off_ring[e] = cur;  if (tape) cur = align256(cur + (size_t)std::max(s.substeps - 1, 0) * block * 4);
    off_adj[e] = cur;   if (tape) cur = align256(cur + (size_t)2 * kComp * n_pad * 4);
    off_perm[e] = cur;  cur = align256(cur + (size_t)ctx->n_slots * n_pad * 4);
    off_grid[e] = cur;  cur = align256(cur + (size_t)(tape ? 4 : 2) * G3 * 16);
    off_tile[e] = cur;  cur = align256(cur + (size_t)TG3 * 4);
    off_pose[e] = cur;  cur = align256(cur + (size_t)ctx->n_slots * 4 * 4);
    off_act[e] = cur;   cur = align256(cur + (size_t)ctx->n_slots * std::max(1, s.n_coll_act + s.n_groups) * 4);
    EnvDesc& d = ctx->desc[e];
    memset(&d, 0, sizeof d);
    d.n = s.n_particles;
    d.n_pad = (int)n_pad;
    d.G = s.grid_res;
    d.S = s.substeps;
    d.bound = s.bound;
    d.n_slots = ctx->n_slots;
    d.material = s.material;
    d.coll_kind = s.collider;
    d.n_coll_act = s.n_coll_act;
    d.n_groups = s.n_groups;
    d.reward_kind = s.reward;
    d.n_sub = s.n_sub;
    d.A = s.n_coll_act + s.n_groups;
    for (int j = 0; j < 4; ++j) {
      d.act_map[j] = s.act_map[j];
      d.coll_dims[j] = s.coll_dims[j];
      d.act_scale[j] = s.act_scale[j];
      d.rparam[j] = s.rparam[j];
    }
    d.dt = s.dt;
    d.dx = 1.0f / (float)s.grid_res;
    d.inv_dx = (float)s.grid_res;
    d.p_vol = s.p_vol;
    d.p_mass = s.rho * s.p_vol;
    for (int i = 0; i < 3; ++i) d.gravity[i] = s.gravity[i];
    if (s.material == 0 || s.material == 1 || s.material == 3) {
      const double E = s.E, nu = s.nu;
      d.mu = (float)(E / (2.0 * (1.0 + nu)));
      d.lam = (float)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    }
    d.cyl = d.mu > 0.f ? (float)((double)s.c_y * s.yield_stress / (2.0 * d.mu)) : 0.f;
    d.bulk = s.bulk;
    d.visc = s.visc;
    d.act_stress = s.act_stress;
    d.coll_mu = s.coll_mu;
    d.alpha = s.alpha;
    d.ground_mu = s.ground_mu;
    d.block = block;
    d.poff = poff;
    d.key_env = (unsigned)e;
    poff += s.n_particles;
  }
  const size_t off_acc = cur;
  cur = align256(cur + ctx->acc_stride * n_envs * 4);
  const size_t off_ctr = cur;
  cur = align256(cur + sizeof(EnvCtr) * n_envs);
  ctx->arena_bytes = cur;
  CK(cudaMalloc(&ctx->arena, ctx->arena_bytes));
  CK(cudaMemset(ctx->arena, 0, ctx->arena_bytes));
  char* A = ctx->arena;
  ctx->acc_all = (float*)(A + off_acc);
  ctx->ctr_all = (EnvCtr*)(A + off_ctr);
  for (int e = 0; e < n_envs; ++e) {
    EnvDesc& d = ctx->desc[e];
    const long long G3 = (long long)d.G * d.G * d.G;
    d.slots = (float*)(A + off_slots[e]);
    d.ring = tape ? (float*)(A + off_ring[e]) : nullptr;
    d.adj0 = tape ? (float*)(A + off_adj[e]) : nullptr;
    d.adj1 = tape ? d.adj0 + (size_t)kComp * d.n_pad : nullptr;
    d.perm = (unsigned*)(A + off_perm[e]);
    float4* g = (float4*)(A + off_grid[e]);
    d.grid_mp = g;
    d.grid_v = g + G3;
    d.grid_vb = tape ? g + 2 * G3 : nullptr;
    d.grid_mpb = tape ? g + 3 * G3 : nullptr;
    d.tile = (unsigned*)(A + off_tile[e]);
    d.pose = (float*)(A + off_pose[e]);
    d.act = (float*)(A + off_act[e]);
    d.acc = ctx->acc_all + ctx->acc_stride * e;
    d.ctr = ctx->ctr_all + e;
  }
  // initial poses (slot 0)
  for (int e = 0; e < n_envs; ++e) CK(cudaMemcpy(ctx->desc[e].pose, ctx->specs[e].pose0, 16, cudaMemcpyHostToDevice));

  // ---- work items: runs of <= chunk particles of one env
  for (int e = 0; e < n_envs; ++e) {
    ctx->env_item0.push_back((int)ctx->items_env_order.size());
    int cnt = 0;
    for (int s0 = 0; s0 < ctx->specs[e].n_particles; s0 += ctx->chunk) {
      WorkItem it{e, s0, std::min(ctx->chunk, ctx->specs[e].n_particles - s0), 0};
      ctx->items_env_order.push_back(it);
      ++cnt;
    }
    ctx->env_nitems.push_back(cnt);
  }
  // particle kernels are compiled per material: group the items by material, and within
  // a group by substep count (descending) so substep k launches a prefix of the group
  ctx->items = ctx->items_env_order;
  std::stable_sort(ctx->items.begin(), ctx->items.end(), [&](const WorkItem& a, const WorkItem& b) {
    const auto &sa = ctx->specs[a.env], &sb = ctx->specs[b.env];
    if (sa.material != sb.material) return sa.material < sb.material;
    return sa.substeps > sb.substeps;
  });
  for (size_t i = 0; i < ctx->items.size(); ++i) {
    const int mat = ctx->specs[ctx->items[i].env].material;
    if (ctx->groups.empty() || ctx->groups.back().material != mat)
      ctx->groups.push_back({mat, (int)i, std::vector<int>(S_max + 1, 0)});
    auto& g = ctx->groups.back();
    for (int k = 0; k <= S_max; ++k)
      if (ctx->specs[ctx->items[i].env].substeps > k) g.n_gt[k] += 1;
  }

  // ---- device arrays
  CK(cudaMalloc(&ctx->d_desc, sizeof(EnvDesc) * n_envs));
  CK(cudaMemcpy(ctx->d_desc, ctx->desc.data(), sizeof(EnvDesc) * n_envs, cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_items, sizeof(WorkItem) * ctx->items.size()));
  CK(cudaMemcpy(ctx->d_items, ctx->items.data(), sizeof(WorkItem) * ctx->items.size(), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&ctx->d_items_env, sizeof(WorkItem) * ctx->items_env_order.size()));
  CK(cudaMemcpy(ctx->d_items_env, ctx->items_env_order.data(), sizeof(WorkItem) * ctx->items_env_order.size(),
                cudaMemcpyHostToDevice));
  ctx->active_cap = tiles_total;
  CK(cudaMalloc(&ctx->active, sizeof(uint2) * std::max<long long>(tiles_total, 1)));
  CK(cudaMalloc(&ctx->active_n, sizeof(int)));
  CK(cudaMemset(ctx->active_n, 0, sizeof(int)));
  const long long sort_blocks = (P + 4095) / 4096;
  for (int i = 0; i < 2; ++i) {
    CK(cudaMalloc(&ctx->sort.keys[i], sizeof(unsigned) * P));
    CK(cudaMalloc(&ctx->sort.vals[i], sizeof(unsigned) * P));
  }
  CK(cudaMalloc(&ctx->sort.hist, sizeof(unsigned) * 256 * std::max<long long>(sort_blocks, 1)));
  ctx->sort.cap = P;
  CK(cudaMalloc(&ctx->act_in, sizeof(float) * n_envs * A_max));
  CK(cudaMemset(ctx->act_in, 0, sizeof(float) * n_envs * A_max));
  CK(cudaMalloc(&ctx->rew, sizeof(float) * n_envs));
  CK(cudaMalloc(&ctx->posebuf, sizeof(float) * n_envs * 4));
  CK(cudaMalloc(&ctx->io, sizeof(float) * P * kComp));
  if (tape) {
    CK(cudaMalloc(&ctx->rbar, sizeof(float) * ctx->T_cap * n_envs));
    CK(cudaMalloc(&ctx->agrad, sizeof(float) * (size_t)ctx->T_cap * n_envs * A_max));
  }
  CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  ctx->total_bytes = ctx->arena_bytes + sizeof(unsigned) * P * 4 + sizeof(float) * P * kComp +
                     sizeof(uint2) * tiles_total + (tape ? sizeof(float) * (size_t)ctx->T_cap * n_envs * (A_max + 1) : 0);
  *out = ctx;
  return MPM_OK;
}

void mpm_destroy(mpm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto& g : ctx->g_fwd)
    if (g) cudaGraphExecDestroy(g);
  if (ctx->g_rev) cudaGraphExecDestroy(ctx->g_rev);
  for (auto e : ctx->ev) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  void* ptrs[] = {ctx->arena, ctx->d_desc, ctx->d_items, ctx->d_items_env, ctx->active, ctx->active_n,
                  ctx->sort.keys[0], ctx->sort.keys[1], ctx->sort.vals[0], ctx->sort.vals[1], ctx->sort.hist,
                  ctx->act_in, ctx->rew, ctx->rbar, ctx->agrad, ctx->io, ctx->posebuf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete ctx;
}

mpm_status mpm_set_state(mpm_ctx* ctx, const float* x, const float* v, const float* C, const float* F,
                         const int32_t* group, const float* pose, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!x || !v || !C || !F) return fail(ctx, MPM_ERR_INVALID_ARG, "x, v, C and F are required");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  const long long P = ctx->P;
  float* io = ctx->io;
  CK(cudaMemcpyAsync(io, x, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(io + P * 3, v, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(io + P * 6, C, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(io + P * 15, F, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  int* gbuf = nullptr;
  if (group) {
    gbuf = (int*)ctx->sort.keys[0];  // scratch, P words
    CK(cudaMemcpyAsync(gbuf, group, sizeof(int) * P, cudaMemcpyDefault, st));
  }
  CK(cudaMemsetAsync(ctx->ctr_all, 0, sizeof(EnvCtr) * ctx->n_envs, st));
  Launch L = make_launch(ctx, st);
  L.items = ctx->d_items_env;
  L.n_items = (int)ctx->items_env_order.size();
  {
    Enqueue q(ctx);
    launch_set_state(L, io, io + P * 3, io + P * 6, io + P * 15, gbuf);
  }
  if (pose) {
    CK(cudaMemcpyAsync(ctx->posebuf, pose, sizeof(float) * 4 * ctx->n_envs, cudaMemcpyDefault, st));
    for (int e = 0; e < ctx->n_envs; ++e)
      CK(cudaMemcpyAsync(ctx->desc[e].pose, ctx->posebuf + 4 * e, 16, cudaMemcpyDeviceToDevice, st));
  } else {
    // keep the current pose: move it to slot 0
    for (int e = 0; e < ctx->n_envs; ++e)
      if (ctx->h_live != 0)
        CK(cudaMemcpyAsync(ctx->desc[e].pose, ctx->desc[e].pose + 4 * ctx->h_live, 16, cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaGetLastError());
  ctx->h_live = ctx->h_base = 0;
  return MPM_OK;
}

mpm_status mpm_get_state(mpm_ctx* ctx, float* x, float* v, float* C, float* F, float* pose, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  const long long P = ctx->P;
  float* io = ctx->io;
  Launch L = make_launch(ctx, st);
  L.items = ctx->d_items_env;
  L.n_items = (int)ctx->items_env_order.size();
  {
    Enqueue q(ctx);
    launch_get_state(L, StateRef{REF_LIVE, 0}, io, io + P * 3, io + P * 6, io + P * 15);
  }
  CK(cudaGetLastError());
  if (x) CK(cudaMemcpyAsync(x, io, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (v) CK(cudaMemcpyAsync(v, io + P * 3, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (C) CK(cudaMemcpyAsync(C, io + P * 6, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (F) CK(cudaMemcpyAsync(F, io + P * 15, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (pose) {
    for (int e = 0; e < ctx->n_envs; ++e)
      CK(cudaMemcpyAsync(ctx->posebuf + 4 * e, ctx->desc[e].pose + 4 * ctx->h_live, 16, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(pose, ctx->posebuf, sizeof(float) * 4 * ctx->n_envs, cudaMemcpyDefault, st));
  }
  return MPM_OK;
}

mpm_status mpm_step(mpm_ctx* ctx, const float* actions, float* reward, uint32_t flags, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  const bool record = (flags & MPM_STEP_RECORD) != 0;
  if (record && (ctx->T_cap == 0 || ctx->h_live + 1 >= ctx->n_slots))
    return fail(ctx, MPM_ERR_STATE, "checkpoint tape full (max_steps=%d)", ctx->T_cap);
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  if (actions)
    CK(cudaMemcpyAsync(ctx->act_in, actions, sizeof(float) * ctx->n_envs * ctx->A_max, cudaMemcpyDefault, st));
  else
    CK(cudaMemsetAsync(ctx->act_in, 0, sizeof(float) * ctx->n_envs * ctx->A_max, st));
  bool rec = record;
  mpm_status s = run_graph_or_direct(ctx, &ctx->g_fwd[record ? 1 : 0], &ctx->g_fwd_kernels[record ? 1 : 0], st, body_fwd, &rec);
  if (s != MPM_OK) return s;
  if (reward) CK(cudaMemcpyAsync(reward, ctx->rew, sizeof(float) * ctx->n_envs, cudaMemcpyDefault, st));
  if (record) {
    ctx->h_live += 1;
  } else {
    ctx->h_live = ctx->h_live == 0 ? 1 : 0;
    ctx->h_base = ctx->h_live;
  }
  return MPM_OK;
}

mpm_status mpm_reset_tape(mpm_ctx* ctx) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  // the live slot stays; it becomes the tape's base (device counters follow on next set)
  ctx->h_base = ctx->h_live;
  CK(cudaDeviceSynchronize());
  std::vector<EnvCtr> c(ctx->n_envs);
  CK(cudaMemcpy(c.data(), ctx->ctr_all, sizeof(EnvCtr) * ctx->n_envs, cudaMemcpyDeviceToHost));
  for (auto& x : c) x.base = x.live;
  CK(cudaMemcpy(ctx->ctr_all, c.data(), sizeof(EnvCtr) * ctx->n_envs, cudaMemcpyHostToDevice));
  return MPM_OK;
}

mpm_status mpm_backward(mpm_ctx* ctx, const float* xb, const float* vb, const float* Cb, const float* Fb,
                        const float* reward_adj, float* action_grad, float* xb0, float* vb0, float* Cb0, float* Fb0,
                        float* pose_grad0, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  const int T = ctx->h_live - ctx->h_base;
  if (T <= 0) return fail(ctx, MPM_ERR_STATE, "no recorded steps");
  if (!action_grad && !xb0 && !vb0 && !Cb0 && !Fb0 && !pose_grad0)
    return fail(ctx, MPM_ERR_INVALID_ARG, "no output requested");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  const long long P = ctx->P;
  float* io = ctx->io;
  if (xb) CK(cudaMemcpyAsync(io, xb, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (vb) CK(cudaMemcpyAsync(io + P * 3, vb, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (Cb) CK(cudaMemcpyAsync(io + P * 6, Cb, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (Fb) CK(cudaMemcpyAsync(io + P * 15, Fb, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  // a NULL reward adjoint is a zero one (keeps a single captured reverse-step graph)
  if (reward_adj)
    CK(cudaMemcpyAsync(ctx->rbar, reward_adj, sizeof(float) * T * ctx->n_envs, cudaMemcpyDefault, st));
  else
    CK(cudaMemsetAsync(ctx->rbar, 0, sizeof(float) * T * ctx->n_envs, st));
  Launch L = make_launch(ctx, st);
  Launch Lio = L;
  Lio.items = ctx->d_items_env;
  Lio.n_items = (int)ctx->items_env_order.size();
  {
    Enqueue q(ctx);
    launch_bwd_init(L, T);
    launch_adj_in(Lio, xb ? io : nullptr, vb ? io + P * 3 : nullptr, Cb ? io + P * 6 : nullptr,
                  Fb ? io + P * 15 : nullptr);
  }
  CK(cudaGetLastError());
  bool have_rbar = true;
  for (int t = T - 1; t >= 0; --t) {
    if (ctx->per_env) {
      Enqueue q(ctx);
      for (int e = 0; e < ctx->n_envs; ++e) {
        Launch Le = env_launch(ctx, e, st);
        const int S = ctx->specs[e].substeps;
        std::vector<mpm_ctx::MatGroup> one{{ctx->specs[e].material, ctx->env_item0[e],
                                            std::vector<int>(S + 1, ctx->env_nitems[e])}};
        one[0].n_gt[S] = 0;
        enqueue_reverse_step(ctx, Le, S, one, have_rbar);
      }
      CK(cudaGetLastError());
    } else {
      mpm_status s = run_graph_or_direct(ctx, &ctx->g_rev, &ctx->g_rev_kernels, st, body_rev, &have_rbar);
      if (s != MPM_OK) return s;
    }
  }
  {
    Enqueue q(ctx);
    launch_adj_out(Lio, StateRef{REF_REV, 0}, io, io + P * 3, io + P * 6, io + P * 15);
  }
  CK(cudaGetLastError());
  if (xb0) CK(cudaMemcpyAsync(xb0, io, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (vb0) CK(cudaMemcpyAsync(vb0, io + P * 3, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (Cb0) CK(cudaMemcpyAsync(Cb0, io + P * 6, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (Fb0) CK(cudaMemcpyAsync(Fb0, io + P * 15, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (action_grad)
    CK(cudaMemcpyAsync(action_grad, ctx->agrad, sizeof(float) * (size_t)T * ctx->n_envs * ctx->A_max, cudaMemcpyDefault,
                       st));
  if (pose_grad0)
    CK(cudaMemcpy2DAsync(pose_grad0, 16, ctx->acc_all + ACC_QB, ctx->acc_stride * 4, 16, ctx->n_envs, cudaMemcpyDefault,
                         st));
  return MPM_OK;
}

mpm_status mpm_check_status(mpm_ctx* ctx, int32_t* flags) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaDeviceSynchronize());
  std::vector<EnvCtr> c(ctx->n_envs);
  CK(cudaMemcpy(c.data(), ctx->ctr_all, sizeof(EnvCtr) * ctx->n_envs, cudaMemcpyDeviceToHost));
  int any = 0;
  for (int e = 0; e < ctx->n_envs; ++e) {
    if (flags) flags[e] = c[e].status;
    any |= c[e].status;
    c[e].status = 0;
  }
  CK(cudaMemcpy(ctx->ctr_all, c.data(), sizeof(EnvCtr) * ctx->n_envs, cudaMemcpyHostToDevice));
  if (any & 6) return fail(ctx, MPM_ERR_NUMERIC, "NaN/Inf or inverted F flagged (bits %d)", any);
  if (any & 1) return fail(ctx, MPM_ERR_DOMAIN, "a particle left the grid");
  return MPM_OK;
}

int64_t mpm_kernel_launches(const mpm_ctx* ctx) { return ctx ? ctx->launches : 0; }

mpm_status mpm_time_kernel(mpm_ctx* ctx, int32_t kernel_class) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (kernel_class < -1 || kernel_class > KC_OTHER) return fail(ctx, MPM_ERR_INVALID_ARG, "kernel_class");
  ctx->time_kc = kernel_class;
  ctx->ev_used = 0;
  return MPM_OK;
}

mpm_status mpm_kernel_time(mpm_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  double tot[KC_OTHER + 1] = {0};
  int64_t cnt[KC_OTHER + 1] = {0};
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float ms = 0.f;
    CK(cudaEventSynchronize(ctx->ev[i + 1]));
    CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
    const int kc = ctx->ev_class[i / 2];
    tot[kc] += ms;
    cnt[kc] += 1;
  }
  // one entry (single class timed) or KC_OTHER + 1 entries indexed by class (all timed)
  if (ctx->time_kc > 0) {
    if (total_ms) *total_ms = tot[ctx->time_kc];
    if (launches) *launches = cnt[ctx->time_kc];
  } else {
    for (int k = 0; k <= KC_OTHER; ++k) {
      if (total_ms) total_ms[k] = tot[k];
      if (launches) launches[k] = cnt[k];
    }
  }
  ctx->ev_used = 0;
  return MPM_OK;
}

int32_t mpm_last_active_tiles(mpm_ctx* ctx) {
  if (!ctx) return -1;
  int n = -1;
  if (cudaMemcpy(&n, ctx->active_n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return n;
}

mpm_status mpm_bin(const float* x, int32_t n, int32_t grid_res, uint32_t* keys, uint32_t* perm, void* stream) {
  if (!x || !keys || !perm || n < 0 || grid_res < 8 || grid_res > 128 || grid_res % 4) return MPM_ERR_INVALID_ARG;
  if (n == 0) return MPM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned *k2 = nullptr, *v2 = nullptr, *v1 = nullptr, *hist = nullptr;
  const long long nb = ((long long)n + 4095) / 4096;
  if (cudaMalloc(&k2, sizeof(unsigned) * n) != cudaSuccess) return MPM_ERR_OOM;
  if (cudaMalloc(&v1, sizeof(unsigned) * n) != cudaSuccess) { cudaFree(k2); return MPM_ERR_OOM; }
  if (cudaMalloc(&v2, sizeof(unsigned) * n) != cudaSuccess) { cudaFree(k2); cudaFree(v1); return MPM_ERR_OOM; }
  if (cudaMalloc(&hist, sizeof(unsigned) * 256 * nb) != cudaSuccess) {
    cudaFree(k2); cudaFree(v1); cudaFree(v2);
    return MPM_ERR_OOM;
  }
  unsigned* k1 = nullptr;
  cudaMalloc(&k1, sizeof(unsigned) * n);
  launch_bin_keys_plain(x, n, grid_res, k1, v1, st);
  cudaMemcpyAsync(keys, k1, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
  const unsigned long long max_cell = (unsigned long long)(grid_res / 4) * (grid_res / 4) * (grid_res / 4) * 64ull - 1ull;
  unsigned* kk[2] = {k1, k2};
  unsigned* vv[2] = {v1, v2};
  int cur = radix_sort(kk, vv, n, bits_for(max_cell), hist, st);
  cudaMemcpyAsync(perm, vv[cur], sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(k1); cudaFree(k2); cudaFree(v1); cudaFree(v2); cudaFree(hist);
  return e == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}

}  // extern "C"
