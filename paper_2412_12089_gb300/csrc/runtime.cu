// runtime.cu -- batch context of the MPM library and the C ABI of include/mpm.h.
//
// A context holds one Group (engine.h): all of its environments advance together, one launch
// per stage.  With MPM_STEP_RECORD the step's start state stays on the checkpoint tape and
// mpm_backward reverses the recorded steps (Sec. 4.1, gradient checkpointing).  Every
// per-step quantity the kernels need lives in device counters, so a captured control-step
// graph (and a reverse-step graph) is replayed unchanged at every step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "kernels.h"
#include "mpm.h"
#include "mpm_types.h"

using namespace mpm;

namespace {
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

struct mpm_ctx {
  int device = 0;
  int n_envs = 0;
  long long P = 0;
  int A_max = 1;
  int T_cap = 0;
  int n_slots = 2;
  bool per_env = false;
  bool use_graphs = false;
  std::vector<mpm_env_spec> specs;
  Group g;
  TuneTimes tune;  // the last autotuning's trial times
  char* arena = nullptr;
  size_t arena_bytes = 0;
  float* act_in = nullptr;   // [n_envs][A_max]
  float* rew = nullptr;      // [n_envs]
  float* rbar = nullptr;     // [T_cap][n_envs]
  float* agrad = nullptr;    // [T_cap][n_envs][A_max]
  float* io = nullptr;       // [P][24] staging
  float* posebuf = nullptr;  // [n_envs][4]
  float* obs_adj = nullptr;  // [T_cap + 1][n_envs][obs_dim] observation adjoints
  int* obs_on = nullptr;     // device flag: obs_adj holds adjoints for the next backward
  int obs_dim = 0, nsub_max = 0;
  size_t acc_stride = 0;
  float* acc_all = nullptr;
  EnvCtr* ctr_all = nullptr;
  int h_live = 0, h_base = 0;  // host mirrors of the device counters (identical in all envs)
  // step-wise reverse pass (mpm_backward_begin / _step / _end): steps recorded when it began
  // and the next step to reverse (-1 when all are done); open between begin and end
  bool bwd_open = false;
  int bwd_T = 0, bwd_next = -1;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t g_fwd[2] = {nullptr, nullptr};
  cudaGraphExec_t g_rev[2] = {nullptr, nullptr};  // reverse step: recomputing, on kept states
  long long g_fwd_kernels[2] = {0, 0};
  long long g_rev_kernels[2] = {0, 0};
  long long launches = 0;        // kernels this context launched (graph replays included)
  int time_kc = 0;               // kernel class timed with events (0 = none, -1 = all)
  std::vector<cudaEvent_t> ev;   // start/stop pairs of timed launches
  std::vector<int> ev_class;     // class of each pair
  size_t ev_used = 0;
  std::string err;
  size_t total_bytes = 0;
};

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

// ---------------------------------------------------------------- instrumentation

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

void body_fwd(mpm_ctx* c, cudaStream_t st, void* arg) {
  enqueue_forward(c->g, st, *(bool*)arg, c->act_in, c->A_max, c->rew, c->per_env);
}

ObsAdj obs_of(const mpm_ctx* c) { return ObsAdj{c->obs_adj, c->obs_on, c->obs_dim, c->nsub_max, c->n_envs}; }

// arg: bool, the step's substep states were kept by the forward pass
void body_rev(mpm_ctx* c, cudaStream_t st, void* arg) {
  const ObsAdj o = obs_of(c);
  enqueue_reverse(c->g, st, c->rbar, c->agrad, c->n_envs, c->A_max, c->per_env, c->obs_adj ? &o : nullptr,
                  *(bool*)arg);
}

Launch io_launch(mpm_ctx* ctx, cudaStream_t st) {
  Launch L = group_launch(ctx->g, st);
  L.items = ctx->g.d_items_env;
  L.n_items = (int)ctx->g.items_env.size();
  return L;
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
int32_t mpm_kept_steps(const mpm_ctx* ctx) { return ctx ? (int32_t)ctx->g.keep_n : 0; }

mpm_status mpm_create(const mpm_env_spec* specs, int n_envs, const mpm_options* opt, mpm_ctx** out) {
  if (!out) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  mpm_ctx* ctx = new mpm_ctx();
  auto bail = [&](mpm_status s) {
    *out = ctx;  // hand back the context so mpm_last_error works; the caller destroys it
    return s;
  };
  if (!specs || n_envs < 1 || n_envs > (1 << 16)) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "n_envs"));
  mpm_options o{};
  if (opt) o = *opt;
  if (o.max_steps < 0 || o.max_steps > 100000) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "max_steps"));
  if (o.chunk != 0 && o.chunk != kChunk) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "chunk (only 256 is built)"));
  ctx->device = o.device;
  ctx->T_cap = o.max_steps;
  ctx->n_slots = std::max(o.max_steps + 1, 2);
  ctx->per_env = o.per_env_launch != 0;
  ctx->use_graphs = o.use_graphs != 0;
  ctx->n_envs = n_envs;
  ctx->specs.assign(specs, specs + n_envs);
  for (int e = 0; e < n_envs; ++e) {
    const char* bad = check_spec(specs[e]);
    if (bad) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "env %d: invalid %s", e, bad));
  }
  int A_max = 1, G_max = 8;
  long long P = 0;
  for (auto& s : ctx->specs) {
    A_max = std::max(A_max, s.n_coll_act + s.n_groups);
    G_max = std::max(G_max, s.grid_res);
    P += s.n_particles;
  }
  {
    int cb = 0, eb = 0;
    for (unsigned long long v = (unsigned long long)(G_max / 4) * (G_max / 4) * (G_max / 4) * 64ull - 1ull; v; v >>= 1)
      ++cb;
    for (unsigned long long v = (unsigned long long)(n_envs - 1); v; v >>= 1) ++eb;
    if (cb + eb > 32) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "too many environments for a 32-bit binning key"));
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return bail(fail(ctx, MPM_ERR_CUDA, "cudaSetDevice(%d)", ctx->device));
  ctx->A_max = A_max;
  ctx->P = P;
  const bool tape = ctx->T_cap > 0;
  ctx->acc_stride = (size_t)ACC_ACT + A_max;

  // ---- every environment's buffers in one arena, then shared accumulators and counters
  std::vector<EnvLayout> lay(n_envs);
  std::vector<size_t> off(n_envs);
  size_t cur = 0;
  for (int e = 0; e < n_envs; ++e) {
    lay[e] = env_layout(ctx->specs[e], ctx->n_slots, tape, false, 0);
    off[e] = cur;
    cur = align256(cur + lay[e].total);
  }
  const size_t off_acc = cur;
  cur = align256(cur + ctx->acc_stride * n_envs * 4);
  const size_t off_ctr = cur;
  cur = align256(cur + sizeof(EnvCtr) * n_envs);
  ctx->arena_bytes = cur;
  if (cudaMalloc(&ctx->arena, ctx->arena_bytes) != cudaSuccess)
    return bail(fail(ctx, MPM_ERR_OOM, "arena of %zu bytes", ctx->arena_bytes));
  if (cudaMemset(ctx->arena, 0, ctx->arena_bytes) != cudaSuccess) return bail(fail(ctx, MPM_ERR_CUDA, "memset"));
  ctx->acc_all = (float*)(ctx->arena + off_acc);
  ctx->ctr_all = (EnvCtr*)(ctx->arena + off_ctr);
  std::vector<EnvDesc> desc(n_envs);
  for (int e = 0; e < n_envs; ++e) {
    env_fill(desc[e], ctx->specs[e], lay[e], ctx->arena + off[e], ctx->acc_all + ctx->acc_stride * e, ctx->ctr_all + e);
    float q0[kPose];
    initial_pose(ctx->specs[e], q0);
    if (cudaMemcpy(desc[e].pose, q0, sizeof q0, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(ctx, MPM_ERR_CUDA, "pose upload"));
    const cudaError_t fe = fem_upload(ctx->specs[e], desc[e]);
    if (fe == cudaErrorInvalidValue) return bail(fail(ctx, MPM_ERR_INVALID_ARG, "env %d: degenerate element", e));
    if (fe != cudaSuccess) return bail(fail(ctx, MPM_ERR_CUDA, "FEM mesh upload"));
  }
  // grid tape for batched reverse passes: a share of the memory left after the arena
  ctx->g.want_tape = o.max_steps > 0 && !o.per_env_launch && o.grid_tape_fraction >= 0.0f;
  ctx->g.tape_T = o.max_steps;
  if (ctx->g.want_tape) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
    const double frac = o.grid_tape_fraction > 0.0f ? std::min(1.0, (double)o.grid_tape_fraction) : 0.5;
    ctx->g.tape_budget = frac * (double)free_b;
    // kept substep states: a share of what the tape leaves, less the staging buffers below
    ctx->g.keep_frac = o.keep_fraction < 0.0f ? 0.0 : (o.keep_fraction > 0.0f ? std::min(1.0, (double)o.keep_fraction) : 0.8);
    ctx->g.keep_reserve = (double)sizeof(float) * (double)P * (kComp + 8) +
                          (double)sizeof(float) * o.max_steps * n_envs * (A_max + 1) * 2.0 + (1u << 30);
  }
  cudaError_t ge = group_build(ctx->g, desc, ctx->specs);
  if (ge != cudaSuccess)
    return bail(fail(ctx, ge == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA, "group: %s", cudaGetErrorString(ge)));

  // ---- staging buffers
  auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess; };
  bool ok = alloc((void**)&ctx->act_in, sizeof(float) * n_envs * A_max) && alloc((void**)&ctx->rew, sizeof(float) * n_envs) &&
            alloc((void**)&ctx->posebuf, sizeof(float) * n_envs * 4) && alloc((void**)&ctx->io, sizeof(float) * P * kComp);
  if (ok && tape)
    ok = alloc((void**)&ctx->rbar, sizeof(float) * ctx->T_cap * n_envs) &&
         alloc((void**)&ctx->agrad, sizeof(float) * (size_t)ctx->T_cap * n_envs * A_max);
  ctx->nsub_max = 0;
  for (const auto& sp : ctx->specs) ctx->nsub_max = std::max(ctx->nsub_max, std::min(sp.n_sub, sp.n_particles));
  ctx->obs_dim = 3 * ctx->nsub_max + 10;
  if (ok && tape)
    ok = alloc((void**)&ctx->obs_adj, sizeof(float) * (size_t)(ctx->T_cap + 1) * n_envs * ctx->obs_dim) &&
         alloc((void**)&ctx->obs_on, sizeof(int));
  if (!ok) return bail(fail(ctx, MPM_ERR_OOM, "staging buffers"));
  if (ctx->obs_on) cudaMemset(ctx->obs_on, 0, sizeof(int));
  cudaMemset(ctx->act_in, 0, sizeof(float) * n_envs * A_max);
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(ctx, MPM_ERR_CUDA, "stream"));
  ctx->total_bytes = ctx->arena_bytes + sizeof(unsigned) * P * 4 + sizeof(float) * P * kComp +
                     sizeof(uint2) * ctx->g.tiles + (tape ? sizeof(float) * (size_t)ctx->T_cap * n_envs * (A_max + 1) : 0) +
                     (size_t)ctx->g.tape.cap * (64 * sizeof(float4) + sizeof(uint2)) + sizeof(float) * ctx->g.keep_cap;
  *out = ctx;
  return MPM_OK;
}

void mpm_destroy(mpm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto& g : ctx->g_fwd)
    if (g) cudaGraphExecDestroy(g);
  for (auto& g : ctx->g_rev)
    if (g) cudaGraphExecDestroy(g);
  for (auto e : ctx->ev) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  ctx->g.release();
  void* ptrs[] = {ctx->arena, ctx->act_in, ctx->rew, ctx->rbar, ctx->agrad, ctx->io, ctx->posebuf, ctx->obs_adj,
                  ctx->obs_on};
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
    gbuf = (int*)ctx->g.sort.keys[0];  // scratch, P words
    CK(cudaMemcpyAsync(gbuf, group, sizeof(int) * P, cudaMemcpyDefault, st));
  }
  if (pose) {
    CK(cudaMemcpyAsync(ctx->posebuf, pose, sizeof(float) * 4 * ctx->n_envs, cudaMemcpyDefault, st));
    launch_pose_io(io_launch(ctx, st), POSE_SET, ctx->posebuf, 0);
  } else if (ctx->h_live != 0) {
    // keep the current pose: move it to slot 0
    launch_pose_io(io_launch(ctx, st), POSE_KEEP, ctx->posebuf, ctx->h_live);
  }
  CK(cudaMemsetAsync(ctx->ctr_all, 0, sizeof(EnvCtr) * ctx->n_envs, st));
  {
    Enqueue q(ctx);
    launch_set_state(io_launch(ctx, st), io, io + P * 3, io + P * 6, io + P * 15, gbuf);
  }
  CK(cudaGetLastError());
  ctx->h_live = ctx->h_base = 0;
  ctx->bwd_open = false;  // the tape an open step-wise reverse pass ran over is gone
  return MPM_OK;
}

mpm_status mpm_get_state(mpm_ctx* ctx, float* x, float* v, float* C, float* F, float* pose, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  const long long P = ctx->P;
  float* io = ctx->io;
  {
    Enqueue q(ctx);
    launch_get_state(io_launch(ctx, st), StateRef{REF_LIVE, 0}, io, io + P * 3, io + P * 6, io + P * 15);
  }
  CK(cudaGetLastError());
  if (x) CK(cudaMemcpyAsync(x, io, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (v) CK(cudaMemcpyAsync(v, io + P * 3, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (C) CK(cudaMemcpyAsync(C, io + P * 6, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (F) CK(cudaMemcpyAsync(F, io + P * 15, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (pose) {
    launch_pose_io(io_launch(ctx, st), POSE_GET, ctx->posebuf, ctx->h_live);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pose, ctx->posebuf, sizeof(float) * 4 * ctx->n_envs, cudaMemcpyDefault, st));
  }
  return MPM_OK;
}

mpm_status mpm_step(mpm_ctx* ctx, const float* actions, float* reward, uint32_t flags, void* stream) {
  if (ctx) ctx->bwd_open = false;  // a new step changes the tape under an open reverse pass
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
  mpm_status s = run_graph_or_direct(ctx, &ctx->g_fwd[record ? 1 : 0], &ctx->g_fwd_kernels[record ? 1 : 0], st,
                                     body_fwd, &rec);
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
  // the live slot stays; it becomes the tape's base
  ctx->h_base = ctx->h_live;
  ctx->bwd_open = false;
  CK(cudaDeviceSynchronize());
  std::vector<EnvCtr> c(ctx->n_envs);
  CK(cudaMemcpy(c.data(), ctx->ctr_all, sizeof(EnvCtr) * ctx->n_envs, cudaMemcpyDeviceToHost));
  for (auto& x : c) x.base = x.live;
  CK(cudaMemcpy(ctx->ctr_all, c.data(), sizeof(EnvCtr) * ctx->n_envs, cudaMemcpyHostToDevice));
  return MPM_OK;
}

// Start of a reverse pass over the T recorded steps: the final state's adjoint in, every
// accumulator zeroed.
static mpm_status bwd_begin(mpm_ctx* ctx, const float* xb, const float* vb, const float* Cb, const float* Fb,
                            cudaStream_t st, int* T_out) {
  const int T = ctx->h_live - ctx->h_base;
  if (T <= 0) return fail(ctx, MPM_ERR_STATE, "no recorded steps");
  CK(cudaSetDevice(ctx->device));
  const long long P = ctx->P;
  float* io = ctx->io;
  if (xb) CK(cudaMemcpyAsync(io, xb, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (vb) CK(cudaMemcpyAsync(io + P * 3, vb, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (Cb) CK(cudaMemcpyAsync(io + P * 6, Cb, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (Fb) CK(cudaMemcpyAsync(io + P * 15, Fb, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  {
    Enqueue q(ctx);
    launch_bwd_init(group_launch(ctx->g, st), T);
    launch_adj_in(io_launch(ctx, st), xb ? io : nullptr, vb ? io + P * 3 : nullptr, Cb ? io + P * 6 : nullptr,
                  Fb ? io + P * 15 : nullptr);
  }
  CK(cudaGetLastError());
  *T_out = T;
  return MPM_OK;
}

// One reverse step (the next one down, t of T recorded), through the captured reverse-step
// graph: the one without the recompute when the forward pass kept the step's substep states.
static mpm_status bwd_step(mpm_ctx* ctx, cudaStream_t st, int t, int T) {
  bool kept = ctx->g.keep_n > 0 && !ctx->per_env && T - t <= ctx->g.keep_n;
  const int i = kept ? 1 : 0;
  return run_graph_or_direct(ctx, &ctx->g_rev[i], &ctx->g_rev_kernels[i], st, body_rev, &kept);
}

// End of a reverse pass: the initial state's observation adjoint (when set), then the initial
// state's and pose's adjoints out.
static mpm_status bwd_end(mpm_ctx* ctx, float* xb0, float* vb0, float* Cb0, float* Fb0, float* pose_grad0,
                          cudaStream_t st) {
  const long long P = ctx->P;
  float* io = ctx->io;
  {
    Enqueue q(ctx);
    if (ctx->obs_adj) {
      launch_obs_adj(group_launch(ctx->g, st), obs_of(ctx), 1);  // observation of the initial state
      CK(cudaMemsetAsync(ctx->obs_on, 0, sizeof(int), st));      // consumed
    }
    launch_adj_out(io_launch(ctx, st), StateRef{REF_REV, 0}, io, io + P * 3, io + P * 6, io + P * 15);
  }
  CK(cudaGetLastError());
  if (xb0) CK(cudaMemcpyAsync(xb0, io, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (vb0) CK(cudaMemcpyAsync(vb0, io + P * 3, sizeof(float) * P * 3, cudaMemcpyDefault, st));
  if (Cb0) CK(cudaMemcpyAsync(Cb0, io + P * 6, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (Fb0) CK(cudaMemcpyAsync(Fb0, io + P * 15, sizeof(float) * P * 9, cudaMemcpyDefault, st));
  if (pose_grad0) {
    launch_pose_io(io_launch(ctx, st), POSE_GRAD, ctx->posebuf, 0);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pose_grad0, ctx->posebuf, sizeof(float) * 4 * ctx->n_envs, cudaMemcpyDefault, st));
  }
  return MPM_OK;
}

mpm_status mpm_backward(mpm_ctx* ctx, const float* xb, const float* vb, const float* Cb, const float* Fb,
                        const float* reward_adj, float* action_grad, float* xb0, float* vb0, float* Cb0, float* Fb0,
                        float* pose_grad0, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!action_grad && !xb0 && !vb0 && !Cb0 && !Fb0 && !pose_grad0)
    return fail(ctx, MPM_ERR_INVALID_ARG, "no output requested");
  if (ctx->bwd_open) return fail(ctx, MPM_ERR_STATE, "a step-wise reverse pass is open");
  cudaStream_t st = (cudaStream_t)stream;
  int T = 0;
  mpm_status s = bwd_begin(ctx, xb, vb, Cb, Fb, st, &T);
  if (s != MPM_OK) return s;
  // a NULL reward adjoint is a zero one (keeps a single captured reverse-step graph)
  if (reward_adj)
    CK(cudaMemcpyAsync(ctx->rbar, reward_adj, sizeof(float) * T * ctx->n_envs, cudaMemcpyDefault, st));
  else
    CK(cudaMemsetAsync(ctx->rbar, 0, sizeof(float) * T * ctx->n_envs, st));
  for (int t = T - 1; t >= 0; --t)
    if ((s = bwd_step(ctx, st, t, T)) != MPM_OK) return s;
  if ((s = bwd_end(ctx, xb0, vb0, Cb0, Fb0, pose_grad0, st)) != MPM_OK) return s;
  if (action_grad)
    CK(cudaMemcpyAsync(action_grad, ctx->agrad, sizeof(float) * (size_t)T * ctx->n_envs * ctx->A_max,
                       cudaMemcpyDefault, st));
  return MPM_OK;
}

mpm_status mpm_backward_begin(mpm_ctx* ctx, const float* xb, const float* vb, const float* Cb, const float* Fb,
                              void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (ctx->bwd_open) return fail(ctx, MPM_ERR_STATE, "a step-wise reverse pass is already open");
  cudaStream_t st = (cudaStream_t)stream;
  int T = 0;
  const mpm_status s = bwd_begin(ctx, xb, vb, Cb, Fb, st, &T);
  if (s != MPM_OK) return s;
  // observation adjoints come step by step now: forget any set for a whole-tape backward
  if (ctx->obs_on) CK(cudaMemsetAsync(ctx->obs_on, 0, sizeof(int), st));
  ctx->bwd_open = true;
  ctx->bwd_T = T;
  ctx->bwd_next = T - 1;
  return MPM_OK;
}

mpm_status mpm_backward_step(mpm_ctx* ctx, const float* reward_adj, const float* obs_adj, float* action_grad,
                             int32_t* step, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!ctx->bwd_open) return fail(ctx, MPM_ERR_STATE, "no step-wise reverse pass is open");
  if (ctx->bwd_next < 0) return fail(ctx, MPM_ERR_STATE, "every recorded step is reversed");
  if (obs_adj && !ctx->obs_adj) return fail(ctx, MPM_ERR_STATE, "observation adjoints need a checkpoint tape");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  const int t = ctx->bwd_next;
  const size_t ne = (size_t)ctx->n_envs;
  if (reward_adj)
    CK(cudaMemcpyAsync(ctx->rbar + (size_t)t * ne, reward_adj, sizeof(float) * ne, cudaMemcpyDefault, st));
  else
    CK(cudaMemsetAsync(ctx->rbar + (size_t)t * ne, 0, sizeof(float) * ne, st));
  if (ctx->obs_adj) {
    // the reverse step adds row t + 1 (its end state) when the flag is set
    if (obs_adj) {
      CK(cudaMemcpyAsync(ctx->obs_adj + (size_t)(t + 1) * ne * ctx->obs_dim, obs_adj,
                         sizeof(float) * ne * ctx->obs_dim, cudaMemcpyDefault, st));
      CK(cudaMemsetAsync(ctx->obs_on, 0x01, 1, st));
    } else {
      CK(cudaMemsetAsync(ctx->obs_on, 0, sizeof(int), st));
    }
  }
  const mpm_status s = bwd_step(ctx, st, t, ctx->bwd_T);
  if (s != MPM_OK) return s;
  if (action_grad)
    CK(cudaMemcpyAsync(action_grad, ctx->agrad + (size_t)t * ne * ctx->A_max, sizeof(float) * ne * ctx->A_max,
                       cudaMemcpyDefault, st));
  if (step) *step = t;
  ctx->bwd_next = t - 1;
  return MPM_OK;
}

mpm_status mpm_backward_end(mpm_ctx* ctx, const float* obs_adj, float* xb0, float* vb0, float* Cb0, float* Fb0,
                            float* pose_grad0, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!ctx->bwd_open) return fail(ctx, MPM_ERR_STATE, "no step-wise reverse pass is open");
  if (ctx->bwd_next >= 0) return fail(ctx, MPM_ERR_STATE, "%d recorded steps are not reversed yet", ctx->bwd_next + 1);
  if (obs_adj && !ctx->obs_adj) return fail(ctx, MPM_ERR_STATE, "observation adjoints need a checkpoint tape");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaSetDevice(ctx->device));
  if (ctx->obs_adj) {
    if (obs_adj) {
      CK(cudaMemcpyAsync(ctx->obs_adj, obs_adj, sizeof(float) * ctx->n_envs * ctx->obs_dim, cudaMemcpyDefault, st));
      CK(cudaMemsetAsync(ctx->obs_on, 0x01, 1, st));
    } else {
      CK(cudaMemsetAsync(ctx->obs_on, 0, sizeof(int), st));
    }
  }
  ctx->bwd_open = false;
  return bwd_end(ctx, xb0, vb0, Cb0, Fb0, pose_grad0, st);
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
  if (any & MPM_FLAG_WAIT) return fail(ctx, MPM_ERR_TIMEOUT, "a bounded wait on an asynchronous copy gave up");
  if (any & (MPM_FLAG_NAN | MPM_FLAG_INVERTED))
    return fail(ctx, MPM_ERR_NUMERIC, "NaN/Inf or inverted F flagged (mask 0x%x)", any);
  if (any & MPM_FLAG_DOMAIN) return fail(ctx, MPM_ERR_DOMAIN, "a particle left the grid");
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
  // one class timed: entry 0; every class timed: entries indexed by class
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
  if (cudaMemcpy(&n, ctx->g.active_n, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return n;
}

int32_t mpm_obs_dim(const mpm_ctx* ctx) { return ctx ? ctx->obs_dim : 0; }

mpm_status mpm_observe(mpm_ctx* ctx, float* obs, void* stream) {
  if (!ctx || !obs) return MPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  {
    Enqueue q(ctx);
    launch_observe(group_launch(ctx->g, st), obs, ctx->obs_dim, ctx->nsub_max);
  }
  CK(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_set_obs_adjoint(mpm_ctx* ctx, const float* obs_adj, void* stream) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (!ctx->obs_adj) return fail(ctx, MPM_ERR_STATE, "observation adjoints need a checkpoint tape (max_steps > 0)");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int T = ctx->h_live - ctx->h_base;
  if (!obs_adj) {
    CK(cudaMemsetAsync(ctx->obs_on, 0, sizeof(int), st));
    return MPM_OK;
  }
  CK(cudaMemcpyAsync(ctx->obs_adj, obs_adj, sizeof(float) * (size_t)(T + 1) * ctx->n_envs * ctx->obs_dim,
                     cudaMemcpyDefault, st));
  CK(cudaMemsetAsync(ctx->obs_on, 0x01, 1, st));
  return MPM_OK;
}

mpm_status mpm_autotune(mpm_ctx* ctx, int32_t trials, int32_t* box_out, float* ms_out) {
  if (!ctx || trials < 1 || trials > 1000) return MPM_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaDeviceSynchronize());  // the state may still be in flight on the caller's stream
  TuneTimes tt;
  cudaError_t e;
  {
    Enqueue q(ctx);
    e = autotune_scatter(ctx->g, ctx->cap_stream, trials, &tt);
  }
  const auto& ms = tt.p2g;
  ctx->tune = tt;
  if (e != cudaSuccess) return fail(ctx, MPM_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  // captured graphs hold the old kernel choice: capture again on the next step
  for (auto& g : ctx->g_fwd)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (auto& g : ctx->g_rev)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (int m = 0; m < 4; ++m) {
    if (box_out) box_out[m] = 0;
    for (int b = 0; b < kNScatterBoxes && ms_out; ++b) ms_out[kNScatterBoxes * m + b] = 0.0f;
  }
  for (size_t i = 0; i < ctx->g.mats.size(); ++i) {
    const int mat = ctx->g.mats[i].material;
    if (mat < 0 || mat > 3) continue;
    if (box_out) box_out[mat] = ctx->g.mats[i].sc_box;
    for (int b = 0; b < kNScatterBoxes && ms_out && (int)ms[i].size() == kNScatterBoxes; ++b)
      ms_out[kNScatterBoxes * mat + b] = ms[i][b];
  }
  return MPM_OK;
}

mpm_status mpm_autotune_config(const mpm_ctx* ctx, int32_t* grid_blocks, float* grid_ms, int32_t* g2p_stage,
                               float* g2p_ms) {
  if (!ctx) return MPM_ERR_INVALID_ARG;
  if (grid_blocks) *grid_blocks = ctx->g.grid_blocks;
  for (int c = 0; c < 4 && grid_ms; ++c) grid_ms[c] = c < (int)ctx->tune.grid.size() ? ctx->tune.grid[c] : 0.0f;
  for (int m = 0; m < 4; ++m) {
    if (g2p_stage) g2p_stage[m] = -1;
    if (g2p_ms) g2p_ms[2 * m] = g2p_ms[2 * m + 1] = 0.0f;
  }
  for (size_t i = 0; i < ctx->g.mats.size(); ++i) {
    const int mat = ctx->g.mats[i].material;
    if (mat < 0 || mat > 3) continue;
    if (g2p_stage) g2p_stage[mat] = ctx->g.mats[i].g2p_stage;
    if (g2p_ms && i < ctx->tune.g2p.size() && ctx->tune.g2p[i].size() == 2) {
      g2p_ms[2 * mat] = ctx->tune.g2p[i][0];
      g2p_ms[2 * mat + 1] = ctx->tune.g2p[i][1];
    }
  }
  return MPM_OK;
}

mpm_status mpm_bin(const float* x, int32_t n, int32_t grid_res, uint32_t* keys, uint32_t* perm, void* stream) {
  if (!x || !keys || !perm || n < 0 || grid_res < 8 || grid_res > 128 || grid_res % 4) return MPM_ERR_INVALID_ARG;
  if (n == 0) return MPM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned *k1 = nullptr, *k2 = nullptr, *v1 = nullptr, *v2 = nullptr, *hist = nullptr;
  bool ok = cudaMalloc(&k1, sizeof(unsigned) * n) == cudaSuccess && cudaMalloc(&k2, sizeof(unsigned) * n) == cudaSuccess &&
            cudaMalloc(&v1, sizeof(unsigned) * n) == cudaSuccess && cudaMalloc(&v2, sizeof(unsigned) * n) == cudaSuccess &&
            cudaMalloc(&hist, sizeof(unsigned) * radix_hist_entries(n)) == cudaSuccess;
  mpm_status res = MPM_OK;
  if (!ok) {
    res = MPM_ERR_OOM;
  } else {
    launch_bin_keys_plain(x, n, grid_res, k1, v1, st);
    cudaMemcpyAsync(keys, k1, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
    int bits = 0;
    for (unsigned long long v = (unsigned long long)(grid_res / 4) * (grid_res / 4) * (grid_res / 4) * 64ull - 1ull; v;
         v >>= 1)
      ++bits;
    unsigned* kk[2] = {k1, k2};
    unsigned* vv[2] = {v1, v2};
    const int cur = radix_sort(kk, vv, n, bits, hist, st);
    cudaMemcpyAsync(perm, vv[cur], sizeof(unsigned) * n, cudaMemcpyDeviceToDevice, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) res = MPM_ERR_CUDA;
  }
  unsigned* ptrs[] = {k1, k2, v1, v2, hist};
  for (unsigned* p : ptrs)
    if (p) cudaFree(p);
  return res;
}

}  // extern "C"
