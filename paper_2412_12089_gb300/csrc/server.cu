// server.cu -- continuous-batching rollout server (mpm_server_* / mpm_submit / mpm_poll).
//
// Requests (an environment spec, its initial state, a horizon of actions, optionally the
// reward adjoints for a gradient) arrive at any time.  A scheduler thread:
//   1. admits queued requests in arrival order while a slot is free and the memory budget
//      (a fraction of device memory) holds their buffers; admission uploads the request's
//      state, actions and reward adjoints once, so its whole rollout stays on the device;
//   2. each tick advances every resident environment in the forward phase by one control
//      step (one launch per stage for all of them, stream A) and every environment in the
//      reverse phase by one reverse control step (stream B), so the two phases overlap;
//   3. retires finished requests: rewards, final positions and (if asked) action
//      gradients go back to host memory, the device buffers are freed and waiters woken.
// A request's result does not depend on what else is resident: every environment keeps its
// own buffers and counters, and the batched kernels never mix environments.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "kernels.h"
#include "mpm.h"
#include "mpm_types.h"

using namespace mpm;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t id = 0;
  mpm_env_spec spec{};
  int T = 0, A = 0;
  bool grad = false;
  std::vector<float> x, v, C, F, actions, rbar;
  std::vector<int32_t> group;
  std::vector<int32_t> fem_tets, fem_group;  // material FEM: the request's mesh
  std::vector<float> fem_rest;
  EnvLayout lay;
  char* mem = nullptr;
  EnvDesc desc{};
  int phase = 0;  // 0 queued, 1 forward, 2 reverse, 3 done
  int steps = 0;  // steps done in the current phase
  bool enter_reverse = false;
  std::vector<float> rewards, agrad, xfinal;
  int status = MPM_OK;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  bool done = false;
};

}  // namespace

struct mpm_server {
  int device = 0;
  double budget = 0;
  int max_resident = 64;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
  std::vector<std::shared_ptr<Req>> resident;  // scheduler thread only
  double used = 0;                             // bytes of resident requests
  bool stop = false;
  std::thread th;
  Group gf, gb;
  cudaStream_t sf = nullptr, sb = nullptr;
  float* io = nullptr;
  size_t io_cap = 0;
  std::string err;
  uint64_t next_id = 1;
  Clock::time_point t0;
};

namespace {

double now_ms(const mpm_server* s) {
  return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

mpm_status sfail(mpm_server* s, mpm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = buf;
  }
  return st;
}

void finish(mpm_server* s, const std::shared_ptr<Req>& r, int status) {
  if (r->mem) cudaFree(r->mem);
  r->mem = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= (double)r->lay.total;
  r->status = status;
  r->phase = 3;
  r->t_finish = now_ms(s);
  r->done = true;
  s->cv_done.notify_all();
}

// Device-side setup of an admitted request (scheduler thread): buffers, state, horizon.
cudaError_t admit(mpm_server* s, Req& r, Group& scratch) {
  cudaError_t e = cudaMalloc(&r.mem, r.lay.total);
  if (e) return e;
  if ((e = cudaMemset(r.mem, 0, r.lay.total))) return e;
  env_fill(r.desc, r.spec, r.lay, r.mem, nullptr, nullptr);
  const size_t P = (size_t)r.spec.n_particles;
  if (s->io_cap < P * (kComp + 1)) {
    if (s->io) cudaFree(s->io);
    s->io = nullptr;
    s->io_cap = 0;
    if ((e = cudaMalloc(&s->io, P * (kComp + 1) * sizeof(float)))) return e;
    s->io_cap = P * (kComp + 1);
  }
  float* io = s->io;
  cudaMemcpy(io, r.x.data(), P * 3 * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(io + P * 3, r.v.data(), P * 3 * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(io + P * 6, r.C.data(), P * 9 * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(io + P * 15, r.F.data(), P * 9 * 4, cudaMemcpyHostToDevice);
  int* gbuf = nullptr;
  if (!r.group.empty()) {
    gbuf = (int*)(io + P * kComp);
    cudaMemcpy(gbuf, r.group.data(), P * 4, cudaMemcpyHostToDevice);
  }
  {
    float q0[kPose];
    initial_pose(r.spec, q0);
    cudaMemcpy(r.desc.pose, q0, sizeof q0, cudaMemcpyHostToDevice);
  }
  if ((e = fem_upload(r.spec, r.desc))) return e;
  if (r.A > 0) cudaMemcpy((void*)r.desc.act_env, r.actions.data(), (size_t)r.T * r.A * 4, cudaMemcpyHostToDevice);
  cudaMemcpy((void*)r.desc.rbar_env, r.rbar.data(), (size_t)r.T * 4, cudaMemcpyHostToDevice);
  // a one-environment group writes the state into slot 0
  std::vector<EnvDesc> d{r.desc};
  std::vector<mpm_env_spec> sp{r.spec};
  if ((e = group_build(scratch, d, sp))) return e;
  launch_set_state(env_launch(scratch, 0, 0), io, io + P * 3, io + P * 6, io + P * 15, gbuf);
  return cudaDeviceSynchronize();
}

// Results of a request whose forward phase ended (final positions, rewards, status bits).
cudaError_t collect_forward(mpm_server* s, Req& r, Group& scratch, int* status_bits) {
  const size_t P = (size_t)r.spec.n_particles;
  std::vector<EnvDesc> d{r.desc};
  std::vector<mpm_env_spec> sp{r.spec};
  cudaError_t e = group_build(scratch, d, sp);
  if (e) return e;
  float* xout = (float*)(r.mem + r.lay.xout);
  launch_get_state(env_launch(scratch, 0, 0), StateRef{REF_LIVE, 0}, xout, nullptr, nullptr, nullptr);
  if ((e = cudaDeviceSynchronize())) return e;
  r.xfinal.resize(P * 3);
  r.rewards.resize(r.T);
  cudaMemcpy(r.xfinal.data(), xout, P * 3 * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(r.rewards.data(), r.desc.rew_env, (size_t)r.T * 4, cudaMemcpyDeviceToHost);
  EnvCtr c;
  cudaMemcpy(&c, r.desc.ctr, sizeof c, cudaMemcpyDeviceToHost);
  *status_bits = c.status;
  (void)s;
  return cudaGetLastError();
}

int status_of(int bits) {
  if (bits & 6) return MPM_ERR_NUMERIC;
  if (bits & 1) return MPM_ERR_DOMAIN;
  return MPM_OK;
}

void scheduler(mpm_server* s) {
  cudaSetDevice(s->device);
  Group scratch;
  bool layout_changed = true;
  for (;;) {
    // ---- admission (arrival order; the head waits until it fits)
    std::vector<std::shared_ptr<Req>> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->resident.empty() && s->pending.empty() && !s->stop)
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      if (s->stop) break;
      while (!s->pending.empty() && (int)(s->resident.size() + admitted.size()) < s->max_resident) {
        auto& r = s->pending.front();
        if (s->used + (double)r->lay.total > s->budget) break;
        s->used += (double)r->lay.total;
        admitted.push_back(r);
        s->pending.pop_front();
      }
    }
    for (auto& r : admitted) {
      cudaError_t e = admit(s, *r, scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        finish(s, r, e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA);
        continue;
      }
      r->t_admit = now_ms(s);
      r->phase = 1;
      r->steps = 0;
      s->resident.push_back(r);
      layout_changed = true;
    }
    if (s->resident.empty()) continue;
    // ---- groups: forward-phase and reverse-phase environments
    std::vector<std::shared_ptr<Req>> fw, bw;
    for (auto& r : s->resident) (r->phase == 1 ? fw : bw).push_back(r);
    if (layout_changed) {
      std::vector<EnvDesc> df, db;
      std::vector<mpm_env_spec> sf, sbv;
      for (auto& r : fw) df.push_back(r->desc), sf.push_back(r->spec);
      for (auto& r : bw) db.push_back(r->desc), sbv.push_back(r->spec);
      if (group_build(s->gf, df, sf) != cudaSuccess || group_build(s->gb, db, sbv) != cudaSuccess) {
        cudaGetLastError();
        for (auto& r : s->resident) finish(s, r, MPM_ERR_OOM);
        s->resident.clear();
        continue;
      }
      layout_changed = false;
    }
    // ---- one tick: forward step (stream A) and reverse step (stream B) overlap
    if (!fw.empty()) enqueue_forward(s->gf, s->sf, true, nullptr, s->gf.A_max, nullptr, false);
    if (!bw.empty()) {
      for (int e = 0; e < (int)bw.size(); ++e)
        if (bw[e]->enter_reverse) {
          const Launch Le = env_launch(s->gb, e, s->sb);
          launch_bwd_init(Le, bw[e]->T);
          launch_adj_in(Le, nullptr, nullptr, nullptr, nullptr);
          bw[e]->enter_reverse = false;
        }
      enqueue_reverse(s->gb, s->sb, nullptr, nullptr, s->gb.n_envs, s->gb.A_max, false);
    }
    cudaError_t ef = cudaStreamSynchronize(s->sf);
    cudaError_t eb = cudaStreamSynchronize(s->sb);
    if (ef != cudaSuccess || eb != cudaSuccess) {
      cudaGetLastError();
      for (auto& r : s->resident) finish(s, r, MPM_ERR_CUDA);
      s->resident.clear();
      layout_changed = true;
      continue;
    }
    // ---- bookkeeping and retirement
    std::vector<std::shared_ptr<Req>> keep;
    for (auto& r : s->resident) {
      r->steps += 1;
      bool retire = false;
      int status = MPM_OK;
      if (r->phase == 1 && r->steps == r->T) {
        int bits = 0;
        if (collect_forward(s, *r, scratch, &bits) != cudaSuccess) {
          cudaGetLastError();
          retire = true;
          status = MPM_ERR_CUDA;
        } else if (r->grad && !(bits & 6)) {
          r->phase = 2;
          r->steps = 0;
          r->enter_reverse = true;
          layout_changed = true;
        } else {
          retire = true;
          status = status_of(bits);
        }
      } else if (r->phase == 2 && r->steps == r->T) {
        r->agrad.resize((size_t)r->T * r->A);
        if (r->A > 0) cudaMemcpy(r->agrad.data(), r->desc.agrad_env, (size_t)r->T * r->A * 4, cudaMemcpyDeviceToHost);
        EnvCtr c;
        cudaMemcpy(&c, r->desc.ctr, sizeof c, cudaMemcpyDeviceToHost);
        retire = true;
        status = status_of(c.status);
      }
      if (retire) {
        finish(s, r, status);
        layout_changed = true;
      } else {
        keep.push_back(r);
      }
    }
    s->resident.swap(keep);
  }
  for (auto& r : s->resident) finish(s, r, MPM_ERR_STATE);
  s->resident.clear();
  scratch.release();
}

}  // namespace

extern "C" {

mpm_status mpm_server_create(const mpm_server_options* opt, mpm_server** out) {
  if (!out) return MPM_ERR_INVALID_ARG;
  *out = nullptr;
  mpm_server_options o{0.8, 64, 0, 0};
  if (opt) o = *opt;
  if (!(o.mem_fraction > 0.0 && o.mem_fraction <= 1.0) || o.max_resident < 1) return MPM_ERR_INVALID_ARG;
  if (o.chunk != 0 && o.chunk != kChunk) return MPM_ERR_INVALID_ARG;
  mpm_server* s = new mpm_server();
  s->device = o.device;
  s->max_resident = o.max_resident;
  s->t0 = Clock::now();
  if (cudaSetDevice(s->device) != cudaSuccess) {
    delete s;
    return MPM_ERR_CUDA;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete s;
    return MPM_ERR_CUDA;
  }
  s->budget = o.mem_fraction * (double)tot;
  if (cudaStreamCreateWithFlags(&s->sf, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->sb, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return MPM_ERR_CUDA;
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return MPM_OK;
}

void mpm_server_destroy(mpm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->pending) {
      r->status = MPM_ERR_STATE;
      r->done = true;
    }
    s->pending.clear();
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  s->gf.release();
  s->gb.release();
  if (s->io) cudaFree(s->io);
  if (s->sf) cudaStreamDestroy(s->sf);
  if (s->sb) cudaStreamDestroy(s->sb);
  delete s;
}

const char* mpm_server_last_error(const mpm_server* s) { return s ? s->err.c_str() : "null server"; }

mpm_status mpm_submit(mpm_server* s, const mpm_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return MPM_ERR_INVALID_ARG;
  const char* bad = check_spec(q->spec);
  if (bad) return sfail(s, MPM_ERR_INVALID_ARG, "invalid %s", bad);
  if (q->horizon < 1 || q->horizon > 100000) return sfail(s, MPM_ERR_INVALID_ARG, "horizon");
  if (!q->x || !q->v || !q->C || !q->F) return sfail(s, MPM_ERR_INVALID_ARG, "x, v, C and F are required");
  const int A = q->spec.n_coll_act + q->spec.n_groups;
  if (A > 0 && !q->actions) return sfail(s, MPM_ERR_INVALID_ARG, "actions are required");
  auto r = std::make_shared<Req>();
  r->spec = q->spec;
  if (q->spec.material == kMatFem) {  // the mesh is read at admission: keep a copy
    r->fem_tets.assign(q->spec.fem_tets, q->spec.fem_tets + 4 * (size_t)q->spec.n_tets);
    r->fem_rest.assign(q->spec.fem_rest, q->spec.fem_rest + 3 * (size_t)q->spec.n_particles);
    if (q->spec.fem_group) r->fem_group.assign(q->spec.fem_group, q->spec.fem_group + q->spec.n_tets);
    r->spec.fem_tets = r->fem_tets.data();
    r->spec.fem_rest = r->fem_rest.data();
    r->spec.fem_group = q->spec.fem_group ? r->fem_group.data() : nullptr;
  }
  r->T = q->horizon;
  r->A = A;
  r->grad = q->want_grad != 0;
  const size_t P = (size_t)q->spec.n_particles;
  r->x.assign(q->x, q->x + P * 3);
  r->v.assign(q->v, q->v + P * 3);
  r->C.assign(q->C, q->C + P * 9);
  r->F.assign(q->F, q->F + P * 9);
  if (q->group) r->group.assign(q->group, q->group + P);
  if (A > 0) r->actions.assign(q->actions, q->actions + (size_t)r->T * A);
  if (q->reward_adj)
    r->rbar.assign(q->reward_adj, q->reward_adj + r->T);
  else
    r->rbar.assign(r->T, 1.0f);
  r->lay = env_layout(r->spec, r->T + 1, r->grad, true, r->T);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((double)r->lay.total > s->budget) {
      s->err = "request exceeds the memory budget";
      return MPM_ERR_BUDGET;
    }
    r->id = s->next_id++;
    r->t_submit = now_ms(s);
    s->tickets[r->id] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_all();
  *ticket = r->id;
  return MPM_OK;
}

static void fill_result(const Req& r, mpm_result* out) {
  out->status = r.status;
  out->horizon = r.T;
  out->action_dim = r.A;
  out->n_particles = r.spec.n_particles;
  out->rewards = r.rewards.empty() ? nullptr : r.rewards.data();
  out->action_grad = (r.grad && !r.agrad.empty()) ? r.agrad.data() : nullptr;
  out->x_final = r.xfinal.empty() ? nullptr : r.xfinal.data();
  out->submit_ms = r.t_submit;
  out->admit_ms = r.t_admit;
  out->finish_ms = r.t_finish;
}

mpm_status mpm_poll(mpm_server* s, uint64_t ticket, mpm_result* out) {
  if (!s) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return MPM_ERR_INVALID_ARG;
  if (!it->second->done) return MPM_NOT_READY;
  if (out) fill_result(*it->second, out);
  return MPM_OK;
}

mpm_status mpm_wait(mpm_server* s, uint64_t ticket, double timeout_ms, mpm_result* out) {
  if (!s) return MPM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return MPM_ERR_INVALID_ARG;
  auto r = it->second;
  const auto deadline = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1000.0));
  while (!r->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return MPM_ERR_TIMEOUT;
  }
  if (out) fill_result(*r, out);
  return MPM_OK;
}

mpm_status mpm_release(mpm_server* s, uint64_t ticket) {
  if (!s) return MPM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return MPM_ERR_INVALID_ARG;
  if (!it->second->done) return MPM_NOT_READY;
  s->tickets.erase(it);
  return MPM_OK;
}

}  // extern "C"
