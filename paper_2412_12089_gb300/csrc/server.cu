// server.cu -- continuous-batching rollout server (mpm_server_* / mpm_submit / mpm_poll).
//
// Requests (an environment spec, its initial state, a horizon of actions, optionally the
// reward adjoints for a gradient) arrive at any time.  A scheduler thread:
//   1. enqueues one control step of every resident environment in the forward phase (one
//      launch per stage for all of them, stream A) and, independently, one reverse control
//      step of every environment in the reverse phase (stream B): each lane starts its next
//      tick as soon as its last one has finished, so the two phases overlap;
//   2. while that runs, admits queued requests in arrival order as long as a slot is free
//      and the memory budget (a fraction of device memory) holds their buffers: their
//      buffers are carved from the server's device pool and their state, actions and reward
//      adjoints uploaded on a third stream (C), once, so each whole rollout stays on the
//      device; they join the resident set at the next tick;
//   3. when a lane's tick has finished, retires its finished requests: rewards, final
//      positions and (if asked) action gradients go back to host memory, the buffers go back
//      to the pool and waiters are woken; requests that asked for gradients move from the
//      forward lane to the reverse lane.
// The pool grows by cudaMalloc up to the budget and is freed only when the server is
// destroyed, so admissions and retirements make no cudaMalloc or cudaFree (a cudaFree
// synchronises the whole device and would stall the streams of the running requests).
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
#include <map>
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

// Device memory of the admitted requests: chunks taken with cudaMalloc as needed, up to the
// budget, carved first-fit into 256-byte aligned blocks and coalesced when given back.
struct Pool {
  struct Chunk {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free;  // offset -> bytes
  };
  std::vector<Chunk> chunks;
  size_t reserved = 0;
  static constexpr size_t kAlign = 256;
  static constexpr size_t kMinChunk = size_t(1) << 30;

  static size_t round(size_t n) { return (std::max<size_t>(n, 1) + kAlign - 1) / kAlign * kAlign; }

  char* take(size_t n) {
    n = round(n);
    for (auto& c : chunks)
      for (auto it = c.free.begin(); it != c.free.end(); ++it)
        if (it->second >= n) {
          const size_t off = it->first, left = it->second - n;
          c.free.erase(it);
          if (left) c.free[off + n] = left;
          return c.base + off;
        }
    return nullptr;
  }
  void give(char* p, size_t n) {
    n = round(n);
    for (auto& c : chunks) {
      if (p < c.base || p >= c.base + c.size) continue;
      size_t off = (size_t)(p - c.base);
      auto nx = c.free.lower_bound(off);
      if (nx != c.free.end() && off + n == nx->first) {  // merge with the next block
        n += nx->second;
        nx = c.free.erase(nx);
      }
      if (nx != c.free.begin()) {  // merge with the previous block
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
          pv->second += n;
          return;
        }
      }
      c.free[off] = n;
      return;
    }
  }
  // A new chunk that holds at least n bytes, if the budget allows it.
  cudaError_t grow(size_t n, double budget) {
    n = round(n);
    size_t want = std::max(n, kMinChunk);
    if ((double)(reserved + want) > budget) want = n;
    if ((double)(reserved + want) > budget) return cudaErrorMemoryAllocation;
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    Chunk c;
    c.base = p;
    c.size = want;
    c.free[0] = want;
    chunks.push_back(std::move(c));
    reserved += want;
    return cudaSuccess;
  }
  char* alloc(size_t n, double budget) {
    char* p = take(n);
    if (!p && grow(n, budget) == cudaSuccess) p = take(n);
    return p;
  }
  bool idle() const {
    for (auto& c : chunks)
      if (c.free.size() != 1 || c.free.begin()->second != c.size) return false;
    return true;
  }
  void release() {  // only with nothing carved out and no work in flight
    for (auto& c : chunks) cudaFree(c.base);
    chunks.clear();
    reserved = 0;
  }
};

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
  char* io = nullptr;  // upload staging (caller-order state), given back once uploaded
  size_t io_bytes = 0;
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
  double used = 0;                             // bytes of resident requests
  bool stop = false;
  std::thread th;
  Group gf, gb;
  cudaStream_t sf = nullptr, sb = nullptr, su = nullptr;
  Pool pool;  // scheduler thread only
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
  if (r->mem) s->pool.give(r->mem, r->lay.total);
  r->mem = nullptr;
  if (r->io) s->pool.give(r->io, r->io_bytes);
  r->io = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= (double)r->lay.total;
  r->status = status;
  r->phase = 3;
  r->t_finish = now_ms(s);
  r->done = true;
  s->cv_done.notify_all();
}

// Device-side setup of an admitted request (scheduler thread), enqueued on the upload
// stream: buffers carved from the pool (the caller checked that they fit), zeroed, then
// the state, horizon arrays and poses uploaded and the state laid into slot 0.  The caller
// synchronises the upload stream.
cudaError_t admit(mpm_server* s, Req& r, Group& scratch) {
  const size_t P = (size_t)r.spec.n_particles;
  cudaStream_t su = s->su;
  cudaError_t e;
  if ((e = cudaMemsetAsync(r.mem, 0, r.lay.total, su))) return e;
  env_fill(r.desc, r.spec, r.lay, r.mem, nullptr, nullptr);
  float* io = reinterpret_cast<float*>(r.io);
  if ((e = cudaMemcpyAsync(io, r.x.data(), P * 3 * 4, cudaMemcpyHostToDevice, su)) ||
      (e = cudaMemcpyAsync(io + P * 3, r.v.data(), P * 3 * 4, cudaMemcpyHostToDevice, su)) ||
      (e = cudaMemcpyAsync(io + P * 6, r.C.data(), P * 9 * 4, cudaMemcpyHostToDevice, su)) ||
      (e = cudaMemcpyAsync(io + P * 15, r.F.data(), P * 9 * 4, cudaMemcpyHostToDevice, su)))
    return e;
  int* gbuf = nullptr;
  if (!r.group.empty()) {
    gbuf = (int*)(io + P * kComp);
    if ((e = cudaMemcpyAsync(gbuf, r.group.data(), P * 4, cudaMemcpyHostToDevice, su))) return e;
  }
  float q0[kPose];
  initial_pose(r.spec, q0);
  if ((e = cudaMemcpyAsync(r.desc.pose, q0, sizeof q0, cudaMemcpyHostToDevice, su))) return e;
  if (r.A > 0 &&
      (e = cudaMemcpyAsync((void*)r.desc.act_env, r.actions.data(), (size_t)r.T * r.A * 4, cudaMemcpyHostToDevice, su)))
    return e;
  if ((e = cudaMemcpyAsync((void*)r.desc.rbar_env, r.rbar.data(), (size_t)r.T * 4, cudaMemcpyHostToDevice, su)))
    return e;
  // q0 lives on this stack frame: the copies must finish before it goes
  if ((e = cudaStreamSynchronize(su))) return e;
  if ((e = fem_upload(r.spec, r.desc))) return e;
  // a one-environment group writes the state into slot 0
  std::vector<EnvDesc> d{r.desc};
  std::vector<mpm_env_spec> sp{r.spec};
  if ((e = group_build(scratch, d, sp))) return e;
  launch_set_state(env_launch(scratch, 0, su), io, io + P * 3, io + P * 6, io + P * 15, gbuf);
  return cudaStreamSynchronize(su);
}

// Results of a request whose forward phase ended (final positions, rewards, status bits).
cudaError_t collect_forward(mpm_server* s, Req& r, Group& scratch, int* status_bits) {
  const size_t P = (size_t)r.spec.n_particles;
  std::vector<EnvDesc> d{r.desc};
  std::vector<mpm_env_spec> sp{r.spec};
  cudaError_t e = group_build(scratch, d, sp);
  if (e) return e;
  float* xout = (float*)(r.mem + r.lay.xout);
  launch_get_state(env_launch(scratch, 0, s->su), StateRef{REF_LIVE, 0}, xout, nullptr, nullptr, nullptr);
  if ((e = cudaStreamSynchronize(s->su))) return e;
  r.xfinal.resize(P * 3);
  r.rewards.resize(r.T);
  cudaMemcpy(r.xfinal.data(), xout, P * 3 * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(r.rewards.data(), r.desc.rew_env, (size_t)r.T * 4, cudaMemcpyDeviceToHost);
  EnvCtr c;
  cudaMemcpy(&c, r.desc.ctr, sizeof c, cudaMemcpyDeviceToHost);
  *status_bits = c.status;
  return cudaGetLastError();
}

int status_of(int bits) {
  if (bits & 6) return MPM_ERR_NUMERIC;
  if (bits & 1) return MPM_ERR_DOMAIN;
  return MPM_OK;
}

// Take queued requests (arrival order; the head waits until it fits) and upload them on
// stream C while the tick runs.  Returns the requests that will join at the next tick.
std::vector<std::shared_ptr<Req>> admit_pending(mpm_server* s, Group& scratch, size_t resident) {
  std::vector<std::shared_ptr<Req>> admitted;
  for (;;) {
    std::shared_ptr<Req> r;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->pending.empty() || resident + admitted.size() >= (size_t)s->max_resident) break;
      r = s->pending.front();
      if (s->used + (double)r->lay.total > s->budget) break;
    }
    const size_t P = (size_t)r->spec.n_particles;
    r->io_bytes = P * (kComp + 1) * sizeof(float);
    r->mem = s->pool.alloc(r->lay.total, s->budget + (double)r->io_bytes);
    r->io = r->mem ? s->pool.alloc(r->io_bytes, s->budget + (double)r->io_bytes) : nullptr;
    if (!r->mem || !r->io) {  // no contiguous room now: wait for retirements
      if (r->mem) s->pool.give(r->mem, r->lay.total);
      if (r->io) s->pool.give(r->io, r->io_bytes);
      r->mem = r->io = nullptr;
      if (resident + admitted.size() == 0 && s->pool.idle()) {
        // nothing runs and the pool is empty, yet fragmented or too small: start it over
        s->pool.release();
        r->mem = s->pool.alloc(r->lay.total, s->budget + (double)r->io_bytes);
        r->io = r->mem ? s->pool.alloc(r->io_bytes, s->budget + (double)r->io_bytes) : nullptr;
      }
      if (!r->mem || !r->io) {
        if (r->mem) s->pool.give(r->mem, r->lay.total);
        r->mem = nullptr;
        if (resident + admitted.size() == 0) {  // it can never be placed
          {
            std::lock_guard<std::mutex> lk(s->mu);
            s->pending.pop_front();
            s->used += (double)r->lay.total;
          }
          finish(s, r, MPM_ERR_OOM);
          continue;
        }
        break;
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->pending.pop_front();
      s->used += (double)r->lay.total;
    }
    cudaError_t e = admit(s, *r, scratch);
    s->pool.give(r->io, r->io_bytes);  // uploaded (or failed): the staging goes back
    r->io = nullptr;
    if (e != cudaSuccess) {
      cudaGetLastError();
      finish(s, r, MPM_ERR_CUDA);
      continue;
    }
    r->t_admit = now_ms(s);
    admitted.push_back(r);
  }
  return admitted;
}

// A lane's tick as a captured CUDA graph while the lane's group stays the same: the first tick
// after a change runs directly, the second is captured, later ones replay it (the step index
// and tape positions live in device counters, so a replay advances like a direct launch).
struct LaneGraph {
  cudaGraphExec_t exec = nullptr;
  int stable = 0;  // ticks run since the group last changed
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    stable = 0;
  }
  template <class Body>
  cudaError_t run(bool changed, cudaStream_t st, Body body) {
    if (changed) reset();
    if (stable >= 1) {
      if (!exec) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          body(st);
          if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) {
            if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
          }
          if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        if (!exec) {  // capture failed: stay with direct launches for this group
          stable = -1000000;
          body(st);
          return cudaGetLastError();
        }
      }
      return cudaGraphLaunch(exec, st);
    }
    body(st);
    ++stable;
    return cudaGetLastError();
  }
};

// Forward and reverse environments run as two lanes, each on its own stream with its own
// group: a lane enqueues its next tick as soon as its last one has finished, so a long reverse
// tick does not hold up the forward lane (or the other way round).  Requests whose forward
// phase ends wait for the reverse lane's next tick to join it; admitted requests join the
// forward lane at its next tick.
void scheduler(mpm_server* s) {
  cudaSetDevice(s->device);
  Group scratch;
  std::vector<std::shared_ptr<Req>> fw, bw, to_bw, incoming;
  bool fw_busy = false, bw_busy = false, fw_changed = true, bw_changed = true;
  LaneGraph fg, bg;
  cudaEvent_t ev_f = nullptr, ev_b = nullptr;
  cudaEventCreateWithFlags(&ev_f, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev_b, cudaEventDisableTiming);
  auto lanes = [&]() { return fw.size() + bw.size() + to_bw.size(); };
  auto fail_all = [&](std::vector<std::shared_ptr<Req>>& v, int status) {
    for (auto& r : v) finish(s, r, status);
    v.clear();
  };
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (lanes() == 0 && incoming.empty() && s->pending.empty() && !s->stop)
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      if (s->stop) break;
    }
    // ---- forward lane: bookkeeping of its finished tick, then its next tick
    if (fw_busy && cudaEventQuery(ev_f) != cudaErrorNotReady) {
      fw_busy = false;
      if (cudaEventSynchronize(ev_f) != cudaSuccess) {
        cudaGetLastError();
        fail_all(fw, MPM_ERR_CUDA);
        fw_changed = true;
      } else {
        std::vector<std::shared_ptr<Req>> keep;
        for (auto& r : fw) {
          if (++r->steps < r->T) {
            keep.push_back(r);
            continue;
          }
          fw_changed = true;
          int bits = 0;
          if (collect_forward(s, *r, scratch, &bits) != cudaSuccess) {
            cudaGetLastError();
            finish(s, r, MPM_ERR_CUDA);
          } else if (r->grad && !(bits & 6)) {
            r->phase = 2;
            r->steps = 0;
            r->enter_reverse = true;
            to_bw.push_back(r);
          } else {
            finish(s, r, status_of(bits));
          }
        }
        fw.swap(keep);
      }
    }
    if (!fw_busy) {
      for (auto& r : incoming) {
        r->phase = 1;
        r->steps = 0;
        fw.push_back(r);
        fw_changed = true;
      }
      incoming.clear();
      const bool rebuilt = !fw.empty() && fw_changed;
      if (rebuilt) {
        std::vector<EnvDesc> d;
        std::vector<mpm_env_spec> sp;
        for (auto& r : fw) d.push_back(r->desc), sp.push_back(r->spec);
        if (group_build(s->gf, d, sp) != cudaSuccess) {
          cudaGetLastError();
          fail_all(fw, MPM_ERR_OOM);
        }
        fw_changed = false;
      }
      if (!fw.empty()) {
        if (fg.run(rebuilt, s->sf, [&](cudaStream_t st) {
              enqueue_forward(s->gf, st, true, nullptr, s->gf.A_max, nullptr, false);
            }) != cudaSuccess) {
          cudaGetLastError();
        }
        cudaEventRecord(ev_f, s->sf);
        fw_busy = true;
      }
    }
    // ---- reverse lane
    if (bw_busy && cudaEventQuery(ev_b) != cudaErrorNotReady) {
      bw_busy = false;
      if (cudaEventSynchronize(ev_b) != cudaSuccess) {
        cudaGetLastError();
        fail_all(bw, MPM_ERR_CUDA);
        bw_changed = true;
      } else {
        std::vector<std::shared_ptr<Req>> keep;
        for (auto& r : bw) {
          if (++r->steps < r->T) {
            keep.push_back(r);
            continue;
          }
          bw_changed = true;
          r->agrad.resize((size_t)r->T * r->A);
          if (r->A > 0) cudaMemcpy(r->agrad.data(), r->desc.agrad_env, (size_t)r->T * r->A * 4, cudaMemcpyDeviceToHost);
          EnvCtr c;
          cudaMemcpy(&c, r->desc.ctr, sizeof c, cudaMemcpyDeviceToHost);
          finish(s, r, status_of(c.status));
        }
        bw.swap(keep);
      }
    }
    if (!bw_busy) {
      for (auto& r : to_bw) {
        bw.push_back(r);
        bw_changed = true;
      }
      to_bw.clear();
      const bool rebuilt = !bw.empty() && bw_changed;
      if (rebuilt) {
        std::vector<EnvDesc> d;
        std::vector<mpm_env_spec> sp;
        for (auto& r : bw) d.push_back(r->desc), sp.push_back(r->spec);
        if (group_build(s->gb, d, sp) != cudaSuccess) {
          cudaGetLastError();
          fail_all(bw, MPM_ERR_OOM);
        }
        bw_changed = false;
      }
      if (!bw.empty()) {
        // a request's first reverse tick starts its pass (only on ticks after a change)
        for (int e = 0; e < (int)bw.size(); ++e)
          if (bw[e]->enter_reverse) {
            const Launch Le = env_launch(s->gb, e, s->sb);
            launch_bwd_init(Le, bw[e]->T);
            launch_adj_in(Le, nullptr, nullptr, nullptr, nullptr);
            bw[e]->enter_reverse = false;
          }
        if (bg.run(rebuilt, s->sb, [&](cudaStream_t st) {
              enqueue_reverse(s->gb, st, nullptr, nullptr, s->gb.n_envs, s->gb.A_max, false);
            }) != cudaSuccess) {
          cudaGetLastError();
        }
        cudaEventRecord(ev_b, s->sb);
        bw_busy = true;
      }
    }
    // ---- admissions upload on stream C while the lanes run; then wait for either lane
    for (;;) {
      if (incoming.empty()) incoming = admit_pending(s, scratch, lanes());
      const bool f_done = !fw_busy || cudaEventQuery(ev_f) != cudaErrorNotReady;
      const bool b_done = !bw_busy || cudaEventQuery(ev_b) != cudaErrorNotReady;
      if (!fw_busy && !bw_busy) break;  // nothing in flight: back to the top (idle wait)
      if ((fw_busy && f_done) || (bw_busy && b_done)) break;
      if (!fw_busy && !incoming.empty()) break;  // the idle forward lane can start them
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) break;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  cudaStreamSynchronize(s->sf);
  cudaStreamSynchronize(s->sb);
  cudaGetLastError();
  fail_all(incoming, MPM_ERR_STATE);
  fail_all(fw, MPM_ERR_STATE);
  fail_all(bw, MPM_ERR_STATE);
  fail_all(to_bw, MPM_ERR_STATE);
  if (ev_f) cudaEventDestroy(ev_f);
  if (ev_b) cudaEventDestroy(ev_b);
  fg.reset();
  bg.reset();
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
      cudaStreamCreateWithFlags(&s->sb, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->su, cudaStreamNonBlocking) != cudaSuccess) {
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
  s->pool.release();
  if (s->sf) cudaStreamDestroy(s->sf);
  if (s->sb) cudaStreamDestroy(s->sb);
  if (s->su) cudaStreamDestroy(s->su);
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
