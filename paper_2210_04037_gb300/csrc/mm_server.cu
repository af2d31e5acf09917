// Served runs with continuous batching.  A scheduler thread owns the GPU
// work: it admits queued runs while the device memory they need fits a
// budget (creating their grids), steps every admitted run together (one
// batch per group of runs sharing dimension, precision, material layout and
// CFL number, each group on its own stream so the groups overlap on the
// device), and retires finished runs (primitive fields to host memory, grid
// freed), which lets the next queued runs in.  Runs submitted while others
// are on the GPU join at the next tick.  A batched member computes exactly
// what the same grid computes alone, so a run's result does not depend on
// the mix it was served in.  Built on the public C ABI (grids, batches).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "mm_internal.h"
#include "mmfrac.h"

namespace {

typedef std::chrono::steady_clock Clock;

struct Run {
  int64_t id = 0;
  mm_grid_desc desc;
  std::vector<mm_material> mats;
  std::vector<double> prim;
  std::vector<float> phi0;
  mm_init init;
  int n_steps = 0;
  double cfl = 0.0;
  size_t bytes = 0;
  long long ncell = 0;
  int nfield = 0;
  // progress (scheduler thread until finished)
  mm_grid* g = nullptr;
  long long steps_done = 0;
  double t_sim = 0.0;
  int status = MM_OK;
  std::string msg;
  bool finished = false;
  double t_submit = 0.0, t_admit = -1.0, t_done = -1.0;
  std::vector<double> result;
};

typedef std::shared_ptr<Run> RunP;
typedef std::tuple<int, int, int, int, double> GroupKey;  // dim, precision, nmat, nhist, cfl

struct Group {
  std::vector<RunP> members;
  mm_batch* batch = nullptr;
  cudaStream_t stream = nullptr;
  int q = 0;
};

int plastic_count(const mm_material* m, int n) {
  int h = 0;
  for (int l = 0; l < n; ++l) h += m[l].plasticity == MM_PL_JOHNSON_COOK;
  return h;
}

}  // namespace

struct mm_server {
  size_t budget = 0, used = 0;
  int quantum = 8;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<RunP> pending;
  std::map<int64_t, RunP> runs;  // submitted and not yet collected
  int64_t next_id = 1;
  bool stop = false;
  long long admitted = 0, retired = 0;
  // scheduler thread only
  std::vector<RunP> active;
  std::map<GroupKey, Group> groups;
  cudaStream_t admit_stream = nullptr;
  Clock::time_point t0;
  std::thread worker;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void finish(mm_server* s, const RunP& r, int status) {
  if (r->g) {
    if (status == MM_OK) {
      r->result.resize((size_t)r->nfield * r->ncell);
      mm_status st = mm_read_fields(r->g, ~0ull, 1, r->result.data(), r->result.size());
      if (st != MM_OK) {
        status = st;
        r->msg = mm_last_error();
        r->result.clear();
      }
    }
    mm_destroy(r->g);
    r->g = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  r->status = status;
  r->finished = true;
  r->t_done = s->now();
  s->used -= r->bytes;
  ++s->retired;
  s->cv_done.notify_all();
}

void fail_run(mm_server* s, const RunP& r, int status) {
  r->msg = mm_last_error();
  finish(s, r, status);
}

// Rebuild the batch of every group whose membership changed.
bool regroup(mm_server* s) {
  std::map<GroupKey, std::vector<RunP>> want;
  for (const RunP& r : s->active)
    want[GroupKey(r->desc.dim, r->desc.precision, r->desc.n_materials,
                  plastic_count(r->mats.data(), (int)r->mats.size()), r->cfl)]
        .push_back(r);
  for (auto it = s->groups.begin(); it != s->groups.end();) {
    auto w = want.find(it->first);
    const bool same = w != want.end() && w->second == it->second.members;
    if (!same && it->second.batch) {
      mm_batch_destroy(it->second.batch);
      it->second.batch = nullptr;
      it->second.members.clear();
    }
    if (w == want.end()) {
      if (it->second.stream) cudaStreamDestroy(it->second.stream);
      it = s->groups.erase(it);
    } else {
      ++it;
    }
  }
  for (auto& kv : want) {
    Group& gr = s->groups[kv.first];
    if (gr.batch) continue;
    if (!gr.stream && cudaStreamCreateWithFlags(&gr.stream, cudaStreamNonBlocking) != cudaSuccess)
      return false;
    std::vector<mm_grid*> gs;
    for (const RunP& r : kv.second) gs.push_back(r->g);
    if (mm_batch_create(gs.data(), (int)gs.size(), gr.stream, &gr.batch) != MM_OK) return false;
    gr.members = kv.second;
  }
  return true;
}

void serve(mm_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<RunP> admit;
    std::vector<RunP> cancelled;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty())
        s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
      if (s->stop) {
        for (RunP& r : s->pending) cancelled.push_back(r);
        s->pending.clear();
      }
      // first come, first served, while the device memory fits
      while (!s->pending.empty() && s->used + s->pending.front()->bytes <= s->budget) {
        admit.push_back(s->pending.front());
        s->used += s->pending.front()->bytes;
        s->pending.pop_front();
        ++s->admitted;
      }
    }
    for (RunP& r : cancelled) {
      r->msg = "cancelled: the server was destroyed before the run was admitted";
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = MM_ESTATE;
      r->finished = true;
      r->t_done = s->now();
      s->cv_done.notify_all();
    }
    for (RunP& r : admit) {
      r->t_admit = s->now();
      mm_status st = mm_create_grid(&r->desc, s->admit_stream, &r->g);
      if (st == MM_OK) st = mm_set_materials(r->g, r->mats.data(), (int)r->mats.size(), &r->init);
      if (st != MM_OK) {
        fail_run(s, r, st);
        continue;
      }
      if (r->n_steps == 0) {
        finish(s, r, MM_OK);
        continue;
      }
      s->active.push_back(r);
    }
    if (s->active.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop && s->pending.empty()) break;
      continue;
    }
    if (!regroup(s)) {
      // a batch could not be built: fail the runs rather than spin
      for (RunP& r : s->active) fail_run(s, r, MM_ECUDA);
      s->active.clear();
      regroup(s);
      continue;
    }
    // one tick: every group advances by its quantum, all enqueued before any wait
    for (auto& kv : s->groups) {
      Group& gr = kv.second;
      long long q = s->quantum;
      for (const RunP& r : gr.members) q = std::min(q, (long long)r->n_steps - r->steps_done);
      gr.q = (int)q;
      if (mm_batch_step(gr.batch, gr.q, std::get<4>(kv.first)) != MM_OK) gr.q = -1;
    }
    std::vector<RunP> still;
    for (auto& kv : s->groups) {
      Group& gr = kv.second;
      cudaStreamSynchronize(gr.stream);
      for (const RunP& r : gr.members) {
        mm_step_info info;
        mm_status st = gr.q < 0 ? MM_ECUDA : mm_synchronize(r->g, &info);
        if (st != MM_OK) {
          fail_run(s, r, st);
          continue;
        }
        r->steps_done += gr.q;
        r->t_sim = info.t;
        if (r->steps_done >= r->n_steps)
          finish(s, r, MM_OK);
        else
          still.push_back(r);
      }
    }
    s->active.swap(still);
  }
  for (auto& kv : s->groups) {
    if (kv.second.batch) mm_batch_destroy(kv.second.batch);
    if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
  }
  s->groups.clear();
}

}  // namespace

mm_status mm_server_create(size_t memory_budget, int steps_per_tick, mm_server** out) {
  if (!out) {
    mm_internal_set_error("mm_server_create: null argument");
    return MM_EINVAL;
  }
  *out = nullptr;
  int dev = 0;
  size_t free_b = 0, total_b = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    mm_internal_set_error("mm_server_create: no CUDA device");
    return MM_ECUDA;
  }
  mm_server* s = new mm_server();
  s->device = dev;
  s->budget = memory_budget ? memory_budget : free_b / 10 * 9;
  s->quantum = steps_per_tick > 0 ? steps_per_tick : 8;
  s->t0 = Clock::now();
  if (cudaStreamCreateWithFlags(&s->admit_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    mm_internal_set_error("mm_server_create: cudaStreamCreate failed");
    return MM_ECUDA;
  }
  s->worker = std::thread(serve, s);
  *out = s;
  return MM_OK;
}

mm_status mm_server_submit(mm_server* s, const mm_grid_desc* desc, const mm_material* mats,
                           int n_mat, const mm_init* init, int n_steps, double cfl,
                           int64_t* id) {
  if (!s || !desc || !mats || !init || !init->prim || !id) {
    mm_internal_set_error("mm_server_submit: null argument");
    return MM_EINVAL;
  }
  if (desc->dim < 1 || desc->dim > 3 || n_mat != desc->n_materials || n_mat != 2 || n_steps < 0 ||
      !(cfl > 0.0) || !(cfl <= 1.0) || mats[0].eos == MM_EOS_VOID ||
      mats[1].eos == MM_EOS_VOID || plastic_count(mats, n_mat) > 1 ||
      (desc->precision != MM_FP64 && desc->precision != MM_FP32_SPLIT)) {
    mm_internal_set_error(
        "mm_server_submit: dim 1..3, two materials (no void, at most one plastic), n_steps >= 0, "
        "cfl in (0, 1] and a known precision are required");
    return MM_EINVAL;
  }
  RunP r = std::make_shared<Run>();
  r->desc = *desc;
  r->mats.assign(mats, mats + n_mat);
  r->ncell = 1;
  for (int k = 0; k < desc->dim; ++k) {
    if (desc->n[k] < 2) {
      mm_internal_set_error("mm_server_submit: n[k] >= 2 required");
      return MM_EINVAL;
    }
    r->ncell *= desc->n[k];
  }
  const int dim = desc->dim, nF = dim == 1 ? 3 : (dim == 2 ? 5 : 9);
  r->nfield = (n_mat - 1) + n_mat + dim + 1 + nF + 2 * plastic_count(mats, n_mat) + dim;
  r->prim.assign(init->prim, init->prim + (size_t)r->nfield * r->ncell);
  long long np = 0;
  if (init->phi0) {
    np = 1;
    for (int k = 0; k < dim; ++k) np *= init->phi0_n[k] > 0 ? init->phi0_n[k] : 0;
    r->phi0.assign(init->phi0, init->phi0 + np);
  }
  r->init = *init;
  r->init.prim = r->prim.data();
  r->init.phi0 = init->phi0 ? r->phi0.data() : nullptr;
  r->n_steps = n_steps;
  r->cfl = cfl;
  // device bytes of the grid: two state copies, the FP64 staging fields, the lattice
  const size_t per = desc->precision == MM_FP64 ? 8 * (size_t)r->nfield : 4 * ((size_t)r->nfield + 1) + 8;
  r->bytes = (size_t)r->ncell * (2 * per + 8 * (size_t)r->nfield) + 4 * (size_t)np + (1u << 20);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    mm_internal_set_error("mm_server_submit: the server is shutting down");
    return MM_ESTATE;
  }
  if (r->bytes > s->budget) {
    mm_internal_set_error("mm_server_submit: the run needs more device memory than the budget");
    return MM_EINVAL;
  }
  r->id = s->next_id++;
  r->t_submit = s->now();
  s->runs[r->id] = r;
  s->pending.push_back(r);
  *id = r->id;
  s->cv_work.notify_all();
  return MM_OK;
}

mm_status mm_server_wait(mm_server* s, int64_t id, int timeout_ms, mm_run_info* info,
                         double* host_dst, size_t dst_len) {
  if (!s) {
    mm_internal_set_error("mm_server_wait: null server");
    return MM_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->runs.find(id);
  if (it == s->runs.end()) {
    mm_internal_set_error("mm_server_wait: unknown or already collected run");
    return MM_EINVAL;
  }
  RunP r = it->second;
  auto done = [&] { return r->finished; };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, done);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    mm_internal_set_error("mm_server_wait: the run has not finished within the timeout");
    return MM_ETIMEOUT;
  }
  if (info) {
    info->id = r->id;
    info->status = r->status;
    info->nfield = r->nfield;
    info->ncell = r->ncell;
    info->steps_done = r->steps_done;
    info->t = r->t_sim;
    info->submit_s = r->t_submit;
    info->admit_s = r->t_admit;
    info->done_s = r->t_done;
  }
  if (r->status != MM_OK) {
    mm_internal_set_error(r->msg.c_str());
    s->runs.erase(it);
    return (mm_status)r->status;
  }
  if (host_dst) {
    if (dst_len < r->result.size()) {
      mm_internal_set_error("mm_server_wait: destination smaller than nfield x ncell doubles");
      return MM_EINVAL;
    }
    std::memcpy(host_dst, r->result.data(), sizeof(double) * r->result.size());
    s->runs.erase(it);
  }
  return MM_OK;
}

mm_status mm_server_stats(mm_server* s, mm_server_info* info) {
  if (!s || !info) {
    mm_internal_set_error("mm_server_stats: null argument");
    return MM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  info->budget_bytes = s->budget;
  info->used_bytes = s->used;
  info->pending = (int64_t)s->pending.size();
  info->admitted = s->admitted;
  info->retired = s->retired;
  return MM_OK;
}

mm_status mm_server_destroy(mm_server* s) {
  if (!s) return MM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->admit_stream) cudaStreamDestroy(s->admit_stream);
  delete s;
  return MM_OK;
}
