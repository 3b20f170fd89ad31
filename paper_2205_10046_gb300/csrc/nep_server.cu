// Serving: a persistent request loop with iteration-level (continuous) batching
// (include/nep.h, nep_server_*).
//
// Jobs enter a FIFO queue. One scheduler thread owns a library handle and a CUDA stream and
// runs the batched engine: every running job is one structure of a batch, and one iteration
// advances all of them together — one velocity-Verlet (NVE) or FIRE step each, or, in a job's
// first iteration, its initial evaluation (which is all a single-point job needs). Between
// iterations finished jobs leave (their arrays are copied out) and queued jobs join, first
// in first out, while the batch has a free job slot and the admitted jobs' workspace
// estimates fit the memory budget. A job's arithmetic uses only its own structure (own cell
// grid, lists, sums in a fixed order), so its results do not depend on the other jobs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/nep.h"
#include "nep_internal.cuh"

namespace nep {
void set_create_error(const char *msg);
}  // namespace nep

namespace {

// Atoms one batch may hold: a neighbour-list entry packs the atom index with three 3-bit image
// offsets into 32 bits, so the batch's atom index has 23 bits. Admission keeps the running
// jobs' atoms within it (a job alone above it is refused at submission).
constexpr long long kEngineMaxAtoms = 1LL << 23;

struct Job {
  long long id = 0;
  nep_job spec{};
  std::vector<double> pos, vel;
  std::vector<int> types;
  double t_submit = 0, t_start = 0;
  size_t est = 0;
  bool finished = false;  // results delivered; frozen in the batch until the next layout change
};

struct Arrays {
  std::vector<double> pos, force, vel;
};

double now_since(const std::chrono::steady_clock::time_point &t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// The server type stays internal to the library; the C entry points below are exported
// explicitly (a function taking a hidden type would otherwise be hidden too).
#define NEP_SERVER_API __attribute__((visibility("default")))

struct __attribute__((visibility("hidden"))) nep_server {
  // model (deep copy of the parameters)
  nep_params p{};
  std::vector<double> cR, cA, w0, b0, w1, mass;
  nep_server_config cfg{};
  std::chrono::steady_clock::time_point t0;
  // queue and results
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::deque<nep_result> done;
  std::map<long long, Arrays> arrays;
  long long next_id = 1;
  bool stopping = false;
  int running = 0;
  size_t reserved = 0, peak_reserved = 0, peak_workspace = 0;
  long long completed = 0, failed = 0;
  double atom_evals = 0;
  // where the scheduler's time goes (host wall clock)
  long long iterations = 0, relayouts = 0, builds = 0;
  double t_relayout = 0, t_step = 0, t_fetch = 0;
  std::thread scheduler;

  // Device workspace estimate of one job (bytes): its per-atom arrays in the batch,
  // neighbour lists sized for twice the expected neighbour count (the handle grows lists to
  // 2 m + 16 for a largest count m), staging and cell arrays, plus a fixed part.
  size_t estimate(int N, const double *box) const {
    const double det = std::fabs(box[0] * (box[4] * box[8] - box[5] * box[7]) -
                                 box[1] * (box[3] * box[8] - box[5] * box[6]) +
                                 box[2] * (box[3] * box[7] - box[4] * box[6]));
    const double rho = det > 0 ? N / det : 1.0;
    const double skin = p.skin > 0 ? p.skin : 1.0;
    const double pi = 3.14159265358979323846;
    const double nr = 4.0 / 3.0 * pi * std::pow(p.rc_radial + skin, 3) * rho;
    const double na = 4.0 / 3.0 * pi * std::pow(p.rc_angular + skin, 3) * rho;
    const double cap_r = std::min(512.0, 2.0 * std::ceil(1.3 * nr) + 20);
    const double cap_a = std::min(512.0, 2.0 * std::ceil(1.3 * na) + 20);
    const int T = p.n_types;
    const double est = ((p.basis_radial + 2) + 3) / 4 * 4;
    const double per_atom = 16 * 24.0 + 16 * 4.0 + 4.0 * T + 48 + 4.0 * T * est + 9 * cap_r +
                            cap_a * (4 + 4 + 16) + 3 * 4 * 4.0 + 8 + 72;
    return (size_t)(1.25 * per_atom * N) + ((size_t)1 << 20);
  }

  void scheduler_main();
};

// Scheduler: between iterations, finished jobs leave and queued jobs join the batch.
void nep_server::scheduler_main() {
  cudaStream_t s = nullptr;
  nep_handle *h = nullptr;
  int rc = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess ? NEP_OK : NEP_ERR_CUDA;
  std::string setup_error = rc ? "stream creation failed" : "";
  if (rc == NEP_OK) {
    nep::set_thread_alloc_stream(s);
    rc = nep_create(&p, &h);
    if (rc == NEP_OK && cfg.precision) rc = nep_set_precision(h, cfg.precision);
    if (rc != NEP_OK) setup_error = nep_last_error(h);
  }
  std::vector<Job> active;  // in batch order
  bool relaid = false;      // the layout changed since the last iteration (force a build)
  // finished jobs have left `active` but not yet the engine's layout: the next layout change
  // (with the jobs admitted then) keeps only these engine job indices, so one relayout per
  // iteration serves both the leaving and the joining jobs
  bool compact = false;
  std::vector<int> pending_keep;
  auto timed = [](double &acc, auto &&fn) {
    const auto a = std::chrono::steady_clock::now();
    auto r = fn();
    acc += std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
    return r;
  };
  for (;;) {
    // 1. admit queued jobs (first in first out) while a job slot and the budget allow
    std::vector<Job> add;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (active.empty()) cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
      if (stopping) break;
      long long batch_atoms = 0;
      int live = 0;
      for (const Job &j : active)
        if (!j.finished) {
          batch_atoms += j.spec.n_atoms;
          ++live;
        }
      // lazy leaving (compact_every > 0): while jobs run, admit only once a 1/compact_every
      // share of the slots and of the budget is free, so that one layout change takes many
      // jobs in (and the finished ones out)
      const bool gate_open = cfg.compact_every <= 0 || live == 0 ||
                             (cfg.workers - live >= std::max(1, cfg.workers / cfg.compact_every) &&
                              cfg.memory_budget - std::min(reserved, cfg.memory_budget) >=
                                  cfg.memory_budget / (size_t)cfg.compact_every);
      while (gate_open && !queue.empty() && live + (int)add.size() < cfg.workers &&
             batch_atoms + queue.front().spec.n_atoms <= kEngineMaxAtoms &&
             (live == 0 && add.empty() ? true : reserved + queue.front().est <= cfg.memory_budget)) {
        Job j = std::move(queue.front());
        queue.pop_front();
        batch_atoms += j.spec.n_atoms;
        reserved += j.est;
        peak_reserved = std::max(peak_reserved, reserved);
        ++running;
        add.push_back(std::move(j));
      }
    }
    const double t_admit = now_since(t0);
    for (Job &j : add) j.t_start = t_admit;
    auto fail_jobs = [&](std::vector<Job> &jobs, int code, const std::string &msg) {
      std::lock_guard<std::mutex> lk(mu);
      for (Job &j : jobs) {
        nep_result r{};
        r.id = j.id;
        r.kind = j.spec.kind;
        r.n_atoms = j.spec.n_atoms;
        r.status = code;
        r.t_submit = j.t_submit;
        r.t_start = j.t_start;
        r.t_done = now_since(t0);
        r.workspace_est = j.est;
        std::snprintf(r.message, sizeof(r.message), "%s", msg.c_str());
        --running;
        reserved -= j.est;
        ++failed;
        done.push_back(r);
      }
      jobs.clear();
      cv_done.notify_all();
    };
    if (!h) {
      fail_jobs(add, rc ? rc : NEP_ERR_STATE, "server has no handle: " + setup_error);
      continue;
    }
    // 2. new layout: the running jobs, then the admitted ones (and the finished jobs out)
    if (!add.empty() || (compact && !active.empty())) {
      // any layout change also drops the finished jobs still frozen in the batch
      std::vector<int> keep;
      if (compact) keep = pending_keep;
      else
        for (size_t k = 0; k < active.size(); ++k) keep.push_back((int)k);
      {
        std::vector<int> live_keep;
        std::vector<Job> still;
        for (size_t k = 0; k < active.size(); ++k)
          if (!active[k].finished) {
            live_keep.push_back(keep[k]);
            still.push_back(std::move(active[k]));
          }
        keep = std::move(live_keep);
        active = std::move(still);
      }
      compact = false;
      std::vector<nep::EngineJob> in;
      for (Job &j : add) {
        nep::EngineJob e{};
        e.kind = j.spec.kind;
        e.n = j.spec.n_atoms;
        e.n_steps = j.spec.n_steps;
        std::memcpy(e.box, j.spec.box, sizeof(e.box));
        e.dt = j.spec.dt_fs;
        e.fmax = j.spec.fmax;
        e.pos = j.pos.data();
        e.vel = (j.spec.kind == NEP_JOB_NVE && !j.vel.empty()) ? j.vel.data() : nullptr;
        e.types = j.types.data();
        in.push_back(e);
      }
      size_t target = 0;
      for (const Job &j : active) target += j.est;
      for (const Job &j : add) target += j.est;
      const int r = timed(t_relayout, [&] { return nep::engine_relayout(h, keep, in, s, target); });
      {
        std::lock_guard<std::mutex> lk(mu);
        ++relayouts;
      }
      if (r != NEP_OK) {
        // the admitted jobs cannot be laid out: report them and restore the running batch
        const std::string msg = nep_last_error(h);
        fail_jobs(add, r, msg);
        if (nep::engine_relayout(h, keep, {}, s) != NEP_OK) fail_jobs(active, r, msg);
        relaid = true;
        continue;
      }
      for (Job &j : add) active.push_back(std::move(j));
      add.clear();
      relaid = true;
    }
    if (active.empty()) {
      if (compact) nep::engine_relayout(h, {}, {}, s);  // the last jobs left: an empty layout
      compact = false;
      continue;
    }
    // 3. a chunk of iterations of every job: one while jobs wait or start (to admit and finish
    // them promptly), else up to the first job's completion (at most 32)
    int n_iter = 32;
    {
      // one iteration when a queued job could join now (lazy leaving: once the slots and the
      // budget have the free share that opens admission)
      std::lock_guard<std::mutex> lk(mu);
      if (!queue.empty()) {
        int live = 0;
        for (const Job &j : active) live += j.finished ? 0 : 1;
        const bool slot_free = cfg.compact_every <= 0
                                   ? live < cfg.workers
                                   : cfg.workers - live >= std::max(1, cfg.workers / cfg.compact_every);
        const bool budget_free = cfg.compact_every <= 0 ||
                                 cfg.memory_budget - std::min(reserved, cfg.memory_budget) >=
                                     cfg.memory_budget / (size_t)cfg.compact_every;
        if (slot_free && budget_free) n_iter = 1;
      }
    }
    for (size_t k = 0; k < active.size() && n_iter > 1; ++k) {
      if (active[k].finished) continue;  // frozen until the next layout change
      const nep::EngineSlot &sl = nep::engine_slot(h, (int)k);
      if (sl.phase != 1) n_iter = 1;
      else n_iter = std::max(1, std::min(n_iter, sl.n_steps - sl.steps_done));
    }
    // at least min_chunk iterations: a job that finishes earlier is frozen (phase 2: no drift,
    // no kick, its energy, forces and state unchanged) until the chunk ends
    n_iter = std::max(n_iter, std::min(cfg.min_chunk, 32));
    const int r = timed(t_step, [&] { return nep::engine_step(h, s, n_iter, relaid); });
    relaid = false;
    {
      std::lock_guard<std::mutex> lk(mu);
      iterations += n_iter;
      builds = nep::engine_builds(h);
    }
    {
      const size_t ws = nep::workspace_bytes(h);
      std::lock_guard<std::mutex> lk(mu);
      peak_workspace = std::max(peak_workspace, ws);
    }
    if (r != NEP_OK) {
      std::vector<Job> unfinished;
      for (Job &j : active)
        if (!j.finished) unfinished.push_back(std::move(j));
      active.clear();
      fail_jobs(unfinished, r, nep_last_error(h));
      nep::engine_relayout(h, {}, {}, s);
      compact = false;
      continue;
    }
    const auto t_fetch0 = std::chrono::steady_clock::now();
    // 4. finished jobs hand over their results at once; they leave the batch at the next
    // layout change, or now if (lazy leaving) they make up a 1/compact_every share of it
    std::vector<nep_result> out;
    std::vector<std::pair<long long, Arrays>> outa;
    double evals = 0;
    int n_finished = 0;
    for (size_t k = 0; k < active.size(); ++k) {
      Job &j = active[k];
      if (j.finished) {
        ++n_finished;
        continue;
      }
      const nep::EngineSlot &sl = nep::engine_slot(h, (int)k);
      if (sl.phase != 2) continue;
      nep_result res{};
      res.id = j.id;
      res.kind = j.spec.kind;
      res.n_atoms = j.spec.n_atoms;
      res.steps = sl.steps_done;
      res.energy = nep::engine_energy(h, (int)k);
      std::memcpy(res.virial, nep::engine_virial(h, (int)k), sizeof(res.virial));
      res.t_submit = j.t_submit;
      res.t_start = j.t_start;
      res.workspace_est = j.est;
      const size_t n3 = 3 * (size_t)j.spec.n_atoms;
      Arrays a;
      a.pos.resize(n3);
      a.force.resize(n3);
      if (j.spec.kind == NEP_JOB_NVE) a.vel.resize(n3);
      res.status = nep::engine_fetch(h, (int)k, a.pos.data(), a.force.data(), a.vel.empty() ? nullptr : a.vel.data(), s);
      if (res.status != NEP_OK) std::snprintf(res.message, sizeof(res.message), "%s", nep_last_error(h));
      res.workspace_used = nep::workspace_bytes(h);
      res.t_done = now_since(t0);
      evals += (double)j.spec.n_atoms * (1 + sl.steps_done);
      out.push_back(res);
      outa.emplace_back(j.id, std::move(a));
      j.finished = true;
      ++n_finished;
    }
    if (!out.empty()) {
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t q = 0; q < out.size(); ++q) {
          --running;
          reserved -= out[q].workspace_est;
          if (out[q].status == NEP_OK) {
            ++completed;
            arrays.emplace(outa[q].first, std::move(outa[q].second));
          } else {
            ++failed;
          }
          done.push_back(out[q]);
        }
        atom_evals += evals;
      }
      cv_done.notify_all();
    }
    if (n_finished > 0 && (cfg.compact_every <= 0 || n_finished == (int)active.size() ||
                           n_finished * cfg.compact_every >= (int)active.size())) {
      // the engine keeps the finished jobs until the next layout change (step 2)
      std::vector<int> keep;
      std::vector<Job> still;
      for (size_t k = 0; k < active.size(); ++k)
        if (!active[k].finished) {
          keep.push_back((int)k);
          still.push_back(std::move(active[k]));
        }
      active = std::move(still);
      pending_keep = std::move(keep);
      compact = true;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      t_fetch += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_fetch0).count();
    }
  }
  if (h) {
    nep::release_workspace(h);
    nep_destroy(h);
  }
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
}

extern "C" {

NEP_SERVER_API int nep_server_create(const nep_params *params, const nep_server_config *cfg, nep_server **out) {
  if (!out || !params || !cfg) {
    nep::set_create_error("null argument");
    return NEP_ERR_ARG;
  }
  *out = nullptr;
  if (cfg->workers < 1 || cfg->workers > 65536 || cfg->memory_budget == 0 ||
      cfg->precision < 0 || cfg->precision > 2 || cfg->compact_every < 0 || cfg->compact_every > 1024 ||
      cfg->min_chunk < 0 || cfg->min_chunk > 32) {
    nep::set_create_error("need 1 <= workers <= 65536, memory_budget > 0, precision 0, 1 or 2, "
                          "0 <= compact_every <= 1024, 0 <= min_chunk <= 32");
    return NEP_ERR_ARG;
  }
  if (!params->mass) {
    nep::set_create_error("serving needs params->mass (FIRE and NVE jobs)");
    return NEP_ERR_ARG;
  }
  // validate the parameters once on this thread (and find the compiled shape)
  nep_handle *probe = nullptr;
  int rc = nep_create(params, &probe);
  if (rc) return rc;
  const int n_des = nep_n_des(probe);
  nep_destroy(probe);
  nep_server *s = new nep_server();
  s->cfg = *cfg;
  s->p = *params;
  const int T = params->n_types;
  const size_t ncr = (size_t)T * T * (params->n_max_radial + 1) * (params->basis_radial + 1);
  const size_t nca = (size_t)T * T * (params->n_max_angular + 1) * (params->basis_angular + 1);
  s->cR.assign(params->c_radial, params->c_radial + ncr);
  s->cA.assign(params->c_angular, params->c_angular + nca);
  s->w0.assign(params->w0, params->w0 + (size_t)params->n_neuron * n_des);
  s->b0.assign(params->b0, params->b0 + params->n_neuron);
  s->w1.assign(params->w1, params->w1 + params->n_neuron);
  s->mass.assign(params->mass, params->mass + T);
  s->p.c_radial = s->cR.data();
  s->p.c_angular = s->cA.data();
  s->p.w0 = s->w0.data();
  s->p.b0 = s->b0.data();
  s->p.w1 = s->w1.data();
  s->p.mass = s->mass.data();
  // keep freed stream-ordered memory in the pool (up to the budget) for the next layouts
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = cfg->memory_budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  s->t0 = std::chrono::steady_clock::now();
  s->scheduler = std::thread([s, dev] {
    cudaSetDevice(dev);
    s->scheduler_main();
  });
  *out = s;
  return NEP_OK;
}

NEP_SERVER_API int nep_server_submit(nep_server *s, const nep_job *job, long long *id) {
  if (!s || !job) return NEP_ERR_ARG;
  const int N = job->n_atoms;
  if (job->kind < NEP_JOB_SINGLE || job->kind > NEP_JOB_NVE || N < 1 || !job->pos || !job->types)
    return NEP_ERR_ARG;
  if (job->kind != NEP_JOB_SINGLE && (job->n_steps < 0 || !(job->dt_fs > 0) || !std::isfinite(job->dt_fs)))
    return NEP_ERR_ARG;
  if (job->kind == NEP_JOB_FIRE && !(job->fmax >= 0)) return NEP_ERR_ARG;
  // checked here, so that a bad job cannot stop the batch it would join
  for (int i = 0; i < N; ++i)
    if (job->types[i] < 0 || job->types[i] >= s->p.n_types) return NEP_ERR_ARG;
  for (size_t k = 0; k < 3 * (size_t)N; ++k)
    if (!std::isfinite(job->pos[k])) return NEP_ERR_NONFINITE;
  Job j;
  j.spec = *job;
  j.pos.assign(job->pos, job->pos + 3 * (size_t)N);
  j.types.assign(job->types, job->types + N);
  if (job->kind == NEP_JOB_NVE && job->vel) j.vel.assign(job->vel, job->vel + 3 * (size_t)N);
  j.spec.pos = nullptr;
  j.spec.types = nullptr;
  j.spec.vel = nullptr;
  if (N > kEngineMaxAtoms) return NEP_ERR_UNSUPPORTED;
  j.est = s->estimate(N, job->box);
  if (j.est > s->cfg.memory_budget) return NEP_ERR_OOM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return NEP_ERR_STATE;
    j.id = s->next_id++;
    j.t_submit = now_since(s->t0);
    if (id) *id = j.id;
    s->queue.push_back(std::move(j));
  }
  s->cv_work.notify_all();
  return NEP_OK;
}

NEP_SERVER_API int nep_server_wait(nep_server *s, double timeout_s, nep_result *out) {
  if (!s || !out) return NEP_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return !s->done.empty(); };
  if (timeout_s < 0) s->cv_done.wait(lk, ready);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return NEP_ERR_TIMEOUT;
  *out = s->done.front();
  s->done.pop_front();
  return NEP_OK;
}

NEP_SERVER_API int nep_server_arrays(nep_server *s, long long id, double *pos, double *force, double *vel) {
  if (!s) return NEP_ERR_ARG;
  Arrays a;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->arrays.find(id);
    if (it == s->arrays.end()) return NEP_ERR_ARG;
    a = std::move(it->second);
    s->arrays.erase(it);
  }
  if (pos) std::memcpy(pos, a.pos.data(), a.pos.size() * sizeof(double));
  if (force) std::memcpy(force, a.force.data(), a.force.size() * sizeof(double));
  if (vel) {
    if (a.vel.empty()) std::memset(vel, 0, a.pos.size() * sizeof(double));
    else std::memcpy(vel, a.vel.data(), a.vel.size() * sizeof(double));
  }
  return NEP_OK;
}

NEP_SERVER_API int nep_server_stats_get(nep_server *s, nep_server_stats *out) {
  if (!s || !out) return NEP_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int)s->queue.size();
  out->running = s->running;
  out->completed = s->completed;
  out->failed = s->failed;
  out->bytes_reserved = s->reserved;
  out->peak_bytes_reserved = s->peak_reserved;
  out->peak_workspace_bytes = s->peak_workspace;
  out->atom_evaluations = s->atom_evals;
  out->iterations = s->iterations;
  out->relayouts = s->relayouts;
  out->relayout_seconds = s->t_relayout;
  out->step_seconds = s->t_step;
  out->fetch_seconds = s->t_fetch;
  out->builds = s->builds;
  return NEP_OK;
}

NEP_SERVER_API int nep_server_destroy(nep_server *s) {
  if (!s) return NEP_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  if (s->scheduler.joinable()) s->scheduler.join();
  delete s;
  return NEP_OK;
}

}  // extern "C"
