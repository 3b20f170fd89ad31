// Serving: a persistent request loop with continuous batching (include/nep.h, nep_server_*).
//
// Jobs enter a FIFO queue. A pool of workers (one host thread, one non-blocking CUDA stream
// and one library handle each) takes the head job as soon as a worker is free and the job's
// estimated device workspace fits into what the running jobs leave of the memory budget.
// A worker runs its job to completion with the ordinary entry points (nep_compute, md_init
// + md_run, md_init + fire_run), so a job computes exactly what it computes alone; the
// overlap of jobs on the device comes from the workers' streams. Every device buffer of a
// worker is a stream-ordered allocation on its stream and is released when the job ends,
// so neither growing nor freeing a workspace synchronises the device.
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

namespace nep {
void set_thread_alloc_stream(cudaStream_t s);
void release_workspace(nep_handle *h);
size_t workspace_bytes(nep_handle *h);
void set_create_error(const char *msg);
cudaError_t stream_sync(cudaStream_t s);
}  // namespace nep

namespace {

struct Job {
  long long id = 0;
  nep_job spec{};
  std::vector<double> pos, vel;
  std::vector<int> types;
  double t_submit = 0;
  size_t est = 0;
};

struct Arrays {
  std::vector<double> pos, force, vel;
};

// Stream-ordered device buffer of a worker.
struct WBuf {
  void *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes, cudaStream_t s) {
    if (bytes <= n && p) return cudaSuccess;
    release(s);
    cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s);
    if (e == cudaSuccess) n = bytes;
    else p = nullptr;
    return e;
  }
  void release(cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
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
  int n_des = 0;
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
  size_t reserved = 0, peak_reserved = 0;
  long long completed = 0, failed = 0;
  double atom_evals = 0;
  std::vector<std::thread> workers;
  int worker_error = 0;
  std::string worker_message;

  // Device workspace estimate of one job (bytes): per-atom arrays of the handle and the
  // worker, neighbour lists sized for twice the expected neighbour count (the handle grows
  // lists to 2 m + 16 for a largest count m) and the cell grid, plus a fixed part.
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
    const double per_atom = 11 * 24.0 + 5 * 24.0 + 12 * 4.0 + 4.0 * T + 16 + 4.0 * T * est + 4 * cap_r +
                            cap_a * (4 + 4 + 16) + 3 * 4 * 4.0 + 16 + 72;
    return (size_t)(1.25 * per_atom * N) + ((size_t)8 << 20);
  }

  void worker_main(int w);
  void run_job(nep_handle *h, cudaStream_t s, Job &job, nep_result &r, Arrays &out, WBuf *buf, double &evals_out);
};

#define SCK(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      r.status = e_ == cudaErrorMemoryAllocation ? NEP_ERR_OOM : NEP_ERR_CUDA;                     \
      std::snprintf(r.message, sizeof(r.message), "%s", cudaGetErrorString(e_));                   \
      return;                                                                                      \
    }                                                                                              \
  } while (0)

#define SNEP(call)                                                                                 \
  do {                                                                                             \
    const int rc_ = (call);                                                                        \
    if (rc_ != NEP_OK) {                                                                           \
      r.status = rc_;                                                                              \
      std::snprintf(r.message, sizeof(r.message), "%s", nep_last_error(h));                        \
      return;                                                                                      \
    }                                                                                              \
  } while (0)

void nep_server::run_job(nep_handle *h, cudaStream_t s, Job &job, nep_result &r, Arrays &out, WBuf *buf,
                         double &evals_out) {
  const nep_job &J = job.spec;
  const int N = J.n_atoms;
  const size_t b3 = sizeof(double) * 3 * (size_t)N;
  enum { POS, TYPES, VEL, F, E, W, NBUF };
  SCK(buf[POS].ensure(b3, s));
  SCK(buf[TYPES].ensure(sizeof(int) * (size_t)N, s));
  SCK(buf[VEL].ensure(b3, s));
  SCK(buf[F].ensure(b3, s));
  SCK(buf[E].ensure(sizeof(double), s));
  SCK(buf[W].ensure(9 * sizeof(double), s));
  double *d_pos = static_cast<double *>(buf[POS].p), *d_vel = static_cast<double *>(buf[VEL].p);
  double *d_F = static_cast<double *>(buf[F].p), *d_E = static_cast<double *>(buf[E].p);
  double *d_W = static_cast<double *>(buf[W].p);
  int *d_types = static_cast<int *>(buf[TYPES].p);
  SCK(cudaMemcpyAsync(d_pos, job.pos.data(), b3, cudaMemcpyHostToDevice, s));
  SCK(cudaMemcpyAsync(d_types, job.types.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, s));
  r.steps = 0;
  double evals = 1;
  out.vel.clear();
  if (J.kind == NEP_JOB_FIRE) {
    SNEP(md_init(h, N, d_pos, d_types, J.box, nullptr, s));
    int steps = 0;
    SNEP(fire_run(h, J.n_steps, J.dt_fs, J.fmax, nullptr, &steps, s));
    SNEP(md_get_state(h, d_pos, nullptr, nullptr, s));
    r.steps = steps;
    evals += 1 + steps;
  } else if (J.kind == NEP_JOB_NVE) {
    if (!job.vel.empty()) SCK(cudaMemcpyAsync(d_vel, job.vel.data(), b3, cudaMemcpyHostToDevice, s));
    SNEP(md_init(h, N, d_pos, d_types, J.box, job.vel.empty() ? nullptr : d_vel, s));
    SNEP(md_run(h, J.n_steps, J.dt_fs, std::max(1, J.n_steps), nullptr, s));
    SNEP(md_get_state(h, d_pos, d_vel, nullptr, s));
    r.steps = J.n_steps;
    evals += 1 + J.n_steps;
    out.vel.resize(3 * (size_t)N);
  }
  // the final state: energy, forces and virial at the final positions
  SNEP(nep_compute(h, N, d_pos, d_types, J.box, nullptr, d_E, d_F, nullptr, d_W, s));
  out.pos.resize(3 * (size_t)N);
  out.force.resize(3 * (size_t)N);
  SCK(cudaMemcpyAsync(out.pos.data(), d_pos, b3, cudaMemcpyDeviceToHost, s));
  SCK(cudaMemcpyAsync(out.force.data(), d_F, b3, cudaMemcpyDeviceToHost, s));
  if (!out.vel.empty()) SCK(cudaMemcpyAsync(out.vel.data(), d_vel, b3, cudaMemcpyDeviceToHost, s));
  SCK(cudaMemcpyAsync(&r.energy, d_E, sizeof(double), cudaMemcpyDeviceToHost, s));
  SCK(cudaMemcpyAsync(r.virial, d_W, 9 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SCK(nep::stream_sync(s));
  r.workspace_used = nep::workspace_bytes(h);
  for (int k = 0; k < NBUF; ++k) r.workspace_used += buf[k].n;
  // the positions are reported wrapped into the cell, like md_get_state
  if (J.kind == NEP_JOB_SINGLE) {
    const double *H = J.box;
    double inv[9];
    const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                       H[2] * (H[3] * H[7] - H[4] * H[6]);
    inv[0] = (H[4] * H[8] - H[5] * H[7]) / det;
    inv[1] = (H[2] * H[7] - H[1] * H[8]) / det;
    inv[2] = (H[1] * H[5] - H[2] * H[4]) / det;
    inv[3] = (H[5] * H[6] - H[3] * H[8]) / det;
    inv[4] = (H[0] * H[8] - H[2] * H[6]) / det;
    inv[5] = (H[2] * H[3] - H[0] * H[5]) / det;
    inv[6] = (H[3] * H[7] - H[4] * H[6]) / det;
    inv[7] = (H[1] * H[6] - H[0] * H[7]) / det;
    inv[8] = (H[0] * H[4] - H[1] * H[3]) / det;
    for (int i = 0; i < N; ++i) {
      double *x = out.pos.data() + 3 * (size_t)i, sf[3];
      for (int b = 0; b < 3; ++b) {
        sf[b] = x[0] * inv[b] + x[1] * inv[3 + b] + x[2] * inv[6 + b];
        sf[b] -= std::floor(sf[b]);
      }
      for (int b = 0; b < 3; ++b) x[b] = sf[0] * H[b] + sf[1] * H[3 + b] + sf[2] * H[6 + b];
    }
  }
  r.status = NEP_OK;
  evals_out = evals * N;
}

void nep_server::worker_main(int w) {
  cudaStream_t s = nullptr;
  nep_handle *h = nullptr;
  int rc = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess ? NEP_OK : NEP_ERR_CUDA;
  if (rc == NEP_OK) {
    nep::set_thread_alloc_stream(s);
    rc = nep_create(&p, &h);
    if (rc == NEP_OK && cfg.precision) rc = nep_set_precision(h, cfg.precision);
  }
  if (rc != NEP_OK) {
    std::lock_guard<std::mutex> lk(mu);
    worker_error = rc;
    worker_message = "worker " + std::to_string(w) + ": " + nep_last_error(h);
  }
  WBuf buf[6];
  for (;;) {
    Job job;
    {
      std::unique_lock<std::mutex> lk(mu);
      // FIFO admission: the head job starts when a worker is free (this one) and its workspace
      // fits next to the running jobs' (a job always starts when nothing else runs)
      cv_work.wait(lk, [&] {
        return stopping || (!queue.empty() && (running == 0 || reserved + queue.front().est <= cfg.memory_budget));
      });
      if (stopping) break;
      job = std::move(queue.front());
      queue.pop_front();
      ++running;
      reserved += job.est;
      peak_reserved = std::max(peak_reserved, reserved);
    }
    cv_work.notify_all();  // the next head may fit as well
    nep_result r{};
    r.id = job.id;
    r.kind = job.spec.kind;
    r.n_atoms = job.spec.n_atoms;
    r.t_submit = job.t_submit;
    r.t_start = now_since(t0);
    r.workspace_est = job.est;
    Arrays out;
    double evals = 0;
    if (!h) {
      r.status = worker_error ? worker_error : NEP_ERR_STATE;
      std::snprintf(r.message, sizeof(r.message), "%s", "worker has no handle");
    } else {
      run_job(h, s, job, r, out, buf, evals);
      nep::release_workspace(h);
      for (auto &b : buf) b.release(s);
      nep::stream_sync(s);
    }
    r.t_done = now_since(t0);
    {
      std::lock_guard<std::mutex> lk(mu);
      --running;
      reserved -= job.est;
      if (r.status == NEP_OK) {
        ++completed;
        atom_evals += evals;
        arrays.emplace(r.id, std::move(out));
      } else {
        ++failed;
      }
      done.push_back(r);
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (h) {
    nep::release_workspace(h);
    nep_destroy(h);
  }
  for (auto &b : buf) b.release(s);
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
  if (cfg->workers < 1 || cfg->workers > 256 || cfg->memory_budget == 0 || (cfg->precision != 0 && cfg->precision != 1)) {
    nep::set_create_error("need 1 <= workers <= 256, memory_budget > 0, precision 0 or 1");
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
  nep_server *s = new nep_server();
  s->n_des = nep_n_des(probe);
  nep_destroy(probe);
  s->cfg = *cfg;
  s->p = *params;
  const int T = params->n_types;
  const size_t ncr = (size_t)T * T * (params->n_max_radial + 1) * (params->basis_radial + 1);
  const size_t nca = (size_t)T * T * (params->n_max_angular + 1) * (params->basis_angular + 1);
  s->cR.assign(params->c_radial, params->c_radial + ncr);
  s->cA.assign(params->c_angular, params->c_angular + nca);
  s->w0.assign(params->w0, params->w0 + (size_t)params->n_neuron * s->n_des);
  s->b0.assign(params->b0, params->b0 + params->n_neuron);
  s->w1.assign(params->w1, params->w1 + params->n_neuron);
  s->mass.assign(params->mass, params->mass + T);
  s->p.c_radial = s->cR.data();
  s->p.c_angular = s->cA.data();
  s->p.w0 = s->w0.data();
  s->p.b0 = s->b0.data();
  s->p.w1 = s->w1.data();
  s->p.mass = s->mass.data();
  // keep freed stream-ordered memory in the pool (up to the budget) for the next jobs
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = cfg->memory_budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  s->t0 = std::chrono::steady_clock::now();
  for (int w = 0; w < cfg->workers; ++w)
    s->workers.emplace_back([s, w, dev] {
      cudaSetDevice(dev);
      s->worker_main(w);
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
  Job j;
  j.spec = *job;
  j.pos.assign(job->pos, job->pos + 3 * (size_t)N);
  j.types.assign(job->types, job->types + N);
  if (job->kind == NEP_JOB_NVE && job->vel) j.vel.assign(job->vel, job->vel + 3 * (size_t)N);
  j.spec.pos = nullptr;
  j.spec.types = nullptr;
  j.spec.vel = nullptr;
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
  out->atom_evaluations = s->atom_evals;
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
  for (auto &t : s->workers) t.join();
  delete s;
  return NEP_OK;
}

}  // extern "C"
