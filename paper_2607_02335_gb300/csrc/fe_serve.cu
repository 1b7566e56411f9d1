// fe_serve.cu -- request server with continuous batching of cell-wise CG solves.
//
// Clients submit solves (mesh description, right-hand side, CG options) from any thread.  A
// worker thread owns the GPU work: it admits queued requests in arrival order while a slot is
// free and the request's device-memory estimate fits the budget, builds each admitted problem
// (mesh, geometry, workspace, Jacobi diagonal, right-hand side) and joins it to a running batch.
// FP64 requests join the FP64 batch at once; mixed-precision requests join the mixed batch at its
// next outer-iteration boundary.  Every batch iteration applies the operators of all its problems
// in one persistent launch (fe_batch.cu).  Converged solves retire: the solution is copied to the
// host, the problem's device memory returns to the library pool and its slot frees up for the next
// request.  A problem's arithmetic does not depend on the other problems in its batch, so every
// result is bitwise the same as when it is served alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fe_batch.h"

namespace {

using Clock = std::chrono::steady_clock;
double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Request {
  long long ticket = 0;
  fe_mesh_desc desc;
  std::vector<double> b_host;  // empty: the manufactured sine load (FE_RHS_SINE)
  fe_cg_opts opts;
  bool mixed = false;
  size_t mem = 0;
  double t_arrive = 0.0, t_done = 0.0;
  int state = RQ_QUEUED;
  fe_mesh* mesh = nullptr;
  CgWork* w = nullptr;
  double* b_dev = nullptr;
  double bscale = 1.0;  // the exact power of two the request's system is scaled by
  fe_cg_result result;
  std::vector<double> x_host;
};

// device bytes of one request at its peak (set-up holds the FP64 geometry until the diagonal and
// the copies that the solve reads exist)
size_t estimate_bytes(const fe_mesh_desc& d, bool mixed) {
  const long long n = d.degree + 1;
  const long long ncw = (long long)d.mx * d.my * d.mz * n * n * n;
  size_t per = 0;
  if (d.geom_mode == FE_GEOM_STORED) per += FE_GEO_COMPS * (8 + 8 + (mixed ? 4 : 0));
  per += 6 * 8 + 8 + 4 + 4 + 8;  // FP64 CG vectors, inverse diagonals, 1/mult, b
  if (mixed) per += 6 * 4;
  return (size_t)ncw * per + (size_t)(1 << 20);
}

}  // namespace

struct fe_server {
  size_t budget = 0;
  int max_slots = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<long long, Request*> reqs;
  long long next_ticket = 1;
  size_t mem_used = 0;
  int slots_used = 0;
  bool stop = false;
  fe_status worker_status = FE_OK;
  std::vector<double> latencies;
  double t_first = -1.0, t_last = -1.0;
  long long n_done = 0;
  std::thread worker;
  // worker-owned
  cudaStream_t st = nullptr;
  FeBatch b64, b32;
  std::vector<Request*> run64, run32, pending32;
};

namespace {

fe_status alloc_hsc(FeBatch& B, size_t n) {
  if (B.cap_hsc >= 2 * n && B.hsc) return FE_OK;
  if (B.hsc) cudaFreeHost(B.hsc);
  B.hsc = nullptr;
  const size_t cap = std::max<size_t>(2 * n, 64);
  FE_CUDA(cudaMallocHost(&B.hsc, cap * sizeof(CgScal)), "server scalars");
  B.cap_hsc = cap;
  return FE_OK;
}

// (re)build a batch over the given requests
fe_status rebuild(fe_server* S, FeBatch& B, std::vector<Request*>& run) {
  B.hp.resize(run.size());
  B.active.assign(run.size(), 1);
  B.any_flexible = 0;
  for (size_t i = 0; i < run.size(); ++i) {
    FE_TRY(fe_batch_fill(&B, (int)i, run[i]->mesh, run[i]->w, run[i]->b_dev, &run[i]->opts));
    B.any_flexible |= B.hp[i].flexible;
  }
  FE_TRY(alloc_hsc(B, run.size()));
  return run.empty() ? FE_OK : fe_batch_build(&B);
}

fe_status setup_request(fe_server* S, Request* r) {
  FE_TRY(fe_mesh_create(&r->desc, S->st, &r->mesh));
  FE_TRY(fe_cg_get_work(r->mesh, r->mixed, &r->w));
  FE_TRY(fe_ensure_geometry(r->mesh, FE_F64, false));
  if (r->mixed) FE_TRY(fe_ensure_geometry(r->mesh, FE_F32, false));
  FE_TRY(fe_cg_ensure_diag(r->mesh, r->w, FE_LAPLACE));
  const long long n = r->mesh->ncw;
  FE_TRY(fe_dalloc((void**)&r->b_dev, n * sizeof(double), r->w->st, "server rhs"));
  if (r->b_host.empty()) {
    FE_TRY(fe_rhs(r->mesh, FE_RHS_SINE, r->b_dev, r->w->st));
  } else {
    FE_CUDA(cudaMemcpyAsync(r->b_dev, r->b_host.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                            r->w->st),
            "server rhs upload");
  }
  // the request's system scaled by an exact power of two (fe_cg_rhs_scale); x0 = 0
  FE_TRY(fe_cg_rhs_scale(r->w, r->b_dev, n, &r->bscale));
  FE_TRY(fe_cg_scale(r->b_dev, r->b_dev, r->bscale, n, r->w->st));
  FE_CUDA(cudaMemsetAsync(r->w->x, 0, n * sizeof(double), r->w->st), "server x0");
  FE_CUDA(cudaStreamSynchronize(r->w->st), "server set-up");
  if (r->mesh->d.geom_mode == FE_GEOM_STORED) fe_mesh_drop_geo64(r->mesh, S->st);
  std::vector<double>().swap(r->b_host);
  return FE_OK;
}

void release_request(fe_server* S, Request* r) {
  if (r->mesh) fe_mesh_release_async(r->mesh, S->st);  // also frees the CG workspace
  fe_dfree(r->b_dev, S->st);
  r->mesh = nullptr;
  r->w = nullptr;
  r->b_dev = nullptr;
}

void finish_request(fe_server* S, Request* r, fe_status st, const CgScal* sc) {
  if (sc) {
    r->result.status = (fe_status)sc[0].status;
    r->result.rel_res = sc[0].relres;
    r->result.iters = r->mixed ? sc[1].stall_total : sc[0].iter;
    r->result.outer_iters = r->mixed ? sc[0].iter : 1;
  } else {
    r->result.status = st;
  }
  if (sc && r->w) {
    r->x_host.resize(r->mesh->ncw);
    fe_cg_scale(r->w->x, r->w->x, 1.0 / r->bscale, r->mesh->ncw, S->st);  // exact: a power of two
    cudaMemcpyAsync(r->x_host.data(), r->w->x, r->mesh->ncw * sizeof(double), cudaMemcpyDeviceToHost,
                    S->st);
    cudaStreamSynchronize(S->st);
  }
  release_request(S, r);
  std::lock_guard<std::mutex> lock(S->mu);
  S->mem_used -= r->mem;
  S->slots_used -= 1;
  r->t_done = now_s();
  r->state = RQ_DONE;
  S->latencies.push_back(r->t_done - r->t_arrive);
  S->n_done += 1;
  S->t_last = r->t_done;
  S->cv.notify_all();
}

// set up the joining requests alone (fresh scalars, initial residual, first direction or
// residual check), then add them to the running batch
fe_status join(fe_server* S, FeBatch& B, std::vector<Request*>& run, std::vector<Request*>& news,
               bool mixed) {
  if (news.empty()) return FE_OK;
  {
    FeBatch J;
    J.st = S->st;
    J.own_stream = false;
    FE_TRY(rebuild(S, J, news));
    FE_TRY(fe_batch_start(&J, mixed));
    FE_CUDA(cudaStreamSynchronize(S->st), "join");
  }
  run.insert(run.end(), news.begin(), news.end());
  news.clear();
  return rebuild(S, B, run);
}

// retire finished problems of a batch (scalars already read back)
fe_status retire(fe_server* S, FeBatch& B, std::vector<Request*>& run) {
  std::vector<Request*> keep;
  bool changed = false;
  for (size_t i = 0; i < run.size(); ++i) {
    const CgScal* sc = &B.hsc[2 * i];
    if (sc[0].done) {
      finish_request(S, run[i], FE_OK, sc);
      changed = true;
    } else {
      keep.push_back(run[i]);
    }
  }
  if (!changed) return FE_OK;
  run.swap(keep);
  return rebuild(S, B, run);
}

fe_status step_fp64(fe_server* S, std::vector<Request*>& news) {
  FE_TRY(join(S, S->b64, S->run64, news, false));
  if (S->run64.empty()) return FE_OK;
  for (int k = 0; k < 4; ++k) FE_TRY(fe_batch_iteration<double>(&S->b64, 0, 0));
  FE_TRY(fe_batch_read(&S->b64));
  return retire(S, S->b64, S->run64);
}

// Reliable updates (or, for new requests, the initial residual check) of the given requests alone,
// in a temporary batch; the converged ones go to `leaving`, the others start their next FP32 run
// and go to `cont`.  The requests keep their device state, so the running batch needs no rebuild
// for the ones that continue.
fe_status update_runs(fe_server* S, std::vector<Request*>& reqs, bool fresh,
                      std::vector<Request*>* cont, std::vector<std::pair<Request*, CgScal[2]>>* leaving) {
  std::vector<Request*> go;
  {
    FeBatch J;
    J.st = S->st;
    J.own_stream = false;
    FE_TRY(rebuild(S, J, reqs));
    if (fresh)
      FE_TRY(fe_batch_start(&J, true));
    else
      FE_TRY(fe_batch_inner_finish(&J));
    FE_TRY(fe_batch_read(&J));
    for (size_t i = 0; i < reqs.size(); ++i) {
      const CgScal* sc = &J.hsc[2 * i];
      if (sc[0].done) {
        leaving->emplace_back();
        leaving->back().first = reqs[i];
        leaving->back().second[0] = sc[0];
        leaving->back().second[1] = sc[1];
      } else {
        go.push_back(reqs[i]);
      }
    }
  }
  if (!go.empty()) {
    FeBatch K;
    K.st = S->st;
    K.own_stream = false;
    FE_TRY(rebuild(S, K, go));
    FE_TRY(fe_batch_inner_start(&K));
  }
  cont->insert(cont->end(), go.begin(), go.end());
  return FE_OK;
}

// Mixed requests run their FP32 runs independently: a round advances every running request by
// four FP32 iterations (a request whose run has ended is skipped by the kernels); then the
// requests whose run ended take their reliable update alone and leave converged or start their
// next run, so no request waits for another's run.  New requests join between rounds.
fe_status step_mixed(fe_server* S) {
  std::vector<std::pair<Request*, CgScal[2]>> leaving;
  bool changed = false;
  if (!S->pending32.empty()) {
    std::vector<Request*> news;
    news.swap(S->pending32);
    FE_TRY(update_runs(S, news, true, &S->run32, &leaving));
    changed = true;
  }
  if (!S->run32.empty()) {
    if (changed) FE_TRY(rebuild(S, S->b32, S->run32));
    changed = false;
    for (int k = 0; k < 4; ++k) FE_TRY(fe_batch_iteration<float>(&S->b32, 1, 1));
    FE_TRY(fe_batch_read(&S->b32));
    std::vector<Request*> ended, keep;
    for (size_t i = 0; i < S->run32.size(); ++i)
      (S->b32.hsc[2 * i + 1].done ? ended : keep).push_back(S->run32[i]);
    if (!ended.empty()) {
      const size_t before = leaving.size();
      std::vector<Request*> cont;
      FE_TRY(update_runs(S, ended, false, &cont, &leaving));
      if (leaving.size() > before) {  // the running batch must stop referencing them first
        keep.insert(keep.end(), cont.begin(), cont.end());
        S->run32.swap(keep);
        changed = true;
      }
    }
  }
  if (changed) FE_TRY(rebuild(S, S->b32, S->run32));
  for (auto& l : leaving) finish_request(S, l.first, FE_OK, l.second);
  return FE_OK;
}

void worker_main(fe_server* S) {
  cudaSetDevice(S->device);
  fe_status st = fe_cuda_check(cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking), "server stream");
  if (st == FE_OK) st = fe_batch_prepare();
  S->b64.st = S->b32.st = S->st;
  S->b64.own_stream = S->b32.own_stream = false;
  while (st == FE_OK) {
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      const bool busy = !S->run64.empty() || !S->run32.empty() || !S->pending32.empty();
      if (S->stop && S->queue.empty() && !busy) break;
      while (!S->queue.empty()) {
        Request* r = S->queue.front();
        if (S->slots_used >= S->max_slots || S->mem_used + r->mem > S->budget) break;
        S->queue.pop_front();
        S->slots_used += 1;
        S->mem_used += r->mem;
        r->state = RQ_RUNNING;
        admit.push_back(r);
      }
      if (admit.empty() && !busy) {
        S->cv.wait_for(lock, std::chrono::milliseconds(2));
        continue;
      }
    }
    std::vector<Request*> news64;
    for (Request* r : admit) {
      const fe_status s = setup_request(S, r);
      if (s != FE_OK) {
        finish_request(S, r, s, nullptr);
        continue;
      }
      (r->mixed ? S->pending32 : news64).push_back(r);
    }
    st = step_fp64(S, news64);
    if (st == FE_OK) st = step_mixed(S);
  }
  if (st != FE_OK) {
    std::lock_guard<std::mutex> lock(S->mu);
    S->worker_status = st;
    S->cv.notify_all();
  }
  if (S->st) cudaStreamSynchronize(S->st);
}

}  // namespace

extern "C" fe_status fe_serve_create(size_t mem_budget, int max_slots, int device,
                                     fe_server** out) {
  if (!out || max_slots < 1 || mem_budget == 0) {
    fe_set_error("fe_serve_create: invalid argument");
    return FE_ERR_INVALID;
  }
  *out = nullptr;
  fe_server* S = new (std::nothrow) fe_server();
  if (!S) {
    fe_set_error("fe_serve_create: host allocation failed");
    return FE_ERR_OOM;
  }
  S->budget = mem_budget;
  S->max_slots = max_slots;
  S->device = device;
  S->worker = std::thread(worker_main, S);
  *out = S;
  return FE_OK;
}

extern "C" fe_status fe_serve_submit(fe_server* S, const fe_mesh_desc* desc, const double* b_host,
                                     const fe_cg_opts* opts, long long* ticket) {
  if (!S || !desc || !opts || !ticket) {
    fe_set_error("fe_serve_submit: null argument");
    return FE_ERR_INVALID;
  }
  if (desc->degree < 1 || desc->degree > 7 || desc->mx < 1 || desc->my < 1 || desc->mz < 1 ||
      desc->geom_mode == FE_GEOM_RECOMPUTE || desc->layout != FE_LAYOUT_CELLS ||
      desc->device != S->device) {
    fe_set_error("fe_serve_submit: invalid mesh description");
    return FE_ERR_INVALID;
  }
  if (opts->maxit < 1 || !(opts->rtol >= 0.0) || (opts->mixed != 0 && opts->mixed != FE_F32)) {
    fe_set_error("fe_serve_submit: invalid options");
    return FE_ERR_INVALID;
  }
  Request* r = new (std::nothrow) Request();
  if (!r) {
    fe_set_error("fe_serve_submit: host allocation failed");
    return FE_ERR_OOM;
  }
  r->desc = *desc;
  r->opts = *opts;
  r->opts.history = nullptr;
  r->mixed = opts->mixed == FE_F32;
  r->mem = estimate_bytes(*desc, r->mixed);
  if (r->mem > S->budget) {
    delete r;
    fe_set_error("fe_serve_submit: the request needs more device memory than the budget");
    return FE_ERR_OOM;
  }
  std::memset(&r->result, 0, sizeof(r->result));
  if (b_host) {
    const long long n = (long long)(desc->degree + 1) * (desc->degree + 1) * (desc->degree + 1) *
                        desc->mx * desc->my * desc->mz;
    r->b_host.assign(b_host, b_host + n);
  }
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->worker_status != FE_OK) {
    delete r;
    fe_set_error("fe_serve_submit: the server worker stopped with an error");
    return S->worker_status;
  }
  r->ticket = S->next_ticket++;
  r->t_arrive = now_s();
  if (S->t_first < 0.0) S->t_first = r->t_arrive;
  S->reqs[r->ticket] = r;
  S->queue.push_back(r);
  *ticket = r->ticket;
  S->cv.notify_all();
  return FE_OK;
}

extern "C" fe_status fe_serve_poll(fe_server* S, long long ticket, fe_cg_result* res,
                                   double* x_host) {
  if (!S || !res) {
    fe_set_error("fe_serve_poll: null argument");
    return FE_ERR_INVALID;
  }
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
      fe_set_error("fe_serve_poll: unknown ticket %lld", ticket);
      return FE_ERR_INVALID;
    }
    if (it->second->state != RQ_DONE) {
      if (S->worker_status != FE_OK) return S->worker_status;
      return FE_ERR_BUSY;
    }
    r = it->second;
    S->reqs.erase(it);
  }
  *res = r->result;
  if (x_host && !r->x_host.empty()) std::memcpy(x_host, r->x_host.data(), r->x_host.size() * sizeof(double));
  delete r;
  return FE_OK;
}

extern "C" fe_status fe_serve_stats(fe_server* S, double* p50_s, double* p99_s,
                                    double* solves_per_s) {
  if (!S) {
    fe_set_error("fe_serve_stats: null server");
    return FE_ERR_INVALID;
  }
  std::vector<double> lat;
  double t0, t1;
  long long n;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    lat = S->latencies;
    t0 = S->t_first;
    t1 = S->t_last;
    n = S->n_done;
  }
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    const size_t k = std::min(lat.size() - 1, (size_t)std::ceil(q * lat.size()) - (q > 0 ? 1 : 0));
    std::nth_element(lat.begin(), lat.begin() + k, lat.end());
    return lat[k];
  };
  if (p50_s) *p50_s = pct(0.50);
  if (p99_s) *p99_s = pct(0.99);
  if (solves_per_s) *solves_per_s = (n > 0 && t1 > t0) ? n / (t1 - t0) : 0.0;
  return FE_OK;
}

extern "C" fe_status fe_serve_destroy(fe_server* S) {
  if (!S) return FE_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    for (Request* r : S->queue) {  // never admitted: dropped
      S->reqs.erase(r->ticket);
      delete r;
    }
    S->queue.clear();
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  FeDeviceGuard device_guard;
  device_guard.set(S->device);
  for (auto& kv : S->reqs) {
    if (kv.second->mesh) release_request(S, kv.second);
    delete kv.second;
  }
  const fe_status st = S->worker_status;
  cudaStream_t stream = S->st;
  delete S;  // the batches free their work lists on `stream`
  if (stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  }
  fe_pool_trim();
  return st;
}
