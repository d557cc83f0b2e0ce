// server.cu -- request server with continuous batching (serving workload;
// the paper solves one problem at a time).
//
// Callers submit steady-flow requests from any thread.  One worker thread
// owns the context's stream and loops:
//   1. admit queued requests while the HBM budget allows (a request is
//      admitted by building its problem; a build that would exceed the
//      context's budget waits for running requests to finish);
//   2. run one outer iteration of every running request together
//      (batch_iterate: one cooperative Krylov launch per solve for all);
//   3. for each request, apply the paper's time-step logic (Sec. 3.2:
//      outer iterations until Delta < tol, tol = 1e-4 then min(1e-4,
//      dt * eps_s)); after a step, test the steady residual; a request
//      that reaches its tolerance (or fails) leaves with its fields copied
//      to host memory and its device memory freed.
// New requests join, and finished ones leave, at outer-iteration
// boundaries, so the device always works on whatever is running.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "abi_guard.cuh"
#include "batch.cuh"
#include "problem.cuh"

using namespace rbffd;

namespace {

using Clock = std::chrono::steady_clock;

double secs(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

struct Request {
  uint64_t id = 0;
  std::vector<double> x, y, nx, ny, ubc, vbc;
  std::vector<int8_t> tag;
  rbffd_problem_desc desc{};
  rbffd_solve_params sp{};
  rbffd_step_params step{};
  Clock::time_point t_arrive, t_admit, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done
  int status = RBFFD_OK;
  rbffd_problem *P = nullptr;
  double tol = 1e-4;
  int outer_in_step = 0;
  int steps = 0;
  int admit_attempts = 0;  // hierarchy uploads tried (the build itself runs once)
  int builds = 0;          // problem builds (clouds, weights, operators) made
  bool admitted = false;   // joined the running batch (t_admit set)
  int64_t outer_total = 0;
  double resid[4] = {1, 1, 1, 0};
  std::vector<double> u, v, p;
};

}  // namespace

struct rbffd_server {
  rbffd_ctx *ctx = nullptr;
  int max_active = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::vector<Request *> running;
  std::unordered_map<uint64_t, Request *> all;
  uint64_t next_id = 1;
  int unfinished = 0;
  bool stop = false;
  int fatal = RBFFD_OK;
  BatchScratch scratch;
  Clock::time_point t0 = Clock::now();  // the clock of rbffd_result admit_s / done_s

  void finish(Request *r, int status) {
    r->status = status;
    if (r->P) {
      if (status == RBFFD_OK) {
        r->u.resize(r->desc.n);
        r->v.resize(r->desc.n);
        r->p.resize(r->desc.n);
        int rc = rbffd_get_field(r->P, RBFFD_FIELD_U, r->u.data());
        if (rc == RBFFD_OK) rc = rbffd_get_field(r->P, RBFFD_FIELD_V, r->v.data());
        if (rc == RBFFD_OK) rc = rbffd_get_field(r->P, RBFFD_FIELD_P, r->p.data());
        if (rc != RBFFD_OK) r->status = rc;
      }
      rbffd_problem_destroy(r->P);
      r->P = nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    r->t_done = Clock::now();
    r->state = 2;
    --unfinished;
    cv_done.notify_all();
  }

  void admit() {
    for (;;) {
      Request *r = nullptr;
      {
        std::lock_guard<std::mutex> g(mu);
        if (queue.empty() || (int)running.size() >= max_active) return;
        r = queue.front();
      }
      // A request whose problem was built on an earlier attempt keeps it:
      // only its hierarchy upload, which found no device memory then, is
      // retried (the clouds, weights, operators and the host part of the
      // hierarchy are not built again).
      int rc = RBFFD_OK;
      if (!r->P) {
        ++r->builds;
        rc = rbffd_problem_create(ctx, &r->desc, &r->P);
      }
      if (rc == RBFFD_OK) {
        ++r->admit_attempts;
        // the hierarchy's device memory counts against the budget now
        rc = rbffd::amg_ready(r->P);
        if (rc == RBFFD_OK) rc = rbffd::compat_ready(r->P);
        if (rc == RBFFD_ENOMEM && !running.empty()) return;  // keep r->P; wait for memory
      } else {
        r->P = nullptr;
        if (rc == RBFFD_ENOMEM && !running.empty()) return;  // wait for memory
      }
      {
        std::lock_guard<std::mutex> g(mu);
        queue.pop_front();
      }
      if (rc != RBFFD_OK) {
        finish(r, rc);  // frees a problem built on the way
        continue;
      }
      r->t_admit = Clock::now();
      r->admitted = true;
      r->state = 1;
      running.push_back(r);
    }
  }

  void step_all() {
    const int m = (int)running.size();
    std::vector<rbffd_problem *> P(m);
    std::vector<const rbffd_step_params *> spv(m);
    for (int i = 0; i < m; ++i) {
      P[i] = running[i]->P;
      spv[i] = &running[i]->step;
    }
    std::vector<double> delta(m);
    std::vector<int> status(m);
    int rc = batch_iterate(scratch, P.data(), m, spv.data(), delta.data(), nullptr,
                           status.data());
    if (rc != RBFFD_OK) {  // a launch-level failure ends every running request
      for (int i = 0; i < m; ++i) finish(running[i], rc);
      running.clear();
      return;
    }
    std::vector<Request *> keep;
    for (int i = 0; i < m; ++i) {
      Request *r = running[i];
      if (status[i] != RBFFD_OK) {
        finish(r, status[i]);
        continue;
      }
      r->outer_in_step++;
      r->outer_total++;
      if (delta[i] < r->tol || r->outer_in_step >= r->sp.max_outer) {
        double change = 0.0;
        int e = problem_step_end(r->P, &change);
        if (e == RBFFD_OK) e = rbffd_steady_residual(r->P, r->resid);
        if (e != RBFFD_OK) {
          finish(r, e);
          continue;
        }
        r->steps++;
        r->outer_in_step = 0;
        r->tol = change < 1e-4 ? change : 1e-4;
        if (steady_done(&r->sp, r->resid[2], change, r->steps)) {
          finish(r, RBFFD_OK);
          continue;
        }
        if (r->steps >= r->sp.max_steps) {
          finish(r, RBFFD_ENOCONV);
          continue;
        }
      }
      keep.push_back(r);
    }
    running.swap(keep);
  }

  void loop() {
    cudaSetDevice(ctx->device);
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop && queue.empty() && running.empty()) return;
        if (queue.empty() && running.empty()) {
          cv_work.wait_for(lk, std::chrono::milliseconds(20));
          continue;
        }
      }
      const int rc = guarded([&] {
        admit();
        if (!running.empty()) step_all();
        return RBFFD_OK;
      });
      if (rc != RBFFD_OK) {  // host memory exhausted: end the running requests
        for (Request *r : running) finish(r, rc);
        running.clear();
      }
    }
  }
};

extern "C" int rbffd_server_create(rbffd_ctx *ctx, const rbffd_server_params *prm,
                                   rbffd_server **out) {
  return guarded([&]() -> int {
    if (!ctx || !out) return RBFFD_EINVAL;
    *out = nullptr;
    RBFFD_CK(cudaSetDevice(ctx->device));
    rbffd_server *s = new rbffd_server();
    s->ctx = ctx;
    ctx_ref(ctx);
    size_t budget = prm ? prm->hbm_budget_bytes : 0;
    if (budget == 0) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = ctx->used.load() + fr / 10 * 8;
    }
    if (budget && (ctx->budget == 0 || budget < ctx->budget)) ctx->budget = budget;
    int cap = krylov_batch_max_ctas(ctx, 2);
    s->max_active = (prm && prm->max_active > 0) ? prm->max_active : cap;
    if (s->max_active > cap) s->max_active = cap;
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_server_submit(rbffd_server *s, const rbffd_problem_desc *d,
                                   const rbffd_solve_params *sp, uint64_t *ticket) {
  return guarded([&]() -> int {
    if (!s || !d || !sp || !ticket || d->n < 1 || !d->x || !d->y || !d->tag || !d->nx || !d->ny ||
        !d->ubc || !d->vbc || sp->max_outer < 1 || sp->max_steps < 1 || !(sp->dt > 0))
      return RBFFD_EINVAL;
    if (d->precision != RBFFD_PREC_FP64 && d->precond == RBFFD_PRECOND_JACOBI) {
      set_error("rbffd_server_submit: a mixed-precision request needs a multigrid p' solver");
      return RBFFD_EINVAL;
    }
    Request *r = new Request();
    const size_t n = d->n;
    // host copies of the inputs (the caller's buffers may go away)
    auto cp = [n](std::vector<double> &v, const double *src) { v.assign(src, src + n); };
    cp(r->x, d->x);
    cp(r->y, d->y);
    cp(r->nx, d->nx);
    cp(r->ny, d->ny);
    cp(r->ubc, d->ubc);
    cp(r->vbc, d->vbc);
    r->tag.assign(d->tag, d->tag + n);
    r->desc = *d;
    r->desc.x = r->x.data();
    r->desc.y = r->y.data();
    r->desc.nx = r->nx.data();
    r->desc.ny = r->ny.data();
    r->desc.ubc = r->ubc.data();
    r->desc.vbc = r->vbc.data();
    r->desc.tag = r->tag.data();
    r->sp = *sp;
    r->step.dt = sp->dt;
    r->step.alpha[0] = 1.5;
    r->step.alpha[1] = -2.0;
    r->step.alpha[2] = 0.5;
    r->step.krylov_tol = sp->krylov_tol;
    r->step.krylov_maxit = sp->krylov_maxit;
    r->t_arrive = Clock::now();
    {
      std::lock_guard<std::mutex> g(s->mu);
      r->id = s->next_id++;
      s->all[r->id] = r;
      s->queue.push_back(r);
      s->unfinished++;
    }
    s->cv_work.notify_one();
    *ticket = r->id;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_server_poll(rbffd_server *s, uint64_t ticket, rbffd_result *res, double *u,
                                 double *v, double *p) {
  return guarded([&]() -> int {
    if (!s || !res) return RBFFD_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return RBFFD_EINVAL;
    Request *r = it->second;
    memset(res, 0, sizeof(*res));
    res->state = r->state;
    res->status = r->status;
    res->steps = r->steps;
    res->outer_iters = r->outer_total;
    for (int k = 0; k < 4; ++k) res->resid[k] = r->resid[k];
    res->admit_attempts = r->admit_attempts;
    res->builds = r->builds;
    res->arrive_s = secs(s->t0, r->t_arrive);
    if (r->admitted) res->admit_s = secs(s->t0, r->t_admit);
    if (r->state == 2) res->done_s = secs(s->t0, r->t_done);
    if (r->admitted) res->queue_s = secs(r->t_arrive, r->t_admit);
    if (r->state == 2) {
      res->latency_s = secs(r->t_arrive, r->t_done);
      if (r->status == RBFFD_OK && !r->u.empty()) {
        const size_t nb = sizeof(double) * r->u.size();
        if (u) memcpy(u, r->u.data(), nb);
        if (v) memcpy(v, r->v.data(), nb);
        if (p) memcpy(p, r->p.data(), nb);
      }
    }
    return RBFFD_OK;
  });
}

extern "C" int rbffd_server_drain(rbffd_server *s) {
  return guarded([&]() -> int {
    if (!s) return RBFFD_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [s] { return s->unfinished == 0; });
    return RBFFD_OK;
  });
}

extern "C" void rbffd_server_destroy(rbffd_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  rbffd_ctx *ctx = s->ctx;
  for (auto &kv : s->all) {
    if (kv.second->P) rbffd_problem_destroy(kv.second->P);
    delete kv.second;
  }
  s->all.clear();
  delete s;  // frees the batch scratch through ctx, still alive here
  ctx_unref(ctx);
}
