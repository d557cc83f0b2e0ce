// batch.cu -- many independent flow problems advanced together: one outer
// iteration of every active member per call, with the two Krylov solves of
// all members in one cooperative launch each (k_bicgstab_batch: each member
// gets its own consecutive CTAs and synchronises only among them, so members
// iterate independently and one member's grid-exchange latency is hidden
// behind the others' work).  The row kernels of the outer iteration are a
// few microseconds per member and run per member on the same stream.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "abi_guard.cuh"
#include "batch.cuh"
#include "fgmres.cuh"
#include "krylov_dev.cuh"
#include "ops.cuh"
#include "problem.cuh"

using namespace rbffd;

namespace {

// Per member result of one batched outer iteration, gathered on the device.
struct MemberOut {
  double delta;
  double relres[3];
  int iters[3];
  int status[3];
};

__global__ void k_gather_out(int m, IterRecord *const *recs, const KrylovOut *const *kouts,
                             MemberOut *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  out[i].delta = recs[i]->delta;
  for (int k = 0; k < 3; ++k) {
    out[i].relres[k] = kouts[i][k].relres;
    out[i].iters[k] = kouts[i][k].iters;
    out[i].status[k] = kouts[i][k].status;
  }
}

int status_of(int s) {
  switch (s) {
    case KRY_OK: return RBFFD_OK;
    case KRY_NOCONV: return RBFFD_ENOCONV;
    case KRY_DIVERGED: return RBFFD_EDIVERGED;
    case KRY_TIMEOUT: return RBFFD_ETIMEOUT;
    default: return RBFFD_ECUDA;
  }
}

}  // namespace

namespace rbffd {

void BatchScratch::drop_graph() {
  if (exec) cudaGraphExecDestroy(exec);
  exec = nullptr;
  key.clear();
  graph_launches = 0;
}

BatchScratch::~BatchScratch() {
  for (auto &e : ev)
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  if (ctx) {
    drop_graph();
    dev_free(ctx, dmem, dbytes);
    if (hmem) cudaFreeHost(hmem);
  }
}

int BatchScratch::reserve(rbffd_ctx *c, int members) {
  ctx = c;
  if (members <= cap) return RBFFD_OK;
  drop_graph();  // it refers to the buffers replaced here
  if (dmem) {
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, dmem, dbytes);
    dmem = nullptr;
  }
  if (hmem) {
    cudaFreeHost(hmem);
    hmem = nullptr;
  }
  cap = std::max(members, 16);
  maxc = std::max({krylov_batch_max_ctas(ctx, 1), krylov_batch_max_ctas(ctx, 2),
                   fgmres_batch_max_ctas(ctx), krylov_ir_batch_max_ctas(ctx, 1, INNER_F32),
                   krylov_ir_batch_max_ctas(ctx, 2, INNER_F32),
                   krylov_ir_batch_max_ctas(ctx, 1, INNER_FF),
                   krylov_ir_batch_max_ctas(ctx, 2, INNER_FF)});
  // device: per slot sys args, cta tables, flags, barriers; record
  // pointers, outputs.  The pinned host copy has the same layout.
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t a = o;
    o += (b + 255) / 256 * 256;
    return a;
  };
  for (int k = 0; k < NSLOT; ++k) {
    off_sys[k] = take(std::max({sizeof(KrylovArgs), sizeof(FgmresArgs), sizeof(MixedArgs)}) * cap);
    off_cta_sys[k] = take(sizeof(int) * maxc);
    team_words = 4 * maxc + cap;
    off_cta_first[k] = take(sizeof(int) * team_words);
    off_flags[k] = take(sizeof(unsigned int) * maxc);
    off_bars[k] = take(sizeof(GridBarrier) * cap);
  }
  off_recs = take(sizeof(void *) * cap);
  off_kouts = take(sizeof(void *) * cap);
  off_out = take(sizeof(MemberOut) * cap);
  dbytes = o;
  RBFFD_TRY(dev_alloc(ctx, &dmem, dbytes));
  hbytes = dbytes;
  RBFFD_CK(cudaMallocHost(&hmem, hbytes));
  return RBFFD_OK;
}

// Persistent work list of a batched launch: the CTAs form nteams teams of
// `team` consecutive CTAs; every system goes to one team, and a team solves
// its systems one after another (the kernels loop over the team's list).
// The host plans it from an estimate of each system's work (its rows times
// the iterations its last solve took, 1 before any):
//   - the team size makes the largest system fit a team's average share of
//     the work (team >= cmax * wmax / total), so no single system outlasts
//     the rest, capped by what every system's partial sums hold (cap[i]) and
//     by 8 threads per row of the smallest system's rows per CTA;
//   - teams = cmax / team (at most one per system, and then larger teams);
//   - largest work first, each system to the least-loaded team (LPT).
// Tables (device copies of the host arrays): cta_team[c] = the team of CTA
// c; team info[4 t ..] = first CTA, CTAs, list begin, list end, the list
// being positions in the same array (after the 4 * nteams info words)
// holding system indices.  Returns the CTAs launched; nb[i] = CTAs of
// system i's team.
struct TeamPlan {
  int nctas = 0;
  std::vector<int> cta_team, info_and_list, nb;
};

static TeamPlan plan_teams(const std::vector<double> &work, const std::vector<int> &cap,
                           const std::vector<int> &rows, int cmax, double scale = 1.0) {
  const int m = (int)work.size();
  TeamPlan T;
  double total = 0.0, wmax = 0.0;
  int capmin = kdev::MAXB, rmin = 1 << 30;
  for (int i = 0; i < m; ++i) {
    total += work[i];
    wmax = std::max(wmax, work[i]);
    capmin = std::min(capmin, cap[i]);
    rmin = std::min(rmin, rows[i]);
  }
  // CTAs beyond 8 threads per row of the smallest system only add waits
  const int rowcap = std::max(1, (int)((rmin * 8LL + KB_NT - 1) / KB_NT));
  const int tmax = std::max(1, std::min(capmin, kdev::MAXB));
  int team = total > 0 ? (int)std::ceil(cmax * wmax / total) : 1;
  team = std::max(1, (int)std::lround(team * scale));  // the autotuner's scale
  team = std::max(1, std::min(team, tmax));
  int nteams = std::max(1, std::min(cmax / team, m));
  // fewer teams than the grid holds: spread the CTAs over them
  team = std::max(1, std::min({cmax / nteams, tmax, std::max(team, rowcap)}));
  T.nctas = nteams * team;
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return work[a] > work[b]; });
  std::vector<double> load(nteams, 0.0);
  std::vector<std::vector<int>> lists(nteams);
  for (int i : order) {
    int best = 0;
    for (int t = 1; t < nteams; ++t)
      if (load[t] < load[best]) best = t;
    load[best] += work[i];
    lists[best].push_back(i);
  }
  T.cta_team.resize(T.nctas);
  for (int c = 0; c < T.nctas; ++c) T.cta_team[c] = c / team;
  T.info_and_list.assign(4 * nteams, 0);
  T.nb.assign(m, team);
  for (int t = 0; t < nteams; ++t) {
    T.info_and_list[4 * t] = t * team;
    T.info_and_list[4 * t + 1] = team;
    T.info_and_list[4 * t + 2] = (int)T.info_and_list.size();
    for (int i : lists[t]) T.info_and_list.push_back(i);
    T.info_and_list[4 * t + 3] = (int)T.info_and_list.size();
  }
  return T;
}

// The planner on its own, for the host tests (no device work): the team of
// every member and the plan's sizes.
extern "C" int rbffd_plan_work_lists(int32_t m, const double *work, const int32_t *cap,
                                     const int32_t *rows, int32_t cmax, double scale,
                                     int32_t *nctas, int32_t *team_size, int32_t *nteams,
                                     int32_t *member_team) {
  return guarded([&]() -> int {
    if (m < 1 || cmax < 1 || !work || !cap || !rows || !member_team || !(scale > 0.0))
      return RBFFD_EINVAL;
    for (int i = 0; i < m; ++i)
      if (!(work[i] >= 0.0) || cap[i] < 1 || rows[i] < 1) return RBFFD_EINVAL;
    const TeamPlan T = plan_teams(std::vector<double>(work, work + m),
                                  std::vector<int>(cap, cap + m), std::vector<int>(rows, rows + m),
                                  cmax, scale);
    // every team has the same size; nctas = teams x size
    const int size = T.nb[0], teams = T.nctas / size;
    for (int i = 0; i < m; ++i) member_team[i] = -1;
    for (int t = 0; t < teams; ++t)
      for (int k = T.info_and_list[4 * t + 2]; k < T.info_and_list[4 * t + 3]; ++k)
        member_team[T.info_and_list[k]] = t;
    if (nctas) *nctas = T.nctas;
    if (team_size) *team_size = size;
    if (nteams) *nteams = teams;
    return RBFFD_OK;
  });
}

// Autotuner events around the launch of one slot (only while tuning; such
// iterations are never captured).
static int tune_mark(BatchScratch &S, int slot, int end) {
  if (!S.timing) return RBFFD_OK;
  if (!S.ev[slot][end]) RBFFD_CK(cudaEventCreate(&S.ev[slot][end]));
  RBFFD_CK(cudaEventRecord(S.ev[slot][end], S.ctx->stream));
  S.slot_used[slot] = true;
  return RBFFD_OK;
}

// Work of one of a member's solves for the work-list plan: its rows times
// the iterations its last solve of that kind took (1 before any).
static double work_of(const rbffd_problem *Q, int kind) {
  return (double)Q->n * (double)std::max(1, Q->it_hist[kind]);
}

// Copy a launch's system arguments (m of `argbytes` each, already in the
// pinned host slot) and its work-list tables to the device, stream-ordered
// (captured as copies of the pinned host tables).
static int put_tables(BatchScratch &S, int slot, const TeamPlan &T, int m, size_t argbytes) {
  char *hb = (char *)S.hmem;
  char *db = (char *)S.dmem;
  if ((int)T.cta_team.size() > S.maxc || (int)T.info_and_list.size() > S.team_words) {
    set_error("batch: work-list tables exceed their slots");
    return RBFFD_EINVAL;
  }
  memcpy(hb + S.off_cta_sys[slot], T.cta_team.data(), sizeof(int) * T.cta_team.size());
  memcpy(hb + S.off_cta_first[slot], T.info_and_list.data(),
         sizeof(int) * T.info_and_list.size());
  RBFFD_CK(cudaMemcpyAsync(db + S.off_sys[slot], hb + S.off_sys[slot], argbytes * m,
                           cudaMemcpyHostToDevice, S.ctx->stream));
  RBFFD_CK(cudaMemcpyAsync(db + S.off_cta_sys[slot], hb + S.off_cta_sys[slot],
                           sizeof(int) * T.cta_team.size(), cudaMemcpyHostToDevice,
                           S.ctx->stream));
  RBFFD_CK(cudaMemcpyAsync(db + S.off_cta_first[slot], hb + S.off_cta_first[slot],
                           sizeof(int) * T.info_and_list.size(), cudaMemcpyHostToDevice,
                           S.ctx->stream));
  return RBFFD_OK;
}

// Threads per row: cover a CTA's rows (kdev::cta_rows) in one pass.
static int tpr_for(int n, int nb) {
  const long long R = (n + (long long)nb - 1) / nb;
  int T = 1;
  for (int t = 2; t <= 8; ++t)
    if ((long long)(32 / t) * (KB_NT / 32) >= R) T = t;
  return T;
}

// One batched Krylov launch for the systems args[0..m) (args filled except
// nblocks, tpr, flags and bar, which are set here), with table slot `slot`,
// planned as a persistent work list from the systems' work (plan_teams).
static int launch_krylov(BatchScratch &S, int slot, int nr, std::vector<KrylovArgs> &args,
                         const std::vector<double> &work, const std::vector<int> &rows,
                         bool amg = false) {
  rbffd_ctx *ctx = S.ctx;
  const int m = (int)args.size();
  const int cmax = krylov_batch_max_ctas(ctx, nr);
  if (m > cmax) {
    set_error("batch: %d members exceed the %d co-resident CTAs of one launch", m, cmax);
    return RBFFD_EINVAL;
  }
  std::vector<int> cap(m);
  for (int i = 0; i < m; ++i) cap[i] = args[i].nblocks;
  const TeamPlan T = plan_teams(work, cap, rows, cmax, S.scale[slot]);
  char *hb = (char *)S.hmem;
  char *db = (char *)S.dmem;
  KrylovArgs *hsys = (KrylovArgs *)(hb + S.off_sys[slot]);
  unsigned int *dflags = (unsigned int *)(db + S.off_flags[slot]);
  GridBarrier *dbars = (GridBarrier *)(db + S.off_bars[slot]);
  for (int i = 0; i < m; ++i) {
    KrylovArgs a = args[i];
    a.nblocks = T.nb[i];
    a.tpr = tpr_for(a.n, a.nblocks);
    a.flags = dflags + i;  // one arrival counter per system
    a.bar = dbars + i;
    hsys[i] = a;
  }
  RBFFD_TRY(put_tables(S, slot, T, m, sizeof(KrylovArgs)));
  RBFFD_CK(cudaMemsetAsync(dflags, 0, sizeof(unsigned int) * m, ctx->stream));
  RBFFD_TRY(reset_barriers(ctx, dbars, m));
  RBFFD_TRY(krylov_batch_launch(ctx, nr, T.nctas, (const KrylovArgs *)(db + S.off_sys[slot]),
                                (const int *)(db + S.off_cta_sys[slot]),
                                (const int *)(db + S.off_cta_first[slot]), amg));
  return RBFFD_OK;
}

// One batched mixed-precision launch (FP32 or float-float BiCGSTAB inside
// FP64 refinement) for the momentum systems args[0..m) of one inner
// arithmetic, with table slot `slot`: a persistent work list as in
// launch_krylov.
static int launch_mixed(BatchScratch &S, int slot, int nr, int inner,
                        std::vector<MixedArgs> &args, const std::vector<double> &work,
                        const std::vector<int> &rows) {
  rbffd_ctx *ctx = S.ctx;
  const int m = (int)args.size();
  const int cmax = krylov_ir_batch_max_ctas(ctx, nr, inner);
  if (m > cmax) {
    set_error("batch: %d members exceed the %d co-resident CTAs of one launch", m, cmax);
    return RBFFD_EINVAL;
  }
  std::vector<int> cap(m);
  for (int i = 0; i < m; ++i) cap[i] = args[i].nblocks;
  const TeamPlan T = plan_teams(work, cap, rows, cmax, S.scale[slot]);
  char *hb = (char *)S.hmem;
  char *db = (char *)S.dmem;
  MixedArgs *hsys = (MixedArgs *)(hb + S.off_sys[slot]);
  unsigned int *dflags = (unsigned int *)(db + S.off_flags[slot]);
  GridBarrier *dbars = (GridBarrier *)(db + S.off_bars[slot]);
  for (int i = 0; i < m; ++i) {
    MixedArgs a = args[i];
    a.nblocks = T.nb[i];
    a.tpr = tpr_for(a.n, a.nblocks);
    a.flags = dflags + i;
    a.bar = dbars + i;
    hsys[i] = a;
  }
  RBFFD_TRY(put_tables(S, slot, T, m, sizeof(MixedArgs)));
  RBFFD_CK(cudaMemsetAsync(dflags, 0, sizeof(unsigned int) * m, ctx->stream));
  RBFFD_TRY(reset_barriers(ctx, dbars, m));
  return krylov_ir_batch_launch(ctx, nr, inner, T.nctas, (const MixedArgs *)(db + S.off_sys[slot]),
                                (const int *)(db + S.off_cta_sys[slot]),
                                (const int *)(db + S.off_cta_first[slot]));
}

// One batched flexible-GMRES launch for the pressure-correction systems
// args[0..m) (filled except nblocks, flags and bar), with table slot `slot`:
// a persistent work list as in launch_krylov.
static int launch_fgmres(BatchScratch &S, int slot, std::vector<FgmresArgs> &args,
                         const std::vector<double> &work, const std::vector<int> &rows) {
  rbffd_ctx *ctx = S.ctx;
  const int m = (int)args.size();
  const int cmax = fgmres_batch_max_ctas(ctx);
  if (m > cmax) {
    set_error("batch: %d members exceed the %d co-resident CTAs of one launch", m, cmax);
    return RBFFD_EINVAL;
  }
  const TeamPlan T = plan_teams(work, std::vector<int>(m, kdev::MAXB), rows, cmax, S.scale[slot]);
  char *hb = (char *)S.hmem;
  char *db = (char *)S.dmem;
  FgmresArgs *hsys = (FgmresArgs *)(hb + S.off_sys[slot]);
  unsigned int *dflags = (unsigned int *)(db + S.off_flags[slot]);
  GridBarrier *dbars = (GridBarrier *)(db + S.off_bars[slot]);
  for (int i = 0; i < m; ++i) {
    FgmresArgs a = args[i];
    a.nblocks = T.nb[i];
    a.tpr = tpr_for(a.n, a.nblocks);
    a.flags = dflags + i;
    a.bar = dbars + i;
    hsys[i] = a;
  }
  RBFFD_TRY(put_tables(S, slot, T, m, sizeof(FgmresArgs)));
  RBFFD_CK(cudaMemsetAsync(dflags, 0, sizeof(unsigned int) * m, ctx->stream));
  RBFFD_TRY(reset_barriers(ctx, dbars, m));
  return fgmres_batch_launch(ctx, T.nctas, (const FgmresArgs *)(db + S.off_sys[slot]),
                             (const int *)(db + S.off_cta_sys[slot]),
                             (const int *)(db + S.off_cta_first[slot]));
}

// One batched pressure-correction solve M x_i = b_i of the members sel
// (one launch per solver: Jacobi BiCGSTAB, multigrid BiCGSTAB, flexible
// GMRES), issued on the context's stream with no host synchronisation.
// Its outcome goes to each member's kout[2].  a1 holds the members'
// common Krylov arguments.
static int launch_pcorr(BatchScratch &S, rbffd_problem *const *P, const std::vector<int> &sel,
                        const std::vector<const double *> &b, const std::vector<double *> &x,
                        const std::vector<double> &tol, const std::vector<int> &maxit) {
  std::vector<KrylovArgs> pj, pa;
  std::vector<FgmresArgs> pf;
  std::vector<int> rj, ra, rf;
  std::vector<double> wj, wa, wf;
  std::vector<std::pair<int, int>> mj, ma, mf;
  for (size_t s = 0; s < sel.size(); ++s) {
    rbffd_problem *Q = P[sel[s]];
    if (Q->amgf) {
      FgmresArgs f;
      memset(&f, 0, sizeof(f));
      f.n = Q->n;
      f.q = Q->q;
      f.ldn = Q->ldn;
      f.tpr = 1;
      f.m = Q->fg_m;
      f.col = Q->col;
      f.val = Q->Pp;
      f.val32 = Q->amgf_host.a0;
      f.b = b[s];
      f.x = x[s];
      f.r = Q->fgR;
      f.V = Q->fgV;
      f.Z = Q->fgZ;
      f.part = Q->fgpart;
      f.out = Q->kout + 2;
      f.tol = tol[s];
      f.maxit = maxit[s];
      f.amg = Q->amgf;
      f.reorth = Q->ctx->fgmres_reorth;
      pf.push_back(f);
      rf.push_back(Q->n);
      wf.push_back(work_of(Q, 1));
      mf.push_back({sel[s], 1});
      continue;
    }
    KrylovArgs a;
    memset(&a, 0, sizeof(a));
    a.n = Q->n;
    a.q = Q->q;
    a.ldn = Q->ldn;
    a.col = Q->col;
    a.part = Q->part;
    a.tol = tol[s];
    a.maxit = maxit[s];
    a.val = Q->Pp;
    a.dinv = Q->p_dinv;
    a.b[0] = b[s];
    a.x[0] = x[s];
    a.w[0] = Q->kv[0];
    a.out = Q->kout + 2;
    a.nblocks = 2 * std::max(Q->kblocks1, Q->kblocks2);
    if (Q->amg) {
      a.amg = Q->amg;
      pa.push_back(a);
      ra.push_back(Q->n);
      wa.push_back(work_of(Q, 1));
      ma.push_back({sel[s], 1});
    } else {
      pj.push_back(a);
      rj.push_back(Q->n);
      wj.push_back(work_of(Q, 1));
      mj.push_back({sel[s], 1});
    }
  }
  if (!pj.empty()) {
    RBFFD_TRY(tune_mark(S, 2, 0));
    RBFFD_TRY(launch_krylov(S, 2, 1, pj, wj, rj));
    S.slot_sys[2] = mj;
    RBFFD_TRY(tune_mark(S, 2, 1));
  }
  if (!pa.empty()) {
    RBFFD_TRY(tune_mark(S, 3, 0));
    RBFFD_TRY(launch_krylov(S, 3, 1, pa, wa, ra, true));
    S.slot_sys[3] = ma;
    RBFFD_TRY(tune_mark(S, 3, 1));
  }
  if (!pf.empty()) {
    RBFFD_TRY(tune_mark(S, 4, 0));
    RBFFD_TRY(launch_fgmres(S, 4, pf, wf, rf));
    S.slot_sys[4] = mf;
    RBFFD_TRY(tune_mark(S, 4, 1));
  }
  return RBFFD_OK;
}

// Issue one batched outer iteration on the context's stream, ending with
// the members' results copied to the pinned host table: no host
// synchronisation, so it can be captured.
static int issue_batch(BatchScratch &S, rbffd_problem *const *P, int m,
                       const rbffd_step_params *const *spv) {
  rbffd_ctx *ctx = P[0]->ctx;
  // momentum predictor of every member, then one launch for the two-RHS
  // solves of all members (and one for the single-RHS pairs, if any)
  std::vector<KrylovArgs> a2, a1s;
  std::vector<int> rows2, rows1s;
  std::vector<double> work2, work1s;
  std::vector<std::pair<int, int>> mem2, mem1s, xmem2[2], xmem1s[2];
  // mixed-precision members by inner arithmetic (0 FP32, 1 float-float)
  std::vector<MixedArgs> x2[2], x1s[2];
  std::vector<int> xr2[2], xr1s[2];
  std::vector<double> xw2[2], xw1s[2];
  for (int i = 0; i < m; ++i) {
    const rbffd_step_params *sp = spv[i];
    RBFFD_TRY(ops_momentum(P[i], sp));
    if (P[i]->precision != RBFFD_PREC_FP64) {
      rbffd_problem *Q = P[i];
      const int ia = Q->inner == INNER_FF ? 1 : 0;
      RBFFD_TRY(ops_to_inner(Q, Q->Am, Q->Ain, (int64_t)Q->ldn * Q->q));
      RBFFD_TRY(ops_to_inner(Q, Q->m_dinv, Q->mdin, Q->ldn));
      MixedArgs x;
      memset(&x, 0, sizeof(x));
      x.inner = Q->inner;
      x.n = Q->n;
      x.q = Q->q;
      x.ldn = Q->ldn;
      x.col = Q->col;
      x.part64 = Q->part64;
      x.partin = Q->partin;
      x.tol = sp->krylov_tol;
      x.maxit = sp->krylov_maxit;
      x.inner_tol = sp->inner_tol > 0 ? sp->inner_tol : 1e-3;
      x.inner_maxit = sp->inner_maxit > 0 ? sp->inner_maxit : 4000;
      x.max_sweeps = 60;
      x.val64 = Q->Am;
      x.valin = Q->Ain;
      x.dinvin = Q->mdin;
      x.b[0] = Q->bu;
      x.b[1] = Q->bv;
      x.x[0] = Q->ut;
      x.x[1] = Q->vt;
      x.w[0] = Q->mv[0];
      x.w[1] = Q->mv[1];
      x.out = Q->kout;
      x.nblocks = std::max(Q->kblocks1, Q->kblocks2);  // partial-sum capacity
      if (!Q->has_sym) {
        x2[ia].push_back(x);
        xr2[ia].push_back(Q->n);
        xw2[ia].push_back(work_of(Q, 0));
        xmem2[ia].push_back({i, 0});
      } else {
        // the u~ and v~ systems differ on symmetry lines: two single-RHS
        // systems, the second on its own partial sums (second half)
        RBFFD_TRY(ops_to_inner(Q, Q->Am2, Q->Ain2, (int64_t)Q->ldn * Q->q));
        RBFFD_TRY(ops_to_inner(Q, Q->m_dinv2, Q->mdin2, Q->ldn));
        MixedArgs xu = x;
        xu.b[1] = nullptr;
        xu.x[1] = nullptr;
        MixedArgs xv = xu;
        xv.val64 = Q->Am2;
        xv.valin = Q->Ain2;
        xv.dinvin = Q->mdin2;
        xv.b[0] = Q->bv;
        xv.x[0] = Q->vt;
        xv.w[0] = Q->mv[1];
        xv.out = Q->kout + 1;
        xv.part64 = Q->part64 + krylov_ir_partials64(1, x.nblocks);
        xv.partin = (char *)Q->partin + krylov_ir_partials_inner_bytes(1, x.nblocks, Q->inner);
        x1s[ia].push_back(xu);
        x1s[ia].push_back(xv);
        xr1s[ia].push_back(Q->n);
        xr1s[ia].push_back(Q->n);
        xw1s[ia].push_back(work_of(Q, 0));
        xw1s[ia].push_back(work_of(Q, 0));
        xmem1s[ia].push_back({i, 0});
        xmem1s[ia].push_back({i, 0});
      }
      continue;
    }
    KrylovArgs a;
    memset(&a, 0, sizeof(a));
    a.n = P[i]->n;
    a.q = P[i]->q;
    a.ldn = P[i]->ldn;
    a.col = P[i]->col;
    a.part = P[i]->part;
    a.tol = sp->krylov_tol;
    a.maxit = sp->krylov_maxit;
    a.val = P[i]->Am;
    a.dinv = P[i]->m_dinv;
    a.b[0] = P[i]->bu;
    a.b[1] = P[i]->bv;
    a.x[0] = P[i]->ut;
    a.x[1] = P[i]->vt;
    a.w[0] = P[i]->kv[0];
    a.w[1] = P[i]->kv[1];
    a.out = P[i]->kout;
    const int capb = std::max(P[i]->kblocks1, P[i]->kblocks2);  // partial-sum capacity
    a.nblocks = capb;
    if (!P[i]->has_sym) {
      a2.push_back(a);
      rows2.push_back(P[i]->n);
      work2.push_back(work_of(P[i], 0));
      mem2.push_back({i, 0});
    } else {
      KrylovArgs au = a;
      au.b[1] = nullptr;
      au.x[1] = nullptr;
      KrylovArgs av = au;
      av.val = P[i]->Am2;
      av.dinv = P[i]->m_dinv2;
      av.b[0] = P[i]->bv;
      av.x[0] = P[i]->vt;
      av.w[0] = P[i]->kv[1];
      av.out = P[i]->kout + 1;
      av.part = P[i]->part + krylov_partials_doubles(1, capb);  // second half
      a1s.push_back(au);
      a1s.push_back(av);
      rows1s.push_back(P[i]->n);
      rows1s.push_back(P[i]->n);
      work1s.push_back(work_of(P[i], 0));
      work1s.push_back(work_of(P[i], 0));
      mem1s.push_back({i, 0});
      mem1s.push_back({i, 0});
    }
  }
  prof_begin(ctx, 0);
  if (!a2.empty()) {
    RBFFD_TRY(tune_mark(S, 0, 0));
    RBFFD_TRY(launch_krylov(S, 0, 2, a2, work2, rows2));
    S.slot_sys[0] = mem2;
    RBFFD_TRY(tune_mark(S, 0, 1));
  }
  if (!a1s.empty()) {
    RBFFD_TRY(tune_mark(S, 1, 0));
    RBFFD_TRY(launch_krylov(S, 1, 1, a1s, work1s, rows1s));
    S.slot_sys[1] = mem1s;
    RBFFD_TRY(tune_mark(S, 1, 1));
  }
  for (int ia = 0; ia < 2; ++ia) {
    const int inner = ia ? INNER_FF : INNER_F32;
    if (!x2[ia].empty()) {
      RBFFD_TRY(tune_mark(S, 5 + 2 * ia, 0));
      RBFFD_TRY(launch_mixed(S, 5 + 2 * ia, 2, inner, x2[ia], xw2[ia], xr2[ia]));
      S.slot_sys[5 + 2 * ia] = xmem2[ia];
      RBFFD_TRY(tune_mark(S, 5 + 2 * ia, 1));
    }
    if (!x1s[ia].empty()) {
      RBFFD_TRY(tune_mark(S, 6 + 2 * ia, 0));
      RBFFD_TRY(launch_mixed(S, 6 + 2 * ia, 1, inner, x1s[ia], xw1s[ia], xr1s[ia]));
      S.slot_sys[6 + 2 * ia] = xmem1s[ia];
      RBFFD_TRY(tune_mark(S, 6 + 2 * ia, 1));
    }
  }
  prof_end(ctx, 0);
  // p' solves: one launch per solver -- Jacobi BiCGSTAB, multigrid
  // BiCGSTAB, flexible GMRES
  std::vector<const double *> bs(m);
  std::vector<double *> xs(m);
  std::vector<double> tols(m);
  std::vector<int> maxits(m), sel(m);
  for (int i = 0; i < m; ++i) {
    RBFFD_TRY(ops_divergence(P[i], spv[i]));
    bs[i] = P[i]->bp;
    xs[i] = P[i]->pc;
    tols[i] = spv[i]->krylov_tol;
    maxits[i] = spv[i]->krylov_maxit;
    sel[i] = i;
  }
  prof_begin(ctx, 1);
  RBFFD_TRY(launch_pcorr(S, P, sel, bs, xs, tols, maxits));
  prof_end(ctx, 1);
  for (int i = 0; i < m; ++i) {
    RBFFD_TRY(ops_pressure(P[i], spv[i]));
    RBFFD_TRY(ops_correct(P[i], spv[i]));
  }
  // gather every member's Delta and Krylov outcome with one read-back
  char *hb = (char *)S.hmem;
  char *db = (char *)S.dmem;
  IterRecord **hrec = (IterRecord **)(hb + S.off_recs);
  KrylovOut **hko = (KrylovOut **)(hb + S.off_kouts);
  for (int i = 0; i < m; ++i) {
    hrec[i] = P[i]->rec;
    hko[i] = P[i]->kout;
  }
  RBFFD_CK(cudaMemcpyAsync(db + S.off_recs, hb + S.off_recs, S.off_out - S.off_recs,
                           cudaMemcpyHostToDevice, ctx->stream));
  k_gather_out<<<(m + 127) / 128, 128, 0, ctx->stream>>>(
      m, (IterRecord *const *)(db + S.off_recs), (const KrylovOut *const *)(db + S.off_kouts),
      (MemberOut *)(db + S.off_out));
  RBFFD_TRY(after_launch(ctx, "k_gather_out"));
  RBFFD_CK(cudaMemcpyAsync(hb + S.off_out, db + S.off_out, sizeof(MemberOut) * m,
                           cudaMemcpyDeviceToHost, ctx->stream));
  return RBFFD_OK;
}

// what a captured iteration depends on beyond device memory: the members,
// their builds, and the step parameters baked into kernel arguments and
// Krylov tables
static std::vector<uint64_t> graph_key(rbffd_problem *const *P, int m,
                                       const rbffd_step_params *const *spv) {
  std::vector<uint64_t> k;
  k.reserve(1 + 8 * (size_t)m);
  k.push_back((uint64_t)m);
  auto bits = [](double v) {
    uint64_t u;
    memcpy(&u, &v, sizeof(u));
    return u;
  };
  for (int i = 0; i < m; ++i) {
    const rbffd_step_params *sp = spv[i];
    k.push_back((uint64_t)(uintptr_t)P[i]);
    k.push_back(P[i]->gen);
    k.push_back(bits(sp->dt));
    for (int a = 0; a < 3; ++a) k.push_back(bits(sp->alpha[a]));
    k.push_back(bits(sp->krylov_tol));
    k.push_back((uint64_t)(uint32_t)sp->krylov_maxit);
  }
  return k;
}

// The compatible p' of the pinned members built since their last
// iteration needs z = M^{-1} e_I (problem.cu: compat_ready): solved here for
// all of them in one batched launch per solver, before anything is issued
// or captured.  The launch tables it writes are those a captured iteration
// copies at replay, so a captured graph is dropped first (a build changes
// the graph key anyway).
static int batch_compat(BatchScratch &S, rbffd_problem *const *P, int m) {
  std::vector<int> sel;
  for (int i = 0; i < m; ++i)
    if (P[i]->compat && !P[i]->z_ready) sel.push_back(i);
  if (sel.empty()) return RBFFD_OK;
  rbffd_ctx *ctx = P[0]->ctx;
  S.drop_graph();
  std::vector<const double *> b;
  std::vector<double *> x;
  for (int i : sel) {
    RBFFD_TRY(ops_interior_ones(P[i], P[i]->pcs, P[i]->zc));
    b.push_back(P[i]->pcs);
    x.push_back(P[i]->zc);
  }
  std::vector<double> tol;
  std::vector<int> maxit;
  for (int i : sel) {
    tol.push_back(compat_tol(P[i]));
    maxit.push_back(compat_maxit(P[i]));
  }
  RBFFD_TRY(launch_pcorr(S, P, sel, b, x, tol, maxit));
  std::vector<KrylovOut> ko(sel.size());
  for (size_t s = 0; s < sel.size(); ++s)
    RBFFD_CK(cudaMemcpyAsync(&ko[s], P[sel[s]]->kout + 2, sizeof(KrylovOut),
                             cudaMemcpyDeviceToHost, ctx->stream));
  RBFFD_CK(cudaStreamSynchronize(ctx->stream));
  for (size_t s = 0; s < sel.size(); ++s) {
    int rc = status_of(ko[s].status);
    // the same acceptance and fallback as compat_ready (z carries the pin's
    // response; a stalled multigrid solve is redone with FP64 Jacobi)
    if (rc == RBFFD_ENOCONV && ko[s].relres <= compat_accept()) rc = RBFFD_OK;
    rbffd_problem *Q = P[sel[s]];
    if ((rc == RBFFD_ENOCONV || rc == RBFFD_EDIVERGED) && (Q->amg || Q->amgf))
      rc = compat_fallback(Q, &ko[s].relres);
    if (rc != RBFFD_OK) {
      set_error("batch member %d: compatible p': the solve of M z = e_I ended with status %d "
                "(relres %.3e)", sel[s], rc, ko[s].relres);
      return rc;
    }
    P[sel[s]]->z_ready = true;
  }
  return RBFFD_OK;
}

int batch_iterate(BatchScratch &S, rbffd_problem *const *P, int m,
                  const rbffd_step_params *const *spv, double *deltas, rbffd_iter_stats *stats,
                  int *status) {
  if (m <= 0) return RBFFD_OK;
  rbffd_ctx *ctx = P[0]->ctx;
  for (int i = 0; i < m; ++i) {
    if (P[i]->ctx != ctx ||
        (P[i]->precision != RBFFD_PREC_FP64 && P[i]->precond == RBFFD_PRECOND_JACOBI)) {
      set_error("batch: members must share one context; mixed-precision members need a "
                "multigrid p' solver");
      return RBFFD_EINVAL;
    }
  }
  // hierarchies still being built are finished before anything is issued
  // (the iteration may be captured as a graph)
  for (int i = 0; i < m; ++i) RBFFD_TRY(amg_ready(P[i]));
  // a member with symmetry lines solves u~ and v~ as two single-RHS systems
  // (their rows differ there), so a launch may hold up to 2m systems
  RBFFD_TRY(S.reserve(ctx, 2 * m));
  RBFFD_TRY(batch_compat(S, P, m));
  // replay the captured iteration when it was captured for exactly these
  // members, builds and step parameters.  A new set runs directly once and
  // is captured when it comes back, so one-off iterations (a rebuild before
  // every call) pay no capture.  Live kernel timing records events per
  // phase: launched directly.
  // the work-list autotuner's iterations run directly, timed per slot
  S.timing = !S.tuned && !S.tune_off && !ctx->prof;
  const double cand[BatchScratch::NCAND] = {1.0, 2.0, 0.5, 4.0};
  const int tc = S.timing ? BatchScratch::tune_cand(S.tune_step) : -1;
  if (S.timing) {
    for (int k = 0; k < BatchScratch::NSLOT; ++k) {
      S.scale[k] = tc < 0 ? 1.0 : cand[tc];
      S.slot_used[k] = false;
    }
  }
  const bool want = !ctx->prof && !S.graph_off && !S.timing;
  std::vector<uint64_t> key;
  if (want) key = graph_key(P, m, spv);
  if (S.timing) {
    S.drop_graph();
    RBFFD_TRY(issue_batch(S, P, m, spv));
  } else if (want && S.exec && key == S.key) {
    RBFFD_CK(cudaGraphLaunch(S.exec, ctx->stream));
    ctx->launches += S.graph_launches;
    S.replays++;
  } else {
    S.drop_graph();
    const bool again = want && key == S.seen;
    if (want && !again) S.seen = key;
    bool done = false;
    if (again && cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      const int64_t l0 = ctx->launches;
      const int rc = issue_batch(S, P, m, spv);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
      ctx->launches = l0;
      if (rc != RBFFD_OK) {  // an error of the iteration itself, not of the capture
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc;
      }
      if (e == cudaSuccess && g && cudaGraphInstantiate(&S.exec, g, 0) == cudaSuccess) {
        S.graph_launches = 0;
        size_t nn = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
          std::vector<cudaGraphNode_t> nodes(nn);
          cudaGraphGetNodes(g, nodes.data(), &nn);
          for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
              S.graph_launches++;
          }
        }
        S.key = std::move(key);
        S.captures++;
        done = true;
      } else {
        // the capture did not hold: launch directly from now on
        S.exec = nullptr;
        S.graph_off = true;
        cudaGetLastError();
      }
      if (g) cudaGraphDestroy(g);
      if (done) {
        RBFFD_CK(cudaGraphLaunch(S.exec, ctx->stream));
        ctx->launches += S.graph_launches;
      }
    }
    if (!done) RBFFD_TRY(issue_batch(S, P, m, spv));
  }
  RBFFD_CK(cudaStreamSynchronize(ctx->stream));
  char *hb = (char *)S.hmem;
  const MemberOut *mo = (const MemberOut *)(hb + S.off_out);
  if (ctx->prof) {
    // units: rows x iterations of every member (the launch's work)
    double um = 0, up = 0, bm = 0, bp = 0;
    for (int i = 0; i < m; ++i) {
      const double n = P[i]->n, q = P[i]->q;
      const double im = std::max(mo[i].iters[0], mo[i].iters[1]), ip = mo[i].iters[2];
      um += n * im;
      up += n * ip;
      bm += n * im * (2 * q * 12.0 + 28 * 8.0);
      bp += pcorr_bytes(P[i], mo[i].iters[2]);
    }
    prof_collect(ctx, 0, RBFFD_KSTAT_KRYLOV_MOM, um, bm);
    prof_collect(ctx, 1, RBFFD_KSTAT_KRYLOV_P, up, bp);
  }
  if (S.timing) {
    // time per unit of work (rows x iterations) of every slot's launch
    for (int k = 0; k < BatchScratch::NSLOT && tc >= 0; ++k) {
      if (!S.slot_used[k]) continue;
      float ms = 0.0f;
      RBFFD_CK(cudaEventElapsedTime(&ms, S.ev[k][0], S.ev[k][1]));
      double work = 0.0;
      for (const auto &pr : S.slot_sys[k]) {
        const MemberOut &o = mo[pr.first];
        const int it = pr.second == 0 ? std::max(o.iters[0], o.iters[1]) : o.iters[2];
        work += (double)P[pr.first]->n * std::max(1, it);
      }
      if (work > 0.0) S.cost[k][tc] += 0.5 * ms / work;
    }
    S.timing = false;
    if (++S.tune_step == BatchScratch::NTUNE) {
      for (int k = 0; k < BatchScratch::NSLOT; ++k) {
        int best = 0;
        for (int c = 1; c < BatchScratch::NCAND; ++c)
          if (S.cost[k][c] > 0.0 && (S.cost[k][best] <= 0.0 || S.cost[k][c] < S.cost[k][best]))
            best = c;
        S.scale[k] = cand[best];
      }
      S.tuned = true;
    }
  }
  // iteration history for the next plan of the work lists (plan_teams)
  for (int i = 0; i < m; ++i) {
    P[i]->it_hist[0] = std::max(mo[i].iters[0], mo[i].iters[1]);
    P[i]->it_hist[1] = mo[i].iters[2];
  }
  int rc = RBFFD_OK;
  for (int i = 0; i < m; ++i) {
    if (deltas) deltas[i] = mo[i].delta;
    if (stats) {
      for (int k = 0; k < 3; ++k) {
        stats[i].iters[k] = mo[i].iters[k];
        stats[i].relres[k] = mo[i].relres[k];
        stats[i].sweeps[k] = 0;
      }
    }
    int st = RBFFD_OK;
    for (int k = 0; k < 3 && st == RBFFD_OK; ++k) st = status_of(mo[i].status[k]);
    if (st == RBFFD_OK && !std::isfinite(mo[i].delta)) st = RBFFD_EDIVERGED;
    if (status) status[i] = st;
    if (st != RBFFD_OK && rc == RBFFD_OK) rc = st;
  }
  return status ? RBFFD_OK : rc;
}

}  // namespace rbffd

// ------------------------------------------------------------------ C ABI

struct rbffd_batch {
  rbffd_ctx *ctx = nullptr;
  std::vector<rbffd_problem *> members;
  BatchScratch scratch;
};

extern "C" int rbffd_batch_create(rbffd_ctx *ctx, int32_t count, rbffd_problem *const *members,
                                  rbffd_batch **out) {
  return guarded([&]() -> int {
    if (!ctx || !out || count < 1 || !members) return RBFFD_EINVAL;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
      if (!members[i] || members[i]->ctx != ctx ||
          (members[i]->precision != RBFFD_PREC_FP64 &&
           members[i]->precond == RBFFD_PRECOND_JACOBI)) {
        set_error("rbffd_batch_create: member %d is null, on another context, or mixed-precision "
                  "with a Jacobi p' solver", i);
        return RBFFD_EINVAL;
      }
    }
    rbffd_batch *b = new rbffd_batch();
    b->ctx = ctx;
    ctx_ref(ctx);
    b->members.assign(members, members + count);
    int rc = b->scratch.reserve(ctx, count);
    if (rc != RBFFD_OK) {
      delete b;
      ctx_unref(ctx);
      return rc;
    }
    *out = b;
    return RBFFD_OK;
  });
}

extern "C" void rbffd_batch_destroy(rbffd_batch *b) {
  if (!b) return;
  rbffd_ctx *ctx = b->ctx;
  cudaStreamSynchronize(ctx->stream);
  delete b;  // frees the scratch through ctx, which is still alive here
  ctx_unref(ctx);
}

extern "C" int rbffd_batch_graph_stats(const rbffd_batch *b, int64_t *captures,
                                       int64_t *replays, int64_t *kernels) {
  return guarded([&]() -> int {
    if (!b) return RBFFD_EINVAL;
    if (captures) *captures = b->scratch.captures;
    if (replays) *replays = b->scratch.replays;
    if (kernels) *kernels = b->scratch.graph_off ? 0 : b->scratch.graph_launches;
    return RBFFD_OK;
  });
}

extern "C" int rbffd_batch_tuning(const rbffd_batch *b, int32_t *tuned, double *scales,
                                  double *cost) {
  return guarded([&]() -> int {
    if (!b) return RBFFD_EINVAL;
    const BatchScratch &S = b->scratch;
    if (tuned) *tuned = S.tuned ? 1 : 0;
    for (int k = 0; k < BatchScratch::NSLOT; ++k) {
      if (scales) scales[k] = S.scale[k];
      for (int c = 0; c < BatchScratch::NCAND; ++c)
        if (cost) cost[k * BatchScratch::NCAND + c] = S.cost[k][c];
    }
    return RBFFD_OK;
  });
}

extern "C" int rbffd_batch_set_autotune(rbffd_batch *b, int on) {
  return guarded([&]() -> int {
    if (!b) return RBFFD_EINVAL;
    BatchScratch &S = b->scratch;
    S.tune_off = !on;
    S.tuned = false;
    S.tune_step = 0;
    for (int k = 0; k < BatchScratch::NSLOT; ++k) {
      S.scale[k] = 1.0;
      for (int c = 0; c < BatchScratch::NCAND; ++c) S.cost[k][c] = 0.0;
    }
    return RBFFD_OK;
  });
}

extern "C" int rbffd_batch_iterate(rbffd_batch *b, const rbffd_step_params *sp,
                                   const double *dt, const int32_t *active, double *deltas,
                                   rbffd_iter_stats *stats, int32_t *status) {
  return guarded([&]() -> int {
    if (!b || !sp) return RBFFD_EINVAL;
    if (!(sp->dt > 0) || !(sp->krylov_tol > 0) || sp->krylov_maxit < 1 || sp->alpha[0] == 0.0)
      return RBFFD_EINVAL;
    RBFFD_CK(cudaSetDevice(b->ctx->device));
    const int count = (int)b->members.size();
    std::vector<rbffd_problem *> act;
    std::vector<int> where;
    for (int i = 0; i < count; ++i)
      if (!active || active[i]) {
        act.push_back(b->members[i]);
        where.push_back(i);
      }
    std::vector<double> d(act.size());
    std::vector<rbffd_iter_stats> st(act.size());
    std::vector<int> sts(act.size());
    std::vector<rbffd_step_params> own(act.size(), *sp);
    std::vector<const rbffd_step_params *> spv(act.size());
    for (size_t k = 0; k < act.size(); ++k) {
      if (dt) {
        if (!(dt[where[k]] > 0)) return RBFFD_EINVAL;
        own[k].dt = dt[where[k]];
      }
      spv[k] = &own[k];
    }
    int rc = batch_iterate(b->scratch, act.data(), (int)act.size(), spv.data(), d.data(),
                           st.data(), sts.data());
    if (rc != RBFFD_OK) return rc;
    int worst = RBFFD_OK;
    for (size_t k = 0; k < act.size(); ++k) {
      const int i = where[k];
      if (deltas) deltas[i] = d[k];
      if (stats) stats[i] = st[k];
      if (status) status[i] = sts[k];
      if (sts[k] != RBFFD_OK && worst == RBFFD_OK) worst = sts[k];
    }
    if (worst != RBFFD_OK && !status) set_error("a batch member's solve failed (%d)", worst);
    return status ? RBFFD_OK : worst;
  });
}
