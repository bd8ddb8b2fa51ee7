// Batching pattern: several independent problems (uneven grids, wavelengths,
// permittivities, sources) solved by FGMRES in lock step.  Every Arnoldi
// step applies the neural local solves of ALL windows of ALL still-active
// problems as one batch (one launch per neural-operator stage, in chunks of
// the batch's window capacity, Fig. 1a "multi-wavelength simulations in
// parallel"); the Krylov kernels then run per problem.  Each problem keeps
// its own restart position, FP64 iterate and FP64 true residual at restarts,
// exactly as fdfd_solve does.
#include <math.h>
#include <string.h>
#include <vector>
#include "ctx.cuh"
#include "nno.cuh"

int schwarz_inner_iters(fdfd_ctx* h);
int schwarz_coarse(fdfd_ctx* h, float2* z);

struct fdfd_batch_ctx {
  std::vector<fdfd_ctx*> hs;
  int cap = 0;                 // windows per neural-operator pass
  NnoWork work;
  int2* wtab_d = nullptr;      // [total windows]
  ProbGeom* ptab_d = nullptr;  // [n]
  int2* wtab_h = nullptr;      // pinned
  ProbGeom* ptab_h = nullptr;  // pinned
  double* flags_h = nullptr;   // pinned, 2 per problem
  size_t bytes = 0;
};

namespace {

struct PState {
  int j = 0, iters = 0, cycles = 0, status = FDFD_NOT_CONVERGED, stalls = 0;
  bool active = true;
  double est = 1.0, relres = 1.0, prev = INFINITY;
  double rs = 1.0;  // power-of-two scaling of the system, ||rs b|| in [1, 2)
};

__global__ void bnorm_kernel(KrylovState* st) {
  st->bnorm = sqrt(st->resid);
  st->nonfinite = 0;
  st->breakdown = 0;
}

int n_windows(const fdfd_ctx* h) { return (h->nx / FDFD_CORE) * (h->ny / FDFD_CORE); }

}  // namespace

extern "C" int fdfd_batch_create(fdfd_handle* hs, int n, int max_windows, fdfd_batch* out) {
  if (!out) return FDFD_EINVAL;
  *out = nullptr;
  if (!hs || n < 1 || max_windows < 0) return FDFD_EINVAL;
  int total = 0;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->stream != hs[0]->stream) return FDFD_EINVAL;
    total += n_windows(hs[i]);
  }
  fdfd_batch_ctx* b = new fdfd_batch_ctx();
  b->hs.assign(hs, hs + n);
  b->cap = max_windows > 0 ? (max_windows < total ? max_windows : total) : (total < 8192 ? total : 8192);
  int rc = FDFD_OK;
  if (schwarz_weights(hs[0])) {
    rc = nno_alloc_work(&b->work, b->cap, &b->bytes);
    if (!rc) rc = nno_autotune(schwarz_weights(hs[0]), &b->work, b->cap, hs[0]->stream);
  }
  if (!rc) {
    if (cudaMalloc((void**)&b->wtab_d, (size_t)total * sizeof(int2)) != cudaSuccess ||
        cudaMalloc((void**)&b->ptab_d, (size_t)n * sizeof(ProbGeom)) != cudaSuccess ||
        cudaMallocHost((void**)&b->wtab_h, (size_t)total * sizeof(int2)) != cudaSuccess ||
        cudaMallocHost((void**)&b->ptab_h, (size_t)n * sizeof(ProbGeom)) != cudaSuccess ||
        cudaMallocHost((void**)&b->flags_h, (size_t)n * 2 * sizeof(double)) != cudaSuccess)
      rc = FDFD_ENOMEM;
  }
  if (rc) { fdfd_batch_destroy(b); return rc; }
  *out = b;
  return FDFD_OK;
}

extern "C" void fdfd_batch_destroy(fdfd_batch b) {
  if (!b) return;
  if (!b->hs.empty()) cudaStreamSynchronize(b->hs[0]->stream);
  nno_free_work(&b->work);
  if (b->wtab_d) cudaFree(b->wtab_d);
  if (b->ptab_d) cudaFree(b->ptab_d);
  if (b->wtab_h) cudaFreeHost(b->wtab_h);
  if (b->ptab_h) cudaFreeHost(b->ptab_h);
  if (b->flags_h) cudaFreeHost(b->flags_h);
  delete b;
}

extern "C" int fdfd_solve_batched(fdfd_batch bt, const fdfd_c64* const* Jp, fdfd_c64* const* Ep,
                                  const fdfd_solve_opts* o, fdfd_solve_stats* stats) {
  if (!bt || !Jp || !Ep || !o) return FDFD_EINVAL;
  const int n = (int)bt->hs.size();
  fdfd_ctx* h0 = bt->hs[0];
  if (o->restart < 1 || o->restart > h0->rmax || o->max_iters < 0 || !(o->tol > 0)) return FDFD_EINVAL;
  if (o->precond < FDFD_PRECOND_NONE || o->precond > FDFD_PRECOND_SCHWARZ) return FDFD_EINVAL;
  const bool schwarz = o->precond == FDFD_PRECOND_SCHWARZ;
  for (int p = 0; p < n; ++p) {
    if (!Jp[p] || !Ep[p]) return FDFD_EINVAL;
    if (schwarz && !schwarz_weights(bt->hs[p])) return FDFD_ENOSETUP;
  }
  if (schwarz && !bt->work.X) return FDFD_ENOSETUP;
  cudaStream_t s = h0->stream;
  const int m = o->restart;
  std::vector<PState> ps(n);
  auto Jf = [&](int p) { return reinterpret_cast<const float2*>(Jp[p]); };
  auto Ef = [&](int p) { return reinterpret_cast<float2*>(Ep[p]); };
  int rc;
  CK(cudaEventRecord(h0->ev0, s));
  // ||b|| of every problem
  for (int p = 0; p < n; ++p) {
    fdfd_ctx* h = bt->hs[p];
    CK(cudaMemsetAsync(h->x64, 0, h->n * sizeof(double2), s));
    ProfScope ps_(h0, 3, 2);
    if ((rc = launch_residual64(nullptr, Jf(p), h->sb, 1, 1.0, h->eps, h->cx64, h->cy64, h->k2, h->nx, h->ny, h->V,
                                h->partials, h->counter, &h->st->resid, s)))
      return rc;
    bnorm_kernel<<<1, 1, 0, s>>>(h->st);
    CKL();
    CK(cudaMemcpyAsync(&bt->flags_h[2 * p], &h->st->bnorm, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  for (int p = 0; p < n; ++p) {
    const double bn = bt->flags_h[2 * p];
    if (!isfinite(bn)) { ps[p].status = FDFD_ENUMERIC; ps[p].active = false; }
    else if (bn == 0.0) {
      CK(cudaMemsetAsync(Ef(p), 0, bt->hs[p]->n * sizeof(float2), s));
      ps[p].status = FDFD_OK; ps[p].active = false; ps[p].relres = 0.0; ps[p].est = 0.0;
    } else {
      fdfd_ctx* h = bt->hs[p];
      ps[p].rs = ldexp(1.0, -ilogb(bn));
      if (ps[p].rs != 1.0) {  // ||rs b|| and, from x = 0, the first residual
        if ((rc = launch_residual64(nullptr, Jf(p), h->sb, 1, ps[p].rs, h->eps, h->cx64, h->cy64, h->k2, h->nx,
                                    h->ny, h->V, h->partials, h->counter, &h->st->resid, s)))
          return rc;
        bnorm_kernel<<<1, 1, 0, s>>>(h->st);
        CKL();
      }
      if (o->use_x0) {
        if ((rc = launch_load_field(Ef(p), h->x64, h->n, ps[p].rs, s))) return rc;
        if ((rc = launch_residual64(h->x64, Jf(p), h->sb, 1, ps[p].rs, h->eps, h->cx64, h->cy64, h->k2, h->nx,
                                    h->ny, h->V, h->partials, h->counter, &h->st->resid, s)))
          return rc;
      }
    }
  }
  // start of a cycle for the problems in `list`: beta, g0, true relres -> host
  auto cycle_start = [&](const std::vector<int>& list) -> int {
    for (int p : list) {
      fdfd_ctx* h = bt->hs[p];
      int r = launch_cycle_start(h->st, s);
      if (r) return r;
      CK(cudaMemcpyAsync(&bt->flags_h[2 * p], &h->st->est, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (int p : list) {
      PState& q = ps[p];
      double est = bt->flags_h[2 * p];
      int fl[2];
      memcpy(fl, &bt->flags_h[2 * p + 1], sizeof(fl));
      q.relres = q.est = est;
      q.j = 0;
      if (fl[0] || !isfinite(est)) { q.status = FDFD_ENUMERIC; q.active = false; continue; }
      if (est <= o->tol) { q.status = FDFD_OK; q.active = false; continue; }
      if (q.iters >= o->max_iters) { q.status = FDFD_NOT_CONVERGED; q.active = false; continue; }
      if (est > 0.99 * q.prev) { if (++q.stalls >= 3) { q.status = FDFD_STAGNATED; q.active = false; continue; } }
      else q.stalls = 0;
      q.prev = est;
    }
    return FDFD_OK;
  };
  {
    std::vector<int> all;
    for (int p = 0; p < n; ++p) if (ps[p].active) all.push_back(p);
    if ((rc = cycle_start(all))) return rc;
  }
  std::vector<int> finished;
  auto finish = [&](int p) -> int {
    fdfd_ctx* h = bt->hs[p];
    ProfScope ps_(h0, 4, 1);
    return launch_store_field(h->x64, Ef(p), h->n, 1.0 / ps[p].rs, s);
  };
  for (int p = 0; p < n; ++p)
    if (!ps[p].active && ps[p].status != FDFD_ENUMERIC && ps[p].relres > 0.0)
      if ((rc = finish(p))) return rc;
  int last_set = -1;
  for (;;) {
    std::vector<int> act;
    for (int p = 0; p < n; ++p) if (ps[p].active) act.push_back(p);
    if (act.empty()) break;
    // ---- preconditioner: one neural pass over all windows of all active problems whose
    // local solve is one network application; a problem whose local solver runs
    // NN-FGMRES steps applies its own preconditioner (local FGMRES and coarse correction) ----
    if (schwarz) {
      std::vector<int> one;
      for (int p : act) {
        fdfd_ctx* h = bt->hs[p];
        if (schwarz_inner_iters(h) == 0) { one.push_back(p); continue; }
        const size_t off = (size_t)ps[p].j * h->n;
        if ((rc = schwarz_apply(h, h->V + off, &h->st->vscale[ps[p].j], h->Z + off, 0))) return rc;
      }
      int nent = 0;
      for (int p : one) {
        fdfd_ctx* h = bt->hs[p];
        const size_t off = (size_t)ps[p].j * h->n;
        bt->ptab_h[p] = ProbGeom{h->nx, h->ny, h->nx / FDFD_CORE, (float)h->k2, h->eps, h->isx, h->isy,
                                 h->V + off, h->Z + off, &h->st->vscale[ps[p].j], schwarz_modulation(h)};
        for (int w = 0; w < n_windows(h); ++w) bt->wtab_h[nent++] = make_int2(p, w);
      }
      CK(cudaMemcpyAsync(bt->ptab_d, bt->ptab_h, (size_t)n * sizeof(ProbGeom), cudaMemcpyHostToDevice, s));
      if (last_set != (int)one.size()) {
        CK(cudaMemcpyAsync(bt->wtab_d, bt->wtab_h, (size_t)nent * sizeof(int2), cudaMemcpyHostToDevice, s));
        last_set = (int)one.size();
      }
      GridGeom g{h0->nx, h0->ny, h0->nx / FDFD_CORE, (float)h0->k2, h0->eps, h0->isx, h0->isy,
                 nullptr};  // entries take their problem's modulation from the table
      for (int st0 = 0; st0 < nent; st0 += bt->cap) {
        const int cnt = nent - st0 < bt->cap ? nent - st0 : bt->cap;
        NnoInput in;
        in.wtab = bt->wtab_d + st0;
        in.ptab = bt->ptab_d;
        NnoOutput out;  // outputs and scales come from the problem table
        if ((rc = nno_forward(schwarz_weights(h0), &bt->work, g, in, out, cnt, s, h0))) return rc;
      }
      // (the pinned tables are rewritten only after the flag read below has synchronised the stream)
      for (int p : one)
        if ((rc = schwarz_coarse(bt->hs[p], bt->hs[p]->Z + (size_t)ps[p].j * bt->hs[p]->n))) return rc;
    }
    // ---- per-problem Arnoldi step ----
    for (int p : act) {
      fdfd_ctx* h = bt->hs[p];
      const int j = ps[p].j;
      float2* vj = h->V + (size_t)j * h->n;
      float2* zj = h->Z + (size_t)j * h->n;
      const double* scj = &h->st->vscale[j];
      const float k2 = (float)h->k2;
      {
        ProfScope ps_(h0, 0, 1);
        if (o->precond == FDFD_PRECOND_JACOBI)
          rc = launch_stencil_jacobi(vj, scj, h->w, h->eps, h->cx, h->cy, k2, h->nx, h->ny, s);
        else {
          if (o->precond == FDFD_PRECOND_NONE && (rc = launch_scale_copy(vj, scj, zj, h->n, s))) return rc;
          rc = launch_stencil(zj, h->w, h->eps, h->cx, h->cy, k2, h->nx, h->ny, s);
        }
        if (rc) return rc;
      }
      {
        ProfScope ps_(h0, 1, (j + 32) / 32);
        if ((rc = launch_cgs_dots(h->V, h->n, j, h->w, h->n, h->st, h->partials, h->counter, s))) return rc;
      }
      {
        ProfScope ps_(h0, 2, (j + 32) / 32);
        if ((rc = launch_cgs_update(h->V, h->n, j, h->w, h->V + (size_t)(j + 1) * h->n, h->n, h->st, h->partials,
                                    h->counter, m, s)))
          return rc;
      }
      CK(cudaMemcpyAsync(&bt->flags_h[2 * p], &h->st->est, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    std::vector<int> ending;
    for (int p : act) {
      PState& q = ps[p];
      const double est = bt->flags_h[2 * p];
      int fl[2];
      memcpy(fl, &bt->flags_h[2 * p + 1], sizeof(fl));
      ++q.iters;
      q.est = est;
      if (fl[0]) { q.status = FDFD_ENUMERIC; q.active = false; continue; }
      if (est <= o->tol || fl[1] || q.iters >= o->max_iters || q.j + 1 == m) ending.push_back(p);
      else ++q.j;
    }
    // ---- end of a cycle: x += Z y, FP64 true residual, next cycle ----
    for (int p : ending) {
      fdfd_ctx* h = bt->hs[p];
      const int k = ps[p].j + 1;
      ProfScope ps_(h0, 4, 2);
      if ((rc = launch_solve_y(h->st, k, m, s))) return rc;
      if (o->precond == FDFD_PRECOND_JACOBI)
        rc = launch_x_update_jacobi(h->x64, h->V, h->n, k, h->n, h->st, h->eps, h->cx, h->cy, (float)h->k2, h->nx, s);
      else
        rc = launch_x_update(h->x64, h->Z, h->n, k, h->n, h->st, s);
      if (rc) return rc;
      ++ps[p].cycles;
      if ((rc = launch_residual64(h->x64, Jf(p), h->sb, 1, ps[p].rs, h->eps, h->cx64, h->cy64, h->k2, h->nx, h->ny, h->V,
                                  h->partials, h->counter, &h->st->resid, s)))
        return rc;
    }
    if (!ending.empty()) {
      if ((rc = cycle_start(ending))) return rc;
      for (int p : ending)
        if (!ps[p].active && ps[p].status != FDFD_ENUMERIC)
          if ((rc = finish(p))) return rc;
    }
  }
  CK(cudaEventRecord(h0->ev1, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h0->ev0, h0->ev1);
  int worst = FDFD_OK;
  for (int p = 0; p < n; ++p) {
    if (stats) {
      stats[p].iters = ps[p].iters;
      stats[p].restarts = ps[p].cycles;
      stats[p].status = ps[p].status;
      stats[p].relres_true = ps[p].relres;
      stats[p].relres_est = ps[p].est;
      stats[p].t_solve_ms = ms;
    }
    if (ps[p].status < 0) worst = ps[p].status;
    else if (worst >= 0 && ps[p].status > worst) worst = ps[p].status;
  }
  return worst;
}
