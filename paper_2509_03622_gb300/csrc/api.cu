// C-ABI entry points (include/fdfd.h): handle life cycle, UPML set-up,
// and the flexible GMRES driver of Algorithm 1 with restarts.
//
// The driver keeps the iterate in FP64 and recomputes the true residual
// b~ - A~ x in FP64 at every restart (iterative refinement); inside a
// cycle the Krylov vectors are complex64 and the dots / norms / Hessenberg
// least squares are FP64.  The host only reads one 16-byte status word per
// Arnoldi step (the least-squares residual estimate and error flags).
#include <math.h>
#include <string.h>
#include <vector>
#include <complex>
#include "ctx.cuh"
#include "nno.cuh"
#include "local.cuh"

void graphs_invalidate(fdfd_ctx* h) {
  for (auto& g : h->graphs) {
    for (auto& e : g.exec)
      if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    g.key = -1;
  }
}

namespace {

constexpr double MU0 = 1.25663706212e-6;    // vacuum permeability (CODATA 2018)
constexpr double C0 = 299792458.0;          // speed of light
constexpr int RESTART_CAP = 32;
const double kOne = 1.0;

typedef std::complex<double> zd;

// UPML stretching along one axis (Methods, Eq. 6): s = 1 - j sigma/(w eps0),
// sigma/(w eps0) = -(m+1) lnR / (2 npml k0dx) * (depth/npml)^m, depth measured
// in cells from the inner PML interface; nodes at i + 1/2, faces at i.
void stretch(int n, int lo, int hi, double k0dx, double m, double lnR, std::vector<zd>& sn,
             std::vector<zd>& sh) {
  sn.assign(n, zd(1, 0));
  sh.assign(n + 1, zd(1, 0));
  auto s_at = [&](double p) {
    double sig = 0;
    if (lo > 0 && p < lo) sig += -(m + 1) * lnR / (2.0 * lo * k0dx) * pow((lo - p) / lo, m);
    if (hi > 0 && p > n - hi) sig += -(m + 1) * lnR / (2.0 * hi * k0dx) * pow((p - (n - hi)) / hi, m);
    return zd(1.0, -sig);
  };
  for (int i = 0; i < n; ++i) sn[i] = s_at(i + 0.5);
  for (int i = 0; i <= n; ++i) sh[i] = s_at((double)i);
}

void axis_coefs(int n, const std::vector<zd>& sn, const std::vector<zd>& sh, std::vector<AxisCoef64>& A,
                std::vector<AxisCoef64>& AT) {
  std::vector<zd> lo(n), hi(n);
  for (int i = 0; i < n; ++i) {
    lo[i] = 1.0 / (sn[i] * sh[i]);
    hi[i] = 1.0 / (sn[i] * sh[i + 1]);
  }
  A.resize(n);
  AT.resize(n);
  for (int i = 0; i < n; ++i) {
    zd dg = -(lo[i] + hi[i]);
    zd loT = i > 0 ? hi[i - 1] : zd(0, 0);
    zd hiT = i + 1 < n ? lo[i + 1] : zd(0, 0);
    A[i] = {make_double2(lo[i].real(), lo[i].imag()), make_double2(hi[i].real(), hi[i].imag()),
            make_double2(dg.real(), dg.imag())};
    AT[i] = {make_double2(loT.real(), loT.imag()), make_double2(hiT.real(), hiT.imag()),
             make_double2(dg.real(), dg.imag())};
  }
}

std::vector<AxisCoef> to_f32(const std::vector<AxisCoef64>& a) {
  std::vector<AxisCoef> o(a.size());
  for (size_t i = 0; i < a.size(); ++i)
    o[i] = {make_float2((float)a[i].lo.x, (float)a[i].lo.y), make_float2((float)a[i].hi.x, (float)a[i].hi.y),
            make_float2((float)a[i].dg.x, (float)a[i].dg.y)};
  return o;
}

template <class T>
int dalloc(fdfd_ctx* h, T** p, size_t count) {
  const size_t b = count * sizeof(T);
  if (cudaMalloc((void**)p, b) != cudaSuccess) { *p = nullptr; return FDFD_ENOMEM; }
  h->bytes += b;
  return FDFD_OK;
}

template <class T>
int upload(fdfd_ctx* h, T** p, const std::vector<T>& v) {
  int rc = dalloc(h, p, v.size());
  if (rc) return rc;
  CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FDFD_OK;
}

int setup_coefs(fdfd_ctx* h) {
  std::vector<zd> sxn, sxh, syn, syh;
  stretch(h->nx, h->npml[0], h->npml[1], h->k0dx, h->pml_m, h->pml_lnR, sxn, sxh);
  stretch(h->ny, h->npml[2], h->npml[3], h->k0dx, h->pml_m, h->pml_lnR, syn, syh);
  std::vector<AxisCoef64> ax, axT, ay, ayT;
  axis_coefs(h->nx, sxn, sxh, ax, axT);
  axis_coefs(h->ny, syn, syh, ay, ayT);
  int rc;
  if ((rc = upload(h, &h->cx64, ax)) || (rc = upload(h, &h->cxT64, axT)) || (rc = upload(h, &h->cy64, ay)) ||
      (rc = upload(h, &h->cyT64, ayT)))
    return rc;
  if ((rc = upload(h, &h->cx, to_f32(ax))) || (rc = upload(h, &h->cxT, to_f32(axT))) ||
      (rc = upload(h, &h->cy, to_f32(ay))) || (rc = upload(h, &h->cyT, to_f32(ayT))))
    return rc;
  std::vector<float2> ix(h->nx), iy(h->ny);
  for (int i = 0; i < h->nx; ++i) { zd v = 1.0 / sxn[i]; ix[i] = make_float2((float)v.real(), (float)v.imag()); }
  for (int j = 0; j < h->ny; ++j) { zd v = 1.0 / syn[j]; iy[j] = make_float2((float)v.real(), (float)v.imag()); }
  if ((rc = upload(h, &h->isx, ix)) || (rc = upload(h, &h->isy, iy))) return rc;
  return FDFD_OK;
}

void release(fdfd_ctx* h) {
  if (!h) return;
  graphs_invalidate(h);
  schwarz_destroy(h);
  void* ptrs[] = {h->eps, h->cx, h->cy, h->cxT, h->cyT, h->cx64, h->cy64, h->cxT64, h->cyT64, h->isx, h->isy,
                  h->V, h->Z, h->w, h->x64, h->st, h->partials, h->counter, h->hostJ, h->hostE, h->d_one,
                  h->adj};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->flag_host) cudaFreeHost(h->flag_host);
  if (h->prof_ev) {
    for (int i = 0; i < 2 * PROF_POOL; ++i) cudaEventDestroy(h->prof_ev[i]);
    delete[] h->prof_ev;
    delete[] h->prof_cls;
  }
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

int read_flags(fdfd_ctx* h, double* est, int* nonfinite, int* breakdown) {
  CK(cudaMemcpyAsync(h->flag_host, &h->st->est, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *est = h->flag_host[0];
  int fl[2];
  memcpy(fl, &h->flag_host[1], sizeof(fl));
  *nonfinite = fl[0];
  *breakdown = fl[1];
  return FDFD_OK;
}

int read_double(fdfd_ctx* h, const double* dev, double* out) {
  CK(cudaMemcpyAsync(h->flag_host, dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = h->flag_host[0];
  return FDFD_OK;
}

__global__ void to_f64_kernel(const float2* __restrict__ u, double2* __restrict__ x, size_t n) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    x[c] = make_double2((double)u[c].x, (double)u[c].y);
}

__global__ void set_bnorm_kernel(KrylovState* st) {
  st->bnorm = sqrt(st->resid);
  st->nonfinite = 0;
  st->breakdown = 0;
}

// CUDA graphs of the m Arnoldi steps for `key`, captured on first use (the
// capture only records launches; nothing runs).  Kernels counted during the
// capture are booked per replay instead.  Returns nullptr (eager launches)
// if any capture fails, and stops trying for this handle.
template <class Step>
fdfd_ctx::StepGraphs* step_graphs(fdfd_ctx* h, int key, int m, Step& issue_step) {
  for (auto& g : h->graphs)
    if (g.key == key) return &g;
  fdfd_ctx::StepGraphs& g = h->graphs[h->graph_next];
  h->graph_next = (h->graph_next + 1) % 4;
  for (auto& e : g.exec)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  g.key = -1;
  // capture on the handle's private stream (the caller's may be the legacy
  // default stream, which cannot be captured); replays go to the caller's
  cudaStream_t user = h->stream;
  h->stream = h->cap_stream;
  for (int j = 0; j < m; ++j) {
    const long long before = h->launches_total;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();
      h->graphs_ok = false;
      break;
    }
    const int rc = issue_step(j);
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    g.nk[j] = h->launches_total - before;
    h->launches_total = before;
    if (rc || ce != cudaSuccess || !graph || cudaGraphInstantiate(&g.exec[j], graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      h->graphs_ok = false;
      break;
    }
    cudaGraphDestroy(graph);
  }
  h->stream = user;
  cudaGetLastError();
  if (!h->graphs_ok) {
    for (auto& e : g.exec)
      if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    return nullptr;
  }
  g.key = key;
  return &g;
}

// One FGMRES(restart) solve of A~ x = rhs (or A~^T x = rhs).
int solve_impl(fdfd_ctx* h, const float2* rhs, int rhs_is_source, int transpose, float2* E,
               const fdfd_solve_opts* o, fdfd_solve_stats* stats) {
  if (!h || !rhs || !E || !o) return FDFD_EINVAL;
  if (o->restart < 1 || o->restart > h->rmax || o->max_iters < 0 || !(o->tol > 0)) return FDFD_EINVAL;
  if (o->precond < FDFD_PRECOND_NONE || o->precond > FDFD_PRECOND_SCHWARZ) return FDFD_EINVAL;
  if (o->precond == FDFD_PRECOND_SCHWARZ && !h->sw) return FDFD_ENOSETUP;
  cudaStream_t s = h->stream;
  const AxisCoef* cx = transpose ? h->cxT : h->cx;
  const AxisCoef* cy = transpose ? h->cyT : h->cy;
  const AxisCoef64* cx64 = transpose ? h->cxT64 : h->cx64;
  const AxisCoef64* cy64 = transpose ? h->cyT64 : h->cy64;
  const size_t n = h->n;
  const int m = o->restart;
  const float k2 = (float)h->k2;
  int rc;
  fdfd_solve_stats loc{};
  CK(cudaEventRecord(h->ev0, s));
  // ||b|| via the residual of x = 0
  CK(cudaMemsetAsync(h->x64, 0, n * sizeof(double2), s));
  {
    ProfScope ps(h, 16, 2);
    if ((rc = launch_residual64(nullptr, rhs, h->sb, rhs_is_source, 1.0, h->eps, cx64, cy64, h->k2, h->nx, h->ny,
                                h->V, h->partials, h->counter, &h->st->resid, s)))
      return rc;
    set_bnorm_kernel<<<1, 1, 0, s>>>(h->st);
    CKL();
  }
  double bnorm;
  if ((rc = read_double(h, &h->st->bnorm, &bnorm))) return rc;
  if (!isfinite(bnorm)) return FDFD_ENUMERIC;
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(E, 0, n * sizeof(float2), s));
    CK(cudaStreamSynchronize(s));
    if (stats) { *stats = loc; stats->status = FDFD_OK; }
    return FDFD_OK;
  }
  // Solve the system scaled by a power of two so that ||rs b|| is in [1, 2):
  // right-hand sides of any magnitude (an adjoint source is often ~1e-20)
  // then keep the FP32 sums of squares inside the preconditioner and the
  // local solves far from underflow.  x64 holds rs x; the scaling is exact.
  const double rs = ldexp(1.0, -ilogb(bnorm));
  if (rs != 1.0) {
    ProfScope ps(h, 16, 2);
    if ((rc = launch_residual64(nullptr, rhs, h->sb, rhs_is_source, rs, h->eps, cx64, cy64, h->k2, h->nx, h->ny,
                                h->V, h->partials, h->counter, &h->st->resid, s)))
      return rc;
    set_bnorm_kernel<<<1, 1, 0, s>>>(h->st);
    CKL();
  }
  if (o->use_x0) {
    ProfScope ps(h, 4, 1);
    if ((rc = launch_load_field(E, h->x64, n, rs, s))) return rc;
  }
  // one Arnoldi step j: z_j = M v_j, w = A~ z_j, CGS against v_0..v_j, v_{j+1}
  auto issue_step = [&](int j) -> int {
    int r;
    cudaStream_t s = h->stream;  // the private capture stream while a graph is recorded
    float2* vj = h->V + (size_t)j * n;
    float2* zj = h->Z + (size_t)j * n;
    const double* scj = &h->st->vscale[j];
    if (o->precond == FDFD_PRECOND_JACOBI) {
      ProfScope ps(h, 0, 1);
      r = launch_stencil_jacobi(vj, scj, h->w, h->eps, cx, cy, k2, h->nx, h->ny, s);
    } else {
      if (o->precond == FDFD_PRECOND_NONE) {
        ProfScope ps(h, 4, 1);
        r = launch_scale_copy(vj, scj, zj, n, s);
      } else {
        r = schwarz_apply(h, vj, scj, zj, transpose);
      }
      if (r) return r;
      ProfScope ps(h, 0, 1);
      r = launch_stencil(zj, h->w, h->eps, cx, cy, k2, h->nx, h->ny, s);
    }
    if (r) return r;
    {
      ProfScope ps(h, 1, (j + 16) / 16);
      if ((r = launch_cgs_dots(h->V, n, j, h->w, n, h->st, h->partials, h->counter, s))) return r;
    }
    ProfScope ps(h, 2, (j + 16) / 16);
    return launch_cgs_update(h->V, n, j, h->w, h->V + (size_t)(j + 1) * n, n, h->st, h->partials, h->counter, m,
                             s);
  };
  fdfd_ctx::StepGraphs* G = nullptr;
  if (o->use_graphs && !h->prof_on && h->graphs_ok)
    G = step_graphs(h, o->precond + 3 * transpose + 6 * m, m, issue_step);
  int iters = 0, cycles = 0, status = FDFD_NOT_CONVERGED;
  double est = 1.0, relres = 1.0, prev_relres = INFINITY;
  int stalls = 0;
  for (;;) {
    if (cycles > 0 || o->use_x0) {
      ProfScope ps(h, 3, 1);
      if ((rc = launch_residual64(h->x64, rhs, h->sb, rhs_is_source, rs, h->eps, cx64, cy64, h->k2, h->nx,
                                  h->ny, h->V, h->partials, h->counter, &h->st->resid, s)))
        return rc;
    }
    {
      ProfScope ps(h, 4, 1);
      if ((rc = launch_cycle_start(h->st, s))) return rc;
    }
    int nonfinite = 0, breakdown = 0;
    if ((rc = read_flags(h, &relres, &nonfinite, &breakdown))) return rc;
    if (nonfinite) { status = FDFD_ENUMERIC; break; }
    if (o->precond == FDFD_PRECOND_SCHWARZ && (rc = schwarz_error(h))) { status = rc; break; }
    est = relres;
    if (relres <= o->tol) { status = FDFD_OK; break; }
    if (iters >= o->max_iters) { status = FDFD_NOT_CONVERGED; break; }
    // stagnation: three cycles in a row that do not lower the true residual by 1%
    if (relres > 0.99 * prev_relres) { if (++stalls >= 3) { status = FDFD_STAGNATED; break; } }
    else stalls = 0;
    prev_relres = relres;
    int k = 0;
    for (int j = 0; j < m; ++j) {
      if (G) {
        CK(cudaGraphLaunch(G->exec[j], s));
        h->launches_total += G->nk[j];
      } else if ((rc = issue_step(j))) {
        return rc;
      }
      ++iters;
      k = j + 1;
      if ((rc = read_flags(h, &est, &nonfinite, &breakdown))) return rc;
      if (nonfinite) { status = FDFD_ENUMERIC; break; }
      if (est <= o->tol || breakdown || iters >= o->max_iters) break;
    }
    if (status == FDFD_ENUMERIC) break;
    if (o->precond == FDFD_PRECOND_SCHWARZ && (rc = schwarz_error(h))) { status = rc; break; }
    ProfScope ps(h, 4, 2);
    if ((rc = launch_solve_y(h->st, k, m, s))) return rc;
    if (o->precond == FDFD_PRECOND_JACOBI)
      rc = launch_x_update_jacobi(h->x64, h->V, n, k, n, h->st, h->eps, cx, cy, k2, h->nx, s);
    else
      rc = launch_x_update(h->x64, h->Z, n, k, n, h->st, s);
    if (rc) return rc;
    ++cycles;
  }
  if (status != FDFD_ENUMERIC && status != FDFD_ETIMEOUT) {
    ProfScope ps(h, 4, 1);
    if ((rc = launch_store_field(h->x64, E, n, 1.0 / rs, s))) return rc;
  }
  CK(cudaEventRecord(h->ev1, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  if (stats) {
    stats->iters = iters;
    stats->restarts = cycles;
    stats->status = status;
    stats->relres_true = relres;
    stats->relres_est = est;
    stats->t_solve_ms = ms;
  }
  return status;
}

}  // namespace

extern "C" {

const char* fdfd_status_string(int code) {
  switch (code) {
    case FDFD_OK: return "ok";
    case FDFD_NOT_CONVERGED: return "not converged (max_iters reached)";
    case FDFD_STAGNATED: return "stagnated (restart cycles made no progress)";
    case FDFD_EINVAL: return "invalid argument";
    case FDFD_ECUDA: return "CUDA error";
    case FDFD_ENUMERIC: return "NaN or Inf in the iteration";
    case FDFD_ETIMEOUT: return "bounded device wait expired";
    case FDFD_ENOSETUP: return "schwarz_setup required";
    case FDFD_ENOMEM: return "device allocation failed";
    default: return "unknown status";
  }
}

int fdfd_create(const fdfd_desc* d, fdfd_handle* out) {
  if (!out) return FDFD_EINVAL;
  *out = nullptr;
  if (!d || !d->eps) return FDFD_EINVAL;
  if (d->nx < 2 * FDFD_CORE || d->ny < 2 * FDFD_CORE || d->nx % FDFD_CORE || d->ny % FDFD_CORE) return FDFD_EINVAL;
  if (!(d->dx > 0) || !(d->wavelength > 0) || !(d->pml_m >= 0) || !(d->pml_lnR < 0)) return FDFD_EINVAL;
  for (int i = 0; i < 4; ++i) {
    const int n = i < 2 ? d->nx : d->ny;
    if (d->npml[i] < 0 || 2 * d->npml[i] >= n) return FDFD_EINVAL;
  }
  if (d->max_restart < 0 || d->max_restart > FDFD_MAXRESTART) return FDFD_EINVAL;
  fdfd_ctx* h = new fdfd_ctx();
  h->nx = d->nx; h->ny = d->ny; h->n = (size_t)d->nx * d->ny;
  h->dx = d->dx; h->wavelength = d->wavelength; h->pml_m = d->pml_m; h->pml_lnR = d->pml_lnR;
  memcpy(h->npml, d->npml, sizeof(h->npml));
  h->k0dx = 2.0 * M_PI * d->dx / d->wavelength;
  h->k2 = h->k0dx * h->k0dx;
  const double omega = 2.0 * M_PI * C0 / d->wavelength;
  h->sb = d->dx * d->dx * omega * MU0;
  h->stream = (cudaStream_t)d->stream;
  h->rmax = d->max_restart ? d->max_restart : RESTART_CAP;
  int rc = FDFD_OK;
  const size_t n = h->n;
  if ((rc = dalloc(h, &h->eps, n)) || (rc = setup_coefs(h)) ||
      (rc = dalloc(h, &h->V, (size_t)(h->rmax + 1) * n)) || (rc = dalloc(h, &h->Z, (size_t)h->rmax * n)) ||
      (rc = dalloc(h, &h->w, n)) || (rc = dalloc(h, &h->x64, n)) || (rc = dalloc(h, &h->st, 1)) ||
      (rc = dalloc(h, &h->partials, (size_t)8192 * FDFD_MAXRESTART * 2)) || (rc = dalloc(h, &h->counter, 4)) ||
      (rc = dalloc(h, &h->d_one, 1)) || (rc = dalloc(h, &h->adj, n))) {
    release(h);
    return rc;
  }
  if (cudaMemcpy(h->eps, d->eps, n * sizeof(float), cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemset(h->counter, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->st, 0, sizeof(KrylovState)) != cudaSuccess ||
      cudaMemcpy(h->d_one, &kOne, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMallocHost((void**)&h->flag_host, 4 * sizeof(double)) != cudaSuccess ||
      cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    release(h);
    return FDFD_ECUDA;
  }
  *out = h;
  return FDFD_OK;
}

int fdfd_set_eps(fdfd_handle h, const float* eps_dev) {
  if (!h || !eps_dev) return FDFD_EINVAL;
  CK(cudaMemcpyAsync(h->eps, eps_dev, h->n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  graphs_invalidate(h);
  schwarz_destroy(h);
  return FDFD_OK;
}

int schwarz_setup(fdfd_handle h, const schwarz_desc* sd) {
  if (!h || !sd) return FDFD_EINVAL;
  graphs_invalidate(h);
  schwarz_destroy(h);
  return schwarz_create(h, sd);
}

void fdfd_destroy(fdfd_handle h) { release(h); }

int fdfd_get_info(fdfd_handle h, fdfd_info* info) {
  if (!h || !info) return FDFD_EINVAL;
  memset(info, 0, sizeof(*info));
  info->nwx = h->nx / FDFD_CORE;
  info->nwy = h->ny / FDFD_CORE;
  info->n_win = info->nwx * info->nwy;
  info->workspace_bytes = h->bytes;
  for (auto& g : h->graphs) info->graphs_cached += g.key >= 0;
  info->graphs_ok = h->graphs_ok;
  if (h->sw) schwarz_info(h, info);
  return FDFD_OK;
}

int fdfd_solve(fdfd_handle h, const fdfd_c64* J, fdfd_c64* E, const fdfd_solve_opts* o, fdfd_solve_stats* st) {
  return solve_impl(h, reinterpret_cast<const float2*>(J), 1, 0, reinterpret_cast<float2*>(E), o, st);
}

int fdfd_solve_host(fdfd_handle h, const fdfd_c64* J, fdfd_c64* E, const fdfd_solve_opts* o,
                    fdfd_solve_stats* st) {
  if (!h || !J || !E) return FDFD_EINVAL;
  if (!h->hostJ) {
    int rc;
    if ((rc = dalloc(h, &h->hostJ, h->n)) || (rc = dalloc(h, &h->hostE, h->n))) return rc;
  }
  CK(cudaMemcpyAsync(h->hostJ, J, h->n * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
  if (o && o->use_x0) CK(cudaMemcpyAsync(h->hostE, E, h->n * sizeof(float2), cudaMemcpyHostToDevice, h->stream));
  const int rc = solve_impl(h, h->hostJ, 1, 0, h->hostE, o, st);
  if (rc >= 0) {
    CK(cudaMemcpyAsync(E, h->hostE, h->n * sizeof(float2), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return rc;
}

// Adjoint solve through the symmetrised operator: with D = diag(s_x s_y)
// (UPML factors at cell centres), D A~ is complex symmetric, so
// A~^T = D A~ D^-1 and  A~^T lam = g  <=>  A~ mu = D^-1 g,  lam = D mu.
// The forward machinery (and its preconditioner, built for A~) then solves
// the adjoint exactly; the reported relres is the adjoint's own FP64 one.
int fdfd_solve_adjoint(fdfd_handle h, const fdfd_c64* g, fdfd_c64* lam, const fdfd_solve_opts* o,
                       fdfd_solve_stats* st) {
  if (!h || !g || !lam || !o) return FDFD_EINVAL;
  float2* L = reinterpret_cast<float2*>(lam);
  const float2* G = reinterpret_cast<const float2*>(g);
  cudaStream_t s = h->stream;
  int rc;
  {
    ProfScope ps(h, 4, o->use_x0 ? 2 : 1);
    if (o->use_x0 && (rc = launch_scale_d(L, L, h->isx, h->isy, h->nx, h->n, 1, s))) return rc;
    if ((rc = launch_scale_d(G, h->adj, h->isx, h->isy, h->nx, h->n, 1, s))) return rc;
  }
  fdfd_solve_stats loc{};
  const int status = solve_impl(h, h->adj, 0, 0, L, o, &loc);
  if (status < 0) { if (st) *st = loc; return status; }
  {
    ProfScope ps(h, 4, 1);
    if ((rc = launch_scale_d(L, L, h->isx, h->isy, h->nx, h->n, 0, s))) return rc;
  }
  // ||g - A~^T lam|| / ||g|| in FP64
  double r2[2];
  for (int pass = 0; pass < 2; ++pass) {
    ProfScope ps(h, 3, 2);
    if (pass == 1 && (rc = launch_load_field(L, h->x64, h->n, 1.0, s))) return rc;
    if ((rc = launch_residual64(pass ? h->x64 : nullptr, G, h->sb, 0, 1.0, h->eps, h->cxT64, h->cyT64, h->k2, h->nx, h->ny, h->V,
                                h->partials, h->counter, &h->st->resid, s)))
      return rc;
    if ((rc = read_double(h, &h->st->resid, &r2[pass]))) return rc;
  }
  loc.relres_true = r2[0] > 0 ? sqrt(r2[1] / r2[0]) : 0.0;
  if (st) *st = loc;
  return status;
}

int fdfd_grad_eps(fdfd_handle h, const fdfd_c64* E, const fdfd_c64* lam, float* grad, int accumulate) {
  if (!h || !E || !lam || !grad) return FDFD_EINVAL;
  int rc = launch_grad_eps(reinterpret_cast<const float2*>(E), reinterpret_cast<const float2*>(lam), grad,
                           (float)h->k2, (int)h->n, accumulate, h->stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_apply_A(fdfd_handle h, const fdfd_c64* x, fdfd_c64* y, int transpose) {
  if (!h || !x || !y) return FDFD_EINVAL;
  ProfScope ps(h, 0, 1);
  int rc = launch_stencil(reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y), h->eps,
                          transpose ? h->cxT : h->cx, transpose ? h->cyT : h->cy, (float)h->k2, h->nx, h->ny,
                          h->stream);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_precond_apply(fdfd_handle h, const fdfd_c64* v, fdfd_c64* z) {
  if (!h || !v || !z) return FDFD_EINVAL;
  if (!h->sw) return FDFD_ENOSETUP;
  int rc = schwarz_apply(h, reinterpret_cast<const float2*>(v), h->d_one, reinterpret_cast<float2*>(z), 0);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_nno_solve(fdfd_handle h, const fdfd_c64* r_win, const fdfd_c64* g_win, const int* win_id, int n,
                   fdfd_c64* e_win) {
  if (!h || !r_win || !g_win || !win_id || !e_win || n < 0) return FDFD_EINVAL;
  if (!h->sw) return FDFD_ENOSETUP;
  int rc = schwarz_nno_solve(h, reinterpret_cast<const float2*>(r_win), reinterpret_cast<const float2*>(g_win),
                             win_id, n, reinterpret_cast<float2*>(e_win));
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_local_apply(fdfd_handle h, const fdfd_c64* x, fdfd_c64* y, const int* win_id, int n) {
  if (!h || !x || !y || !win_id || n < 0) return FDFD_EINVAL;
  if (n == 0) return FDFD_OK;
  int rc = local_apply_windows(h, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y), win_id, n);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_trace_extract(fdfd_handle h, const fdfd_c64* u, fdfd_c64* g) {
  if (!h || !u || !g) return FDFD_EINVAL;
  int rc = schwarz_traces(h, reinterpret_cast<const float2*>(u), reinterpret_cast<float2*>(g));
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_schwarz_stationary(fdfd_handle h, const fdfd_c64* b_dev, fdfd_c64* u_dev, int max_iters, double tol,
                            double momentum, int* iters, double* relres) {
  if (!h || !b_dev || !u_dev || max_iters < 1 || !(tol >= 0.0) || !(momentum >= 0.0 && momentum < 1.0))
    return FDFD_EINVAL;
  if (!h->sw) return FDFD_ENOSETUP;
  const float2* b = reinterpret_cast<const float2*>(b_dev);
  float2* u = reinterpret_cast<float2*>(u_dev);
  cudaStream_t s = h->stream;
  const size_t n_win = (size_t)(h->nx / FDFD_CORE) * (h->ny / FDFD_CORE), nt = n_win * 4 * FDFD_WIN;
  // Robin data, new traces and the inner solver's window right-hand sides
  // live in the FGMRES search-direction space Z (rmax x n >= 1.8 n)
  float2 *g = h->Z, *g_new = h->Z + nt, *rhs = h->Z + 2 * nt;
  int rc;
  if ((rc = schwarz_error(h))) return rc;
  CK(cudaMemsetAsync(g, 0, nt * sizeof(float2), s));
  double b2 = 0.0, r2 = 0.0;
  if ((rc = launch_residual64(nullptr, b, h->sb, 0, 1.0, h->eps, h->cx64, h->cy64, h->k2, h->nx, h->ny, h->w,
                              h->partials, h->counter, &h->st->resid, s)) ||
      (rc = read_double(h, &h->st->resid, &b2)))
    return rc;
  int it = 0;
  double rr = 0.0;
  if (b2 == 0.0) {  // u = 0 solves it exactly
    CK(cudaMemsetAsync(u, 0, h->n * sizeof(float2), s));
  } else {
    for (it = 1; it <= max_iters; ++it) {
      if ((rc = schwarz_sweep_data(h, b, g, u, rhs)) || (rc = schwarz_stationary_update(h, u, g, g_new, momentum)))
        return rc;
      to_f64_kernel<<<krylov_grid(h->n), 256, 0, s>>>(u, h->x64, h->n);
      CKL();
      if ((rc = launch_residual64(h->x64, b, h->sb, 0, 1.0, h->eps, h->cx64, h->cy64, h->k2, h->nx, h->ny, h->w,
                                  h->partials, h->counter, &h->st->resid, s)) ||
          (rc = read_double(h, &h->st->resid, &r2)) || (rc = schwarz_error(h)))
        return rc;
      rr = sqrt(r2 / b2);
      if (!isfinite(rr) || rr <= tol) break;
    }
    if (it > max_iters) it = max_iters;
  }
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return isfinite(rr) ? FDFD_OK : FDFD_ENUMERIC;
}

int fdfd_profile_start(fdfd_handle h) {
  if (!h || h->prof_on) return FDFD_EINVAL;
  if (!h->prof_ev) {
    h->prof_ev = new cudaEvent_t[2 * PROF_POOL];
    h->prof_cls = new int[PROF_POOL];
    for (int i = 0; i < 2 * PROF_POOL; ++i) CK(cudaEventCreate(&h->prof_ev[i]));
  }
  h->prof_on = true;
  h->prof_next = 0;
  for (int c = 0; c < FDFD_PROF_NCLASS; ++c) h->prof_launch[c] = 0;
  h->launches_total = 0;
  return FDFD_OK;
}

int fdfd_profile_stop(fdfd_handle h, fdfd_profile* out) {
  if (!h || !h->prof_on || !out) return FDFD_EINVAL;
  h->prof_on = false;
  CK(cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof(*out));
  for (int i = 0; i < h->prof_next; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    out->ms[h->prof_cls[i]] += ms;
  }
  for (int c = 0; c < FDFD_PROF_NCLASS; ++c) out->launches[c] = h->prof_launch[c];
  out->total_launches = h->launches_total;
  return FDFD_OK;
}

int fdfd_selftest_wait(void) {
  int r = 0;
  const int rc = nno_wait_selftest(&r, 0);
  if (rc) return rc;
  return r == 2 ? FDFD_ETIMEOUT : FDFD_OK;
}

int fdfd_nno_mark_failed(fdfd_handle h) { return schwarz_mark_failed(h); }

int fdfd_selftest_gemm(const void* A, const void* B, float* C, int M, int N, int K, int a_mn) {
  if (!A || !B || !C || M <= 0) return FDFD_EINVAL;
  int* err = nullptr;
  CK(cudaMalloc(&err, sizeof(int)));
  CK(cudaMemset(err, 0, sizeof(int)));
  int rc = nno_gemm_selftest(reinterpret_cast<const bf16*>(A), reinterpret_cast<const bf16*>(B), C, M, N, K, a_mn,
                             err, 0);
  int e = 0;
  if (!rc) {
    if (cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = FDFD_ECUDA;
  }
  cudaFree(err);
  if (!rc && e) rc = FDFD_ETIMEOUT;
  return rc;
}

int fdfd_coarse_ritz(fdfd_handle h, double* eta_host, double* H_host) {
  if (!h) return FDFD_EINVAL;
  if (!h->sw) return FDFD_ENOSETUP;
  return schwarz_ritz_export(h, eta_host, H_host);
}

int fdfd_coarse_export(fdfd_handle h, double* Q, double* G) {
  if (!h) return FDFD_EINVAL;
  if (!h->sw) return FDFD_ENOSETUP;
  return schwarz_export(h, Q, G);
}

int fdfd_coarse_solve(fdfd_handle h, const fdfd_c64* ebc, fdfd_c64* z) {
  if (!h || !ebc || !z) return FDFD_EINVAL;
  if (!h->sw) return FDFD_ENOSETUP;
  return schwarz_coarse_solve(h, reinterpret_cast<const float2*>(ebc), reinterpret_cast<float2*>(z));
}

}  // extern "C"
