// Two-level Schwarz preconditioner (Algorithm 3 as one sweep from a zero
// guess): partition kernels, neural local solves and the coarse space.
#include "ctx.cuh"
#include "nno.cuh"
#include "local.cuh"

struct CoarseData;
void coarse_free(CoarseData* c);
int coarse_setup(fdfd_ctx* h, const NnoWeights* W, NnoWork* work, LocalWork* L, int k, double ritz_tol,
                 CoarseData** out, size_t* bytes);
int coarse_kept(CoarseData* c);
int coarse_ritz_export(fdfd_ctx* h, CoarseData* c, double* eta_host, double* H_host);
int coarse_apply(fdfd_ctx* h, CoarseData* c, float2* u, const float2* g_ref = nullptr);
int coarse_export(fdfd_ctx* h, CoarseData* c, double* Qh, double* Gh);
int coarse_solve_mismatch(fdfd_ctx* h, CoarseData* c, const float2* ebc, float2* z);

struct SchwarzData {
  int k = 0, n_win = 0, nwx = 0, precision = 0, inner = 0;
  NnoWeights W;
  NnoWork work;
  LocalWork local;
  CoarseData* coarse = nullptr;
  float* mod = nullptr;  // per-window modulation [n_win][4][512] of the modified FNO, or nullptr
  size_t bytes = 0;
};

namespace {

// Robin traces (Eq. 2, dx-scaled): g = u_o - u_b + j kd_b u_b on the
// interface sides of every window; zero on grid-edge sides.
__global__ void traces_kernel(const float2* __restrict__ u, const float* __restrict__ eps, float k0dx,
                              int nx, int ny, int nwx, int n_win, float2* __restrict__ g) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_win * 4 * FDFD_WIN) return;
  const int t = idx % FDFD_WIN, s = (idx / FDFD_WIN) % 4, w = idx / (4 * FDFD_WIN);
  const int a = w % nwx, b = w / nwx;
  const int x0 = min(max(FDFD_CORE * a - FDFD_OVL, 0), nx - FDFD_WIN);
  const int y0 = min(max(FDFD_CORE * b - FDFD_OVL, 0), ny - FDFD_WIN);
  int bx, by, ox, oy;
  bool iface;
  if (s == 0) { bx = x0; by = y0 + t; ox = bx - 1; oy = by; iface = x0 > 0; }
  else if (s == 1) { bx = x0 + FDFD_WIN - 1; by = y0 + t; ox = bx + 1; oy = by; iface = x0 + FDFD_WIN < nx; }
  else if (s == 2) { bx = x0 + t; by = y0; ox = bx; oy = by - 1; iface = y0 > 0; }
  else { bx = x0 + t; by = y0 + FDFD_WIN - 1; ox = bx; oy = by + 1; iface = y0 + FDFD_WIN < ny; }
  float2 r = make_float2(0.f, 0.f);
  if (iface) {
    const float2 ub = u[(size_t)by * nx + bx], uo = u[(size_t)oy * nx + ox];
    const float kd = k0dx * sqrtf(eps[(size_t)by * nx + bx]);
    r = make_float2(uo.x - ub.x - kd * ub.y, uo.y - ub.y + kd * ub.x);
  }
  g[idx] = r;
}

// rhs_w += R_w b: the restricted source joins the Robin data's right-hand side.
__global__ void add_restricted_kernel(float2* __restrict__ rhs, const float2* __restrict__ b, int nx, int ny,
                                      int nwx) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x, w = blockIdx.y;
  if (p >= FDFD_WIN * FDFD_WIN) return;
  const int a = w % nwx, bb = w / nwx;
  const int x0 = min(max(FDFD_CORE * a - FDFD_OVL, 0), nx - FDFD_WIN);
  const int y0 = min(max(FDFD_CORE * bb - FDFD_OVL, 0), ny - FDFD_WIN);
  const float2 v = b[(size_t)(y0 + p / FDFD_WIN) * nx + x0 + p % FDFD_WIN];
  float2& r = rhs[(size_t)w * FDFD_WIN * FDFD_WIN + p];
  r = make_float2(r.x + v.x, r.y + v.y);
}

// Momentum blend of the Robin data: g = m g + (1 - m) g_new.
__global__ void blend_kernel(float2* __restrict__ g, const float2* __restrict__ g_new, float m, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 a = g[i], c = g_new[i];
    g[i] = make_float2(m * a.x + (1.f - m) * c.x, m * a.y + (1.f - m) * c.y);
  }
}

}  // namespace

int schwarz_traces(fdfd_ctx* h, const float2* u, float2* g) {
  const int nwx = h->nx / FDFD_CORE, n_win = nwx * (h->ny / FDFD_CORE);
  const int tot = n_win * 4 * FDFD_WIN;
  traces_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(u, h->eps, (float)h->k0dx, h->nx, h->ny, nwx, n_win, g);
  CKL();
  return FDFD_OK;
}

const float* schwarz_modulation(fdfd_ctx* h) { return (h && h->sw) ? h->sw->mod : nullptr; }

static GridGeom geom(fdfd_ctx* h) {
  return GridGeom{h->nx, h->ny, h->nx / FDFD_CORE, (float)h->k2, h->eps, h->isx, h->isy, schwarz_modulation(h)};
}

// Seeded uniform complex field in [-1, 1)^2 (counter-based splitmix64), the
// residual-like input of the FP8 calibration forward.
__global__ void fill_uniform_kernel(float2* v, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float a = (float)(uint32_t)(z >> 32) * (1.f / 4294967296.f), b = (float)(uint32_t)z * (1.f / 4294967296.f);
    v[i] = make_float2(2.f * a - 1.f, 2.f * b - 1.f);
  }
}

static int check_err(fdfd_ctx* h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->sw->work.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return e ? FDFD_ETIMEOUT : FDFD_OK;
}

int schwarz_error(fdfd_ctx* h) { return (h && h->sw) ? check_err(h) : FDFD_OK; }

int schwarz_mark_failed(fdfd_ctx* h) {
  if (!h || !h->sw) return FDFD_ENOSETUP;
  const int one = 1;
  CK(cudaMemcpyAsync(h->sw->work.err, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int schwarz_create(fdfd_ctx* h, const schwarz_desc* sd) {
  if (sd->k_coarse < 0 || sd->k_coarse > 256) return FDFD_EINVAL;
  if (sd->precision != FDFD_PREC_BF16 && sd->precision != FDFD_PREC_FP8) return FDFD_EINVAL;
  if (sd->inner_iters < 0 || sd->inner_iters > LOCAL_MAXM) return FDFD_EINVAL;
  if (sd->r_rank < 0 || sd->r_rank > 512 || (sd->modulation != 0 && sd->modulation != 1)) return FDFD_EINVAL;
  // the FP8 calibration folds scales into the plain network's weights only
  if ((sd->r_rank || sd->modulation) && sd->precision == FDFD_PREC_FP8) return FDFD_EINVAL;
  SchwarzData* S = new SchwarzData();
  S->nwx = h->nx / FDFD_CORE;
  S->n_win = S->nwx * (h->ny / FDFD_CORE);
  S->precision = sd->precision;
  S->inner = sd->inner_iters;
  int rc = nno_upload_weights(&S->W, sd->weights, sd->n_weights, sd->r_rank, sd->modulation, &S->bytes);
  if (!rc && S->W.mod) {  // modulation of every window: it depends on eps and the PML maps only
    if (cudaMalloc((void**)&S->mod, (size_t)S->n_win * 2048 * sizeof(float)) != cudaSuccess) rc = FDFD_ENOMEM;
    else S->bytes += (size_t)S->n_win * 2048 * sizeof(float);
    if (!rc) rc = nno_modulation(&S->W, geom(h), S->n_win, S->mod, h->stream);
  }
  if (!rc) rc = nno_alloc_work(&S->work, S->n_win < 64 ? 64 : S->n_win, &S->bytes);
  if (!rc) rc = nno_autotune(&S->W, &S->work, S->n_win, h->stream);
  if (!rc && sd->precision == FDFD_PREC_FP8) {  // calibrate the activation scales on random inputs
    fill_uniform_kernel<<<1024, 256, 0, h->stream>>>(h->w, h->n, 0x5EEDull);
    // calibrate on both kinds of input the network meets: residual windows
    // (the sweeps and local solves) and Robin data with no source (the
    // coarse set-up's trials); the random field doubles as that Robin data
    // (n_win x 320 values, fewer than the grid's cells)
    NnoInput in[2];
    in[0].v_global = h->w;
    in[1].g_win = h->w;
    rc = nno_enable_fp8(&S->W, &S->work, geom(h), in, 2, S->n_win, sd->weights, sd->n_weights, &S->bytes,
                        h->stream);
  }
  if (!rc && S->inner > 0) rc = local_alloc(&S->local, S->n_win, S->inner, &S->bytes);
  h->sw = S;
  if (!rc && sd->k_coarse > 0) {
    S->k = sd->k_coarse;
    rc = coarse_setup(h, &S->W, &S->work, S->inner > 0 ? &S->local : nullptr, sd->k_coarse, sd->ritz_tol,
                      &S->coarse, &S->bytes);
    if (!rc) rc = check_err(h);
  }
  if (rc) { schwarz_destroy(h); return rc; }
  h->bytes += S->bytes;
  return FDFD_OK;
}

void schwarz_destroy(fdfd_ctx* h) {
  if (!h || !h->sw) return;
  SchwarzData* S = h->sw;
  cudaStreamSynchronize(h->stream);
  if (S->coarse) coarse_free(S->coarse);
  if (S->mod) cudaFree(S->mod);
  nno_free_weights(&S->W);
  nno_free_work(&S->work);
  local_free(&S->local);
  h->bytes -= (h->bytes >= S->bytes ? S->bytes : h->bytes);
  delete S;
  h->sw = nullptr;
}

int schwarz_apply(fdfd_ctx* h, const float2* v, const double* scale_dev, float2* z, int transpose) {
  SchwarzData* S = h->sw;
  NnoInput in;
  in.v_global = v;
  NnoOutput out;
  out.z_global = z;
  out.scale = scale_dev;
  int rc;
  if (S->inner > 0)
    rc = local_fgmres(h, &S->local, &S->W, &S->work, v, nullptr, z, nullptr, scale_dev, transpose);
  else
    rc = nno_forward(&S->W, &S->work, geom(h), in, out, S->n_win, h->stream, h);
  if (rc) return rc;
  if (S->coarse) {
    if ((rc = coarse_apply(h, S->coarse, z))) return rc;
  }
  return FDFD_OK;
}

int schwarz_nno_solve(fdfd_ctx* h, const float2* r_win, const float2* g_win, const int* win_id, int n,
                      float2* e_win) {
  SchwarzData* S = h->sw;
  if (n > S->work.cap) return FDFD_EINVAL;
  NnoInput in;
  in.r_win = r_win;
  in.g_win = g_win;
  in.win_id = win_id;
  NnoOutput out;
  out.e_win = e_win;
  int rc = nno_forward(&S->W, &S->work, geom(h), in, out, n, h->stream);
  if (rc) return rc;
  return check_err(h);
}

// Local solves of Algorithm 3 with data: every window's problem has the
// restricted source R_w b and the Robin data g_win [n_win][4][80] on its
// interface sides; the solutions are assembled into u by restricted
// prolongation (each cell from its owning window's core).
int schwarz_sweep_data(fdfd_ctx* h, const float2* b, const float2* g_win, float2* u, float2* rhs_scratch) {
  SchwarzData* S = h->sw;
  if (S->inner > 0) {  // k steps of NN-preconditioned FGMRES on R_w b - sum_sides c_bo g
    int rc = local_robin_rhs(h, g_win, rhs_scratch, S->n_win);
    if (rc) return rc;
    add_restricted_kernel<<<dim3((FDFD_WIN * FDFD_WIN + 255) / 256, S->n_win), 256, 0, h->stream>>>(
        rhs_scratch, b, h->nx, h->ny, S->nwx);
    CKL();
    return local_fgmres(h, &S->local, &S->W, &S->work, nullptr, rhs_scratch, u, nullptr, h->d_one, 0);
  }
  NnoInput in;  // one neural application to (source, Robin data)
  in.v_global = b;
  in.g_win = g_win;
  NnoOutput out;
  out.z_global = u;
  out.scale = h->d_one;
  return nno_forward(&S->W, &S->work, geom(h), in, out, S->n_win, h->stream, h);
}

// The rest of one iteration of Algorithm 3 after the local solves: new Robin
// data from the assembled field u (traces, Eq. 2); with a coarse space, u is
// first corrected for the boundary mismatch between those traces and the
// data g the local solves used (Eq. 8) and the traces are taken again; then
// g = m g + (1 - m) g_new.  g_new is scratch of the same size as g.
int schwarz_stationary_update(fdfd_ctx* h, float2* u, float2* g, float2* g_new, double momentum) {
  SchwarzData* S = h->sw;
  int rc = schwarz_traces(h, u, g_new);
  if (!rc && S->coarse) {
    if (!(rc = coarse_apply(h, S->coarse, u, g))) rc = schwarz_traces(h, u, g_new);
  }
  if (rc) return rc;
  const int tot = S->n_win * 4 * FDFD_WIN;
  blend_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(g, g_new, (float)momentum, tot);
  CKL();
  return FDFD_OK;
}

const NnoWeights* schwarz_weights(fdfd_ctx* h) { return (h && h->sw) ? &h->sw->W : nullptr; }

int schwarz_inner_iters(fdfd_ctx* h) { return (h && h->sw) ? h->sw->inner : 0; }

int schwarz_dfty_variant(fdfd_ctx* h) { return (h && h->sw) ? h->sw->work.g2_split : 0; }

// Coarse correction of a one-level sweep result z (no-op without a coarse space).
int schwarz_coarse(fdfd_ctx* h, float2* z) {
  if (!h->sw || !h->sw->coarse) return FDFD_OK;
  return coarse_apply(h, h->sw->coarse, z);
}

int schwarz_ritz_export(fdfd_ctx* h, double* eta, double* H) {
  if (!h->sw->coarse) return FDFD_ENOSETUP;
  return coarse_ritz_export(h, h->sw->coarse, eta, H);
}

int schwarz_export(fdfd_ctx* h, double* Q, double* G) {
  if (!h->sw->coarse) return FDFD_ENOSETUP;
  return coarse_export(h, h->sw->coarse, Q, G);
}

int schwarz_coarse_solve(fdfd_ctx* h, const float2* ebc, float2* z) {
  if (!h->sw->coarse) return FDFD_ENOSETUP;
  return coarse_solve_mismatch(h, h->sw->coarse, ebc, z);
}

int schwarz_info(fdfd_ctx* h, fdfd_info* info) {
  info->k_coarse = h->sw->k;
  info->n_coarse = h->sw->k * h->sw->n_win;
  info->n_coarse_kept = coarse_kept(h->sw->coarse);
  info->tuned_dfty_split = h->sw->work.g2_split;
  return FDFD_OK;
}
