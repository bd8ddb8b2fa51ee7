// Two-level Schwarz preconditioner (Algorithm 3 as one sweep from a zero
// guess): partition kernels, neural local solves and the coarse space.
#include "ctx.cuh"

struct SchwarzData {
  int k = 0;
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

}  // namespace

int schwarz_traces(fdfd_ctx* h, const float2* u, float2* g) {
  const int nwx = h->nx / FDFD_CORE, n_win = nwx * (h->ny / FDFD_CORE);
  const int tot = n_win * 4 * FDFD_WIN;
  traces_kernel<<<(tot + 255) / 256, 256, 0, h->stream>>>(u, h->eps, (float)h->k0dx, h->nx, h->ny, nwx, n_win, g);
  CKL();
  return FDFD_OK;
}

int schwarz_create(fdfd_ctx*, const schwarz_desc*) { return FDFD_ENOSETUP; }
void schwarz_destroy(fdfd_ctx* h) {
  if (h && h->sw) { delete h->sw; h->sw = nullptr; }
}
int schwarz_apply(fdfd_ctx*, const float2*, const double*, float2*, int) { return FDFD_ENOSETUP; }
int schwarz_nno_solve(fdfd_ctx*, const float2*, const float2*, const int*, int, float2*) { return FDFD_ENOSETUP; }
int schwarz_export(fdfd_ctx*, double*, double*) { return FDFD_ENOSETUP; }
int schwarz_info(fdfd_ctx*, fdfd_info*) { return FDFD_OK; }
