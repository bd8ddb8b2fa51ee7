// Inverse-design parameterisation and optimiser (Sec. 2.2, inverse design:
// density-based optimisation, differentiable filtering and projection, Adam
// ascent with adjoint gradients).  The design variable rho in [0, 1] lives
// on a rectangle of the grid; rho_f = W rho is a cone filter of radius R
// (weights max(0, R - |d|) over the offsets that stay in the rectangle,
// each output divided by its own weight sum); the projection
// P(x) = (tanh(beta eta) + tanh(beta (x - eta))) / (tanh(beta eta) +
// tanh(beta (1 - eta))) maps it to eps = eps_lo + P(rho_f) (eps_hi - eps_lo);
// the chain rule runs back as g_rho = W^T (P'(rho_f) (eps_hi - eps_lo) g_eps);
// Adam (Kingma and Ba) with bias correction ascends the figure of merit.
// The rectangle is a few hundred cells square: these are small
// bandwidth-bound kernels next to the solves that produce g_eps.
#include <math.h>
#include "ctx.cuh"

namespace {
constexpr int DT = 256;
constexpr int DMAXR = 16;  // largest filter radius in cells

struct DesignK {
  int x0, y0, w, h, nx, r;
  float R, beta, eta, lo, hi, a, den;  // a = tanh(beta eta), den = a + tanh(beta (1 - eta))
};

__device__ __forceinline__ float cone_w(const DesignK& k, int dy, int dx) {
  return k.R - sqrtf((float)(dy * dy + dx * dx));
}

// rho_f and the permittivity of the rectangle
__global__ void __launch_bounds__(DT) design_fwd_kernel(const float* __restrict__ rho, float* __restrict__ rho_f,
                                                        float* __restrict__ eps, DesignK k) {
  const int c = blockIdx.x * DT + threadIdx.x;
  if (c >= k.w * k.h) return;
  const int i = c / k.w, j = c % k.w;
  float num = 0.f, S = 0.f;
  for (int dy = -k.r; dy <= k.r; ++dy) {
    if (i + dy < 0 || i + dy >= k.h) continue;
    for (int dx = -k.r; dx <= k.r; ++dx) {
      const float wgt = cone_w(k, dy, dx);
      if (wgt <= 0.f || j + dx < 0 || j + dx >= k.w) continue;
      num += wgt * rho[(i + dy) * k.w + j + dx];
      S += wgt;
    }
  }
  const float rf = num / S;
  rho_f[c] = rf;
  const float p = (k.a + tanhf(k.beta * (rf - k.eta))) / k.den;
  eps[(size_t)(k.y0 + i) * k.nx + k.x0 + j] = k.lo + p * (k.hi - k.lo);
}

// t = P'(rho_f) (eps_hi - eps_lo) g_eps / S  (S: the output's weight sum)
__global__ void __launch_bounds__(DT) design_bwd1_kernel(const float* __restrict__ g_eps,
                                                         const float* __restrict__ rho_f, float* __restrict__ t,
                                                         DesignK k) {
  const int c = blockIdx.x * DT + threadIdx.x;
  if (c >= k.w * k.h) return;
  const int i = c / k.w, j = c % k.w;
  float S = 0.f;
  for (int dy = -k.r; dy <= k.r; ++dy) {
    if (i + dy < 0 || i + dy >= k.h) continue;
    for (int dx = -k.r; dx <= k.r; ++dx) {
      const float wgt = cone_w(k, dy, dx);
      if (wgt > 0.f && j + dx >= 0 && j + dx < k.w) S += wgt;
    }
  }
  const float th = tanhf(k.beta * (rho_f[c] - k.eta));
  const float dp = k.beta * (1.f - th * th) / k.den;
  t[c] = dp * (k.hi - k.lo) * g_eps[(size_t)(k.y0 + i) * k.nx + k.x0 + j] / S;
}

// g_rho[j] = sum over outputs i = j - d of w_d t_i
__global__ void __launch_bounds__(DT) design_bwd2_kernel(const float* __restrict__ t, float* __restrict__ g_rho,
                                                         DesignK k) {
  const int c = blockIdx.x * DT + threadIdx.x;
  if (c >= k.w * k.h) return;
  const int i = c / k.w, j = c % k.w;
  float acc = 0.f;
  for (int dy = -k.r; dy <= k.r; ++dy) {
    if (i - dy < 0 || i - dy >= k.h) continue;
    for (int dx = -k.r; dx <= k.r; ++dx) {
      const float wgt = cone_w(k, dy, dx);
      if (wgt <= 0.f || j - dx < 0 || j - dx >= k.w) continue;
      acc += wgt * t[(i - dy) * k.w + j - dx];
    }
  }
  g_rho[c] = acc;
}

// Adam ascent with bias correction (c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t));
// the gradient is multiplied by g_scale first; theta stays in [0, 1].
__global__ void __launch_bounds__(DT) adam_kernel(float* __restrict__ theta, const float* __restrict__ g,
                                                  float* __restrict__ m, float* __restrict__ v, int n, float lr,
                                                  float b1, float b2, float eps, float c1, float c2, float g_scale) {
  const int c = blockIdx.x * DT + threadIdx.x;
  if (c >= n) return;
  const float gg = g[c] * g_scale;
  const float mm = b1 * m[c] + (1.f - b1) * gg, vv = b2 * v[c] + (1.f - b2) * gg * gg;
  m[c] = mm;
  v[c] = vv;
  theta[c] = fminf(fmaxf(theta[c] + lr * (mm * c1) / (sqrtf(vv * c2) + eps), 0.f), 1.f);
}

int make_k(fdfd_ctx* h, const fdfd_design* d, DesignK* k) {
  if (!h || !d || d->w < 1 || d->h < 1 || d->x0 < 0 || d->y0 < 0 || d->x0 + d->w > h->nx ||
      d->y0 + d->h > h->ny || !(d->radius > 0.f && d->radius <= (float)DMAXR) || !(d->beta > 0.f) ||
      !(d->eta > 0.f && d->eta < 1.f))
    return FDFD_EINVAL;
  k->x0 = d->x0; k->y0 = d->y0; k->w = d->w; k->h = d->h; k->nx = h->nx;
  k->R = d->radius; k->r = (int)ceilf(d->radius);
  k->beta = d->beta; k->eta = d->eta; k->lo = d->eps_lo; k->hi = d->eps_hi;
  const double a = tanh((double)d->beta * d->eta), b = tanh((double)d->beta * (1.0 - d->eta));
  k->a = (float)a;
  k->den = (float)(a + b);
  return FDFD_OK;
}

}  // namespace

int fdfd_design_eps(fdfd_handle h, const fdfd_design* d, const float* rho, float* rho_f, float* eps) {
  DesignK k;
  int rc = make_k(h, d, &k);
  if (rc) return rc;
  if (!rho || !rho_f || !eps) return FDFD_EINVAL;
  const int n = k.w * k.h;
  design_fwd_kernel<<<(n + DT - 1) / DT, DT, 0, h->stream>>>(rho, rho_f, eps, k);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_design_grad(fdfd_handle h, const fdfd_design* d, const float* rho_f, const float* g_eps, float* work,
                     float* g_rho) {
  DesignK k;
  int rc = make_k(h, d, &k);
  if (rc) return rc;
  if (!rho_f || !g_eps || !work || !g_rho) return FDFD_EINVAL;
  const int n = k.w * k.h;
  design_bwd1_kernel<<<(n + DT - 1) / DT, DT, 0, h->stream>>>(g_eps, rho_f, work, k);
  design_bwd2_kernel<<<(n + DT - 1) / DT, DT, 0, h->stream>>>(work, g_rho, k);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

int fdfd_adam_step(fdfd_handle h, const fdfd_adam* a, int t, float g_scale, float* theta, const float* g, float* m,
                   float* v, int n) {
  if (!h || !a || t < 1 || n < 0 || !(a->lr > 0.f) || !(a->beta1 >= 0.f && a->beta1 < 1.f) ||
      !(a->beta2 >= 0.f && a->beta2 < 1.f) || !(a->eps > 0.f))
    return FDFD_EINVAL;
  if (n == 0) return FDFD_OK;
  if (!theta || !g || !m || !v) return FDFD_EINVAL;
  const float c1 = (float)(1.0 / (1.0 - pow((double)a->beta1, t)));
  const float c2 = (float)(1.0 / (1.0 - pow((double)a->beta2, t)));
  adam_kernel<<<(n + DT - 1) / DT, DT, 0, h->stream>>>(theta, g, m, v, n, a->lr, a->beta1, a->beta2, a->eps, c1, c2,
                                                       g_scale);
  CKL();
  CK(cudaStreamSynchronize(h->stream));
  return FDFD_OK;
}

// ---- figure of merit: port mode overlaps (Sec. 2.2, inverse design) ----
// c = dx sum_i conj(m_i) E[y0 + i][port_x] is linear (holomorphic) in E with
// dc/dE = conj(m_i) dx on the port line.  PyTorch passes gradients of a real
// loss L as G_z = 2 dL/d conj(z); the chain rule through c is then
// G_E = G_c conj(dc/dE) = G_c m_i dx, and the adjoint right-hand side of the
// adjoint variable method is dL/dE = conj(G_E) / 2.
namespace {
constexpr int OT = 256;

__global__ void __launch_bounds__(OT) overlap_kernel(const float2* __restrict__ E, const float2* __restrict__ m,
                                                     int nm, int nx, int port_x, int y0, double dx,
                                                     double* __restrict__ c) {
  __shared__ double sr[OT / 32], si[OT / 32];
  double ar = 0.0, ai = 0.0;
  for (int i = threadIdx.x; i < nm; i += OT) {
    const float2 e = E[(size_t)(y0 + i) * nx + port_x], w = m[i];
    // conj(w) e = (w.x e.x + w.y e.y) + j (w.x e.y - w.y e.x)
    ar += (double)w.x * e.x + (double)w.y * e.y;
    ai += (double)w.x * e.y - (double)w.y * e.x;
  }
  for (int o = 16; o; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sr[warp] = ar; si[warp] = ai; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < OT / 32; ++w) { tr += sr[w]; ti += si[w]; }
    c[0] = tr * dx;
    c[1] = ti * dx;
  }
}

__global__ void __launch_bounds__(OT) overlap_grad_kernel(const float2* __restrict__ m, int nm, int nx, int port_x,
                                                          int y0, double gr, double gi, float2* __restrict__ G,
                                                          int accumulate) {
  const int i = blockIdx.x * OT + threadIdx.x;
  if (i >= nm) return;
  const float2 w = m[i];
  float2* p = G + (size_t)(y0 + i) * nx + port_x;
  // (gr + j gi) dx (w.x + j w.y); gr, gi already carry dx
  float2 v = make_float2((float)(gr * w.x - gi * w.y), (float)(gr * w.y + gi * w.x));
  if (accumulate) {
    const float2 o = *p;
    v.x += o.x;
    v.y += o.y;
  }
  *p = v;
}

// g = conj(G) / 2 (8-byte loads: any complex64 field is 8-byte aligned)
__global__ void __launch_bounds__(OT) adjoint_rhs_kernel(const float2* __restrict__ G, float2* __restrict__ g,
                                                         size_t n) {
  const size_t stride = (size_t)gridDim.x * OT;
  for (size_t i = (size_t)blockIdx.x * OT + threadIdx.x; i < n; i += stride) {
    const float2 v = G[i];
    g[i] = make_float2(0.5f * v.x, -0.5f * v.y);
  }
}

bool port_ok(int nx, int ny, int nm, int port_x, int y0) {
  return nx >= 1 && ny >= 1 && nm >= 1 && port_x >= 0 && port_x < nx && y0 >= 0 && (long long)y0 + nm <= ny;
}
}  // namespace

int fdfd_mode_overlap(const fdfd_c64* E, int nx, int ny, const fdfd_c64* mode, int nm, int port_x, int y0,
                      double dx, double* c_dev, void* stream) {
  if (!E || !mode || !c_dev || !port_ok(nx, ny, nm, port_x, y0) || !(dx > 0.0)) return FDFD_EINVAL;
  overlap_kernel<<<1, OT, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float2*>(E),
                                                     reinterpret_cast<const float2*>(mode), nm, nx, port_x, y0, dx,
                                                     c_dev);
  CKL();
  return FDFD_OK;
}

int fdfd_mode_overlap_grad(int nx, int ny, const fdfd_c64* mode, int nm, int port_x, int y0, double dx,
                           double gc_re, double gc_im, fdfd_c64* grad_E, int accumulate, void* stream) {
  if (!mode || !grad_E || !port_ok(nx, ny, nm, port_x, y0) || !(dx > 0.0)) return FDFD_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!accumulate) CK(cudaMemsetAsync(grad_E, 0, (size_t)nx * ny * sizeof(fdfd_c64), s));
  overlap_grad_kernel<<<(nm + OT - 1) / OT, OT, 0, s>>>(reinterpret_cast<const float2*>(mode), nm, nx, port_x, y0,
                                                        gc_re * dx, gc_im * dx, reinterpret_cast<float2*>(grad_E),
                                                        accumulate);
  CKL();
  return FDFD_OK;
}

int fdfd_adjoint_rhs(fdfd_handle h, const fdfd_c64* grad_E, fdfd_c64* g) {
  if (!h || !grad_E || !g) return FDFD_EINVAL;
  const size_t n = (size_t)h->nx * h->ny;
  size_t blocks = (n + OT - 1) / OT;
  if (blocks > 8192) blocks = 8192;
  adjoint_rhs_kernel<<<(unsigned)blocks, OT, 0, h->stream>>>(reinterpret_cast<const float2*>(grad_E),
                                                             reinterpret_cast<float2*>(g), n);
  CKL();
  return FDFD_OK;
}
