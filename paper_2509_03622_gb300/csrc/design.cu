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
