// 5-point stencil of the dx^2-scaled operator of Eq. 1 with UPML (Methods):
//   (A~x)_ij = hi_x(i) x_{i+1,j} + lo_x(i) x_{i-1,j} + hi_y(j) x_{i,j+1}
//            + lo_y(j) x_{i,j-1} + (dg_x(i) + dg_y(j) + (k0 dx)^2 eps_ij) x_ij,
// zero outside the grid.  For A~ the coefficients are lo = 1/(s_n(i) s_h(i)),
// hi = 1/(s_n(i) s_h(i+1)), dg = -(lo + hi); for A~^T the host passes
// lo(i) = hi(i-1), hi(i) = lo(i+1) with the same dg.
//
// Complex64 kernel: one thread computes two adjacent cells (one float4) in
// each of SR consecutive rows; left/right neighbours come from the
// neighbouring lanes by shuffle, the rows above and below from the thread's
// own registers.  Algorithmic HBM traffic 20 B per cell (x 8 + eps 4 + y 8).
#include "common.cuh"
#include "reduce.cuh"

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ float2 ax_apply(const AxisCoef& c, float2 xm, float2 xp) {
  return cadd(cmul(c.lo, xm), cmul(c.hi, xp));
}

// Each warp owns 32 cell pairs (one float4 each) of a column chunk and
// marches down SR rows: the SR + 2 rows of x it needs (one above, one below)
// and the SR rows of eps are all loaded before any arithmetic, so every x
// row is read once per chunk (the two halo rows through L2) and each thread
// keeps its loads in flight; the left and right neighbours of the chunk's
// edge lanes are loaded up front too.  eps and y are touched once, so they
// bypass L1 with streaming loads and stores.
constexpr int SW = 4;  // warps (column chunks) per block
constexpr int SR = 4;  // rows per thread (measured at 4096^2: 4 beats 2, 8 and 16)
__global__ void __launch_bounds__(32 * SW)
stencil_c64(const float4* __restrict__ x, float4* __restrict__ y, const float2* __restrict__ eps,
            const AxisCoef* __restrict__ cx, const AxisCoef* __restrict__ cy, float k2, int nx,
            int ny) {
  const int lane = threadIdx.x & 31;
  const int np = nx >> 1;
  const int chunk = blockIdx.x * SW + (threadIdx.x >> 5);
  if (chunk * 32 >= np) return;                    // whole warps only (np is a multiple of 32)
  const int p = chunk * 32 + lane;                 // float4 (cell pair) column
  const int j0 = blockIdx.y * SR;                  // ny is a multiple of SR
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 r[SR + 2];
#pragma unroll
  for (int t = 0; t < SR + 2; ++t) {
    const int j = j0 - 1 + t;
    r[t] = (j >= 0 && j < ny) ? __ldg(x + (size_t)j * np + p) : zero4;
  }
  float2 e[SR];
#pragma unroll
  for (int t = 0; t < SR; ++t) e[t] = __ldcs(eps + (size_t)(j0 + t) * np + p);  // read once: streaming
  // the x neighbour across the chunk edge: lane 0 needs cell 2p - 1, lane 31 cell 2p + 2
  const bool edge_l = lane == 0 && p > 0, edge_r = lane == 31 && p + 1 < np;
  float2 h[SR];
#pragma unroll
  for (int t = 0; t < SR; ++t) {
    h[t] = make_float2(0.f, 0.f);
    const float2* xr = reinterpret_cast<const float2*>(x + (size_t)(j0 + t) * np);
    if (edge_l) h[t] = __ldg(xr + 2 * p - 1);
    if (edge_r) h[t] = __ldg(xr + 2 * p + 2);
  }
  const int i0 = 2 * p;
  const AxisCoef a0 = cx[i0], a1 = cx[i0 + 1];
#pragma unroll
  for (int t = 0; t < SR; ++t) {
    const int j = j0 + t;
    const float4 c = r[t + 1], up = r[t + 2], dn = r[t];
    float lx = __shfl_up_sync(0xffffffffu, c.z, 1), ly = __shfl_up_sync(0xffffffffu, c.w, 1);
    float rx = __shfl_down_sync(0xffffffffu, c.x, 1), ry = __shfl_down_sync(0xffffffffu, c.y, 1);
    if (lane == 0) { lx = h[t].x; ly = h[t].y; }
    if (lane == 31) { rx = h[t].x; ry = h[t].y; }
    const AxisCoef b = cy[j];
    const float2 x0 = make_float2(c.x, c.y), x1 = make_float2(c.z, c.w);
    float2 y0 = ax_apply(a0, make_float2(lx, ly), x1);
    float2 y1 = ax_apply(a1, x0, make_float2(rx, ry));
    y0 = cadd(y0, ax_apply(b, make_float2(dn.x, dn.y), make_float2(up.x, up.y)));
    y1 = cadd(y1, ax_apply(b, make_float2(dn.z, dn.w), make_float2(up.z, up.w)));
    const float2 d0 = make_float2(a0.dg.x + b.dg.x + k2 * e[t].x, a0.dg.y + b.dg.y);
    const float2 d1 = make_float2(a1.dg.x + b.dg.x + k2 * e[t].y, a1.dg.y + b.dg.y);
    y0 = cadd(y0, cmul(d0, x0));
    y1 = cadd(y1, cmul(d1, x1));
    __stcs(y + (size_t)j * np + p, make_float4(y0.x, y0.y, y1.x, y1.y));  // written once: streaming
  }
}

// w = A~ (D^-1 v * s): the Jacobi-preconditioned operator in one sweep
// (D = diagonal of A~, recomputed from eps and the PML coefficients).
__device__ __forceinline__ float2 cdiv(float2 a, float2 d) {
  const float inv = 1.f / (d.x * d.x + d.y * d.y);
  return make_float2((a.x * d.x + a.y * d.y) * inv, (a.y * d.x - a.x * d.y) * inv);
}

__device__ __forceinline__ float2 diag_at(const AxisCoef* cx, const AxisCoef* cy, const float* eps,
                                          float k2, int i, int j, int nx) {
  const float2 dx_ = cx[i].dg, dy_ = cy[j].dg;
  return make_float2(dx_.x + dy_.x + k2 * __ldg(eps + (size_t)j * nx + i), dx_.y + dy_.y);
}

__global__ void __launch_bounds__(BX * BY)
stencil_jacobi_c64(const float4* __restrict__ v, const double* __restrict__ vscale,
                   float4* __restrict__ w, const float* __restrict__ eps,
                   const AxisCoef* __restrict__ cx, const AxisCoef* __restrict__ cy, float k2,
                   int nx, int ny) {
  const int lane = threadIdx.x;
  const int p = blockIdx.x * BX + lane;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int np = nx >> 1;
  const size_t row = (size_t)j * np;
  const float s = (float)(*vscale);
  const int i0 = 2 * p;
  auto u_of = [&](float4 q, int ii, int jj) -> float4 {  // D^-1 v s at (ii, jj), (ii+1, jj)
    float2 a = cdiv(make_float2(q.x * s, q.y * s), diag_at(cx, cy, eps, k2, ii, jj, nx));
    float2 b = cdiv(make_float2(q.z * s, q.w * s), diag_at(cx, cy, eps, k2, ii + 1, jj, nx));
    return make_float4(a.x, a.y, b.x, b.y);
  };
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 c = u_of(__ldg(v + row + p), i0, j);
  const float4 up = (j + 1 < ny) ? u_of(__ldg(v + row + np + p), i0, j + 1) : zero4;
  const float4 dn = (j > 0) ? u_of(__ldg(v + row - np + p), i0, j - 1) : zero4;
  float lx = __shfl_up_sync(0xffffffffu, c.z, 1), ly = __shfl_up_sync(0xffffffffu, c.w, 1);
  float rx = __shfl_down_sync(0xffffffffu, c.x, 1), ry = __shfl_down_sync(0xffffffffu, c.y, 1);
  if (lane == 0) {
    if (p > 0) { float4 t = u_of(__ldg(v + row + p - 1), i0 - 2, j); lx = t.z; ly = t.w; } else { lx = 0.f; ly = 0.f; }
  }
  if (lane == BX - 1) {
    if (p + 1 < np) { float4 t = u_of(__ldg(v + row + p + 1), i0 + 2, j); rx = t.x; ry = t.y; } else { rx = 0.f; ry = 0.f; }
  }
  const AxisCoef a0 = cx[i0], a1 = cx[i0 + 1], b = cy[j];
  const float2 x0 = make_float2(c.x, c.y), x1 = make_float2(c.z, c.w);
  float2 y0 = ax_apply(a0, make_float2(lx, ly), x1);
  float2 y1 = ax_apply(a1, x0, make_float2(rx, ry));
  y0 = cadd(y0, ax_apply(b, make_float2(dn.x, dn.y), make_float2(up.x, up.y)));
  y1 = cadd(y1, ax_apply(b, make_float2(dn.z, dn.w), make_float2(up.z, up.w)));
  const float2 e = __ldg(reinterpret_cast<const float2*>(eps) + row + p);
  const float2 d0 = make_float2(a0.dg.x + b.dg.x + k2 * e.x, a0.dg.y + b.dg.y);
  const float2 d1 = make_float2(a1.dg.x + b.dg.x + k2 * e.y, a1.dg.y + b.dg.y);
  y0 = cadd(y0, cmul(d0, x0));
  y1 = cadd(y1, cmul(d1, x1));
  w[row + p] = make_float4(y0.x, y0.y, y1.x, y1.y);
}

// z = D^-1 v s (stored, for the flexible basis when Jacobi is used as M).
__global__ void jacobi_apply(const float2* __restrict__ v, const double* __restrict__ vscale,
                             float2* __restrict__ z, const float* __restrict__ eps,
                             const AxisCoef* __restrict__ cx, const AxisCoef* __restrict__ cy,
                             float k2, int nx, size_t n) {
  const float s = (float)(*vscale);
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)(c / nx);
    const float2 q = v[c];
    z[c] = cdiv(make_float2(q.x * s, q.y * s), diag_at(cx, cy, eps, k2, i, j, nx));
  }
}

// FP64 residual r = rs b - A~ x with FP64 coefficients, x in FP64; b = j sb J
// (source form) or b = J (adjoint right-hand side); rs rescales the system
// (a power of two, so exactly); x == nullptr means x = 0.  Writes r rounded
// to complex64 and reduces ||r||^2 (FP64) into *result.  FP64 arithmetic is
// scarce on this GPU, so cells whose coefficients are all real (everywhere
// outside the PML) take a real-coefficient path with the same roundings.
constexpr int RT = 256;
__global__ void __launch_bounds__(RT)
residual64(const double2* __restrict__ x, const float2* __restrict__ J, double sb, int src, double rs,
           const float* __restrict__ eps, const AxisCoef64* __restrict__ cx,
           const AxisCoef64* __restrict__ cy, double k2, int nx, int ny,
           float2* __restrict__ r_out, double* __restrict__ partials, unsigned* counter,
           double* result) {
  __shared__ double sh[RT / 32];
  double acc = 0.0;
  const size_t n = (size_t)nx * ny;
  for (size_t c = blockIdx.x * (size_t)RT + threadIdx.x; c < n; c += (size_t)gridDim.x * RT) {
    double2 Ax = make_double2(0.0, 0.0);
    if (x) {
      const int i = (int)(c % nx), j = (int)(c / nx);
      const AxisCoef64 a = cx[i], b = cy[j];
      const double2 xc = x[c];
      const double2 z = make_double2(0.0, 0.0);
      const double2 xl = i > 0 ? x[c - 1] : z, xr = i + 1 < nx ? x[c + 1] : z;
      const double2 xd = j > 0 ? x[c - nx] : z, xu = j + 1 < ny ? x[c + nx] : z;
      const double dre = a.dg.x + b.dg.x + k2 * (double)eps[c];
      if (a.lo.y == 0.0 && a.hi.y == 0.0 && b.lo.y == 0.0 && b.hi.y == 0.0 && a.dg.y + b.dg.y == 0.0) {
        Ax.x = dre * xc.x + a.lo.x * xl.x + a.hi.x * xr.x + b.lo.x * xd.x + b.hi.x * xu.x;
        Ax.y = dre * xc.y + a.lo.x * xl.y + a.hi.x * xr.y + b.lo.x * xd.y + b.hi.x * xu.y;
      } else {
        Ax = zmul(make_double2(dre, a.dg.y + b.dg.y), xc);
        Ax = zadd(Ax, zmul(a.lo, xl));
        Ax = zadd(Ax, zmul(a.hi, xr));
        Ax = zadd(Ax, zmul(b.lo, xd));
        Ax = zadd(Ax, zmul(b.hi, xu));
      }
    }
    const float2 Jc = J[c];
    const double2 bc = src ? make_double2(-sb * rs * (double)Jc.y, sb * rs * (double)Jc.x)
                           : make_double2(rs * (double)Jc.x, rs * (double)Jc.y);
    const double2 r = zsub(bc, Ax);
    r_out[c] = make_float2((float)r.x, (float)r.y);
    acc += r.x * r.x + r.y * r.y;
  }
  const double t = block_sum<RT>(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (last_block(counter)) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += RT) s += partials[b];
    s = block_sum<RT>(s, sh);
    if (threadIdx.x == 0) { *result = s; *counter = 0u; }
  }
}

__global__ void grad_eps_kernel(const float2* __restrict__ E, const float2* __restrict__ lam,
                                float* __restrict__ grad, float k2, size_t n, int acc) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const float2 e = E[c], l = lam[c];
    const float g = -2.f * k2 * (l.x * e.x - l.y * e.y);
    grad[c] = acc ? grad[c] + g : g;
  }
}

__global__ void scale_d_kernel(const float2* in, float2* out, const float2* __restrict__ isx,
                               const float2* __restrict__ isy, int nx, size_t n, int inverse) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    const float2 dinv = cmul(isx[c % nx], isy[c / nx]);  // 1 / (s_x s_y)
    float2 f = dinv;
    if (!inverse) {
      const float m = dinv.x * dinv.x + dinv.y * dinv.y;
      f = make_float2(dinv.x / m, -dinv.y / m);
    }
    out[c] = cmul(in[c], f);
  }
}

}  // namespace

int launch_scale_d(const float2* in, float2* out, const float2* isx, const float2* isy, int nx, size_t n,
                   int inverse, cudaStream_t s) {
  scale_d_kernel<<<krylov_grid(n), 256, 0, s>>>(in, out, isx, isy, nx, n, inverse);
  CKL();
  return FDFD_OK;
}

int launch_stencil(const float2* x, float2* y, const float* eps, const AxisCoef* cx,
                   const AxisCoef* cy, float k2, int nx, int ny, cudaStream_t s) {
  dim3 grid((nx / 64 + SW - 1) / SW, ny / SR), block(32 * SW);
  stencil_c64<<<grid, block, 0, s>>>(reinterpret_cast<const float4*>(x), reinterpret_cast<float4*>(y),
                                     reinterpret_cast<const float2*>(eps), cx, cy, k2, nx, ny);
  CKL();
  return FDFD_OK;
}

int launch_stencil_jacobi(const float2* v, const double* vscale, float2* w, const float* eps,
                          const AxisCoef* cx, const AxisCoef* cy, float k2, int nx, int ny,
                          cudaStream_t s) {
  dim3 grid(nx / (2 * BX), ny / BY), block(BX, BY);
  stencil_jacobi_c64<<<grid, block, 0, s>>>(reinterpret_cast<const float4*>(v), vscale,
                                            reinterpret_cast<float4*>(w), eps, cx, cy, k2, nx, ny);
  CKL();
  return FDFD_OK;
}

int launch_jacobi_apply(const float2* v, const double* vscale, float2* z, const float* eps,
                        const AxisCoef* cx, const AxisCoef* cy, float k2, int nx, int ny,
                        cudaStream_t s) {
  jacobi_apply<<<krylov_grid((size_t)nx * ny), 256, 0, s>>>(v, vscale, z, eps, cx, cy, k2, nx,
                                                             (size_t)nx * ny);
  CKL();
  return FDFD_OK;
}

int launch_residual64(const double2* x, const float2* J, double sb, int rhs_is_source, double rs,
                      const float* eps, const AxisCoef64* cx, const AxisCoef64* cy, double k2,
                      int nx, int ny, float2* r_out, double* partials, unsigned* counter,
                      double* result, cudaStream_t s) {
  residual64<<<krylov_grid((size_t)nx * ny), RT, 0, s>>>(x, J, sb, rhs_is_source, rs, eps, cx, cy, k2,
                                                          nx, ny, r_out, partials, counter, result);
  CKL();
  return FDFD_OK;
}

int launch_grad_eps(const float2* E, const float2* lam, float* grad, float k2, int n,
                    int accumulate, cudaStream_t s) {
  grad_eps_kernel<<<krylov_grid((size_t)n), 256, 0, s>>>(E, lam, grad, k2, (size_t)n, accumulate);
  CKL();
  return FDFD_OK;
}
