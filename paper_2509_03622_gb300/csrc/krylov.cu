// Flexible GMRES building blocks (Algorithm 1 with restarts):
//   cgs_dots    h_i = (w, v_i) = v_i^H w, i = 0..j  (one pass over V and w)
//   cgs_update  w' = w - sum_i h_i v_i, ||w'||^2, stored as v_{j+1};
//               the last block then does the Hessenberg/Givens update of
//               column j in FP64 and the least-squares residual estimate.
//   solve_y     back substitution of the rotated Hessenberg system
//   x_update    x += sum_j y_j z_j (x in FP64; the sum in FP32)
// Vectors are complex64, stored v_i = (1/vscale_i) * true v_i (the norm of
// v_{j+1} is only known after its pass, so scaling is deferred to readers).
// Products run in FP32, per-thread partial sums in FP32 over a few dozen
// terms, block and grid sums in FP64, summed in a fixed order (no float
// atomics): results are bitwise reproducible for a given launch shape.
#include "common.cuh"
#include "reduce.cuh"

namespace {
constexpr int KT = 256;

template <int NV>
__global__ void __launch_bounds__(KT)
cgs_dots_kernel(const float4* __restrict__ V, size_t ld4, int v0, int nv, const float4* __restrict__ w,
                size_t n4, KrylovState* st, double2* __restrict__ partials, unsigned* counter) {
  __shared__ double sh[KT / 32];
  float ar[NV], ai[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) { ar[i] = 0.f; ai[i] = 0.f; }
  // two float4 of w per thread and iteration; the loads of each group of
  // four vectors are issued together (8 x 16 B in flight per thread)
  const size_t stride = (size_t)gridDim.x * KT;
  for (size_t c0 = blockIdx.x * (size_t)KT + threadIdx.x; c0 < n4; c0 += 2 * stride) {
    const size_t c1 = c0 + stride;
    const bool has1 = c1 < n4;
    const float4 q0 = __ldg(w + c0);
    const float4 q1 = has1 ? __ldg(w + c1) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int g = 0; g < NV; g += 4) {
      float4 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool on = g + i < nv;
        const float4* vi = V + (size_t)(v0 + g + i) * ld4;
        a[i] = on ? __ldg(vi + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
        b[i] = (on && has1) ? __ldg(vi + c1) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        // conj(v) * w for both complex entries of each float4
        ar[g + i] += a[i].x * q0.x + a[i].y * q0.y + a[i].z * q0.z + a[i].w * q0.w
                   + b[i].x * q1.x + b[i].y * q1.y + b[i].z * q1.z + b[i].w * q1.w;
        ai[g + i] += a[i].x * q0.y - a[i].y * q0.x + a[i].z * q0.w - a[i].w * q0.z
                   + b[i].x * q1.y - b[i].y * q1.x + b[i].z * q1.w - b[i].w * q1.z;
      }
    }
  }
  // warp sums (FP64) of all nv accumulators, then one pass over the 8 warps
  __shared__ double2 wsum[KT / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < nv) {
      double tr = (double)ar[i], ti = (double)ai[i];
      for (int o = 16; o > 0; o >>= 1) {
        tr += __shfl_xor_sync(0xffffffffu, tr, o);
        ti += __shfl_xor_sync(0xffffffffu, ti, o);
      }
      if (lane == 0) wsum[wid][i] = make_double2(tr, ti);
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double tr = 0.0, ti = 0.0;
    for (int q = 0; q < KT / 32; ++q) { tr += wsum[q][threadIdx.x].x; ti += wsum[q][threadIdx.x].y; }
    partials[(size_t)blockIdx.x * FDFD_MAXRESTART + threadIdx.x] = make_double2(tr, ti);
  }
  if (last_block(counter)) {
    const int nb = gridDim.x;
    for (int i = 0; i < nv; ++i) {
      double sr = 0.0, si = 0.0;
      for (int b = threadIdx.x; b < nb; b += KT) {
        const double2 p = partials[(size_t)b * FDFD_MAXRESTART + i];
        sr += p.x; si += p.y;
      }
      sr = block_sum<KT>(sr, sh);
      si = block_sum<KT>(si, sh);
      if (threadIdx.x == 0) {
        const double s = st->vscale[v0 + i];
        st->h[v0 + i] = make_double2(sr * s, si * s);
      }
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// Serial FP64 Givens update of Hessenberg column j (thread 0 only).
__device__ void givens_column(KrylovState* st, int j, int ld, double hnext) {
  double2* Hc = st->H + (size_t)j * ld;
  for (int i = 0; i <= j; ++i) Hc[i] = st->h[i];
  Hc[j + 1] = make_double2(hnext, 0.0);
  for (int i = 0; i < j; ++i) {  // earlier rotations
    const double c = st->cs[i];
    const double2 s = st->sn[i];
    const double2 a = Hc[i], b = Hc[i + 1];
    Hc[i] = zadd(make_double2(c * a.x, c * a.y), zmul(s, b));
    Hc[i + 1] = zsub(make_double2(c * b.x, c * b.y), zmul(zconj(s), a));
  }
  const double2 a = Hc[j], b = Hc[j + 1];
  const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
  double c; double2 s;
  if (bb == 0.0) { c = 1.0; s = make_double2(0.0, 0.0); }
  else if (aa == 0.0) { c = 0.0; s = make_double2(b.x / bb, -b.y / bb); }
  else {
    const double t = hypot(aa, bb);
    c = aa / t;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    s = zmul(ph, make_double2(b.x / t, -b.y / t));
  }
  st->cs[j] = c; st->sn[j] = s;
  Hc[j] = zadd(make_double2(c * a.x, c * a.y), zmul(s, b));
  Hc[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = st->g[j];
  st->g[j + 1] = zmul(make_double2(-s.x, s.y), gj);   // -conj(s) g_j
  st->g[j] = make_double2(c * gj.x, c * gj.y);
  const double2 gn = st->g[j + 1];
  st->est = hypot(gn.x, gn.y) / st->bnorm;
  if (!isfinite(hnext) || !isfinite(st->est)) st->nonfinite = 1;
  st->breakdown = (hnext == 0.0);
  st->vscale[j + 1] = (hnext > 0.0) ? 1.0 / hnext : 0.0;
}

template <int NV>
__global__ void __launch_bounds__(KT)
cgs_update_kernel(const float4* __restrict__ V, size_t ld4, int v0, int nv, float4* __restrict__ w,
                  float4* __restrict__ vnext, size_t n4, KrylovState* st, double* __restrict__ partials,
                  unsigned* counter, int j_col, int ld, int final_chunk) {
  __shared__ double sh[KT / 32];
  __shared__ float2 coef[NV];
  if (threadIdx.x < nv) {
    const double2 h = st->h[v0 + threadIdx.x];
    const double s = st->vscale[v0 + threadIdx.x];
    coef[threadIdx.x] = make_float2((float)(h.x * s), (float)(h.y * s));
  }
  __syncthreads();
  float acc = 0.f;
  // two float4 per thread and iteration; each group of four vectors' loads
  // is issued together (8 x 16 B in flight per thread)
  const size_t stride = (size_t)gridDim.x * KT;
  for (size_t c0 = blockIdx.x * (size_t)KT + threadIdx.x; c0 < n4; c0 += 2 * stride) {
    const size_t c1 = c0 + stride;
    const bool has1 = c1 < n4;
    float4 q[2] = {w[c0], has1 ? w[c1] : make_float4(0.f, 0.f, 0.f, 0.f)};
#pragma unroll(NV <= 16 ? NV / 4 : 4)
    for (int g = 0; g < NV; g += 4) {
      float4 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool on = g + i < nv;
        const float4* vi = V + (size_t)(v0 + g + i) * ld4;
        a[i] = on ? __ldg(vi + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
        b[i] = (on && has1) ? __ldg(vi + c1) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 h = coef[g + i < NV ? g + i : 0];
        const float hx = g + i < nv ? h.x : 0.f, hy = g + i < nv ? h.y : 0.f;
        q[0].x -= hx * a[i].x - hy * a[i].y; q[0].y -= hx * a[i].y + hy * a[i].x;
        q[0].z -= hx * a[i].z - hy * a[i].w; q[0].w -= hx * a[i].w + hy * a[i].z;
        q[1].x -= hx * b[i].x - hy * b[i].y; q[1].y -= hx * b[i].y + hy * b[i].x;
        q[1].z -= hx * b[i].z - hy * b[i].w; q[1].w -= hx * b[i].w + hy * b[i].z;
      }
    }
    if (final_chunk) {
      vnext[c0] = q[0];
      acc += q[0].x * q[0].x + q[0].y * q[0].y + q[0].z * q[0].z + q[0].w * q[0].w;
      if (has1) {
        vnext[c1] = q[1];
        acc += q[1].x * q[1].x + q[1].y * q[1].y + q[1].z * q[1].z + q[1].w * q[1].w;
      }
    } else {
      w[c0] = q[0];
      if (has1) w[c1] = q[1];
    }
  }
  if (!final_chunk) return;
  const double t = block_sum<KT>((double)acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (last_block(counter)) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += KT) s += partials[b];
    s = block_sum<KT>(s, sh);
    if (threadIdx.x == 0) {
      *counter = 0u;
      givens_column(st, j_col, ld, sqrt(s));
    }
  }
}

__global__ void cycle_start_kernel(KrylovState* st) {
  const double beta = sqrt(st->resid);
  st->beta = beta;
  st->g[0] = make_double2(beta, 0.0);
  st->vscale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
  st->est = beta / st->bnorm;
  if (!isfinite(beta)) st->nonfinite = 1;
}

__global__ void solve_y_kernel(KrylovState* st, int k, int ld) {
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = st->g[i];
    for (int l = i + 1; l < k; ++l) acc = zsub(acc, zmul(st->H[(size_t)l * ld + i], st->y[l]));
    const double2 d = st->H[(size_t)i * ld + i];
    const double den = d.x * d.x + d.y * d.y;
    st->y[i] = den > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den)
                       : make_double2(0.0, 0.0);
  }
}

__global__ void x_update_kernel(double2* __restrict__ x, const float2* __restrict__ Z, size_t ld, int k,
                                size_t n, const KrylovState* __restrict__ st) {
  __shared__ float2 y[FDFD_MAXRESTART];
  if (threadIdx.x < k) y[threadIdx.x] = make_float2((float)st->y[threadIdx.x].x, (float)st->y[threadIdx.x].y);
  __syncthreads();
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    float2 d = make_float2(0.f, 0.f);
    for (int jj = 0; jj < k; ++jj) d = cadd(d, cmul(y[jj], __ldg(Z + (size_t)jj * ld + c)));
    double2 xc = x[c];
    xc.x += (double)d.x; xc.y += (double)d.y;
    x[c] = xc;
  }
}

__global__ void x_update_jacobi_kernel(double2* __restrict__ x, const float2* __restrict__ V, size_t ld,
                                       int k, size_t n, const KrylovState* __restrict__ st,
                                       const float* __restrict__ eps, const AxisCoef* __restrict__ cx,
                                       const AxisCoef* __restrict__ cy, float k2, int nx) {
  __shared__ float2 y[FDFD_MAXRESTART];
  if (threadIdx.x < k) {
    const double s = st->vscale[threadIdx.x];
    y[threadIdx.x] = make_float2((float)(st->y[threadIdx.x].x * s), (float)(st->y[threadIdx.x].y * s));
  }
  __syncthreads();
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    float2 d = make_float2(0.f, 0.f);
    for (int jj = 0; jj < k; ++jj) d = cadd(d, cmul(y[jj], __ldg(V + (size_t)jj * ld + c)));
    const int i = (int)(c % nx), j = (int)(c / nx);
    const float2 dg = make_float2(cx[i].dg.x + cy[j].dg.x + k2 * eps[c], cx[i].dg.y + cy[j].dg.y);
    const float inv = 1.f / (dg.x * dg.x + dg.y * dg.y);
    const float2 q = make_float2((d.x * dg.x + d.y * dg.y) * inv, (d.y * dg.x - d.x * dg.y) * inv);
    double2 xc = x[c];
    xc.x += (double)q.x; xc.y += (double)q.y;
    x[c] = xc;
  }
}

__global__ void store_field_kernel(const double2* __restrict__ x, float2* __restrict__ E, size_t n, double f) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    E[c] = make_float2((float)(f * x[c].x), (float)(f * x[c].y));
}
__global__ void load_field_kernel(const float2* __restrict__ E, double2* __restrict__ x, size_t n, double f) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    x[c] = make_double2(f * (double)E[c].x, f * (double)E[c].y);
}
__global__ void scale_copy_kernel(const float2* __restrict__ v, const double* __restrict__ sc,
                                  float2* __restrict__ z, size_t n) {
  const float s = (float)(*sc);
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
    z[c] = make_float2(v[c].x * s, v[c].y * s);
}

template <int NV>
int dots_nv(const float2* V, size_t ld, int v0, int nv, const float2* w, size_t n, KrylovState* st,
            double* partials, unsigned* counter, cudaStream_t s) {
  static int resident = 0;  // one wave of resident blocks: fewer partial sums to combine
  if (!resident) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs_dots_kernel<NV>, KT, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    resident = nsm * per_sm;
  }
  const int grid = krylov_grid(n) < resident ? krylov_grid(n) : resident;
  cgs_dots_kernel<NV><<<grid, KT, 0, s>>>(
      reinterpret_cast<const float4*>(V), ld / 2, v0, nv, reinterpret_cast<const float4*>(w), n / 2, st,
      reinterpret_cast<double2*>(partials), counter);
  CKL();
  return FDFD_OK;
}

template <int NV>
int update_nv(const float2* V, size_t ld, int v0, int nv, float2* w, float2* vnext, size_t n,
              KrylovState* st, double* partials, unsigned* counter, int j, int ldH, int fin,
              cudaStream_t s) {
  static int resident = 0;  // one wave of resident blocks (as for the dots)
  if (!resident) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs_update_kernel<NV>, KT, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    resident = nsm * per_sm;
  }
  const int grid = krylov_grid(n) < resident ? krylov_grid(n) : resident;
  cgs_update_kernel<NV><<<grid, KT, 0, s>>>(
      reinterpret_cast<const float4*>(V), ld / 2, v0, nv, reinterpret_cast<float4*>(w),
      reinterpret_cast<float4*>(vnext), n / 2, st, partials, counter, j, ldH, fin);
  CKL();
  return FDFD_OK;
}

}  // namespace

int krylov_grid(size_t n) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  const size_t want = (n / 2 + KT - 1) / KT;
  const size_t cap = (size_t)nsm * 8;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

int launch_cgs_dots(const float2* V, size_t ld, int j, const float2* w, size_t n, KrylovState* st,
                    double* partials, unsigned* counter, cudaStream_t s) {
  int rc = FDFD_OK;
  // at most 16 vectors per pass: more would cost occupancy (registers) than
  // the extra read of w saves
  for (int v0 = 0; v0 <= j && rc == FDFD_OK; v0 += 16) {
    const int nv = (j + 1 - v0) < 16 ? (j + 1 - v0) : 16;
    if (nv <= 8) rc = dots_nv<8>(V, ld, v0, nv, w, n, st, partials, counter, s);
    else rc = dots_nv<16>(V, ld, v0, nv, w, n, st, partials, counter, s);
  }
  return rc;
}

int launch_cgs_update(const float2* V, size_t ld, int j, float2* w, float2* vnext, size_t n,
                      KrylovState* st, double* partials, unsigned* counter, int restart,
                      cudaStream_t s) {
  int rc = FDFD_OK;
  const int ldH = restart + 1;
  // up to 32 vectors per pass: the update's registers do not grow with the
  // pass (its coefficients sit in shared memory), and every extra pass reads
  // and writes w once more
  for (int v0 = 0; v0 <= j && rc == FDFD_OK; v0 += 32) {
    const int nv = (j + 1 - v0) < 32 ? (j + 1 - v0) : 32;
    const int fin = (v0 + 32 > j);
    if (nv <= 8) rc = update_nv<8>(V, ld, v0, nv, w, vnext, n, st, partials, counter, j, ldH, fin, s);
    else if (nv <= 16) rc = update_nv<16>(V, ld, v0, nv, w, vnext, n, st, partials, counter, j, ldH, fin, s);
    else rc = update_nv<32>(V, ld, v0, nv, w, vnext, n, st, partials, counter, j, ldH, fin, s);
  }
  return rc;
}

int launch_cycle_start(KrylovState* st, cudaStream_t s) {
  cycle_start_kernel<<<1, 1, 0, s>>>(st);
  CKL();
  return FDFD_OK;
}

int launch_solve_y(KrylovState* st, int k, int restart, cudaStream_t s) {
  solve_y_kernel<<<1, 1, 0, s>>>(st, k, restart + 1);
  CKL();
  return FDFD_OK;
}

int launch_x_update(double2* x, const float2* Z, size_t ld, int k, size_t n, const KrylovState* st,
                    cudaStream_t s) {
  x_update_kernel<<<krylov_grid(n), 256, 0, s>>>(x, Z, ld, k, n, st);
  CKL();
  return FDFD_OK;
}

int launch_x_update_jacobi(double2* x, const float2* V, size_t ld, int k, size_t n,
                           const KrylovState* st, const float* eps, const AxisCoef* cx,
                           const AxisCoef* cy, float k2, int nx, cudaStream_t s) {
  x_update_jacobi_kernel<<<krylov_grid(n), 256, 0, s>>>(x, V, ld, k, n, st, eps, cx, cy, k2, nx);
  CKL();
  return FDFD_OK;
}

int launch_store_field(const double2* x, float2* E, size_t n, double f, cudaStream_t s) {
  store_field_kernel<<<krylov_grid(n), 256, 0, s>>>(x, E, n, f);
  CKL();
  return FDFD_OK;
}
int launch_load_field(const float2* E, double2* x, size_t n, double f, cudaStream_t s) {
  load_field_kernel<<<krylov_grid(n), 256, 0, s>>>(E, x, n, f);
  CKL();
  return FDFD_OK;
}
int launch_scale_copy(const float2* v, const double* sc, float2* z, size_t n, cudaStream_t s) {
  scale_copy_kernel<<<krylov_grid(n), 256, 0, s>>>(v, sc, z, n);
  CKL();
  return FDFD_OK;
}
