// Batched per-window NN-preconditioned flexible GMRES (Algorithm 1) on the
// local Robin problems of Algorithm 3's M.solve: every window runs m Arnoldi
// steps in lock step, the neural operator (Fig. 2) as the flexible
// preconditioner, the local Robin operator A_w of Eq. 1-2 as the matrix.
//
//   local_apply : y = A_w x on [n][80][80] window fields: the global 5-point
//                 UPML stencil restricted to the window, interface ghosts
//                 eliminated with zero Robin data (u_o = (1 - j kd_b) u_b),
//                 grid-edge ghosts zero.
//   local_cgs   : one CTA per window: h_i = (w, v_i), w -= sum h_i v_i,
//                 h_{j+1,j} = ||w||, v_{j+1} = w, FP64 Givens update.
//   local_sum   : e = sum_j y_j z_j after back substitution, written to the
//                 window's core of a global field (restricted prolongation)
//                 or to a window array.
#include "ctx.cuh"
#include "reduce.cuh"
#include "local.cuh"

namespace {

constexpr double kTiny = 1e-30;  // below this a window norm counts as zero


constexpr int LT = 256;
constexpr int NP = FDFD_WIN * FDFD_WIN;

__device__ inline void window_origin(int w, int nx, int ny, int nwx, int& x0, int& y0) {
  const int a = w % nwx, b = w / nwx;
  x0 = min(max(FDFD_CORE * a - FDFD_OVL, 0), nx - FDFD_WIN);
  y0 = min(max(FDFD_CORE * b - FDFD_OVL, 0), ny - FDFD_WIN);
}

__global__ void __launch_bounds__(LT) local_apply_kernel(const float2* __restrict__ x, float2* __restrict__ y,
                                                         const int* __restrict__ win_id, const float* __restrict__ eps,
                                                         const AxisCoef* __restrict__ cx,
                                                         const AxisCoef* __restrict__ cy, float k2, float k0dx,
                                                         int nx, int ny, int nwx) {
  const int b = blockIdx.y;
  const int w = win_id ? win_id[b] : b;
  int x0, y0;
  window_origin(w, nx, ny, nwx, x0, y0);
  const bool il = x0 > 0, ir = x0 + FDFD_WIN < nx, ib = y0 > 0, it = y0 + FDFD_WIN < ny;
  const float2* xb = x + (size_t)b * NP;
#pragma unroll 5
  for (int p = blockIdx.x * LT + threadIdx.x; p < NP; p += gridDim.x * LT) {
    const int ly = p / FDFD_WIN, lx = p % FDFD_WIN, gx = x0 + lx, gy = y0 + ly;
    const AxisCoef a = cx[gx], c = cy[gy];
    const float e = eps[(size_t)gy * nx + gx];
    const float2 xc = xb[p];
    float2 d = make_float2(a.dg.x + c.dg.x + k2 * e, a.dg.y + c.dg.y);
    const float kd = k0dx * sqrtf(e);
    const float2 f = make_float2(1.f, -kd);  // 1 - j kd
    float2 acc = make_float2(0.f, 0.f);
    if (lx > 0) acc = cadd(acc, cmul(a.lo, xb[p - 1])); else if (il) d = cadd(d, cmul(a.lo, f));
    if (lx < FDFD_WIN - 1) acc = cadd(acc, cmul(a.hi, xb[p + 1])); else if (ir) d = cadd(d, cmul(a.hi, f));
    if (ly > 0) acc = cadd(acc, cmul(c.lo, xb[p - FDFD_WIN])); else if (ib) d = cadd(d, cmul(c.lo, f));
    if (ly < FDFD_WIN - 1) acc = cadd(acc, cmul(c.hi, xb[p + FDFD_WIN])); else if (it) d = cadd(d, cmul(c.hi, f));
    y[(size_t)b * NP + p] = cadd(acc, cmul(d, xc));
  }
}

// Robin data -> right-hand side: rhs_b = -c_bo g on interface boundary cells.
__global__ void __launch_bounds__(LT) robin_rhs_kernel(const float2* __restrict__ g, float2* __restrict__ rhs,
                                                       const AxisCoef* __restrict__ cx,
                                                       const AxisCoef* __restrict__ cy, int nx, int ny, int nwx) {
  const int b = blockIdx.x;
  int x0, y0;
  window_origin(b, nx, ny, nwx, x0, y0);
  const bool iface[4] = {x0 > 0, x0 + FDFD_WIN < nx, y0 > 0, y0 + FDFD_WIN < ny};
  float2* r = rhs + (size_t)b * NP;
  for (int p = threadIdx.x; p < NP; p += LT) r[p] = make_float2(0.f, 0.f);
  __syncthreads();
  // one thread per t, one side at a time (corner cells get two terms)
  const float2* gw = g + (size_t)b * 320;
  for (int s = 0; s < 4; ++s) {
    if (threadIdx.x < FDFD_WIN && iface[s]) {
      const int t = threadIdx.x;
      int lx, ly;
      float2 cbo;
      if (s == 0) { lx = 0; ly = t; cbo = cx[x0].lo; }
      else if (s == 1) { lx = FDFD_WIN - 1; ly = t; cbo = cx[x0 + FDFD_WIN - 1].hi; }
      else if (s == 2) { lx = t; ly = 0; cbo = cy[y0].lo; }
      else { lx = t; ly = FDFD_WIN - 1; cbo = cy[y0 + FDFD_WIN - 1].hi; }
      const float2 v = cmul(cbo, gw[s * 80 + t]);
      float2& dst = r[ly * FDFD_WIN + lx];
      dst = make_float2(dst.x - v.x, dst.y - v.y);
    }
    __syncthreads();
  }
}

// Window reductions.  GB300 issues FP64 at a small fraction of the FP32 rate
// (tens of cycles per warp instruction), so per-pixel FP64 products and
// FP64 warp shuffles cost more than a window's loads: each thread sums its
// 25 pixels in FP32, each warp its 32 threads in FP32, and only the block's
// eight warp partials are added in FP64.
__device__ __forceinline__ float warp_sum_f32(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// FP64 sum of the block's per-thread values v (valid in thread 0).
__device__ __forceinline__ double block_sum_warps(float v, double* sh) {
  v = warp_sum_f32(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < LT / 32; ++w) t += sh[w];
  return t;
}
// A thread's share of a window's squared norm, acc32 being its FP32 sum of
// squares.  Where that sum may have underflowed or overflowed although the
// thread's values are not all zero (very small or very large window values,
// e.g. an unscaled source in the stationary solver), the thread sums its
// pixels again, from the vector it has just written, in FP64 into acc64 and
// sets exact64; all-zero windows (frequent while the Krylov vectors are
// still local) take the FP32 path.
__device__ __forceinline__ float norm2_share(float acc32, bool nonzero, const float2* __restrict__ win, bool& exact64,
                                             double& acc64) {
  exact64 = nonzero && !(acc32 >= 1e-30f && acc32 <= 1e36f);
  if (!exact64) return acc32;
  double acc = 0.0;
  for (int p = threadIdx.x; p < NP; p += LT) {
    const float2 q = win[p];
    acc += (double)q.x * q.x + (double)q.y * q.y;
  }
  acc64 = acc;
  return 0.f;
}
// Block sum of the norm shares: FP32 warp sums where every thread took the
// FP32 path, else (rare) an FP64 sum of all threads' shares.
__device__ __forceinline__ double block_norm2(float share, bool exact64, double acc64, double* sh) {
  if (!__syncthreads_or(exact64)) return block_sum_warps(share, sh);
  const double v = exact64 ? acc64 : (double)share;
  return block_sum<LT>(v, sh);
}

// Restriction of a global field into window arrays, and initial norms.
__global__ void __launch_bounds__(LT) local_start_kernel(const float2* __restrict__ v, const float2* __restrict__ rhs_win,
                                                         float2* __restrict__ V0, LocalState* st, int nx, int ny,
                                                         int nwx) {
  __shared__ double sh[LT / 32];
  const int b = blockIdx.x;
  int x0, y0;
  window_origin(b, nx, ny, nwx, x0, y0);
  float acc32 = 0.f;
  bool nz = false;
#pragma unroll 5
  for (int t = 0; t < NP / LT; ++t) {  // five pixels' loads in flight per thread
    const int p = threadIdx.x + t * LT;
    const float2 q = rhs_win ? rhs_win[(size_t)b * NP + p]
                             : v[(size_t)(y0 + p / FDFD_WIN) * nx + x0 + p % FDFD_WIN];
    V0[(size_t)b * NP + p] = q;
    acc32 += q.x * q.x + q.y * q.y;
    nz |= (q.x != 0.f) | (q.y != 0.f);
  }
  bool ex; double a64 = 0.0;
  const float share = norm2_share(acc32, nz, V0 + (size_t)b * NP, ex, a64);
  const double t = block_norm2(share, ex, a64, sh);
  if (threadIdx.x == 0) {
    LocalState& s = st[b];
    const double beta = sqrt(t);
    s.beta = beta;
    s.g[0] = make_double2(beta, 0.0);
    // the outer solve's vectors are O(1) overall; a window whose restriction is
    // below kTiny carries nothing of weight and its 1/beta would leave the FP32
    // range of the network's scaling, so it is treated as empty
    s.vscale[0] = beta > kTiny ? 1.0 / beta : 0.0;
    s.k = 0;
  }
}

// One CGS step of window b's Arnoldi process plus its Givens update.  JT >= 0
// fixes j = JT at compile time (accumulators for the j + 1 dots only, more
// windows resident per SM); JT = -1 takes j at run time.  Both forms add in
// the same order, so they give the same bits.
static_assert(NP % LT == 0, "whole pixel rounds per thread");
template <int JT>
__global__ void __launch_bounds__(LT) local_cgs_kernel(const float2* __restrict__ Vw, float2* __restrict__ w_io,
                                                       float2* __restrict__ vnext, LocalState* st, int j_rt,
                                                       size_t ldv) {
  constexpr int NA = JT >= 0 ? JT + 1 : LOCAL_MAXM + 1;  // accumulator pairs
  const int j = JT >= 0 ? JT : j_rt;
  __shared__ double sh[LT / 32];
  __shared__ double2 hs[LOCAL_MAXM + 1];
  __shared__ double part[LT / 32][2 * (LOCAL_MAXM + 1)];
  __shared__ float2 hf[LOCAL_MAXM + 1];
  const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  LocalState& s = st[b];
  const float2* w = w_io + (size_t)b * NP;
  // all dots (w, v_i), i <= j, in one pass: FP32 sums over each thread's 25
  // pixels, FP64 across the block
  float dr[NA], di[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) { dr[i] = 0.f; di[i] = 0.f; }
#pragma unroll(JT >= 0 ? 5 : 1)
  for (int t = 0; t < NP / LT; ++t) {
    const int p = threadIdx.x + t * LT;
    const float2 q = w[p];
#pragma unroll
    for (int i = 0; i < NA; ++i)
      if (i <= j) {
        const float2 a = Vw[(size_t)i * ldv + (size_t)b * NP + p];
        dr[i] += a.x * q.x + a.y * q.y;
        di[i] += a.x * q.y - a.y * q.x;
      }
  }
#pragma unroll
  for (int i = 0; i < NA; ++i)
    if (i <= j) {
      const float r = warp_sum_f32(dr[i]), m = warp_sum_f32(di[i]);
      if (lane == 0) { part[warp][2 * i] = (double)r; part[warp][2 * i + 1] = (double)m; }
    }
  __syncthreads();
  if (threadIdx.x <= j) {
    const int i = threadIdx.x;
    double r = 0.0, m = 0.0;
    for (int q = 0; q < LT / 32; ++q) { r += part[q][2 * i]; m += part[q][2 * i + 1]; }
    hs[i] = make_double2(r * s.vscale[i], m * s.vscale[i]);
    hf[i] = make_float2((float)(hs[i].x * s.vscale[i]), (float)(hs[i].y * s.vscale[i]));
  }
  __syncthreads();
  float acc32 = 0.f;
  bool nz = false;
#pragma unroll(JT >= 0 ? 5 : 1)
  for (int t = 0; t < NP / LT; ++t) {
    const int p = threadIdx.x + t * LT;
    float2 q = w[p];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      if (i > j) break;
      const float2 a = Vw[(size_t)i * ldv + (size_t)b * NP + p];
      const float hr = hf[i].x, hi = hf[i].y;
      q.x -= hr * a.x - hi * a.y;
      q.y -= hr * a.y + hi * a.x;
    }
    vnext[(size_t)b * NP + p] = q;
    acc32 += q.x * q.x + q.y * q.y;
    nz |= (q.x != 0.f) | (q.y != 0.f);
  }
  bool ex; double a64 = 0.0;
  const float share = norm2_share(acc32, nz, vnext + (size_t)b * NP, ex, a64);
  const double nrm2 = block_norm2(share, ex, a64, sh);
  if (threadIdx.x == 0) {
    const double hn = sqrt(nrm2);
    double2 Hc[LOCAL_MAXM + 1];
    for (int i = 0; i <= j; ++i) Hc[i] = hs[i];
    Hc[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const double c = s.cs[i];
      const double2 sn = s.sn[i], a = Hc[i], bb = Hc[i + 1];
      Hc[i] = zadd(make_double2(c * a.x, c * a.y), zmul(sn, bb));
      Hc[i + 1] = zsub(make_double2(c * bb.x, c * bb.y), zmul(zconj(sn), a));
    }
    const double2 a = Hc[j], bb = Hc[j + 1];
    const double aa = hypot(a.x, a.y), bm = hypot(bb.x, bb.y);
    double c; double2 sn;
    if (bm == 0.0) { c = 1.0; sn = make_double2(0.0, 0.0); }
    else if (aa == 0.0) { c = 0.0; sn = make_double2(bb.x / bm, -bb.y / bm); }
    else {
      const double t = hypot(aa, bm);
      c = aa / t;
      sn = zmul(make_double2(a.x / aa, a.y / aa), make_double2(bb.x / t, -bb.y / t));
    }
    s.cs[j] = c; s.sn[j] = sn;
    Hc[j] = zadd(make_double2(c * a.x, c * a.y), zmul(sn, bb));
    for (int i = 0; i <= j; ++i) s.H[j * (LOCAL_MAXM + 1) + i] = Hc[i];
    const double2 gj = s.g[j];
    s.g[j + 1] = zmul(make_double2(-sn.x, sn.y), gj);
    s.g[j] = make_double2(c * gj.x, c * gj.y);
    s.vscale[j + 1] = hn > kTiny ? 1.0 / hn : 0.0;
    s.k = j + 1;
  }
}

__global__ void local_solve_y_kernel(LocalState* st, int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  LocalState& s = st[b];
  const int k = s.k;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = s.g[i];
    for (int l = i + 1; l < k; ++l) acc = zsub(acc, zmul(s.H[l * (LOCAL_MAXM + 1) + i], s.y[l]));
    const double2 d = s.H[i * (LOCAL_MAXM + 1) + i];
    const double den = d.x * d.x + d.y * d.y;
    s.y[i] = (den > 0 && s.beta > 0)
                 ? make_double2((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den)
                 : make_double2(0.0, 0.0);
  }
}

// e = sum_j y_j z_j, into the core of a global field (x outer scale) or a window array.
__global__ void __launch_bounds__(LT) local_sum_kernel(const float2* __restrict__ Zw, size_t ldz, const LocalState* st,
                                                       float2* __restrict__ z_global, float2* __restrict__ e_win,
                                                       const double* __restrict__ scale, int nx, int ny, int nwx) {
  const int b = blockIdx.y;
  int x0, y0;
  window_origin(b, nx, ny, nwx, x0, y0);
  const LocalState& s = st[b];
  const float f = scale ? (float)(*scale) : 1.f;
  float2 y[LOCAL_MAXM];
  for (int i = 0; i < s.k; ++i) y[i] = make_float2((float)s.y[i].x * f, (float)s.y[i].y * f);
  const int a = b % nwx, bb = b / nwx;
  const int cx0 = FDFD_CORE * a - x0, cy0 = FDFD_CORE * bb - y0;
#pragma unroll 5
  for (int p = blockIdx.x * LT + threadIdx.x; p < NP; p += gridDim.x * LT) {
    const int ly = p / FDFD_WIN, lx = p % FDFD_WIN;
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < s.k; ++i) acc = cadd(acc, cmul(y[i], Zw[(size_t)i * ldz + (size_t)b * NP + p]));
    if (e_win) { e_win[(size_t)b * NP + p] = acc; continue; }
    if (lx < cx0 || lx >= cx0 + FDFD_CORE || ly < cy0 || ly >= cy0 + FDFD_CORE) continue;
    z_global[(size_t)(y0 + ly) * nx + x0 + lx] = acc;
  }
}

__global__ void vscale_copy_kernel(const LocalState* st, double* out, int j, int n) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) out[b] = st[b].vscale[j];
}

}  // namespace

int local_alloc(LocalWork* L, int n_win, int m, size_t* bytes) {
  if (m < 1 || m > LOCAL_MAXM) return FDFD_EINVAL;
  L->m = m;
  L->n = n_win;
  const size_t nv = (size_t)n_win * NP;
  struct { void** p; size_t b; } a[] = {{(void**)&L->V, (size_t)(m + 1) * nv * 8}, {(void**)&L->Z, (size_t)m * nv * 8},
                                        {(void**)&L->w, nv * 8}, {(void**)&L->st, (size_t)n_win * sizeof(LocalState)},
                                        {(void**)&L->escale, (size_t)n_win * 8}};
  for (auto& e : a) {
    if (cudaMalloc(e.p, e.b) != cudaSuccess) return FDFD_ENOMEM;
    *bytes += e.b;
  }
  return FDFD_OK;
}

void local_free(LocalWork* L) {
  void* ptrs[] = {L->V, L->Z, L->w, L->st, L->escale};
  for (void* p : ptrs) if (p) cudaFree(p);
  *L = LocalWork();
}

int local_robin_rhs(fdfd_ctx* h, const float2* g, float2* rhs, int n_win) {
  robin_rhs_kernel<<<n_win, LT, 0, h->stream>>>(g, rhs, h->cx, h->cy, h->nx, h->ny, h->nx / FDFD_CORE);
  CKL();
  return FDFD_OK;
}

int local_fgmres(fdfd_ctx* h, LocalWork* L, const NnoWeights* W, NnoWork* work, const float2* v_global,
                 const float2* rhs_win, float2* z_global, float2* e_win, const double* scale, int transpose) {
  const int n = L->n, nwx = h->nx / FDFD_CORE;
  // for the adjoint solve the local problems use the transposed couplings
  const AxisCoef* lcx = transpose ? h->cxT : h->cx;
  const AxisCoef* lcy = transpose ? h->cyT : h->cy;
  const size_t ld = (size_t)n * NP;
  cudaStream_t s = h->stream;
  GridGeom g{h->nx, h->ny, nwx, (float)h->k2, h->eps, h->isx, h->isy, schwarz_modulation(h)};
  int rc;
  {
    ProfScope ps(h, 4, 1);
    local_start_kernel<<<n, LT, 0, s>>>(v_global, rhs_win, L->V, L->st, h->nx, h->ny, nwx);
    CKL();
  }
  for (int j = 0; j < L->m; ++j) {
    {
      ProfScope ps(h, 4, 1);
      vscale_copy_kernel<<<(n + 255) / 256, 256, 0, s>>>(L->st, L->escale, j, n);
      CKL();
    }
    NnoInput in;
    in.r_win = L->V + (size_t)j * ld;
    NnoOutput out;
    out.e_win = L->Z + (size_t)j * ld;
    out.scale_win = L->escale;
    if ((rc = nno_forward(W, work, g, in, out, n, s, h))) return rc;
    {
      ProfScope ps(h, 15, 2);
      local_apply_kernel<<<dim3(NP / LT / 5, n), LT, 0, s>>>(L->Z + (size_t)j * ld, L->w, nullptr, h->eps, lcx,
                                                              lcy, (float)h->k2, (float)h->k0dx, h->nx, h->ny, nwx);
      float2* vn = L->V + (size_t)(j + 1) * ld;
      switch (j) {  // the first steps (the usual inner counts) with j fixed at compile time
        case 0: local_cgs_kernel<0><<<n, LT, 0, s>>>(L->V, L->w, vn, L->st, j, ld); break;
        case 1: local_cgs_kernel<1><<<n, LT, 0, s>>>(L->V, L->w, vn, L->st, j, ld); break;
        case 2: local_cgs_kernel<2><<<n, LT, 0, s>>>(L->V, L->w, vn, L->st, j, ld); break;
        case 3: local_cgs_kernel<3><<<n, LT, 0, s>>>(L->V, L->w, vn, L->st, j, ld); break;
        default: local_cgs_kernel<-1><<<n, LT, 0, s>>>(L->V, L->w, vn, L->st, j, ld); break;
      }
      CKL();
    }
  }
  ProfScope ps(h, 4, 2);
  local_solve_y_kernel<<<(n + 127) / 128, 128, 0, s>>>(L->st, n);
  local_sum_kernel<<<dim3(5, n), LT, 0, s>>>(L->Z, ld, L->st, z_global, e_win, scale, h->nx, h->ny, nwx);
  CKL();
  return FDFD_OK;
}

int local_apply_windows(fdfd_ctx* h, const float2* x, float2* y, const int* win_id, int n) {
  local_apply_kernel<<<dim3(NP / LT / 5, n), LT, 0, h->stream>>>(x, y, win_id, h->eps, h->cx, h->cy, (float)h->k2,
                                                                  (float)h->k0dx, h->nx, h->ny, h->nx / FDFD_CORE);
  CKL();
  return FDFD_OK;
}
