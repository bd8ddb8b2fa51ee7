// Coarse space of the two-level Schwarz method (Sec. 2.2; Methods,
// Algorithm 3 set-up and correction; Eq. 7-8).
//
// Set-up: pseudo-plane-wave Robin trials walked around each window with
// the local wavenumber, modified Gram-Schmidt in FP64, homogeneous neural
// solves for each trial, the traces of the restricted basis fields on the
// neighbours' boundaries minus the window's own data (C = BQ - Q, stored as
// 9 neighbour blocks per window).  Optional Rayleigh-Ritz truncation
// (Algorithm 3 set-up: eta, u = eig(H); Sec. 2.2: the slowly decaying modes
// above a threshold): per window the Ritz matrix H = Q^H Y of the
// Robin-to-Robin map (Y: the data each basis field hands to the neighbours,
// read on their sides facing the window), its eigenpairs (one thread per
// window, eig.cuh), and Q, Phi and the window's columns of C combined by the
// eigenvectors with |eta| >= ritz_tol; the other directions become zero
// columns, pinned like dependent trials.
//
// Coarse equation (reading of Eq. 7 with the Rayleigh-Ritz step): the
// Galerkin projection of the interface operator onto the trial space,
//     G z = -Q^H e_bc,   G = Q^H C   (blocks G[i][j] = Q_i^H C[i][j]),
// a 9-block stencil over the window grid.  Ordered by window rows it is
// block tridiagonal, G = tridiag(L_b, D_b, U_b) with blocks of size
// D = nwx k, and is factored once by block elimination over the rows:
//     S_0 = D_0,   S_b = D_b - L_b S_{b-1}^-1 U_{b-1},
// each S_b inverted explicitly (FP32 LU with partial pivoting, cuSOLVER, at
// set-up; the block-sparse products L_b S^-1 U are this file's kernels).
// Apply: e_bc = traces of the one-level field, r = -Q^H e_bc, a forward
// sweep y_b = S_b^-1 (r_b - L_b y_{b-1}) and a backward sweep
// z_b = y_b - S_b^-1 U_b z_{b+1} (dense GEMVs, HBM-bound), then
// u += sum_w R~_w^T sum_m z_{w,m} Phi_{w,m}.  Storage grows as
// nwy D^2 (8.6 GB at 4096^2, k = 64) instead of the (nwx nwy k)^2 of a
// dense inverse.
#include <math.h>
#include <vector>
#include <cusolverDn.h>
#include <cuda_fp16.h>
#include "ctx.cuh"
#include "nno.cuh"
#include "local.cuh"
#include "reduce.cuh"
#include "eig.cuh"

struct CoarseData {
  int k = 0, nc = 0, nwx = 0, nwy = 0, D = 0;
  double2* Q = nullptr;      // [n_win][k][320]
  float2* Qf = nullptr;      // [k][n_win][320]
  float2* Phi = nullptr;     // [n_win][k][64*64] core of each basis field (set-up only)
  __half2* Phih = nullptr;   // the same, complex half: what the correction reads
  double2* C = nullptr;      // [n_win][9][320][k]   (set-up only)
  double2* G = nullptr;      // [n_win][9][k][k]     Galerkin blocks, FP64
  float2* Gf = nullptr;      // [n_win][9][k][k]     FP32 copy used by the sweeps
  __half2* Sinv = nullptr;   // [nwy][D][D]          row-major S_b^-1, complex half (re, im)
  float2* rcf = nullptr;     // [nc] right-hand side -Q^H e_bc
  float2* ycf = nullptr;     // [nc] forward sweep
  float2* zcf = nullptr;     // [nc] coarse solution
  float2* tcf = nullptr;     // [D]  row temporary
  float2* ebc = nullptr;     // [n_win][320]
  float2* tmp = nullptr;     // [n_win][6400] window fields during set-up
  int* dropped = nullptr;    // [nc]
  double2* eta = nullptr;    // [n_win][k] Ritz values (Ritz step only)
  double2* H = nullptr;      // [n_win][k][k] Ritz matrices (Ritz step only)
  int n_kept = 0;            // unknowns not dropped
};

namespace {

struct Win {
  int x0, y0, a, b;
  bool iface[4];
};

__host__ __device__ inline Win win_of(int w, int nx, int ny, int nwx) {
  Win r;
  r.a = w % nwx; r.b = w / nwx;
  r.x0 = min(max(FDFD_CORE * r.a - FDFD_OVL, 0), nx - FDFD_WIN);
  r.y0 = min(max(FDFD_CORE * r.b - FDFD_OVL, 0), ny - FDFD_WIN);
  r.iface[0] = r.x0 > 0; r.iface[1] = r.x0 + FDFD_WIN < nx;
  r.iface[2] = r.y0 > 0; r.iface[3] = r.y0 + FDFD_WIN < ny;
  return r;
}

// boundary cell b and ghost o of slot (side s, t)
__device__ inline void slot_cells(const Win& W, int s, int t, int& bx, int& by, int& ox, int& oy) {
  if (s == 0) { bx = W.x0; by = W.y0 + t; ox = bx - 1; oy = by; }
  else if (s == 1) { bx = W.x0 + FDFD_WIN - 1; by = W.y0 + t; ox = bx + 1; oy = by; }
  else if (s == 2) { bx = W.x0 + t; by = W.y0; ox = bx; oy = by - 1; }
  else { bx = W.x0 + t; by = W.y0 + FDFD_WIN - 1; ox = bx; oy = by + 1; }
}

// Counter-clockwise walk: bottom (t up), right (t up), top (t down), left (t down).
__device__ inline void walk_step(int n, int& s, int& t) {
  const int seg = n / FDFD_WIN, r = n % FDFD_WIN;
  if (seg == 0) { s = 2; t = r; }
  else if (seg == 1) { s = 1; t = r; }
  else if (seg == 2) { s = 3; t = FDFD_WIN - 1 - r; }
  else { s = 0; t = FDFD_WIN - 1 - r; }
}

__global__ void __launch_bounds__(256) trials_gs_kernel(double2* Q, float2* Qf, int k, const float* eps, double k0dx,
                                                        int nx, int ny, int nwx, int n_win) {
  __shared__ double sh[8];
  __shared__ double2 s_dot;
  __shared__ double s_norm;
  const int w = blockIdx.x;
  const Win W = win_of(w, nx, ny, nwx);
  double2* Qw = Q + (size_t)w * k * 320;
  // trial data: phase accumulated along the perimeter with the local wavenumber
  for (int m = threadIdx.x; m < k; m += blockDim.x) {
    const double th = 2.0 * M_PI * m / k, dxh = cos(th), dyh = sin(th);
    double phi = 0.0, kprev = 0.0;
    int px = 0, py = 0;
    for (int n = 0; n < 320; ++n) {
      int s, t, bx, by, ox, oy;
      walk_step(n, s, t);
      slot_cells(W, s, t, bx, by, ox, oy);
      const double kd = k0dx * sqrt((double)eps[(size_t)by * nx + bx]);
      if (n > 0) phi += 0.5 * (kprev + kd) * (dxh * (bx - px) + dyh * (by - py));
      kprev = kd; px = bx; py = by;
      Qw[(size_t)m * 320 + s * 80 + t] = W.iface[s] ? make_double2(cos(phi), -sin(phi)) : make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  // modified Gram-Schmidt in FP64 (l2 over the 320 slots)
  for (int m = 0; m < k; ++m) {
    double2* v = Qw + (size_t)m * 320;
    double a0 = 0.0;
    for (int t = threadIdx.x; t < 320; t += blockDim.x) a0 += v[t].x * v[t].x + v[t].y * v[t].y;
    a0 = block_sum<256>(a0, sh);
    if (threadIdx.x == 0) s_norm = sqrt(a0);
    __syncthreads();
    const double n0 = s_norm;
    for (int i = 0; i < m; ++i) {
      const double2* qi = Qw + (size_t)i * 320;
      double dr = 0.0, di = 0.0;
      for (int t = threadIdx.x; t < 320; t += blockDim.x) {  // conj(q_i) . v
        dr += qi[t].x * v[t].x + qi[t].y * v[t].y;
        di += qi[t].x * v[t].y - qi[t].y * v[t].x;
      }
      dr = block_sum<256>(dr, sh);
      di = block_sum<256>(di, sh);
      if (threadIdx.x == 0) s_dot = make_double2(dr, di);
      __syncthreads();
      const double2 d = s_dot;
      for (int t = threadIdx.x; t < 320; t += blockDim.x) v[t] = zsub(v[t], zmul(d, qi[t]));
      __syncthreads();
    }
    double a = 0.0;
    for (int t = threadIdx.x; t < 320; t += blockDim.x) a += v[t].x * v[t].x + v[t].y * v[t].y;
    a = block_sum<256>(a, sh);
    if (threadIdx.x == 0) s_norm = sqrt(a);
    __syncthreads();
    const double nv = s_norm;
    const double f = (n0 == 0.0 || nv <= 1e-10 * n0) ? 0.0 : 1.0 / nv;
    for (int t = threadIdx.x; t < 320; t += blockDim.x) {
      v[t] = make_double2(v[t].x * f, v[t].y * f);
      Qf[((size_t)m * n_win + w) * 320 + t] = make_float2((float)v[t].x, (float)v[t].y);
    }
    __syncthreads();
  }
}

__global__ void copy_core_kernel(const float2* tmp, float2* Phi, int m, int k, int nx, int ny, int nwx, int n_win) {
  const int w = blockIdx.x;
  const Win W = win_of(w, nx, ny, nwx);
  const int cx = FDFD_CORE * W.a - W.x0, cy = FDFD_CORE * W.b - W.y0;
  for (int p = threadIdx.x; p < FDFD_CORE * FDFD_CORE; p += blockDim.x) {
    const int y = p / FDFD_CORE, x = p % FDFD_CORE;
    Phi[((size_t)w * k + m) * 4096 + p] = tmp[(size_t)w * 6400 + (cy + y) * 80 + cx + x];
  }
}

// C[i][j][slot][m] = trace on window i's slot of R~_J^T Phi_{J,m} (J = neighbour j of i), minus Q_i on j = self.
__global__ void assemble_C_kernel(double2* C, const double2* Q, const float2* Phi, int k, const float* eps,
                                  double k0dx, int nx, int ny, int nwx, int nwy) {
  const int i = blockIdx.x, j = blockIdx.y;
  const int n_win = nwx * nwy;
  const Win Wi = win_of(i, nx, ny, nwx);
  const int dx = j % 3 - 1, dy = j / 3 - 1;
  const int aJ = Wi.a + dx, bJ = Wi.b + dy;
  const bool hasJ = aJ >= 0 && aJ < nwx && bJ >= 0 && bJ < nwy;
  const int J = bJ * nwx + aJ;
  for (int e = threadIdx.x; e < 320 * k; e += blockDim.x) {
    const int slot = e / k, m = e % k, s = slot / 80, t = slot % 80;
    double2 val = make_double2(0.0, 0.0);
    if (Wi.iface[s] && hasJ) {
      int bx, by, ox, oy;
      slot_cells(Wi, s, t, bx, by, ox, oy);
      auto core_val = [&](int gx, int gy) -> double2 {
        const int cx = gx - FDFD_CORE * aJ, cy = gy - FDFD_CORE * bJ;
        if (cx < 0 || cx >= FDFD_CORE || cy < 0 || cy >= FDFD_CORE) return make_double2(0.0, 0.0);
        const float2 f = Phi[((size_t)J * k + m) * 4096 + cy * FDFD_CORE + cx];
        return make_double2(f.x, f.y);
      };
      const double2 ub = core_val(bx, by), uo = core_val(ox, oy);
      const double kd = k0dx * sqrt((double)eps[(size_t)by * nx + bx]);
      // u_o - (1 - j kd) u_b
      val = make_double2(uo.x - ub.x - kd * ub.y, uo.y - ub.y + kd * ub.x);
      if (j == 4) val = zsub(val, Q[((size_t)i * k + m) * 320 + slot]);
    }
    (void)n_win;
    C[(((size_t)i * 9 + j) * 320 + slot) * k + m] = val;
  }
}

// Galerkin blocks G[i][j][p][q] = sum_slot conj(Q_i[p][slot]) C[i][j][slot][q]
// (window i's test functions against the basis of J = i + offset j).
// Unknowns with a zero trial vector (dropped) get a unit diagonal.
__global__ void assemble_G_kernel(double2* __restrict__ G, const double2* __restrict__ Q,
                                  const double2* __restrict__ C, int k) {
  const int i = blockIdx.x, j = blockIdx.y;
  const double2* Qi = Q + (size_t)i * k * 320;
  const double2* Cij = C + ((size_t)i * 9 + j) * 320 * k;
  double2* Gij = G + ((size_t)i * 9 + j) * k * k;
  for (int pq = threadIdx.x; pq < k * k; pq += blockDim.x) {
    const int p = pq / k, q = pq % k;
    double sr = 0.0, si = 0.0, qn = 0.0;
    for (int sl = 0; sl < 320; ++sl) {
      const double2 a = Qi[(size_t)p * 320 + sl], c = Cij[(size_t)sl * k + q];  // conj(a) * c
      sr += a.x * c.x + a.y * c.y;
      si += a.x * c.y - a.y * c.x;
      qn += a.x * a.x + a.y * a.y;
    }
    if (j == 4 && p == q && qn == 0.0) { sr = 1.0; si = 0.0; }
    Gij[pq] = make_double2(sr, si);
  }
}

__global__ void dropped_kernel(int* dropped, const double2* Q, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double2* q = Q + (size_t)c * 320;
  bool any = false;
  for (int t = 0; t < 320; ++t) any |= (q[t].x != 0.0 || q[t].y != 0.0);
  dropped[c] = !any;
}

// Q [w][k][320] FP64 -> Qf [k][w][320] FP32 (after the Ritz rotation).
__global__ void q_to_f32_kernel(float2* Qf, const double2* Q, int k, int n_win) {
  const int w = blockIdx.x;
  for (int e = threadIdx.x; e < k * 320; e += blockDim.x) {
    const int m = e / 320, sl = e % 320;
    const double2 v = Q[((size_t)w * k + m) * 320 + sl];
    Qf[((size_t)m * n_win + w) * 320 + sl] = make_float2((float)v.x, (float)v.y);
  }
}

// S (row-major D x D) = D_b: the blocks of window row b coupling windows
// of the same row (offsets j = 3, 4, 5).
__global__ void build_S_kernel(float2* __restrict__ S, const float2* __restrict__ Gf, int k, int nwx, int b) {
  const int D = nwx * k;
  const size_t n = (size_t)D * D;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / D), c = (int)(e % D);
    const int a = r / k, p = r % k, a2 = c / k, q = c % k;
    const int d = a2 - a;
    float2 v = make_float2(0.f, 0.f);
    if (d >= -1 && d <= 1) v = Gf[(((size_t)(b * nwx + a) * 9 + 4 + d) * k + p) * k + q];
    S[e] = v;
  }
}

// T = Sinv_{b-1} U_{b-1}: U couples window (a, b-1) to (a + d, b), offset
// j = 7 + d.  T[r][(a2, q)] = sum_{a = a2-1..a2+1} sum_p Sinv[r][(a, p)]
// U[(a, p)][(a2, q)].  Each thread: RT rows of one column.
constexpr int RT = 4;
__global__ void __launch_bounds__(256) schur_T_kernel(float2* __restrict__ T, const float2* __restrict__ Sinv,
                                                      const float2* __restrict__ Gf, int k, int nwx, int b) {
  const int D = nwx * k;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * RT;
  if (c >= D) return;
  const int a2 = c / k, q = c % k;
  float2 acc[RT];
#pragma unroll
  for (int t = 0; t < RT; ++t) acc[t] = make_float2(0.f, 0.f);
  for (int a = max(a2 - 1, 0); a <= min(a2 + 1, nwx - 1); ++a) {
    const float2* Ub = Gf + ((size_t)((b - 1) * nwx + a) * 9 + 7 + (a2 - a)) * k * k + q;
    for (int p = 0; p < k; ++p) {
      const float2 u = __ldg(Ub + (size_t)p * k);
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        const int r = r0 + t;
        if (r < D) acc[t] = cadd(acc[t], cmul(__ldg(Sinv + (size_t)r * D + a * k + p), u));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < RT; ++t)
    if (r0 + t < D) T[(size_t)(r0 + t) * D + c] = acc[t];
}

// S -= L_b T: L couples window (a, b) to (a + d, b - 1), offset j = 1 + d.
// S[(a, p)][c] -= sum_{a3 = a-1..a+1} sum_p3 L[(a, p)][(a3, p3)] T[(a3, p3)][c].
// Each thread: RT consecutive rows (which may straddle two windows) of one column.
__global__ void __launch_bounds__(256) schur_update_kernel(float2* __restrict__ S, const float2* __restrict__ T,
                                                           const float2* __restrict__ Gf, int k, int nwx, int b) {
  const int D = nwx * k;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * RT;
  if (c >= D || r0 >= D) return;
  const int alo = r0 / k, ahi = min(r0 + RT - 1, D - 1) / k;
  float2 acc[RT];
#pragma unroll
  for (int t = 0; t < RT; ++t) acc[t] = make_float2(0.f, 0.f);
  for (int a3 = max(alo - 1, 0); a3 <= min(ahi + 1, nwx - 1); ++a3) {
    for (int p3 = 0; p3 < k; ++p3) {
      const float2 tv = __ldg(T + (size_t)(a3 * k + p3) * D + c);
#pragma unroll
      for (int t = 0; t < RT; ++t) {
        const int r = r0 + t;
        if (r >= D) continue;
        const int a = r / k, d = a3 - a;
        if (d < -1 || d > 1) continue;
        const float2 l = __ldg(Gf + (((size_t)(b * nwx + a) * 9 + 1 + d) * k + r % k) * k + p3);
        acc[t] = cadd(acc[t], cmul(l, tv));
      }
    }
  }
#pragma unroll
  for (int t = 0; t < RT; ++t) {
    if (r0 + t >= D) continue;
    float2& d = S[(size_t)(r0 + t) * D + c];
    d = make_float2(d.x - acc[t].x, d.y - acc[t].y);
  }
}

__global__ void nonfinite_kernel(const float2* __restrict__ a, size_t n, int* flag) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(a[e].x) || !isfinite(a[e].y)) { atomicExch(flag, 1); return; }
}

__global__ void identity_kernel(float2* X, int D) {
  const size_t n = (size_t)D * D;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    X[e] = make_float2((e / D == e % D) ? 1.f : 0.f, 0.f);
}

// r[w][m] = -sum_slot conj(Qf[m][w][slot]) e_bc[w][slot]  (warp per m)
__global__ void __launch_bounds__(256) galerkin_rhs_kernel(float2* __restrict__ r, const float2* __restrict__ Qf,
                                                           const float2* __restrict__ ebc, int k, int n_win) {
  const int w = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int m = warp; m < k; m += blockDim.x / 32) {
    const float2* q = Qf + ((size_t)m * n_win + w) * 320;
    const float2* e = ebc + (size_t)w * 320;
    float sr = 0.f, si = 0.f;
    for (int t = lane; t < 320; t += 32) {
      const float2 a = q[t], b = e[t];
      sr += a.x * b.x + a.y * b.y;
      si += a.x * b.y - a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) r[(size_t)w * k + m] = make_float2(-sr, -si);
  }
}

// Row temporary of the sweeps (warp per entry (a, p) of window row b):
//   forward  (jbase = 0): t = r_b - L_b y_{b-1}   (x = y of row b-1)
//   backward (jbase = 6): t = U_b z_{b+1}          (x = z of row b+1, r = NULL)
__global__ void __launch_bounds__(256) sweep_t_kernel(float2* __restrict__ t, const float2* __restrict__ r,
                                                      const float2* __restrict__ x, const float2* __restrict__ Gf,
                                                      int k, int nwx, int b, int jbase) {
  const int D = nwx * k;
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= D) return;
  const int a = row / k, p = row % k;
  float sr = 0.f, si = 0.f;
  for (int a3 = max(a - 1, 0); a3 <= min(a + 1, nwx - 1); ++a3) {
    const float2* g = Gf + (((size_t)(b * nwx + a) * 9 + jbase + 1 + (a3 - a)) * k + p) * k;
    const float2* xv = x + (size_t)a3 * k;
    for (int p3 = lane; p3 < k; p3 += 32) {
      const float2 v = cmul(g[p3], xv[p3]);
      sr += v.x; si += v.y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) t[row] = r ? make_float2(r[row].x - sr, r[row].y - si) : make_float2(sr, si);
}

// out = base + sgn * A t for a row-major D x D complex matrix A stored as
// complex half: each row is split over GW warps (GEMV_ROWS rows per CTA, so
// enough loads are in flight to stream A at HBM rate), four complex entries
// per 16-byte load, FP32 products and sums; base may be NULL.  Four warps per
// row: alone (back-to-back GEMVs) two warps per row streamed a 4096 x 4096
// block 6% faster, but inside the sweeps, between the coupling kernels, they
// made the coarse solve 11% slower; eight warps per row or a persistent grid
// were slower in both.
constexpr int GW = 4, GEMV_ROWS = 8 / GW;
__global__ void __launch_bounds__(256) gemv_rows_kernel(float2* __restrict__ out, const float2* __restrict__ base,
                                                        const __half2* __restrict__ A, const float2* __restrict__ t,
                                                        int D, float sgn) {
  __shared__ float2 red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * GEMV_ROWS + warp / GW, part = warp % GW;
  float sr = 0.f, si = 0.f;
  if (row < D) {
    const __half2* a = A + (size_t)row * D;
    const uint4* a4 = reinterpret_cast<const uint4*>(a);
    const float4* t4 = reinterpret_cast<const float4*>(t);
    // 16-byte loads need every row 16-byte aligned (D a multiple of 4);
    // otherwise the scalar loop below takes the whole row
    const int n4 = (D & 3) ? 0 : D / 4;
#pragma unroll 4
    for (int j = part * 32 + lane; j < n4; j += 32 * GW) {
      const uint4 m = __ldcs(a4 + j);
      const float4 v0 = __ldg(t4 + 2 * j), v1 = __ldg(t4 + 2 * j + 1);
      const float2 m0 = __half22float2(*reinterpret_cast<const __half2*>(&m.x));
      const float2 m1 = __half22float2(*reinterpret_cast<const __half2*>(&m.y));
      const float2 m2 = __half22float2(*reinterpret_cast<const __half2*>(&m.z));
      const float2 m3 = __half22float2(*reinterpret_cast<const __half2*>(&m.w));
      sr += m0.x * v0.x - m0.y * v0.y + m1.x * v0.z - m1.y * v0.w + m2.x * v1.x - m2.y * v1.y + m3.x * v1.z - m3.y * v1.w;
      si += m0.x * v0.y + m0.y * v0.x + m1.x * v0.w + m1.y * v0.z + m2.x * v1.y + m2.y * v1.x + m3.x * v1.w + m3.y * v1.z;
    }
    for (int j = 4 * n4 + part * 32 + lane; j < D; j += 32 * GW) {  // D not a multiple of 4
      const float2 m = __half22float2(a[j]), v = t[j];
      sr += m.x * v.x - m.y * v.y;
      si += m.x * v.y + m.y * v.x;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) red[warp] = make_float2(sr, si);
  __syncthreads();
  if (part == 0 && lane == 0 && row < D) {
    float2 acc = red[warp];
    for (int q = 1; q < GW; ++q) acc = make_float2(acc.x + red[warp + q].x, acc.y + red[warp + q].y);
    const float2 b0 = base ? base[row] : make_float2(0.f, 0.f);
    out[row] = make_float2(b0.x + sgn * acc.x, b0.y + sgn * acc.y);
  }
}

__global__ void to_half_kernel(__half2* dst, const float2* src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __floats2half2_rn(src[i].x, src[i].y);
}

__global__ void nonfinite_half_kernel(const __half2* __restrict__ a, size_t n, int* flag) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 v = __half22float2(a[e]);
    if (!isfinite(v.x) || !isfinite(v.y)) { atomicExch(flag, 1); return; }
  }
}

// H[w][p][q] = sum over w's interface sides s of conj(Q_w[p][s]) . Y_w[q][s],
// Y_w[q][s] = the trace basis field (w, q) leaves on the neighbour across s,
// on its side facing w: C block (neighbour i, j = w's offset from i).
__global__ void ritz_H_kernel(const double2* __restrict__ Q, const double2* __restrict__ C, double2* __restrict__ H,
                              int k, int nx, int ny, int nwx) {
  const int w = blockIdx.x;
  const Win W = win_of(w, nx, ny, nwx);
  // side s: neighbour offset (di), block index of w seen from it (j), its facing side (f)
  const int di[4] = {-1, 1, -nwx, nwx}, jb[4] = {5, 3, 7, 1}, fs[4] = {1, 0, 3, 2};
  for (int pq = threadIdx.x; pq < k * k; pq += blockDim.x) {
    const int p = pq / k, q = pq % k;
    double sr = 0.0, si = 0.0;
    for (int sd = 0; sd < 4; ++sd) {
      if (!W.iface[sd]) continue;
      const int i = w + di[sd];
      const double2* qp = Q + ((size_t)w * k + p) * 320 + sd * 80;
      const double2* cy = C + (((size_t)i * 9 + jb[sd]) * 320 + fs[sd] * 80) * k + q;
      for (int t = 0; t < 80; ++t) {  // conj(q) . y
        const double2 a = qp[t], b = cy[(size_t)t * k];
        sr += a.x * b.x + a.y * b.y;
        si += a.x * b.y - a.y * b.x;
      }
    }
    H[((size_t)w * k + p) * k + q] = make_double2(sr, si);
  }
}

// Eigenpairs of each window's Ritz matrix (one thread per window); the
// eigenvectors with |eta| < tol become zero columns of U.
__global__ void ritz_eig_kernel(double2* H, double2* Z, double2* U, double2* eta, int k, int n_win, double tol,
                                int* fail) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_win) return;
  const size_t o = (size_t)w * k * k;
  ecd* e = reinterpret_cast<ecd*>(eta + (size_t)w * k);
  ecd* u = reinterpret_cast<ecd*>(U + o);
  if (!eig_small(reinterpret_cast<ecd*>(H + o), reinterpret_cast<ecd*>(Z + o), e, u, k)) atomicExch(fail, 1);
  for (int q = 0; q < k; ++q)
    if (e_abs(e[q]) < tol)
      for (int m = 0; m < k; ++m) u[m * k + q] = {0.0, 0.0};
}

// out[w][q][e] = sum_m in[w][m][e] U[w][m][q]  (Q: L = 320, Phi: L = 4096)
template <typename T>
__global__ void ritz_rotate_kernel(const T* __restrict__ in, T* __restrict__ out, const double2* __restrict__ U,
                                   int k, int L) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x, w = blockIdx.y;
  if (e >= L) return;
  const double2* Uw = U + (size_t)w * k * k;
  for (int q = 0; q < k; ++q) {
    double sr = 0.0, si = 0.0;
    for (int m = 0; m < k; ++m) {
      const T x = in[((size_t)w * k + m) * L + e];
      const double2 c = Uw[m * k + q];
      sr += (double)x.x * c.x - (double)x.y * c.y;
      si += (double)x.x * c.y + (double)x.y * c.x;
    }
    T r;
    r.x = sr; r.y = si;
    out[((size_t)w * k + q) * L + e] = r;
  }
}

// C rows of window i, block j (columns of window J = i + offset j): the
// k-vector of each slot times U_J.
__global__ void ritz_rotate_C_kernel(const double2* __restrict__ C, double2* __restrict__ out,
                                     const double2* __restrict__ U, int k, int nwx, int nwy) {
  const int ij = blockIdx.x, i = ij / 9, j = ij % 9;
  const int aJ = i % nwx + j % 3 - 1, bJ = i / nwx + j / 3 - 1;
  const bool hasJ = aJ >= 0 && aJ < nwx && bJ >= 0 && bJ < nwy;
  const double2* UJ = U + (size_t)(hasJ ? bJ * nwx + aJ : 0) * k * k;
  for (int slot = threadIdx.x; slot < 320; slot += blockDim.x) {
    const double2* x = C + ((size_t)ij * 320 + slot) * k;
    double2* y = out + ((size_t)ij * 320 + slot) * k;
    for (int q = 0; q < k; ++q) {
      double sr = 0.0, si = 0.0;
      if (hasJ)
        for (int m = 0; m < k; ++m) {
          const double2 a = x[m], c = UJ[m * k + q];
          sr += a.x * c.x - a.y * c.y;
          si += a.x * c.y + a.y * c.x;
        }
      y[q] = make_double2(sr, si);
    }
  }
}

__global__ void sub_kernel(float2* a, const float2* b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = make_float2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void to_f32_kernel(float2* dst, const double2* src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

// u[core(w)] += sum_m z[w,m] Phi[w][m]
__global__ void correction_kernel(float2* u, const __half2* Phi, const float2* z, int k, int nx, int nwx) {
  const int w = blockIdx.y;
  const int a = w % nwx, b = w / nwx;
  __shared__ float2 zw[256];
  for (int m = threadIdx.x; m < k; m += blockDim.x) zw[m] = z[w * k + m];
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= 4096) return;
  const __half2* ph = Phi + (size_t)w * k * 4096 + p;
  float2 acc = make_float2(0.f, 0.f);
  for (int m = 0; m < k; ++m) acc = cadd(acc, cmul(zw[m], __half22float2(__ldcs(ph + (size_t)m * 4096))));
  const size_t g = (size_t)(FDFD_CORE * b + p / 64) * nx + FDFD_CORE * a + p % 64;
  u[g] = cadd(u[g], acc);
}

template <class T>
int ca(T** p, size_t n, size_t* bytes) {
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) return FDFD_ENOMEM;
  *bytes += n * sizeof(T);
  return FDFD_OK;
}

}  // namespace

void coarse_free(CoarseData* c) {
  if (!c) return;
  void* ptrs[] = {c->Q, c->Qf, c->Phi, c->Phih, c->C, c->G, c->Gf, c->Sinv, c->rcf, c->ycf, c->zcf, c->tcf, c->ebc,
                  c->tmp, c->dropped, c->eta, c->H};
  for (void* p : ptrs) if (p) cudaFree(p);
  delete c;
}

// The Rayleigh-Ritz truncation of a set-up whose C is assembled: Q, Phi
// and C are replaced by their combinations with the kept eigenvectors.
static int ritz_truncate(fdfd_ctx* h, CoarseData* c, double tol, size_t* bytes) {
  const int nwx = h->nx / FDFD_CORE, nwy = h->ny / FDFD_CORE, n_win = nwx * nwy, k = c->k, nc = c->nc;
  cudaStream_t s = h->stream;
  double2 *H = nullptr, *Z = nullptr, *U = nullptr, *Q2 = nullptr, *C2 = nullptr;
  float2* P2 = nullptr;
  int* fail = nullptr;
  size_t tb = 0;  // temporaries, released before returning
  int rc = FDFD_OK, f = 0;
  if ((rc = ca(&c->eta, (size_t)n_win * k, bytes)) || (rc = ca(&c->H, (size_t)n_win * k * k, bytes)) ||
      (rc = ca(&H, (size_t)n_win * k * k, &tb)) ||
      (rc = ca(&Z, (size_t)n_win * k * k, &tb)) || (rc = ca(&U, (size_t)n_win * k * k, &tb)) ||
      (rc = ca(&Q2, (size_t)nc * 320, &tb)) || (rc = ca(&P2, (size_t)nc * 4096, &tb)) ||
      (rc = ca(&C2, (size_t)n_win * 9 * 320 * k, &tb)) || (rc = ca(&fail, 1, &tb)))
    goto done;
  ritz_H_kernel<<<n_win, 256, 0, s>>>(c->Q, c->C, H, k, h->nx, h->ny, nwx);
  if (cudaMemcpyAsync(c->H, H, (size_t)n_win * k * k * sizeof(double2), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    rc = FDFD_ECUDA;
    goto done;
  }
  ritz_eig_kernel<<<(n_win + 31) / 32, 32, 0, s>>>(H, Z, U, c->eta, k, n_win, tol, fail);
  ritz_rotate_kernel<double2><<<dim3((320 + 255) / 256, n_win), 256, 0, s>>>(c->Q, Q2, U, k, 320);
  ritz_rotate_kernel<float2><<<dim3(4096 / 256, n_win), 256, 0, s>>>(c->Phi, P2, U, k, 4096);
  ritz_rotate_C_kernel<<<n_win * 9, 256, 0, s>>>(c->C, C2, U, k, nwx, nwy);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&f, fail, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = FDFD_ECUDA;
    goto done;
  }
  if (f) { rc = FDFD_ENUMERIC; goto done; }  // a QR iteration did not converge
  { double2* t = c->Q; c->Q = Q2; Q2 = t; }
  { float2* t = c->Phi; c->Phi = P2; P2 = t; }
  { double2* t = c->C; c->C = C2; C2 = t; }
done:
  cudaStreamSynchronize(s);
  void* tmp[] = {H, Z, U, Q2, P2, C2, fail};
  for (void* p : tmp) if (p) cudaFree(p);
  return rc;
}


// Block elimination over the window rows of G: S_b^-1 for every row b
// (row-major, FP32).  cuSOLVER sees each row-major S as its transpose, so
// getrf/getrs with the identity as right-hand side return inv(S^T) in
// column-major order, which is inv(S) in row-major order.
static int factor_rows(fdfd_ctx* h, CoarseData* c) {
  const int k = c->k, nwx = c->nwx, nwy = c->nwy, D = c->D;
  cudaStream_t s = h->stream;
  float2 *S = nullptr, *T = nullptr, *X = nullptr;  // X: this row's inverse in FP32 (the next update reads it)
  int *ipiv = nullptr, *info = nullptr;
  cuComplex* work = nullptr;
  cusolverDnHandle_t sh = nullptr;
  size_t tb = 0;
  int rc = FDFD_OK, lwork = 0;
  std::vector<int> hinfo(2 * nwy + 1, 0);  // getrf / getrs info per row, then the FP32 non-finite flag
  const size_t DD = (size_t)D * D;
  const dim3 tile((D + 255) / 256, (D + RT - 1) / RT);
  if ((rc = ca(&S, DD, &tb)) || (rc = ca(&T, DD, &tb)) || (rc = ca(&X, DD, &tb)) || (rc = ca(&ipiv, (size_t)D, &tb)) ||
      (rc = ca(&info, (size_t)2 * nwy + 1, &tb)))
    goto done;
  if (cusolverDnCreate(&sh) != CUSOLVER_STATUS_SUCCESS || cusolverDnSetStream(sh, s) != CUSOLVER_STATUS_SUCCESS ||
      cusolverDnCgetrf_bufferSize(sh, D, D, reinterpret_cast<cuComplex*>(S), D, &lwork) != CUSOLVER_STATUS_SUCCESS) {
    rc = FDFD_ECUDA;
    goto done;
  }
  if ((rc = ca(&work, (size_t)(lwork > 0 ? lwork : 1), &tb))) goto done;
  if (cudaMemsetAsync(info + 2 * nwy, 0, sizeof(int), s) != cudaSuccess) { rc = FDFD_ECUDA; goto done; }
  for (int b = 0; b < nwy; ++b) {
    build_S_kernel<<<2048, 256, 0, s>>>(S, c->Gf, k, nwx, b);
    if (b > 0) {  // X holds S_{b-1}^-1 in FP32
      schur_T_kernel<<<tile, 256, 0, s>>>(T, X, c->Gf, k, nwx, b);
      schur_update_kernel<<<tile, 256, 0, s>>>(S, T, c->Gf, k, nwx, b);
    }
    identity_kernel<<<2048, 256, 0, s>>>(X, D);
    if (cudaGetLastError() != cudaSuccess ||
        cusolverDnCgetrf(sh, D, D, reinterpret_cast<cuComplex*>(S), D, work, ipiv, info + 2 * b) !=
            CUSOLVER_STATUS_SUCCESS ||
        cusolverDnCgetrs(sh, CUBLAS_OP_N, D, D, reinterpret_cast<const cuComplex*>(S), D, ipiv,
                         reinterpret_cast<cuComplex*>(X), D, info + 2 * b + 1) != CUSOLVER_STATUS_SUCCESS) {
      rc = FDFD_ECUDA;
      goto done;
    }
    // a Schur complement that is numerically singular leaves non-finite or
    // overflowing entries in its inverse; flag them instead of solving with them
    nonfinite_kernel<<<1024, 256, 0, s>>>(X, DD, info + 2 * nwy);
    to_half_kernel<<<2048, 256, 0, s>>>(c->Sinv + (size_t)b * DD, X, DD);  // the stored copy the sweeps read
  }
  if (cudaMemsetAsync(ipiv, 0, sizeof(int), s) != cudaSuccess) { rc = FDFD_ECUDA; goto done; }
  nonfinite_half_kernel<<<4096, 256, 0, s>>>(c->Sinv, (size_t)nwy * DD, ipiv);  // beyond the half range
  nonfinite_kernel<<<1024, 256, 0, s>>>(c->Gf, (size_t)nwx * nwy * 9 * k * k, ipiv);
  if (cudaMemcpyAsync(hinfo.data(), ipiv, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = FDFD_ECUDA;
    goto done;
  }
  if (hinfo[0]) { rc = FDFD_ENUMERIC; goto done; }
  if (cudaMemcpyAsync(hinfo.data(), info, hinfo.size() * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    rc = FDFD_ECUDA;
    goto done;
  }
  for (int v : hinfo)
    if (v != 0) rc = FDFD_ENUMERIC;  // a singular Schur complement (or a bad argument)
done:
  cudaStreamSynchronize(s);
  if (sh) cusolverDnDestroy(sh);
  void* tmp[] = {S, T, X, ipiv, info, work};
  for (void* p : tmp) if (p) cudaFree(p);
  return rc;
}

int coarse_setup(fdfd_ctx* h, const NnoWeights* W, NnoWork* work, LocalWork* L, int k, double ritz_tol,
                 CoarseData** out, size_t* bytes) {
  const int nwx = h->nx / FDFD_CORE, nwy = h->ny / FDFD_CORE, n_win = nwx * nwy;
  const int nc = n_win * k;
  if (k < 1 || k > 256) return FDFD_EINVAL;
  if (!(ritz_tol >= 0.0) || (ritz_tol > 0.0 && k > EIG_KMAX)) return FDFD_EINVAL;
  CoarseData* c = new CoarseData();
  c->k = k; c->nc = nc; c->nwx = nwx; c->nwy = nwy; c->D = nwx * k;
  const size_t DD = (size_t)c->D * c->D;
  const size_t c_bytes = (size_t)n_win * 9 * 320 * k * sizeof(double2);
  int rc;
  if ((rc = ca(&c->Q, (size_t)nc * 320, bytes)) || (rc = ca(&c->Qf, (size_t)nc * 320, bytes)) ||
      (rc = ca(&c->Phi, (size_t)nc * 4096, bytes)) || (rc = ca(&c->C, (size_t)n_win * 9 * 320 * k, bytes)) ||
      (rc = ca(&c->G, (size_t)n_win * 9 * k * k, bytes)) || (rc = ca(&c->Gf, (size_t)n_win * 9 * k * k, bytes)) ||
      (rc = ca(&c->Sinv, (size_t)nwy * DD, bytes)) || (rc = ca(&c->rcf, (size_t)nc, bytes)) ||
      (rc = ca(&c->ycf, (size_t)nc, bytes)) || (rc = ca(&c->zcf, (size_t)nc, bytes)) ||
      (rc = ca(&c->tcf, (size_t)c->D, bytes)) || (rc = ca(&c->ebc, (size_t)n_win * 320, bytes)) ||
      (rc = ca(&c->tmp, (size_t)n_win * 6400, bytes)) || (rc = ca(&c->dropped, (size_t)nc, bytes))) {
    coarse_free(c);
    return rc;
  }
  cudaStream_t s = h->stream;
  trials_gs_kernel<<<n_win, 256, 0, s>>>(c->Q, c->Qf, k, h->eps, h->k0dx, h->nx, h->ny, nwx, n_win);
  CKL();
  GridGeom g{h->nx, h->ny, nwx, (float)h->k2, h->eps, h->isx, h->isy, schwarz_modulation(h)};
  float2* rhs = nullptr;
  if (L && (rc = ca(&rhs, (size_t)n_win * 6400, bytes))) { coarse_free(c); return rc; }
  for (int m = 0; m < k; ++m) {
    const float2* qm = c->Qf + (size_t)m * n_win * 320;
    if (L) {  // homogeneous Robin problem solved by the local NN-FGMRES
      if ((rc = local_robin_rhs(h, qm, rhs, n_win)) ||
          (rc = local_fgmres(h, L, W, work, nullptr, rhs, nullptr, c->tmp, nullptr))) {
        cudaFree(rhs); coarse_free(c); return rc;
      }
    } else {  // one neural application with the Robin data as input
      NnoInput in;
      in.g_win = qm;
      NnoOutput o;
      o.e_win = c->tmp;
      if ((rc = nno_forward(W, work, g, in, o, n_win, s))) { cudaFree(rhs); coarse_free(c); return rc; }
    }
    copy_core_kernel<<<n_win, 256, 0, s>>>(c->tmp, c->Phi, m, k, h->nx, h->ny, nwx, n_win);
    CKL();
  }
  if (rhs) { cudaStreamSynchronize(s); cudaFree(rhs); *bytes -= (size_t)n_win * 6400 * sizeof(float2); }
  assemble_C_kernel<<<dim3(n_win, 9), 256, 0, s>>>(c->C, c->Q, c->Phi, k, h->eps, h->k0dx, h->nx, h->ny, nwx, nwy);
  CKL();
  if (ritz_tol > 0.0) {
    if ((rc = ritz_truncate(h, c, ritz_tol, bytes))) { coarse_free(c); return rc; }
    q_to_f32_kernel<<<n_win, 256, 0, s>>>(c->Qf, c->Q, k, n_win);  // rotated test functions
    CKL();
  }
  assemble_G_kernel<<<dim3(n_win, 9), 256, 0, s>>>(c->G, c->Q, c->C, k);
  to_f32_kernel<<<1024, 256, 0, s>>>(c->Gf, c->G, (size_t)n_win * 9 * k * k);
  dropped_kernel<<<(nc + 255) / 256, 256, 0, s>>>(c->dropped, c->Q, nc);
  CKL();
  // C and the FP32 basis fields are set-up temporaries: the Galerkin blocks
  // and a complex-half copy of the fields replace them
  if ((rc = ca(&c->Phih, (size_t)nc * 4096, bytes))) { coarse_free(c); return rc; }
  to_half_kernel<<<2048, 256, 0, s>>>(c->Phih, c->Phi, (size_t)nc * 4096);
  CKL();
  cudaStreamSynchronize(s);
  cudaFree(c->C);
  c->C = nullptr;
  cudaFree(c->Phi);
  c->Phi = nullptr;
  *bytes -= c_bytes + (size_t)nc * 4096 * sizeof(float2);
  if ((rc = factor_rows(h, c))) { coarse_free(c); return rc; }
  {
    std::vector<int> dr(nc);
    if (cudaMemcpyAsync(dr.data(), c->dropped, (size_t)nc * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      coarse_free(c);
      return FDFD_ECUDA;
    }
    c->n_kept = 0;
    for (int d : dr) c->n_kept += d ? 0 : 1;
  }
  *out = c;
  return FDFD_OK;
}

int coarse_kept(CoarseData* c) { return c ? c->n_kept : 0; }

int coarse_ritz_export(fdfd_ctx* h, CoarseData* c, double* eta_host, double* H_host) {
  if (!c->eta) return FDFD_ENOSETUP;
  const size_t n = (size_t)(h->nx / FDFD_CORE) * (h->ny / FDFD_CORE) * c->k;
  if (eta_host) CK(cudaMemcpy(eta_host, c->eta, n * sizeof(double2), cudaMemcpyDeviceToHost));
  if (H_host) CK(cudaMemcpy(H_host, c->H, n * c->k * sizeof(double2), cudaMemcpyDeviceToHost));
  return FDFD_OK;
}

// Kernel launches of one coarse solve (right-hand side, both sweeps).
static int solve_launches(const CoarseData* c) { return 1 + (2 * c->nwy - 1) + 2 * (c->nwy - 1); }

// z = G^-1 r (rcf -> zcf): forward then backward sweep over the window rows.
static int solve_rows(fdfd_ctx* h, CoarseData* c) {
  const int D = c->D, k = c->k, nwx = c->nwx, nwy = c->nwy;
  const size_t DD = (size_t)D * D;
  const int grid = (D + 7) / 8, ggrid = (D + GEMV_ROWS - 1) / GEMV_ROWS;
  cudaStream_t s = h->stream;
  for (int b = 0; b < nwy; ++b) {
    const float2* t = c->rcf + (size_t)b * D;
    if (b > 0) {
      sweep_t_kernel<<<grid, 256, 0, s>>>(c->tcf, c->rcf + (size_t)b * D, c->ycf + (size_t)(b - 1) * D, c->Gf, k,
                                          nwx, b, 0);
      t = c->tcf;
    }
    gemv_rows_kernel<<<ggrid, 256, 0, s>>>(c->ycf + (size_t)b * D, nullptr, c->Sinv + (size_t)b * DD, t, D, 1.f);
  }
  CK(cudaMemcpyAsync(c->zcf + (size_t)(nwy - 1) * D, c->ycf + (size_t)(nwy - 1) * D, (size_t)D * sizeof(float2),
                     cudaMemcpyDeviceToDevice, s));
  for (int b = nwy - 2; b >= 0; --b) {
    sweep_t_kernel<<<grid, 256, 0, s>>>(c->tcf, nullptr, c->zcf + (size_t)(b + 1) * D, c->Gf, k, nwx, b, 6);
    gemv_rows_kernel<<<ggrid, 256, 0, s>>>(c->zcf + (size_t)b * D, c->ycf + (size_t)b * D, c->Sinv + (size_t)b * DD,
                                          c->tcf, D, -1.f);
  }
  CKL();
  return FDFD_OK;
}

int coarse_apply(fdfd_ctx* h, CoarseData* c, float2* u, const float2* g_ref) {
  const int nwx = c->nwx, n_win = c->nwx * c->nwy;
  cudaStream_t s = h->stream;
  int rc;
  {
    ProfScope ps(h, 6, g_ref ? 2 : 1);
    if ((rc = schwarz_traces(h, u, c->ebc))) return rc;
    if (g_ref) {  // boundary mismatch against the Robin data the local solves used
      const int tot = n_win * 320;
      sub_kernel<<<(tot + 255) / 256, 256, 0, s>>>(c->ebc, g_ref, tot);
      CKL();
    }
  }
  ProfScope ps(h, 7, solve_launches(c) + 1);
  galerkin_rhs_kernel<<<n_win, 256, 0, s>>>(c->rcf, c->Qf, c->ebc, c->k, n_win);
  CKL();
  if ((rc = solve_rows(h, c))) return rc;
  correction_kernel<<<dim3(4096 / 256, n_win), 256, 0, s>>>(u, c->Phih, c->zcf, c->k, h->nx, nwx);
  CKL();
  return FDFD_OK;
}

int coarse_solve_mismatch(fdfd_ctx* h, CoarseData* c, const float2* ebc, float2* z) {
  const int n_win = c->nwx * c->nwy;
  cudaStream_t s = h->stream;
  galerkin_rhs_kernel<<<n_win, 256, 0, s>>>(c->rcf, c->Qf, ebc, c->k, n_win);
  CKL();
  int rc;
  if ((rc = solve_rows(h, c))) return rc;
  CK(cudaMemcpyAsync(z, c->zcf, (size_t)c->nc * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return FDFD_OK;
}

int coarse_export(fdfd_ctx* h, CoarseData* c, double* Qh, double* Gh) {
  const int n_win = c->nwx * c->nwy;
  (void)h;
  if (Qh) CK(cudaMemcpy(Qh, c->Q, (size_t)c->nc * 320 * sizeof(double2), cudaMemcpyDeviceToHost));
  if (Gh) CK(cudaMemcpy(Gh, c->G, (size_t)n_win * 9 * c->k * c->k * sizeof(double2), cudaMemcpyDeviceToHost));
  return FDFD_OK;
}
