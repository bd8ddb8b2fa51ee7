// Coarse space of the two-level Schwarz method (Sec. 2.2; Methods,
// Algorithm 3 set-up and correction; Eq. 7-8).
//
// Set-up: pseudo-plane-wave Robin trials walked around each window with
// the local wavenumber, modified Gram-Schmidt in FP64, homogeneous neural
// solves for each trial, the traces of the restricted basis fields on the
// neighbours' boundaries minus the window's own data (C = BQ - Q, stored as
// 9 neighbour blocks per window), the normal matrix C^H C (Eq. 8) and its
// inverse (FP64 Gauss-Jordan; the matrix is Hermitian positive definite).
// Optional Rayleigh-Ritz truncation (Algorithm 3 set-up: eta, u = eig(H);
// Sec. 2.2: the slowly decaying modes above a threshold): per window the
// Ritz matrix H = Q^H Y of the Robin-to-Robin map (Y: the data each basis
// field hands to the neighbours, read on their sides facing the window),
// its eigenpairs (one thread per window, eig.cuh), and Q, Phi and the
// window's columns of C combined by the eigenvectors with |eta| >= ritz_tol;
// the other directions become zero columns, pinned like dependent trials.
// Apply: e_bc = traces of the one-level field, r_c = -C^H e_bc, z = N^-1 r_c,
// u += sum_w R~_w^T sum_m z_{w,m} Phi_{w,m}.
#include <math.h>
#include <vector>
#include "ctx.cuh"
#include "nno.cuh"
#include "local.cuh"
#include "reduce.cuh"
#include "eig.cuh"

struct CoarseData {
  int k = 0, nc = 0;
  double2* Q = nullptr;      // [n_win][k][320]
  float2* Qf = nullptr;      // [k][n_win][320]
  float2* Phi = nullptr;     // [n_win][k][64*64] core of each basis field
  double2* C = nullptr;      // [n_win][9][320][k]
  double2* N = nullptr;      // [nc][nc]  -> inverse after set-up
  double2* Nd = nullptr;     // [n_win][k][k] diagonal blocks of the normal matrix
  double2* rc = nullptr;     // [nc]
  double2* zc = nullptr;     // [nc]
  float2* ebc = nullptr;     // [n_win][320]
  float2* tmp = nullptr;     // [n_win][6400] window fields during set-up
  int* dropped = nullptr;    // [nc]
  double2* eta = nullptr;    // [n_win][k] Ritz values (Ritz step only)
  double2* H = nullptr;      // [n_win][k][k] Ritz matrices (Ritz step only)
  int n_kept = 0;            // unknowns not dropped
  // FP32 copies used by the per-iteration apply (the correction is part of a
  // flexible preconditioner, and FP64 arithmetic is scarce on this GPU)
  float2* Cf = nullptr;      // [n_win][9][320][k]
  float2* Nf = nullptr;      // [nc][nc] inverse normal matrix
  float2* rcf = nullptr;     // [nc]
  float2* zcf = nullptr;     // [nc]
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

// Normal-matrix block (w, w' = w + (ex, ey)): sum over windows i adjacent to both.
__global__ void assemble_N_kernel(double2* N, double2* Nd, const double2* C, int k, int nwx, int nwy) {
  const int w = blockIdx.x, e = blockIdx.y;
  const int ex = e % 5 - 2, ey = e / 5 - 2;
  const int aw = w % nwx, bw = w / nwx, aw2 = aw + ex, bw2 = bw + ey;
  if (aw2 < 0 || aw2 >= nwx || bw2 < 0 || bw2 >= nwy) return;
  const int w2 = bw2 * nwx + aw2;
  const int nc = nwx * nwy * k;
  for (int pq = threadIdx.x; pq < k * k; pq += blockDim.x) {
    const int p = pq / k, q = pq % k;
    double sr = 0.0, si = 0.0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int ai = aw - dx, bi = bw - dy;            // w = i + (dx, dy)
        if (ai < 0 || ai >= nwx || bi < 0 || bi >= nwy) continue;
        const int dx2 = aw2 - ai, dy2 = bw2 - bi;        // w2 = i + (dx2, dy2)
        if (dx2 < -1 || dx2 > 1 || dy2 < -1 || dy2 > 1) continue;
        const int i = bi * nwx + ai;
        const double2* c1 = C + (((size_t)i * 9 + (dy + 1) * 3 + dx + 1) * 320) * k;
        const double2* c2 = C + (((size_t)i * 9 + (dy2 + 1) * 3 + dx2 + 1) * 320) * k;
        for (int sl = 0; sl < 320; ++sl) {
          const double2 a = c1[sl * k + p], b = c2[sl * k + q];  // conj(a) * b
          sr += a.x * b.x + a.y * b.y;
          si += a.x * b.y - a.y * b.x;
        }
      }
    N[(size_t)(w * k + p) * nc + w2 * k + q] = make_double2(sr, si);
    if (w2 == w) Nd[((size_t)w * k + p) * k + q] = make_double2(sr, si);
  }
}

__global__ void dropped_kernel(double2* N, int* dropped, const double2* Q, int nc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double2* q = Q + (size_t)c * 320;
  bool any = false;
  for (int t = 0; t < 320; ++t) any |= (q[t].x != 0.0 || q[t].y != 0.0);
  dropped[c] = !any;
  if (!any) N[(size_t)c * nc + c] = make_double2(1.0, 0.0);
}

// Gauss-Jordan inversion in place (no pivoting; the matrix is HPD).
__global__ void gj_row_kernel(double2* A, int n, int p, double2* prow) {
  const double2 piv = A[(size_t)p * n + p];
  const double den = piv.x * piv.x + piv.y * piv.y;
  const double2 inv = make_double2(piv.x / den, -piv.y / den);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double2 a = (j == p) ? make_double2(1.0, 0.0) : A[(size_t)p * n + j];
    const double2 r = zmul(a, inv);
    A[(size_t)p * n + j] = r;
    prow[j] = r;
  }
}
__global__ void gj_elim_kernel(double2* A, int n, int p, const double2* prow, double2* pcol) {
  // pcol holds column p before elimination (copied by gj_col_kernel)
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i == p) continue;
    const double2 f = pcol[i];
    const double2 a = (j == p) ? make_double2(0.0, 0.0) : A[e];
    A[e] = zsub(a, zmul(f, prow[j]));
  }
}
__global__ void gj_col_kernel(const double2* A, int n, int p, double2* pcol) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pcol[i] = A[(size_t)i * n + p];
}

// r_c[(w,m)] = -sum_{i adjacent to w} sum_slot conj(C[i][j(w)][slot][m]) e_bc[i][slot]
// FP32 apply: r_c[w][m] = -sum C[i][d][sl][m]^H e_bc[i][sl] over the window and
// its 8 neighbours (warp per basis vector m, lanes over the 9 x 320 terms)
__global__ void __launch_bounds__(256) coarse_rhs32_kernel(float2* rc, const float2* C, const float2* ebc, int k,
                                                           int nwx, int nwy) {
  const int w = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int aw = w % nwx, bw = w / nwx;
  for (int m = warp; m < k; m += blockDim.x / 32) {
    float sr = 0.f, si = 0.f;
    for (int t = lane; t < 9 * 320; t += 32) {
      const int d = t / 320, sl = t % 320, dy = d / 3 - 1, dx = d % 3 - 1;
      const int ai = aw - dx, bi = bw - dy;
      if (ai < 0 || ai >= nwx || bi < 0 || bi >= nwy) continue;
      const int i = bi * nwx + ai;
      const float2 a = C[(((size_t)i * 9 + d) * 320 + sl) * k + m];
      const float2 e = ebc[(size_t)i * 320 + sl];
      sr += a.x * e.x + a.y * e.y;
      si += a.x * e.y - a.y * e.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) rc[w * k + m] = make_float2(-sr, -si);
  }
}

// z = Ninv r_c in FP32 (one warp per row)
__global__ void gemv32_kernel(float2* z, const float2* A, const float2* x, const int* dropped, int n) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (row >= n) return;
  float sr = 0.f, si = 0.f;
  const float2* a = A + (size_t)row * n;
  for (int j = lane; j < n; j += 32) {
    if (dropped[j]) continue;
    const float2 p = cmul(a[j], x[j]);
    sr += p.x; si += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) z[row] = dropped[row] ? make_float2(0.f, 0.f) : make_float2(sr, si);
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
__global__ void correction_kernel(float2* u, const float2* Phi, const float2* z, int k, int nx, int nwx) {
  const int w = blockIdx.y;
  const int a = w % nwx, b = w / nwx;
  __shared__ float2 zw[256];
  for (int m = threadIdx.x; m < k; m += blockDim.x) zw[m] = z[w * k + m];
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= 4096) return;
  const float2* ph = Phi + (size_t)w * k * 4096 + p;
  float2 acc = make_float2(0.f, 0.f);
  for (int m = 0; m < k; ++m) acc = cadd(acc, cmul(zw[m], __ldg(ph + (size_t)m * 4096)));
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
  void* ptrs[] = {c->Q, c->Qf, c->Phi, c->C, c->N, c->Nd, c->rc, c->zc, c->ebc, c->tmp, c->dropped,
                  c->Cf, c->Nf, c->rcf, c->zcf, c->eta, c->H};
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

int coarse_setup(fdfd_ctx* h, const NnoWeights* W, NnoWork* work, LocalWork* L, int k, double ritz_tol,
                 CoarseData** out, size_t* bytes) {
  const int nwx = h->nx / FDFD_CORE, nwy = h->ny / FDFD_CORE, n_win = nwx * nwy;
  const int nc = n_win * k;
  if (k < 1 || k > 256 || (size_t)nc * nc * 16 > ((size_t)16 << 30)) return FDFD_EINVAL;
  if (!(ritz_tol >= 0.0) || (ritz_tol > 0.0 && k > EIG_KMAX)) return FDFD_EINVAL;
  CoarseData* c = new CoarseData();
  c->k = k; c->nc = nc;
  int rc;
  if ((rc = ca(&c->Q, (size_t)nc * 320, bytes)) || (rc = ca(&c->Qf, (size_t)nc * 320, bytes)) ||
      (rc = ca(&c->Phi, (size_t)nc * 4096, bytes)) || (rc = ca(&c->C, (size_t)n_win * 9 * 320 * k, bytes)) ||
      (rc = ca(&c->N, (size_t)nc * nc, bytes)) || (rc = ca(&c->Nd, (size_t)n_win * k * k, bytes)) ||
      (rc = ca(&c->rc, (size_t)nc, bytes)) || (rc = ca(&c->zc, (size_t)nc, bytes)) ||
      (rc = ca(&c->ebc, (size_t)n_win * 320, bytes)) || (rc = ca(&c->tmp, (size_t)n_win * 6400, bytes)) ||
      (rc = ca(&c->dropped, (size_t)nc, bytes)) || (rc = ca(&c->Cf, (size_t)n_win * 9 * 320 * k, bytes)) ||
      (rc = ca(&c->Nf, (size_t)nc * nc, bytes)) || (rc = ca(&c->rcf, (size_t)nc, bytes)) ||
      (rc = ca(&c->zcf, (size_t)nc, bytes))) {
    coarse_free(c);
    return rc;
  }
  cudaStream_t s = h->stream;
  trials_gs_kernel<<<n_win, 256, 0, s>>>(c->Q, c->Qf, k, h->eps, h->k0dx, h->nx, h->ny, nwx, n_win);
  CKL();
  GridGeom g{h->nx, h->ny, nwx, (float)h->k2, h->eps, h->isx, h->isy};
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
  if (ritz_tol > 0.0 && (rc = ritz_truncate(h, c, ritz_tol, bytes))) { coarse_free(c); return rc; }
  if (cudaMemsetAsync(c->N, 0, (size_t)nc * nc * sizeof(double2), s) != cudaSuccess) { coarse_free(c); return FDFD_ECUDA; }
  assemble_N_kernel<<<dim3(n_win, 25), 256, 0, s>>>(c->N, c->Nd, c->C, k, nwx, nwy);
  CKL();
  dropped_kernel<<<(nc + 255) / 256, 256, 0, s>>>(c->N, c->dropped, c->Q, nc);
  CKL();
  // Gauss-Jordan inverse (rc, zc reused as the pivot row / column buffers)
  const int gb = 1024;
  for (int p = 0; p < nc; ++p) {
    gj_col_kernel<<<(nc + 255) / 256, 256, 0, s>>>(c->N, nc, p, c->zc);
    gj_row_kernel<<<(nc + 255) / 256, 256, 0, s>>>(c->N, nc, p, c->rc);
    gj_elim_kernel<<<gb, 256, 0, s>>>(c->N, nc, p, c->rc, c->zc);
  }
  to_f32_kernel<<<1024, 256, 0, s>>>(c->Cf, c->C, (size_t)n_win * 9 * 320 * k);
  to_f32_kernel<<<1024, 256, 0, s>>>(c->Nf, c->N, (size_t)nc * nc);
  CKL();
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

int coarse_apply(fdfd_ctx* h, CoarseData* c, float2* u, const float2* g_ref) {
  const int nwx = h->nx / FDFD_CORE, nwy = h->ny / FDFD_CORE, n_win = nwx * nwy;
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
  ProfScope ps(h, 7, 3);
  coarse_rhs32_kernel<<<n_win, 256, 0, s>>>(c->rcf, c->Cf, c->ebc, c->k, nwx, nwy);
  gemv32_kernel<<<(c->nc + 7) / 8, 256, 0, s>>>(c->zcf, c->Nf, c->rcf, c->dropped, c->nc);
  correction_kernel<<<dim3(4096 / 256, n_win), 256, 0, s>>>(u, c->Phi, c->zcf, c->k, h->nx, nwx);
  CKL();
  return FDFD_OK;
}

int coarse_export(fdfd_ctx* h, CoarseData* c, double* Qh, double* Ndh) {
  const int n_win = (h->nx / FDFD_CORE) * (h->ny / FDFD_CORE);
  if (Qh) CK(cudaMemcpy(Qh, c->Q, (size_t)c->nc * 320 * sizeof(double2), cudaMemcpyDeviceToHost));
  if (Ndh) CK(cudaMemcpy(Ndh, c->Nd, (size_t)n_win * c->k * c->k * sizeof(double2), cudaMemcpyDeviceToHost));
  return FDFD_OK;
}
