// Eigenpairs of one small dense complex matrix (k <= EIG_KMAX), FP64, by
// one thread: Householder reduction to upper Hessenberg form, the shifted
// QR iteration (Wilkinson shifts, deflation on negligible subdiagonals) to
// the complex Schur form T = Z^H A Z, and the eigenvectors of T by back
// substitution, mapped back by Z (Golub & Van Loan, Matrix Computations,
// Sec. 7.4-7.6).  Used for the Rayleigh-Ritz step of the coarse-space
// set-up (Algorithm 3: eta, u = eig(H)), one matrix per window.  Plain C++
// with host/device qualifiers, so the same code can run on either side.
#pragma once
#include <math.h>

#ifdef __CUDACC__
#define EIG_HD __host__ __device__ __forceinline__
#else
#define EIG_HD inline
#endif

constexpr int EIG_KMAX = 64;

struct ecd { double r, i; };
EIG_HD ecd e_add(ecd a, ecd b) { return {a.r + b.r, a.i + b.i}; }
EIG_HD ecd e_sub(ecd a, ecd b) { return {a.r - b.r, a.i - b.i}; }
EIG_HD ecd e_mul(ecd a, ecd b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
EIG_HD ecd e_cmul(ecd a, ecd b) { return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r}; }  // conj(a) b
EIG_HD ecd e_conj(ecd a) { return {a.r, -a.i}; }
EIG_HD ecd e_scale(ecd a, double s) { return {a.r * s, a.i * s}; }
EIG_HD double e_abs(ecd a) { return hypot(a.r, a.i); }
EIG_HD double e_abs1(ecd a) { return fabs(a.r) + fabs(a.i); }
EIG_HD ecd e_div(ecd a, ecd b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
EIG_HD ecd e_sqrt(ecd a) {  // principal square root
  const double m = e_abs(a);
  if (m == 0.0) return {0.0, 0.0};
  const double re = sqrt(0.5 * (m + fabs(a.r))), im = 0.5 * fabs(a.i) / re;
  if (a.r >= 0.0) return {re, a.i >= 0.0 ? im : -im};
  return {im, a.i >= 0.0 ? re : -re};
}

// A: k x k row-major (overwritten by the Schur form T); Z: k x k (out, the
// unitary Schur vectors); eta: k eigenvalues; U: k x k row-major, column q
// the unit eigenvector of eta[q].  Returns false if the QR iteration did
// not converge (30 sweeps per eigenvalue).
EIG_HD bool eig_small(ecd* A, ecd* Z, ecd* eta, ecd* U, int k) {
  if (k < 1 || k > EIG_KMAX) return false;
  auto a = [&](int i, int j) -> ecd& { return A[i * k + j]; };
  auto z = [&](int i, int j) -> ecd& { return Z[i * k + j]; };
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) z(i, j) = {i == j ? 1.0 : 0.0, 0.0};
  ecd v[EIG_KMAX];
  // 1. Hessenberg form: P = I - 2 v v^H / (v^H v) zeroes column j below j + 1
  for (int j = 0; j + 2 < k; ++j) {
    double alpha = 0.0;
    for (int i = j + 1; i < k; ++i) alpha += a(i, j).r * a(i, j).r + a(i, j).i * a(i, j).i;
    alpha = sqrt(alpha);
    if (alpha == 0.0) continue;
    const ecd x0 = a(j + 1, j);
    const double m0 = e_abs(x0);
    const ecd ph = m0 > 0.0 ? e_scale(x0, 1.0 / m0) : ecd{1.0, 0.0};
    double vv = 0.0;
    for (int i = j + 1; i < k; ++i) {
      v[i] = a(i, j);
      if (i == j + 1) v[i] = e_add(v[i], e_scale(ph, alpha));
      vv += v[i].r * v[i].r + v[i].i * v[i].i;
    }
    if (vv == 0.0) continue;
    for (int c = j; c < k; ++c) {  // A <- P A (rows j+1..)
      ecd s = {0.0, 0.0};
      for (int i = j + 1; i < k; ++i) s = e_add(s, e_cmul(v[i], a(i, c)));
      const ecd f = e_scale(s, 2.0 / vv);
      for (int i = j + 1; i < k; ++i) a(i, c) = e_sub(a(i, c), e_mul(f, v[i]));
    }
    for (int r = 0; r < k; ++r) {  // A <- A P, Z <- Z P (columns j+1..)
      ecd s = {0.0, 0.0}, t = {0.0, 0.0};
      for (int i = j + 1; i < k; ++i) { s = e_add(s, e_mul(a(r, i), v[i])); t = e_add(t, e_mul(z(r, i), v[i])); }
      const ecd f = e_scale(s, 2.0 / vv), g = e_scale(t, 2.0 / vv);
      for (int i = j + 1; i < k; ++i) {
        a(r, i) = e_sub(a(r, i), e_mul(f, e_conj(v[i])));
        z(r, i) = e_sub(z(r, i), e_mul(g, e_conj(v[i])));
      }
    }
    for (int i = j + 2; i < k; ++i) a(i, j) = {0.0, 0.0};
  }
  double anorm = 0.0;
  for (int i = 0; i < k * k; ++i) anorm = fmax(anorm, e_abs1(A[i]));
  const double eps = 2.220446049250313e-16;
  // 2. shifted QR on the active block l..hi; rotations applied to the whole
  // matrix and to Z so that T = Z^H A Z stays exact
  double cs[EIG_KMAX];
  ecd sn[EIG_KMAX];
  int hi = k - 1, its = 0, total = 0;
  while (hi > 0) {
    int l = hi;
    for (; l > 0; --l) {
      double s = e_abs1(a(l - 1, l - 1)) + e_abs1(a(l, l));
      if (s == 0.0) s = anorm;
      if (e_abs1(a(l, l - 1)) <= eps * s) { a(l, l - 1) = {0.0, 0.0}; break; }
    }
    if (l == hi) { --hi; its = 0; continue; }
    if (++its > 30 || ++total > 30 * k) return false;
    ecd mu;
    if (its % 10 == 0) {  // exceptional shift
      mu = e_add(a(hi, hi), ecd{0.75 * e_abs1(a(hi, hi - 1)), 0.0});
    } else {  // eigenvalue of the trailing 2 x 2 block nearer to its last diagonal entry
      const ecd p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), d = a(hi, hi);
      const ecd half = e_scale(e_sub(p, d), 0.5);
      const ecd disc = e_sqrt(e_add(e_mul(half, half), e_mul(q, r)));
      const ecd mid = e_scale(e_add(p, d), 0.5);
      const ecd m1 = e_add(mid, disc), m2 = e_sub(mid, disc);
      mu = e_abs(e_sub(m1, d)) <= e_abs(e_sub(m2, d)) ? m1 : m2;
    }
    for (int i = l; i <= hi; ++i) a(i, i) = e_sub(a(i, i), mu);
    for (int i = l; i < hi; ++i) {  // A - mu I = Q R: Givens rotations on rows i, i + 1
      const ecd x = a(i, i), y = a(i + 1, i);
      const double ax = e_abs(x), nr = hypot(ax, e_abs(y));
      double c;
      ecd s;
      if (nr == 0.0) { c = 1.0; s = {0.0, 0.0}; }
      else if (ax == 0.0) { c = 0.0; s = e_scale(e_conj(y), 1.0 / e_abs(y)); }
      else { c = ax / nr; s = e_scale(e_mul(e_scale(x, 1.0 / ax), e_conj(y)), 1.0 / nr); }
      cs[i] = c; sn[i] = s;
      for (int col = i; col < k; ++col) {
        const ecd p = a(i, col), q = a(i + 1, col);
        a(i, col) = e_add(e_scale(p, c), e_mul(s, q));
        a(i + 1, col) = e_sub(e_scale(q, c), e_mul(e_conj(s), p));
      }
    }
    for (int i = l; i < hi; ++i) {  // R Q: the conjugate rotations on columns i, i + 1
      const double c = cs[i];
      const ecd s = sn[i];
      for (int r = 0; r <= i + 1; ++r) {
        const ecd p = a(r, i), q = a(r, i + 1);
        a(r, i) = e_add(e_scale(p, c), e_mul(e_conj(s), q));
        a(r, i + 1) = e_sub(e_scale(q, c), e_mul(s, p));
      }
      for (int r = 0; r < k; ++r) {
        const ecd p = z(r, i), q = z(r, i + 1);
        z(r, i) = e_add(e_scale(p, c), e_mul(e_conj(s), q));
        z(r, i + 1) = e_sub(e_scale(q, c), e_mul(s, p));
      }
    }
    for (int i = l; i <= hi; ++i) a(i, i) = e_add(a(i, i), mu);
  }
  // 3. eigenvectors: T x = t_jj x by back substitution, u = Z x / ||Z x||
  const double small = fmax(anorm, 1e-300) * eps;
  for (int j = 0; j < k; ++j) {
    eta[j] = a(j, j);
    v[j] = {1.0, 0.0};
    for (int i = j - 1; i >= 0; --i) {
      ecd s = {0.0, 0.0};
      for (int m = i + 1; m <= j; ++m) s = e_add(s, e_mul(a(i, m), v[m]));
      ecd den = e_sub(a(i, i), a(j, j));
      if (e_abs1(den) < small) den = {small, 0.0};
      v[i] = e_scale(e_div(s, den), -1.0);
    }
    double nrm = 0.0;
    for (int r = 0; r < k; ++r) {
      ecd s = {0.0, 0.0};
      for (int m = 0; m <= j; ++m) s = e_add(s, e_mul(z(r, m), v[m]));
      U[r * k + j] = s;
      nrm += s.r * s.r + s.i * s.i;
    }
    nrm = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int r = 0; r < k; ++r) U[r * k + j] = e_scale(U[r * k + j], nrm);
  }
  return true;
}
