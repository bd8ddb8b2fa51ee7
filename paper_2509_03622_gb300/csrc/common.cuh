// Internal declarations shared by the CUDA translation units of libfdfd.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include "../../include/fdfd.h"

#define FDFD_WIN 80
#define FDFD_CORE 64
#define FDFD_OVL 8
#define FDFD_MAXRESTART 64
#define FDFD_CH 32      // neural-operator width
#define FDFD_CIN 15     // input channels
#define FDFD_HID 128    // projection hidden width
#define FDFD_MY 32      // retained ky modes
#define FDFD_MX 16      // retained kx modes
#define FDFD_NMODE (FDFD_MY * FDFD_MX)

#define CK(call)                                                               \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      fprintf(stderr, "libfdfd: %s failed: %s (%s:%d)\n", #call,               \
              cudaGetErrorString(e_), __FILE__, __LINE__);                     \
      return FDFD_ECUDA;                                                       \
    }                                                                          \
  } while (0)

#define CKL()                                                                  \
  do {                                                                         \
    cudaError_t e_ = cudaGetLastError();                                       \
    if (e_ != cudaSuccess) {                                                   \
      fprintf(stderr, "libfdfd: launch failed: %s (%s:%d)\n",                  \
              cudaGetErrorString(e_), __FILE__, __LINE__);                     \
      return FDFD_ECUDA;                                                       \
    }                                                                          \
  } while (0)

// Per-axis 5-point coefficients: lo multiplies x_{i-1}, hi multiplies
// x_{i+1}, dg is the axis' share of the diagonal.
struct AxisCoef { float2 lo, hi, dg; };
struct AxisCoef64 { double2 lo, hi, dg; };

// Device-side state of one FGMRES solve (FP64 scalars).
struct KrylovState {
  double2 H[(FDFD_MAXRESTART + 1) * FDFD_MAXRESTART];  // column-major, ld = restart+1
  double cs[FDFD_MAXRESTART];
  double2 sn[FDFD_MAXRESTART];
  double2 g[FDFD_MAXRESTART + 1];
  double2 y[FDFD_MAXRESTART];
  double2 h[FDFD_MAXRESTART + 1];        // current column (dots)
  double vscale[FDFD_MAXRESTART + 1];    // stored v_i = vscale_i^-1 * true v_i
  double beta;                           // ||r0|| of the cycle
  double bnorm;                          // ||b||
  double resid;                          // FP64 scratch norm result
  double est;                            // |g_{j+1}| / ||b||
  int    nonfinite;                      // NaN/Inf seen
  int    breakdown;                      // h_{j+1,j} == 0
};

// ---- complex helpers --------------------------------------------------
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// ---- kernels/launchers implemented in the .cu files --------------------
// stencil.cu
int launch_stencil(const float2* x, float2* y, const float* eps, const AxisCoef* cx,
                   const AxisCoef* cy, float k2, int nx, int ny, cudaStream_t s);
int launch_stencil_jacobi(const float2* v, const double* vscale_dev, float2* w, const float* eps,
                          const AxisCoef* cx, const AxisCoef* cy, float k2, int nx, int ny,
                          cudaStream_t s);
int launch_residual64(const double2* x, const float2* J, double sb, int rhs_is_source, double rs,
                      const float* eps, const AxisCoef64* cx, const AxisCoef64* cy, double k2,
                      int nx, int ny, float2* r_out, double* partials, unsigned* counter,
                      double* result, cudaStream_t s);
int launch_grad_eps(const float2* E, const float2* lam, float* grad, float k2, int n,
                    int accumulate, cudaStream_t s);
// out = in * D^-1 (inverse = 1) or in * D (inverse = 0), D = s_x s_y at cell centres
// (isx, isy hold 1/s); in and out may alias.
int launch_scale_d(const float2* in, float2* out, const float2* isx, const float2* isy, int nx, size_t n,
                   int inverse, cudaStream_t s);
// krylov.cu
int krylov_grid(size_t n);
int launch_cgs_dots(const float2* V, size_t ld, int j, const float2* w, size_t n,
                    KrylovState* st, double* partials, unsigned* counter, cudaStream_t s);
int launch_cgs_update(const float2* V, size_t ld, int j, float2* w_inout, float2* vnext, size_t n,
                      KrylovState* st, double* partials, unsigned* counter, int restart,
                      cudaStream_t s);
int launch_cycle_start(KrylovState* st, cudaStream_t s);
int launch_solve_y(KrylovState* st, int k, int restart, cudaStream_t s);
int launch_x_update(double2* x, const float2* Z, size_t ld, int k, size_t n, const KrylovState* st,
                    cudaStream_t s);
int launch_x_update_jacobi(double2* x, const float2* V, size_t ld, int k, size_t n,
                           const KrylovState* st, const float* eps, const AxisCoef* cx,
                           const AxisCoef* cy, float k2, int nx, cudaStream_t s);
// E = f x (complex128 -> complex64) and x = f E
int launch_store_field(const double2* x, float2* E, size_t n, double f, cudaStream_t s);
int launch_load_field(const float2* E, double2* x, size_t n, double f, cudaStream_t s);
int launch_scale_copy(const float2* v, const double* scale_dev, float2* z, size_t n, cudaStream_t s);
int launch_jacobi_apply(const float2* v, const double* scale_dev, float2* z, const float* eps,
                        const AxisCoef* cx, const AxisCoef* cy, float k2, int nx, int ny,
                        cudaStream_t s);
