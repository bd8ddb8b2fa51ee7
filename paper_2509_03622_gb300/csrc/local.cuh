// Batched per-window NN-preconditioned FGMRES (Algorithm 1) for the local
// Robin problems of Algorithm 3; see local.cu.
#pragma once
#include "common.cuh"
#include "nno.cuh"

#define LOCAL_MAXM 16

struct LocalState {
  double2 H[LOCAL_MAXM * (LOCAL_MAXM + 1)];  // rotated Hessenberg, column-major, ld = MAXM+1
  double cs[LOCAL_MAXM];
  double2 sn[LOCAL_MAXM];
  double2 g[LOCAL_MAXM + 1];
  double2 y[LOCAL_MAXM];
  double vscale[LOCAL_MAXM + 1];             // stored v_i = true v_i / vscale_i
  double beta;
  int k;
};

struct LocalWork {
  int m = 0, n = 0;            // inner steps, windows
  float2* V = nullptr;         // [m+1][n][6400]
  float2* Z = nullptr;         // [m][n][6400]
  float2* w = nullptr;         // [n][6400]
  LocalState* st = nullptr;    // [n]
  double* escale = nullptr;    // [n] per-window output scale of the current step
};

struct fdfd_ctx;
int local_alloc(LocalWork* L, int n_win, int m, size_t* bytes);
void local_free(LocalWork* L);
// rhs [n_win][80][80] = -c_bo g on interface boundary cells (Robin data g [n_win][4][80]).
int local_robin_rhs(fdfd_ctx* h, const float2* g, float2* rhs, int n_win);
// m steps of FGMRES on every window: right-hand side from the global field
// v_global (restricted) or from rhs_win; result prolonged (restricted, times
// *scale) into z_global, or written whole to e_win.
int local_fgmres(fdfd_ctx* h, LocalWork* L, const NnoWeights* W, NnoWork* work, const float2* v_global,
                 const float2* rhs_win, float2* z_global, float2* e_win, const double* scale, int transpose = 0);
// y = A_w x for n windows (x, y [n][80][80]; win_id nullable = identity).
int local_apply_windows(fdfd_ctx* h, const float2* x, float2* y, const int* win_id, int n);
