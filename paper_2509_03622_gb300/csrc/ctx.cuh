// Handle layout shared by api.cu and the Schwarz translation units.
#pragma once
#include "common.cuh"

struct SchwarzData;  // defined in schwarz.cu

struct fdfd_ctx {
  int nx = 0, ny = 0;
  size_t n = 0;
  double dx = 0, wavelength = 0, pml_m = 3, pml_lnR = -30;
  int npml[4] = {0, 0, 0, 0};
  double k0dx = 0, k2 = 0, sb = 0;   // k0 dx, (k0 dx)^2, dx^2 w mu0
  cudaStream_t stream = nullptr;
  float* eps = nullptr;
  AxisCoef *cx = nullptr, *cy = nullptr, *cxT = nullptr, *cyT = nullptr;
  AxisCoef64 *cx64 = nullptr, *cy64 = nullptr, *cxT64 = nullptr, *cyT64 = nullptr;
  float2 *isx = nullptr, *isy = nullptr;  // 1/s at cell centres
  // Krylov workspace
  int rmax = 0;
  float2 *V = nullptr, *Z = nullptr, *w = nullptr;
  double2* x64 = nullptr;
  KrylovState* st = nullptr;
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* d_one = nullptr;      // device constant 1.0 (unit scale)
  double* flag_host = nullptr;  // pinned: est, nonfinite|breakdown
  float2 *hostJ = nullptr, *hostE = nullptr;  // device staging for host-buffer solves
  float2* adj = nullptr;                       // D^-1 g of the adjoint solve
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  size_t bytes = 0;
  SchwarzData* sw = nullptr;
  // live profiling
  bool prof_on = false;
  int prof_next = 0;
  cudaEvent_t* prof_ev = nullptr;   // 2 * PROF_POOL events
  int* prof_cls = nullptr;          // class of each recorded pair
  long long prof_launch[FDFD_PROF_NCLASS] = {0};
  long long launches_total = 0;
  // CUDA graphs of the Arnoldi steps (key = precond + 3 transpose + 6 restart)
  struct StepGraphs {
    int key = -1;
    cudaGraphExec_t exec[FDFD_MAXRESTART] = {};
    long long nk[FDFD_MAXRESTART] = {};  // kernels in each graph
  };
  StepGraphs graphs[4];
  cudaStream_t cap_stream = nullptr;     // private stream the graphs are captured on
  int graph_next = 0;
  bool graphs_ok = true;                 // false after a failed capture
};

// Drop every captured step graph (buffers or the preconditioner changed).
void graphs_invalidate(fdfd_ctx* h);

#define PROF_POOL 16384
// Bracket `nk` kernel launches of class `cls` issued by `body`.
struct ProfScope {
  fdfd_ctx* h; int cls; int slot;
  ProfScope(fdfd_ctx* h_, int cls_, int nk) : h(h_), cls(cls_), slot(-1) {
    if (!h) return;
    h->launches_total += nk;
    if (!h->prof_on) return;
    h->prof_launch[cls] += nk;
    if (h->prof_next < PROF_POOL) {
      slot = h->prof_next++;
      h->prof_cls[slot] = cls;
      cudaEventRecord(h->prof_ev[2 * slot], h->stream);
    }
  }
  ~ProfScope() { if (slot >= 0) cudaEventRecord(h->prof_ev[2 * slot + 1], h->stream); }
};

// schwarz.cu
int schwarz_create(fdfd_ctx* h, const schwarz_desc* sd);
void schwarz_destroy(fdfd_ctx* h);
// z = M(v * (*scale)) for the global vector v (complex64).
int schwarz_apply(fdfd_ctx* h, const float2* v, const double* scale_dev, float2* z, int transpose);
int schwarz_nno_solve(fdfd_ctx* h, const float2* r_win, const float2* g_win, const int* win_id,
                      int n, float2* e_win);
int schwarz_traces(fdfd_ctx* h, const float2* u, float2* g);
// Algorithm 3 pieces: local solves with source b and Robin data g_win,
// assembled into u (rhs_scratch: n_win x 6400 complex64, used with inner
// FGMRES local solves) ...
int schwarz_sweep_data(fdfd_ctx* h, const float2* b, const float2* g_win, float2* u, float2* rhs_scratch);
// ... then new traces, the coarse correction of their mismatch with g, and
// the momentum blend of g (g_new: scratch, n_win x 320 complex64).
int schwarz_stationary_update(fdfd_ctx* h, float2* u, float2* g, float2* g_new, double momentum);
// FDFD_ETIMEOUT once a bounded wait inside a neural-operator kernel ran out
// (the flag stays set: later neural passes of the handle skip their work).
int schwarz_error(fdfd_ctx* h);
// Set that flag from the host (failure injection for tests).
int schwarz_mark_failed(fdfd_ctx* h);
int schwarz_export(fdfd_ctx* h, double* Q, double* G);
int schwarz_coarse_solve(fdfd_ctx* h, const float2* ebc, float2* z);
int schwarz_ritz_export(fdfd_ctx* h, double* eta, double* H);
struct NnoWeights;
const NnoWeights* schwarz_weights(fdfd_ctx* h);  // nullptr before schwarz_setup
int schwarz_info(fdfd_ctx* h, fdfd_info* info);
int schwarz_dfty_variant(fdfd_ctx* h);  // the DFT-y GEMM variant autotuned at set-up
// Per-window modulation of the modified FNO ([n_win][4][512]), nullptr if none.
const float* schwarz_modulation(fdfd_ctx* h);
