// Neural-operator (Fig. 2) device data and the host driver's interface.
#pragma once
#include "common.cuh"

typedef __nv_bfloat16 bf16;

struct NnoWeights {
  bf16* lift_w = nullptr;   // [32][16]      (15 inputs, padded)
  float* lift_b = nullptr;  // [32]
  bf16* Fx = nullptr;       // [32 (kx,ri)][80 x]           forward DFT along x
  bf16* Fy = nullptr;       // [64 (q,ri)][160 (ri',y)]     forward DFT along y (realified)
  bf16* R[4] = {};          // [512 mode][64 (o,ri)][64 (c,ri')]  realified spectral weights,
                            // rows swizzled like Xh (r_off)
  bf16* Gy = nullptr;       // [160 (y,ri)][64 (q,ri')]     inverse DFT along y (1/80)
  bf16* Gx = nullptr;       // [128 x][32 (kx,ri)]          inverse real DFT along x (1/80), rows >= 80 zero
  bf16* W[4] = {};          // [32 o][32 c]
  float* bias[4] = {};      // [32]
  bf16* W0L = nullptr;      // [32][16]  W[0] lift_w: block 0's residual path applied to the inputs
  float* bias0L = nullptr;  // [32]      W[0] lift_b + bias[0]
  bf16* P1 = nullptr;       // [144][32]: P1, then 0.01 P2 P1 (the leaky-ReLU's linear part), 0
  float p2w[256] = {};      // 0.99 P2 [2][128]  (host copies: kernel parameters)
  float nb[128] = {};       // -p1b
  float p2b[2] = {0.f, 0.f};  // p2b + P2 p1b
  // FP8 activations (precision pattern): the activation entering block b
  // (b = 0..3) and the projection (b = 4) is stored as E4M3 q with
  // x = q * s[b][c] (power-of-two per-channel scales from a calibration pass);
  // the scales are folded into the weights that read it.
  bool fp8 = false;
  float* qinv = nullptr;    // [5][32]  1 / s[b][c], used by the writers
  bf16* W8[4] = {};         // [32 o][32 c]  W[b] diag(s[b])
  bf16* P18 = nullptr;      // [144][32]     P1 (extended as above) diag(s[4])
  // Modulation path of the modified FNO (Sec. 2.1, Fig. 2), FP32: 3x3
  // stride-2 valid convolution of the five auxiliary channels to 16, leaky-
  // ReLU, 13x13 average pooling (3 x 3 cells), fully connected 144 -> 2048.
  bool mod = false;
  float* mod_conv_w = nullptr;  // [16][5][3][3]
  float* mod_conv_b = nullptr;  // [16]
  float* mod_fc_w = nullptr;    // [2048][144]
  float* mod_fc_b = nullptr;    // [2048]
};

// Rows of the spectrum per mode: the windows rounded up to a whole 8-row
// group of the tiled layout.
__host__ __device__ constexpr int xh_rows(int cap) { return (cap + 7) & ~7; }
// Spectrum: element (mode md, window w, k = (c,ri)).  Each window's 64
// values of a mode are one 128-byte row (written whole by the DFT-y
// epilogue) with its 16-byte chunk k/8 stored at chunk (k/8) ^ (w % 8): the
// 128-byte swizzled K-major operand layout, so a tile of up to 128
// consecutive windows of one mode is one contiguous bulk copy that the
// tensor core reads as it lands.
__host__ __device__ constexpr size_t xh_off(int md, int w, int k, int rows) {
  return ((size_t)md * rows + w) * 64 + ((((k >> 3) ^ (w & 7)) << 3) | (k & 7));
}
// Spectral weights: element (mode, n = (o,ri), k = (c,ri')), same layout.
__host__ __device__ constexpr size_t r_off(int md, int n, int k) {
  return (size_t)md * 4096 + (size_t)n * 64 + ((((k >> 3) ^ (n & 7)) << 3) | (k & 7));
}

// Mixed spectrum: element (window w, m = (o,kx), k = (q,ri)); each 128-byte
// row (w, m) keeps its 16-byte chunk k/8 at chunk (k/8) ^ (m % 8), the
// 128-byte swizzled K-major operand layout, so a tile of 128 rows of one
// window is one contiguous bulk copy for the inverse DFT along y.
__host__ __device__ constexpr size_t yh_off(int w, int m, int k) {
  return ((size_t)w * 512 + m) * 64 + ((((k >> 3) ^ (m & 7)) << 3) | (k & 7));
}

struct NnoWork {
  int cap = 0;              // windows per batch
  bf16* X = nullptr;        // [cap][80 y][x/8][c/8][x%8][c%8]  activations, tiled (in place)
  bf16* T1 = nullptr;       // [cap][160 (ri,y)][512 (kx,c)]
  bf16* Xh = nullptr;       // [512 mode][xh_rows(cap) w][64 (c,ri)], chunks swizzled: xh_off
  bf16* Yh = nullptr;       // [cap][512 (o,kx)][64 (q,ri)], chunks swizzled: yh_off
  bf16* T3 = nullptr;       // [cap][80 y][o/8][k/8][o%8][k%8]  k = (kx,ri), tiled
  float* rho = nullptr;     // [cap]
  uint8_t* packed = nullptr;  // [cap][20 units][4 rows][x/8][k/8][x%8][k%8] BF16 input channels (16 per
                              // pixel, the lift's A tiles); nullptr: the G5 kernels build them in place
  int* err = nullptr;       // bounded-wait failure flag
  int g2_split = 0;         // DFT-y GEMM variant, set by nno_autotune: 0 = A tiles by TMA,
                            // 1 or 2 = cp.async gather with that K split
};

// One problem of a multi-problem window batch (batching pattern).
struct ProbGeom {
  int nx, ny, nwx;
  float k2;
  const float* eps;
  const float2* isx;
  const float2* isy;
  const float2* v;       // preconditioner input field of this problem
  float2* z;             // output field (restricted prolongation)
  const double* scale;   // output scale (device scalar)
  const float* mod;      // this problem's per-window modulation [n_win][4][512] or nullptr
};

// Where the packed inputs come from.
struct NnoInput {
  const float2* v_global = nullptr;  // residual source: global field (restricted per window), or
  const float2* r_win = nullptr;     //   per-window residuals [n][80][80], or neither (zero)
  const float2* g_win = nullptr;     // Robin data [n][4][80] (nullptr = zero)
  const int* win_id = nullptr;       // window of each batch entry (nullptr = identity)
  // multi-problem batch: entry b is window wtab[b].y of problem ptab[wtab[b].x]
  // (geometry, input and output then come from the table)
  const int2* wtab = nullptr;
  const ProbGeom* ptab = nullptr;
};

// Where the output goes.
struct NnoOutput {
  float2* z_global = nullptr;        // restricted prolongation into a global field, or
  float2* e_win = nullptr;           // per-window fields [n][80][80]
  const double* scale = nullptr;     // multiply by *scale (nullptr = 1)
  const double* scale_win = nullptr; // and by scale_win[b] per batch entry (nullptr = 1)
};

struct GridGeom {
  int nx, ny, nwx;
  float k2;                          // (k0 dx)^2
  const float* eps;
  const float2* isx;
  const float2* isy;
  const float* mod;                  // per-window modulation [n_win][4][512] (modified FNO) or nullptr
};

// Blob layout (include/fdfd.h): rank > 0 gives each block's R as rank-r
// factors (expanded here, in FP64, into the tiled R); modulation appends the
// modulation path's weights.
int nno_upload_weights(NnoWeights* W, const float* blob, size_t nfloats, int rank, int modulation,
                       size_t* bytes);
// Floats in a weight blob of that layout.
size_t nno_blob_floats(int rank, int modulation);
// The modulation of every window of a grid, once per set-up (it depends on
// the permittivity and PML maps only): out [n_win][4][512].
int nno_modulation(const NnoWeights* W, const GridGeom& g, int n_win, float* out, cudaStream_t s);
void nno_free_weights(NnoWeights* W);
int nno_alloc_work(NnoWork* w, int cap, size_t* bytes);
// Autotuner: time the variants of the shape-dependent stage (the DFT-y
// GEMM: TMA-loaded operand tiles, or the gather with K split 1 or 2) on n
// windows of the work buffers with CUDA events and keep the fastest in `work`.
int nno_autotune(const NnoWeights* W, NnoWork* work, int n, cudaStream_t s);
void nno_free_work(NnoWork* w);
struct fdfd_ctx;
// Run the neural operator on n windows (n <= work->cap); h (nullable) only
// receives the per-stage profiling scopes.
int nno_forward(const NnoWeights* W, NnoWork* work, const GridGeom& g, const NnoInput& in,
                const NnoOutput& out, int n, cudaStream_t s, fdfd_ctx* h = nullptr,
                unsigned* calib = nullptr);
// Switch W to FP8 activations: calibrate the per-channel scales on BF16
// forwards of `n` windows of each of the n_in inputs in[] (max |x| per
// channel at the five activation points over all of them, with 4x headroom,
// rounded up to a power of two) and upload the scale-folded weights.  `blob`
// is the weight blob W was made from.
int nno_enable_fp8(NnoWeights* W, NnoWork* work, const GridGeom& g, const NnoInput* in, int n_in, int n,
                   const float* blob, size_t nfloats, size_t* bytes, cudaStream_t s);
// Direct access to the tcgen05 GEMM for self-tests: C[M][N] (fp32) =
// A[M][K] . B[N][K]^T with A K-major (a_mn = 0, row stride K) or MN-major
// (a_mn = 1, stored [K][M]); supported (N, K): (32,80) (64,160) (64,64)
// (160,64) (32,16) (128,32).
// Diagnostic of the bounded waits: *result = 2 if a wait that can never
// complete gave up as it must, 1 if it (wrongly) completed.
int nno_wait_selftest(int* result, cudaStream_t s);
int nno_gemm_selftest(const bf16* A, const bf16* B, float* C, int M, int N, int K, int a_mn, int* err,
                      cudaStream_t s);
