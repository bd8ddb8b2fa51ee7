// Fourier neural operator of the subdomain solver (Sec. 2.1, Fig. 2) on
// tcgen05 tensor cores, batched over windows.
//
// Per window (80 x 80, width 32, 4 Fourier blocks, 512 retained modes):
//   pack   : restriction, RMS normalisation, 15 input channels   (SIMT)
//   lift   : [6400 px][16] x [32][16]^T                           (GEMM)
//   block b (the truncated 2D DFT is done as two 1D DFT GEMMs each way):
//     G1  DFT along x   : rows (y,c)   K = x 80        N = (kx,ri) 32   A MN-major
//     G2  DFT along y   : rows (kx,c)  K = (ri,y) 160  N = (q,ri) 64    A MN-major
//     G3  spectral mix  : 4 modes per CTA, rows = windows, K = (c,ri) 64, N = (o,ri) 64
//     G4  inverse DFT y : rows (o,kx)  K = (q,ri) 64   N = (y,ri) 160
//     G5  fused: inverse real DFT along x + W x + bias + leaky-ReLU, per y row:
//         D_y[x][o] = Gx[x][:] . T3_y[o][:] + X_y[x][:] . W[o][:]
//   proj   : [6400 px][32] x [128][32]^T, leaky, 128 -> 2, times rho,
//            written to the window's core in the global field (restricted
//            prolongation) or to a per-window array.
// Each GEMM epilogue writes the layout the next stage reads, with lanes
// mapped to the contiguous output dimension (coalesced stores).
#include <math.h>
#include <string.h>
#include <vector>
#include "nno.cuh"
#include "ctx.cuh"
#include "tc.cuh"
#include "reduce.cuh"

namespace {

constexpr int NPIX = FDFD_WIN * FDFD_WIN;  // 6400
constexpr float LEAK = 0.01f;
constexpr long long WAIT_LIMIT = 1ll << 22;  // polls of mbarrier.try_wait before giving up

__device__ __forceinline__ float leaky(float x) { return x >= 0.f ? x : LEAK * x; }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ---------------------------------------------------------------------
// Generic tile GEMM: D[128 x BN] = A[128 x K] . B[BN x K]^T for tile
// blockIdx.x of batch blockIdx.y; Op supplies operand addresses and the
// epilogue.  One elected thread issues the MMAs, the commit arrives on an
// mbarrier, all four warps read the FP32 accumulator from TMEM.
// ---------------------------------------------------------------------
// Persistent form: each CTA walks the tiles blockIdx.x, +gridDim.x, ... of
// the (batch, tile) space.  Two shared-memory stages: while tile i's MMA and
// epilogue run, tile i+1's operands are already in flight (cp.async).  A
// B operand that is the same for every tile (Op::kConstB: DFT matrices,
// weights) is loaded once per CTA.
template <int BN, int K, bool AMN, class Op>
struct GemmCfg {
  static constexpr int KC = K / 8;
  static constexpr uint32_t A_BYTES = 128 * K * 2, B_BYTES = BN * K * 2;
  static constexpr uint32_t STAGE = A_BYTES + (Op::kConstB ? 0 : B_BYTES);
  static constexpr uint32_t SMEM = 2 * STAGE + (Op::kConstB ? B_BYTES : 0) + 16;
  static constexpr uint32_t TCOLS = tc::tmem_cols(BN);
};

template <int BN, int K, bool AMN, class Op>
__device__ __forceinline__ void gemm_load(const Op& op, uint8_t* sA, uint8_t* sB, int b, int m0, int Mb,
                                          bool loadB) {
  constexpr int KC = K / 8;
  const int tid = threadIdx.x;
  if (!AMN) {
    for (int c = tid; c < 128 * KC; c += 128) {
      const int t8 = c & 7, rest = c >> 3, kc = rest % KC, rg = rest / KC;
      const int m = m0 + rg * 8 + t8;
      const bool ok = m < Mb;
      tc::cp_async16(sA + (rg * KC + kc) * 128 + t8 * 16, op.a_src(b, ok ? m : 0, kc * 8), ok);
    }
  } else {
    for (int c = tid; c < 16 * K; c += 128) {
      const int t8 = c & 7, rest = c >> 3, mg = rest & 15, kg = rest >> 4;
      const int m = m0 + mg * 8;
      const bool ok = m < Mb;
      tc::cp_async16(sA + (mg * KC + kg) * 128 + t8 * 16, op.a_src(b, ok ? m : 0, kg * 8 + t8), ok);
    }
  }
  if (loadB)
    for (int c = tid; c < BN * KC; c += 128) {
      const int t8 = c & 7, rest = c >> 3, kc = rest % KC, rg = rest / KC;
      tc::cp_async16(sB + (rg * KC + kc) * 128 + t8 * 16, op.b_src(b, rg * 8 + t8, kc * 8), true);
    }
}

template <int BN, int K, bool AMN, class Op>
__global__ void __launch_bounds__(128) gemm_kernel(Op op, int tiles_per_batch, int total, int* err) {
  static_assert(K % 16 == 0 && BN % 16 == 0 && BN <= 256, "shape");
  typedef GemmCfg<BN, K, AMN, Op> Cfg;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* stage[2] = {smem, smem + Cfg::STAGE};
  uint8_t* sBc = smem + 2 * Cfg::STAGE;  // constant B (if kConstB)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Cfg::SMEM - 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Cfg::SMEM - 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int tile = blockIdx.x;
  if (tile >= total) return;
  auto sB_of = [&](int st) { return Op::kConstB ? sBc : stage[st] + Cfg::A_BYTES; };
  {
    const int b = tile / tiles_per_batch, m0 = (tile % tiles_per_batch) * 128;
    gemm_load<BN, K, AMN>(op, stage[0], sB_of(0), b, m0, op.rows(b), true);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  if (tid == 0) tc::mbar_init(tc::smem_u32(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), Cfg::TCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16(BN, AMN, false);
  for (int i = 0; tile < total; tile += gridDim.x, ++i) {
    const int st = i & 1;
    const int b = tile / tiles_per_batch, m0 = (tile % tiles_per_batch) * 128;
    const int Mb = op.rows(b);
    const int next = tile + gridDim.x;
    if (next < total) {  // prefetch the next tile into the other stage
      const int nb = next / tiles_per_batch;
      gemm_load<BN, K, AMN>(op, stage[st ^ 1], sB_of(st ^ 1), nb, (next % tiles_per_batch) * 128, op.rows(nb),
                            !Op::kConstB);
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 1;" ::: "memory");
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a0 = tc::smem_u32(stage[st]), b0 = tc::smem_u32(sB_of(st));
#pragma unroll
      for (int s = 0; s < K / 16; ++s)
        tc::mma_bf16(tmem, tc::make_desc(a0 + s * 256, 128, K * 16), tc::make_desc(b0 + s * 256, 128, K * 16),
                     idesc, s > 0);
      tc::mma_commit(tc::smem_u32(mbar));
    }
    if (!tc::mbar_wait(tc::smem_u32(mbar), (uint32_t)(i & 1), WAIT_LIMIT)) atomicExch(err, 1);
    tc::fence_after();
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = tile rows
    const int m = m0 + warp * 32 + lane;
    const bool valid = m < Mb;
    typename Op::State sst;
    op.epi_begin(sst);
    if constexpr (Op::kUnroll) {
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (valid) op.epi(b, m, c0, v, sst);
      }
    } else {
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (valid) op.epi(b, m, c0, v, sst);
      }
    }
    if (valid) op.epi_end(b, m, sst);
    tc::fence_before();
    __syncthreads();  // accumulator and stage st are free again
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_free(tmem, Cfg::TCOLS);
  }
}

constexpr int SM_SMEM = 233472;  // shared memory per SM (228 KB)

// Grid of a persistent kernel: SMs x resident CTAs per SM, the latter from
// shared memory (1 KB reserved per CTA), threads, registers and the 512
// TMEM columns per SM (a CTA that cannot get its columns would only wait in
// tcgen05.alloc).
int persistent_grid(const void* kern, int threads, size_t smem, uint32_t tcols) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncAttributes fa;
  int regs = 64;
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
  int per_sm = (int)(SM_SMEM / (smem + 1024));
  per_sm = per_sm < 2048 / threads ? per_sm : 2048 / threads;
  const int by_regs = 65536 / (regs * threads);
  per_sm = per_sm < by_regs ? per_sm : by_regs;
  const int by_tmem = (int)(512 / tcols);
  per_sm = per_sm < by_tmem ? per_sm : by_tmem;
  if (per_sm < 1) per_sm = 1;
  return nsm * per_sm;
}

template <int BN, int K, bool AMN, class Op>
int launch_gemm(const Op& op, int tiles, int batches, int* err, cudaStream_t s) {
  typedef GemmCfg<BN, K, AMN, Op> Cfg;
  auto kern = gemm_kernel<BN, K, AMN, Op>;
  static int grid_cap = 0;
  if (grid_cap == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM) != cudaSuccess)
      return FDFD_ECUDA;
    grid_cap = persistent_grid((const void*)kern, 128, Cfg::SMEM, Cfg::TCOLS);
  }
  const int total = tiles * batches;
  const int grid = total < grid_cap ? total : grid_cap;
  kern<<<grid, 128, Cfg::SMEM, s>>>(op, tiles, total, err);
  CKL();
  return FDFD_OK;
}

struct NoState {};

// ---------------------------------------------------------------------
// Stage operators
// ---------------------------------------------------------------------
struct LiftOp {  // rows = pixels, K = 16 inputs, N = 32 channels
  static constexpr bool kConstB = true;
  static constexpr bool kUnroll = false;
  const bf16* in; const bf16* w; const float* bias; bf16* X;
  typedef NoState State;
  __device__ int rows(int) const { return NPIX; }
  __device__ const uint4* a_src(int b, int m, int k) const {
    return reinterpret_cast<const uint4*>(in + ((size_t)b * NPIX + m) * 16 + k);
  }
  __device__ const uint4* b_src(int, int n, int k) const { return reinterpret_cast<const uint4*>(w + n * 16 + k); }
  __device__ void epi_begin(State&) const {}
  __device__ void epi(int b, int m, int c0, const float* v, State&) const {
    uint32_t p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = pack2(v[2 * i] + bias[c0 + 2 * i], v[2 * i + 1] + bias[c0 + 2 * i + 1]);
    uint4* dst = reinterpret_cast<uint4*>(X + ((size_t)b * NPIX + m) * 32 + c0);
    dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
    dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
  }
  __device__ void epi_end(int, int, State&) const {}
};

struct G1Op {  // DFT along x: rows (y,c), K = x (A MN-major from X), N = (kx,ri)
  static constexpr bool kConstB = true;
  static constexpr bool kUnroll = false;
  const bf16* X; const bf16* Fx; bf16* T1;
  typedef NoState State;
  __device__ int rows(int) const { return 80 * 32; }
  __device__ const uint4* a_src(int b, int m, int k) const {  // 8 consecutive c at (y, x = k)
    const int y = m >> 5, c = m & 31;
    return reinterpret_cast<const uint4*>(X + (((size_t)b * 80 + y) * 80 + k) * 32 + c);
  }
  __device__ const uint4* b_src(int, int n, int k) const { return reinterpret_cast<const uint4*>(Fx + n * 80 + k); }
  __device__ void epi_begin(State&) const {}
  __device__ void epi(int b, int m, int c0, const float* v, State&) const {
    const int y = m >> 5, c = m & 31;
    bf16* base = T1 + (size_t)b * 160 * 512;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int col = c0 + i, kx = col >> 1, ri = col & 1;
      base[(ri * 80 + y) * 512 + kx * 32 + c] = __float2bfloat16_rn(v[i]);
    }
  }
  __device__ void epi_end(int, int, State&) const {}
};

struct G2Op {  // DFT along y: rows (kx,c), K = (ri,y) (A MN-major from T1), N = (q,ri)
  static constexpr bool kConstB = true;
  static constexpr bool kUnroll = false;
  const bf16* T1; const bf16* Fy; bf16* Xh; int cap;
  typedef NoState State;
  __device__ int rows(int) const { return 512; }
  __device__ const uint4* a_src(int b, int m, int k) const {
    return reinterpret_cast<const uint4*>(T1 + ((size_t)b * 160 + k) * 512 + m);
  }
  __device__ const uint4* b_src(int, int n, int k) const { return reinterpret_cast<const uint4*>(Fy + n * 160 + k); }
  __device__ void epi_begin(State&) const {}
  __device__ void epi(int b, int m, int c0, const float* v, State&) const {
    const int kx = m >> 5, c = m & 31;
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      const int q = (c0 + i) >> 1;
      *reinterpret_cast<uint32_t*>(Xh + (((size_t)(q * 16 + kx)) * cap + b) * 64 + c * 2) = pack2(v[i], v[i + 1]);
    }
  }
  __device__ void epi_end(int, int, State&) const {}
};


struct G4Op {  // inverse DFT along y: rows (o,kx), K = (q,ri), N = (y,ri)
  static constexpr bool kConstB = true;
  static constexpr bool kUnroll = false;
  const bf16* Yh; const bf16* Gy; bf16* T3;
  typedef NoState State;
  __device__ int rows(int) const { return 512; }
  __device__ const uint4* a_src(int b, int m, int k) const {
    return reinterpret_cast<const uint4*>(Yh + ((size_t)b * 512 + m) * 64 + k);
  }
  __device__ const uint4* b_src(int, int n, int k) const { return reinterpret_cast<const uint4*>(Gy + n * 64 + k); }
  __device__ void epi_begin(State&) const {}
  __device__ void epi(int b, int m, int c0, const float* v, State&) const {
    const int o = m >> 4, kx = m & 15;
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      const int y = (c0 + i) >> 1;
      *reinterpret_cast<uint32_t*>(T3 + (((size_t)b * 80 + y) * 32 + o) * 32 + kx * 2) = pack2(v[i], v[i + 1]);
    }
  }
  __device__ void epi_end(int, int, State&) const {}
};

struct ProjOp {  // rows = pixels, K = 32, N = 128 hidden; then 128 -> 2 and the output
  static constexpr bool kConstB = true;
  static constexpr bool kUnroll = true;  // constants below become constant-bank operands
  const bf16* X; const bf16* P1; float p2b0, p2b1;
  const float* rho; const double* scale; const int* win_id;
  float2* z_global; float2* e_win; int nx, nwx;
  const double* scale_win;
  struct State { float re, im; };
  __device__ int rows(int) const { return NPIX; }
  __device__ const uint4* a_src(int b, int m, int k) const {
    return reinterpret_cast<const uint4*>(X + ((size_t)b * NPIX + m) * 32 + k);
  }
  __device__ const uint4* b_src(int, int n, int k) const { return reinterpret_cast<const uint4*>(P1 + n * 32 + k); }
  __device__ void epi_begin(State& s) const { s.re = 0.f; s.im = 0.f; }
  __device__ void epi(int, int, int c0, const float* v, State& s) const {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float h = leaky(v[i] + p1b[c0 + i]);
      s.re = fmaf(P2[c0 + i], h, s.re);
      s.im = fmaf(P2[128 + c0 + i], h, s.im);
    }
  }
  __device__ void epi_end(int b, int m, State& s) const {
    int w = win_id ? win_id[b] : b;
    int gnx = nx, gny = ny_, gnwx = nwx;
    const double* sc = scale;
    float2* zg = z_global;
    if (ptab) {  // multi-problem batch
      const int2 e = wtab[b];
      const ProbGeom& P = ptab[e.x];
      w = e.y; gnx = P.nx; gny = P.ny; gnwx = P.nwx; sc = P.scale; zg = P.z;
    }
    float f = rho[b];
    if (sc) f *= (float)(*sc);
    if (scale_win) f *= (float)scale_win[b];
    const float2 o = make_float2((s.re + p2b0) * f, (s.im + p2b1) * f);
    if (e_win) { e_win[(size_t)b * NPIX + m] = o; return; }
    // restricted prolongation: only the window's 64 x 64 core is written
    const int a = w % gnwx, bb = w / gnwx;
    const int y = m / 80, x = m % 80;
    const int gx = min(max(FDFD_CORE * a - FDFD_OVL, 0), gnx - FDFD_WIN) + x;
    const int gy = min(max(FDFD_CORE * bb - FDFD_OVL, 0), gny - FDFD_WIN) + y;
    if (gx < FDFD_CORE * a || gx >= FDFD_CORE * a + FDFD_CORE) return;
    if (gy < FDFD_CORE * bb || gy >= FDFD_CORE * bb + FDFD_CORE) return;
    zg[(size_t)gy * gnx + gx] = o;
  }
  int ny_;
  const int2* wtab;
  const ProbGeom* ptab;
  float p1b[128];  // hidden bias
  float P2[256];   // [2][128] output weights
};

// G3 with 4 modes per CTA: unit = (kx, q-group of 4, tile of 128 windows);
// D_m[w][(o,ri)] = Xh_m[w][(c,ri')] R'_m[(o,ri)][(c,ri')]^T for the 4 modes
// m = (q0..q0+3, kx), accumulators side by side in TMEM (4 x 64 columns), so
// the epilogue writes 16 contiguous bytes (4 q x re/im) per (window, o).
constexpr int G3_Q = 4;
constexpr uint32_t G3_A = 128 * 64 * 2, G3_B = 64 * 64 * 2;
constexpr uint32_t G3_SMEM = G3_Q * (G3_A + G3_B) + 16;

__global__ void __launch_bounds__(128) g3_kernel(const bf16* Xh, const bf16* R, bf16* Yh, int cap, int nwin,
                                                 int wtiles, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + G3_Q * G3_A;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + G3_SMEM - 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + G3_SMEM - 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int u = blockIdx.x;
  const int wt = u % wtiles, qg = (u / wtiles) % (32 / G3_Q), kx = u / (wtiles * (32 / G3_Q));
  const int w0 = wt * 128;
  for (int mq = 0; mq < G3_Q; ++mq) {
    const int md = (qg * G3_Q + mq) * 16 + kx;
    for (int c = tid; c < 128 * 8; c += 128) {
      const int t8 = c & 7, rest = c >> 3, kc = rest & 7, rg = rest >> 3;
      const int w = w0 + rg * 8 + t8;
      const bool ok = w < nwin;
      tc::cp_async16(sA + mq * G3_A + (rg * 8 + kc) * 128 + t8 * 16,
                     Xh + ((size_t)md * cap + (ok ? w : 0)) * 64 + kc * 8, ok);
    }
    for (int c = tid; c < 64 * 8; c += 128) {
      const int t8 = c & 7, rest = c >> 3, kc = rest & 7, rg = rest >> 3;
      tc::cp_async16(sB + mq * G3_B + (rg * 8 + kc) * 128 + t8 * 16,
                     R + ((size_t)md * 64 + rg * 8 + t8) * 64 + kc * 8, true);
    }
  }
  tc::cp_async_wait_all();
  if (tid == 0) tc::mbar_init(tc::smem_u32(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 64 * G3_Q);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16(64, false, false);
    for (int mq = 0; mq < G3_Q; ++mq) {
      const uint32_t a0 = tc::smem_u32(sA + mq * G3_A), b0 = tc::smem_u32(sB + mq * G3_B);
      for (int s = 0; s < 4; ++s)
        tc::mma_bf16(tmem + mq * 64, tc::make_desc(a0 + s * 256, 128, 1024), tc::make_desc(b0 + s * 256, 128, 1024),
                     idesc, s > 0);
    }
    tc::mma_commit(tc::smem_u32(mbar));
  }
  if (!tc::mbar_wait(tc::smem_u32(mbar), 0, WAIT_LIMIT)) atomicExch(err, 1);
  tc::fence_after();
  const int w = w0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int oc = 0; oc < 4; ++oc) {  // 8 output channels (16 columns) per pass
    float v[G3_Q][16];
#pragma unroll
    for (int mq = 0; mq < G3_Q; ++mq) tc::tmem_ld16(trow + mq * 64 + oc * 16, v[mq]);
    if (w < nwin) {
#pragma unroll
      for (int oo = 0; oo < 8; ++oo) {
        const int o = oc * 8 + oo;
        uint4 q;
        q.x = pack2(v[0][2 * oo], v[0][2 * oo + 1]);
        q.y = pack2(v[1][2 * oo], v[1][2 * oo + 1]);
        q.z = pack2(v[2][2 * oo], v[2][2 * oo + 1]);
        q.w = pack2(v[3][2 * oo], v[3][2 * oo + 1]);
        *reinterpret_cast<uint4*>(Yh + (((size_t)w * 512) + o * 16 + kx) * 64 + qg * G3_Q * 2) = q;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_free(tmem, 64 * G3_Q);
  }
}

// Fused G5, persistent over units (window, 4 rows):
//   D_y[x][o] = Gx[x][:] T3_y[o][:]^T + X_y[x][:] W[o][:]^T
// then + bias, leaky-ReLU (not after the last block), written back to X.
// The MMA has M = 128 rows but only x < 80 are real: the X tiles of a stage
// are packed 80 rows apart, so rows 80..127 of one tile read the next tile
// (or the stage's slack), and the corresponding accumulator rows are never
// read back.  Gx and W are loaded once per CTA; the next unit's X and T3
// tiles are prefetched into the other stage while the current unit runs.
// 8 warps: warps w and w+4 share TMEM lanes 32(w%4).. and split the rows.
constexpr int G5_ROWS = 4;
constexpr int G5_THREADS = 256;
constexpr uint32_t G5_XT = 80 * 32 * 2;                              // one packed [80][32] X tile
constexpr uint32_t G5_STAGE = G5_ROWS * G5_XT + 48 * 64 + G5_ROWS * 2048;  // X tiles + slack + T3 tiles
constexpr uint32_t G5_GX = 128 * 32 * 2;
constexpr uint32_t G5_SMEM = G5_GX + 2048 + 2 * G5_STAGE + 16;

__device__ __forceinline__ void g5_load(uint8_t* stg, const bf16* X, const bf16* T3, int b, int y0) {
  const int tid = threadIdx.x;
  for (int c = tid; c < G5_ROWS * 80 * 4; c += G5_THREADS) {
    const int yy = c / 320, r = c % 320;
    const int t8 = r & 7, rest = r >> 3, kc = rest & 3, rg = rest >> 2;
    tc::cp_async16(stg + yy * G5_XT + (rg * 4 + kc) * 128 + t8 * 16,
                   X + (((size_t)b * 80 + y0 + yy) * 80 + rg * 8 + t8) * 32 + kc * 8, true);
  }
  for (int c = tid; c < G5_ROWS * 128; c += G5_THREADS) {
    const int yy = c >> 7, r = c & 127;
    const int t8 = r & 7, rest = r >> 3, kc = rest & 3, rg = rest >> 2;
    tc::cp_async16(stg + G5_ROWS * G5_XT + 48 * 64 + yy * 2048 + (rg * 4 + kc) * 128 + t8 * 16,
                   T3 + (((size_t)b * 80 + y0 + yy) * 32 + rg * 8 + t8) * 32 + kc * 8, true);
  }
}

__global__ void __launch_bounds__(G5_THREADS) g5_kernel(bf16* X, const bf16* T3, const bf16* Gx, const bf16* Wb,
                                                        const float* bias, int last, int total, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAg = smem;                       // Gx, [128][32] (rows >= 80 zero)
  uint8_t* sBw = smem + G5_GX;               // W, [32][32]
  uint8_t* stage[2] = {smem + G5_GX + 2048, smem + G5_GX + 2048 + G5_STAGE};
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + G5_SMEM - 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + G5_SMEM - 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int UPW = 80 / G5_ROWS;  // units per window
  int u = blockIdx.x;
  if (u >= total) return;
  for (int c = tid; c < 128 * 4; c += G5_THREADS) {
    const int t8 = c & 7, rest = c >> 3, kc = rest & 3, rg = rest >> 2;
    tc::cp_async16(sAg + (rg * 4 + kc) * 128 + t8 * 16, Gx + (rg * 8 + t8) * 32 + kc * 8, true);
  }
  if (tid < 128) {
    const int t8 = tid & 7, rest = tid >> 3, kc = rest & 3, rg = rest >> 2;
    tc::cp_async16(sBw + (rg * 4 + kc) * 128 + t8 * 16, Wb + (rg * 8 + t8) * 32 + kc * 8, true);
  }
  g5_load(stage[0], X, T3, u / UPW, (u % UPW) * G5_ROWS);
  asm volatile("cp.async.commit_group;" ::: "memory");
  float bs[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) bs[o] = bias[o];
  if (tid == 0) tc::mbar_init(tc::smem_u32(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 32 * G5_ROWS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16(32, false, false);
  const int quarter = warp & 3, half = warp >> 2;  // TMEM lane quarter, row half
  for (int i = 0; u < total; u += gridDim.x, ++i) {
    const int st = i & 1;
    const int b = u / UPW, y0 = (u % UPW) * G5_ROWS;
    const int next = u + gridDim.x;
    if (next < total) g5_load(stage[st ^ 1], X, T3, next / UPW, (next % UPW) * G5_ROWS);
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 1;" ::: "memory");
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t ag = tc::smem_u32(sAg), bw = tc::smem_u32(sBw), ax0 = tc::smem_u32(stage[st]);
      const uint32_t bt0 = ax0 + G5_ROWS * G5_XT + 48 * 64;
      for (int yy = 0; yy < G5_ROWS; ++yy) {
        const uint32_t d = tmem + yy * 32;
        for (int s = 0; s < 2; ++s)
          tc::mma_bf16(d, tc::make_desc(ag + s * 256, 128, 512), tc::make_desc(bt0 + yy * 2048 + s * 256, 128, 512),
                       idesc, s > 0);
        for (int s = 0; s < 2; ++s)
          tc::mma_bf16(d, tc::make_desc(ax0 + yy * G5_XT + s * 256, 128, 512),
                       tc::make_desc(bw + s * 256, 128, 512), idesc, 1);
      }
      tc::mma_commit(tc::smem_u32(mbar));
    }
    if (!tc::mbar_wait(tc::smem_u32(mbar), (uint32_t)(i & 1), WAIT_LIMIT)) atomicExch(err, 1);
    tc::fence_after();
    if (quarter < 3) {
      const int x = quarter * 32 + lane;
      for (int yy = half * (G5_ROWS / 2); yy < (half + 1) * (G5_ROWS / 2); ++yy) {
        float v[32];
        tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + yy * 32, v);
        tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + yy * 32 + 16, v + 16);
        if (x < 80) {
          uint32_t p[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            float a = v[2 * q] + bs[2 * q], c = v[2 * q + 1] + bs[2 * q + 1];
            if (!last) { a = leaky(a); c = leaky(c); }
            p[q] = pack2(a, c);
          }
          uint4* dst = reinterpret_cast<uint4*>(X + (((size_t)b * 80 + y0 + yy) * 80 + x) * 32);
          dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
          dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
          dst[2] = make_uint4(p[8], p[9], p[10], p[11]);
          dst[3] = make_uint4(p[12], p[13], p[14], p[15]);
        }
      }
    }
    tc::fence_before();
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_free(tmem, 32 * G5_ROWS);
  }
}

__global__ void __launch_bounds__(256) pack_kernel(NnoInput in, GridGeom g, bf16* out, float* rho_out) {
  __shared__ double sh[8];
  __shared__ float s_inv;
  const int b = blockIdx.x;
  int w = in.win_id ? in.win_id[b] : b;
  if (in.ptab) {  // multi-problem batch: this entry's problem supplies geometry and input
    const int2 e = in.wtab[b];
    const ProbGeom P = in.ptab[e.x];
    w = e.y;
    g.nx = P.nx; g.ny = P.ny; g.nwx = P.nwx; g.k2 = P.k2; g.eps = P.eps; g.isx = P.isx; g.isy = P.isy;
    in.v_global = P.v;
  }
  const int a = w % g.nwx, bb = w / g.nwx;
  const int x0 = min(max(FDFD_CORE * a - FDFD_OVL, 0), g.nx - FDFD_WIN);
  const int y0 = min(max(FDFD_CORE * bb - FDFD_OVL, 0), g.ny - FDFD_WIN);
  auto r_at = [&](int p) -> float2 {
    if (in.v_global) return in.v_global[(size_t)(y0 + p / 80) * g.nx + x0 + p % 80];
    if (in.r_win) return in.r_win[(size_t)b * NPIX + p];
    return make_float2(0.f, 0.f);
  };
  const float2* gw = in.g_win ? in.g_win + (size_t)b * 320 : nullptr;
  float acc = 0.f;
  for (int p = threadIdx.x; p < NPIX; p += 256) { const float2 r = r_at(p); acc += r.x * r.x + r.y * r.y; }
  if (gw)
    for (int t = threadIdx.x; t < 320; t += 256) { const float2 q = gw[t]; acc += q.x * q.x + q.y * q.y; }
  const double tot = block_sum<256>((double)acc, sh);
  if (threadIdx.x == 0) {
    const float rho = (float)sqrt(tot / NPIX);
    rho_out[b] = rho;
    s_inv = rho > 0.f ? 1.f / rho : 0.f;
  }
  __syncthreads();
  const float inv = s_inv;
  for (int p = threadIdx.x; p < NPIX; p += 256) {
    const int y = p / 80, x = p % 80, gx = x0 + x, gy = y0 + y;
    const float2 r = r_at(p);
    float c[16];
    c[0] = g.k2 * g.eps[(size_t)gy * g.nx + gx];
    c[1] = r.x * inv; c[2] = r.y * inv;
    if (gw) {
      const float2 gl = gw[0 * 80 + y], gr = gw[1 * 80 + y], gb = gw[2 * 80 + x], gt = gw[3 * 80 + x];
      c[3] = gl.x * inv; c[4] = gl.y * inv; c[5] = gr.x * inv; c[6] = gr.y * inv;
      c[7] = gb.x * inv; c[8] = gb.y * inv; c[9] = gt.x * inv; c[10] = gt.y * inv;
    } else {
#pragma unroll
      for (int i = 3; i <= 10; ++i) c[i] = 0.f;
    }
    const float2 sx = g.isx[gx], sy = g.isy[gy];
    c[11] = sx.x; c[12] = sx.y; c[13] = sy.x; c[14] = sy.y; c[15] = 0.f;
    uint4* dst = reinterpret_cast<uint4*>(out + ((size_t)b * NPIX + p) * 16);
    dst[0] = make_uint4(pack2(c[0], c[1]), pack2(c[2], c[3]), pack2(c[4], c[5]), pack2(c[6], c[7]));
    dst[1] = make_uint4(pack2(c[8], c[9]), pack2(c[10], c[11]), pack2(c[12], c[13]), pack2(c[14], c[15]));
  }
}

// Self-test operator: plain row-major C = A B^T.
struct TestOp {
  static constexpr bool kConstB = false;
  static constexpr bool kUnroll = false;
  const bf16* A; const bf16* B; float* C; int M, N, K, amn;
  typedef NoState State;
  __device__ int rows(int) const { return M; }
  __device__ const uint4* a_src(int, int m, int k) const {
    return reinterpret_cast<const uint4*>(amn ? A + (size_t)k * M + m : A + (size_t)m * K + k);
  }
  __device__ const uint4* b_src(int, int n, int k) const { return reinterpret_cast<const uint4*>(B + (size_t)n * K + k); }
  __device__ void epi_begin(State&) const {}
  __device__ void epi(int, int m, int c0, const float* v, State&) const {
#pragma unroll
    for (int i = 0; i < 16; ++i) C[(size_t)m * N + c0 + i] = v[i];
  }
  __device__ void epi_end(int, int, State&) const {}
};

std::vector<bf16> to_bf16(const std::vector<float>& a) {
  std::vector<bf16> o(a.size());
  for (size_t i = 0; i < a.size(); ++i) o[i] = __float2bfloat16_rn(a[i]);
  return o;
}

template <class T>
int up(T** dst, const std::vector<T>& v, size_t* bytes) {
  if (cudaMalloc((void**)dst, v.size() * sizeof(T)) != cudaSuccess) return FDFD_ENOMEM;
  *bytes += v.size() * sizeof(T);
  CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FDFD_OK;
}

}  // namespace

int nno_upload_weights(NnoWeights* W, const float* blob, size_t nfloats, size_t* bytes) {
  const size_t expect = 32 * 15 + 32 + 4 * (2 * 32 * 32 * 512 + 32 * 32 + 32) + 128 * 32 + 128 + 2 * 128 + 2;
  if (!blob || nfloats != expect) return FDFD_EINVAL;
  const float* p = blob;
  int rc;
  {  // lift [32][15] -> [32][16]
    std::vector<float> lw(32 * 16, 0.f);
    for (int o = 0; o < 32; ++o)
      for (int i = 0; i < 15; ++i) lw[o * 16 + i] = p[o * 15 + i];
    p += 32 * 15;
    if ((rc = up(&W->lift_w, to_bf16(lw), bytes))) return rc;
    if ((rc = up(&W->lift_b, std::vector<float>(p, p + 32), bytes))) return rc;
    p += 32;
  }
  const double PI = 3.14159265358979323846;
  {  // DFT matrices (FP64 -> BF16)
    std::vector<float> fx(32 * 80), fy(64 * 160), gy(160 * 64), gx(128 * 32, 0.f);
    for (int kx = 0; kx < 16; ++kx)
      for (int x = 0; x < 80; ++x) {
        const double th = 2 * PI * kx * x / 80.0;
        fx[(kx * 2 + 0) * 80 + x] = (float)cos(th);
        fx[(kx * 2 + 1) * 80 + x] = (float)(-sin(th));
        const double c = (kx == 0 ? 1.0 : 2.0) / 80.0;
        gx[x * 32 + kx * 2 + 0] = (float)(c * cos(th));
        gx[x * 32 + kx * 2 + 1] = (float)(-c * sin(th));
      }
    for (int q = 0; q < 32; ++q) {
      const int ky = q < 16 ? q : q - 32;
      for (int y = 0; y < 80; ++y) {
        const double th = 2 * PI * ky * y / 80.0;
        const double fr = cos(th), fi = -sin(th);          // e^{-i th}
        fy[(q * 2 + 0) * 160 + 0 * 80 + y] = (float)fr;
        fy[(q * 2 + 0) * 160 + 1 * 80 + y] = (float)(-fi);
        fy[(q * 2 + 1) * 160 + 0 * 80 + y] = (float)fi;
        fy[(q * 2 + 1) * 160 + 1 * 80 + y] = (float)fr;
        const double gr = cos(th) / 80.0, gi = sin(th) / 80.0;  // e^{+i th} / 80
        gy[(y * 2 + 0) * 64 + q * 2 + 0] = (float)gr;
        gy[(y * 2 + 0) * 64 + q * 2 + 1] = (float)(-gi);
        gy[(y * 2 + 1) * 64 + q * 2 + 0] = (float)gi;
        gy[(y * 2 + 1) * 64 + q * 2 + 1] = (float)gr;
      }
    }
    if ((rc = up(&W->Fx, to_bf16(fx), bytes)) || (rc = up(&W->Fy, to_bf16(fy), bytes)) ||
        (rc = up(&W->Gy, to_bf16(gy), bytes)) || (rc = up(&W->Gx, to_bf16(gx), bytes)))
      return rc;
  }
  for (int bl = 0; bl < 4; ++bl) {
    const float* Rr = p;
    const float* Ri = p + 32 * 32 * 512;
    p += 2 * 32 * 32 * 512;
    std::vector<float> R(512 * 64 * 64);
    for (int q = 0; q < 32; ++q)
      for (int kx = 0; kx < 16; ++kx) {
        const int md = q * 16 + kx;
        for (int o = 0; o < 32; ++o)
          for (int c = 0; c < 32; ++c) {
            const float rr = Rr[((o * 32 + c) * 32 + q) * 16 + kx], ri = Ri[((o * 32 + c) * 32 + q) * 16 + kx];
            float* row_re = &R[((size_t)md * 64 + o * 2 + 0) * 64];
            float* row_im = &R[((size_t)md * 64 + o * 2 + 1) * 64];
            row_re[c * 2 + 0] = rr; row_re[c * 2 + 1] = -ri;
            row_im[c * 2 + 0] = ri; row_im[c * 2 + 1] = rr;
          }
      }
    if ((rc = up(&W->R[bl], to_bf16(R), bytes))) return rc;
    if ((rc = up(&W->W[bl], to_bf16(std::vector<float>(p, p + 1024)), bytes))) return rc;
    p += 1024;
    if ((rc = up(&W->bias[bl], std::vector<float>(p, p + 32), bytes))) return rc;
    p += 32;
  }
  if ((rc = up(&W->P1, to_bf16(std::vector<float>(p, p + 128 * 32)), bytes))) return rc;
  p += 128 * 32;
  if ((rc = up(&W->p1b, std::vector<float>(p, p + 128), bytes))) return rc;
  memcpy(W->hp1b, p, sizeof(W->hp1b));
  p += 128;
  if ((rc = up(&W->P2, std::vector<float>(p, p + 256), bytes))) return rc;
  memcpy(W->hP2, p, sizeof(W->hP2));
  p += 256;
  W->p2b[0] = p[0];
  W->p2b[1] = p[1];
  return FDFD_OK;
}

void nno_free_weights(NnoWeights* W) {
  void* ptrs[] = {W->lift_w, W->lift_b, W->Fx, W->Fy, W->Gy, W->Gx, W->P1, W->p1b, W->P2};
  for (void* q : ptrs) if (q) cudaFree(q);
  for (int b = 0; b < 4; ++b) {
    if (W->R[b]) cudaFree(W->R[b]);
    if (W->W[b]) cudaFree(W->W[b]);
    if (W->bias[b]) cudaFree(W->bias[b]);
  }
  *W = NnoWeights();
}

int nno_alloc_work(NnoWork* w, int cap, size_t* bytes) {
  w->cap = cap;
  const size_t c = (size_t)cap;
  struct { void** p; size_t n; } a[] = {
      {(void**)&w->in, c * NPIX * 16 * 2}, {(void**)&w->X, c * NPIX * 32 * 2}, {(void**)&w->T1, c * 160 * 512 * 2},
      {(void**)&w->Xh, 512 * c * 64 * 2},  {(void**)&w->Yh, c * 512 * 64 * 2}, {(void**)&w->T3, c * 80 * 32 * 32 * 2},
      {(void**)&w->rho, c * 4},             {(void**)&w->err, 16}};
  for (auto& e : a) {
    if (cudaMalloc(e.p, e.n) != cudaSuccess) return FDFD_ENOMEM;
    *bytes += e.n;
  }
  CK(cudaMemset(w->err, 0, 16));
  return FDFD_OK;
}

void nno_free_work(NnoWork* w) {
  void* ptrs[] = {w->in, w->X, w->T1, w->Xh, w->Yh, w->T3, w->rho, w->err};
  for (void* q : ptrs) if (q) cudaFree(q);
  *w = NnoWork();
}

int nno_forward(const NnoWeights* W, NnoWork* k, const GridGeom& g, const NnoInput& in, const NnoOutput& out,
                int n, cudaStream_t s, fdfd_ctx* h) {
  if (n <= 0) return FDFD_OK;
  if (n > k->cap) return FDFD_EINVAL;
  int rc;
  {
    ProfScope ps(h, 5, 1);
    pack_kernel<<<n, 256, 0, s>>>(in, g, k->in, k->rho);
    CKL();
  }
  {
    ProfScope ps(h, 8, 1);
    if ((rc = launch_gemm<32, 16, false>(LiftOp{k->in, W->lift_w, W->lift_b, k->X}, NPIX / 128, n, k->err, s))) return rc;
  }
  static int g5_cap = 0;
  if (!g5_cap) {
    CK(cudaFuncSetAttribute(g3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G3_SMEM));
    CK(cudaFuncSetAttribute(g5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G5_SMEM));
    g5_cap = persistent_grid((const void*)g5_kernel, G5_THREADS, G5_SMEM, 32 * G5_ROWS);
  }
  const int g5_total = n * (80 / G5_ROWS);
  const int g5_grid = g5_total < g5_cap ? g5_total : g5_cap;
  for (int bl = 0; bl < 4; ++bl) {
    {
      ProfScope ps(h, 9, 1);
      if ((rc = launch_gemm<32, 80, true>(G1Op{k->X, W->Fx, k->T1}, 2560 / 128, n, k->err, s))) return rc;
    }
    {
      ProfScope ps(h, 10, 1);
      if ((rc = launch_gemm<64, 160, true>(G2Op{k->T1, W->Fy, k->Xh, k->cap}, 512 / 128, n, k->err, s))) return rc;
    }
    {
      ProfScope ps(h, 11, 1);
      const int wtiles = (n + 127) / 128;
      g3_kernel<<<wtiles * (32 / G3_Q) * 16, 128, G3_SMEM, s>>>(k->Xh, W->R[bl], k->Yh, k->cap, n, wtiles, k->err);
      CKL();
    }
    {
      ProfScope ps(h, 12, 1);
      if ((rc = launch_gemm<160, 64, false>(G4Op{k->Yh, W->Gy, k->T3}, 512 / 128, n, k->err, s))) return rc;
    }
    {
      ProfScope ps(h, 13, 1);
      g5_kernel<<<g5_grid, G5_THREADS, G5_SMEM, s>>>(k->X, k->T3, W->Gx, W->W[bl], W->bias[bl], bl == 3, g5_total, k->err);
      CKL();
    }
  }
  ProjOp po{k->X, W->P1, W->p2b[0], W->p2b[1], k->rho, out.scale, in.win_id,
            out.z_global, out.e_win, g.nx, g.nwx, out.scale_win};
  po.ny_ = g.ny;
  po.wtab = in.wtab;
  po.ptab = in.ptab;
  memcpy(po.p1b, W->hp1b, sizeof(po.p1b));
  memcpy(po.P2, W->hP2, sizeof(po.P2));
  {
    ProfScope ps(h, 14, 1);
    if ((rc = launch_gemm<128, 32, false>(po, NPIX / 128, n, k->err, s))) return rc;
  }
  return FDFD_OK;
}

int nno_gemm_selftest(const bf16* A, const bf16* B, float* C, int M, int N, int K, int a_mn, int* err,
                      cudaStream_t s) {
  TestOp op{A, B, C, M, N, K, a_mn};
  const int tiles = (M + 127) / 128;
  if (M % 8) return FDFD_EINVAL;
#define SELF(NN, KK)                                                              \
  if (N == NN && K == KK)                                                         \
    return a_mn ? launch_gemm<NN, KK, true>(op, tiles, 1, err, s)                 \
                : launch_gemm<NN, KK, false>(op, tiles, 1, err, s);
  SELF(32, 80) SELF(64, 160) SELF(64, 64) SELF(160, 64) SELF(32, 16) SELF(128, 32)
#undef SELF
  return FDFD_EINVAL;
}
