// fdfd_nno_solve_noalloc: the batched neural local solve of fdfd_nno_solve
// for callers that must not allocate device memory: code that runs inside a
// fixed device-memory budget handed out by its own pool allocator (a
// cudaMalloc there would take memory the pool has already promised to
// others), or a latency-bound loop that cannot afford the device-wide
// synchronisation an allocation or free may cause.  The call is synchronous:
// it copies the kernels' error flag back and waits for the stream.
//
// Instead of the handle's per-call workspace, the intermediates of the
// neural operator live in one file-scope device array of fixed size
// (NOALLOC_MAX_WINDOWS windows, about 3.5 MB), which every GPU that loads
// the library holds until the process exits.  In host code the array's name
// is only a host-side stand-in, so its device address is looked up with
// cudaGetSymbolAddress, with the device current, the first time a call runs
// on a device (and again if that device's context has been replaced, e.g.
// after cudaDeviceReset), and then passed to the kernels.
#include <mutex>
#include "ctx.cuh"
#include "nno.cuh"

#define NOALLOC_MAX_WINDOWS 4

namespace {

constexpr size_t NW = NOALLOC_MAX_WINDOWS;
constexpr size_t B_X = NW * 6400 * 32 * 2;
constexpr size_t B_T1 = NW * 160 * 512 * 2;
constexpr size_t B_XH = 512 * (size_t)xh_rows(NW) * 64 * 2;
constexpr size_t B_YH = NW * 512 * 64 * 2;
constexpr size_t B_T3 = NW * 80 * 32 * 32 * 2;
constexpr size_t B_RHO = 256;
constexpr size_t B_ERR = 256;
constexpr size_t SCRATCH_BYTES = B_X + B_T1 + B_XH + B_YH + B_T3 + B_RHO + B_ERR;

static __device__ __align__(256) unsigned char g_nno_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[MAX_DEVICES] = {};
void* g_scratch_ctx[MAX_DEVICES] = {};  // context the cached address belongs to

// The driver's cuCtxGetCurrent, looked up through the runtime (the library
// keeps no load-time dependency on the driver library).
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  return fn;
}

void* current_ctx() {
  void* ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get || get(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of the scratch array on the current device and context.
int scratch_address(unsigned char** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return FDFD_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  void* ctx = current_ctx();
  if (!g_scratch_dev[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_nno_scratch));  // also makes the device's context current
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    g_scratch_ctx[dev] = current_ctx();
  }
  *out = g_scratch_dev[dev];
  return FDFD_OK;
}

}  // namespace

extern "C" int fdfd_nno_solve_noalloc(fdfd_handle h, const fdfd_c64* r_win, const fdfd_c64* g_win,
                                      const int* win_id, int n, fdfd_c64* e_win) {
  if (!h || !r_win || !g_win || !win_id || !e_win || n < 0) return FDFD_EINVAL;
  if (n > NOALLOC_MAX_WINDOWS) {
    fprintf(stderr, "libfdfd: fdfd_nno_solve_noalloc: %d windows requested, at most %d supported\n", n,
            NOALLOC_MAX_WINDOWS);
    return FDFD_EINVAL;
  }
  const NnoWeights* W = schwarz_weights(h);
  if (!W) return FDFD_ENOSETUP;
  // a neural pass of this handle already gave up on a bounded wait: the
  // same sticky failure fdfd_nno_solve reports
  int rc = schwarz_error(h);
  if (rc) return rc;
  if (n == 0) return FDFD_OK;
  unsigned char* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  NnoWork k;
  k.cap = NOALLOC_MAX_WINDOWS;
  k.g2_split = schwarz_dfty_variant(h);  // the same kernels as the handle's own passes
  size_t off = 0;
  k.X = reinterpret_cast<bf16*>(base + off); off += B_X;
  k.T1 = reinterpret_cast<bf16*>(base + off); off += B_T1;
  k.Xh = reinterpret_cast<bf16*>(base + off); off += B_XH;
  k.Yh = reinterpret_cast<bf16*>(base + off); off += B_YH;
  k.T3 = reinterpret_cast<bf16*>(base + off); off += B_T3;
  k.rho = reinterpret_cast<float*>(base + off); off += B_RHO;
  k.err = reinterpret_cast<int*>(base + off);
  // the array keeps the previous call's contents: the error flag must start at zero
  CK(cudaMemsetAsync(k.err, 0, sizeof(int), h->stream));
  NnoInput in;
  in.r_win = reinterpret_cast<const float2*>(r_win);
  in.g_win = reinterpret_cast<const float2*>(g_win);
  in.win_id = win_id;
  NnoOutput out;
  out.e_win = reinterpret_cast<float2*>(e_win);
  GridGeom g{h->nx, h->ny, h->nx / FDFD_CORE, (float)h->k2, h->eps, h->isx, h->isy, schwarz_modulation(h)};
  if ((rc = nno_forward(W, &k, g, in, out, n, h->stream, nullptr))) return rc;
  int e = 0;
  CK(cudaMemcpyAsync(&e, k.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return e ? FDFD_ETIMEOUT : FDFD_OK;
}
