// fc_noalloc.cu -- a smoother entry point that allocates no device memory.
//
// fc_smooth keeps its padded residual in a buffer that fc_setup allocated.
// fc_smooth_noalloc runs the same residual and patch-apply kernels but takes
// that scratch from one file-scope static device array instead, so a call
// never reaches cudaMalloc/cudaFree or any allocating library routine.  It is
// meant for callers that cannot allocate at call time: a serving runtime
// that has reserved the device memory it may use up front and hands the
// library only the vectors it owns, or a latency-critical loop that must not
// enter the CUDA allocator (which can synchronise the device).
//
// Limits and sharing:
//  - the array holds kNoallocScratchBytes (16 MiB) on every GPU that loads
//    the library, until the process exits;
//  - every call on a device shares the one array and it keeps the contents
//    of the last call: the part a call uses is cleared (zero halo) at the
//    start of the call;
//  - calls whose work overlaps on the GPU (other streams, other host
//    threads) race on the array; serialise them.
//  - the handle's device (current at fc_setup) must be the current device;
//    other devices are rejected with FC_ERR_INVALID;
//  - the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture.
#include <mutex>

#include "fc_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchBytes / sizeof(double)];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the static scratch on the current device (host code
// cannot use the symbol itself: on the host it names a stand-in object).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

fc_status fail(fc_handle h, fc_status st, const char* msg) {
  if (h) h->err = msg;
  return st;
}

}  // namespace

extern "C" fc_status fc_smooth_noalloc(fc_handle h, int level, double* x, const double* b, int nsweeps) {
  using namespace fc;
  if (!h) return FC_ERR_INVALID;
  if (!h->ready) return fail(h, FC_ERR_INVALID, "handle not set up (fc_setup failed)");
  if (level < 2 || level > h->nlev) return fail(h, FC_ERR_INVALID, "level out of range");
  if (!x || !b || nsweeps < 0) return fail(h, FC_ERR_INVALID, "bad smoother arguments");
  if (h->opt.element != 0 || h->opt.amr_uniform >= 0)
    return fail(h, FC_ERR_INVALID, "fc_smooth_noalloc runs the Q1-Q1 pair on uniform grids only");
  {
    // the scratch array is looked up on the current device: it must be the
    // device that holds the handle's operator and patch cache
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
      return fail(h, FC_ERR_INVALID, "fc_smooth_noalloc: the handle's device is not the current device");
  }
  const Level& L = h->lev[level - 1];
  const fc_prec prec = h->opt.prec;
  const bool inverse = h->opt.cache == FC_CACHE_INVERSE;
  // scratch layout per precision: padded residual in float64, float32 pairs
  // or float32 (the format the patch kernels read)
  size_t elem = 8;
  if (inverse && (prec == FC_PREC_FP32 || prec == FC_PREC_BF16)) elem = 4;
  const size_t need = (size_t)pad_nodes(L.g) * L.g.nd * elem;
  if (need > kNoallocScratchBytes)
    return fail(h, FC_ERR_INVALID,
                "level too large for fc_smooth_noalloc: the padded residual exceeds the 16 MiB static scratch");
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return fail(h, FC_ERR_CUDA, cudaGetErrorString(e));
  // the halo must read as zero; the array keeps whatever the last call left
  e = cudaMemsetAsync(scratch, 0, need, h->stream);
  if (e != cudaSuccess) return fail(h, FC_ERR_CUDA, cudaGetErrorString(e));
  double* rpad = (double*)scratch;
  float* rpadf = (float*)scratch;
  for (int s = 0; s < nsweeps; ++s) {
    if (inverse && prec == FC_PREC_DF64) e = launch_residual_df(L.g, L.st, L.mask, x, b, rpadf, h->stream);
    else if (inverse && prec != FC_PREC_FP64) e = launch_residual_f32(L.g, L.st, L.mask, x, b, rpadf, h->stream);
    else e = launch_residual(L.g, L.st, L.mask, x, b, nullptr, rpad, h->stream);
    if (e != cudaSuccess) return fail(h, FC_ERR_CUDA, cudaGetErrorString(e));
    if (inverse)
      e = launch_patch_apply(L.g, prec, L.coef, L.mask, rpad, rpadf, h->opt.omega, x, L.prow, h->stream);
    else if (h->opt.cache == FC_CACHE_MATRIX)
      e = launch_factor_apply(L.g, L.st, factor_store(L), L.mask, rpad, h->opt.omega, x, L.prow, h->stream);
    else
      e = launch_none_sweep(L.g, L.st, L.mask, h->opt.omega, rpad, x, h->d_err, L.lnode, L.nlist, L.ldl_dmin,
                            h->stream);
    if (e != cudaSuccess) return fail(h, FC_ERR_CUDA, cudaGetErrorString(e));
  }
  return FC_OK;
}
