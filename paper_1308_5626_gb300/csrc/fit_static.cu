// psp_fit_band_static: the band fit of Algorithm 2 for callers that cannot allocate device
// memory.  Some callers of this library run where cudaMalloc is not available to them:
// code inside a CUDA-graph-driven or real-time loop that must not allocate, plugins handed
// a fixed memory budget by their host application, or processes whose allocator is owned by
// another framework.  psp_create allocates the whole solver workspace, so those callers
// cannot use the handle-based psp_fit_band; this entry point needs no handle and allocates
// nothing.
//
// Its one piece of scratch memory -- the per-row moments of the fit, 4b+4 doubles per row --
// lives in a file-scope device array sized for at most kStaticFitMaxRows rows (10 MiB of
// device memory, held by every GPU that loads this library until the process exits).  Host
// code cannot use the array's name as a device address (in host code it names a host-side
// stand-in); the address is fetched once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on that device.  That first call should therefore
// happen before any stream capture.  Every call shares the array and it keeps the last
// call's contents; the degenerate-row counter is cleared at the start of every call.  Calls
// whose work overlaps on the GPU (different streams, or different host threads) race on the
// array and must be serialised by the caller.
#include <mutex>
#include <string>

#include "psp_kernels.cuh"

namespace psp {
void set_last_error(const std::string &msg);   // psp_api.cu
}

namespace {

constexpr int64_t kStaticFitMaxRows = 65536;
constexpr int kMomentsPerRow = 4 * psp::kMaxB + 4;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_fit_scratch[kStaticFitMaxRows * kMomentsPerRow];
static __device__ __align__(256) int g_fit_singular[64];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};
int *g_singular_ptr[kMaxDevices] = {};

psp_status err(psp_status s, const std::string &m) {
  psp::set_last_error(m);
  return s;
}

}  // namespace

extern "C" psp_status psp_fit_band_static(const double *Px, const double *Py, int64_t ld, int M, int64_t n,
                                          int b, int intercept, double *N_band, int *singular_rows,
                                          void *cuda_stream) {
  if (!Px || !Py || !N_band) return err(PSP_ERR_ARG, "psp_fit_band_static: NULL array");
  if (b < 1 || b > psp::kMaxB) return err(PSP_ERR_ARG, "psp_fit_band_static: b must be in 1..4");
  if (n < 2 * b + 1) return err(PSP_ERR_ARG, "psp_fit_band_static: need n >= 2b+1");
  if (n > kStaticFitMaxRows)
    return err(PSP_ERR_ARG, "psp_fit_band_static: n = " + std::to_string(n) + " exceeds the static scratch limit of " +
                                std::to_string(kStaticFitMaxRows) + " rows");
  if (M < 1 || ld < n) return err(PSP_ERR_ARG, "psp_fit_band_static: need M >= 1 and ld >= n");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(PSP_ERR_CUDA, "psp_fit_band_static: no current CUDA device");
  double *scratch = nullptr;
  int *count = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      double *s = nullptr;
      int *c = nullptr;
      cudaError_t e1 = cudaGetSymbolAddress((void **)&s, g_fit_scratch);
      cudaError_t e2 = cudaGetSymbolAddress((void **)&c, g_fit_singular);
      if (e1 != cudaSuccess || e2 != cudaSuccess || !s || !c)
        return err(PSP_ERR_CUDA, std::string("psp_fit_band_static: cudaGetSymbolAddress failed: ") +
                                     cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
      g_scratch_ptr[dev] = s;
      g_singular_ptr[dev] = c;
    }
    scratch = g_scratch_ptr[dev];
    count = g_singular_ptr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (singular_rows) {
    // the count is read back with a copy to host memory and a stream synchronisation, and
    // neither may be enqueued while the stream is being captured into a graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess)
      return err(PSP_ERR_CUDA, "psp_fit_band_static: cudaStreamIsCapturing failed");
    if (cs != cudaStreamCaptureStatusNone)
      return err(PSP_ERR_ARG, "psp_fit_band_static: singular_rows must be NULL while the stream is captured");
  }
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return err(PSP_ERR_CUDA, std::string("psp_fit_band_static: ") + cudaGetErrorString(e));
  psp::launch_fit<double>(b, intercept ? 1 : 0, n, M, Px, Py, ld, scratch, N_band, count, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(PSP_ERR_CUDA, std::string("psp_fit_band_static: launch: ") + cudaGetErrorString(e));
  if (singular_rows) {
    e = cudaMemcpyAsync(singular_rows, count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(PSP_ERR_CUDA, std::string("psp_fit_band_static: ") + cudaGetErrorString(e));
  }
  return PSP_OK;
}
