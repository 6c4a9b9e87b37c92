// qrng_minentropy_noalloc: the min-entropy estimate for callers that must not allocate device
// memory. It runs the same histogram and finaliser kernels as qrng_minentropy, but their scratch
// (the histogram counters and the device-side report) lives in fixed arrays compiled into this
// library instead of in context workspace.
//
// Who needs it: acquisition loops that are not allowed to allocate once streaming has started,
// because cudaMalloc/cudaFree can block and synchronise the whole device and would stall the
// stream of ADC samples; and host programs whose device memory is owned by another allocator
// (a framework's caching pool, a fixed partition of the GPU) that forbids third-party
// allocations, or that have no place to keep a context object between calls.
//
// Costs and rules:
//   - every GPU that loads the library holds the arrays below (about 513 KB) until the process
//     exits, whether or not this entry point is used;
//   - all calls on a device share the same arrays: calls whose work overlaps on the GPU (for
//     example on two streams at once) race and give wrong reports; serialise them;
//   - the first call on each device resolves the arrays' device addresses. With CUDA's lazy
//     module loading (the default), that first use is also when the driver loads this library's
//     device code and places its arrays in device memory, so make the first call during set-up,
//     before streaming starts and before any stream capture on that device (or run with
//     CUDA_MODULE_LOADING=EAGER, which places them when the context is created). Later calls
//     allocate nothing.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "qrng_internal.h"

namespace {

constexpr int kNoallocMaxBits = 16;  // 2^16 codes + 1 out-of-range counter = 524,296 bytes
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device; the previous call's contents stay until the next
// call clears the counters (the histogram launcher zeroes them on the stream first).
static __device__ __align__(256) unsigned long long g_noalloc_hist[(1u << kNoallocMaxBits) + 1];
static __device__ __align__(256) qrng::DevHminResult g_noalloc_result;

struct DeviceScratch {
  bool ready = false;
  unsigned long long* hist = nullptr;       // device address of g_noalloc_hist
  qrng::DevHminResult* result = nullptr;    // device address of g_noalloc_result
  int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceScratch g_scratch[kMaxDevices];

// Once per device, with that device current: look up the arrays' device addresses. In host
// code the array names only denote host-side stand-ins, so kernels must be given these.
int setup_device(int dev, DeviceScratch* out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceScratch& d = g_scratch[dev];
  if (!d.ready) {
    void* h = nullptr;
    void* r = nullptr;
    if (cudaGetSymbolAddress(&h, g_noalloc_hist) != cudaSuccess) return QRNG_ECUDA;
    if (cudaGetSymbolAddress(&r, g_noalloc_result) != cudaSuccess) return QRNG_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QRNG_ECUDA;
    d.hist = static_cast<unsigned long long*>(h);
    d.result = static_cast<qrng::DevHminResult*>(r);
    d.num_sms = sms;
    d.ready = true;
  }
  *out = d;
  return QRNG_OK;
}

}  // namespace

extern "C" QRNG_API int qrng_minentropy_noalloc(const void* samples, uint64_t count, int bits, double eps,
                                                qrng_hmin_report* rep, qrng_stream_t stream) {
  if (!samples || !rep || count == 0) return QRNG_EINVAL;
  if (bits < 1 || bits > kNoallocMaxBits) return QRNG_EINVAL;  // more codes than the fixed histogram holds
  if (!(eps > 0.0 && eps < 1.0)) return QRNG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QRNG_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return QRNG_ENOTSUP;
  DeviceScratch sc;
  int st = setup_device(dev, &sc);
  if (st != QRNG_OK) return st;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t kernels = 0;
  if (qrng::launch_histogram(samples, count, bits, sc.hist, sc.num_sms, s, &kernels) != cudaSuccess) return QRNG_ECUDA;
  if (qrng::launch_hmin_finalize(sc.hist, bits, eps, sc.result, s, &kernels) != cudaSuccess) return QRNG_ECUDA;
  qrng::DevHminResult res;
  if (cudaMemcpyAsync(&res, sc.result, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess) return QRNG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QRNG_ECUDA;
  if (res.out_of_range) return QRNG_EINVAL;
  if (res.status != QRNG_OK) return res.status;
  *rep = res.rep;
  return QRNG_OK;
}
