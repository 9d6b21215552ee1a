// Allocation-free misfit: tp_misfit_noalloc (see include/tprobe.h).
//
// Some callers cannot allocate device memory at the point where they need
// the data misfit of a shot record: code that receives all of its device
// memory from a host framework's own pool and may not allocate on its own,
// or a latency-critical loop in which an allocation, and the device
// synchronisation it can bring, is not acceptable.  For them this entry point
// computes J = 1/2 sum (d_syn - d_obs)^2 with its scratch space (one fp64
// partial sum per chunk of the records) in a fixed array of this file,
// instead of the caller-provided workspace the other entry points use.
//
// The array lives in every GPU that loads the library, until the process
// exits.  Host code must not pass the array's name to a kernel: in host code
// it is only a stand-in for the symbol.  The device address comes from
// cudaGetSymbolAddress with the calling device current: on every call made
// outside stream capture, and from the last such call during capture (so the
// first call on a device must come before any capture).  Every call
// overwrites the partials it uses before reading them, so nothing has to
// start at zero; calls that overlap on the GPU (for example on two streams)
// race on the array.
#include <cstdio>
#include <mutex>

#include "tp_internal.h"
#include "tprobe.h"

namespace tp {

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 65536;       // samples reduced by one block
constexpr int NA_MAX_CHUNKS = 4096;         // partial sums the array holds

static __device__ __align__(256) double g_noalloc_partials[NA_MAX_CHUNKS];

__device__ __forceinline__ double na_block_sum(double v) {
  __shared__ double sh[NA_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < NA_THREADS / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// block b: partial[b] = sum over samples [b*CHUNK, (b+1)*CHUNK) of (d - dobs)^2
__global__ void __launch_bounds__(NA_THREADS) na_partial_kernel(const float* __restrict__ d,
                                                                 const float* __restrict__ dobs, long long n,
                                                                 double* partial) {
  const long long lo = blockIdx.x * NA_CHUNK, hi = min(n, lo + NA_CHUNK);
  double acc = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NA_THREADS) {
    const float r = d[i] - dobs[i];
    acc += (double)r * (double)r;
  }
  const double t = na_block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NA_THREADS) na_finalize_kernel(const double* partial, int nchunks, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nchunks; i += NA_THREADS) acc += partial[i];
  const double t = na_block_sum(acc);
  if (threadIdx.x == 0) *out = 0.5 * t;
}

// device address of g_noalloc_partials on each device.  Outside stream capture
// it is looked up again on every call (a cheap host call), so an address made
// stale by a device reset is never used; during capture the address cached by
// the last call outside capture on that device is used, because a lookup then
// could load the module inside the capture.
constexpr int NA_MAX_DEVICES = 64;
double* g_na_ptr[NA_MAX_DEVICES] = {};
std::mutex g_na_mutex;

cudaError_t na_scratch(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (cs == cudaStreamCaptureStatusNone || !g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // the current device is `dev`
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

tp_status na_fail(tp_status st, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
  set_last_error(buf);
  return st;
}

}  // namespace
}  // namespace tp

extern "C" {

tp_status tp_misfit_noalloc(const float* d_syn, const float* d_obs, int64_t n, double* misfit, void* stream) {
  using namespace tp;
  if (!d_syn || !d_obs || !misfit) return na_fail(TP_ERR_ARG, "tp_misfit_noalloc: NULL pointer");
  if (n < 1) return na_fail(TP_ERR_ARG, "tp_misfit_noalloc: n must be >= 1");
  if (n > NA_CHUNK * NA_MAX_CHUNKS)
    return na_fail(TP_ERR_ARG, "tp_misfit_noalloc: n exceeds the fixed scratch (268435456 samples at most)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  cudaError_t e = na_scratch(st, &scratch);
  if (e != cudaSuccess) return na_fail(TP_ERR_CUDA, "tp_misfit_noalloc: scratch lookup failed", e);
  const int nchunks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
  prof_before(4, st);
  na_partial_kernel<<<nchunks, NA_THREADS, 0, st>>>(d_syn, d_obs, n, scratch);
  na_finalize_kernel<<<1, NA_THREADS, 0, st>>>(scratch, nchunks, misfit);
  prof_after(4, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(TP_ERR_CUDA, "tp_misfit_noalloc: launch failed", e);
  return TP_OK;
}

}  // extern "C"
