// hy_dot_noalloc: a dot product of two device vectors that allocates no device memory.
//
// Who needs it: callers that must not allocate device memory once they are running -- code that
// runs after a framework has claimed the whole device budget for its own pool, real-time loops where
// a cudaMalloc/cudaFree could synchronise the device and stall, or hosts that forbid allocation after
// initialisation. hy_dot needs a context whose set-up allocates its scratch; this entry point needs
// neither a context nor an allocation.
//
// How: the per-block partial sums and the result live in one file-scope __device__ array of fixed
// size, which every GPU that loads this library holds until the process exits. Host code cannot use
// the array's name as a device address, so the first call on each device (with that device current)
// looks the address up with cudaGetSymbolAddress and keeps it; later calls reuse it. Make that first
// call before any stream capture begins.
//
// The array is shared by every call: each call writes every entry it reads (partials of its own
// blocks, then the result slot) before reading it, so nothing needs clearing, but two calls that
// overlap on the GPU (different streams, no ordering between them) race on the array and may return
// each other's values. Issue them on one stream, or order them.
#include <mutex>

#include "../../include/hyperelastic.h"

namespace {

constexpr int NA_TPB = 256;
constexpr int NA_PER_THREAD = 16;
constexpr long long NA_CHUNK = (long long)NA_TPB * NA_PER_THREAD;  // elements per block
constexpr int NA_MAX_BLOCKS = 16384;
static_assert((long long)NA_MAX_BLOCKS * NA_CHUNK == HY_DOT_NOALLOC_MAX_N, "limit in the header");
constexpr int NA_MAX_DEVICES = 64;

// NA_MAX_BLOCKS partial sums followed by the result slot: 16385 doubles = 128 KiB + 8 B per device.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS + 1];

__global__ void na_partial_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                  double* __restrict__ scratch) {
  __shared__ double sh[NA_TPB];
  const long long base = blockIdx.x * NA_CHUNK;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < NA_PER_THREAD; ++j) {
    const long long i = base + (long long)j * NA_TPB + threadIdx.x;
    if (i < n) s = fma(a[i], b[i], s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = NA_TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[blockIdx.x] = sh[0];
}

__global__ void na_final_kernel(double* __restrict__ scratch, int nblocks) {
  __shared__ double sh[NA_TPB];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += NA_TPB) s += scratch[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = NA_TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[NA_MAX_BLOCKS] = sh[0];
}

std::mutex g_mu;
double* g_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
hy_status scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HY_ERR_CUDA;
    g_ptr[device] = static_cast<double*>(p);
  }
  *out = g_ptr[device];
  return HY_OK;
}

}  // namespace

namespace {

hy_status dot_noalloc_on_current(int device, void* cuda_stream, const double* a_dev, const double* b_dev,
                                 int64_t n, double* result) {
  if (n == 0) {
    *result = 0.0;
    return HY_OK;
  }
  double* scratch = nullptr;
  const hy_status st = scratch_address(device, &scratch);
  if (st != HY_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nblocks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
  na_partial_kernel<<<nblocks, NA_TPB, 0, s>>>(a_dev, b_dev, (long long)n, scratch);
  na_final_kernel<<<1, NA_TPB, 0, s>>>(scratch, nblocks);
  if (cudaGetLastError() != cudaSuccess) return HY_ERR_CUDA;
  if (cudaMemcpyAsync(result, scratch + NA_MAX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return HY_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HY_ERR_CUDA;
  return HY_OK;
}

}  // namespace

// The call makes `device` current for its own launches and gives the calling thread back the device
// that was current on entry, on every return path.
extern "C" hy_status hy_dot_noalloc(int device, void* cuda_stream, const double* a_dev, const double* b_dev,
                                    int64_t n, double* result) {
  if (!a_dev || !b_dev || !result || n < 0) return HY_ERR_ARG;
  if (n > HY_DOT_NOALLOC_MAX_N) return HY_ERR_ARG;  // the partial sums would not fit the fixed array
  if (device < 0 || device >= NA_MAX_DEVICES) return HY_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return HY_ERR_CUDA;
  if (prev != device && cudaSetDevice(device) != cudaSuccess) return HY_ERR_CUDA;
  const hy_status st = dot_noalloc_on_current(device, cuda_stream, a_dev, b_dev, n, result);
  if (prev != device && cudaSetDevice(prev) != cudaSuccess) return st == HY_OK ? HY_ERR_CUDA : st;
  return st;
}
