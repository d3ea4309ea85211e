// pa_noalloc.cu -- bootstrap errors without any device allocation.
//
// pa_bootstrap stages its inputs and its per-resample results in memory it
// allocates with cudaMallocAsync.  Some callers cannot allow that: code that
// has handed all device memory to its own pool or to another framework and
// must not take memory behind that pool's back, latency-critical loops that
// must not pay for (or risk failing) an allocation while a run is live, and
// embedded or certified deployments where device memory is fixed at start-up.
// pa_bootstrap_noalloc serves them: the caller passes device inputs and a
// device output, and the per-resample scratch is a file-scope device array
// of fixed size that every GPU which loads this library holds until exit.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "pa_engine.h"

// Scratch: per-resample weighted mean [0, B) and -beta F-bar [B, 2B).
static __device__ __align__(256) double g_boot_scratch[2 * PA_BOOTSTRAP_NOALLOC_MAX_B];

// One block: sample standard deviation (ddof 1) of the B resample values of
// each of the two quantities; out[0] = std of the mean, out[1] = std of -beta F-bar.
__global__ void __launch_bounds__(256) k_boot_std(const double* __restrict__ vals, int B,
                                                  double* __restrict__ out) {
  __shared__ double s_part[256 / 32];
  for (int q = 0; q < 2; ++q) {
    const double* v = vals + q * PA_BOOTSTRAP_NOALLOC_MAX_B;
    double acc = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) acc += v[b];
    for (int sh = 16; sh >= 1; sh >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, sh);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    double mean = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mean += s_part[w];
    mean /= (double)B;
    __syncthreads();
    double ss = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) ss += (v[b] - mean) * (v[b] - mean);
    for (int sh = 16; sh >= 1; sh >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, sh);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
      out[q] = sqrt(t / (double)(B - 1));
    }
    __syncthreads();
  }
}

// Device address of the scratch array, looked up once per device and kept for
// the life of the process (a cudaDeviceReset of a device this library has
// used is not supported, see pa.h).
static std::mutex g_scratch_mu;
static double* g_scratch_ptr[64];

static cudaError_t scratch_address(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_boot_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double*)p;
  }
  *ptr = g_scratch_ptr[dev];
  return cudaSuccess;
}

extern "C" int pa_bootstrap_noalloc(int M, const double* x_dev, const double* A_dev, const double* R_dev,
                                    int B, uint64_t seed, double* out_dev, void* stream) {
  if (M < 1 || !x_dev || !out_dev) return PA_ERR_INVALID;
  if (B < 2 || B > PA_BOOTSTRAP_NOALLOC_MAX_B) return PA_ERR_INVALID;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return PA_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // every one of the 2B scratch entries read below is written first by this
  // call, so nothing has to be cleared
  if (pa::launch_bootstrap(M, x_dev, A_dev, R_dev, B, seed, scratch, scratch + PA_BOOTSTRAP_NOALLOC_MAX_B, st) !=
      cudaSuccess)
    return PA_ERR_CUDA;
  k_boot_std<<<1, 256, 0, st>>>(scratch, B, out_dev);
  if (cudaGetLastError() != cudaSuccess) return PA_ERR_CUDA;
  return PA_OK;
}
