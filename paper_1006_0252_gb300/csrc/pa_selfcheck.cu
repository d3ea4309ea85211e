// pa_selfcheck.cu -- the device Philox4x32-10 (both forms the kernels use)
// against cuRAND's Philox4_32_10 generator, run on the device.
//
// After curand_init(seed, subsequence, 4 m), the first curand4 is
// Philox4x32-10 of the counter (m lo, m hi, subsequence lo, subsequence hi)
// under the key (seed lo, seed hi) (the generator's documented layout:
// subsequences advance the upper 64 counter bits, offsets of 4 draws the
// lower), so it must equal philox10(m lo, m hi, s lo, s hi, seed lo, seed hi)
// and philox10_rk with the round keys of the seed.
#include <curand_kernel.h>

#include "pa_device.cuh"
#include "pa_gauss.cuh"

namespace pa {

__global__ void k_check_philox(int64_t n, uint64_t seed0, unsigned long long* __restrict__ mismatches) {
  unsigned long long bad = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // the seed, subsequence and offset of draw i from the generator itself
    const u32x4 h = philox10((uint32_t)i, (uint32_t)(i >> 32), 0x53454C46u, 0x43484B21u,
                             (uint32_t)seed0, (uint32_t)(seed0 >> 32));
    const uint64_t seed = ((uint64_t)h.a << 32) | h.b;
    const uint64_t sub = ((uint64_t)h.c << 32) | (h.d & 0xFFFFu);  // up to 2^48 subsequences
    const uint32_t m = h.d >> 16;                                    // offset 4 m
    curandStatePhilox4_32_10_t st;
    curand_init(seed, sub, 4ull * m, &st);
    const uint4 ref = curand4(&st);
    const u32x4 a = philox10(m, 0u, (uint32_t)sub, (uint32_t)(sub >> 32), (uint32_t)seed, (uint32_t)(seed >> 32));
    const RoundKeys rk = make_round_keys(seed);
    const u32x4 b = philox10_rk(m, 0u, (uint32_t)sub, (uint32_t)(sub >> 32), rk);
    if (a.a != ref.x || a.b != ref.y || a.c != ref.z || a.d != ref.w) bad += 1ull;
    if (b.a != ref.x || b.b != ref.y || b.c != ref.z || b.d != ref.w) bad += 1ull;
  }
#pragma unroll
  for (int sh = 16; sh >= 1; sh >>= 1) bad += __shfl_xor_sync(0xFFFFFFFFu, bad, sh);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mismatches, bad);
}

cudaError_t launch_check_philox(int64_t n, uint64_t seed, unsigned long long* mismatches) {
  k_check_philox<<<152 * 4, 256>>>(n, seed, mismatches);
  return cudaGetLastError();
}

// The integer thresholds of the Gaussian decision (pa_gauss.cuh), one per
// energy change, as the threshold-table kernels compute them.
__global__ void k_gauss_thresholds(int64_t n, double beta, const int32_t* __restrict__ dE,
                                   uint32_t* __restrict__ thr) {
  const float beta_f = __double2float_rn(beta);  // as the sweep kernels round beta'
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    thr[i] = gauss_threshold(dE[i], beta_f);
}

cudaError_t launch_gauss_thresholds(int64_t n, double beta, const int32_t* dE, uint32_t* thr) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
  k_gauss_thresholds<<<blocks, 256>>>(n, beta, dE, thr);
  return cudaGetLastError();
}

}  // namespace pa
