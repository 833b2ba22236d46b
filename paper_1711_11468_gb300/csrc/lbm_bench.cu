// Bandwidth micro-benchmarks of Sec. 4.1, GPU counterparts: copy-19 copies 19
// arrays concurrently (19 read and 19 write streams), update-19 updates 19
// arrays in place. They give the "adjusted" roofline bandwidth for the two-grid
// and the in-place sweeps. Bitwise integer work so any element size is valid.
// fma64 measures the FP64 pipe, the bound of the FP64 sweep on this GPU.
#include "lbm_async.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_copy19(const T* __restrict__ src, T* __restrict__ dst, int64_t n,
                                                int64_t stride) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T v[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) v[i] = __ldcs(src + i * stride + e);
#pragma unroll
    for (int i = 0; i < 19; ++i) __stcs(dst + i * stride + e, v[i]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_update19(T* __restrict__ buf, int64_t n, int64_t stride) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T v[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) v[i] = __ldcs(buf + i * stride + e);
#pragma unroll
    for (int i = 0; i < 19; ++i) __stcs(buf + i * stride + e, (T)(v[i] + (T)1));
  }
}

// One CTA arms an mbarrier for 16 bytes that no copy will deliver and waits
// for at most `polls` polls: the bounded-wait path of the staged sweeps, run
// on purpose. It must give up, set the status bit and return.
__global__ void k_wait_selftest(uint32_t polls, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0, polls) && threadIdx.x == 0) atomicOr(status, kStatusWaitTimeout);
}

// FP64 pipe throughput: sixteen independent chains of fused multiply-adds per
// thread (each 2 flops); the sums go to out[] so nothing is optimised away.
__global__ void __launch_bounds__(256) k_fma64(double* __restrict__ out, int iterations) {
  double a[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const double b = 0.9999999, c = 1e-7;
  for (int it = 0; it < iterations; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = fma(a[k], b, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) sum += a[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

unsigned grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int64_t cap = (int64_t)sms * 8;   // 8 resident blocks of 256 per SM
  return (unsigned)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

cudaError_t launch_copy19(const void* src, void* dst, int64_t n, int64_t stride, int elem, cudaStream_t s) {
  const unsigned g = grid_for(n);
  switch (elem) {
    case 8: k_copy19<unsigned long long><<<g, 256, 0, s>>>((const unsigned long long*)src, (unsigned long long*)dst, n, stride); break;
    case 4: k_copy19<unsigned int><<<g, 256, 0, s>>>((const unsigned int*)src, (unsigned int*)dst, n, stride); break;
    case 2: k_copy19<unsigned short><<<g, 256, 0, s>>>((const unsigned short*)src, (unsigned short*)dst, n, stride); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int fma64_wave_blocks() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma64, 256, 0);
  return std::max(1, sms) * std::max(1, per_sm);
}

cudaError_t launch_fma64(double* out, int blocks, int iterations, cudaStream_t s) {
  k_fma64<<<blocks, 256, 0, s>>>(out, iterations);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint32_t polls, int* status, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(polls, status);
  return cudaGetLastError();
}

cudaError_t launch_update19(void* buf, int64_t n, int64_t stride, int elem, cudaStream_t s) {
  const unsigned g = grid_for(n);
  switch (elem) {
    case 8: k_update19<unsigned long long><<<g, 256, 0, s>>>((unsigned long long*)buf, n, stride); break;
    case 4: k_update19<unsigned int><<<g, 256, 0, s>>>((unsigned int*)buf, n, stride); break;
    case 2: k_update19<unsigned short><<<g, 256, 0, s>>>((unsigned short*)buf, n, stride); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
