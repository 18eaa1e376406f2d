// Test helper (not part of the library): raw outputs of cuRAND's
// Philox4_32_10 device generator, run as a black box so that the oracle's
// Philox4x32-10 can be compared with an implementation it shares nothing with.
#include <cstdint>

#include <curand_kernel.h>

__global__ void philox_raw(const unsigned long long* seeds, const unsigned long long* subseq,
                           const unsigned long long* offsets, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seeds[i], subseq[i], offsets[i], &st);
  out[i] = curand4(&st);
}

// Device pointers; returns the cudaError_t of the launch and synchronisation.
extern "C" int curand_philox_raw(const unsigned long long* seeds, const unsigned long long* subseq,
                                 const unsigned long long* offsets, void* out, int n) {
  if (n <= 0) return 0;
  philox_raw<<<(n + 127) / 128, 128>>>(seeds, subseq, offsets, static_cast<uint4*>(out), n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}
