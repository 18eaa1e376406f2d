// noalloc.cu -- an allocation-free variant of the weights + weighted update.
//
// Some callers cannot allocate device memory once they run: a real-time MPC
// loop (cudaMalloc / cudaFree may synchronise the device and take unbounded
// time, which a fixed-rate controller cannot absorb), or a host program whose
// device memory is entirely owned by another allocator or a fixed memory
// plan.  mppi_jump_update_noalloc serves them: the caller passes the rollout
// costs, the perturbations and the controls, and the kernels' scratch (the
// split-K partial sums, the chunk normalisers, the running minimum and the
// completion ticket) lives in a file-scope __device__ array of fixed size
// that every GPU loading this library holds until the process exits.
//
// Host code must not pass the array's name to a kernel (on the host it names
// a host-side stand-in, not device memory): the device address is looked up
// with cudaGetSymbolAddress once per device, with that device current, by the
// first call made on it.  Every call shares the array and leaves its contents
// behind; each call first clears the words that must start cleared.  Calls
// whose work overlaps on the GPU (on different streams, or from several host
// threads) race on the array and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace mj {
namespace {

constexpr size_t kScratchFloats = size_t(1) << 20;  // 4 MiB of scratch per device
constexpr int kCtlFloats = 64;                      // control words at the start
constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 4;                     // rollouts per thread in a block
constexpr int kNaChunk = kNaThreads * kNaPerThread;  // rollouts per block
constexpr int kNaRows = 8;                          // steps per block
constexpr int kMaxDevices = 64;
constexpr int kMaxGroups = 65535;                   // gridDim.y limit

static __device__ __align__(256) float g_update_scratch[kScratchFloats];

float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_update_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (float*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Running minimum of the costs (order key), one atomic per warp.
__global__ void __launch_bounds__(kNaThreads)
na_min_kernel(const float* __restrict__ costs, int K, uint32_t* __restrict__ key) {
  uint32_t best = kKeyEmpty;
  for (int k = blockIdx.x * kNaThreads + threadIdx.x; k < K; k += gridDim.x * kNaThreads) {
    float c = costs[k];
    if (!isfinite(c)) c = INFINITY;
    best = min(best, order_key(c));
  }
  best = __reduce_min_sync(0xffffffffu, best);
  if ((threadIdx.x & 31) == 0) atomicMin(key, best);
}

// Block (c, g): rollouts c*kNaChunk .. and steps g*kNaRows ..; the weights
// e_k = exp((rho - S~_k)/lambda) of its rollouts in registers, the partial
// sums N_c[j][i] = sum_k e_k delta[j][k][i] and (first step group) Z_c into
// the scratch; the last block to finish combines the chunks in order and
// updates U += alpha sum_c N_c / sum_c Z_c (Eq. 37 / 49, no shift).
template <int M>
__global__ void __launch_bounds__(kNaThreads)
na_update_kernel(const float* __restrict__ costs, const float* __restrict__ noise, int K, int T,
                 float inv_lam, float alpha, float* __restrict__ U, float* __restrict__ scratch) {
  __shared__ float sh_s[kNaThreads / 32], sh_c[kNaThreads / 32];
  __shared__ float red_s[kNaThreads / 32][M], red_c[kNaThreads / 32][M];
  __shared__ unsigned ticket;
  uint32_t* key = reinterpret_cast<uint32_t*>(scratch);
  unsigned* done = reinterpret_cast<unsigned*>(scratch) + 1;
  const int chunks = gridDim.x;
  float* partial = scratch + kCtlFloats;      // [chunks][T][M]
  float* zpart = partial + (size_t)chunks * T * M;  // [chunks]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t kv = __ldcg(key);
  const bool ok = kv < kKeyInf;
  const float rho = ok ? key_to_float(kv) : 0.0f;
  if (ok) {
    float e[kNaPerThread];
    float zs = 0.0f, zc = 0.0f;
#pragma unroll
    for (int t = 0; t < kNaPerThread; ++t) {
      const int k = blockIdx.x * kNaChunk + t * kNaThreads + tid;
      float c = k < K ? costs[k] : INFINITY;
      if (!isfinite(c)) c = INFINITY;
      e[t] = k < K ? expf((rho - c) * inv_lam) : 0.0f;
      two_sum_acc(zs, zc, e[t]);
    }
    if (blockIdx.y == 0) {
      const float z = block_sum2<kNaThreads>(zs, zc, sh_s, sh_c);
      if (tid == 0) zpart[blockIdx.x] = z;
    }
    const int j_end = min(T, (int)(blockIdx.y + 1) * kNaRows);
    for (int j = blockIdx.y * kNaRows; j < j_end; ++j) {
      float acc[M];
#pragma unroll
      for (int i = 0; i < M; ++i) acc[i] = 0.0f;
#pragma unroll
      for (int t = 0; t < kNaPerThread; ++t) {
        const int k = blockIdx.x * kNaChunk + t * kNaThreads + tid;
        if (k < K) {
#pragma unroll
          for (int i = 0; i < M; ++i) acc[i] = fmaf(e[t], noise[((size_t)j * K + k) * M + i], acc[i]);
        }
      }
      float cmp[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        cmp[i] = 0.0f;
        warp_sum2(acc[i], cmp[i]);
      }
      __syncthreads();
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          red_s[wid][i] = acc[i];
          red_c[wid][i] = cmp[i];
        }
      }
      __syncthreads();
      if (wid == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          float s = lane < kNaThreads / 32 ? red_s[lane][i] : 0.0f;
          float c = lane < kNaThreads / 32 ? red_c[lane][i] : 0.0f;
          warp_sum2(s, c);
          if (lane == 0) partial[((size_t)blockIdx.x * T + j) * M + i] = s + c;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    ticket = atomicAdd(done, 1u);
  }
  __syncthreads();
  if (ticket != gridDim.x * gridDim.y - 1) return;
  __threadfence();
  if (!ok) return;  // every cost non-finite: U is left unchanged
  float zs = 0.0f, zc = 0.0f;
  for (int c = tid; c < chunks; c += kNaThreads) two_sum_acc(zs, zc, __ldcg(zpart + c));
  const float Z = block_sum2<kNaThreads>(zs, zc, sh_s, sh_c);
  const int TM = T * M;
  for (int idx = tid; idx < TM; idx += kNaThreads) {
    float s = 0.0f, c = 0.0f;
    for (int ch = 0; ch < chunks; ++ch) two_sum_acc(s, c, __ldcg(partial + (size_t)ch * TM + idx));
    U[idx] = U[idx] + alpha * ((s + c) / Z);
  }
}

}  // namespace
}  // namespace mj

using namespace mj;

extern "C" mppi_status mppi_jump_update_noalloc(const float* costs, const float* noise, int32_t K,
                                                int32_t T, int32_t m, float lambda, float alpha,
                                                float* U, void* stream) {
  if (!costs || !noise || !U || K < 1 || T < 1 || (m != 1 && m != 4) || !(lambda > 0.0f) ||
      !std::isfinite(lambda) || !std::isfinite(alpha))
    return MPPI_EINVAL;
  const int chunks = (K + kNaChunk - 1) / kNaChunk;
  const int groups = (T + kNaRows - 1) / kNaRows;
  // the step groups are the grid's y dimension, which holds at most 65535
  // blocks: T <= 8 * 65535; checked before anything is enqueued
  if (groups > kMaxGroups) return MPPI_EINVAL;
  const size_t need = (size_t)kCtlFloats + (size_t)chunks * T * m + (size_t)chunks;
  if (need > kScratchFloats) return MPPI_ENOMEM;  // beyond the fixed scratch
  float* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return MPPI_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the running minimum starts at "empty", the ticket at zero
  if (cudaMemsetAsync(scratch, 0xff, sizeof(uint32_t), s) != cudaSuccess) return MPPI_ECUDA;
  if (cudaMemsetAsync(scratch + 1, 0, sizeof(unsigned), s) != cudaSuccess) return MPPI_ECUDA;
  const int min_blocks = (K + kNaThreads - 1) / kNaThreads < 1024 ? (K + kNaThreads - 1) / kNaThreads : 1024;
  na_min_kernel<<<min_blocks, kNaThreads, 0, s>>>(costs, K, reinterpret_cast<uint32_t*>(scratch));
  const float inv_lam = (float)(1.0 / (double)lambda);
  if (m == 4)
    na_update_kernel<4><<<dim3(chunks, groups), kNaThreads, 0, s>>>(costs, noise, K, T, inv_lam, alpha,
                                                                   U, scratch);
  else
    na_update_kernel<1><<<dim3(chunks, groups), kNaThreads, 0, s>>>(costs, noise, K, T, inv_lam, alpha,
                                                                   U, scratch);
  return cudaGetLastError() == cudaSuccess ? MPPI_OK : MPPI_ECUDA;
}
