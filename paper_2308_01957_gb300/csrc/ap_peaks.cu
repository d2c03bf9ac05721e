// Throughput probes of the arithmetic pipes the path's kernels are bound by,
// so that their roofline fractions divide by measured rates rather than unit
// counts times a nominal clock: float32 FMA, the special-function unit
// (ex2 / lg2, as the profile math uses them), float64 FMA and the warp-level
// TF32 MMA.  Each probe runs independent dependency chains per thread so the
// pipe, not latency, is the limit; one CTA of 256 threads per block slot.
#include <cuda_runtime.h>

#include "ap_internal.cuh"

namespace ap {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) peak_fma32_kernel(int iters, float* out) {
  float a[PK_CHAINS];
  const float m = 1.0f + 1e-7f * threadIdx.x, c = 1e-9f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == 1234.5f) out[blockIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(PK_THREADS) peak_fma64_kernel(int iters, double* out) {
  double a[PK_CHAINS];
  const double m = 1.0 + 1e-15 * threadIdx.x, c = 1e-18;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == 1234.5) out[blockIdx.x] = s;
}

// one ex2 and one lg2 per chain step: x -> ex2(lg2(x) * 0.999) stays finite
__global__ void __launch_bounds__(PK_THREADS) peak_xu_kernel(int iters, float* out) {
  float a[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = 1.5f + 0.001f * (threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) {
        float l, e;
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(a[k]));
        l *= 0.999f;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(l));
        a[k] = e + 1.0f;
      }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == 1234.5f) out[blockIdx.x] = s;
}

// mma.sync m16n8k8 TF32 with four independent accumulators per warp
__global__ void __launch_bounds__(PK_THREADS) peak_mma_tf32_kernel(int iters, float* out) {
  float d[4][4] = {};
  uint32_t a0 = __float_as_uint(1.0f + threadIdx.x * 1e-3f), a1 = a0 ^ 0x100u, a2 = a0 ^ 0x200u, a3 = a0 ^ 0x300u;
  uint32_t b0 = __float_as_uint(0.5f), b1 = b0 ^ 0x100u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};"
                     : "+f"(d[k][0]), "+f"(d[k][1]), "+f"(d[k][2]), "+f"(d[k][3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1] + d[k][2] + d[k][3];
  if (s == 1234.5f) out[blockIdx.x] = s;
}

}  // namespace ap

extern "C" int ap_measure_pipe(int kind, int iters, double* ms, double* ops, void* stream) {
  if (kind < AP_PIPE_FMA32 || kind > AP_PIPE_MMA_TF32 || iters < 1 || iters > (1 << 24) || !ms || !ops)
    return AP_ERR_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  void* fn = nullptr;
  switch (kind) {
    case AP_PIPE_FMA32: fn = (void*)ap::peak_fma32_kernel; break;
    case AP_PIPE_XU: fn = (void*)ap::peak_xu_kernel; break;
    case AP_PIPE_FMA64: fn = (void*)ap::peak_fma64_kernel; break;
    default: fn = (void*)ap::peak_mma_tf32_kernel; break;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ap::PK_THREADS, 0) != cudaSuccess || per_sm < 1)
    return AP_ERR_CUDA;
  const int blocks = sms * per_sm;
  void* out = nullptr;
  if (cudaMallocAsync(&out, (size_t)blocks * sizeof(double), st) != cudaSuccess) return AP_ERR_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void* args[] = {&iters, &out};
  // one launch to warm up, one timed
  cudaLaunchKernel(fn, dim3(blocks), dim3(ap::PK_THREADS), args, 0, st);
  cudaEventRecord(e0, st);
  cudaLaunchKernel(fn, dim3(blocks), dim3(ap::PK_THREADS), args, 0, st);
  cudaEventRecord(e1, st);
  const cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return AP_ERR_CUDA;
  const double threads = (double)blocks * ap::PK_THREADS;
  double per_thread = 0.0;
  switch (kind) {
    case AP_PIPE_FMA32:
    case AP_PIPE_FMA64: per_thread = 2.0 * 16 * ap::PK_CHAINS * (double)iters; break;   // flops
    case AP_PIPE_XU: per_thread = 2.0 * 8 * ap::PK_CHAINS * (double)iters; break;       // ex2 + lg2
    default: per_thread = 2.0 * 16 * 8 * 8 * 8 * 4 * (double)iters / 32.0; break;      // flops per warp / 32
  }
  *ms = t;
  *ops = threads * per_thread;
  return AP_OK;
}
