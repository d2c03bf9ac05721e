// ap_lm_solve_noalloc: the damped LM solve of one parameter group for callers
// that may not allocate device memory.  Some callers cannot call cudaMalloc:
// code that runs while a CUDA graph is being captured (allocation is not a
// stream operation and is refused during capture), processes that work inside
// a fixed, pre-reserved device-memory budget, and plug-ins whose host
// application owns every device allocation.  This entry point takes its
// scratch from a fixed array in the library's device data segment instead.
//
// The array is a file-scope __device__ array, so every GPU that loads the
// library holds it (AP_NOALLOC_SCRATCH_DOUBLES doubles, 768 KiB) until the
// process exits.  Host code cannot use the array's name as a device address:
// every call made outside a stream capture asks the runtime for the address
// (with the call's device current; the first such call on a device also loads
// the module there) and remembers it per device; a call made while its stream
// is being captured uses the remembered address, so the first call on a
// device must come before any capture.  Asking again outside a capture keeps
// the address right after a device reset, which reloads the module.
#include <cuda_runtime.h>

#include <mutex>

#include "ap_internal.cuh"

namespace ap {

constexpr int NA_THREADS = 1024;
constexpr int NA_MAX_IT = 4000;
constexpr double NA_RTOL = 1e-11;
constexpr double NA_FLOOR = 1e-12;
constexpr int NA_RETRIES = 8;

// six vectors of AP_NOALLOC_MAX_N doubles: D, x, r, z, p, q
static __device__ __align__(256) double g_noalloc_scratch[AP_NOALLOC_SCRATCH_DOUBLES];

__device__ double na_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < NA_THREADS / 32; ++k) s += red[k];
  return s;
}

__device__ double na_block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < NA_THREADS / 32; ++k) s = fmax(s, red[k]);
  return s;
}

// y = (A + lam diag(D)) x, one warp per row (lanes stride the row's entries,
// a fixed shuffle tree sums them), then the row's pq contribution
__device__ double na_spmv(int n, const int64_t* row_ptr, const int32_t* col_idx, const double* vals, const double* D,
                          double lam, const double* x, double* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double pq = 0.0;
  for (int i = warp; i < n; i += NA_THREADS / 32) {
    double s = 0.0;
    for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) s += vals[e] * x[col_idx[e]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s += lam * D[i] * x[i];
    if (lane == 0) {
      y[i] = s;
      pq += x[i] * s;
    }
  }
  return pq;
}

// Jacobi-preconditioned conjugate gradients on (A + lam D) delta = b in one
// CTA, with the same damping, stopping rule and lambda retries as the
// per-group solver of ap_lm_solve().
__global__ void __launch_bounds__(NA_THREADS) noalloc_pcg_kernel(int n, const int64_t* __restrict__ row_ptr,
                                                                 const int32_t* __restrict__ col_idx,
                                                                 const double* __restrict__ vals,
                                                                 const double* __restrict__ b, double* lambda,
                                                                 double* delta, int* status, double* scratch) {
  __shared__ double red[32];
  double* D = scratch;
  double* x = D + AP_NOALLOC_MAX_N;
  double* r = x + AP_NOALLOC_MAX_N;
  double* z = r + AP_NOALLOC_MAX_N;
  double* p = z + AP_NOALLOC_MAX_N;
  double* q = p + AP_NOALLOC_MAX_N;
  const int tid = threadIdx.x;
  // diagonal (the last call's contents are overwritten, nothing is reused);
  // repeated entries of a position add up, as they do in the product below
  double dmax = 0.0, bn2 = 0.0;
  for (int i = tid; i < n; i += NA_THREADS) {
    double d = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col_idx[e] == i) d += vals[e];
    D[i] = d;
    dmax = fmax(dmax, d);
    bn2 += b[i] * b[i];
  }
  dmax = na_block_max(dmax, red);
  bn2 = na_block_sum(bn2, red);
  const double floor_v = dmax > 0.0 ? NA_FLOOR * dmax : 1.0;
  for (int i = tid; i < n; i += NA_THREADS) D[i] = fmax(D[i], floor_v);
  double lam = *lambda;
  int result = AP_ERR_NOT_SPD;
  for (int attempt = 0; attempt <= NA_RETRIES; ++attempt) {
    __syncthreads();
    double rz = 0.0;
    for (int i = tid; i < n; i += NA_THREADS) {
      x[i] = 0.0;
      r[i] = b[i];
      z[i] = b[i] / ((1.0 + lam) * D[i]);
      p[i] = z[i];
      rz += r[i] * z[i];
    }
    rz = na_block_sum(rz, red);
    const double rz0 = rz;
    bool conv = bn2 == 0.0 || rz0 == 0.0, bad = false;
    for (int it = 0; it < NA_MAX_IT && !conv; ++it) {
      __syncthreads();
      double pq = na_spmv(n, row_ptr, col_idx, vals, D, lam, p, q);
      pq = na_block_sum(pq, red);
      if (!(pq > 0.0)) { bad = true; break; }
      const double alpha = rz / pq;
      double rz2 = 0.0;
      for (int i = tid; i < n; i += NA_THREADS) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        z[i] = r[i] / ((1.0 + lam) * D[i]);
        rz2 += r[i] * z[i];
      }
      rz2 = na_block_sum(rz2, red);
      if (rz2 <= NA_RTOL * NA_RTOL * rz0) { conv = true; break; }
      const double beta = rz2 / rz;
      rz = rz2;
      for (int i = tid; i < n; i += NA_THREADS) p[i] = z[i] + beta * p[i];
    }
    __syncthreads();
    if (bad) { lam *= 10.0; continue; }
    result = conv ? AP_OK : AP_ERR_TIMEOUT;
    break;
  }
  for (int i = tid; i < n; i += NA_THREADS) delta[i] = result == AP_ERR_NOT_SPD ? 0.0 : x[i];
  if (tid == 0) {
    *lambda = lam;
    *status = result;
  }
}

}  // namespace ap

extern "C" int ap_lm_solve_noalloc(int n, const int64_t* row_ptr_dev, const int32_t* col_idx_dev,
                                   const double* vals_dev, const double* jtwr_dev, double* lambda_dev,
                                   double* delta_dev, int* status_dev, void* stream) {
  if (n < 1 || n > AP_NOALLOC_MAX_N) return AP_ERR_ARG;
  if (!row_ptr_dev || !col_idx_dev || !vals_dev || !jtwr_dev || !lambda_dev || !delta_dev || !status_dev)
    return AP_ERR_ARG;
  // the device address of the scratch array on the current device: asked
  // for outside a capture (cheap once the module is loaded, and right again
  // after a device reset), remembered for calls made during a capture
  static std::mutex mu;
  static void* scratch_of_device[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return AP_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return AP_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, ap::g_noalloc_scratch) != cudaSuccess || !p) return AP_ERR_CUDA;
      scratch_of_device[dev] = p;
    }
    scratch = scratch_of_device[dev];
  }
  if (!scratch) return AP_ERR_CUDA;   // first call on this device made during a capture
  // the launch's own status (not an error left on the thread by other work)
  void* args[] = {&n, (void*)&row_ptr_dev, (void*)&col_idx_dev, (void*)&vals_dev, (void*)&jtwr_dev,
                  (void*)&lambda_dev, (void*)&delta_dev, (void*)&status_dev, &scratch};
  const cudaError_t e = cudaLaunchKernel((const void*)ap::noalloc_pcg_kernel, dim3(1), dim3(ap::NA_THREADS), args, 0,
                                         (cudaStream_t)stream);
  return e == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}
