// Damped float64 solve of the Levenberg-Marquardt step and the on-device
// accept / reject (Sec. "Optimization methods": Marquardt 1963, Transtrum &
// Sethna 2012, Gavin 2022; the step never meets a singular matrix).
//
// Per group g with parameters gp[0..n):
//   M = (J^T W J)_gg + lambda_g diag(D),  D = diag(J^T W J)_gg floored at
//   1e-12 max(D); solve M delta = (J^T W r)_g.
// A failed factorisation (or a non-positive curvature p^T M p in CG) raises
// lambda_g x10 and retries, at most 8 times; then the status word gets
// AP_ERR_NOT_SPD and delta_g = 0.
#include "ap_internal.cuh"

namespace ap {

constexpr int CHOL_THREADS = 256;
constexpr int PCG_THREADS = 1024;
constexpr int LM_RETRIES = 8;
constexpr double DIAG_FLOOR = 1e-12;
constexpr int PCG_MAX_IT = 4000;
constexpr double PCG_RTOL = 1e-12;

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < nw; ++k) s += red[k];
  return s;
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < nw; ++k) s = fmax(s, red[k]);
  return s;
}

// ---------------------------------------------------------------------------
// dense Cholesky, one CTA per small group; matrix in shared memory
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CHOL_THREADS) chol_kernel(const GroupDev* __restrict__ groups, int n_groups,
                                                            const int* __restrict__ gparams,
                                                            const int* __restrict__ plocal,
                                                            const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col_idx,
                                                            const double* __restrict__ vals,
                                                            const double* __restrict__ jtwr, double* lambda,
                                                            double* delta, int max_n, int* status) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ int fail;
  const int g = blockIdx.x;
  const GroupDev G = groups[g];
  if (!G.dense) return;
  const int n = G.n;
  const int* gp = gparams + G.p0;
  double* A = sm;               // n x n damped copy
  double* A0 = A + max_n * max_n;   // n x n original
  double* D = A0 + max_n * max_n;   // n
  double* y = D + max_n;            // n
  const int tid = threadIdx.x;
  for (int idx = tid; idx < n * n; idx += blockDim.x) A0[idx] = 0.0;
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) {
    const int pr = gp[r];
    for (int64_t e = row_ptr[pr]; e < row_ptr[pr + 1]; ++e) {
      const int lc = plocal[col_idx[e]];
      if (lc >= 0 && lc < n) A0[r * n + lc] = vals[e];
    }
  }
  __syncthreads();
  double dmax = 0.0;
  for (int r = tid; r < n; r += blockDim.x) dmax = fmax(dmax, A0[r * n + r]);
  dmax = block_max(dmax, red);
  const double floor_v = dmax > 0.0 ? DIAG_FLOOR * dmax : 1.0;
  for (int r = tid; r < n; r += blockDim.x) D[r] = fmax(A0[r * n + r], floor_v);
  double lam = lambda[g];
  bool ok = false;
  for (int attempt = 0; attempt <= LM_RETRIES; ++attempt) {
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx - r * n;
      A[idx] = A0[idx] + (r == c ? lam * D[r] : 0.0);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    // right-looking column Cholesky, lower triangle
    for (int k = 0; k < n; ++k) {
      if (tid == 0) {
        const double d = A[k * n + k];
        if (!(d > 0.0) || !isfinite(d)) fail = 1;
        else A[k * n + k] = sqrt(d);
      }
      __syncthreads();
      if (fail) break;
      const double lkk = A[k * n + k];
      for (int r = k + 1 + tid; r < n; r += blockDim.x) A[r * n + k] /= lkk;
      __syncthreads();
      const int m = n - k - 1;
      for (int idx = tid; idx < m * m; idx += blockDim.x) {
        const int r = k + 1 + idx / m, c = k + 1 + idx % m;
        if (c <= r) A[r * n + c] -= A[r * n + k] * A[c * n + k];
      }
      __syncthreads();
    }
    if (!fail) { ok = true; break; }
    lam *= 10.0;
  }
  __syncthreads();
  if (!ok) {
    for (int r = tid; r < n; r += blockDim.x) delta[gp[r]] = 0.0;
    if (tid == 0) { atomicCAS(status, 0, AP_ERR_NOT_SPD); lambda[g] = lam; }
    return;
  }
  // forward and back substitution (one thread: n <= 64)
  if (tid == 0) {
    for (int r = 0; r < n; ++r) {
      double s = jtwr[gp[r]];
      for (int c = 0; c < r; ++c) s -= A[r * n + c] * y[c];
      y[r] = s / A[r * n + r];
    }
    for (int r = n - 1; r >= 0; --r) {
      double s = y[r];
      for (int c = r + 1; c < n; ++c) s -= A[c * n + r] * y[c];
      y[r] = s / A[r * n + r];
    }
    lambda[g] = lam;
  }
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) delta[gp[r]] = y[r];
}

// ---------------------------------------------------------------------------
// block-Jacobi preconditioned conjugate gradients, one CTA per large group.
// Preconditioner blocks (<= 8 consecutive local indices) are factorised once
// per attempt; vectors live in the work buffer (5 n doubles per group).
// ---------------------------------------------------------------------------
__device__ void spmv_damped(const int* gp, const int* plocal, const int64_t* row_ptr, const int32_t* col_idx,
                            const double* vals, const double* D, double lam, const double* x, double* y, int n) {
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int pr = gp[r];
    double s = lam * D[r] * x[r];
    for (int64_t e = row_ptr[pr]; e < row_ptr[pr + 1]; ++e) {
      const int lc = plocal[col_idx[e]];
      s += vals[e] * x[lc];
    }
    y[r] = s;
  }
}

__global__ void __launch_bounds__(PCG_THREADS) pcg_kernel(const GroupDev* __restrict__ groups, int n_groups,
                                                          const int* __restrict__ gparams,
                                                          const int* __restrict__ plocal,
                                                          const int* __restrict__ blk_ptr,
                                                          const int64_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ col_idx,
                                                          const double* __restrict__ vals,
                                                          const double* __restrict__ jtwr, double* lambda,
                                                          double* delta, double* work, double* blk_work,
                                                          int* status) {
  __shared__ double red[32];
  __shared__ int fail;
  const int g = blockIdx.x;
  const GroupDev G = groups[g];
  if (G.dense) return;
  const int n = G.n;
  const int* gp = gparams + G.p0;
  const int* bp = blk_ptr + G.b0;
  double* D = work + (int64_t)6 * G.p0;
  double* x = D + n;
  double* r = x + n;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* Linv = blk_work + (int64_t)64 * G.b0;  // 8x8 factor per block
  const int tid = threadIdx.x;
  double dmax = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    const int pr = gp[i];
    double d = 0.0;
    for (int64_t e = row_ptr[pr]; e < row_ptr[pr + 1]; ++e)
      if (col_idx[e] == pr) d = vals[e];
    D[i] = d;
    dmax = fmax(dmax, d);
  }
  dmax = block_max(dmax, red);
  const double floor_v = dmax > 0.0 ? DIAG_FLOOR * dmax : 1.0;
  for (int i = tid; i < n; i += blockDim.x) D[i] = fmax(D[i], floor_v);
  double bnorm2 = 0.0;
  for (int i = tid; i < n; i += blockDim.x) bnorm2 += jtwr[gp[i]] * jtwr[gp[i]];
  bnorm2 = block_sum(bnorm2, red);
  double lam = lambda[g];
  bool ok = false;
  for (int attempt = 0; attempt <= LM_RETRIES && !ok; ++attempt) {
    __syncthreads();
    if (tid == 0) fail = 0;
    __syncthreads();
    // factorise the damped diagonal blocks: one thread per block
    for (int b = tid; b < G.nblk; b += blockDim.x) {
      const int s0 = bp[b], m = bp[b + 1] - bp[b];
      double L[64];
      for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) {
          const int pr = gp[s0 + a], pc = gp[s0 + c];
          double v = 0.0;
          for (int64_t e = row_ptr[pr]; e < row_ptr[pr + 1]; ++e)
            if (col_idx[e] == pc) { v = vals[e]; break; }
          if (a == c) v += lam * D[s0 + a];
          L[a * 8 + c] = v;
        }
      bool bok = true;
      for (int k = 0; k < m && bok; ++k) {
        double d = L[k * 8 + k];
        for (int t = 0; t < k; ++t) d -= L[k * 8 + t] * L[k * 8 + t];
        if (!(d > 0.0)) { bok = false; break; }
        d = sqrt(d);
        L[k * 8 + k] = d;
        for (int rr = k + 1; rr < m; ++rr) {
          double v = L[rr * 8 + k];
          for (int t = 0; t < k; ++t) v -= L[rr * 8 + t] * L[k * 8 + t];
          L[rr * 8 + k] = v / d;
        }
      }
      if (!bok) fail = 1;
      double* dst = Linv + (int64_t)64 * b;
      for (int t = 0; t < 64; ++t) dst[t] = L[t];
    }
    __syncthreads();
    if (fail) { lam *= 10.0; continue; }
    // x = 0, r = b, z = M^-1 r, p = z
    for (int i = tid; i < n; i += blockDim.x) { x[i] = 0.0; r[i] = jtwr[gp[i]]; }
    __syncthreads();
    auto precond = [&](const double* in, double* out) {
      for (int b = tid; b < G.nblk; b += blockDim.x) {
        const int s0 = bp[b], m = bp[b + 1] - bp[b];
        const double* L = Linv + (int64_t)64 * b;
        double y[8];
        for (int a = 0; a < m; ++a) {
          double v = in[s0 + a];
          for (int t = 0; t < a; ++t) v -= L[a * 8 + t] * y[t];
          y[a] = v / L[a * 8 + a];
        }
        for (int a = m - 1; a >= 0; --a) {
          double v = y[a];
          for (int t = a + 1; t < m; ++t) v -= L[t * 8 + a] * y[t];
          y[a] = v / L[a * 8 + a];
        }
        for (int a = 0; a < m; ++a) out[s0 + a] = y[a];
      }
    };
    precond(r, z);
    __syncthreads();
    double rz = 0.0;
    for (int i = tid; i < n; i += blockDim.x) { p[i] = z[i]; rz += r[i] * z[i]; }
    rz = block_sum(rz, red);
    bool conv = bnorm2 == 0.0;
    for (int it = 0; it < PCG_MAX_IT && !conv; ++it) {
      __syncthreads();
      spmv_damped(gp, plocal, row_ptr, col_idx, vals, D, lam, p, q, n);
      __syncthreads();
      double pq = 0.0;
      for (int i = tid; i < n; i += blockDim.x) pq += p[i] * q[i];
      pq = block_sum(pq, red);
      if (!(pq > 0.0)) { if (tid == 0) fail = 1; break; }
      const double alpha = rz / pq;
      double rr = 0.0;
      for (int i = tid; i < n; i += blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        rr += r[i] * r[i];
      }
      rr = block_sum(rr, red);
      if (rr <= PCG_RTOL * PCG_RTOL * bnorm2) { conv = true; break; }
      __syncthreads();
      precond(r, z);
      __syncthreads();
      double rz2 = 0.0;
      for (int i = tid; i < n; i += blockDim.x) rz2 += r[i] * z[i];
      rz2 = block_sum(rz2, red);
      const double beta = rz2 / rz;
      rz = rz2;
      for (int i = tid; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
    }
    __syncthreads();
    if (fail) { lam *= 10.0; continue; }
    if (!conv && tid == 0) atomicCAS(status, 0, AP_ERR_TIMEOUT);
    ok = true;
  }
  __syncthreads();
  if (!ok) {
    for (int i = tid; i < n; i += blockDim.x) delta[gp[i]] = 0.0;
    if (tid == 0) atomicCAS(status, 0, AP_ERR_NOT_SPD);
  } else {
    for (int i = tid; i < n; i += blockDim.x) delta[gp[i]] = x[i];
  }
  if (tid == 0) lambda[g] = lam;
}

static int g_max_dense = 1;

void configure_solve(int max_dense_n) {
  g_max_dense = max_dense_n < 1 ? 1 : max_dense_n;
  const size_t sm = (size_t)(2 * g_max_dense * g_max_dense + 2 * g_max_dense) * sizeof(double);
  cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

void launch_lm_solve(const GroupDev* groups, int n_groups, const int* gparams, const int* plocal,
                     const int* blk_ptr, const int64_t* row_ptr, const int32_t* col_idx, const double* vals,
                     const double* jtwr, double* lambda, double* delta, double* work, double* blk_work,
                     int max_dense_n, int* status, cudaStream_t st, int any_dense, int any_pcg) {
  if (n_groups <= 0) return;
  if (any_dense) {
    const size_t sm = (size_t)(2 * max_dense_n * max_dense_n + 2 * max_dense_n) * sizeof(double);
    chol_kernel<<<n_groups, CHOL_THREADS, sm, st>>>(groups, n_groups, gparams, plocal, row_ptr, col_idx, vals, jtwr,
                                                    lambda, delta, max_dense_n, status);
  }
  if (any_pcg)
    pcg_kernel<<<n_groups, PCG_THREADS, 0, st>>>(groups, n_groups, gparams, plocal, blk_ptr, row_ptr, col_idx, vals,
                                                 jtwr, lambda, delta, work, blk_work, status);
}

// ---------------------------------------------------------------------------
// trial point and accept / reject
// ---------------------------------------------------------------------------
__global__ void trial_kernel(const double* theta, const double* delta, const double* lo, const double* hi,
                             double* trial, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) trial[p] = fmin(fmax(theta[p] + delta[p], lo[p]), hi[p]);
}

void launch_trial(const double* theta, const double* delta, const double* lo, const double* hi, double* trial, int n,
                  cudaStream_t st) {
  if (n > 0) trial_kernel<<<(n + 255) / 256, 256, 0, st>>>(theta, delta, lo, hi, trial, n);
}

constexpr double LAMBDA_DOWN = 9.0, LAMBDA_UP = 11.0, LAMBDA_MIN = 1e-12, LAMBDA_MAX = 1e12;

__global__ void accept_groups_kernel(const double* chi2_now, const double* chi2_trial, double* lambda,
                                     double* chi2_state, double* log, int* accepted, int n_groups) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const double c0 = chi2_now[g], c1 = chi2_trial[g];
  const int acc = isfinite(c1) && c1 < c0;
  double lam = lambda[g];
  lam = acc ? fmax(lam / LAMBDA_DOWN, LAMBDA_MIN) : fmin(lam * LAMBDA_UP, LAMBDA_MAX);
  lambda[g] = lam;
  accepted[g] = acc;
  chi2_state[g] = acc ? c1 : c0;
  if (log) {
    log[4 * g + 0] = c0;
    log[4 * g + 1] = c1;
    log[4 * g + 2] = lam;
    log[4 * g + 3] = acc;
  }
}

__global__ void accept_params_kernel(const int* param_group, int n_params, const int* accepted, double* theta,
                                     const double* trial) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_params) return;
  const int g = param_group[p];
  if (g >= 0 && accepted[g]) theta[p] = trial[p];
}

void launch_accept_groups(const double* chi2_now, const double* chi2_trial, double* lambda, double* chi2_state,
                          double* log, int* accepted, int n_groups, cudaStream_t st) {
  if (n_groups > 0)
    accept_groups_kernel<<<(n_groups + 255) / 256, 256, 0, st>>>(chi2_now, chi2_trial, lambda, chi2_state, log,
                                                                 accepted, n_groups);
}

void launch_accept_params(const int* param_group, int n_params, const int* accepted, double* theta,
                          const double* trial, cudaStream_t st) {
  if (n_params > 0)
    accept_params_kernel<<<(n_params + 255) / 256, 256, 0, st>>>(param_group, n_params, accepted, theta, trial);
}

__global__ void scale_kernel(const double* in, double* out, double s, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = s * in[p];
}

void launch_scale(const double* in, double* out, double s, int n, cudaStream_t st) {
  if (n > 0) scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(in, out, s, n);
}

}  // namespace ap
