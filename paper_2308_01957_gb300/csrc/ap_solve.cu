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
#include <cooperative_groups.h>

#include "ap_internal.cuh"

namespace cg = cooperative_groups;

namespace ap {

constexpr int CHOL_THREADS = 256;
constexpr int PCG_THREADS = 1024;
constexpr int LM_RETRIES = 8;
constexpr double DIAG_FLOOR = 1e-12;
constexpr int PCG_MAX_IT = 4000;
// stop when the preconditioned residual r^T M^-1 r has fallen by PCG_RTOL^2:
// invariant to the scaling of the parameters (fluxes vs positions)
constexpr double PCG_RTOL = 1e-11;

// Block reductions: warp shuffles, then warp 0 combines the warp partials
// with a fixed shuffle tree and broadcasts through shared memory (one warp
// does the float64 adds, not every thread).  red[] holds 33 doubles.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
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
  __shared__ double red[33];
  __shared__ int fail;
  const int g = blockIdx.x;
  const GroupDev G = groups[g];
  if (G.dense != 1) return;
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
// block-Jacobi preconditioned conjugate gradients, one CTA per group of up to
// PCG_SMEM_N parameters, vectors in shared memory.  Plans precomputed on the
// host: lcol[e] (group-local column of CSR entry e), dpos[p] (CSR position of
// row p's diagonal), bpos[64 b + 8 a + c] (position of entry (a, c) of
// preconditioner block b, -1 if structurally zero).
// ---------------------------------------------------------------------------
constexpr int PCG_SMEM_N = 2048;

// Factorise the damped block and store its explicit inverse (m x m, row
// stride 8): applying the preconditioner is then one small matrix-vector
// product with no float64 division.
__device__ bool factor_block(const int64_t* bpos, const double* vals, const double* D, int s0, int m, double lam,
                             double* dst) {
  double L[64];
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c) {
      const int64_t e = bpos[a * 8 + c];
      double v = e >= 0 ? vals[e] : 0.0;
      if (a == c) v += lam * D[s0 + a];
      L[a * 8 + c] = v;
    }
  double inv_d[8];
  for (int k = 0; k < m; ++k) {
    double d = L[k * 8 + k];
    for (int t = 0; t < k; ++t) d -= L[k * 8 + t] * L[k * 8 + t];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    inv_d[k] = 1.0 / d;
    L[k * 8 + k] = d;
    for (int rr = k + 1; rr < m; ++rr) {
      double v = L[rr * 8 + k];
      for (int t = 0; t < k; ++t) v -= L[rr * 8 + t] * L[k * 8 + t];
      L[rr * 8 + k] = v * inv_d[k];
    }
  }
  // X = L^-1 (lower), then inverse = X^T X
  double X[64];
  for (int c = 0; c < m; ++c)
    for (int a = 0; a < m; ++a) {
      if (a < c) { X[a * 8 + c] = 0.0; continue; }
      double v = (a == c) ? 1.0 : 0.0;
      for (int t = c; t < a; ++t) v -= L[a * 8 + t] * X[t * 8 + c];
      X[a * 8 + c] = v * inv_d[a];
    }
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c) {
      double v = 0.0;
      for (int t = (a > c ? a : c); t < m; ++t) v += X[t * 8 + a] * X[t * 8 + c];
      dst[a * 8 + c] = v;
    }
  return true;
}

__device__ __forceinline__ void apply_block(const double* Minv, const double* in, double* out, int s0, int m) {
  double x[8];
  for (int a = 0; a < m; ++a) x[a] = in[s0 + a];
  for (int a = 0; a < m; ++a) {
    double v = 0.0;
    for (int c = 0; c < m; ++c) v += Minv[a * 8 + c] * x[c];
    out[s0 + a] = v;
  }
}

__global__ void __launch_bounds__(PCG_THREADS) pcg_kernel(const GroupDev* __restrict__ groups, int n_groups,
                                                          const int* __restrict__ gparams,
                                                          const int* __restrict__ blk_ptr,
                                                          const int64_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ lcol,
                                                          const int64_t* __restrict__ dpos,
                                                          const int64_t* __restrict__ bpos,
                                                          const double* __restrict__ vals,
                                                          const double* __restrict__ jtwr, double* lambda,
                                                          double* delta, double* blk_work, int* iters,
                                                          const int64_t* __restrict__ ch_e0,
                                                          const int64_t* __restrict__ ch_e1,
                                                          const int* __restrict__ ch_row, double* ch_part,
                                                          int* status) {
  extern __shared__ double vec[];
  __shared__ double red[33];
  __shared__ int fail;
  const int g = blockIdx.x;
  const GroupDev G = groups[g];
  if (G.dense != 0) return;
  const int n = G.n;
  const int* gp = gparams + G.p0;
  const int* bp = blk_ptr + G.b0;
  double* D = vec;
  double* x = D + n;
  double* r = x + n;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* Linv = blk_work + (int64_t)64 * G.b0;
  const int tid = threadIdx.x;
  double dmax = 0.0, bn2 = 0.0;
  for (int i = tid; i < n; i += blockDim.x) {
    const int pr = gp[i];
    const int64_t e = dpos[pr];
    const double d = e >= 0 ? vals[e] : 0.0;
    D[i] = d;
    dmax = fmax(dmax, d);
    const double b = jtwr[pr];
    bn2 += b * b;
  }
  dmax = block_max(dmax, red);
  bn2 = block_sum(bn2, red);
  const double floor_v = dmax > 0.0 ? DIAG_FLOOR * dmax : 1.0;
  for (int i = tid; i < n; i += blockDim.x) D[i] = fmax(D[i], floor_v);
  double lam = lambda[g];
  bool ok = false;
  int it = 0;
  for (int attempt = 0; attempt <= LM_RETRIES && !ok; ++attempt) {
    __syncthreads();
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int b = tid; b < G.nblk; b += blockDim.x)
      if (!factor_block(bpos + (int64_t)64 * (G.b0 + b), vals, D, bp[b], bp[b + 1] - bp[b], lam, Linv + (int64_t)64 * b))
        fail = 1;
    for (int i = tid; i < n; i += blockDim.x) { x[i] = 0.0; r[i] = jtwr[gp[i]]; }
    __syncthreads();
    if (fail) { lam *= 10.0; continue; }
    for (int b = tid; b < G.nblk; b += blockDim.x) apply_block(Linv + (int64_t)64 * b, r, z, bp[b], bp[b + 1] - bp[b]);
    __syncthreads();
    double rz = 0.0;
    for (int i = tid; i < n; i += blockDim.x) { p[i] = z[i]; rz += r[i] * z[i]; }
    rz = block_sum(rz, red);
    const double rz0 = rz;
    bool conv = bn2 == 0.0 || rz0 == 0.0;
    bool bad = false;
    const int cbeg = ch_row[G.p0], cend = ch_row[G.p0 + n];
    for (it = 0; it < PCG_MAX_IT && !conv; ++it) {
      __syncthreads();
      // SpMV: chunk partial sums, then each row sums its chunks in order
      for (int ch = cbeg + tid; ch < cend; ch += blockDim.x) {
        double sv = 0.0;
        for (int64_t e = ch_e0[ch]; e < ch_e1[ch]; ++e) sv += vals[e] * p[lcol[e]];
        ch_part[ch] = sv;
      }
      __syncthreads();
      double pq = 0.0;
      for (int i = tid; i < n; i += blockDim.x) {
        double sv = lam * D[i] * p[i];
        for (int ch = ch_row[G.p0 + i]; ch < ch_row[G.p0 + i + 1]; ++ch) sv += ch_part[ch];
        q[i] = sv;
        pq += p[i] * sv;
      }
      pq = block_sum(pq, red);
      if (!(pq > 0.0)) { bad = true; break; }
      const double alpha = rz / pq;
      for (int i = tid; i < n; i += blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      __syncthreads();
      for (int b = tid; b < G.nblk; b += blockDim.x) apply_block(Linv + (int64_t)64 * b, r, z, bp[b], bp[b + 1] - bp[b]);
      __syncthreads();
      double rz2 = 0.0;
      for (int i = tid; i < n; i += blockDim.x) rz2 += r[i] * z[i];
      rz2 = block_sum(rz2, red);
      if (rz2 <= PCG_RTOL * PCG_RTOL * rz0) { conv = true; ++it; break; }
      const double beta = rz2 / rz;
      rz = rz2;
      for (int i = tid; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
    }
    __syncthreads();
    if (bad) { lam *= 10.0; continue; }
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
  if (tid == 0) {
    lambda[g] = lam;
    if (iters) iters[g] = it;
  }
}

// ---------------------------------------------------------------------------
// grid-wide block-Jacobi PCG for one large group: every CTA of a cooperative
// launch works on the same system; dot products are block sums written to
// part[], a grid barrier, and the same fixed-order sum in every CTA
// (deterministic).  Three rotating partial buffers separate consecutive
// reductions by at least one barrier.
// ---------------------------------------------------------------------------
__device__ double grid_combine(const double* pb, double* red, bool is_max) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s = is_max ? fmax(s, pb[b]) : s + pb[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, s, o);
      s = is_max ? fmax(s, t) : s + t;
    }
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

__device__ double grid_sum(double v, double* part, int& slot, double* red, cg::grid_group& grid) {
  v = block_sum(v, red);
  double* pb = part + (size_t)slot * gridDim.x;
  if (threadIdx.x == 0) pb[blockIdx.x] = v;
  slot = (slot + 1) % 3;
  grid.sync();
  return grid_combine(pb, red, false);
}

__device__ double grid_max(double v, double* part, int& slot, double* red, cg::grid_group& grid) {
  v = block_max(v, red);
  double* pb = part + (size_t)slot * gridDim.x;
  if (threadIdx.x == 0) pb[blockIdx.x] = v;
  slot = (slot + 1) % 3;
  grid.sync();
  return grid_combine(pb, red, true);
}

__global__ void __launch_bounds__(PCG_THREADS) pcg_grid_kernel(int g, const GroupDev* __restrict__ groups,
                                                               const int* __restrict__ gparams,
                                                               const int* __restrict__ blk_ptr,
                                                               const int64_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ lcol,
                                                               const int64_t* __restrict__ dpos,
                                                               const int64_t* __restrict__ bpos,
                                                               const double* __restrict__ vals,
                                                               const double* __restrict__ jtwr, double* lambda,
                                                               double* delta, double* work, double* blk_work,
                                                               double* part, int* flag, int* iters,
                                                               const int64_t* __restrict__ ch_e0,
                                                               const int64_t* __restrict__ ch_e1,
                                                               const int* __restrict__ ch_row, double* ch_part,
                                                               int* status) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[33];
  const GroupDev G = groups[g];
  const int n = G.n;
  const int* gp = gparams + G.p0;
  const int* bp = blk_ptr + G.b0;
  double* D = work + (int64_t)6 * G.p0;
  double* x = D + n;
  double* r = x + n;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* Linv = blk_work + (int64_t)64 * G.b0;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int gs = gridDim.x * blockDim.x;
  int slot = 0;
  double dmax = 0.0, bn2 = 0.0;
  for (int i = gt; i < n; i += gs) {
    const int pr = gp[i];
    const int64_t e = dpos[pr];
    const double d = e >= 0 ? vals[e] : 0.0;
    D[i] = d;
    dmax = fmax(dmax, d);
    bn2 += jtwr[pr] * jtwr[pr];
  }
  dmax = grid_max(dmax, part, slot, red, grid);
  bn2 = grid_sum(bn2, part, slot, red, grid);
  const double floor_v = dmax > 0.0 ? DIAG_FLOOR * dmax : 1.0;
  for (int i = gt; i < n; i += gs) D[i] = fmax(D[i], floor_v);
  double lam = lambda[g];
  bool ok = false;
  int it = 0;
  for (int attempt = 0; attempt <= LM_RETRIES && !ok; ++attempt) {
    if (gt == 0) flag[0] = 0;
    grid.sync();
    for (int b = gt; b < G.nblk; b += gs)
      if (!factor_block(bpos + (int64_t)64 * (G.b0 + b), vals, D, bp[b], bp[b + 1] - bp[b], lam, Linv + (int64_t)64 * b))
        atomicOr(flag, 1);
    for (int i = gt; i < n; i += gs) { x[i] = 0.0; r[i] = jtwr[gp[i]]; }
    grid.sync();
    const int failed = *(volatile int*)flag;
    grid.sync();   // every CTA has read the flag before the next attempt resets it
    if (failed) { lam *= 10.0; continue; }
    for (int b = gt; b < G.nblk; b += gs) apply_block(Linv + (int64_t)64 * b, r, z, bp[b], bp[b + 1] - bp[b]);
    grid.sync();
    double rz = 0.0;
    for (int i = gt; i < n; i += gs) { p[i] = z[i]; rz += r[i] * z[i]; }
    rz = grid_sum(rz, part, slot, red, grid);
    const double rz0 = rz;
    bool conv = bn2 == 0.0 || rz0 == 0.0;
    bool bad = false;
    const int cbeg = ch_row[G.p0], cend = ch_row[G.p0 + n];
    // one iteration: [chunk SpMV] | [row sums -> q, p.q] | grid sum |
    // [per preconditioner block: x, r, z = M^-1 r, r.z] | grid sum |
    // [per block: p = z + beta p] | -- four grid barriers
    for (it = 0; it < PCG_MAX_IT && !conv; ++it) {
      for (int ch = cbeg + gt; ch < cend; ch += gs) {
        double sv = 0.0;
        for (int64_t e = ch_e0[ch]; e < ch_e1[ch]; ++e) sv += vals[e] * p[lcol[e]];
        ch_part[ch] = sv;
      }
      grid.sync();
      double pq = 0.0;
      for (int i = gt; i < n; i += gs) {
        double sv = lam * D[i] * p[i];
        for (int ch = ch_row[G.p0 + i]; ch < ch_row[G.p0 + i + 1]; ++ch) sv += ch_part[ch];
        q[i] = sv;
        pq += p[i] * sv;
      }
      pq = grid_sum(pq, part, slot, red, grid);
      if (!(pq > 0.0)) { bad = true; break; }
      const double alpha = rz / pq;
      double rz2 = 0.0;
      for (int b = gt; b < G.nblk; b += gs) {
        const int s0 = bp[b], m = bp[b + 1] - bp[b];
        for (int a = 0; a < m; ++a) {
          x[s0 + a] += alpha * p[s0 + a];
          r[s0 + a] -= alpha * q[s0 + a];
        }
        apply_block(Linv + (int64_t)64 * b, r, z, s0, m);
        for (int a = 0; a < m; ++a) rz2 += r[s0 + a] * z[s0 + a];
      }
      rz2 = grid_sum(rz2, part, slot, red, grid);
      if (rz2 <= PCG_RTOL * PCG_RTOL * rz0) { conv = true; ++it; break; }
      const double beta = rz2 / rz;
      rz = rz2;
      for (int b = gt; b < G.nblk; b += gs) {
        const int s0 = bp[b], m = bp[b + 1] - bp[b];
        for (int a = 0; a < m; ++a) p[s0 + a] = z[s0 + a] + beta * p[s0 + a];
      }
      grid.sync();
    }
    if (bad) { lam *= 10.0; grid.sync(); continue; }
    if (!conv && gt == 0) atomicCAS(status, 0, AP_ERR_TIMEOUT);
    ok = true;
  }
  if (!ok) {
    for (int i = gt; i < n; i += gs) delta[gp[i]] = 0.0;
    if (gt == 0) atomicCAS(status, 0, AP_ERR_NOT_SPD);
  } else {
    for (int i = gt; i < n; i += gs) delta[gp[i]] = x[i];
  }
  if (gt == 0) {
    lambda[g] = lam;
    if (iters) iters[g] = it;
  }
}

int grid_pcg_blocks(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_grid_kernel, PCG_THREADS, 0);
  return sms * (per > 0 ? 1 : 0);
}

// one cooperative launch per large group (groups flagged dense == 2)
int launch_pcg_grid(const GroupDev* groups_host, int n_groups, const SolvePlan& sp, const double* vals,
                    const double* jtwr, double* lambda, double* delta, int nblocks, int* status, cudaStream_t st) {
  for (int g = 0; g < n_groups; ++g) {
    if (groups_host[g].dense != 2) continue;
    void* args[] = {(void*)&g, (void*)&sp.groups, (void*)&sp.gparams, (void*)&sp.blk_ptr, (void*)&sp.row_ptr,
                    (void*)&sp.lcol, (void*)&sp.dpos, (void*)&sp.bpos, (void*)&vals, (void*)&jtwr, (void*)&lambda,
                    (void*)&delta, (void*)&sp.work, (void*)&sp.blk_work, (void*)&sp.part, (void*)&sp.flag,
                    (void*)&sp.iters, (void*)&sp.ch_e0, (void*)&sp.ch_e1, (void*)&sp.ch_row, (void*)&sp.ch_part,
                    (void*)&status};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_grid_kernel, dim3(nblocks), dim3(PCG_THREADS), args,
                                                0, st);
    if (e != cudaSuccess) return (int)e;
  }
  return 0;
}

void configure_solve() {
  allow_max_dynamic_smem(chol_kernel);
  allow_max_dynamic_smem(pcg_kernel);
}

void launch_lm_solve(int n_groups, const SolvePlan& sp, const double* vals, const double* jtwr, double* lambda,
                     double* delta, int* status, cudaStream_t st, int any_dense, int any_pcg, int max_dense,
                     int max_pcg) {
  if (n_groups <= 0) return;
  if (any_dense) {
    const size_t sm = (size_t)(2 * max_dense * max_dense + 2 * max_dense) * sizeof(double);
    chol_kernel<<<n_groups, CHOL_THREADS, sm, st>>>(sp.groups, n_groups, sp.gparams, sp.plocal, sp.row_ptr,
                                                    sp.col_idx, vals, jtwr, lambda, delta, max_dense, status);
  }
  if (any_pcg)
    pcg_kernel<<<n_groups, PCG_THREADS, 6 * max_pcg * sizeof(double), st>>>(
        sp.groups, n_groups, sp.gparams, sp.blk_ptr, sp.row_ptr, sp.lcol, sp.dpos, sp.bpos, vals, jtwr, lambda,
        delta, sp.blk_work, sp.iters, sp.ch_e0, sp.ch_e1, sp.ch_row, sp.ch_part, status);
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
