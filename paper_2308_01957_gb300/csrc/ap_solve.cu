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
// row p's diagonal), bpos[PCG_BLK2 b + PCG_BLK a + c] (position of entry
// (a, c) of preconditioner block b, -1 if structurally zero).
// ---------------------------------------------------------------------------
constexpr int PCG_SMEM_N = 2048;

// The damped block (m x m, m <= PCG_BLK) into A (row stride PCG_BLK) and
// its explicit inverse in place, by Gauss-Jordan elimination without
// pivoting (the block is symmetric positive definite, else a pivot fails):
// applying the preconditioner is then one small matrix-vector product with
// no float64 division.
__device__ bool factor_block(const int64_t* bq, const double* vals, const double* D, int s0, int m, double lam,
                             double* A) {
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c) {
      const int64_t e = bq[a * PCG_BLK + c];
      double v = e >= 0 ? vals[e] : 0.0;
      if (a == c) v += lam * D[s0 + a];
      A[a * PCG_BLK + c] = v;
    }
  for (int k = 0; k < m; ++k) {
    const double piv = A[k * PCG_BLK + k];
    if (!(piv > 0.0) || !isfinite(piv)) return false;
    const double ip = 1.0 / piv;
    A[k * PCG_BLK + k] = 1.0;
    for (int c = 0; c < m; ++c) A[k * PCG_BLK + c] *= ip;
    for (int a = 0; a < m; ++a) {
      if (a == k) continue;
      const double f = A[a * PCG_BLK + k];
      A[a * PCG_BLK + k] = 0.0;
      for (int c = 0; c < m; ++c) A[a * PCG_BLK + c] -= f * A[k * PCG_BLK + c];
    }
  }
  return true;
}

__device__ __forceinline__ void apply_block(const double* Minv, const double* in, double* out, int s0, int m) {
  double x[PCG_BLK];
  for (int a = 0; a < m; ++a) x[a] = in[s0 + a];
  for (int a = 0; a < m; ++a) {
    double v = 0.0;
    for (int c = 0; c < m; ++c) v += Minv[a * PCG_BLK + c] * x[c];
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
  double* Linv = blk_work + (int64_t)PCG_BLK2 * G.b0;
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
      if (!factor_block(bpos + (int64_t)PCG_BLK2 * (G.b0 + b), vals, D, bp[b], bp[b + 1] - bp[b], lam,
                        Linv + (int64_t)PCG_BLK2 * b))
        fail = 1;
    for (int i = tid; i < n; i += blockDim.x) { x[i] = 0.0; r[i] = jtwr[gp[i]]; }
    __syncthreads();
    if (fail) { lam *= 10.0; continue; }
    for (int b = tid; b < G.nblk; b += blockDim.x)
      apply_block(Linv + (int64_t)PCG_BLK2 * b, r, z, bp[b], bp[b + 1] - bp[b]);
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
      for (int b = tid; b < G.nblk; b += blockDim.x)
        apply_block(Linv + (int64_t)PCG_BLK2 * b, r, z, bp[b], bp[b + 1] - bp[b]);
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
// Distributed block-Jacobi PCG: one group's system spread over several CTAs,
// either the CTAs of one thread-block cluster (one group per cluster, many
// clusters per launch) or every CTA of a cooperative launch (one large group
// per launch).
//
// The iteration is the Chronopoulos-Gear arrangement of preconditioned CG
// (Chronopoulos & Gear 1989), in which both inner products of an iteration
// are reduced together:
//   u = M^-1 r,  w = A u,  gamma = r.u,  delta = u.w
//   beta = gamma / gamma_old,  alpha = gamma / (delta - beta gamma / alpha_old)
//   p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s
// (first iteration: beta = 0, alpha = gamma / delta).  In exact arithmetic it
// produces the iterates of the textbook PCG in pcg_kernel.  Two barriers per
// iteration: one after the SpMV chunk partials of A u (with delta), one after
// the owners of the rows publish the next u (with gamma).
//
// Ownership: CTA k owns a contiguous run of preconditioner blocks (and so of
// rows), planned on the host; its x, r, p, s, D and block inverses live in
// its shared memory.  The SpMV is cut into chunks that any CTA may compute:
// rows of up to DIST_WARP_ROW entries into thread chunks of DIST_CHUNK
// entries, longer rows (the sky parameters couple to everything) into warp
// chunks of DIST_WCHUNK entries, so that no row has more than a few partials
// to add.  In a cluster, u is broadcast into every CTA's shared memory and
// each chunk partial is stored straight into its row owner's shared memory
// (distributed shared memory); grid-wide, both go through global memory.
// Reductions: every CTA publishes its block totals to slot[parity][rank];
// after the barrier every CTA adds the slots in rank order, so all CTAs hold
// the same bits and take the same branches.
// ---------------------------------------------------------------------------
constexpr int DIST_THREADS = 256;

struct GridBarrier {
  static constexpr bool kCluster = false;
  __device__ void sync() const { cg::this_grid().sync(); }
  __device__ int rank() const { return blockIdx.x; }
  __device__ int size() const { return gridDim.x; }
  __device__ int unit() const { return 0; }
  template <typename T>
  __device__ T* at(T* p, int) const { return p; }
};

struct ClusterBarrier {
  static constexpr bool kCluster = true;
  __device__ void sync() const { cg::this_cluster().sync(); }
  __device__ int rank() const { return (int)cg::this_cluster().block_rank(); }
  __device__ int size() const { return (int)cg::this_cluster().num_blocks(); }
  __device__ int unit() const { return blockIdx.x / size(); }
  // the same shared-memory object in CTA q of the cluster
  template <typename T>
  __device__ T* at(T* p, int q) const { return cg::this_cluster().map_shared_rank(p, q); }
};

// CTA totals of NV <= 3 values (value 0 is a max when max0); every lane of
// warp 0 ends with them.  The tree joining the warp partials is only as wide
// as there are warps (every float64 instruction is costly on this part).
// red[] holds 3 x 32 + 3 doubles.
template <int NV>
__device__ void cta_reduce(double v[3], bool max0, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = (k == 0 && max0) ? fmax(v[k], t) : v[k] + t;
    }
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < NV; ++k) red[warp * 3 + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? red[lane * 3 + k] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        if (o >= nw) continue;   // uniform: the lanes past nw hold zeros
        const double t = __shfl_xor_sync(0xffffffffu, v[k], o);
        v[k] = (k == 0 && max0) ? fmax(v[k], t) : v[k] + t;
      }
      // after the trimmed tree only the lanes below nw hold the total: lane
      // 0's copy goes to every lane (a cluster publishes from lanes 0..nct-1)
      v[k] = __shfl_sync(0xffffffffu, v[k], 0);
    }
  }
}

// publish the CTA totals into slot[par][rank] (every CTA's copy in a
// cluster, the one global copy otherwise), wait at the barrier, add the slots
// in rank order; every thread returns the same NV values
template <int NV, class Bar>
__device__ void dist_reduce(const Bar& bar, double v[3], bool max0, double* slots, int& par, double* red) {
  const int nct = bar.size(), rank = bar.rank();
  cta_reduce<NV>(v, max0, red);
  double* sp = slots + (size_t)par * nct * 4;
  if (Bar::kCluster) {
    // every lane of warp 0 holds the totals; lane q stores them into CTA q
    if (threadIdx.x < nct) {
      double* dst = bar.at(sp, threadIdx.x) + rank * 4;
      for (int k = 0; k < NV; ++k) dst[k] = v[k];
    }
  } else if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) sp[rank * 4 + k] = v[k];
  }
  bar.sync();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double s[3] = {0.0, 0.0, 0.0};
    for (int q = lane; q < nct; q += 32)
      for (int k = 0; k < NV; ++k) {
        const double t = Bar::kCluster ? sp[q * 4 + k] : __ldcg(sp + q * 4 + k);
        s[k] = (k == 0 && max0) ? fmax(s[k], t) : s[k] + t;
      }
#pragma unroll
    for (int k = 0; k < NV; ++k)
      for (int o = 16; o > 0; o >>= 1) {
        if (o >= nct) continue;   // uniform: the lanes past nct hold zeros
        const double t = __shfl_xor_sync(0xffffffffu, s[k], o);
        s[k] = (k == 0 && max0) ? fmax(s[k], t) : s[k] + t;
      }
    if (lane == 0)   // lane 0 holds the complete sum
      for (int k = 0; k < NV; ++k) red[96 + k] = s[k];
  }
  __syncthreads();
  for (int k = 0; k < NV; ++k) v[k] = red[96 + k];
  par ^= 1;
}

// read u: the CTA's own copy in a cluster, global memory (L2) otherwise
template <bool CL>
__device__ __forceinline__ double ld_u(const double* u, int i) {
  if (CL) return u[i];
  return __ldcg(u + i);
}

// thread chunk: at most DIST_CHUNK entries of one row, all loads issued first
template <bool CL>
__device__ __forceinline__ double dist_tchunk(const double* __restrict__ vals, const int32_t* __restrict__ lcol,
                                              const double* u, int64_t e0, int64_t e1) {
  double v[DIST_CHUNK];
  int c[DIST_CHUNK];
#pragma unroll
  for (int k = 0; k < DIST_CHUNK; ++k) {
    const bool in = e0 + k < e1;
    v[k] = in ? vals[e0 + k] : 0.0;
    c[k] = in ? lcol[e0 + k] : -1;
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < DIST_CHUNK; ++k)
    if (c[k] >= 0) acc[k & 3] += v[k] * ld_u<CL>(u, c[k]);
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// warp chunk: at most DIST_WCHUNK entries of one row, lane l takes entries
// l, l + 32, ...; every lane returns the (fixed-order) total
template <bool CL>
__device__ __forceinline__ double dist_wchunk(const double* __restrict__ vals, const int32_t* __restrict__ lcol,
                                              const double* u, int64_t e0, int64_t e1, int lane) {
  double a0 = 0.0, a1 = 0.0;
  int64_t e = e0 + lane;
  for (; e + 32 < e1; e += 64) {
    a0 += vals[e] * ld_u<CL>(u, lcol[e]);
    a1 += vals[e + 32] * ld_u<CL>(u, lcol[e + 32]);
  }
  if (e < e1) a0 += vals[e] * ld_u<CL>(u, lcol[e]);
  double s = a0 + a1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <class Bar>
__global__ void __launch_bounds__(DIST_THREADS, 2) pcg_dist_kernel(int g_fixed, const int* __restrict__ glist,
                                                                const GroupDev* __restrict__ groups,
                                                                const int* __restrict__ gparams,
                                                                const int* __restrict__ blk_ptr,
                                                                const int64_t* __restrict__ dpos,
                                                                const int64_t* __restrict__ bpos,
                                                                const double* __restrict__ vals,
                                                                const double* __restrict__ jtwr, double* lambda,
                                                                double* delta, double* work, double* gslots,
                                                                int* iters, DistPlan dp, DistSmem sz,
                                                                int* status) {
  constexpr bool CL = Bar::kCluster;
  const Bar bar;
  extern __shared__ double sm[];
  __shared__ double red[3 * 32 + 3];
  const int nct = bar.size(), rank = bar.rank();
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = CL ? glist[bar.unit()] : g_fixed;
  const GroupDev G = groups[g];
  const int* gp = gparams + G.p0;
  const int* bp = blk_ptr + G.b0;
  const int ob = dp.own_ptr[g];
  const int b0 = dp.own_blk[ob + rank], b1 = dp.own_blk[ob + rank + 1];
  const int R0 = bp[b0], R1 = bp[b1];
  const int P0 = dp.row[G.p0 + R0];   // first chunk partial of the owned rows
  // shared memory: [slots (cluster)] | x r p s D [nr] | block inverses [nb] | u [nu] | partials [np] (cluster)
  double* slots = CL ? sm : gslots;
  double* X = sm + (CL ? 8 * nct : 0);
  double* Rv = X + sz.nr;
  double* P = Rv + sz.nr;
  double* S = P + sz.nr;
  double* Dv = S + sz.nr;
  double* Lv = Dv + sz.nr;                    // packed block inverses of the owned blocks
  double* U = Lv + sz.nb;                     // cluster: u over the whole group; grid: u of the owned rows
  double* PART = U + sz.nu;                   // cluster: partials of the owned rows
  double* gu = work + (int64_t)6 * G.p0;      // grid: u over the whole group, in global memory
  const double* ug = CL ? U : gu;             // where the SpMV gathers u from
  const int first = rank + nct * tid, stride = nct * (int)blockDim.x;
  const int wfirst = rank + nct * (tid >> 5), wstride = nct * (int)(blockDim.x >> 5);
  int par = 0;
  if (CL) bar.sync();   // every CTA of the cluster is running before any remote store

  double v[3] = {0.0, 0.0, 0.0};
  for (int i = R0 + tid; i < R1; i += blockDim.x) {
    const int pr = gp[i];
    const int64_t e = dpos[pr];
    v[0] = fmax(v[0], e >= 0 ? vals[e] : 0.0);
    v[1] += jtwr[pr] * jtwr[pr];
  }
  dist_reduce<2>(bar, v, true, slots, par, red);
  const double floor_v = v[0] > 0.0 ? DIAG_FLOOR * v[0] : 1.0;
  const double bn2 = v[1];
  double lam = lambda[g];
  bool ok = false;
  int it = 0;
  const int tb = dp.tptr[g], te = dp.tptr[g + 1], wb = dp.wptr[g], we = dp.wptr[g + 1];

  // u of one row: publish to the SpMV (every CTA's copy, or global memory)
  auto publish_u = [&](int i, double val) {
    if (CL) {
      for (int q = 0; q < nct; ++q) bar.at(U, q)[i] = val;
    } else {
      gu[i] = val;
      U[i - R0] = val;
    }
  };
  auto own_u = [&](int i) -> double { return CL ? U[i] : U[i - R0]; };

  // block phases run in teams of PCG_BLK (16) lanes, one team per owned
  // block and one lane per row of it; the rounds are uniform over the CTA so
  // that the team shuffles and warp syncs always see the whole warp
  const int team = tid / PCG_BLK, tl = tid % PCG_BLK, tbase = lane & ~(PCG_BLK - 1);
  const int nteam = blockDim.x / PCG_BLK;
  const int nrounds = (b1 - b0 + nteam - 1) / nteam;

  for (int attempt = 0; attempt <= LM_RETRIES && !ok; ++attempt) {
    double fail = 0.0, gam = 0.0, dd = 0.0;
    for (int rd = 0; rd < nrounds; ++rd) {
      const int b = b0 + rd * nteam + team;
      const bool has = b < b1;
      const int s0 = has ? bp[b] : 0, m = has ? bp[b + 1] - s0 : 0, l0 = s0 - R0;
      const bool row = tl < m;
      double d = 0.0, rr = 0.0;
      if (row) {
        const int pr = gp[s0 + tl];
        const int64_t e = dpos[pr];
        d = fmax(e >= 0 ? vals[e] : 0.0, floor_v);
        rr = jtwr[pr];
        Dv[l0 + tl] = d;
        X[l0 + tl] = 0.0;
        Rv[l0 + tl] = rr;
        P[l0 + tl] = 0.0;
        S[l0 + tl] = 0.0;
      }
      // the damped block into its packed slot (lane tl: row tl), then its
      // inverse in place by Gauss-Jordan elimination without pivoting (M is
      // symmetric positive definite or the block fails), the lanes of the
      // team updating their rows step by step; steps past the warp's largest
      // block are skipped (mw is uniform over the warp)
      double* Li = Lv + (has ? dp.loff[G.b0 + b] : 0);
      if (row) {
        const int64_t* bq = bpos + (int64_t)PCG_BLK2 * (G.b0 + b) + tl * PCG_BLK;
        for (int c = 0; c < m; ++c) {
          const int64_t e = bq[c];
          Li[tl * m + c] = (e >= 0 ? vals[e] : 0.0) + (c == tl ? lam * d : 0.0);
        }
      }
      __syncwarp();
      bool good = true;
      const int mw = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
      for (int k = 0; k < mw; ++k) {
        const bool act = k < m;
        const double piv = act ? Li[k * m + k] : 1.0;
        __syncwarp();   // the pivot is read before row k changes
        good = good && (!act || (piv > 0.0 && isfinite(piv)));
        const double ip = 1.0 / piv;
        if (act && tl == k) {
          Li[k * m + k] = 1.0;
          for (int c = 0; c < m; ++c) Li[k * m + c] *= ip;
        }
        __syncwarp();   // row k is scaled
        if (act && row && tl != k) {
          const double f = Li[tl * m + k];
          Li[tl * m + k] = 0.0;
          for (int c = 0; c < m; ++c) Li[tl * m + c] -= f * Li[k * m + c];
        }
        __syncwarp();   // every row is updated before the next pivot is read
      }
      // every lane of the team saw the same pivots: lane 0 counts a failure
      if (has && tl == 0 && !good) fail += 1.0;
      // u = M^-1 r for the block
      double t = 0.0;
      for (int c = 0; c < mw; ++c) {
        const double rc = __shfl_sync(0xffffffffu, rr, tbase + c);
        if (row && c < m) t += Li[tl * m + c] * rc;
      }
      if (row) {
        gam += rr * t;
        dd += lam * d * t * t;
        publish_u(s0 + tl, t);
      }
    }
    v[0] = fail; v[1] = gam; v[2] = dd;
    dist_reduce<3>(bar, v, false, slots, par, red);
    if (v[0] > 0.0) { lam *= 10.0; continue; }
    gam = v[1];
    dd = v[2];
    const double gamma0 = gam;
    bool conv = bn2 == 0.0 || !(gamma0 > 0.0);
    bool bad = false;
    double gam_old = 1.0, alpha_old = 1.0;
    for (it = 0; it < PCG_MAX_IT && !conv;) {
      // w = A u as chunk partials; delta = u.(A u) + the damping part
      double del = 0.0;
      for (int k = wb + wfirst; k < we; k += wstride) {
        const int c = dp.wlist[k];
        const double sv = dist_wchunk<CL>(vals, dp.lcol, ug, dp.e0[c], dp.e1[c], lane);
        if (lane == 0) {
          if (CL) bar.at(PART, dp.owner[c])[dp.dst[c]] = sv;
          else dp.part[c] = sv;
          del += ld_u<CL>(ug, dp.lrow[c]) * sv;
        }
      }
      for (int k = tb + first; k < te; k += stride) {
        const int c = dp.tlist[k];
        const double sv = dist_tchunk<CL>(vals, dp.lcol, ug, dp.e0[c], dp.e1[c]);
        if (CL) bar.at(PART, dp.owner[c])[dp.dst[c]] = sv;
        else dp.part[c] = sv;
        del += ld_u<CL>(ug, dp.lrow[c]) * sv;
      }
      v[0] = del;
      dist_reduce<1>(bar, v, false, slots, par, red);
      const double dlt = v[0] + dd;
      const double beta = it == 0 ? 0.0 : gam / gam_old;
      const double den = it == 0 ? dlt : dlt - beta * gam / alpha_old;
      if (!(den > 0.0) || !isfinite(den)) { bad = true; break; }
      const double alpha = gam / den;
      double gam2 = 0.0, dd2 = 0.0;
      for (int rd = 0; rd < nrounds; ++rd) {
        const int b = b0 + rd * nteam + team;
        const bool has = b < b1;
        const int s0 = has ? bp[b] : 0, m = has ? bp[b + 1] - s0 : 0, l = s0 - R0 + tl;
        const bool row = tl < m;
        double rr = 0.0;
        if (row) {
          const int i = s0 + tl;
          const int c0 = dp.row[G.p0 + i], c1 = dp.row[G.p0 + i + 1];
          const double ui = own_u(i);
          double w0 = lam * Dv[l] * ui, w1 = 0.0;
          int ch = c0;
          for (; ch + 1 < c1; ch += 2) {
            w0 += CL ? PART[ch - P0] : __ldcg(dp.part + ch);
            w1 += CL ? PART[ch + 1 - P0] : __ldcg(dp.part + ch + 1);
          }
          if (ch < c1) w0 += CL ? PART[ch - P0] : __ldcg(dp.part + ch);
          const double pi = ui + beta * P[l];
          const double si = (w0 + w1) + beta * S[l];
          P[l] = pi;
          S[l] = si;
          X[l] += alpha * pi;
          rr = Rv[l] - alpha * si;
          Rv[l] = rr;
        }
        const double* Li = Lv + (has ? dp.loff[G.b0 + b] : 0) + tl * m;
        // two independent product chains (shorter dependency path), as wide
        // as the warp's largest block
        const int mw = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
        double t0 = 0.0, t1 = 0.0;
        for (int c = 0; c < mw; ++c) {
          const double rc = __shfl_sync(0xffffffffu, rr, tbase + c);
          if (row && c < m) {
            if (c & 1) t1 += Li[c] * rc;
            else t0 += Li[c] * rc;
          }
        }
        const double t = t0 + t1;
        if (row) {
          gam2 += rr * t;
          dd2 += lam * Dv[l] * t * t;
          // the SpMV of this iteration is complete in every CTA (barrier
          // above), so u may be overwritten
          publish_u(s0 + tl, t);
        }
      }
      v[0] = gam2; v[1] = dd2;
      dist_reduce<2>(bar, v, false, slots, par, red);
      gam_old = gam;
      alpha_old = alpha;
      gam = v[0];
      dd = v[1];
      ++it;
      conv = gam <= PCG_RTOL * PCG_RTOL * gamma0;
    }
    if (bad) { lam *= 10.0; continue; }
    if (!conv && rank == 0 && tid == 0) atomicCAS(status, 0, AP_ERR_TIMEOUT);
    ok = true;
  }
  for (int i = R0 + tid; i < R1; i += blockDim.x) delta[gp[i]] = ok ? X[i - R0] : 0.0;
  if (rank == 0 && tid == 0) {
    lambda[g] = lam;
    if (iters) iters[g] = it;
    if (!ok) atomicCAS(status, 0, AP_ERR_NOT_SPD);
  }
  if (CL) bar.sync();   // no CTA leaves while another may still address its shared memory
}

size_t dist_smem_bytes(const DistSmem& sz, int nct, bool cluster) {
  return sizeof(double) * ((cluster ? (size_t)8 * nct : 0) + 5 * (size_t)sz.nr + (size_t)sz.nb + sz.nu + sz.np);
}

int grid_pcg_blocks(int device, size_t smem) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  allow_max_dynamic_smem(pcg_dist_kernel<GridBarrier>);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_dist_kernel<GridBarrier>, DIST_THREADS, smem);
  return sms * std::min(per, 2);
}

int cluster_pcg_size(int device, size_t smem) {
  (void)device;
  allow_max_dynamic_smem(pcg_dist_kernel<ClusterBarrier>);
  cudaFuncSetAttribute(pcg_dist_kernel<ClusterBarrier>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cs : {16, 8, 4}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(DIST_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, pcg_dist_kernel<ClusterBarrier>, &cfg) == cudaSuccess &&
        nclusters > 0)
      return cs;
    cudaGetLastError();
  }
  return 0;
}

// one cooperative launch per grid group (dense == 2), one cluster launch for
// all cluster groups (dense == 3)
int launch_pcg_dist(const GroupDev* groups_host, int n_groups, const SolvePlan& sp, const double* vals,
                    const double* jtwr, double* lambda, double* delta, const DistLaunch& dl, int* status,
                    cudaStream_t st) {
  const int* no_list = nullptr;
  for (int g = 0; g < n_groups; ++g) {
    if (groups_host[g].dense != 2) continue;
    void* args[] = {(void*)&g, (void*)&no_list, (void*)&sp.groups, (void*)&sp.gparams, (void*)&sp.blk_ptr,
                    (void*)&sp.dpos, (void*)&sp.bpos, (void*)&vals, (void*)&jtwr, (void*)&lambda, (void*)&delta,
                    (void*)&sp.work, (void*)&sp.part, (void*)&sp.iters, (void*)&sp.dist, (void*)&dl.grid_sz,
                    (void*)&status};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_dist_kernel<GridBarrier>,
                                                      dim3(dl.grid_blocks), dim3(DIST_THREADS), args,
                                                      dist_smem_bytes(dl.grid_sz, dl.grid_blocks, false), st);
    if (e != cudaSuccess) return (int)e;
  }
  if (dl.n_cluster_groups > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = dl.cluster_size;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(dl.n_cluster_groups * dl.cluster_size);
    cfg.blockDim = dim3(DIST_THREADS);
    cfg.dynamicSmemBytes = dist_smem_bytes(dl.cluster_sz, dl.cluster_size, true);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e =
        cudaLaunchKernelEx(&cfg, pcg_dist_kernel<ClusterBarrier>, -1, sp.cluster_groups, sp.groups, sp.gparams,
                           sp.blk_ptr, sp.dpos, sp.bpos, vals, jtwr, lambda, delta, sp.work, sp.part, sp.iters,
                           sp.dist, dl.cluster_sz, status);
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

// fwd_valid[g] = 1: after this iteration's state copy the group's current
// source records and w r are in place (the trial's if it accepted, else
// those of the unchanged theta), and chi2_state holds its chi^2
__global__ void accept_groups_kernel(const double* chi2_now, const double* chi2_trial, double* lambda,
                                     double* chi2_state, double* log, int* accepted, int* fwd_valid, int n_groups) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const double c0 = chi2_now[g], c1 = chi2_trial[g];
  const int acc = isfinite(c1) && c1 < c0;
  double lam = lambda[g];
  lam = acc ? fmax(lam / LAMBDA_DOWN, LAMBDA_MIN) : fmin(lam * LAMBDA_UP, LAMBDA_MAX);
  lambda[g] = lam;
  accepted[g] = acc;
  chi2_state[g] = acc ? c1 : c0;
  if (fwd_valid) fwd_valid[g] = 1;
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
                          double* log, int* accepted, int* fwd_valid, int n_groups, cudaStream_t st) {
  if (n_groups > 0)
    accept_groups_kernel<<<(n_groups + 255) / 256, 256, 0, st>>>(chi2_now, chi2_trial, lambda, chi2_state, log,
                                                                 accepted, fwd_valid, n_groups);
}

// one CTA per chunk: an accepted group's trial records and w r become its
// current ones (16-byte words where both ends are aligned)
__global__ void __launch_bounds__(256) accept_state_kernel(const StateChunk* __restrict__ chunks,
                                                           const int* __restrict__ accepted) {
  const StateChunk ch = chunks[blockIdx.x];
  if (!accepted[ch.group]) return;
  int done = 0;
  if ((((uintptr_t)ch.src | (uintptr_t)ch.dst) & 15) == 0) {
    const int nq = ch.n_words >> 2;
    const uint4* s4 = reinterpret_cast<const uint4*>(ch.src);
    uint4* d4 = reinterpret_cast<uint4*>(ch.dst);
    for (int i = threadIdx.x; i < nq; i += blockDim.x) d4[i] = s4[i];
    done = nq << 2;
  }
  for (int i = done + threadIdx.x; i < ch.n_words; i += blockDim.x) ch.dst[i] = ch.src[i];
}

void launch_accept_state(const StateChunk* chunks, int n_chunks, const int* accepted, cudaStream_t st) {
  if (n_chunks > 0) accept_state_kernel<<<n_chunks, 256, 0, st>>>(chunks, accepted);
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

// Pointers carried by value in the kernel's arguments: the launch copies them,
// so the caller's host array need not outlive the call (no host sync).
struct PtrRun {
  void* p[PTR_RUN];
  int n;
};

__global__ void store_ptrs_kernel(PtrRun run, void** dst) {
  if ((int)threadIdx.x < run.n) dst[threadIdx.x] = run.p[threadIdx.x];
}

void launch_store_ptrs(void* const* src_host, int n, void** dst_dev, cudaStream_t st) {
  for (int k0 = 0; k0 < n; k0 += PTR_RUN) {
    PtrRun run;
    run.n = n - k0 < PTR_RUN ? n - k0 : PTR_RUN;
    for (int k = 0; k < run.n; ++k) run.p[k] = src_host[k0 + k];
    store_ptrs_kernel<<<1, PTR_RUN, 0, st>>>(run, dst_dev + k0);
  }
}

}  // namespace ap
