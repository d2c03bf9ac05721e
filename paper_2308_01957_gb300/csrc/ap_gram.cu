// J^T W J for the Levenberg-Marquardt step (Sec. "Optimization methods").
//
// J is never stored whole (the paper names its N_pixels x N_parameters memory
// as LM's drawback): the convolved columns of each source are stored on that
// source's support only, the others are its derivative images.
//
// Pass 1: each CTA owns one TILE x TILE image tile.  It loads sqrt(w)
// dm/dtheta_k over the tile for every free slot of every source reaching the
// tile into shared memory (pixel major), forms the tile's Gram matrix (3xTF32
// tensor-core MMAs, or float64 on CUDA cores), and stores it, cut into the
// blocks of its source pairs, into a scratch array where every source pair
// keeps its tiles' blocks one after another (offsets planned on the host).
// Pass 2: one warp per source pair adds its tiles' blocks in tile order and
// writes each sum into the compressed-sparse-row J^T W J (and its mirror),
// with plain stores where no other pair adds to the same entries (a shared
// parameter, as in joint fits, makes float64 atomics necessary).  No
// searches in the CSR and one write per entry instead of one atomic per tile.
#include <algorithm>

#include "ap_internal.cuh"

namespace ap {

template <typename T> struct GramCols { static constexpr int value = 160; };
template <> struct GramCols<double> { static constexpr int value = 80; };

template <typename T> struct Ld4;
template <> struct Ld4<float> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <> struct Ld4<double> {
  __device__ __forceinline__ static void ld(const double* p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

// Row stride of the pixel-major column blocks: for the tensor-core path a
// multiple of 32 plus 8 floats, so the eight rows x four lanes of a fragment
// load hit 32 different banks; cb + 4 for the float64 path.
template <typename T>
__host__ __device__ constexpr int gram_stride(int cb) {
  return sizeof(T) == 4 ? ((cb + 31) / 32) * 32 + 8 : cb + 4;
}

// Column position of element (pixel p, column c) in its pixel row.  Float
// path: c XOR ((p / 4) mod 8), which keeps c in its aligned group of 8 and
// makes both access patterns conflict-free with the stride above (= 8 mod
// 32): the row writes (32 pixels, one column) and the MMA fragment loads (4
// pixels x 8 columns).  Float64 path: unswizzled (4-column vector loads).
template <typename T>
__device__ __forceinline__ int gram_swz(int p, int c) {
  return sizeof(T) == 4 ? (c ^ ((p >> 2) & 7)) : c;
}

// Asynchronous copy of one element global -> shared (cp.async, sm_80+): the
// copies of all of a thread's columns are in flight together.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Load columns [c0, c0 + cb) of the tile (in (source, slot) order) into a
// pixel-major block of row stride CP, scaled by sqrt(w) of the thread's
// pixel; returns the number loaded.  Every thread fills its own row: copies
// are issued for all its in-box values, then awaited, then scaled.
template <typename T>
__device__ __forceinline__ int load_columns(T* blk, int CP, int c0, int cb, const TileWork& w,
                                            const int* __restrict__ jt_src, const SourceDev* __restrict__ srcs,
                                            const T* __restrict__ dbuf, const T* __restrict__ jbuf, int i, int j,
                                            bool inside, T sw, int* colp) {
  T* myrow = blk + threadIdx.x * CP;
  const int p = threadIdx.x;
  int col = 0, n = 0;
  for (int e = w.e0; e < w.e1 && n < cb; ++e) {
    const SourceDev& sd = srcs[jt_src[e]];
    int nfree = 0;
#pragma unroll
    for (int k = 0; k < MAX_SLOTS; ++k) nfree += (k < sd.nslot && sd.pidx[k] >= 0);
    if (col + nfree <= c0) { col += nfree; continue; }
    const int* bx = sd.conv ? sd.sup : sd.box;
    const bool in_b = inside && i >= bx[0] && i < bx[1] && j >= bx[2] && j < bx[3];
    const int bw = bx[3] - bx[2];
    const int64_t area = (int64_t)(bx[1] - bx[0]) * bw;
    const T* base = (sd.conv ? jbuf + sd.j_off : dbuf + sd.d_off) + (in_b ? (int64_t)(i - bx[0]) * bw + (j - bx[2]) : 0);
    int f = 0;
#pragma unroll
    for (int k = 0; k < MAX_SLOTS; ++k) {
      if (k >= sd.nslot || sd.pidx[k] < 0) continue;
      if (col >= c0 && n < cb) {
        if (in_b) cp_async_elem(myrow + gram_swz<T>(p, n), base + k * area);
        else myrow[gram_swz<T>(p, n)] = (T)0;
        // column info: local source index, free-slot index, free columns of the source
        if (threadIdx.x == 0) colp[n] = ((e - w.e0) << 8) | (f << 4) | nfree;
        ++n;
      }
      ++f;
      ++col;
    }
  }
  for (int c = n; c < ((n + 15) & ~15) && c < CP; ++c) myrow[gram_swz<T>(p, c)] = (T)0;
  cp_async_wait_all();
  for (int c = 0; c < n; ++c) myrow[gram_swz<T>(p, c)] *= sw;
  return n;
}

// Store one tile Gram entry (columns ca <= cb with column infos ia, ib) into
// its source pair's block: pairs of the L tile sources are numbered
// row-major over a <= b.
__device__ __forceinline__ void gram_store(double g, int ia, int ib, int L, const int64_t* __restrict__ tab,
                                           const int* __restrict__ tabs, double* __restrict__ scr) {
  const int la = ia >> 8, fa = (ia >> 4) & 15;
  const int lb = ib >> 8, fb = (ib >> 4) & 15, mb = ib & 15;
  const int pidx = la * L - (la * (la - 1)) / 2 + (lb - la);
  scr[tab[pidx] + (int64_t)(fa * mb + fb) * tabs[pidx]] = g;
}

// Gram of column block A (na columns) with column block B (nb_ columns) of
// the tile, stored into the pair blocks; diag = the blocks are the same.
template <typename T>
__device__ void gram_pair(const T* ja, const T* jb, int CP, int na, int nbc, bool diag, const int* colpa,
                          const int* colpb, int L, const int64_t* __restrict__ tab, const int* __restrict__ tabs,
                          double* __restrict__ scr) {
  const int tid = threadIdx.x;
  const int ba = (na + 3) >> 2, bb = (nbc + 3) >> 2;   // 4-column sub-blocks
  const int npb = diag ? ba * (ba + 1) / 2 : ba * bb;
  int NS = 4;
  while (NS < 32 && npb * NS * 2 <= TILE_THREADS) NS <<= 1;
  const int total = npb * NS;
  const int seglen = TILE_THREADS / NS;
  for (int base_idx = 0; base_idx < total; base_idx += TILE_THREADS) {
    const int idx = base_idx + tid;
    const bool active = idx < total;
    const int pb = active ? idx / NS : 0;
    const int seg = idx % NS;
    int A, B;
    if (diag) {
      A = 0;
      int rem = pb;
      while (rem >= ba - A) { rem -= ba - A; ++A; }
      B = A + rem;
    } else {
      A = pb / bb;
      B = pb - A * bb;
    }
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    if (active) {
      const T* pa = ja + 4 * A;
      const T* pbp = jb + 4 * B;
      for (int t = seg * seglen; t < (seg + 1) * seglen; ++t) {
        T va[4], vb[4];
        Ld4<T>::ld(pa + t * CP, va);
        Ld4<T>::ld(pbp + t * CP, vb);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += va[a] * vb[b];
      }
    }
    // segment partial sums (at most 64 pixels each in T) combine in float64
    double accd[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) accd[a][b] = (double)acc[a][b];
    for (int o = NS >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accd[a][b] += __shfl_xor_sync(0xffffffffu, accd[a][b], o);
    if (!active || seg != 0) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int ca = 4 * A + a, cb = 4 * B + b;
        if (ca >= na || cb >= nbc || (diag && cb < ca)) continue;
        gram_store(accd[a][b], colpa[ca], colpb[cb], L, tab, tabs, scr);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 3xTF32 tensor-core Gram (float path).  Each warp owns 16 x 8 output tiles
// of the block pair; for 8 pixels at a time it loads the A fragment (16
// columns of block A) and the B fragment (8 columns of block B) from the
// pixel-major shared blocks, splits every value into a TF32 head and a TF32
// tail, and issues three m16n8k8 MMAs (head*head + head*tail + tail*head,
// the tail*tail term is below float32 rounding).  Products accumulate in
// float32 over 64 pixels, then join a float64 sum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ void gram_pair_tc(const float* ja, const float* jb, int CP, int na, int nbc, bool diag, const int* colpa,
                             const int* colpb, int L, const int64_t* __restrict__ tab, const int* __restrict__ tabs,
                          double* __restrict__ scr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int mt_n = (na + 15) >> 4, nt_n = (nbc + 7) >> 3;
  for (int t = warp; t < mt_n * nt_n; t += TILE_THREADS / 32) {
    const int mt = t / nt_n, nt = t - mt * nt_n;
    const int m0 = 16 * mt, n0 = 8 * nt;
    if (diag && n0 + 8 <= m0) continue;   // entirely below the diagonal: its mirror is computed
    // 64-pixel float32 segments joined by a compensated float32 sum
    // (Knuth's TwoSum: hi + lo carries the exact sum of the segments up to
    // the rounding of lo), converted to float64 once per output
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int seg = 0; seg < TILE_THREADS; seg += 64) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
      for (int k0 = seg; k0 < seg + 64; k0 += 8) {
        // pixels p0 (fragment rows 0-3) and p0 + 4 (rows 4-7), swizzled columns
        const int p0 = k0 + tig, p1 = p0 + 4;
        const int s0 = (p0 >> 2) & 7, s1 = (p1 >> 2) & 7;
        const float* r0 = ja + p0 * CP;
        const float* r1 = ja + p1 * CP;
        uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3, bh0, bl0, bh1, bl1;
        split_tf32(r0[m0 + (gid ^ s0)], ah0, al0);
        split_tf32(r0[m0 + 8 + (gid ^ s0)], ah1, al1);
        split_tf32(r1[m0 + (gid ^ s1)], ah2, al2);
        split_tf32(r1[m0 + 8 + (gid ^ s1)], ah3, al3);
        split_tf32(jb[p0 * CP + n0 + (gid ^ s0)], bh0, bl0);
        split_tf32(jb[p1 * CP + n0 + (gid ^ s1)], bh1, bl1);
        mma_tf32(d, ah0, ah1, ah2, ah3, bl0, bl1);
        mma_tf32(d, al0, al1, al2, al3, bh0, bh1);
        mma_tf32(d, ah0, ah1, ah2, ah3, bh0, bh1);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float sum = __fadd_rn(hi[q], d[q]);
        const float bp = __fsub_rn(sum, hi[q]);
        const float err = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(sum, bp)), __fsub_rn(d[q], bp));
        hi[q] = sum;
        lo[q] = __fadd_rn(lo[q], err);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ca = m0 + gid + (q >> 1) * 8;
      const int cb = n0 + 2 * tig + (q & 1);
      if (ca >= na || cb >= nbc || (diag && cb < ca)) continue;
      gram_store((double)hi[q] + (double)lo[q], colpa[ca], colpb[cb], L, tab, tabs, scr);
    }
  }
}

template <typename T>
__device__ __forceinline__ void gram_pair_any(const T* ja, const T* jb, int CP, int na, int nbc, bool diag,
                                              const int* colpa, const int* colpb, int L, const int64_t* tab,
                                              const int* tabs, double* scr) {
  if constexpr (sizeof(T) == 4)
    gram_pair_tc(reinterpret_cast<const float*>(ja), reinterpret_cast<const float*>(jb), CP, na, nbc, diag, colpa,
                 colpb, L, tab, tabs, scr);
  else
    gram_pair<T>(ja, jb, CP, na, nbc, diag, colpa, colpb, L, tab, tabs, scr);
}

// One CTA per image tile.  The tile's C columns are processed in blocks of
// cb: block I is loaded once, then paired with every block J >= I (the Gram
// is symmetric), so any number of columns fits in two shared blocks.
template <typename T>
__global__ void __launch_bounds__(TILE_THREADS) gram_kernel(const TileWork* __restrict__ work,
                                                            const int* __restrict__ jt_src,
                                                            const SourceDev* __restrict__ srcs,
                                                            const ImageDev* __restrict__ imgs,
                                                            const T* __restrict__ dbuf, const T* __restrict__ jbuf,
                                                            const int64_t* __restrict__ tab0,
                                                            const int64_t* __restrict__ tab_all,
                                                            const int* __restrict__ tabs_all,
                                                            double* __restrict__ scr, int t_first, int cb,
                                                            int two_blocks, int* __restrict__ status) {
  const int CP = gram_stride<T>(cb);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* blk0 = reinterpret_cast<T*>(smem_raw);
  T* blk1 = blk0 + TILE_THREADS * CP;
  int* colp0 = reinterpret_cast<int*>(blk0 + (two_blocks ? 2 : 1) * TILE_THREADS * CP);
  int* colp1 = colp0 + CP;
  const int tile = t_first + blockIdx.x;
  const TileWork w = work[tile];
  const ImageDev& im = imgs[w.image];
  const int tid = threadIdx.x;
  const int i = w.r0 + tid / TILE, j = w.c0 + tid % TILE;
  const bool inside = i < im.H && j < im.W;
  T sw = (T)0;
  if (inside) {
    const size_t o = (size_t)i * im.W + j;
    const float var = im.var[o];
    // sqrt(w) in the column type: float32 (correctly rounded division and
    // root) in the mixed form, float64 in the float64 form
    if ((im.mask == nullptr || im.mask[o] == 0) && var > 0.f && isfinite(var))
      sw = sizeof(T) == 4 ? (T)(1.0f / sqrtf(var)) : (T)sqrt(1.0 / (double)var);
  }
  // total free columns of the tile
  int C = 0;
  for (int e = w.e0; e < w.e1; ++e) {
    const SourceDev& sd = srcs[jt_src[e]];
    for (int k = 0; k < sd.nslot; ++k) C += sd.pidx[k] >= 0;
  }
  const int nblk = (C + cb - 1) / cb;
  if (nblk > 1 && !two_blocks) {
    if (tid == 0) atomicCAS(status, 0, AP_ERR_ARG);
    return;
  }
  const int L = w.e1 - w.e0;
  const int64_t* tab = tab_all + tab0[tile];
  const int* tabs = tabs_all + tab0[tile];
  for (int I = 0; I < nblk; ++I) {
    __syncthreads();
    const int na = load_columns<T>(blk0, CP, I * cb, cb, w, jt_src, srcs, dbuf, jbuf, i, j, inside, sw, colp0);
    __syncthreads();
    gram_pair_any<T>(blk0, blk0, CP, na, na, true, colp0, colp0, L, tab, tabs, scr);
    for (int J = I + 1; J < nblk; ++J) {
      __syncthreads();
      const int nb_ = load_columns<T>(blk1, CP, J * cb, cb, w, jt_src, srcs, dbuf, jbuf, i, j, inside, sw, colp1);
      __syncthreads();
      gram_pair_any<T>(blk0, blk1, CP, na, nb_, false, colp0, colp1, L, tab, tabs, scr);
    }
  }
}

// Pass 2, light pairs: one warp per pair; lane e adds entry e of the pair's
// block over its tiles in tile order (float64) and writes it and its mirror.
__device__ __forceinline__ void gram_write(const GramPair& gp, int64_t pab, int64_t pba, double s,
                                           double* __restrict__ vals) {
  if (gp.excl) {
    vals[pab] = s;
    if (pba >= 0) vals[pba] = s;
  } else {
    atomicAdd(vals + pab, s);
    if (pba >= 0) atomicAdd(vals + pba, s);
  }
}

__global__ void __launch_bounds__(256) gram_reduce_kernel(const GramPair* __restrict__ pairs, int n_pairs,
                                                          const int64_t* __restrict__ pos,
                                                          const double* __restrict__ scr,
                                                          double* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = w0; p < n_pairs; p += nw) {
    const GramPair gp = pairs[p];
    const int ne = gp.ma * gp.mb;
    for (int e = lane; e < ne; e += 32) {
      const int64_t pab = pos[gp.pos + 2 * e], pba = pos[gp.pos + 2 * e + 1];
      if (pab < 0) continue;   // below the diagonal of a source's own block
      const double* src = scr + gp.base + e;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int k = 0;
      for (; k + 3 < gp.cnt; k += 4) {   // four independent loads in flight
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += src[(int64_t)(k + u) * ne];
      }
      double tail = 0.0;
      for (; k < gp.cnt; ++k) tail += src[(int64_t)k * ne];
      gram_write(gp, pab, pba, ((acc[0] + acc[1]) + (acc[2] + acc[3])) + tail, vals);
    }
  }
}

// Pass 2, heavy pairs, entries spanning many tiles (a source and the sky,
// the sky and itself): one CTA per entry from a planned work list; the
// entry's tiles are contiguous, the threads stride over them and a fixed
// tree joins the partials (deterministic).
__global__ void __launch_bounds__(256) gram_reduce_heavy_kernel(const GramPair* __restrict__ pairs,
                                                                const int* __restrict__ items,
                                                                const int64_t* __restrict__ pos,
                                                                const double* __restrict__ scr,
                                                                double* __restrict__ vals) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = items[blockIdx.x];
  const GramPair gp = pairs[item >> 6];
  const int e = item & 63;
  const int64_t pab = pos[gp.pos + 2 * e], pba = pos[gp.pos + 2 * e + 1];
  const double* src = scr + gp.base + (int64_t)e * gp.cnt;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int k = threadIdx.x;
  for (; k + 768 < gp.cnt; k += 1024) {
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += src[k + 256 * u];
  }
  double tail = 0.0;
  for (; k < gp.cnt; k += 256) tail += src[k];
  double s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + tail;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    gram_write(gp, pab, pba, t, vals);
  }
}

// Pass 2, heavy pairs, the other entries (up to GRAM_CTA_TILES tiles): one
// warp per entry, grid-stride over the work list; lane l adds tiles l,
// l + 32, ... in four independent chains and a fixed shuffle tree joins the
// lanes (deterministic).
__global__ void __launch_bounds__(256) gram_reduce_heavy_warp_kernel(const GramPair* __restrict__ pairs,
                                                                     const int* __restrict__ items, int n_items,
                                                                     const int64_t* __restrict__ pos,
                                                                     const double* __restrict__ scr,
                                                                     double* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int it = w0; it < n_items; it += nw) {
    const int item = items[it];
    const GramPair gp = pairs[item >> 6];
    const int e = item & 63;
    const double* src = scr + gp.base + (int64_t)e * gp.cnt;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int k = lane;
    for (; k + 96 < gp.cnt; k += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += src[k + 32 * u];
    }
    double tail = 0.0;
    for (; k < gp.cnt; k += 32) tail += src[k];
    double s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + tail;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) gram_write(gp, pos[gp.pos + 2 * e], pos[gp.pos + 2 * e + 1], s, vals);
  }
}

template <typename T>
size_t gram_smem_bytes(int cb, int two) {
  const int CP = gram_stride<T>(cb);
  return (size_t)(two ? 2 : 1) * TILE_THREADS * CP * sizeof(T) + (size_t)2 * CP * sizeof(int);
}

int gram_max_cols(int is_double) { return is_double ? GramCols<double>::value : GramCols<float>::value; }

// Column block size of a problem: the largest column count of any tile,
// rounded to 16 (float) / 4 (double), capped at 96 (float: one block in about
// 100 KB of shared memory) / 32 (double); two blocks only when some tile needs
// them.
template <typename T>
void gram_blocking(int maxc, int* cb, int* two) {
  const int cap = sizeof(T) == 4 ? 96 : 32;
  const int m = sizeof(T) == 4 ? ((maxc < 16 ? 16 : maxc) + 15) & ~15 : ((maxc < 4 ? 4 : maxc) + 3) & ~3;
  *cb = m < cap ? m : cap;
  *two = m > cap;
}

template <typename T>
void configure_gram(int) {
  allow_max_dynamic_smem(gram_kernel<T>);
}

template <typename T>
void launch_gram(const TileWork* work, const GramRange* ranges, int n_ranges, const int* jt_src,
                 const SourceDev* srcs, const ImageDev* imgs, const T* dbuf, const T* jbuf, const GramPlan& gp,
                 double* vals, int* status, cudaStream_t st, const ForkJoin* fj) {
  // pass 1: the column-blocking classes write disjoint scratch, so they run
  // side by side on the auxiliary streams (their launch tails overlap)
  int used = 0;
  if (fj && n_ranges > 1) cudaEventRecord(fj->fork, st);
  for (int r = 0; r < n_ranges; ++r) {
    const GramRange& g = ranges[r];
    if (g.t1 <= g.t0) continue;
    cudaStream_t s = st;
    if (fj && n_ranges > 1) {
      s = fj->aux[used % N_AUX_STREAMS];
      if (used < N_AUX_STREAMS) cudaStreamWaitEvent(s, fj->fork, 0);
      ++used;
    }
    if constexpr (sizeof(T) == 4) {
      if (g.tc > 0) {
        launch_gram_tc(g.tc, work, g.t0, g.t1, jt_src, srcs, imgs, reinterpret_cast<const float*>(dbuf),
                       reinterpret_cast<const float*>(jbuf), gp, status, s);
        continue;
      }
    }
    gram_kernel<T><<<g.t1 - g.t0, TILE_THREADS, gram_smem_bytes<T>(g.cb, g.two), s>>>(
        work, jt_src, srcs, imgs, dbuf, jbuf, gp.tab0, gp.tab, gp.tabs, gp.scr, g.t0, g.cb, g.two, status);
  }
  for (int k = 0; k < used && k < N_AUX_STREAMS; ++k) {
    cudaEventRecord(fj->join[k], fj->aux[k]);
    cudaStreamWaitEvent(st, fj->join[k], 0);
  }
  if (gp.n_light > 0) {
    const int blocks = (int)std::min<int64_t>(((int64_t)gp.n_light * 32 + 255) / 256, 8192);
    gram_reduce_kernel<<<blocks, 256, 0, st>>>(gp.pairs, gp.n_light, gp.pos, gp.scr, vals);
  }
  if (gp.n_heavy_cta > 0)
    gram_reduce_heavy_kernel<<<gp.n_heavy_cta, 256, 0, st>>>(gp.pairs + gp.n_light, gp.heavy_items, gp.pos, gp.scr,
                                                             vals);
  const int n_warp = gp.n_heavy_items - gp.n_heavy_cta;
  if (n_warp > 0) {
    // a full wave of 8 CTAs of 8 warps per SM, the warps striding over the list
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::min<int64_t>(((int64_t)n_warp * 32 + 255) / 256, (int64_t)std::max(sms, 1) * 8);
    gram_reduce_heavy_warp_kernel<<<blocks, 256, 0, st>>>(gp.pairs + gp.n_light, gp.heavy_items + gp.n_heavy_cta,
                                                          n_warp, gp.pos, gp.scr, vals);
  }
}

template void configure_gram<float>(int);
template void configure_gram<double>(int);
template void launch_gram<float>(const TileWork*, const GramRange*, int, const int*, const SourceDev*,
                                 const ImageDev*, const float*, const float*, const GramPlan&, double*, int*,
                                 cudaStream_t, const ForkJoin*);
template void launch_gram<double>(const TileWork*, const GramRange*, int, const int*, const SourceDev*,
                                  const ImageDev*, const double*, const double*, const GramPlan&, double*, int*,
                                  cudaStream_t, const ForkJoin*);
template void gram_blocking<float>(int, int*, int*);
template void gram_blocking<double>(int, int*, int*);

}  // namespace ap
