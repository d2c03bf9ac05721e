// J^T W J for the Levenberg-Marquardt step (Sec. "Optimization methods").
//
// J is never stored whole (the paper names its N_pixels x N_parameters memory
// as LM's drawback): the convolved columns of each source are stored on that
// source's support only, the others are its derivative images.  Each CTA owns
// one TILE x TILE image tile: it loads sqrt(w) dm/dtheta_k over the tile for
// every free slot of every source reaching the tile into shared memory (pixel
// major, C columns padded to 4), forms the tile's Gram matrix with 4 x 4
// register blocks of column pairs, and adds it into the compressed-sparse-row
// J^T W J with float64 atomics.
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

__device__ __forceinline__ int64_t csr_find(const int64_t* row_ptr, const int32_t* col_idx, int r, int c) {
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    int v = col_idx[mid];
    if (v == c) return mid;
    if (v < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

template <typename T>
__global__ void __launch_bounds__(TILE_THREADS) gram_kernel(const TileWork* __restrict__ work,
                                                            const int* __restrict__ jt_src,
                                                            const SourceDev* __restrict__ srcs,
                                                            const ImageDev* __restrict__ imgs,
                                                            const T* __restrict__ dbuf, const T* __restrict__ jbuf,
                                                            const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col_idx,
                                                            double* __restrict__ vals, int* __restrict__ status) {
  constexpr int MAXC = GramCols<T>::value;
  constexpr int CP = MAXC + 4;                        // row stride of the pixel-major column block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Jt = reinterpret_cast<T*>(smem_raw);             // [256][CP]
  __shared__ int colp[GramCols<float>::value + 4];
  const TileWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  const int tid = threadIdx.x;
  const int i = w.r0 + tid / TILE, j = w.c0 + tid % TILE;
  const bool inside = i < im.H && j < im.W;
  T sw = (T)0;
  if (inside) {
    const size_t o = (size_t)i * im.W + j;
    const double var = (double)im.var[o];
    if ((im.mask == nullptr || im.mask[o] == 0) && var > 0.0 && var < 1e300) sw = (T)sqrt(1.0 / var);
  }
  T* myrow = Jt + tid * CP;
  int ncol = 0;
  for (int e = w.e0; e < w.e1; ++e) {
    const SourceDev& sd = srcs[jt_src[e]];
    const int* bx = sd.conv ? sd.sup : sd.box;
    const bool in_b = inside && i >= bx[0] && i < bx[1] && j >= bx[2] && j < bx[3];
    const int bw = bx[3] - bx[2];
    const int64_t area = (int64_t)(bx[1] - bx[0]) * bw;
    const T* base = sd.conv ? jbuf + sd.j_off : dbuf + sd.d_off;
    const int64_t off = in_b ? (int64_t)(i - bx[0]) * bw + (j - bx[2]) : 0;
    for (int k = 0; k < sd.nslot; ++k) {
      if (sd.pidx[k] < 0) continue;
      if (ncol >= MAXC) {
        if (tid == 0) atomicCAS(status, 0, AP_ERR_ARG);
        continue;
      }
      myrow[ncol] = in_b ? base[k * area + off] * sw : (T)0;
      if (tid == 0) colp[ncol] = sd.pidx[k];
      ++ncol;
    }
  }
  const int nb = (ncol + 3) >> 2;                    // 4-column blocks
  for (int c = ncol; c < 4 * nb; ++c) myrow[c] = (T)0;
  __syncthreads();
  const int npb = nb * (nb + 1) / 2;
  for (int pb = tid; pb < npb; pb += TILE_THREADS) {
    int A = 0, rem = pb;
    while (rem >= nb - A) { rem -= nb - A; ++A; }
    const int B = A + rem;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    const T* pa = Jt + 4 * A;
    const T* pbp = Jt + 4 * B;
    for (int t = 0; t < TILE_THREADS; ++t) {
      T va[4], vb[4];
      Ld4<T>::ld(pa + t * CP, va);
      Ld4<T>::ld(pbp + t * CP, vb);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += va[a] * vb[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int ca = 4 * A + a, cb = 4 * B + b;
        if (ca >= ncol || cb >= ncol || (A == B && b < a)) continue;
        const double g = (double)acc[a][b];
        if (g == 0.0) continue;
        const int ra = colp[ca], rb = colp[cb];
        const int64_t pab = csr_find(row_ptr, col_idx, ra, rb);
        if (pab < 0) { atomicCAS(status, 0, AP_ERR_ARG); continue; }
        atomicAdd(vals + pab, g);
        if (ca != cb) {
          const int64_t pba = csr_find(row_ptr, col_idx, rb, ra);
          if (pba >= 0) atomicAdd(vals + pba, g);
        }
      }
    }
  }
}

template <typename T>
size_t gram_smem_bytes(int) {
  return (size_t)TILE_THREADS * (GramCols<T>::value + 4) * sizeof(T);
}

int gram_max_cols(int is_double) { return is_double ? GramCols<double>::value : GramCols<float>::value; }

template <typename T>
void configure_gram(int Kmax) {
  cudaFuncSetAttribute(gram_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem_bytes<T>(Kmax));
}

template <typename T>
void launch_gram(const TileWork* work, int n_work, const int* jt_src, const SourceDev* srcs, const ImageDev* imgs,
                 const T* dbuf, const T* jbuf, const int64_t* row_ptr, const int32_t* col_idx, double* vals,
                 int* status, cudaStream_t st) {
  if (n_work <= 0) return;
  gram_kernel<T><<<n_work, TILE_THREADS, gram_smem_bytes<T>(0), st>>>(work, jt_src, srcs, imgs, dbuf, jbuf, row_ptr,
                                                                       col_idx, vals, status);
}

template void configure_gram<float>(int);
template void configure_gram<double>(int);
template void launch_gram<float>(const TileWork*, int, const int*, const SourceDev*, const ImageDev*, const float*,
                                 const float*, const int64_t*, const int32_t*, double*, int*, cudaStream_t);
template void launch_gram<double>(const TileWork*, int, const int*, const SourceDev*, const ImageDev*, const double*,
                                  const double*, const int64_t*, const int32_t*, double*, int*, cudaStream_t);

}  // namespace ap
