// Direct PSF correlation through shared memory, with the model / residual /
// chi^2 epilogue (forward) or a plain store (adjoint), and the deterministic
// float64 gathers of chi^2 and gradient partials.
//
// Paper: Sec. "PSF convolution" (direct mode, PSF normalised before
// convolution), Eq. chi2 and the variance / mask maps of Sec. "chi^2
// Optimization".
//
// Both directions are the same correlation
//     out(y, x) = sum_{ty < K, tx < K} Pk[ty][tx] * in(y + ty + off, x + tx + off)
// with in() zero outside its array:
//   forward: in = galaxy layer G (image grown by h), Pk = flipped PSF, off = 0,
//            which is the true convolution M = P * G on the image pixels;
//   adjoint: in = w r on the image, Pk = PSF, off = -2h, out = the galaxy
//            layer; the transpose of the forward map.
//
// Thread layout: a thread owns RY rows x RX = 4 columns of outputs.  For
// every input row it slides a register window of 8 values along the row in
// steps of 4 (one 16-byte shared load per step) and reads the matching PSF
// row chunk for each of its output rows as a broadcast 16-byte load, so the
// loop issues 16 RY FMAs per RY + 1 shared-memory loads.  Tile variants
// (threads BX x BY, RY) are picked per problem by timing them (autotuner in
// ap_api.cu).
#include "ap_internal.cuh"

namespace ap {

constexpr int RX = 4;

template <typename T> struct Limits;
template <> struct Limits<float> { __device__ static constexpr float max_finite() { return 3.402823466e38f; } };
template <> struct Limits<double> { __device__ static constexpr double max_finite() { return 1.7976931348623157e308; } };

template <typename T> struct Vec4;
template <> struct Vec4<float> {
  __device__ __forceinline__ static void ld(const float* p, float& a, float& b, float& c, float& d) {
    float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
  }
};
template <> struct Vec4<double> {
  __device__ __forceinline__ static void ld(const double* p, double& a, double& b, double& c, double& d) {
    double2 v0 = *reinterpret_cast<const double2*>(p);
    double2 v1 = *reinterpret_cast<const double2*>(p + 2);
    a = v0.x; b = v0.y; c = v1.x; d = v1.y;
  }
};

// variant table: threads BX x BY, rows per thread RY
struct ConvShape { int bx, by, ry; };
static const ConvShape kShapes[N_CONV_VARIANTS] = {{16, 16, 4}, {16, 8, 4}, {8, 16, 4}, {16, 16, 2}, {16, 8, 8}, {32, 8, 4},
                                                   {16, 8, 2}};
int conv_tile_w(int v) { return kShapes[v].bx * RX; }
int conv_tile_h(int v) { return kShapes[v].by * kShapes[v].ry; }
int conv_threads(int v) { return kShapes[v].bx * kShapes[v].by; }

template <typename T, int BX, int BY, int RY>
__device__ __forceinline__ void corr_tile(const T* __restrict__ in, int Hi, int Wi, int in_r0, int in_c0,
                                          const T* __restrict__ pk, int K, int K4, T* smem,
                                          T (&acc)[RY][RX]) {
  constexpr int NT = BX * BY;
  constexpr int TW = BX * RX, TH = BY * RY;
  const int SW = TW + K4;           // shared row stride (multiple of 4)
  const int SH = TH + K - 1;
  T* s_in = smem;
  T* s_pk = smem + SH * SW;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < K * K4; idx += NT) s_pk[idx] = pk[idx];
  for (int idx = tid; idx < SH * SW; idx += NT) {
    const int r = idx / SW, c = idx - r * SW;
    const int gr = in_r0 + r, gc = in_c0 + c;
    T v = (T)0;
    if (gr >= 0 && gr < Hi && gc >= 0 && gc < Wi) v = in[(size_t)gr * Wi + gc];
    s_in[idx] = v;
  }
  __syncthreads();
  const int lx = tid % BX, ly = tid / BX;
#pragma unroll
  for (int a = 0; a < RY; ++a)
#pragma unroll
    for (int b = 0; b < RX; ++b) acc[a][b] = (T)0;
  const int nchunk = K4 >> 2;
  for (int ir = 0; ir < RY + K - 1; ++ir) {
    const T* row = s_in + (ly * RY + ir) * SW + lx * RX;
    T w0, w1, w2, w3, w4, w5, w6, w7;
    Vec4<T>::ld(row, w0, w1, w2, w3);
    for (int c = 0; c < nchunk; ++c) {
      Vec4<T>::ld(row + 4 * c + 4, w4, w5, w6, w7);
#pragma unroll
      for (int ry = 0; ry < RY; ++ry) {
        const int ty = ir - ry;
        if (ty >= 0 && ty < K) {
          T p0, p1, p2, p3;
          Vec4<T>::ld(s_pk + ty * K4 + 4 * c, p0, p1, p2, p3);
          acc[ry][0] = fma(p3, w3, fma(p2, w2, fma(p1, w1, fma(p0, w0, acc[ry][0]))));
          acc[ry][1] = fma(p3, w4, fma(p2, w3, fma(p1, w2, fma(p0, w1, acc[ry][1]))));
          acc[ry][2] = fma(p3, w5, fma(p2, w4, fma(p1, w3, fma(p0, w2, acc[ry][2]))));
          acc[ry][3] = fma(p3, w6, fma(p2, w5, fma(p1, w4, fma(p0, w3, acc[ry][3]))));
        }
      }
      w0 = w4; w1 = w5; w2 = w6; w3 = w7;
    }
  }
}

// Fast path for float and PSF rows of NC = K4/4 chunks known at compile time:
// the whole input-row window of 4 NC + 4 values is loaded once per input row
// (NC + 1 shared loads) and every tap chunk of every output row is an
// unrolled block of 16 FMAs with constant register indices.
template <int BX, int BY, int RY, int NC>
__device__ __forceinline__ void corr_tile_nc(const float* __restrict__ in, int Hi, int Wi, int in_r0, int in_c0,
                                             const float* __restrict__ pk, int K, float* smem,
                                             float (&acc)[RY][RX]) {
  constexpr int NT = BX * BY;
  constexpr int TW = BX * RX, TH = BY * RY;
  constexpr int K4 = 4 * NC;
  constexpr int SW = TW + K4;
  const int SH = TH + K - 1;
  float* s_in = smem;
  float* s_pk = smem + SH * SW;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < K * K4; idx += NT) s_pk[idx] = pk[idx];
  for (int idx = tid; idx < SH * SW; idx += NT) {
    const int r = idx / SW, c = idx - r * SW;
    const int gr = in_r0 + r, gc = in_c0 + c;
    float v = 0.f;
    if (gr >= 0 && gr < Hi && gc >= 0 && gc < Wi) v = in[(size_t)gr * Wi + gc];
    s_in[idx] = v;
  }
  __syncthreads();
  const int lx = tid % BX, ly = tid / BX;
#pragma unroll
  for (int a = 0; a < RY; ++a)
#pragma unroll
    for (int b = 0; b < RX; ++b) acc[a][b] = 0.f;
  for (int ir = 0; ir < RY + K - 1; ++ir) {
    const float* row = s_in + (ly * RY + ir) * SW + lx * RX;
    float w[4 * NC + 4];
#pragma unroll
    for (int c = 0; c <= NC; ++c) Vec4<float>::ld(row + 4 * c, w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
#pragma unroll
    for (int ry = 0; ry < RY; ++ry) {
      const int ty = ir - ry;
      if (ty >= 0 && ty < K) {
        const float* prow = s_pk + ty * K4;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          float p0, p1, p2, p3;
          Vec4<float>::ld(prow + 4 * c, p0, p1, p2, p3);
#pragma unroll
          for (int rx = 0; rx < RX; ++rx)
            acc[ry][rx] = fmaf(p3, w[4 * c + rx + 3], fmaf(p2, w[4 * c + rx + 2],
                          fmaf(p1, w[4 * c + rx + 1], fmaf(p0, w[4 * c + rx], acc[ry][rx]))));
        }
      }
    }
  }
}

// dispatch between the generic (runtime K4) tile and the NC-templated one
template <typename T, int BX, int BY, int RY, int NC>
__device__ __forceinline__ void corr_any(const T* __restrict__ in, int Hi, int Wi, int in_r0, int in_c0,
                                         const T* __restrict__ pk, int K, int K4, T* smem, T (&acc)[RY][RX]) {
  if constexpr (NC > 0 && sizeof(T) == 4) {
    corr_tile_nc<BX, BY, RY, NC>(reinterpret_cast<const float*>(in), Hi, Wi, in_r0, in_c0,
                                 reinterpret_cast<const float*>(pk), K, reinterpret_cast<float*>(smem),
                                 reinterpret_cast<float(&)[RY][RX]>(acc));
  } else {
    corr_tile<T, BX, BY, RY>(in, Hi, Wi, in_r0, in_c0, pk, K, K4, smem, acc);
  }
}

// forward: model = P * G + U, r = d - m, w = mask ? 0 : 1/var, chi^2 partial,
// w r stored for the adjoint; model optionally stored
template <typename T, int BX, int BY, int RY, int NC>
__global__ void __launch_bounds__(BX * BY) forward_conv_kernel(const ConvWork* __restrict__ work,
                                                               const ImageDev* __restrict__ imgs,
                                                               double* __restrict__ chi2_partial,
                                                               void* const* __restrict__ model_out,
                                                               const int* __restrict__ skip, int trial,
                                                               int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[32];
  const ConvWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  if (skip && skip[im.group]) return;   // w r already holds this point; the gather keeps its chi^2
  T acc[RY][RX];
  if (im.has_gal) {
    corr_any<T, BX, BY, RY, NC>((const T*)im.gal, im.Hp, im.Wp, w.r0, w.c0, (const T*)im.psf_flip, im.K, im.K4,
                                smem, acc);
  } else {
#pragma unroll
    for (int a = 0; a < RY; ++a)
#pragma unroll
      for (int b = 0; b < RX; ++b) acc[a][b] = (T)0;
  }
  const int lx = threadIdx.x % BX, ly = threadIdx.x / BX;
  const T* U = (const T*)im.unc;
  T* WR = (T*)(trial ? im.wr_trial : im.wr);
  T* M = model_out ? (T*)model_out[w.image] : nullptr;
  // per-pixel residual math in T (float64 is scarce on this GPU); the
  // thread's chi^2 partial of at most RY * 4 terms joins the block sum in
  // float64
  T c2t = (T)0;
  int bad = 0;
#pragma unroll
  for (int ry = 0; ry < RY; ++ry) {
    const int oi = w.r0 + ly * RY + ry;
    if (oi >= im.H) break;
#pragma unroll
    for (int rx = 0; rx < RX; ++rx) {
      const int oj = w.c0 + lx * RX + rx;
      if (oj < im.W) {
        const size_t o = (size_t)oi * im.W + oj;
        const T m = acc[ry][rx] + U[o];
        if (M) M[o] = m;
        const T r = (T)im.data[o] - m;
        const T var = (T)im.var[o];
        T wt = (T)0;
        if (im.mask == nullptr || im.mask[o] == 0) {
          if (var > (T)0 && var <= Limits<T>::max_finite()) wt = (T)1 / var;
          else bad = 1;
        }
        const T wr = wt * r;
        c2t += wr * r;
        WR[o] = wr;
      }
    }
  }
  double c2 = (double)c2t;
  if (bad) atomicCAS(status, 0, AP_ERR_NONFINITE);
  if (chi2_partial) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = c2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int k = 0; k < (BX * BY + 31) / 32; ++k) s += red[k];
      chi2_partial[blockIdx.x] = s;
    }
  }
}

// adjoint: adj(ip, jp) = sum P[ty][tx] wr(ip + ty - 2h, jp + tx - 2h) on the galaxy layer
template <typename T, int BX, int BY, int RY, int NC>
__global__ void __launch_bounds__(BX * BY) adjoint_conv_kernel(const ConvWork* __restrict__ work,
                                                               const ImageDev* __restrict__ imgs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const ConvWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  T acc[RY][RX];
  corr_any<T, BX, BY, RY, NC>((const T*)im.wr, im.H, im.W, w.r0 - 2 * im.h, w.c0 - 2 * im.h, (const T*)im.psf_norm,
                              im.K, im.K4, smem, acc);
  const int lx = threadIdx.x % BX, ly = threadIdx.x / BX;
  T* A = (T*)im.adj;
#pragma unroll
  for (int ry = 0; ry < RY; ++ry) {
    const int oi = w.r0 + ly * RY + ry;
    if (oi >= im.Hp) break;
#pragma unroll
    for (int rx = 0; rx < RX; ++rx) {
      const int oj = w.c0 + lx * RX + rx;
      if (oj < im.Wp) A[(size_t)oi * im.Wp + oj] = acc[ry][rx];
    }
  }
}

// Jacobian columns of convolved sources: J_k = P * (d G_s / d theta_k) on the
// source's Jacobian support (its sampling box grown by h, clipped to the
// image), from the stored derivative images.  One CTA per output tile of one
// source, looping over the source's free slots.
template <typename T, int BX, int BY, int RY, int NC>
__global__ void __launch_bounds__(BX * BY) jcol_kernel(const JcolWork* __restrict__ work,
                                                       const SourceDev* __restrict__ srcs,
                                                       const ImageDev* __restrict__ imgs, const T* __restrict__ dbuf,
                                                       T* __restrict__ jbuf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const JcolWork w = work[blockIdx.x];
  const SourceDev& sd = srcs[w.src];
  const ImageDev& im = imgs[sd.image];
  const int bh = sd.box[1] - sd.box[0], bw = sd.box[3] - sd.box[2];
  const int64_t barea = (int64_t)bh * bw;
  const int sh = sd.sup[1] - sd.sup[0], sw = sd.sup[3] - sd.sup[2];
  const int64_t sarea = (int64_t)sh * sw;
  const int lx = threadIdx.x % BX, ly = threadIdx.x / BX;
  for (int k = 0; k < sd.nslot; ++k) {
    if (sd.pidx[k] < 0) continue;
    T acc[RY][RX];
    corr_any<T, BX, BY, RY, NC>(dbuf + sd.d_off + k * barea, bh, bw, w.r0 - im.h - sd.box[0],
                                w.c0 - im.h - sd.box[2], (const T*)im.psf_flip, im.K, im.K4, smem, acc);
    T* out = jbuf + sd.j_off + k * sarea;
#pragma unroll
    for (int ry = 0; ry < RY; ++ry) {
      const int oi = w.r0 + ly * RY + ry;
      if (oi >= sd.sup[1]) break;
#pragma unroll
      for (int rx = 0; rx < RX; ++rx) {
        const int oj = w.c0 + lx * RX + rx;
        if (oj < sd.sup[3]) out[(int64_t)(oi - sd.sup[0]) * sw + (oj - sd.sup[2])] = acc[ry][rx];
      }
    }
    __syncthreads();   // the next slot reloads the shared tile
  }
}

template <typename T, int BX, int BY, int RY>
static size_t corr_smem_bytes(int Kmax) {
  const int K4 = (Kmax + 3) & ~3;
  return (size_t)((BY * RY + Kmax - 1) * (BX * RX + K4) + Kmax * K4) * sizeof(T);
}

// compile-time PSF chunk counts of the fast path (K4/4); others run generic
__host__ __device__ constexpr bool nc_fast(int nc) { return (nc >= 1 && nc <= 8) || nc == 13; }
int conv_nc_of(int K4, int is_double) { return (!is_double && nc_fast(K4 / 4)) ? K4 / 4 : 0; }

template <typename T, int BX, int BY, int RY, int NC>
static int configure_one(int Kmax) {
  const int need = (int)corr_smem_bytes<T, BX, BY, RY>(Kmax);
  const int a = allow_max_dynamic_smem(forward_conv_kernel<T, BX, BY, RY, NC>);
  const int b = allow_max_dynamic_smem(adjoint_conv_kernel<T, BX, BY, RY, NC>);
  const int c = allow_max_dynamic_smem(jcol_kernel<T, BX, BY, RY, NC>);
  return (a >= need && b >= need && c >= need) ? 1 : 0;
}

// NC dispatch: the fast instantiations exist for float only
#define AP_NC_SWITCH(T, nc, CALL, ...)                                            \
  if (sizeof(T) == 4) {                                                           \
    switch (nc) {                                                                 \
      case 1: CALL(1, __VA_ARGS__); break;                                        \
      case 2: CALL(2, __VA_ARGS__); break;                                        \
      case 3: CALL(3, __VA_ARGS__); break;                                        \
      case 4: CALL(4, __VA_ARGS__); break;                                        \
      case 5: CALL(5, __VA_ARGS__); break;                                        \
      case 6: CALL(6, __VA_ARGS__); break;                                        \
      case 7: CALL(7, __VA_ARGS__); break;                                        \
      case 8: CALL(8, __VA_ARGS__); break;                                        \
      case 13: CALL(13, __VA_ARGS__); break;                                      \
      default: CALL(0, __VA_ARGS__); break;                                       \
    }                                                                             \
  } else {                                                                        \
    CALL(0, __VA_ARGS__);                                                         \
  }

// only the two fast tile shapes get NC instantiations; the others run generic
__host__ __device__ constexpr bool fast_shape(int bx, int by, int ry) {
  return bx == 16 && by == 8 && (ry == 2 || ry == 4 || ry == 8);
}

#define AP_CONV_SWITCH(v, CALL, ...)                     \
  switch (v) {                                           \
    case 0: CALL(16, 16, 4, __VA_ARGS__); break;         \
    case 1: CALL(16, 8, 4, __VA_ARGS__); break;          \
    case 2: CALL(8, 16, 4, __VA_ARGS__); break;          \
    case 3: CALL(16, 16, 2, __VA_ARGS__); break;         \
    case 4: CALL(16, 8, 8, __VA_ARGS__); break;          \
    case 5: CALL(32, 8, 4, __VA_ARGS__); break;          \
    default: CALL(16, 8, 2, __VA_ARGS__); break;         \
  }
static_assert(N_CONV_VARIANTS == 7, "AP_CONV_SWITCH lists every entry of kShapes");

template <typename T, int BX, int BY, int RY>
static int configure_variant(int Kmax) {
  int ok = configure_one<T, BX, BY, RY, 0>(Kmax);
  if constexpr (sizeof(T) == 4 && fast_shape(BX, BY, RY)) {
    ok &= configure_one<T, BX, BY, RY, 1>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 2>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 3>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 4>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 5>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 6>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 7>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 8>(Kmax);
    ok &= configure_one<T, BX, BY, RY, 13>(Kmax);
  }
  return ok;
}

// Set the shared-memory opt-in of every tile variant for PSFs up to Kmax
// (called once per problem, outside any stream capture).  ok[v] tells whether
// variant v fits.
template <typename T>
void configure_conv(int Kmax, int* ok) {
  const int kmax = Kmax < 1 ? 1 : Kmax;
  for (int v = 0; v < N_CONV_VARIANTS; ++v) {
    int r = 0;
#define AP_CFG(BX, BY, RY, dummy) r = configure_variant<T, BX, BY, RY>(kmax)
    AP_CONV_SWITCH(v, AP_CFG, 0)
#undef AP_CFG
    // the kernel the switch launches for v must have v's tile shape (the
    // planner cuts the work items by the table)
    int same = 0;
#define AP_SAME(BX, BY, RY, dummy) same = kShapes[v].bx == BX && kShapes[v].by == BY && kShapes[v].ry == RY
    AP_CONV_SWITCH(v, AP_SAME, 0)
#undef AP_SAME
    if (ok) ok[v] = r && same;
  }
  cudaGetLastError();
}

int conv_variant_fast(int v) {
  int r = 0;
#define AP_FS(BX, BY, RY, dummy) r = fast_shape(BX, BY, RY)
  AP_CONV_SWITCH(v, AP_FS, 0)
#undef AP_FS
  return r;
}

template <typename T, int BX, int BY, int RY, int NC>
static void fwd_launch(const ConvWork* work, int n, const ImageDev* imgs, double* chi2_partial, void* const* model_out,
                       const int* skip, int trial, int* status, int kmax, cudaStream_t st) {
  if constexpr (NC == 0 || (sizeof(T) == 4 && fast_shape(BX, BY, RY)))
    forward_conv_kernel<T, BX, BY, RY, NC><<<n, BX * BY, corr_smem_bytes<T, BX, BY, RY>(kmax), st>>>(
        work, imgs, chi2_partial, model_out, skip, trial, status);
}
template <typename T, int BX, int BY, int RY, int NC>
static void adj_launch(const ConvWork* work, int n, const ImageDev* imgs, int kmax, cudaStream_t st) {
  if constexpr (NC == 0 || (sizeof(T) == 4 && fast_shape(BX, BY, RY)))
    adjoint_conv_kernel<T, BX, BY, RY, NC><<<n, BX * BY, corr_smem_bytes<T, BX, BY, RY>(kmax), st>>>(work, imgs);
}
template <typename T, int BX, int BY, int RY, int NC>
static void jc_launch(const JcolWork* work, int n, const SourceDev* srcs, const ImageDev* imgs, const T* dbuf, T* jbuf,
                      int kmax, cudaStream_t st) {
  if constexpr (NC == 0 || (sizeof(T) == 4 && fast_shape(BX, BY, RY)))
    jcol_kernel<T, BX, BY, RY, NC><<<n, BX * BY, corr_smem_bytes<T, BX, BY, RY>(kmax), st>>>(work, srcs, imgs, dbuf,
                                                                                             jbuf);
}

// Launch one kernel per range of work items sharing a PSF chunk count
// (ranges[k] = {nc, start, count}); nc = 0 runs the generic tile.
template <typename T>
void launch_forward_conv(int v, const ConvWork* work, const ConvRange* ranges, int n_ranges, const ImageDev* imgs,
                         double* chi2_partial, void* const* model_out, const int* skip, int trial, int* status,
                         int kmax, cudaStream_t st) {
  for (int k = 0; k < n_ranges; ++k) {
    const ConvRange r = ranges[k];
    if (r.count <= 0) continue;
    const int nc = conv_variant_fast(v) ? r.nc : 0;
#define AP_FWD_NC(NC, BX, BY, RY) fwd_launch<T, BX, BY, RY, NC>(work + r.start, r.count, imgs, chi2_partial + r.start, model_out, skip, trial, status, kmax, st)
#define AP_FWD(BX, BY, RY, dummy) AP_NC_SWITCH(T, nc, AP_FWD_NC, BX, BY, RY)
    AP_CONV_SWITCH(v, AP_FWD, 0)
#undef AP_FWD
#undef AP_FWD_NC
  }
}

template <typename T>
void launch_adjoint_conv(int v, const ConvWork* work, const ConvRange* ranges, int n_ranges, const ImageDev* imgs,
                         int kmax, cudaStream_t st) {
  for (int k = 0; k < n_ranges; ++k) {
    const ConvRange r = ranges[k];
    if (r.count <= 0) continue;
    const int nc = conv_variant_fast(v) ? r.nc : 0;
#define AP_ADJ_NC(NC, BX, BY, RY) adj_launch<T, BX, BY, RY, NC>(work + r.start, r.count, imgs, kmax, st)
#define AP_ADJ(BX, BY, RY, dummy) AP_NC_SWITCH(T, nc, AP_ADJ_NC, BX, BY, RY)
    AP_CONV_SWITCH(v, AP_ADJ, 0)
#undef AP_ADJ
#undef AP_ADJ_NC
  }
}

template <typename T>
void launch_jcol(int v, const JcolWork* work, const ConvRange* ranges, int n_ranges, const SourceDev* srcs,
                 const ImageDev* imgs, const T* dbuf, T* jbuf, int kmax, cudaStream_t st) {
  for (int k = 0; k < n_ranges; ++k) {
    const ConvRange r = ranges[k];
    if (r.count <= 0) continue;
    const int nc = conv_variant_fast(v) ? r.nc : 0;
#define AP_JC_NC(NC, BX, BY, RY) jc_launch<T, BX, BY, RY, NC>(work + r.start, r.count, srcs, imgs, dbuf, jbuf, kmax, st)
#define AP_JC(BX, BY, RY, dummy) AP_NC_SWITCH(T, nc, AP_JC_NC, BX, BY, RY)
    AP_CONV_SWITCH(v, AP_JC, 0)
#undef AP_JC
#undef AP_JC_NC
  }
}

// ---------------------------------------------------------------------------
// deterministic float64 gathers: one warp per output, lanes stride over the
// output's list in a fixed order, then a fixed shuffle tree
// ---------------------------------------------------------------------------
__global__ void sum_groups_kernel(const double* __restrict__ partial, const int* __restrict__ ptr,
                                  const int* __restrict__ idx, int n_out, double* __restrict__ out, double scale,
                                  const int* __restrict__ skip, const double* __restrict__ keep) {
  const int g = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (g >= n_out) return;
  if (skip && skip[g]) {   // the group's forward did not run: its value is kept
    if (lane == 0) out[g] = keep[g];
    return;
  }
  double s = 0.0;
  for (int k = ptr[g] + lane; k < ptr[g + 1]; k += 32) s += partial[idx[k]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[g] = scale * s;
}

// one 128-thread block per output: the list may be long (a sky parameter has
// one entry per tile it covers)
__global__ void __launch_bounds__(128) sum_contrib_kernel(const double* __restrict__ partial,
                                                          const int64_t* __restrict__ ptr,
                                                          const int64_t* __restrict__ idx, int n_out,
                                                          double* __restrict__ out, double scale) {
  __shared__ double red[4];
  const int g = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s = 0.0;
  for (int64_t k = ptr[g] + threadIdx.x; k < ptr[g + 1]; k += 128) s += partial[idx[k]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) out[g] = scale * (((red[0] + red[1]) + red[2]) + red[3]);
}

void launch_sum_groups(const double* partial, const int* ptr, const int* idx, int n_out, double* out, double scale,
                       const int* skip, const double* keep, cudaStream_t st) {
  if (n_out <= 0) return;
  sum_groups_kernel<<<(n_out + 7) / 8, 256, 0, st>>>(partial, ptr, idx, n_out, out, scale, skip, keep);
}

void launch_sum_contrib(const double* partial, const int64_t* ptr, const int64_t* idx, int n_out, double* out,
                        double scale, cudaStream_t st) {
  if (n_out <= 0) return;
  sum_contrib_kernel<<<n_out, 128, 0, st>>>(partial, ptr, idx, n_out, out, scale);
}

template void configure_conv<float>(int, int*);
template void configure_conv<double>(int, int*);
template void launch_jcol<float>(int, const JcolWork*, const ConvRange*, int, const SourceDev*, const ImageDev*, const float*, float*, int, cudaStream_t);
template void launch_jcol<double>(int, const JcolWork*, const ConvRange*, int, const SourceDev*, const ImageDev*, const double*, double*, int, cudaStream_t);
template void launch_forward_conv<float>(int, const ConvWork*, const ConvRange*, int, const ImageDev*, double*, void* const*, const int*, int, int*, int, cudaStream_t);
template void launch_forward_conv<double>(int, const ConvWork*, const ConvRange*, int, const ImageDev*, double*, void* const*, const int*, int, int*, int, cudaStream_t);
template void launch_adjoint_conv<float>(int, const ConvWork*, const ConvRange*, int, const ImageDev*, int, cudaStream_t);
template void launch_adjoint_conv<double>(int, const ConvWork*, const ConvRange*, int, const ImageDev*, int, cudaStream_t);

}  // namespace ap
