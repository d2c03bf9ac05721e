// FFT mode of the PSF convolution for the Jacobian columns (Sec. "PSF
// convolution": the paper notes that an FFT makes large PSFs affordable).
//
// J_k = P (*) dG/dtheta_k on a source's support is a linear convolution of
// the derivative image (box, bh x bw) with the normalised PSF (K x K).
// Overlap-save on fixed N x N blocks (N = 64 for K <= 33, 128 for K <= 97,
// chosen per source by the estimated cost of its blocks):
// an output block of B = N - K + 1 rows and columns needs the derivative
// image on the block grown by K - 1; its circular convolution of size N
// with the zero-padded PSF equals the linear one at the block's B x B
// outputs (no wrap-around reaches them).  One slot per transform: packing
// two slots into the real and imaginary parts would leak one slot's rounding
// into the other, and a column that is exactly zero (the position angle of a
// round source) must stay zero.
//
// One CTA per (source, slot, output block).  The N x N block lives in
// shared memory; each 1-D pass (rows, then columns) is done by T = 8 threads
// per line with N / T elements in registers: an (N/T)-point DFT per thread,
// twiddles W_N^(n2 k1), an exchange through the line in shared memory, then
// T-point DFTs -- the two-factor split of the DFT
//   X[k1 + E k2] = sum_n2 W_T^(n2 k2) W_N^(n2 k1) sum_n1 x[T n1 + n2] W_E^(n1 k1),
// E = N / T.  Every pass reads and writes natural order, so the product with
// the PSF spectrum (made by the same forward transform and scaled by 1/N^2)
// is elementwise and the inverse passes (conjugate twiddles) return natural
// order.  Float32 throughout; a transform of size N adds O(log N) roundings.
#include <cmath>
#include <vector>

#include "ap_internal.cuh"

namespace ap {

namespace {

constexpr int FFT_T = 8;   // threads per line

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

// W_16^k = exp(-2 pi i k / 16) as literals (cos and sin of multiples of
// pi / 8), so that after unrolling the trivial factors fold away
__device__ __forceinline__ float2 w16(int k) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
  switch (k & 15) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, -s1);
    case 2: return make_float2(r2, -r2);
    case 3: return make_float2(s1, -c1);
    case 4: return make_float2(0.f, -1.f);
    case 5: return make_float2(-s1, -c1);
    case 6: return make_float2(-r2, -r2);
    case 7: return make_float2(-c1, -s1);
    case 8: return make_float2(-1.f, 0.f);
    case 9: return make_float2(-c1, s1);
    case 10: return make_float2(-r2, r2);
    case 11: return make_float2(-s1, c1);
    case 12: return make_float2(0.f, 1.f);
    case 13: return make_float2(s1, c1);
    case 14: return make_float2(r2, r2);
    default: return make_float2(c1, s1);
  }
}

constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// E-point DFT in registers (E = 8 or 16), natural order in and out;
// INV: conjugate roots (unnormalised inverse)
template <int E, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[E]) {
  constexpr int bits = E == 8 ? 3 : 4;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int j = bitrev(i, bits);
    if (j > i) {
      const float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= E; len <<= 1) {
#pragma unroll
    for (int i = 0; i < E; i += len) {
#pragma unroll
      for (int j = 0; j < len / 2; ++j) {
        float2 w = w16(j * (16 / len));
        if (INV) w = c_conj(w);
        const float2 a = v[i + j], b = c_mul(v[i + j + len / 2], w);
        v[i + j] = c_add(a, b);
        v[i + j + len / 2] = c_sub(a, b);
      }
    }
  }
}

// One 1-D pass over all N lines (rows when ROW, else columns) of the N x N
// array a (row stride LD = N + 1).  twN[k] = W_N^k.  The NT threads take
// L = NT / T lines at a time: thread t works on line t mod L as member
// q = t / L of its line, so the 32 lanes of a warp touch 32 different lines
// at the same position -- consecutive (columns) or LD apart (rows, LD odd):
// no shared-memory bank conflicts.  The exchange between the members of a
// line goes through the line itself, separated by block barriers.
template <int N, int NT, int LD, bool ROW, bool INV>
__device__ __forceinline__ void fft_pass(float2* a, const float2* twN) {
  constexpr int T = FFT_T, E = N / T, G = E / T, L = NT / T;
  constexpr int step = ROW ? 1 : LD;
  const int q = threadIdx.x / L;
#pragma unroll 1
  for (int line = threadIdx.x % L; line < N; line += L) {
    float2* base = ROW ? a + line * LD : a + line;
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) v[n1] = base[(T * n1 + q) * step];
    dft_reg<E, INV>(v);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) {
      const float2 w = twN[(q * k1) & (N - 1)];
      v[k1] = c_mul(v[k1], INV ? c_conj(w) : w);
    }
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) base[(q + T * k1) * step] = v[k1];
    __syncthreads();
    float2 u[G][T];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int k1 = q + T * g;
#pragma unroll
      for (int n2 = 0; n2 < T; ++n2) u[g][n2] = base[(n2 + T * k1) * step];
      dft_reg<T, INV>(u[g]);
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int k1 = q + T * g;
#pragma unroll
      for (int k2 = 0; k2 < T; ++k2) base[(k1 + E * k2) * step] = u[g][k2];
    }
  }
}

template <int N>
struct FftShape {
  static constexpr int NT = N * 4;     // threads: N / 2 lines at a time, T members each
  static constexpr int LD = N + 1;     // odd row stride: row passes spread over the banks
  static constexpr size_t smem = (size_t)(N * LD + N) * sizeof(float2);
};

template <int N>
__device__ __forceinline__ void fft2_forward(float2* a, const float2* tw) {
  constexpr int NT = FftShape<N>::NT, LD = FftShape<N>::LD;
  fft_pass<N, NT, LD, true, false>(a, tw);
  __syncthreads();
  fft_pass<N, NT, LD, false, false>(a, tw);
  __syncthreads();
}

template <int N>
__device__ __forceinline__ void fft2_inverse(float2* a, const float2* tw) {
  constexpr int NT = FftShape<N>::NT, LD = FftShape<N>::LD;
  fft_pass<N, NT, LD, false, true>(a, tw);
  __syncthreads();
  fft_pass<N, NT, LD, true, true>(a, tw);
  __syncthreads();
}

// spectrum of the normalised PSF placed at [0, K)^2 of an N x N block,
// scaled by 1 / N^2 (the inverse transform is unnormalised)
template <int N>
__global__ void __launch_bounds__(FftShape<N>::NT) psf_spectrum_kernel(const float* __restrict__ psf, int K, int K4,
                                                                       const float2* __restrict__ tw_g,
                                                                       float2* __restrict__ spec) {
  constexpr int NT = FftShape<N>::NT, LD = FftShape<N>::LD;
  extern __shared__ float2 sm[];
  float2* tw = sm + N * LD;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = tw_g[i];
  for (int idx = threadIdx.x; idx < N * N; idx += NT) {
    const int u = idx / N, v = idx % N;
    sm[u * LD + v] = make_float2(u < K && v < K ? psf[u * K4 + v] : 0.f, 0.f);
  }
  __syncthreads();
  fft2_forward<N>(sm, tw);
  const float s = 1.0f / (float)(N * N);
  for (int idx = threadIdx.x; idx < N * N; idx += NT) {
    const float2 z = sm[(idx / N) * LD + idx % N];
    spec[idx] = make_float2(z.x * s, z.y * s);
  }
}

template <int N>
__global__ void __launch_bounds__(FftShape<N>::NT) jcol_fft_kernel(const JcolFftWork* __restrict__ work,
                                                                   const SourceDev* __restrict__ srcs,
                                                                   const ImageDev* __restrict__ imgs,
                                                                   const float* __restrict__ dbuf,
                                                                   float* __restrict__ jbuf,
                                                                   const float2* __restrict__ tw_g) {
  constexpr int NT = FftShape<N>::NT, LD = FftShape<N>::LD;
  extern __shared__ float2 sm[];
  float2* tw = sm + N * LD;
  const JcolFftWork w = work[blockIdx.x];
  const SourceDev& sd = srcs[w.src];
  const ImageDev& im = imgs[sd.image];
  const int h = im.h, K = im.K, B = N - K + 1;
  const int bh = sd.box[1] - sd.box[0], bw = sd.box[3] - sd.box[2];
  const int64_t barea = (int64_t)bh * bw;
  const float* d1 = dbuf + sd.d_off + w.k * barea;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = tw_g[i];
  // derivative images on the block grown by K - 1 (box coordinates), zero outside the box
  const int y0 = w.by0 - h, x0 = w.bx0 - h;
  for (int idx = threadIdx.x; idx < N * N; idx += NT) {
    const int u = idx / N, v = idx % N;
    const int y = y0 + u, x = x0 + v;
    const bool in = y >= 0 && y < bh && x >= 0 && x < bw;
    const int64_t o = in ? (int64_t)y * bw + x : 0;
    sm[u * LD + v] = make_float2(in ? d1[o] : 0.f, 0.f);
  }
  __syncthreads();
  fft2_forward<N>(sm, tw);
  const float2* S = reinterpret_cast<const float2*>(N == 64 ? im.spec64 : im.spec128);
  for (int idx = threadIdx.x; idx < N * N; idx += NT) {
    float2& z = sm[(idx / N) * LD + idx % N];
    z = c_mul(z, S[idx]);
  }
  __syncthreads();
  fft2_inverse<N>(sm, tw);
  // outputs: block rows / columns [0, B) sit at [K - 1, N) of the circular result
  const int sh = sd.sup[1] - sd.sup[0], sw = sd.sup[3] - sd.sup[2];
  const int64_t sarea = (int64_t)sh * sw;
  float* o1 = jbuf + sd.j_off + w.k * sarea;
  for (int idx = threadIdx.x; idx < B * B; idx += NT) {
    const int i = idx / B, j = idx % B;
    const int oi = sd.box[0] + w.by0 + i, oj = sd.box[2] + w.bx0 + j;
    if (oi < sd.sup[0] || oi >= sd.sup[1] || oj < sd.sup[2] || oj >= sd.sup[3]) continue;
    const float2 z = sm[(i + K - 1) * LD + (j + K - 1)];
    const int64_t o = (int64_t)(oi - sd.sup[0]) * sw + (oj - sd.sup[2]);
    o1[o] = z.x;
  }
}

}  // namespace

// W_N^k, k < N, computed in float64 on the host
std::vector<float2> fft_twiddles(int N) {
  std::vector<float2> t(N);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < N; ++k) {
    const double a = -2.0 * pi * k / N;
    t[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  return t;
}

int configure_fft() {
  const int a = allow_max_dynamic_smem(jcol_fft_kernel<64>);
  const int b = allow_max_dynamic_smem(jcol_fft_kernel<128>);
  allow_max_dynamic_smem(psf_spectrum_kernel<64>);
  allow_max_dynamic_smem(psf_spectrum_kernel<128>);
  return a >= (int)FftShape<64>::smem && b >= (int)FftShape<128>::smem;
}

void launch_psf_spectrum(int N, const float* psf_norm, int K, int K4, const float2* tw, float2* spec,
                         cudaStream_t st) {
  if (N == 64)
    psf_spectrum_kernel<64><<<1, FftShape<64>::NT, FftShape<64>::smem, st>>>(psf_norm, K, K4, tw, spec);
  else if (N == 128)
    psf_spectrum_kernel<128><<<1, FftShape<128>::NT, FftShape<128>::smem, st>>>(psf_norm, K, K4, tw, spec);
}

void launch_jcol_fft(int N, const JcolFftWork* work, int n, const SourceDev* srcs, const ImageDev* imgs,
                     const float* dbuf, float* jbuf, const float2* tw, cudaStream_t st) {
  if (n <= 0) return;
  if (N == 64)
    jcol_fft_kernel<64><<<n, FftShape<64>::NT, FftShape<64>::smem, st>>>(work, srcs, imgs, dbuf, jbuf, tw);
  else if (N == 128)
    jcol_fft_kernel<128><<<n, FftShape<128>::NT, FftShape<128>::smem, st>>>(work, srcs, imgs, dbuf, jbuf, tw);
}

}  // namespace ap
