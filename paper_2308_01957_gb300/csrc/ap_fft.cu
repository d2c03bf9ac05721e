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
// One CTA per (source, slot, output block).  The input is real, so rows 2r
// and 2r + 1 ride in one complex row transform and are separated by
// Hermitian symmetry; only the N/2 + 1 non-redundant columns are transformed
// and multiplied, and the inverse packs the row pairs again (half the work of
// a complex transform; the leakage stays within the slot's own block).  The
// separation of the row pairs, the product with the PSF spectrum and the
// packing are folded into the first or last stage of the neighbouring line
// pass (no pass of their own through shared memory).  The
// block lives in shared memory; each 1-D pass is done by T = 8 threads
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

// a W_16^k (INV: the conjugate root).  k is a constant once the DFT loops
// are unrolled: the multiples of 90 degrees become swaps and sign changes
// (the same values the full complex product gives, without its products by
// 0 and -1, which the compiler keeps: x * 0 is not 0 for infinite or NaN x);
// the other roots take the full product
template <bool INV>
__device__ __forceinline__ float2 mul_w16(float2 a, int k) {
  switch (k & 15) {
    case 0: return a;
    case 4: return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);      // -i
    case 8: return make_float2(-a.x, -a.y);
    case 12: return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);     // +i
    default: {
      const float2 w = w16(k);
      return c_mul(a, INV ? c_conj(w) : w);
    }
  }
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
        const float2 a = v[i + j], b = mul_w16<INV>(v[i + j + len / 2], j * (16 / len));
        v[i + j] = c_add(a, b);
        v[i + j + len / 2] = c_sub(a, b);
      }
    }
  }
}

// One 1-D transform of length LEN on each of nlines lines of the array a:
// element j of line l sits at a[l * LS + j * ES].  twN[k] = W_LEN^k.  The NT
// threads take L = NT / T lines at a time: thread t works on line t mod L as
// member q = t / L of its line, so the 32 lanes of a warp touch 32 different
// lines at the same position -- consecutive (LS = 1) or an odd stride apart:
// no shared-memory bank conflicts.  The exchange between the members of a
// line goes through the line itself, separated by block barriers (rounds are
// uniform over the CTA).  The first stage takes its inputs from ld(line, j)
// and the last stage hands its outputs to st(line, j, value): both may read
// or write another layout of the same buffer (every load of the first stage
// precedes the first barrier, every store of the last stage follows the
// last one), which folds a neighbouring pass into the transform.
template <int LEN, int NT, int ES, int LS, bool INV, class LD, class ST>
__device__ __forceinline__ void fft_lines(float2* a, int nlines, const float2* twN, const LD& ld, const ST& st) {
  constexpr int T = FFT_T, E = LEN / T, G = E / T, L = NT / T;
  const int q = threadIdx.x / L;
  const int rounds = (nlines + L - 1) / L;
#pragma unroll 1
  for (int rd = 0; rd < rounds; ++rd) {
    const int line = rd * L + threadIdx.x % L;
    const bool act = line < nlines;
    float2* base = a + (act ? line : 0) * LS;
    float2 v[E];
    if (act) {
#pragma unroll
      for (int n1 = 0; n1 < E; ++n1) v[n1] = ld(line, T * n1 + q);
      dft_reg<E, INV>(v);
#pragma unroll
      for (int k1 = 1; k1 < E; ++k1) {
        const float2 w = twN[(q * k1) & (LEN - 1)];
        v[k1] = c_mul(v[k1], INV ? c_conj(w) : w);
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) base[(q + T * k1) * ES] = v[k1];
    }
    __syncthreads();
    float2 u[G][T];
    if (act) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int k1 = q + T * g;
#pragma unroll
        for (int n2 = 0; n2 < T; ++n2) u[g][n2] = base[(n2 + T * k1) * ES];
        dft_reg<T, INV>(u[g]);
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int k1 = q + T * g;
#pragma unroll
        for (int k2 = 0; k2 < T; ++k2) st(line, k1 + E * k2, u[g][k2]);
      }
    }
  }
}

// the plain transform: the lines read from and written back to the array
template <int LEN, int NT, int ES, int LS, bool INV>
__device__ __forceinline__ void fft_lines(float2* a, int nlines, const float2* twN) {
  auto ld = [a](int line, int j) { return a[line * LS + j * ES]; };
  auto st = [a](int line, int j, float2 v) { a[line * LS + j * ES] = v; };
  fft_lines<LEN, NT, ES, LS, INV>(a, nlines, twN, ld, st);
}

template <int N>
struct FftShape {
  static constexpr int NT = N * 4;          // threads: N / 2 lines at a time, T members each
  static constexpr int LD = N + 1;          // full complex N x N (PSF spectrum): odd row stride
  static constexpr size_t smem = (size_t)(N * LD + N) * sizeof(float2);
  // real-input transform of the Jacobian blocks: view A = N/2 packed rows of
  // N (row 2r + i row 2r+1), view B = N rows of N/2 + 1 half spectra; both
  // strides odd
  static constexpr int LDA = N + 1, LDB = N / 2 + 1;
  static constexpr int CELLS = (N / 2) * LDA > N * LDB ? (N / 2) * LDA : N * LDB;
  static constexpr size_t smem_r2c = (size_t)(CELLS + N) * sizeof(float2);
  // its threads: T members for each of the N/2 + 1 column lines, so every
  // pass of the real-input transform is one round
  static constexpr int NTR = FFT_T * (N / 2 + 1);
  static constexpr int MINB = N == 64 ? 3 : 2;   // CTAs per SM the register budget allows
};

template <int N>
__device__ __forceinline__ void fft2_forward(float2* a, const float2* tw) {
  constexpr int NT = FftShape<N>::NT, LD = FftShape<N>::LD;
  fft_lines<N, NT, 1, LD, false>(a, N, tw);
  __syncthreads();
  fft_lines<N, NT, LD, 1, false>(a, N, tw);
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
__global__ void __launch_bounds__(FftShape<N>::NTR, FftShape<N>::MINB) jcol_fft_kernel(const JcolFftWork* __restrict__ work,
                                                                   const SourceDev* __restrict__ srcs,
                                                                   const ImageDev* __restrict__ imgs,
                                                                   const float* __restrict__ dbuf,
                                                                   float* __restrict__ jbuf,
                                                                   const float2* __restrict__ tw_g) {
  constexpr int NT = FftShape<N>::NTR, LDA = FftShape<N>::LDA, LDB = FftShape<N>::LDB;
  constexpr int H = N / 2;                       // packed rows; half-spectrum length H + 1
  extern __shared__ float2 sm[];
  float2* tw = sm + FftShape<N>::CELLS;
  const JcolFftWork w = work[blockIdx.x];
  const SourceDev& sd = srcs[w.src];
  const ImageDev& im = imgs[sd.image];
  const int h = im.h, K = im.K, B = N - K + 1;
  const int bh = sd.box[1] - sd.box[0], bw = sd.box[3] - sd.box[2];
  const float* d1 = dbuf + sd.d_off + w.k * (int64_t)bh * bw;
  for (int i = threadIdx.x; i < N; i += NT) tw[i] = tw_g[i];
  // rows: view A row r = block rows 2r (real part) and 2r + 1 (imaginary
  // part) of the derivative image on the block grown by K - 1, zero outside
  // the box; loaded with consecutive threads on consecutive pixels of a row
  // (coalesced), then transformed in place
  const int y0 = w.by0 - h, x0 = w.bx0 - h;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < H * N; idx += NT) {
    const int r = idx / N, v = idx % N;
    const int y = y0 + 2 * r, x = x0 + v;
    const bool inx = x >= 0 && x < bw;
    const float a = (inx && y >= 0 && y < bh) ? d1[(int64_t)y * bw + x] : 0.f;
    const float b = (inx && y + 1 >= 0 && y + 1 < bh) ? d1[(int64_t)(y + 1) * bw + x] : 0.f;
    sm[r * LDA + v] = make_float2(a, b);
  }
  __syncthreads();
  auto ld_rows = [&](int r, int v) { return sm[r * LDA + v]; };
  auto st_a = [&](int r, int k, float2 z) { sm[r * LDA + k] = z; };
  fft_lines<N, NT, 1, LDA, false>(sm, H, tw, ld_rows, st_a);
  __syncthreads();
  // columns of view B (N rows of N/2 + 1 half spectra), the split of each
  // packed row spectrum Z into the spectra of its two real rows taken by the
  // first stage -- X_a[k] = (Z[k] + conj Z[N-k]) / 2,
  // X_b[k] = (Z[k] - conj Z[N-k]) / 2i, k = 0..N/2 (the rest is their
  // conjugate mirror) -- and the product with the PSF spectrum by the last
  auto ld_split = [&](int k, int n) {
    const int r = n >> 1;
    const float2 zk = sm[r * LDA + k], zm = c_conj(sm[r * LDA + ((N - k) & (N - 1))]);
    if (n & 1) {
      const float2 d = make_float2(0.5f * (zk.x - zm.x), 0.5f * (zk.y - zm.y));
      return make_float2(d.y, -d.x);
    }
    return make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
  };
  const float2* S = reinterpret_cast<const float2*>(N == 64 ? im.spec64 : im.spec128);
  auto st_mul = [&](int k, int n, float2 z) { sm[n * LDB + k] = c_mul(z, S[n * N + k]); };
  fft_lines<N, NT, LDB, 1, false>(sm, H + 1, tw, ld_split, st_mul);
  __syncthreads();
  fft_lines<N, NT, LDB, 1, true>(sm, H + 1, tw);
  __syncthreads();
  // inverse rows: the first stage packs the row pairs again, W = Y_a + i Y_b
  // over the full row (Hermitian extension of the half spectra); the
  // inverse of W is row a + i row b
  auto ld_pack = [&](int r, int k) {
    const bool lo = k <= H;
    const int kk = lo ? k : N - k;
    float2 ya = sm[(2 * r) * LDB + kk], yb = sm[(2 * r + 1) * LDB + kk];
    if (!lo) {
      ya = c_conj(ya);
      yb = c_conj(yb);
    }
    return make_float2(ya.x - yb.y, ya.y + yb.x);
  };
  fft_lines<N, NT, 1, LDA, true>(sm, H, tw, ld_pack, st_a);
  __syncthreads();
  // outputs: block rows / columns [0, B) sit at [K - 1, N) of the circular
  // result; thread t takes column t mod N of rows t / N, t / N + NT / N, ...
  const int sw = sd.sup[3] - sd.sup[2];
  float* o1 = jbuf + sd.j_off + w.k * (int64_t)(sd.sup[1] - sd.sup[0]) * sw;
  constexpr int RSTEP = NT / N;   // rows per sweep (the threads past RSTEP * N idle)
  const int j = threadIdx.x % N;
  const int oj = sd.box[2] + w.bx0 + j;
  if (threadIdx.x < RSTEP * N && j < B && oj >= sd.sup[2] && oj < sd.sup[3]) {
    for (int i = threadIdx.x / N; i < B; i += RSTEP) {
      const int oi = sd.box[0] + w.by0 + i;
      if (oi < sd.sup[0] || oi >= sd.sup[1]) continue;
      const int rho = i + K - 1;
      const float2 z = sm[(rho >> 1) * LDA + (j + K - 1)];
      o1[(int64_t)(oi - sd.sup[0]) * sw + (oj - sd.sup[2])] = (rho & 1) ? z.y : z.x;
    }
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
  const int c = allow_max_dynamic_smem(psf_spectrum_kernel<64>);
  const int d = allow_max_dynamic_smem(psf_spectrum_kernel<128>);
  return a >= (int)FftShape<64>::smem_r2c && b >= (int)FftShape<128>::smem_r2c && c >= (int)FftShape<64>::smem &&
         d >= (int)FftShape<128>::smem;
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
    jcol_fft_kernel<64><<<n, FftShape<64>::NTR, FftShape<64>::smem_r2c, st>>>(work, srcs, imgs, dbuf, jbuf, tw);
  else if (N == 128)
    jcol_fft_kernel<128><<<n, FftShape<128>::NTR, FftShape<128>::smem_r2c, st>>>(work, srcs, imgs, dbuf, jbuf,
                                                                                   tw);
}

}  // namespace ap
