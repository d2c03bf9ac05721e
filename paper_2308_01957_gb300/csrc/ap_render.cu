// Source preparation (Sersic b_n in float64), per-pixel Gauss-Legendre
// render and the derivative (adjoint) render.
//
// Paper: Sec. "A Zoo of Models" (profiles), Sec. "Pixel Integration" (order-Q
// Gauss-Legendre per pixel, Q^2 evaluations), Sec. "Implementation with
// PyTorch" (gradient of chi^2 by back-propagation, here a hand-written adjoint).
#include <math.h>

#include <cmath>
#include <vector>

#include "ap_internal.cuh"

namespace ap {

// ---------------------------------------------------------------------------
// Gauss-Legendre rules for Q = 1..7, built on the host by Newton iteration on
// the Legendre recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; weights
// w = 2 / ((1 - x^2) P_Q'(x)^2).  Stored as half offsets u/2 (a node of pixel
// (i, j) sits at (j + 1/2 + u_a/2, i + 1/2 + u_b/2)) and half weights w/2, so a
// pixel value is area * sum_ab (w_a/2)(w_b/2) I(node).
// ---------------------------------------------------------------------------
__constant__ float c_hu_f[8][8];
__constant__ float c_hw_f[8][8];
__constant__ double c_hu_d[8][8];
__constant__ double c_hw_d[8][8];

static void legendre_rule(int Q, double* x, double* w) {
  for (int i = 0; i < Q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (Q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < Q; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      double pq = (Q == 0) ? 1.0 : p1;      // P_Q(z)
      double pqm = (Q == 1) ? 1.0 : p0;     // P_{Q-1}(z)
      if (Q == 1) { pq = z; pqm = 1.0; }
      dp = Q * (z * pq - pqm) / (z * z - 1.0);
      double dz = pq / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute the derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < Q; ++k) {
      double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    double pq = p1, pqm = (Q == 1) ? 1.0 : p0;
    dp = Q * (z * pq - pqm) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void upload_gl_rule(int /*Q*/) {
  static bool done = false;
  if (done) return;
  float hu_f[8][8] = {}, hw_f[8][8] = {};
  double hu_d[8][8] = {}, hw_d[8][8] = {};
  for (int Q = 1; Q <= 7; ++Q) {
    double x[8], w[8];
    legendre_rule(Q, x, w);
    for (int a = 0; a < Q; ++a) {
      hu_d[Q][a] = 0.5 * x[a];
      hw_d[Q][a] = 0.5 * w[a];
      hu_f[Q][a] = (float)hu_d[Q][a];
      hw_f[Q][a] = (float)hw_d[Q][a];
    }
  }
  cudaMemcpyToSymbol(c_hu_f, hu_f, sizeof(hu_f));
  cudaMemcpyToSymbol(c_hw_f, hw_f, sizeof(hw_f));
  cudaMemcpyToSymbol(c_hu_d, hu_d, sizeof(hu_d));
  cudaMemcpyToSymbol(c_hw_d, hw_d, sizeof(hw_d));
  done = true;
}

template <typename T> __device__ __forceinline__ T gl_hu(int Q, int a);
template <> __device__ __forceinline__ float gl_hu<float>(int Q, int a) { return c_hu_f[Q][a]; }
template <> __device__ __forceinline__ double gl_hu<double>(int Q, int a) { return c_hu_d[Q][a]; }
template <typename T> __device__ __forceinline__ T gl_hw(int Q, int a);
template <> __device__ __forceinline__ float gl_hw<float>(int Q, int a) { return c_hw_f[Q][a]; }
template <> __device__ __forceinline__ double gl_hw<double>(int Q, int a) { return c_hw_d[Q][a]; }

// math in the path's precision
__device__ __forceinline__ float p_exp2(float x) { return exp2f(x); }
__device__ __forceinline__ double p_exp2(double x) { return exp2(x); }
__device__ __forceinline__ float p_log2(float x) { return __log2f(x); }
__device__ __forceinline__ double p_log2(double x) { return log2(x); }
// logarithms of the derivative render: the hardware log2 (its absolute error,
// about 2^-22, reaches t = 2^(k0 log2 u) and ln u as a relative error of the
// order of float32 rounding; the J^T W J and step parity tests hold with it)
__device__ __forceinline__ float d_log2(float x) { return __log2f(x); }
__device__ __forceinline__ double d_log2(double x) { return log2(x); }

constexpr double LOG2E = 1.4426950408889634074;
constexpr double LN2 = 0.69314718055994530942;

// ---------------------------------------------------------------------------
// Sersic b_n in float64 (Sersic 1963; half the light inside Re):
// root of P(2n, b) = 1/2 with P the regularised lower incomplete gamma.
//  * P(a, x) by its power series x^a e^-x / Gamma(a+1) sum_k x^k / prod_{j<=k}(a+j)
//    (the root satisfies x < a + 1, where the series converges geometrically);
//  * dP/da by differentiating the series term by term, with the digamma
//    function from its recurrence and asymptotic (Bernoulli) expansion;
//  * safeguarded Newton from the Ciotti & Bertin (1999) asymptotic start,
//    inside the bracket [0, a + 2];
//  * db/dn = -2 (dP/da) / (dP/dx), dP/dx = x^(a-1) e^-x / Gamma(a).
// ---------------------------------------------------------------------------
__device__ double digamma_pos(double z) {
  double acc = 0.0;
  while (z < 10.0) {
    acc -= 1.0 / z;
    z += 1.0;
  }
  double iz = 1.0 / z, iz2 = iz * iz;
  double series = iz2 * (1.0 / 12.0 - iz2 * (1.0 / 120.0 - iz2 * (1.0 / 252.0 - iz2 * (1.0 / 240.0 - iz2 * (1.0 / 132.0)))));
  return acc + log(z) - 0.5 * iz - series;
}

// Reciprocal in float64 by two Newton-Raphson steps r <- r (2 - d r) from a
// float32 seed (relative error squares each step: 1e-7 -> 1e-14 -> 1e-28).
__device__ __forceinline__ double recip64(double d) {
  double r = (double)(1.0f / (float)d);
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}

// One warp sums the series S = sum_{k>=0} x^k / prod_{j<=k}(a+j) and its
// a-derivative dS = -sum_k t_k H_k, H_k = sum_{j<=k} 1/(a+j).  Lane l holds
// the factor x/(a+k) of term k = 32c + l + 1; an inclusive multiplicative
// shuffle scan gives a chunk of 32 terms, an additive scan the harmonic sums;
// chunks continue from the previous chunk's last lane until a term drops
// below 1e-18 (S >= 1).  Every lane returns the totals.
__device__ void gamma_series_warp(double a, double x, double* S, double* dS) {
  const int lane = threadIdx.x & 31;
  double sum = 0.0, dsum = 0.0, carry_t = 1.0, carry_h = 0.0;
  for (int chunk = 0; chunk < 8; ++chunk) {
    const double ak = recip64(a + (double)(32 * chunk + lane + 1));
    double t = x * ak, hs = ak;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double tv = __shfl_up_sync(0xffffffffu, t, o);
      const double hv = __shfl_up_sync(0xffffffffu, hs, o);
      if (lane >= o) { t *= tv; hs += hv; }
    }
    t *= carry_t;
    hs += carry_h;
    sum += t;
    dsum -= t * hs;
    carry_t = __shfl_sync(0xffffffffu, t, 31);
    carry_h = __shfl_sync(0xffffffffu, hs, 31);
    if (carry_t < 1e-18) break;   // uniform: every lane holds the same carry
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  }
  *S = 1.0 + sum;
  *dS = dsum;
}

// All 32 lanes of a warp call this with the same n and get the same result.
// With f'(b) = b^(a-1) e^-b / Gamma(a), P(a, b) = (b / a) f'(b) S(a, b), so an
// iteration costs one exp, one log and one warp series.  Halley steps
// (f''/f' = (a-1)/b - 1) inside the bracket [0, a + 2], bisection if a step
// leaves it.
__device__ void sersic_bn(double n, double* b_out, double* db_out, int* ok) {
  const double a = 2.0 * n;
  const double lga = lgamma(a);
  double lo = 0.0, hi = a + 2.0;
  double b = 2.0 * n - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n * n);
  if (!(b > lo && b < hi)) b = 0.5 * (lo + hi);
  int conv = 0;
  double fp = 0.0, S = 1.0, dS = 0.0;
  for (int it = 0; it < 60; ++it) {
    fp = exp((a - 1.0) * log(b) - b - lga);
    gamma_series_warp(a, b, &S, &dS);
    const double f = b * fp * S / a - 0.5;
    if (f < 0.0) lo = b; else hi = b;
    const double h = f / fp;
    const double c = (a - 1.0) / b - 1.0;
    const double step = h / (1.0 - 0.5 * h * c);
    // Halley converges cubically: once a step is below 1e-9 b the stepped
    // iterate is accurate to float64 rounding.  (Tested before the bracket:
    // a last step smaller than half an ulp lands on the bracket end.)
    if (fabs(step) <= 1e-9 * b) { b -= step; conv = 1; break; }
    double nb = b - step;
    if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
    b = nb;
    if (hi - lo <= 4e-16 * b) { conv = 1; break; }
  }
  fp = exp((a - 1.0) * log(b) - b - lga);
  gamma_series_warp(a, b, &S, &dS);
  const double P = b * fp * S / a;
  const double dPda = P * (log(b) - digamma_pos(a + 1.0)) + b * fp / a * dS;
  *b_out = b;
  *db_out = -2.0 * dPda / fp;
  *ok = conv && isfinite(b) && isfinite(*db_out);
}

// ---------------------------------------------------------------------------
// prepare: one warp per source, float64, from theta to the SrcPar record
// (the warp shares the b_n series; lane 0 stores the record)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void prepare_kernel(const SourceDev* __restrict__ srcs, const ImageDev* __restrict__ imgs, int n_src,
                               const double* __restrict__ theta, SrcPar<T>* __restrict__ par, double* bn_memo,
                               const int* __restrict__ skip, int* status) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (s >= n_src) return;   // whole warps exit together
  const SourceDev& sd = srcs[s];
  const ImageDev& im = imgs[sd.image];
  if (skip && skip[im.group]) return;   // the record already holds this point
  double p[MAX_SLOTS];
  for (int k = 0; k < MAX_SLOTS; ++k) p[k] = (k < sd.nslot) ? (sd.pidx[k] >= 0 ? theta[sd.pidx[k]] : sd.pfix[k]) : 0.0;
  SrcPar<T> r;
  for (int k = 0; k < MAX_SLOTS; ++k) r.pv[k] = (T)p[k];
  r.area = (T)im.area;
  r.m00 = r.m01 = r.m10 = r.m11 = r.invq = r.fx = r.fy = r.c = r.s = (T)0;
  r.k0 = r.k1 = r.k2 = r.k3 = r.k4 = r.k5 = r.k6 = (T)0;
  r.jc = r.ic = 0;
  r.pad_[0] = r.pad_[1] = 0;
  bool good = true;
  if (sd.type == AP_SKY_PLANE) {
    // the plane's geometry in T, so that the per-pixel code converts nothing
    // from float64: pixel -> world matrix and the image centre in pixels
    r.m00 = (T)im.A[0];
    r.m01 = (T)im.A[1];
    r.m10 = (T)im.A[2];
    r.m11 = (T)im.A[3];
    r.fx = (T)(0.5 * im.W);
    r.fy = (T)(0.5 * im.H);
  }
  if (sd.type == AP_PSF_STAR) {
    // pixel position of the star; the pixel -> map frame needs A^-1 for the
    // position derivatives; k0 = F, k1 = the map's centre index (K - 1) / 2
    double wx = p[0] - im.origin[0], wy = p[1] - im.origin[1];
    double u = im.Ainv[0] * wx + im.Ainv[1] * wy;
    double v = im.Ainv[2] * wx + im.Ainv[3] * wy;
    double fu = floor(u), fv = floor(v);
    good = isfinite(u) && isfinite(v) && fabs(u) < 1e9 && fabs(v) < 1e9 && im.K > 0;
    r.jc = good ? (int)fu : 0;
    r.ic = good ? (int)fv : 0;
    r.fx = (T)(u - fu);
    r.fy = (T)(v - fv);
    r.m00 = (T)im.Ainv[0];
    r.m01 = (T)im.Ainv[1];
    r.m10 = (T)im.Ainv[2];
    r.m11 = (T)im.Ainv[3];
    r.k0 = (T)p[2];
    r.k1 = (T)(0.5 * (im.K - 1));
  }
  if (sd.type <= AP_MOFFAT) {
    double x0 = p[0], y0 = p[1], q = p[2], PA = p[3];
    double wx = x0 - im.origin[0], wy = y0 - im.origin[1];
    double u = im.Ainv[0] * wx + im.Ainv[1] * wy;
    double v = im.Ainv[2] * wx + im.Ainv[3] * wy;
    double fu = floor(u), fv = floor(v);
    good = good && isfinite(u) && isfinite(v) && fabs(u) < 1e9 && fabs(v) < 1e9 && q > 0.0;
    r.jc = good ? (int)fu : 0;
    r.ic = good ? (int)fv : 0;
    r.fx = (T)(u - fu);
    r.fy = (T)(v - fv);
    double c = cos(PA), sn = sin(PA);
    r.c = (T)c;
    r.s = (T)sn;
    r.m00 = (T)(c * im.A[0] + sn * im.A[2]);
    r.m01 = (T)(c * im.A[1] + sn * im.A[3]);
    r.m10 = (T)(-sn * im.A[0] + c * im.A[2]);
    r.m11 = (T)(-sn * im.A[1] + c * im.A[3]);
    r.invq = (T)(1.0 / q);
    if (sd.type == AP_SERSIC || sd.type == AP_EXPONENTIAL) {
      double n = (sd.type == AP_SERSIC) ? p[4] : 1.0;
      double Re = (sd.type == AP_SERSIC) ? p[5] : p[4];
      double Ie = (sd.type == AP_SERSIC) ? p[6] : p[5];
      double b = 0.0, db = 0.0;
      int ok = 0;
      if (n >= 0.05 && n <= 20.0) {
        // b_n is a function of n alone: a two-entry memo per source (the
        // current point and the last trial point) keyed on the bits of n.
        // Every lane reads the same entries, so the branch is warp-uniform.
        double* mc = bn_memo + 8 * (int64_t)s;
        const long long key = __double_as_longlong(n);
        bool hit = false;
        for (int slot = 0; slot < 2 && !hit; ++slot)
          if (__double_as_longlong(mc[3 * slot]) == key) {
            b = mc[3 * slot + 1];
            db = mc[3 * slot + 2];
            ok = 1;
            hit = true;
          }
        if (!hit) {
          sersic_bn(n, &b, &db, &ok);
          if (ok && (threadIdx.x & 31) == 0) {
            const int slot = mc[6] == 1.0 ? 1 : 0;   // the older entry (a NaN start reads as 0)
            mc[3 * slot] = n;
            mc[3 * slot + 1] = b;
            mc[3 * slot + 2] = db;
            mc[6] = 1.0 - slot;
          }
        }
      }
      good = good && ok && Re > 0.0;
      r.k0 = (T)(0.5 / n);
      r.k1 = (T)(1.0 / (Re * Re));
      r.k2 = (T)(b * LOG2E);
      r.k3 = (T)Ie;
      r.k4 = (T)b;
      r.k5 = (T)db;
      r.k6 = (T)n;
    } else if (sd.type == AP_GAUSSIAN) {
      double sg = p[4], F = p[5];
      good = good && sg > 0.0;
      double nrm = 1.0 / (2.0 * M_PI * sg * sg * q);
      r.k0 = (T)(-LOG2E / (2.0 * sg * sg));
      r.k1 = (T)(F * nrm);
      r.k2 = (T)(1.0 / (sg * sg));
      r.k3 = (T)nrm;
    } else {  // Moffat
      double n = p[4], Rd = p[5], F = p[6];
      good = good && Rd > 0.0 && n > 1.0;
      double nrm = (n - 1.0) / (M_PI * Rd * Rd * q);
      r.k0 = (T)(1.0 / (Rd * Rd));
      r.k1 = (T)(F * nrm);
      r.k2 = (T)n;
      r.k3 = (T)nrm;
      r.k4 = (T)(1.0 / (n - 1.0));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    if (!good) atomicCAS(status, 0, AP_ERR_NONFINITE);
    par[s] = r;
  }
}

template <typename T>
void launch_prepare(const SourceDev* srcs, const ImageDev* imgs, int n_src, const double* theta, SrcPar<T>* par,
                    double* bn_memo, const int* skip, int* status, cudaStream_t st) {
  if (n_src <= 0) return;
  prepare_kernel<T><<<n_src, 32, 0, st>>>(srcs, imgs, n_src, theta, par, bn_memo, skip, status);
}

// ---------------------------------------------------------------------------
// PSF star (Sec. "A Zoo of Models"): the bilinear interpolant B of the
// image's normalised PSF map at the continuous map index (X, Y) (pixel
// centres at integers, X along columns, zero beyond the map), and its
// derivatives along X and Y (constant inside a map cell).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void psf_bilinear(const T* __restrict__ map, int K, int K4, T X, T Y, T& B, T& dX, T& dY) {
  const T fx = floor(X), fy = floor(Y);
  const int bx = (int)fx, by = (int)fy;
  const T tx = X - fx, ty = Y - fy;
  auto at = [&](int r, int q) -> T { return (r >= 0 && r < K && q >= 0 && q < K) ? map[r * K4 + q] : (T)0; };
  const T p00 = at(by, bx), p01 = at(by, bx + 1), p10 = at(by + 1, bx), p11 = at(by + 1, bx + 1);
  const T top = p00 + tx * (p01 - p00), bot = p10 + tx * (p11 - p10);
  B = top + ty * (bot - top);
  dX = (p01 - p00) + ty * ((p11 - p10) - (p01 - p00));
  dY = bot - top;
}

// ---------------------------------------------------------------------------
// value of one source on one pixel: area * sum_ab (w_a/2)(w_b/2) I(node_ab)
// ---------------------------------------------------------------------------
template <typename T, int Q>
__device__ __forceinline__ T pixel_value(int type, const SrcPar<T>& P, int i, int j, const ImageDev& im) {
  if (type == AP_LIVE_PSF_SRC) return (T)0;   // a live PSF draws nothing itself
  if (type == AP_SKY_FLAT) return P.area * P.pv[0];
  if (type == AP_PSF_STAR) {
    // F times the pixel integral of B (light per unit pixel area F B)
    const T* map = (const T*)im.psf_norm;
    const T X0 = P.k1 + (T)(j - P.jc) + ((T)0.5 - P.fx);
    const T Y0 = P.k1 + (T)(i - P.ic) + ((T)0.5 - P.fy);
    T acc = (T)0;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const T Y = Y0 + gl_hu<T>(Q, b);
      T accb = (T)0;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        T B, dX, dY;
        psf_bilinear<T>(map, im.K, im.K4, X0 + gl_hu<T>(Q, a), Y, B, dX, dY);
        accb += gl_hw<T>(Q, a) * B;
      }
      acc += gl_hw<T>(Q, b) * accb;
    }
    return P.k0 * acc;
  }
  if (type == AP_SKY_PLANE) {
    T du = (T)j + (T)0.5 - P.fx;
    T dv = (T)i + (T)0.5 - P.fy;
    T dxw = P.m00 * du + P.m01 * dv;
    T dyw = P.m10 * du + P.m11 * dv;
    return P.area * (P.pv[0] + P.pv[1] * dxw + P.pv[2] * dyw);
  }
  const T du0 = (T)(j - P.jc) + ((T)0.5 - P.fx);
  const T dv0 = (T)(i - P.ic) + ((T)0.5 - P.fy);
  const T X0 = P.m00 * du0 + P.m01 * dv0;
  const T Y0 = P.m10 * du0 + P.m11 * dv0;
  T acc = (T)0;
  if (type == AP_SERSIC || type == AP_EXPONENTIAL) {
    const T eps2 = (T)1e-8 * P.area;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const T hb = gl_hu<T>(Q, b);
      const T Xb = X0 + P.m01 * hb, Yb = Y0 + P.m11 * hb;
      T accb = (T)0;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const T ha = gl_hu<T>(Q, a);
        const T X = Xb + P.m00 * ha;
        const T Yq = (Yb + P.m10 * ha) * P.invq;
        const T r2 = X * X + Yq * Yq + eps2;
        const T t = p_exp2(P.k0 * p_log2(r2 * P.k1));
        accb += gl_hw<T>(Q, a) * p_exp2(P.k2 * ((T)1 - t));
      }
      acc += gl_hw<T>(Q, b) * accb;
    }
    return P.area * P.k3 * acc;
  }
  if (type == AP_GAUSSIAN) {
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const T hb = gl_hu<T>(Q, b);
      const T Xb = X0 + P.m01 * hb, Yb = Y0 + P.m11 * hb;
      T accb = (T)0;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const T ha = gl_hu<T>(Q, a);
        const T X = Xb + P.m00 * ha;
        const T Yq = (Yb + P.m10 * ha) * P.invq;
        accb += gl_hw<T>(Q, a) * p_exp2(P.k0 * (X * X + Yq * Yq));
      }
      acc += gl_hw<T>(Q, b) * accb;
    }
    return P.area * P.k1 * acc;
  }
  // Moffat: I0 (1 + rho^2/Rd^2)^-n
#pragma unroll
  for (int b = 0; b < Q; ++b) {
    const T hb = gl_hu<T>(Q, b);
    const T Xb = X0 + P.m01 * hb, Yb = Y0 + P.m11 * hb;
    T accb = (T)0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const T ha = gl_hu<T>(Q, a);
      const T X = Xb + P.m00 * ha;
      const T Yq = (Yb + P.m10 * ha) * P.invq;
      const T v = (T)1 + (X * X + Yq * Yq) * P.k0;
      accb += gl_hw<T>(Q, a) * p_exp2(-P.k2 * p_log2(v));
    }
    acc += gl_hw<T>(Q, b) * accb;
  }
  return P.area * P.k1 * acc;
}

// ---------------------------------------------------------------------------
// render: one CTA per TILE x TILE tile of a layer, 128 threads, each thread
// two pixels of one column (rows ly and ly + 8), looping over the sources
// whose sampling box meets the tile.  A gather: every pixel is written once,
// in a fixed order, so the result is deterministic.  Two pixels per thread
// halve the per-source parameter loads per quadrature node and give the two
// independent node chains to interleave.
// ---------------------------------------------------------------------------
constexpr int RENDER_THREADS = TILE_THREADS / 2;

template <typename T, int Q>
__global__ void __launch_bounds__(RENDER_THREADS) render_kernel(const TileWork* __restrict__ work,
                                                                const int* __restrict__ tile_src,
                                                                const SourceDev* __restrict__ srcs,
                                                                const SrcPar<T>* __restrict__ par,
                                                                const ImageDev* __restrict__ imgs,
                                                                const int* __restrict__ skip) {
  const TileWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  if (skip && skip[im.group]) return;   // the layer already holds this point
  const int j = w.c0 + (int)(threadIdx.x % TILE);
  const int i0 = w.r0 + (int)(threadIdx.x / TILE), i1 = i0 + TILE / 2;
  const int h = w.plane == 0 ? im.h : 0;
  const int rows = w.plane == 0 ? im.Hp : im.H;
  const int cols = w.plane == 0 ? im.Wp : im.W;
  T acc0 = (T)0, acc1 = (T)0;
  for (int e = w.e0; e < w.e1; ++e) {
    const int s = tile_src[e];
    const SourceDev& sd = srcs[s];
    const bool cin = j >= sd.box[2] && j < sd.box[3];
    const bool in0 = cin && i0 >= sd.box[0] && i0 < sd.box[1];
    const bool in1 = cin && i1 >= sd.box[0] && i1 < sd.box[1];
    if (in0 || in1) {
      const SrcPar<T> P = par[s];
      const T v0 = pixel_value<T, Q>(sd.type, P, i0, j, im);
      const T v1 = pixel_value<T, Q>(sd.type, P, i1, j, im);
      acc0 += in0 ? v0 : (T)0;
      acc1 += in1 ? v1 : (T)0;
    }
  }
  T* out = (T*)(w.plane == 0 ? im.gal : im.unc);
  if (j + h < cols) {
    if (i0 + h < rows) out[(size_t)(i0 + h) * cols + (j + h)] = acc0;
    if (i1 + h < rows) out[(size_t)(i1 + h) * cols + (j + h)] = acc1;
  }
}

template <typename T>
void launch_render(int Q, const TileWork* work, int n_work, const int* tile_src, const SourceDev* srcs,
                   const SrcPar<T>* par, const ImageDev* imgs, const int* skip, cudaStream_t st) {
  if (n_work <= 0) return;
  switch (Q) {
    case 1: render_kernel<T, 1><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, skip); break;
    case 3: render_kernel<T, 3><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, skip); break;
    case 5: render_kernel<T, 5><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, skip); break;
    default: render_kernel<T, 7><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, skip); break;
  }
}

// ---------------------------------------------------------------------------
// derivative render: d(pixel value)/d(slot) for every slot of one source
// ---------------------------------------------------------------------------
template <typename T, int Q>
__device__ __forceinline__ void pixel_derivs(int type, const SrcPar<T>& P, int i, int j, const ImageDev& im,
                                             T* D) {
#pragma unroll
  for (int k = 0; k < MAX_SLOTS; ++k) D[k] = (T)0;
  if (type == AP_SKY_FLAT) {
    D[0] = P.area;
    return;
  }
  if (type == AP_SKY_PLANE) {
    T du = (T)j + (T)0.5 - P.fx;
    T dv = (T)i + (T)0.5 - P.fy;
    D[0] = P.area;
    D[1] = P.area * (P.m00 * du + P.m01 * dv);
    D[2] = P.area * (P.m10 * du + P.m11 * dv);
    return;
  }
  if (type == AP_PSF_STAR) {
    // X = c + u - u0(x0, y0): dX/dx0 = -A^-1_00, dX/dy0 = -A^-1_01, Y likewise
    const T* map = (const T*)im.psf_norm;
    const T X0 = P.k1 + (T)(j - P.jc) + ((T)0.5 - P.fx);
    const T Y0 = P.k1 + (T)(i - P.ic) + ((T)0.5 - P.fy);
    T sB = (T)0, sX = (T)0, sY = (T)0;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const T Y = Y0 + gl_hu<T>(Q, b);
      const T wb = gl_hw<T>(Q, b);
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        T B, dX, dY;
        psf_bilinear<T>(map, im.K, im.K4, X0 + gl_hu<T>(Q, a), Y, B, dX, dY);
        const T w = wb * gl_hw<T>(Q, a);
        sB += w * B;
        sX += w * dX;
        sY += w * dY;
      }
    }
    D[0] = -P.k0 * (P.m00 * sX + P.m10 * sY);
    D[1] = -P.k0 * (P.m01 * sX + P.m11 * sY);
    D[2] = sB;
    return;
  }
  const T du0 = (T)(j - P.jc) + ((T)0.5 - P.fx);
  const T dv0 = (T)(i - P.ic) + ((T)0.5 - P.fy);
  const T X0 = P.m00 * du0 + P.m01 * dv0;
  const T Y0 = P.m10 * du0 + P.m11 * dv0;
  const T c = P.c, s = P.s, iq = P.invq;
  const T iq2 = iq * iq;
  // accumulate d I / d rho^2 times the pieces of d rho^2 / d(x0, y0, q, PA)
  T a_x0 = 0, a_y0 = 0, a_q = 0, a_pa = 0, a_4 = 0, a_5 = 0, a_6 = 0;
  if (type == AP_SERSIC || type == AP_EXPONENTIAL) {
    const T eps2 = (T)1e-8 * P.area;
    const T k0 = P.k0, k1 = P.k1, k2 = P.k2, b = P.k4, db = P.k5, n = P.k6;
    const T Ie = P.k3;
#pragma unroll
    for (int bb = 0; bb < Q; ++bb) {
      const T hb = gl_hu<T>(Q, bb);
      const T wb = gl_hw<T>(Q, bb);
      const T Xb = X0 + P.m01 * hb, Yb = Y0 + P.m11 * hb;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const T ha = gl_hu<T>(Q, a);
        const T w = wb * gl_hw<T>(Q, a);
        const T X = Xb + P.m00 * ha;
        const T Y = Yb + P.m10 * ha;
        const T Yq = Y * iq;
        const T r2 = X * X + Yq * Yq + eps2;
        const T lt = k0 * d_log2(r2 * k1);       // log2 t
        const T t = p_exp2(lt);                  // (R/Re)^(1/n)
        const T e = p_exp2(k2 * ((T)1 - t));     // exp(-b (t - 1))
        const T we = w * e;
        const T g = -we * Ie * b * t * k0 / r2;  // w dI/d rho^2
        const T YqQ = Yq * iq;                   // Y / q^2
        a_x0 += g * (-X * c + YqQ * s);
        a_y0 += g * (-X * s - YqQ * c);
        a_q += g * (Yq * Yq * iq);
        a_pa += g * (X * Y);
        a_5 += we * t;                           // -> dI/dRe = I b t / (n Re)
        a_6 += we;                               // -> dI/dIe = e
        a_4 += we * (-db * (t - (T)1) + b * t * (T)LN2 * lt / n);  // -> dI/dn / Ie
      }
    }
    D[0] = (T)2 * a_x0;
    D[1] = (T)2 * a_y0;
    D[2] = (T)-2 * a_q;
    D[3] = (T)2 * (1 - iq2) * a_pa;
    if (type == AP_SERSIC) {
      D[4] = Ie * a_4;
      D[5] = Ie * b * a_5 / (n * P.pv[5]);
      D[6] = a_6;
    } else {
      D[4] = Ie * b * a_5 / (n * P.pv[4]);
      D[5] = a_6;
    }
  } else if (type == AP_GAUSSIAN) {
    const T k0 = P.k0, F = P.pv[5], sg = P.pv[4], isg2 = P.k2, nrm = P.k3;
    T a_r2 = 0;
#pragma unroll
    for (int bb = 0; bb < Q; ++bb) {
      const T hb = gl_hu<T>(Q, bb);
      const T wb = gl_hw<T>(Q, bb);
      const T Xb = X0 + P.m01 * hb, Yb = Y0 + P.m11 * hb;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const T ha = gl_hu<T>(Q, a);
        const T w = wb * gl_hw<T>(Q, a);
        const T X = Xb + P.m00 * ha;
        const T Y = Yb + P.m10 * ha;
        const T Yq = Y * iq;
        const T r2 = X * X + Yq * Yq;
        const T we = w * p_exp2(k0 * r2) * nrm;  // w e, I = F e
        const T g = -we * F * (T)0.5 * isg2;      // w dI/d rho^2
        const T YqQ = Yq * iq;
        a_x0 += g * (-X * c + YqQ * s);
        a_y0 += g * (-X * s - YqQ * c);
        a_q += g * (Yq * Yq * iq);
        a_pa += g * (X * Y);
        a_6 += we;
        a_r2 += we * r2;
      }
    }
    D[0] = (T)2 * a_x0;
    D[1] = (T)2 * a_y0;
    D[2] = (T)-2 * a_q - F * a_6 * iq;
    D[3] = (T)2 * (1 - iq2) * a_pa;
    D[4] = F * (-(T)2 * a_6 + a_r2 * isg2) / sg;
    D[5] = a_6;
  } else {  // Moffat
    const T k0 = P.k0, n = P.k2, nrm = P.k3, inm1 = P.k4, F = P.pv[6], Rd = P.pv[5];
    T a_lv = 0, a_rv = 0;
#pragma unroll
    for (int bb = 0; bb < Q; ++bb) {
      const T hb = gl_hu<T>(Q, bb);
      const T wb = gl_hw<T>(Q, bb);
      const T Xb = X0 + P.m01 * hb, Yb = Y0 + P.m11 * hb;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const T ha = gl_hu<T>(Q, a);
        const T w = wb * gl_hw<T>(Q, a);
        const T X = Xb + P.m00 * ha;
        const T Y = Yb + P.m10 * ha;
        const T Yq = Y * iq;
        const T r2 = X * X + Yq * Yq;
        const T v = (T)1 + r2 * k0;
        const T lv = d_log2(v);
        const T we = w * p_exp2(-n * lv) * nrm;  // w e, I = F e
        const T iv = (T)1 / v;
        const T g = -we * F * n * k0 * iv;       // w dI/d rho^2
        const T YqQ = Yq * iq;
        a_x0 += g * (-X * c + YqQ * s);
        a_y0 += g * (-X * s - YqQ * c);
        a_q += g * (Yq * Yq * iq);
        a_pa += g * (X * Y);
        a_6 += we;
        a_lv += we * lv;
        a_rv += we * r2 * iv;
      }
    }
    D[0] = (T)2 * a_x0;
    D[1] = (T)2 * a_y0;
    D[2] = (T)-2 * a_q - F * a_6 * iq;
    D[3] = (T)2 * (1 - iq2) * a_pa;
    D[4] = F * (inm1 * a_6 - (T)LN2 * a_lv);
    D[5] = F * (T)2 / Rd * (-a_6 + n * k0 * a_rv);
    D[6] = a_6;
  }
#pragma unroll
  for (int k = 0; k < MAX_SLOTS; ++k) D[k] *= P.area;
}

// adjoint render: per tile, per source meeting the tile, the block sum over
// the tile's pixels of adj(p) * dm_s(p)/d(slot) into partial[e][slot]
// (float64).  adj is the PSF-correlated w r on the galaxy layer, w r itself
// on the unconvolved layer.  Optionally stores the derivative images.  Same
// thread layout as the render: two pixels of one column per thread.
template <typename T>
__device__ __forceinline__ void store_derivs(T* dbuf, const SourceDev& sd, int i, int j, const T (&D)[MAX_SLOTS]) {
  const int bw = sd.box[3] - sd.box[2];
  const int64_t barea = (int64_t)(sd.box[1] - sd.box[0]) * bw;
  T* dst = dbuf + sd.d_off + (int64_t)(i - sd.box[0]) * bw + (j - sd.box[2]);
#pragma unroll
  for (int k = 0; k < MAX_SLOTS; ++k)
    if (k < sd.nslot) dst[k * barea] = D[k];
}

template <typename T, int Q>
__global__ void __launch_bounds__(RENDER_THREADS) render_adjoint_kernel(
    const TileWork* __restrict__ work, const int* __restrict__ tile_src, const SourceDev* __restrict__ srcs,
    const SrcPar<T>* __restrict__ par, const ImageDev* __restrict__ imgs, double* __restrict__ partial,
    T* __restrict__ dbuf) {
  constexpr int NW = RENDER_THREADS / 32;
  __shared__ T red[NW][MAX_SLOTS];
  const TileWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = w.c0 + (int)(threadIdx.x % TILE);
  const int i0 = w.r0 + (int)(threadIdx.x / TILE), i1 = i0 + TILE / 2;
  const int h = w.plane == 0 ? im.h : 0;
  const int rows = w.plane == 0 ? im.Hp : im.H;
  const int cols = w.plane == 0 ? im.Wp : im.W;
  const bool jin = j + h < cols;
  const bool ok0 = jin && i0 + h < rows, ok1 = jin && i1 + h < rows;
  const T* a = (const T*)(w.plane == 0 ? im.adj : im.wr);
  const T adj0 = ok0 ? a[(size_t)(i0 + h) * cols + (j + h)] : (T)0;
  const T adj1 = ok1 ? a[(size_t)(i1 + h) * cols + (j + h)] : (T)0;
  for (int e = w.e0; e < w.e1; ++e) {
    const int s = tile_src[e];
    const SourceDev& sd = srcs[s];
    const bool cin = j >= sd.box[2] && j < sd.box[3];
    const bool in0 = ok0 && cin && i0 >= sd.box[0] && i0 < sd.box[1];
    const bool in1 = ok1 && cin && i1 >= sd.box[0] && i1 < sd.box[1];
    T v[MAX_SLOTS];
#pragma unroll
    for (int k = 0; k < MAX_SLOTS; ++k) v[k] = (T)0;
    if (in0 || in1) {
      const SrcPar<T> P = par[s];
      T D0[MAX_SLOTS], D1[MAX_SLOTS];
      if (sd.type == AP_LIVE_PSF_SRC) {
        // a live PSF's derivative images were made by the column kernel
        const T* lc = (const T*)im.live_cols;
        const size_t plane = (size_t)im.H * im.W;
#pragma unroll
        for (int k = 0; k < MAX_SLOTS; ++k) {
          D0[k] = (k < 2 && in0) ? lc[k * plane + (size_t)i0 * im.W + j] : (T)0;
          D1[k] = (k < 2 && in1) ? lc[k * plane + (size_t)i1 * im.W + j] : (T)0;
        }
      } else {
        pixel_derivs<T, Q>(sd.type, P, i0, j, im, D0);
        pixel_derivs<T, Q>(sd.type, P, i1, j, im, D1);
      }
      const T w0 = in0 ? adj0 : (T)0, w1 = in1 ? adj1 : (T)0;
#pragma unroll
      for (int k = 0; k < MAX_SLOTS; ++k) v[k] = D0[k] * w0 + D1[k] * w1;
      if (dbuf != nullptr && sd.d_off >= 0) {
        if (in0) store_derivs(dbuf, sd, i0, j, D0);
        if (in1) store_derivs(dbuf, sd, i1, j, D1);
      }
    }
    // block reduction over the tile's 256 pixels in T (warp shuffles, then
    // the warp sums in a fixed order); the per-tile partial joins the
    // per-parameter sums in float64
#pragma unroll
    for (int k = 0; k < MAX_SLOTS; ++k) {
      T x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < MAX_SLOTS) {
      T acc = (T)0;
#pragma unroll
      for (int wv = 0; wv < NW; ++wv) acc += red[wv][threadIdx.x];
      partial[(int64_t)e * MAX_SLOTS + threadIdx.x] = (double)acc;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_render_adjoint(int Q, const TileWork* work, int n_work, const int* tile_src, const SourceDev* srcs,
                           const SrcPar<T>* par, const ImageDev* imgs, double* partial, T* dbuf, cudaStream_t st) {
  if (n_work <= 0) return;
  switch (Q) {
    case 1: render_adjoint_kernel<T, 1><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, partial, dbuf); break;
    case 3: render_adjoint_kernel<T, 3><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, partial, dbuf); break;
    case 5: render_adjoint_kernel<T, 5><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, partial, dbuf); break;
    default: render_adjoint_kernel<T, 7><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, partial, dbuf); break;
  }
}

// ---------------------------------------------------------------------------
// Adaptive pixel integration (Sec. "Pixel Integration")
// ---------------------------------------------------------------------------

// surface brightness of one source at a node (du, dv pixels from its centre),
// with the profile's normalisation (the per-pixel code of pixel_value)
template <typename T>
__device__ __forceinline__ T node_brightness(int type, const SrcPar<T>& P, T du, T dv) {
  const T X = P.m00 * du + P.m01 * dv;
  const T Yq = (P.m10 * du + P.m11 * dv) * P.invq;
  const T r2 = X * X + Yq * Yq;
  if (type == AP_SERSIC || type == AP_EXPONENTIAL) {
    const T t = p_exp2(P.k0 * p_log2((r2 + (T)1e-8 * P.area) * P.k1));
    return P.k3 * p_exp2(P.k2 * ((T)1 - t));
  }
  if (type == AP_GAUSSIAN) return P.k1 * p_exp2(P.k0 * r2);
  return P.k1 * p_exp2(-P.k2 * p_log2((T)1 + r2 * P.k0));
}

// order-Q Gauss-Legendre integral over the square of side s (pixels) whose
// lower-left corner is (du0, dv0) pixels from the source centre
template <typename T, int Q>
__device__ __forceinline__ T rect_sum(int type, const SrcPar<T>& P, T du0, T dv0, T s) {
  T acc = (T)0;
#pragma unroll
  for (int b = 0; b < Q; ++b) {
    const T dv = dv0 + s * ((T)0.5 + gl_hu<T>(Q, b));
    T accb = (T)0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const T du = du0 + s * ((T)0.5 + gl_hu<T>(Q, a));
      accb += gl_hw<T>(Q, a) * node_brightness<T>(type, P, du, dv);
    }
    acc += gl_hw<T>(Q, b) * accb;
  }
  return P.area * s * s * acc;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// midpoint pass: one thread per sample, per-block sums of the values (fixed
// order, in T: the budget needs no more) for the sources' budgets
template <typename T>
__global__ void __launch_bounds__(ADAPT_THREADS) adapt_mid_kernel(const AdaptBlock* __restrict__ blocks,
                                                                  const SourceDev* __restrict__ srcs,
                                                                  const SrcPar<T>* __restrict__ par,
                                                                  const int64_t* __restrict__ aoff,
                                                                  T* __restrict__ v0buf, double* __restrict__ part) {
  __shared__ T red[ADAPT_THREADS / 32];
  const AdaptBlock B = blocks[blockIdx.x];
  const SourceDev& sd = srcs[B.src];
  const int bw = sd.box[3] - sd.box[2];
  const int n = (sd.box[1] - sd.box[0]) * bw;
  const int l = B.l0 + (int)threadIdx.x;
  T v = (T)0;
  if (l < n) {
    const SrcPar<T> P = par[B.src];
    const int i = sd.box[0] + l / bw, j = sd.box[2] + l % bw;
    v = rect_sum<T, 1>(sd.type, P, (T)(j - P.jc) - P.fx, (T)(i - P.ic) - P.fy, (T)1);
    v0buf[aoff[B.src] + l] = v;
  }
  v = warp_sum_t(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = (T)0;
    for (int k = 0; k < ADAPT_THREADS / 32; ++k) t += red[k];
    part[blockIdx.x] = (double)t;
  }
}

// budget e = tol |F| / N per sampled source: one warp each, fixed order
template <typename T>
__global__ void adapt_budget_kernel(const int* __restrict__ asrc, int n_asrc, const int* __restrict__ blk_ptr,
                                    const double* __restrict__ part, const SourceDev* __restrict__ srcs, double tol,
                                    T* __restrict__ ebud) {
  const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (k >= n_asrc) return;   // whole warps
  double F = 0.0;
  for (int b = blk_ptr[k] + lane; b < blk_ptr[k + 1]; b += 32) F += part[b];
  F = warp_sum_t(F);
  if (lane == 0) {
    const SourceDev& sd = srcs[asrc[k]];
    const double N = (double)(sd.box[1] - sd.box[0]) * (double)(sd.box[3] - sd.box[2]);
    ebud[asrc[k]] = (T)(tol * fabs(F) / N);
  }
}

// selection and order 3: one thread per sample.  The discrete Laplacian of
// the midpoint values (second differences of the three nearest pixels of each
// axis inside the box) / 24 estimates the midpoint rule's error; pixels above
// the budget take order 3, and those where order 3 and order 2 differ by more
// than the budget are listed for the deep pass.
template <typename T>
__global__ void __launch_bounds__(ADAPT_THREADS) adapt_select_kernel(
    const AdaptBlock* __restrict__ blocks, const SourceDev* __restrict__ srcs, const SrcPar<T>* __restrict__ par,
    const int64_t* __restrict__ aoff, const T* __restrict__ v0buf, const T* __restrict__ ebud,
    T* __restrict__ vbuf, uint8_t* __restrict__ level, int2* __restrict__ list, int* __restrict__ n_list,
    unsigned long long* __restrict__ counts) {
  __shared__ int cnt[2];
  if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
  __syncthreads();
  const AdaptBlock B = blocks[blockIdx.x];
  const SourceDev& sd = srcs[B.src];
  const int bw = sd.box[3] - sd.box[2], nr = sd.box[1] - sd.box[0];
  const int l = B.l0 + (int)threadIdx.x;
  int lev = -1;
  if (l < nr * bw) {
    const int64_t o = aoff[B.src];
    const T* V = v0buf + o;
    const int a = l / bw, b = l % bw;
    const T v0 = V[l];
    T L = (T)0;
    if (nr >= 3) {
      const int m = min(max(a, 1), nr - 2);
      L += V[(m - 1) * bw + b] - (T)2 * V[m * bw + b] + V[(m + 1) * bw + b];
    }
    if (bw >= 3) {
      const int m = min(max(b, 1), bw - 2);
      L += V[a * bw + m - 1] - (T)2 * V[a * bw + m] + V[a * bw + m + 1];
    }
    const T e = ebud[B.src];
    T out = v0;
    lev = 0;
    if (fabs(L) / (T)24 > e) {
      const SrcPar<T> P = par[B.src];
      const int i = sd.box[0] + a, j = sd.box[2] + b;
      const T du0 = (T)(j - P.jc) - P.fx, dv0 = (T)(i - P.ic) - P.fy;
      const T v1 = rect_sum<T, 3>(sd.type, P, du0, dv0, (T)1);
      const T w1 = rect_sum<T, 2>(sd.type, P, du0, dv0, (T)1);
      out = v1;
      lev = 1;
      if (fabs(v1 - w1) > e) {
        lev = 2;   // provisional: the deep pass decides 2 or 3
        list[atomicAdd(n_list, 1)] = make_int2(B.src, l);
      }
    }
    vbuf[o + l] = out;
    level[o + l] = (uint8_t)lev;
  }
  // per-warp counts of the final levels 0 and 1, one shared atomic each
  const unsigned c0 = __ballot_sync(0xffffffffu, lev == 0), c1 = __ballot_sync(0xffffffffu, lev == 1);
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd(&cnt[0], __popc(c0));
    if (c1) atomicAdd(&cnt[1], __popc(c1));
  }
  __syncthreads();
  if (threadIdx.x < 2 && cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)cnt[threadIdx.x]);
}

// deep pass A: one warp per listed pixel (grid-stride over the list).  Lanes
// 0..24 own the 5 x 5 sub-pixels (orders 5 and 4).  If the summed order-5 and
// order-4 values agree within the budget the pixel ends at level 2; otherwise
// it is at level 3: the sub-pixels whose own order-5 and order-4 values differ
// by more than e/25 are marked to be split again (refbits) and the pixel gets
// the order-5 sum of the others, to which pass B adds the split ones.
template <typename T>
__global__ void __launch_bounds__(256) adapt_deep_kernel(const int2* __restrict__ list, const int* __restrict__ n_list,
                                                         const SourceDev* __restrict__ srcs,
                                                         const SrcPar<T>* __restrict__ par,
                                                         const int64_t* __restrict__ aoff,
                                                         const T* __restrict__ ebud, T* __restrict__ vbuf,
                                                         uint8_t* __restrict__ level, uint32_t* __restrict__ refbits,
                                                         unsigned long long* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int warp0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int n = *n_list;
  const T sub = (T)1 / (T)5;
  const int qx = lane % 5, qy = lane / 5;
  for (int k = warp0; k < n; k += nwarps) {
    const int2 ent = list[k];
    const SourceDev& sd = srcs[ent.x];
    const SrcPar<T> P = par[ent.x];
    const int bw = sd.box[3] - sd.box[2];
    const int i = sd.box[0] + ent.y / bw, j = sd.box[2] + ent.y % bw;
    const T du0 = (T)(j - P.jc) - P.fx, dv0 = (T)(i - P.ic) - P.fy;
    const T e = ebud[ent.x];
    const int64_t o = aoff[ent.x] + ent.y;
    const T qu = du0 + sub * (T)qx, qv = dv0 + sub * (T)qy;
    const T g5 = lane < 25 ? rect_sum<T, 5>(sd.type, P, qu, qv, sub) : (T)0;
    const T g4 = lane < 25 ? rect_sum<T, 4>(sd.type, P, qu, qv, sub) : (T)0;
    const T v2 = warp_sum_t(g5);
    const T w2 = warp_sum_t(g4);
    if (fabs(v2 - w2) <= e) {
      if (lane == 0) {
        vbuf[o] = v2;
        level[o] = 2;
        atomicAdd(&counts[2], 1ull);
      }
      continue;
    }
    const unsigned refm = __ballot_sync(0xffffffffu, lane < 25 && fabs(g5 - g4) > e / (T)25);
    const T keep = warp_sum_t((lane < 25 && !((refm >> lane) & 1u)) ? g5 : (T)0);
    if (lane == 0) {
      vbuf[o] = keep;
      refbits[o] = refm;
      level[o] = 3;
      atomicAdd(&counts[3], 1ull);
      atomicAdd(&counts[4], (unsigned long long)__popc(refm));
    }
  }
}

// deep pass B: one CTA per listed pixel at level 3 (grid-stride over the list,
// other pixels skipped): the 25 x 49 order-7 nodes of every sub-pixel marked
// to be split again form one run spread over the CTA's threads (nodes and
// weights from shared memory); the CTA's sum (fixed order) is added to the
// pixel's value.
template <typename T>
__global__ void __launch_bounds__(ADAPT_THREADS) adapt_split_kernel(
    const int2* __restrict__ list, const int* __restrict__ n_list, const SourceDev* __restrict__ srcs,
    const SrcPar<T>* __restrict__ par, const int64_t* __restrict__ aoff, T* __restrict__ vbuf,
    const uint8_t* __restrict__ level, const uint32_t* __restrict__ refbits) {
  __shared__ T s_hu7[8], s_hw7[8];
  __shared__ T red[ADAPT_THREADS / 32];
  if (threadIdx.x < 7) {
    s_hu7[threadIdx.x] = gl_hu<T>(7, threadIdx.x);
    s_hw7[threadIdx.x] = gl_hw<T>(7, threadIdx.x);
  }
  __syncthreads();
  constexpr int NODES7 = 25 * 49;   // order-7 nodes of one sub-pixel split 5 x 5
  const T sub = (T)1 / (T)5, sub2 = (T)1 / (T)25;
  const int n = *n_list;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    const int2 ent = list[k];
    const int64_t o = aoff[ent.x] + ent.y;
    if (level[o] != 3) continue;   // uniform over the CTA
    const SourceDev& sd = srcs[ent.x];
    const SrcPar<T> P = par[ent.x];
    const int bw = sd.box[3] - sd.box[2];
    const int i = sd.box[0] + ent.y / bw, j = sd.box[2] + ent.y % bw;
    const T du0 = (T)(j - P.jc) - P.fx, dv0 = (T)(i - P.ic) - P.fy;
    const unsigned refm = refbits[o];
    const int n_ref = __popc(refm);
    // node t of the run: split sub-pixel t / NODES7 (in bit order), then piece
    // ss and node (a, b) inside it; each thread steps its sub-pixel along
    unsigned m = refm;
    int qi = 0, q = __ffs(m) - 1;
    T acc = (T)0;
    for (int t = (int)threadIdx.x; t < n_ref * NODES7; t += ADAPT_THREADS) {
      while (t >= (qi + 1) * NODES7) {
        ++qi;
        m &= m - 1;
        q = __ffs(m) - 1;
      }
      const int rem = t - qi * NODES7;
      const int ss = rem / 49, nd = rem - ss * 49, a = nd % 7, b = nd / 7;
      const T du = du0 + sub * (T)(q % 5) + sub2 * ((T)(ss % 5) + (T)0.5 + s_hu7[a]);
      const T dv = dv0 + sub * (T)(q / 5) + sub2 * ((T)(ss / 5) + (T)0.5 + s_hu7[b]);
      acc += s_hw7[a] * s_hw7[b] * node_brightness<T>(sd.type, P, du, dv);
    }
    acc = warp_sum_t(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      T tot = (T)0;
      for (int w = 0; w < ADAPT_THREADS / 32; ++w) tot += red[w];
      vbuf[o] += P.area * sub2 * sub2 * tot;
    }
    __syncthreads();   // red[] is reused by the next pixel
  }
}

template <typename T>
void launch_adaptive(const AdaptPlan& ap, const SourceDev* srcs, const SrcPar<T>* par, double tol, T* v0buf, T* vbuf,
                     cudaStream_t st) {
  if (ap.n_blocks <= 0) return;
  adapt_mid_kernel<T><<<ap.n_blocks, ADAPT_THREADS, 0, st>>>(ap.blocks, srcs, par, ap.aoff, v0buf, ap.part);
  T* ebud = (T*)ap.ebud;
  adapt_budget_kernel<T><<<(ap.n_asrc + 7) / 8, 256, 0, st>>>(ap.asrc, ap.n_asrc, ap.blk_ptr, ap.part, srcs, tol,
                                                             ebud);
  adapt_select_kernel<T><<<ap.n_blocks, ADAPT_THREADS, 0, st>>>(ap.blocks, srcs, par, ap.aoff, v0buf, ebud, vbuf,
                                                                ap.level, ap.list, ap.n_list, ap.counts);
  adapt_deep_kernel<T><<<ap.deep_blocks, 256, 0, st>>>(ap.list, ap.n_list, srcs, par, ap.aoff, ebud, vbuf, ap.level,
                                                        ap.refbits, ap.counts);
  adapt_split_kernel<T><<<ap.deep_blocks, ADAPT_THREADS, 0, st>>>(ap.list, ap.n_list, srcs, par, ap.aoff, vbuf,
                                                                  ap.level, ap.refbits);
}

// the render kernel's tile gather, reading each sampled source's adaptive
// value instead of evaluating it
template <typename T>
__global__ void __launch_bounds__(RENDER_THREADS) render_samples_kernel(const TileWork* __restrict__ work,
                                                                        const int* __restrict__ tile_src,
                                                                        const SourceDev* __restrict__ srcs,
                                                                        const SrcPar<T>* __restrict__ par,
                                                                        const ImageDev* __restrict__ imgs,
                                                                        const int64_t* __restrict__ aoff,
                                                                        const T* __restrict__ vbuf) {
  const TileWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  const int j = w.c0 + (int)(threadIdx.x % TILE);
  const int i0 = w.r0 + (int)(threadIdx.x / TILE), i1 = i0 + TILE / 2;
  const int h = w.plane == 0 ? im.h : 0;
  const int rows = w.plane == 0 ? im.Hp : im.H;
  const int cols = w.plane == 0 ? im.Wp : im.W;
  T acc0 = (T)0, acc1 = (T)0;
  for (int e = w.e0; e < w.e1; ++e) {
    const int s = tile_src[e];
    const SourceDev& sd = srcs[s];
    const bool cin = j >= sd.box[2] && j < sd.box[3];
    const bool in0 = cin && i0 >= sd.box[0] && i0 < sd.box[1];
    const bool in1 = cin && i1 >= sd.box[0] && i1 < sd.box[1];
    if (!(in0 || in1)) continue;
    const int64_t o = aoff[s];
    if (o < 0) {   // a sky: linear in position, its midpoint is exact
      const SrcPar<T> P = par[s];
      if (in0) acc0 += pixel_value<T, 1>(sd.type, P, i0, j, im);
      if (in1) acc1 += pixel_value<T, 1>(sd.type, P, i1, j, im);
    } else {
      const int bw = sd.box[3] - sd.box[2];
      if (in0) acc0 += vbuf[o + (int64_t)(i0 - sd.box[0]) * bw + (j - sd.box[2])];
      if (in1) acc1 += vbuf[o + (int64_t)(i1 - sd.box[0]) * bw + (j - sd.box[2])];
    }
  }
  T* out = (T*)(w.plane == 0 ? im.gal : im.unc);
  if (j + h < cols) {
    if (i0 + h < rows) out[(size_t)(i0 + h) * cols + (j + h)] = acc0;
    if (i1 + h < rows) out[(size_t)(i1 + h) * cols + (j + h)] = acc1;
  }
}

template <typename T>
void launch_render_samples(const TileWork* work, int n_work, const int* tile_src, const SourceDev* srcs,
                           const SrcPar<T>* par, const ImageDev* imgs, const int64_t* aoff, const T* vbuf,
                           cudaStream_t st) {
  if (n_work <= 0) return;
  render_samples_kernel<T><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, aoff, vbuf);
}

// ---------------------------------------------------------------------------
// Pixel-centred sampling with an interpolated re-shift (Sec. "PSF
// convolution"): each convolved profile source is sampled with its centre on
// the centre of the pixel that holds it, moved back by its sub-pixel offset
// (du, dv) in [-1/2, 1/2) with Lanczos (a = 3, weights normalised to unit
// sum) or bilinear interpolation on its sampling box (zero beyond it), and
// then joins the galaxy layer; the interpolation is a discrete convolution,
// so this equals convolving first and shifting after.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T p_sinpi(T x);
template <> __device__ __forceinline__ float p_sinpi<float>(float x) { return sinpif(x); }
template <> __device__ __forceinline__ double p_sinpi<double>(double x) { return sinpi(x); }

// weights of taps t = -3..3 of a shift by d: shifted(p) = sum_t w[t + 3] f(p - t)
template <typename T>
__device__ __forceinline__ void shift_weights(T d, int method, T (&w)[7]) {
  T sum = (T)0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const T x = (T)(k - 3) - d;
    const T ax = fabs(x);
    T v;
    if (method == AP_SHIFT_BILINEAR) {
      v = ax < (T)1 ? (T)1 - ax : (T)0;
    } else {
      const T pi = (T)3.14159265358979323846;
      const T s1 = ax == (T)0 ? (T)1 : p_sinpi<T>(x) / (pi * x);
      const T s3 = ax == (T)0 ? (T)1 : p_sinpi<T>(x / (T)3) / (pi * x / (T)3);
      v = ax < (T)3 ? s1 * s3 : (T)0;
    }
    w[k] = v;
    sum += v;
  }
  if (method != AP_SHIFT_BILINEAR) {
    const T inv = (T)1 / sum;
#pragma unroll
    for (int k = 0; k < 7; ++k) w[k] *= inv;
  }
}

// records with the shifted sources' centres on their pixel centres, and
// their offsets back to the true centres
template <typename T>
__global__ void snap_kernel(const SrcPar<T>* __restrict__ par, const int64_t* __restrict__ soff, int n_src,
                            SrcPar<T>* __restrict__ snap, T* __restrict__ shift) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_src) return;
  SrcPar<T> r = par[s];
  if (soff[s] >= 0) {
    shift[2 * s] = r.fx - (T)0.5;
    shift[2 * s + 1] = r.fy - (T)0.5;
    r.fx = (T)0.5;
    r.fy = (T)0.5;
  }
  snap[s] = r;
}

// one thread per pixel of a shifted source's sampling box
template <typename T, int Q>
__global__ void __launch_bounds__(ADAPT_THREADS) sample_snapped_kernel(const AdaptBlock* __restrict__ blocks,
                                                                       const SourceDev* __restrict__ srcs,
                                                                       const SrcPar<T>* __restrict__ snap,
                                                                       const ImageDev* __restrict__ imgs,
                                                                       const int64_t* __restrict__ soff,
                                                                       T* __restrict__ R) {
  const AdaptBlock bk = blocks[blockIdx.x];
  const SourceDev& sd = srcs[bk.src];
  const int bw = sd.box[3] - sd.box[2];
  const int n = (sd.box[1] - sd.box[0]) * bw;
  const int l = bk.l0 + (int)threadIdx.x;
  if (l >= n) return;
  const int i = sd.box[0] + l / bw, j = sd.box[2] + l % bw;
  R[soff[bk.src] + l] = pixel_value<T, Q>(sd.type, snap[bk.src], i, j, imgs[sd.image]);
}

template <typename T>
__global__ void __launch_bounds__(ADAPT_THREADS) shift_box_kernel(const AdaptBlock* __restrict__ blocks,
                                                                  const SourceDev* __restrict__ srcs,
                                                                  const int64_t* __restrict__ soff,
                                                                  const T* __restrict__ shift, int method,
                                                                  const T* __restrict__ R, T* __restrict__ S) {
  const AdaptBlock bk = blocks[blockIdx.x];
  const SourceDev& sd = srcs[bk.src];
  const int bw = sd.box[3] - sd.box[2], bh = sd.box[1] - sd.box[0];
  const int l = bk.l0 + (int)threadIdx.x;
  if (l >= bh * bw) return;
  const int ri = l / bw, rj = l % bw;
  T wu[7], wv[7];
  shift_weights<T>(shift[2 * bk.src], method, wu);
  shift_weights<T>(shift[2 * bk.src + 1], method, wv);
  const T* Rs = R + soff[bk.src];
  T acc = (T)0;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    const int ii = ri - (a - 3);
    if (ii < 0 || ii >= bh || wv[a] == (T)0) continue;
    T row = (T)0;
#pragma unroll
    for (int b = 0; b < 7; ++b) {
      const int jj = rj - (b - 3);
      if (jj >= 0 && jj < bw) row += wu[b] * Rs[(int64_t)ii * bw + jj];
    }
    acc += wv[a] * row;
  }
  S[soff[bk.src] + l] = acc;
}

// the layers: shifted sources from their stored boxes, the others in place
template <typename T, int Q>
__global__ void __launch_bounds__(RENDER_THREADS) render_shifted_kernel(const TileWork* __restrict__ work,
                                                                        const int* __restrict__ tile_src,
                                                                        const SourceDev* __restrict__ srcs,
                                                                        const SrcPar<T>* __restrict__ par,
                                                                        const ImageDev* __restrict__ imgs,
                                                                        const int64_t* __restrict__ soff,
                                                                        const T* __restrict__ S) {
  const TileWork w = work[blockIdx.x];
  const ImageDev& im = imgs[w.image];
  const int j = w.c0 + (int)(threadIdx.x % TILE);
  const int i0 = w.r0 + (int)(threadIdx.x / TILE), i1 = i0 + TILE / 2;
  const int h = w.plane == 0 ? im.h : 0;
  const int rows = w.plane == 0 ? im.Hp : im.H;
  const int cols = w.plane == 0 ? im.Wp : im.W;
  T acc0 = (T)0, acc1 = (T)0;
  for (int e = w.e0; e < w.e1; ++e) {
    const int s = tile_src[e];
    const SourceDev& sd = srcs[s];
    const bool cin = j >= sd.box[2] && j < sd.box[3];
    const bool in0 = cin && i0 >= sd.box[0] && i0 < sd.box[1];
    const bool in1 = cin && i1 >= sd.box[0] && i1 < sd.box[1];
    if (!(in0 || in1)) continue;
    const int64_t o = soff[s];
    if (o < 0) {
      const SrcPar<T> P = par[s];
      if (in0) acc0 += pixel_value<T, Q>(sd.type, P, i0, j, im);
      if (in1) acc1 += pixel_value<T, Q>(sd.type, P, i1, j, im);
    } else {
      const int bw = sd.box[3] - sd.box[2];
      if (in0) acc0 += S[o + (int64_t)(i0 - sd.box[0]) * bw + (j - sd.box[2])];
      if (in1) acc1 += S[o + (int64_t)(i1 - sd.box[0]) * bw + (j - sd.box[2])];
    }
  }
  T* out = (T*)(w.plane == 0 ? im.gal : im.unc);
  if (j + h < cols) {
    if (i0 + h < rows) out[(size_t)(i0 + h) * cols + (j + h)] = acc0;
    if (i1 + h < rows) out[(size_t)(i1 + h) * cols + (j + h)] = acc1;
  }
}

template <typename T>
void launch_shifted_render(int Q, int method, const ShiftPlan& sp, const TileWork* work, int n_work,
                           const int* tile_src, const SourceDev* srcs, const SrcPar<T>* par, const ImageDev* imgs,
                           int n_src, cudaStream_t st) {
  SrcPar<T>* snap = (SrcPar<T>*)sp.snap;
  T* shift = (T*)sp.shift;
  T* R = (T*)sp.R;
  T* S = (T*)sp.S;
  if (n_src > 0) snap_kernel<T><<<(n_src + 127) / 128, 128, 0, st>>>(par, sp.soff, n_src, snap, shift);
  if (sp.n_blocks > 0) {
    switch (Q) {
      case 1: sample_snapped_kernel<T, 1><<<sp.n_blocks, ADAPT_THREADS, 0, st>>>(sp.blocks, srcs, snap, imgs, sp.soff, R); break;
      case 3: sample_snapped_kernel<T, 3><<<sp.n_blocks, ADAPT_THREADS, 0, st>>>(sp.blocks, srcs, snap, imgs, sp.soff, R); break;
      case 5: sample_snapped_kernel<T, 5><<<sp.n_blocks, ADAPT_THREADS, 0, st>>>(sp.blocks, srcs, snap, imgs, sp.soff, R); break;
      default: sample_snapped_kernel<T, 7><<<sp.n_blocks, ADAPT_THREADS, 0, st>>>(sp.blocks, srcs, snap, imgs, sp.soff, R); break;
    }
    shift_box_kernel<T><<<sp.n_blocks, ADAPT_THREADS, 0, st>>>(sp.blocks, srcs, sp.soff, shift, method, R, S);
  }
  if (n_work <= 0) return;
  switch (Q) {
    case 1: render_shifted_kernel<T, 1><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, sp.soff, S); break;
    case 3: render_shifted_kernel<T, 3><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, sp.soff, S); break;
    case 5: render_shifted_kernel<T, 5><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, sp.soff, S); break;
    default: render_shifted_kernel<T, 7><<<n_work, RENDER_THREADS, 0, st>>>(work, tile_src, srcs, par, imgs, sp.soff, S); break;
  }
}

// ---------------------------------------------------------------------------
// Live PSF (Sec. "PSF convolution": the PSF as a model fitted with the
// sources).  One CTA per live image renders the circular Moffat
// I = (n - 1) / (pi Rd^2) (1 + r^2 / Rd^2)^-n of unit flux over the K x K map
// pixels (the context's order-Q rule, offsets A (du, dv) from the centre of
// the middle pixel, times |det A|), with dI/dn = I (1/(n-1) - ln v) and
// dI/dRd = I (-2/Rd + 2 n r^2 / (v Rd^3)), v = 1 + r^2/Rd^2, all in float64;
// then P = Praw / S, dP = (dPraw - P dS) / S, S = sum Praw.
// ---------------------------------------------------------------------------
constexpr int LIVE_THREADS = 256;

template <typename T, int Q>
__global__ void __launch_bounds__(LIVE_THREADS) live_psf_kernel(const int* __restrict__ live_imgs,
                                                                const SourceDev* __restrict__ srcs,
                                                                const ImageDev* __restrict__ imgs,
                                                                const double* __restrict__ theta,
                                                                int* __restrict__ status) {
  __shared__ double red[3][LIVE_THREADS / 32];
  const ImageDev& im = imgs[live_imgs[blockIdx.x]];
  const SourceDev& sd = srcs[im.live_src];
  const double n = sd.pidx[0] >= 0 ? theta[sd.pidx[0]] : sd.pfix[0];
  const double Rd = sd.pidx[1] >= 0 ? theta[sd.pidx[1]] : sd.pfix[1];
  const int K = im.K, K4 = im.K4, KK = K * K;
  const double c = 0.5 * (K - 1);
  const bool good = n > 1.0 && Rd > 0.0 && isfinite(n) && isfinite(Rd);
  const double iR2 = 1.0 / (Rd * Rd), nrm = (n - 1.0) / (M_PI * Rd * Rd);
  T* pn = (T*)im.psf_norm;
  T* pf = (T*)im.psf_flip;
  // dpsf_flip holds 4 planes of K x K4: the flipped normalised derivatives by
  // n and Rd (planes 0, 1, read by the column kernel) and the raw derivatives
  // (planes 2, 3, scratch of this kernel)
  const int PL = K * K4;
  T* dpf = (T*)im.dpsf_flip;
  // first pass: raw values into the plain map and the raw derivative planes,
  // and the three sums
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int t = threadIdx.x; t < KK; t += LIVE_THREADS) {
    const int a = t / K, b = t % K;
    double P = 0.0, Pn = 0.0, Pr = 0.0;
    if (good) {
      for (int qb = 0; qb < Q; ++qb) {
        const double dv = (a - c) + gl_hu<double>(Q, qb);
        for (int qa = 0; qa < Q; ++qa) {
          const double du = (b - c) + gl_hu<double>(Q, qa);
          const double x = im.A[0] * du + im.A[1] * dv, y = im.A[2] * du + im.A[3] * dv;
          const double r2 = x * x + y * y;
          const double v = 1.0 + r2 * iR2;
          const double I = nrm * exp(-n * log(v));
          const double w = gl_hw<double>(Q, qa) * gl_hw<double>(Q, qb);
          P += w * I;
          Pn += w * I * (1.0 / (n - 1.0) - log(v));
          Pr += w * I * (-2.0 / Rd + 2.0 * n * r2 * iR2 / (v * Rd));
        }
      }
    }
    P *= im.area;
    Pn *= im.area;
    Pr *= im.area;
    pn[a * K4 + b] = (T)P;
    dpf[2 * PL + a * K4 + b] = (T)Pn;
    dpf[3 * PL + a * K4 + b] = (T)Pr;
    s0 += P;
    s1 += Pn;
    s2 += Pr;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    red[0][warp] = s0;
    red[1][warp] = s1;
    red[2][warp] = s2;
  }
  __syncthreads();
  double S = 0.0, Sn = 0.0, Sr = 0.0;
  for (int k = 0; k < LIVE_THREADS / 32; ++k) {
    S += red[0][k];
    Sn += red[1][k];
    Sr += red[2][k];
  }
  if (!(S > 0.0) || !isfinite(S)) {
    if (threadIdx.x == 0) atomicCAS(status, 0, AP_ERR_NONFINITE);
    S = 1.0;
  }
  // second pass (each thread its own entries of the first pass): normalise,
  // and write the flipped copies
  for (int t = threadIdx.x; t < KK; t += LIVE_THREADS) {
    const int a = t / K, b = t % K;
    const int fo = (K - 1 - a) * K4 + (K - 1 - b);
    const double P = (double)pn[a * K4 + b] / S;
    pn[a * K4 + b] = (T)P;
    pf[fo] = (T)P;
    dpf[fo] = (T)(((double)dpf[2 * PL + a * K4 + b] - P * Sn) / S);
    dpf[PL + fo] = (T)(((double)dpf[3 * PL + a * K4 + b] - P * Sr) / S);
  }
}

// the live columns dm/dphi_k = (dP/dphi_k) * G on the image: with the
// flipped kernel F, out(i, j) = sum_{ty, tx} F[ty][tx] Gpad(i + ty, j + tx)
// (Gpad the galaxy layer, image pixel (i, j) at (i + h, j + h)).  One CTA per
// 16 x 16 output tile of one live image, the layer's (16 + K - 1)^2 window
// and both kernels staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(TILE_THREADS) live_cols_kernel(const int* __restrict__ live_imgs,
                                                                 const ImageDev* __restrict__ imgs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ImageDev& im = imgs[live_imgs[blockIdx.y]];
  const int ntc = (im.W + TILE - 1) / TILE, ntr = (im.H + TILE - 1) / TILE;
  if ((int)blockIdx.x >= ntc * ntr) return;
  const int r0 = (blockIdx.x / ntc) * TILE, c0 = (blockIdx.x % ntc) * TILE;
  const int K = im.K, K4 = im.K4, L = TILE + K - 1;
  T* g = reinterpret_cast<T*>(smem_raw);   // L x L window of the layer
  T* f = g + L * L;                         // 2 K x K kernels
  const T* G = (const T*)im.gal;
  const T* dpf = (const T*)im.dpsf_flip;
  for (int t = threadIdx.x; t < L * L; t += TILE_THREADS) {
    const int a = t / L, b = t % L;
    const int gi = r0 + a, gj = c0 + b;   // layer coordinates (image pixel + h)
    g[t] = (im.has_gal && gi < im.Hp && gj < im.Wp) ? G[(size_t)gi * im.Wp + gj] : (T)0;
  }
  for (int t = threadIdx.x; t < 2 * K * K; t += TILE_THREADS) {
    const int k = t / (K * K), u = t % (K * K);
    f[t] = dpf[k * K * K4 + (u / K) * K4 + (u % K)];
  }
  __syncthreads();
  const int li = threadIdx.x / TILE, lj = threadIdx.x % TILE;
  const int i = r0 + li, j = c0 + lj;
  T a0 = (T)0, a1 = (T)0;
  for (int ty = 0; ty < K; ++ty) {
    const T* grow = g + (li + ty) * L + lj;
    const T* f0 = f + ty * K;
    const T* f1 = f + K * K + ty * K;
    for (int tx = 0; tx < K; ++tx) {
      const T v = grow[tx];
      a0 += f0[tx] * v;
      a1 += f1[tx] * v;
    }
  }
  if (i < im.H && j < im.W) {
    T* out = (T*)im.live_cols;
    const size_t plane = (size_t)im.H * im.W;
    out[(size_t)i * im.W + j] = a0;
    out[plane + (size_t)i * im.W + j] = a1;
  }
}

template <typename T>
void launch_live_psf(int Q, const int* live_imgs, int n_live, const SourceDev* srcs, const ImageDev* imgs,
                     const double* theta, int* status, cudaStream_t st) {
  if (n_live <= 0) return;
  switch (Q) {
    case 1: live_psf_kernel<T, 1><<<n_live, LIVE_THREADS, 0, st>>>(live_imgs, srcs, imgs, theta, status); break;
    case 3: live_psf_kernel<T, 3><<<n_live, LIVE_THREADS, 0, st>>>(live_imgs, srcs, imgs, theta, status); break;
    case 5: live_psf_kernel<T, 5><<<n_live, LIVE_THREADS, 0, st>>>(live_imgs, srcs, imgs, theta, status); break;
    default: live_psf_kernel<T, 7><<<n_live, LIVE_THREADS, 0, st>>>(live_imgs, srcs, imgs, theta, status); break;
  }
}

template <typename T>
size_t live_cols_smem(int K) {
  const int L = TILE + K - 1;
  return (size_t)(L * L + 2 * K * K) * sizeof(T);
}

template <typename T>
void launch_live_cols(const int* live_imgs, int n_live, const ImageDev* imgs, int max_tiles, int Kmax,
                      cudaStream_t st) {
  if (n_live <= 0 || max_tiles <= 0) return;
  live_cols_kernel<T><<<dim3(max_tiles, n_live), TILE_THREADS, live_cols_smem<T>(Kmax), st>>>(live_imgs, imgs);
}

int configure_live(int Kmax, int is_double) {
  const size_t need = is_double ? live_cols_smem<double>(Kmax) : live_cols_smem<float>(Kmax);
  const int a = is_double ? allow_max_dynamic_smem(live_cols_kernel<double>) : allow_max_dynamic_smem(live_cols_kernel<float>);
  return a >= (int)need ? 1 : 0;
}

template void launch_live_psf<float>(int, const int*, int, const SourceDev*, const ImageDev*, const double*, int*,
                                     cudaStream_t);
template void launch_live_psf<double>(int, const int*, int, const SourceDev*, const ImageDev*, const double*, int*,
                                      cudaStream_t);
template void launch_live_cols<float>(const int*, int, const ImageDev*, int, int, cudaStream_t);
template void launch_live_cols<double>(const int*, int, const ImageDev*, int, int, cudaStream_t);

template void launch_shifted_render<float>(int, int, const ShiftPlan&, const TileWork*, int, const int*,
                                           const SourceDev*, const SrcPar<float>*, const ImageDev*, int, cudaStream_t);
template void launch_shifted_render<double>(int, int, const ShiftPlan&, const TileWork*, int, const int*,
                                            const SourceDev*, const SrcPar<double>*, const ImageDev*, int,
                                            cudaStream_t);

template void launch_adaptive<float>(const AdaptPlan&, const SourceDev*, const SrcPar<float>*, double, float*, float*,
                                     cudaStream_t);
template void launch_adaptive<double>(const AdaptPlan&, const SourceDev*, const SrcPar<double>*, double, double*,
                                      double*, cudaStream_t);
template void launch_render_samples<float>(const TileWork*, int, const int*, const SourceDev*, const SrcPar<float>*,
                                           const ImageDev*, const int64_t*, const float*, cudaStream_t);
template void launch_render_samples<double>(const TileWork*, int, const int*, const SourceDev*, const SrcPar<double>*,
                                            const ImageDev*, const int64_t*, const double*, cudaStream_t);
template void launch_prepare<float>(const SourceDev*, const ImageDev*, int, const double*, SrcPar<float>*, double*,
                                    const int*, int*, cudaStream_t);
template void launch_prepare<double>(const SourceDev*, const ImageDev*, int, const double*, SrcPar<double>*, double*,
                                     const int*, int*, cudaStream_t);
template void launch_render<float>(int, const TileWork*, int, const int*, const SourceDev*, const SrcPar<float>*, const ImageDev*, const int*, cudaStream_t);
template void launch_render<double>(int, const TileWork*, int, const int*, const SourceDev*, const SrcPar<double>*, const ImageDev*, const int*, cudaStream_t);
template void launch_render_adjoint<float>(int, const TileWork*, int, const int*, const SourceDev*, const SrcPar<float>*, const ImageDev*, double*, float*, cudaStream_t);
template void launch_render_adjoint<double>(int, const TileWork*, int, const int*, const SourceDev*, const SrcPar<double>*, const ImageDev*, double*, double*, cudaStream_t);

}  // namespace ap
