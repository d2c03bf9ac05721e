// Internal declarations shared by the translation units of libastrophot_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "astrophot_gb300.h"

namespace ap {

// Render / adjoint / Jacobian tiles are TILE x TILE pixels, one thread per
// pixel.  16 x 16 = 256 threads keeps every warp on two rows of one tile.
constexpr int TILE = 16;
constexpr int TILE_THREADS = TILE * TILE;
constexpr int MAX_SLOTS = 8;
constexpr int GRAM_MAX_COLS = 160;   // Jacobian columns one image tile may hold

// ---------------------------------------------------------------------------
// device-side descriptors (uploaded once per problem)
// ---------------------------------------------------------------------------
struct ImageDev {
  int H, W;          // image rows, columns
  int K, h;          // PSF size and half width (K = 0, h = 0 without PSF)
  int Hp, Wp;        // galaxy layer size: H + 2h, W + 2h
  int has_gal;       // image has a PSF and at least one convolved source
  int group;
  double A[4];       // pixel -> world
  double origin[2];
  double Ainv[4];    // world -> pixel
  double area;       // |det A|
  double hx, hy;     // A (W/2, H/2): the image centre relative to the origin
  const float* data;
  const float* var;
  const uint8_t* mask;
  void* gal;         // Hp*Wp: galaxy layer G (T)
  void* unc;         // H*W:   unconvolved layer U (T)
  void* wr;          // H*W:   w r (T)
  void* adj;         // Hp*Wp: P-correlated w r (T)
  void* psf_flip;    // K*K4:  normalised PSF, flipped, rows padded to K4 (T)
  void* psf_norm;    // K*K4:  normalised PSF, rows padded to K4 (T)
  int K4;            // K rounded up to a multiple of 4
};

struct SourceDev {
  int type, image, conv, nslot;
  int box[4];        // r0, r1, c0, c1: sampling box (image pixel indices; a
                     // convolved source's box reaches into the PSF halo)
  int pidx[MAX_SLOTS];
  double pfix[MAX_SLOTS];
  int64_t d_off;     // element offset of this source's derivative images
  int sup[4];        // Jacobian support: r0, r1, c0, c1 in image pixels
  int64_t j_off;     // element offset of this source's convolved columns (-1: none)
};

// Per-evaluation source record, prepared from theta on the device.
template <typename T>
struct SrcPar {
  T m00, m01, m10, m11;  // X = m00 du + m01 dv, Y = m10 du + m11 dv (du, dv pixel offsets)
  T invq;
  T fx, fy;              // centre's fractional position in its reference pixel
  T area;
  T c, s;                // cos PA, sin PA
  T k0, k1, k2, k3, k4, k5, k6;  // profile constants (see ap_render.cu)
  T pv[MAX_SLOTS];       // slot values
  int jc, ic;            // reference pixel (column, row)
  int pad_[2];
};

// Work items.
struct TileWork {        // one TILE x TILE tile of a layer
  int image;
  int plane;             // 0 = galaxy layer (coords offset by h), 1 = unconvolved layer
  int r0, c0;            // tile origin in image pixel coordinates
  int e0, e1;            // range in the tile->source list
};

struct ConvWork {        // one output tile of a correlation
  int image;
  int r0, c0;            // tile origin in output coordinates
};

struct JcolWork {        // one output tile of one source's Jacobian columns
  int src;
  int r0, c0;            // tile origin in image pixels
};

// ---------------------------------------------------------------------------
// launchers (each TU owns its kernels; T = float or double)
// ---------------------------------------------------------------------------
void upload_gl_rule(int Q);  // Gauss-Legendre nodes/weights to constant memory

// Let a kernel use as much dynamic shared memory as the device allows next to
// its static shared memory (the opt-in is a cap; every launch asks for what
// it needs).  Returns that amount, or -1 if the runtime refuses.
template <typename F>
inline int allow_max_dynamic_smem(F* func) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return -1;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, func) != cudaSuccess) return -1;
  const int maxdyn = optin - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn) != cudaSuccess) return -1;
  return maxdyn;
}

template <typename T>
void launch_prepare(const SourceDev* srcs, const ImageDev* imgs, int n_src, const double* theta,
                    SrcPar<T>* par, int* status, cudaStream_t st);

template <typename T>
void launch_render(int Q, const TileWork* work, int n_work, const int* tile_src, const SourceDev* srcs,
                   const SrcPar<T>* par, const ImageDev* imgs, cudaStream_t st);

template <typename T>
void launch_render_adjoint(int Q, const TileWork* work, int n_work, const int* tile_src,
                           const SourceDev* srcs, const SrcPar<T>* par, const ImageDev* imgs,
                           double* partial, T* dbuf, cudaStream_t st);

// a run of correlation work items sharing one PSF chunk count (K4/4);
// nc = 0 selects the generic tile code
struct ConvRange {
  int nc, start, count;
};
int conv_nc_of(int K4, int is_double);

// forward correlation of the galaxy layer with the flipped PSF + model
// assembly + residual + chi^2 partials (and the model into model_out)
template <typename T>
void launch_forward_conv(int tile_variant, const ConvWork* work, const ConvRange* ranges, int n_ranges,
                         const ImageDev* imgs, double* chi2_partial, void* const* model_out, int* status, int kmax,
                         cudaStream_t st);

// adjoint correlation: adj = P (correlate) w r over the galaxy layer
template <typename T>
void launch_adjoint_conv(int tile_variant, const ConvWork* work, const ConvRange* ranges, int n_ranges,
                         const ImageDev* imgs, int kmax, cudaStream_t st);

template <typename T> void configure_conv(int Kmax, int* ok);
template <typename T>
void launch_jcol(int variant, const JcolWork* work, const ConvRange* ranges, int n_ranges, const SourceDev* srcs,
                 const ImageDev* imgs, const T* dbuf, T* jbuf, int kmax, cudaStream_t st);
template <typename T> void configure_gram(int unused);
template <typename T> void gram_blocking(int maxc, int* cb, int* two);
int gram_max_cols(int is_double);
int conv_tile_w(int variant);
int conv_tile_h(int variant);
constexpr int N_CONV_VARIANTS = 7;

void launch_sum_groups(const double* partial, const int* ptr, const int* idx, int n_out, double* out,
                       double scale, cudaStream_t st);
void launch_sum_contrib(const double* partial, const int64_t* ptr, const int64_t* idx, int n_out, double* out,
                        double scale, cudaStream_t st);

template <typename T>
void launch_gram(const TileWork* work, int n_work, const int* jt_src, const SourceDev* srcs,
                 const ImageDev* imgs, const T* dbuf, const T* jbuf, const int64_t* row_ptr,
                 const int32_t* col_idx, double* vals, int cb, int two, int* status, cudaStream_t st);

// solver
struct GroupDev {
  int n;               // parameters in the group
  int p0;              // offset into the group's parameter list
  int dense;           // 1: dense Cholesky, 0: one-CTA PCG, 2: grid-wide PCG
  int nblk;            // preconditioner blocks
  int b0;              // offset into the block list
};

// device plan of the damped solves (see ap_solve.cu)
struct SolvePlan {
  const GroupDev* groups;
  const int* gparams;     // parameters of each group, concatenated
  const int* plocal;      // theta index -> index within its group
  const int* blk_ptr;     // preconditioner block starts per group (with a closing entry)
  const int64_t* row_ptr; // CSR of J^T W J
  const int32_t* col_idx;
  const int32_t* lcol;    // group-local column of each CSR entry
  const int64_t* dpos;    // CSR position of each row's diagonal (-1: none)
  const int64_t* bpos;    // 64 CSR positions per preconditioner block (-1: zero)
  double* work;           // 6 n doubles per group (grid PCG vectors)
  double* blk_work;       // 64 doubles per preconditioner block (factors)
  double* part;           // 3 x grid blocks partial sums (grid PCG)
  int* flag;              // retry flag (grid PCG)
  int* iters;             // CG iterations of each group's last solve
  const int64_t* ch_e0;   // SpMV chunks (<= 32 CSR entries of one row): first entry
  const int64_t* ch_e1;   //   one past the last entry
  const int* ch_row;      // chunks of group row r (concatenated over groups): [ch_row[r], ch_row[r+1])
  double* ch_part;        // chunk partial sums
};

constexpr int PCG_ONE_CTA_MAX = 2048;   // groups above use the grid-wide PCG

void configure_solve();
int grid_pcg_blocks(int device);
void launch_lm_solve(int n_groups, const SolvePlan& sp, const double* vals, const double* jtwr, double* lambda,
                     double* delta, int* status, cudaStream_t st, int any_dense, int any_pcg, int max_dense,
                     int max_pcg);
int launch_pcg_grid(const GroupDev* groups_host, int n_groups, const SolvePlan& sp, const double* vals,
                    const double* jtwr, double* lambda, double* delta, int nblocks, int* status, cudaStream_t st);

void launch_trial(const double* theta, const double* delta, const double* lo, const double* hi,
                  double* trial, int n, cudaStream_t st);
void launch_accept(const int* param_group, int n_params, const double* chi2_now, const double* chi2_trial,
                   double* theta, const double* trial, double* lambda, double* chi2_state, double* log,
                   int n_groups, cudaStream_t st);
void launch_accept_params(const int* param_group, int n_params, const int* accepted, double* theta,
                          const double* trial, cudaStream_t st);
void launch_accept_groups(const double* chi2_now, const double* chi2_trial, double* lambda,
                          double* chi2_state, double* log, int* accepted, int n_groups, cudaStream_t st);
void launch_scale(const double* in, double* out, double s, int n, cudaStream_t st);

}  // namespace ap
