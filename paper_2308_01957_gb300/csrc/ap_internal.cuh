// Internal declarations shared by the translation units of libastrophot_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
  void* wr_trial;    // H*W:   w r at the LM trial point (T)
  void* adj;         // Hp*Wp: P-correlated w r (T)
  void* psf_flip;    // K*K4:  normalised PSF, flipped, rows padded to K4 (T)
  void* psf_norm;    // K*K4:  normalised PSF, rows padded to K4 (T)
  int K4;            // K rounded up to a multiple of 4
  const void* spec64;   // 64 x 64 complex float: spectrum of the padded PSF / 64^2 (null: K > 33)
  const void* spec128;  // 128 x 128 likewise (null: K > 97)
  int live_src;         // live PSF: index of its internal source (-1: a fixed PSF)
  void* live_cols;      // live PSF: 2 H*W (T): dm/dn, dm/dRd = (dP/dphi) * G on the image
  void* dpsf_flip;      // live PSF: 4 K*K4 (T): d(normalised PSF)/d(n, Rd) flipped, then 2 scratch planes
};

// The internal source of a live PSF (one per such image): slots n, Rd; its
// box is the whole image; it draws nothing itself, its derivative images are
// the live_cols of its image.
constexpr int AP_LIVE_PSF_SRC = 7;

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
  T m00, m01, m10, m11;  // X = m00 du + m01 dv, Y = m10 du + m11 dv (du, dv pixel offsets);
                         // sky plane: the pixel -> world matrix A
  T invq;
  T fx, fy;              // centre's fractional position in its reference pixel; sky plane:
                         // the image centre in pixels (W/2, H/2)
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

struct JcolFftWork {     // one FFT block of one free slot of one source's Jacobian columns
  int src;
  int k;                 // slot
  int by0, bx0;          // block origin in the source's box coordinates
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

// The forward launches (prepare, render, forward correlation, chi^2 gather)
// take an optional per-group flag array `skip` (device, n_groups ints,
// nullable): the work items of a group whose flag is set return at once,
// leaving that group's source records and w r as they are (the chi^2 gather
// copies the group's kept value instead).  The LM iteration sets the flags
// once its current point's records and w r are in place.

// bn_memo: 8 doubles per source (two (n, b_n, db/dn) entries and the slot to
// replace next), filled with NaN bytes when the problem is set
template <typename T>
void launch_prepare(const SourceDev* srcs, const ImageDev* imgs, int n_src, const double* theta,
                    SrcPar<T>* par, double* bn_memo, const int* skip, int* status, cudaStream_t st);

template <typename T>
void launch_render(int Q, const TileWork* work, int n_work, const int* tile_src, const SourceDev* srcs,
                   const SrcPar<T>* par, const ImageDev* imgs, const int* skip, cudaStream_t st);

// Adaptive pixel integration (Sec. "Pixel Integration"), per source on its
// sampling box: a midpoint pass, the budget e = tol |F| / N of the source,
// order 3 on the pixels whose discrete Laplacian exceeds 24 e, the pixel split
// 5 x 5 with order 5 where orders 3 and 2 differ by more than e, and, where
// the summed orders 5 and 4 still differ by more than e, the sub-pixels whose
// order-5 and order-4 values differ by more than e / 25 split 5 x 5 again with
// order 7.  Samples are stored per source, box
// row-major, from aoff[s] (-1: a sky or an empty box, not sampled).
constexpr int ADAPT_THREADS = 256;
struct AdaptBlock {      // ADAPT_THREADS consecutive samples of one source's box
  int src;
  int l0;
};
struct AdaptPlan {
  const AdaptBlock* blocks;
  int n_blocks;
  const int* asrc;        // the sampled sources
  int n_asrc;
  const int* blk_ptr;     // blocks of asrc[k]: blk_ptr[k] .. blk_ptr[k + 1]
  const int64_t* aoff;    // per source: first sample (-1 none)
  double* part;           // per block: midpoint sum
  void* ebud;             // per source: budget e (T)
  int2* list;             // (source, box index) of the pixels past order 3
  int* n_list;
  unsigned long long* counts;   // final levels 0..3, refined sub-pixels
  uint8_t* level;         // per sample: final level
  uint32_t* refbits;      // per sample at the last level: its sub-pixels to split again (bit q = sub-pixel q)
  int deep_blocks;        // grid of the deep passes (persistent, grid-stride)
};
constexpr int ADAPT_COUNTS = 5;

template <typename T>
void launch_adaptive(const AdaptPlan& ap, const SourceDev* srcs, const SrcPar<T>* par, double tol, T* v0buf, T* vbuf,
                     cudaStream_t st);

// the layers from the adaptive samples (skies computed in place)
template <typename T>
void launch_render_samples(const TileWork* work, int n_work, const int* tile_src, const SourceDev* srcs,
                           const SrcPar<T>* par, const ImageDev* imgs, const int64_t* aoff, const T* vbuf,
                           cudaStream_t st);

// Pixel-centred sampling with an interpolated re-shift (see ap_render.cu):
// per shifted source (a convolved profile source) its box's samples at the
// snapped centre (R) and shifted back (S) from soff[s] (-1: not shifted).
struct ShiftPlan {
  const AdaptBlock* blocks;   // ADAPT_THREADS consecutive box pixels of one shifted source
  int n_blocks;
  const int64_t* soff;
  void* snap;                 // per source: the record with a snapped centre (SrcPar<T>)
  void* shift;                // per source: (du, dv) (T)
  void* R;                    // box samples at the snapped centre (T)
  void* S;                    // the same moved back (T)
};
template <typename T>
void launch_shifted_render(int Q, int method, const ShiftPlan& sp, const TileWork* work, int n_work,
                           const int* tile_src, const SourceDev* srcs, const SrcPar<T>* par, const ImageDev* imgs,
                           int n_src, cudaStream_t st);

// live PSFs: render the normalised PSF (plain and flipped, rows of K4) and
// its flipped derivatives of every live image from theta; the columns
// (dP/dphi) * G on the image from the galaxy layer
template <typename T>
void launch_live_psf(int Q, const int* live_imgs, int n_live, const SourceDev* srcs, const ImageDev* imgs,
                     const double* theta, int* status, cudaStream_t st);
template <typename T>
void launch_live_cols(const int* live_imgs, int n_live, const ImageDev* imgs, int max_tiles, int Kmax,
                      cudaStream_t st);
int configure_live(int Kmax, int is_double);   // shared-memory opt-in of the column kernel; 0: does not fit

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
                         const ImageDev* imgs, double* chi2_partial, void* const* model_out, const int* skip,
                         int trial, int* status, int kmax, cudaStream_t st);

// adjoint correlation: adj = P (correlate) w r over the galaxy layer
template <typename T>
void launch_adjoint_conv(int tile_variant, const ConvWork* work, const ConvRange* ranges, int n_ranges,
                         const ImageDev* imgs, int kmax, cudaStream_t st);

template <typename T> void configure_conv(int Kmax, int* ok);
template <typename T>
void launch_jcol(int variant, const JcolWork* work, const ConvRange* ranges, int n_ranges, const SourceDev* srcs,
                 const ImageDev* imgs, const T* dbuf, T* jbuf, int kmax, cudaStream_t st);
// FFT mode of the Jacobian-column convolution (float only; see ap_fft.cu)
constexpr int FFT_MAX_K64 = 33, FFT_MAX_K128 = 97;   // largest PSF per FFT block size (B >= 32)
int configure_fft();
std::vector<float2> fft_twiddles(int N);
void launch_psf_spectrum(int N, const float* psf_norm, int K, int K4, const float2* tw, float2* spec,
                         cudaStream_t st);
void launch_jcol_fft(int N, const JcolFftWork* work, int n, const SourceDev* srcs, const ImageDev* imgs,
                     const float* dbuf, float* jbuf, const float2* tw, cudaStream_t st);
template <typename T> void configure_gram(int unused);
template <typename T> void gram_blocking(int maxc, int* cb, int* two);
int gram_max_cols(int is_double);
int conv_tile_w(int variant);
int conv_tile_h(int variant);
int conv_threads(int variant);
constexpr int N_CONV_VARIANTS = 7;

void launch_sum_groups(const double* partial, const int* ptr, const int* idx, int n_out, double* out,
                       double scale, const int* skip, const double* keep, cudaStream_t st);
void launch_sum_contrib(const double* partial, const int64_t* ptr, const int64_t* idx, int n_out, double* out,
                        double scale, cudaStream_t st);

// J^T W J in two passes (see ap_gram.cu).  A source pair is two sources
// (A <= B) reaching a common image tile; its block holds the m_A x m_B
// products of their free columns.
struct GramPair {
  int64_t base;   // first scratch value: the block of each tile the pair meets, tile after tile
  int64_t pos;    // first of its 2 m_A m_B CSR positions ((row A, col B), (row B, col A); -1 = none)
  int cnt;        // tiles the pair meets
  int ma, mb;     // free columns of A and B
  int excl;       // 1: no other pair adds to its CSR entries (plain stores)
};

// A pair meeting more than GRAM_HEAVY_TILES tiles keeps its scratch entry
// by entry (the tiles of one entry contiguous); each entry is summed by one
// warp, or by a whole CTA when it spans more than GRAM_CTA_TILES tiles (a
// source and the sky, the sky and itself).  The other pairs keep it tile by
// tile and are summed by one warp per pair.
constexpr int GRAM_HEAVY_TILES = 64;
constexpr int GRAM_CTA_TILES = 2048;

struct GramRange {     // tiles [t0, t1) of the tile list share one column blocking
  int t0, t1, cb, two;
  int tc;              // float path: tcgen05 kernel form (gram_tc_kind: 1, 2, 3), 0 = warp MMA
};

// One free Jacobian column of a tile, as the tensor-core tile Gram reads it
// (planned on the host): the column image at element offset `off` of the
// convolved-column buffer (info bit 30 set) or of the derivative buffer, its
// row pitch bw, the offset off0 of the tile's pixel (0, 0) in it (may lie
// outside the image), its box in tile coordinates clamped to 0..16 (rows
// [b0, b1), columns [b2, b3), a byte each) and
// info = (local source << 8) | (free slot << 4) | free slots of the source.
struct GramCol {
  int64_t off;
  int off0;
  int bw;
  uint32_t bounds;
  int info;
};
constexpr int GRAM_COL_CONV = 1 << 30;

struct GramPlan {
  const int64_t* tab0;   // per tile: first entry of its pair table
  const int64_t* tab;    // per tile, per local pair (a <= b): scratch offset of its block
  const int* tabs;       //   and the stride between the block's entries (1, or the pair's tile count)
  double* scr;           // per-tile pair blocks
  const GramPair* pairs; // light pairs first, then the heavy ones
  const int64_t* pos;    // CSR positions of the pair blocks' entries
  int n_light, n_heavy;
  const int* heavy_items; // (heavy pair << 6) | entry, for every stored entry of the heavy pairs:
  int n_heavy_items;      //   first the n_heavy_cta entries summed by a CTA each, then those summed by a warp
  int n_heavy_cta;
  const int64_t* col_ptr; // float path: per tile, its first column in cols (with a closing entry)
  const GramCol* cols;    //   the tiles' free columns in (source, slot) order
};

// independent launches forked from a stream onto auxiliary streams and
// joined back (in a captured graph they become parallel branches)
constexpr int N_AUX_STREAMS = 4;
struct ForkJoin {
  cudaStream_t aux[N_AUX_STREAMS];
  cudaEvent_t fork;
  cudaEvent_t join[N_AUX_STREAMS];
};

// tcgen05 tile Grams (float path, tiles of up to gram_tc_max_cols() columns;
// see ap_gram_tc.cu)
int gram_tc_max_cols();
constexpr int GRAM_TC_MIN_DEFAULT = 33;   // before the planner has timed the two kernels
// kernel form of a tile of `cols` columns: 1 (up to 64), 2 (up to 128), 3 (up to 256)
int gram_tc_kind(int cols);
void configure_gram_tc();
void launch_gram_tc(int kind, const TileWork* work, int t0, int t1, const int* jt_src, const SourceDev* srcs,
                    const ImageDev* imgs, const float* dbuf, const float* jbuf, const GramPlan& gp, int* status,
                    cudaStream_t st);

template <typename T>
void launch_gram(const TileWork* work, const GramRange* ranges, int n_ranges, const int* jt_src,
                 const SourceDev* srcs, const ImageDev* imgs, const T* dbuf, const T* jbuf, const GramPlan& gp,
                 double* vals, int* status, cudaStream_t st, const ForkJoin* fj);

// solver
// Preconditioner blocks of the block-Jacobi PCG: the parameters of one
// object (the sources that share parameters, as one galaxy's shape and its
// per-band fluxes in a joint fit), at most PCG_BLK of them in a block.
constexpr int PCG_BLK = 16;
constexpr int PCG_BLK2 = PCG_BLK * PCG_BLK;
struct GroupDev {
  int n;               // parameters in the group
  int p0;              // offset into the group's parameter list
  int dense;           // 1: dense Cholesky, 0: one-CTA PCG, 2: grid-wide PCG, 3: cluster PCG
  int nblk;            // preconditioner blocks
  int b0;              // offset into the block list
};

// SpMV chunks of the PCG solvers: rows of up to DIST_WARP_ROW entries are cut
// into thread chunks of at most DIST_CHUNK entries, longer rows into warp
// chunks of DIST_WCHUNK entries (more for rows that would otherwise have more
// than DIST_MAX_PARTS chunks)
constexpr int DIST_CHUNK = 16;
constexpr int DIST_WARP_ROW = 64;
constexpr int DIST_WCHUNK = 128;
constexpr int DIST_MAX_PARTS = 16;

// the distributed PCG's plan (device pointers; see ap_solve.cu)
struct DistPlan {
  const int64_t* e0;      // first CSR entry of each chunk (chunks row-contiguous, rows in group order)
  const int64_t* e1;      // one past the last
  const int* lrow;        // group-local row of each chunk
  const int* row;         // chunks of group row r (concatenated over groups): [row[r], row[r+1])
  const int* tlist;       // thread chunks of group g: tlist[tptr[g] .. tptr[g+1])
  const int* tptr;
  const int* wlist;       // warp chunks of group g: wlist[wptr[g] .. wptr[g+1])
  const int* wptr;
  const int* owner;       // rank of the CTA owning each chunk's row (cluster groups)
  const int* dst;         // offset of each chunk's partial in its owner's partial array (cluster groups)
  const int* own_blk;     // per group, nct + 1 block boundaries of the CTAs' runs, at own_ptr[g]
  const int* own_ptr;
  const int* loff;        // offset of each block's packed inverse (m x m) in its owner's array
  const int32_t* lcol;    // group-local column of each CSR entry
  double* part;           // chunk partial sums in global memory (grid groups)
};

// per-CTA shared-memory extents of a distributed-PCG launch
struct DistSmem {
  int nr;   // most rows owned by one CTA
  int nb;   // most block-inverse doubles (sum of m^2 over owned blocks) of one CTA
  int nu;   // u copy: the group's rows (cluster) or the owned rows (grid)
  int np;   // most chunk partials of one CTA's rows (cluster; 0 on the grid)
};

struct DistLaunch {
  int grid_blocks = 0;        // CTAs of a grid-wide launch
  int cluster_size = 0;       // CTAs per cluster
  int n_cluster_groups = 0;   // clusters (one group each)
  DistSmem grid_sz{}, cluster_sz{};
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
  const int64_t* bpos;    // PCG_BLK2 CSR positions per preconditioner block (row stride PCG_BLK; -1: zero)
  double* work;           // 6 n doubles per group (grid PCG vectors)
  double* blk_work;       // PCG_BLK2 doubles per preconditioner block (its inverse, row stride PCG_BLK)
  double* part;           // grid-wide PCG reduction slots: 8 doubles per CTA
  int* iters;             // CG iterations of each group's last solve
  const int64_t* ch_e0;   // SpMV chunks (<= DIST_CHUNK CSR entries of one row): first entry
  const int64_t* ch_e1;   //   one past the last entry
  const int* ch_row;      // chunks of group row r (concatenated over groups): [ch_row[r], ch_row[r+1])
  double* ch_part;        // chunk partial sums
  const int* cluster_groups;  // groups solved by the cluster PCG, one per cluster
  DistPlan dist;          // the chunk and ownership plan of the distributed PCG
};

constexpr int PCG_ONE_CTA_MAX = 2048;     // largest group for the one-CTA PCG
constexpr int64_t CLUSTER_NNZ_MAX = 262144;  // largest J^T W J block of a group for the cluster PCG
constexpr int CLUSTER_N_MAX = 8192;          // largest group for the cluster PCG
constexpr size_t CLUSTER_SMEM_MAX = 200 * 1024;  // shared memory of one cluster-PCG CTA at most

void configure_solve();
size_t dist_smem_bytes(const DistSmem& sz, int nct, bool cluster);
int grid_pcg_blocks(int device, size_t smem);
int cluster_pcg_size(int device, size_t smem);
void launch_lm_solve(int n_groups, const SolvePlan& sp, const double* vals, const double* jtwr, double* lambda,
                     double* delta, int* status, cudaStream_t st, int any_dense, int any_pcg, int max_dense,
                     int max_pcg);
int launch_pcg_dist(const GroupDev* groups_host, int n_groups, const SolvePlan& sp, const double* vals,
                    const double* jtwr, double* lambda, double* delta, const DistLaunch& dl, int* status,
                    cudaStream_t st);

void launch_trial(const double* theta, const double* delta, const double* lo, const double* hi,
                  double* trial, int n, cudaStream_t st);
void launch_accept(const int* param_group, int n_params, const double* chi2_now, const double* chi2_trial,
                   double* theta, const double* trial, double* lambda, double* chi2_state, double* log,
                   int n_groups, cudaStream_t st);
void launch_accept_params(const int* param_group, int n_params, const int* accepted, double* theta,
                          const double* trial, cudaStream_t st);
void launch_accept_groups(const double* chi2_now, const double* chi2_trial, double* lambda,
                          double* chi2_state, double* log, int* accepted, int* fwd_valid, int n_groups,
                          cudaStream_t st);

// A run of 32-bit words of the trial point's forward state (source records,
// w r) and where it goes when the group accepts: the copy makes them the
// current point's.
struct StateChunk {
  const uint32_t* src;
  uint32_t* dst;
  int n_words;
  int group;
};
constexpr int STATE_CHUNK_WORDS = 16384;
void launch_accept_state(const StateChunk* chunks, int n_chunks, const int* accepted, cudaStream_t st);
void launch_scale(const double* in, double* out, double s, int n, cudaStream_t st);
// dst_dev[0..n) = src_host[0..n), stream-ordered, the values passed in kernel
// arguments (runs of PTR_RUN pointers per launch)
constexpr int PTR_RUN = 256;
void launch_store_ptrs(void* const* src_host, int n, void** dst_dev, cudaStream_t st);

}  // namespace ap
