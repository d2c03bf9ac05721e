// C-ABI entry points of libastrophot_gb300: the context, the host-side plans
// built once per problem (tile -> source lists, Jacobian tiles, the sparse
// J^T W J pattern, parameter groups) and the launch sequences of every call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ap_internal.cuh"

using namespace ap;

namespace {

const int SLOTS_OF[7] = {7, 6, 6, 7, 1, 3, 3};

struct Timer {
  std::string name;
  cudaEvent_t a, b;
};

struct TimingStats {
  std::vector<std::string> names;
  std::vector<double> total_ms;
  std::vector<long> count;
};

}  // namespace

struct ap_ctx {
  ap_options opt{};
  bool f64 = false;
  std::string err;
  // problem sizes
  int n_img = 0, n_src = 0, n_params = 0, n_groups = 0;
  bool have_problem = false;
  std::vector<ImageDev> h_imgs;
  std::vector<SourceDev> h_srcs;
  std::vector<void*> allocs;  // every device allocation of the problem
  ImageDev* d_imgs = nullptr;
  SourceDev* d_srcs = nullptr;
  void* d_par = nullptr;
  void* d_par_trial = nullptr;           // source records at the LM trial point
  int* d_fwd_valid = nullptr;            // per group: current records / w r / chi2_state in place
  StateChunk* d_state_chunks = nullptr;  // trial -> current copies of an accepted group
  int n_state_chunks = 0;
  double* d_bn_memo = nullptr;   // per source: the last two (n, b_n, db/dn) of prepare_kernel
  // render / adjoint-render plan
  TileWork* d_rwork = nullptr;
  int n_rwork = 0;
  int* d_tile_src = nullptr;
  int64_t n_tile_entries = 0;
  double* d_grad_partial = nullptr;
  int64_t* d_gc_ptr = nullptr;
  int64_t* d_gc_idx = nullptr;
  // correlation plans, one per tile variant (the autotuner picks one)
  int conv_variant = 0;
  ConvWork* d_fwork = nullptr;
  int n_fwork = 0;
  ConvWork* d_awork = nullptr;
  int n_awork = 0;
  int* d_grp_ptr = nullptr;
  int* d_grp_idx = nullptr;
  ConvWork* v_fwork[N_CONV_VARIANTS] = {};
  int v_nf[N_CONV_VARIANTS] = {};
  ConvWork* v_awork[N_CONV_VARIANTS] = {};
  int v_na[N_CONV_VARIANTS] = {};
  int* v_grp_ptr[N_CONV_VARIANTS] = {};
  int* v_grp_idx[N_CONV_VARIANTS] = {};
  double conv_ms[N_CONV_VARIANTS] = {};
  std::vector<ConvRange> v_frange[N_CONV_VARIANTS], v_arange[N_CONV_VARIANTS];
  std::vector<ConvRange> frange, arange, jcrange;
  double* d_chi2_partial = nullptr;
  int Kmax = 1;
  // Jacobian columns of convolved sources
  JcolWork* d_jcwork = nullptr;
  int n_jcwork = 0;
  // FFT mode of the Jacobian columns (float only): work per block size,
  // chosen over the direct correlation by timing at set_problem
  JcolFftWork* d_jfwork = nullptr;
  int n_jf64 = 0, n_jf128 = 0;
  float2* d_tw64 = nullptr;
  float2* d_tw128 = nullptr;
  int jcol_fft = 0;
  ForkJoin fj{};            // auxiliary streams for independent launches
  bool have_fj = false;
  double jcol_ms_direct = -1.0, jcol_ms_fft = -1.0;
  void* d_jbuf = nullptr;
  int64_t jbuf_elems = 0;
  // Jacobian plan
  TileWork* d_jwork = nullptr;
  int n_jwork = 0;
  int* d_jt_src = nullptr;
  GramPlan gplan{};
  std::vector<GramRange> gram_ranges;
  std::vector<int> h_tile_ncol;   // columns of every Gram tile (sorted)
  int gram_tc_min = 0;            // float path: tiles with tc_min .. tc_max columns run on tcgen05
  int gram_tc_max = 0;
  void* d_dbuf = nullptr;
  int64_t dbuf_elems = 0;
  std::vector<int64_t> h_row_ptr;
  std::vector<int32_t> h_col_idx;
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col_idx = nullptr;
  double* d_vals = nullptr;
  int64_t nnz = 0;
  // solver
  std::vector<int> h_param_group;
  GroupDev* d_groups = nullptr;
  int* d_gparams = nullptr;
  int* d_plocal = nullptr;
  int* d_blk_ptr = nullptr;
  double* d_work = nullptr;
  double* d_blk_work = nullptr;
  int max_dense_n = 1, max_pcg_n = 1;
  int any_dense = 0, any_pcg = 0, any_grid = 0;
  std::vector<GroupDev> h_groups;
  SolvePlan sp{};
  DistLaunch dl;
  int* d_param_group = nullptr;
  double* d_lo = nullptr;
  double* d_hi = nullptr;
  // LM state
  double* d_theta = nullptr;
  double* d_trial = nullptr;
  double* d_delta = nullptr;
  double* d_jtwr = nullptr;
  double* d_grad = nullptr;
  double* d_chi2 = nullptr;
  double* d_chi2_trial = nullptr;
  double* d_chi2_state = nullptr;
  double* d_lambda = nullptr;
  int* d_accepted = nullptr;
  int* d_cg_iters = nullptr;
  double* d_log = nullptr;
  int* d_log_iter = nullptr;
  int log_cap = 1024;
  int* d_status = nullptr;
  void** d_model_ptrs = nullptr;
  int64_t iterations = 0;
  bool lm_started = false;   // ap_lm_iterate has run since the problem was set
  // CUDA graph of one LM iteration
  cudaGraphExec_t lm_exec = nullptr;
  cudaGraph_t lm_graph = nullptr;
  int launches_last_eval = 0;
  // timing
  bool timing = false;
  std::vector<Timer> pending;
  std::vector<cudaEvent_t> event_pool;
  TimingStats stats;

  // adaptive pixel integration: built by the first call that needs it
  bool have_adapt = false;
  AdaptPlan adapt{};
  int64_t n_asamples = 0;
  std::vector<int64_t> h_aoff;
  void* d_av0 = nullptr;   // midpoint values
  void* d_av = nullptr;    // adaptive values

  // pixel-centred sampling with a re-shift: built by the first call that needs it
  bool have_shift = false;
  ShiftPlan shift{};

  // live PSFs: the images that have one (their internal sources follow the
  // caller's n_src_user sources)
  int* d_live_imgs = nullptr;
  int n_live = 0;
  int n_src_user = 0;
  int max_live_tiles = 0;   // 16 x 16 output tiles of the largest live-PSF image
};

namespace {

int fail(ap_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CUDA_TRY(ctx, call)                                                                         \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? AP_ERR_NOMEM : AP_ERR_CUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    }                                                                                               \
  } while (0)

cudaEvent_t take_event(ap_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Launch bracket: records an event pair around a launch when timing is on.
struct Bracket {
  ap_ctx* c;
  cudaStream_t st;
  Timer t;
  bool on;
  Bracket(ap_ctx* c_, cudaStream_t st_, const char* name) : c(c_), st(st_), on(c_->timing) {
    if (on) {
      t.name = name;
      t.a = take_event(c);
      t.b = take_event(c);
      cudaEventRecord(t.a, st);
    }
  }
  ~Bracket() {
    if (on) {
      cudaEventRecord(t.b, st);
      c->pending.push_back(t);
    }
  }
};

template <typename T>
int64_t alloc_bytes(int64_t n) { return n * (int64_t)sizeof(T); }

int dev_alloc(ap_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, e == cudaErrorMemoryAllocation ? AP_ERR_NOMEM : AP_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return AP_OK;
}

template <typename V>
int upload(ap_ctx* c, V** dst, const std::vector<typename std::remove_const<V>::type>& src) {
  int rc = dev_alloc(c, (void**)dst, src.size() * sizeof(V));
  if (rc) return rc;
  if (!src.empty()) CUDA_TRY(c, cudaMemcpy((void*)*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice));
  return AP_OK;
}

void free_problem(ap_ctx* c) {
  if (c->lm_exec) cudaGraphExecDestroy(c->lm_exec);
  if (c->lm_graph) cudaGraphDestroy(c->lm_graph);
  c->lm_exec = nullptr;
  c->lm_graph = nullptr;
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->d_tw64 = c->d_tw128 = nullptr;
  c->d_jfwork = nullptr;
  c->n_jf64 = c->n_jf128 = 0;
  c->jcol_fft = 0;
  c->jcol_ms_direct = c->jcol_ms_fft = -1.0;
  c->have_problem = false;
  c->lm_started = false;
  c->have_adapt = false;
  c->adapt = AdaptPlan{};
  c->n_asamples = 0;
  c->h_aoff.clear();
  c->d_av0 = c->d_av = nullptr;
  c->have_shift = false;
  c->shift = ShiftPlan{};
  c->d_live_imgs = nullptr;
  c->n_live = 0;
  c->n_src_user = 0;
  c->h_tile_ncol.clear();
  c->gram_tc_min = GRAM_TC_MIN_DEFAULT;
}

// Parameter box applied after each LM update: q in [0.05, 1], Sersic n in
// [0.36, 8], Moffat n in [1.05, 50], Re / Rd / sigma >= 1e-3; a shared index
// takes the intersection of its slots' boxes.
void param_bounds(const std::vector<SourceDev>& srcs, int n_params, std::vector<double>& lo, std::vector<double>& hi) {
  lo.assign(n_params, -INFINITY);
  hi.assign(n_params, INFINITY);
  for (const auto& s : srcs) {
    for (int k = 0; k < s.nslot; ++k) {
      const int p = s.pidx[k];
      if (p < 0) continue;
      double a = -INFINITY, b = INFINITY;
      if (s.type <= AP_MOFFAT && k == 2) { a = 0.05; b = 1.0; }
      else if (s.type == AP_SERSIC && k == 4) { a = 0.36; b = 8.0; }
      else if (s.type == AP_MOFFAT && k == 4) { a = 1.05; b = 50.0; }
      else if ((s.type == AP_SERSIC && k == 5) || ((s.type == AP_EXPONENTIAL || s.type == AP_GAUSSIAN) && k == 4) ||
               (s.type == AP_MOFFAT && k == 5)) { a = 1e-3; }
      else if (s.type == AP_LIVE_PSF_SRC && k == 0) { a = 1.05; b = 50.0; }   // live Moffat PSF n, Rd
      else if (s.type == AP_LIVE_PSF_SRC && k == 1) { a = 1e-3; }
      lo[p] = std::max(lo[p], a);
      hi[p] = std::min(hi[p], b);
    }
  }
}

// skip (device, per group, nullable): groups whose source records, w r and
// chi^2 (d_chi2_state) at theta are already in place keep them; the gradient
// and everything after it run for every group.  trial: the forward state goes
// to the trial buffers (d_par_trial, wr_trial), leaving the current point's.
template <typename T>
int do_eval(ap_ctx* c, const double* theta, double* chi2_out, double* grad_out, void* const* model_ptrs_dev,
            bool want_D, const int* skip, bool trial, cudaStream_t st) {
  SrcPar<T>* par = (SrcPar<T>*)(trial ? c->d_par_trial : c->d_par);
  c->launches_last_eval = (c->n_src > 0) + (c->n_rwork > 0) + (c->n_fwork > 0) + (chi2_out && c->n_groups > 0) +
                          (grad_out ? (c->n_awork > 0) + (c->n_rwork > 0) + (c->n_params > 0) : 0);
  {
    Bracket b(c, st, "prepare");
    launch_prepare<T>(c->d_srcs, c->d_imgs, c->n_src, theta, par, c->d_bn_memo, skip, c->d_status, st);
  }
  if (c->n_live > 0) {
    // every evaluation renders the live PSFs at its theta (never skipped: the
    // trial evaluation leaves its own PSF behind)
    Bracket b(c, st, "live_psf");
    launch_live_psf<T>(c->opt.quad_order, c->d_live_imgs, c->n_live, c->d_srcs, c->d_imgs, theta, c->d_status, st);
  }
  {
    Bracket b(c, st, "render");
    launch_render<T>(c->opt.quad_order, c->d_rwork, c->n_rwork, c->d_tile_src, c->d_srcs, par, c->d_imgs, skip, st);
  }
  {
    Bracket b(c, st, "forward_conv_chi2");
    launch_forward_conv<T>(c->conv_variant, c->d_fwork, c->frange.data(), (int)c->frange.size(), c->d_imgs,
                           c->d_chi2_partial, model_ptrs_dev, skip, trial ? 1 : 0, c->d_status, c->Kmax, st);
  }
  if (chi2_out) {
    Bracket b(c, st, "chi2_gather");
    launch_sum_groups(c->d_chi2_partial, c->d_grp_ptr, c->d_grp_idx, c->n_groups, chi2_out, 1.0, skip,
                      c->d_chi2_state, st);
  }
  if (grad_out) {
    {
      Bracket b(c, st, "adjoint_conv");
      launch_adjoint_conv<T>(c->conv_variant, c->d_awork, c->arange.data(), (int)c->arange.size(), c->d_imgs, c->Kmax,
                             st);
    }
    if (c->n_live > 0) {
      Bracket b(c, st, "live_psf_columns");
      launch_live_cols<T>(c->d_live_imgs, c->n_live, c->d_imgs, c->max_live_tiles, c->Kmax, st);
    }
    {
      Bracket b(c, st, "render_adjoint");
      launch_render_adjoint<T>(c->opt.quad_order, c->d_rwork, c->n_rwork, c->d_tile_src, c->d_srcs,
                               (const SrcPar<T>*)c->d_par, c->d_imgs, c->d_grad_partial,
                               want_D ? (T*)c->d_dbuf : nullptr, st);
    }
    {
      Bracket b(c, st, "grad_gather");
      launch_sum_contrib(c->d_grad_partial, c->d_gc_ptr, c->d_gc_idx, c->n_params, grad_out, -2.0, st);
    }
  }
  return AP_OK;
}

int eval_any(ap_ctx* c, const double* theta, double* chi2_out, double* grad_out, void* const* model_ptrs_dev,
             bool want_D, cudaStream_t st, const int* skip = nullptr, bool trial = false) {
  return c->f64 ? do_eval<double>(c, theta, chi2_out, grad_out, model_ptrs_dev, want_D, skip, trial, st)
                : do_eval<float>(c, theta, chi2_out, grad_out, model_ptrs_dev, want_D, skip, trial, st);
}

void launch_jcol_fft_all(ap_ctx* c, cudaStream_t st) {
  // the two block sizes write disjoint columns: side by side when both exist
  const bool both = c->have_fj && c->n_jf64 > 0 && c->n_jf128 > 0;
  cudaStream_t s64 = st;
  if (both) {
    cudaEventRecord(c->fj.fork, st);
    cudaStreamWaitEvent(c->fj.aux[0], c->fj.fork, 0);
    s64 = c->fj.aux[0];
  }
  launch_jcol_fft(64, c->d_jfwork, c->n_jf64, c->d_srcs, c->d_imgs, (const float*)c->d_dbuf, (float*)c->d_jbuf,
                  c->d_tw64, s64);
  launch_jcol_fft(128, c->d_jfwork + c->n_jf64, c->n_jf128, c->d_srcs, c->d_imgs, (const float*)c->d_dbuf,
                  (float*)c->d_jbuf, c->d_tw128, st);
  if (both) {
    cudaEventRecord(c->fj.join[0], c->fj.aux[0]);
    cudaStreamWaitEvent(st, c->fj.join[0], 0);
  }
}

int normal_eq_any(ap_ctx* c, const double* theta, double* jtwr_out, cudaStream_t st, const int* skip = nullptr) {
  int rc = eval_any(c, theta, c->d_chi2, c->d_grad, nullptr, true, st, skip);
  if (rc) return rc;
  {
    Bracket b(c, st, "jtwr_scale");
    launch_scale(c->d_grad, jtwr_out, -0.5, c->n_params, st);
  }
  cudaMemsetAsync(c->d_vals, 0, (size_t)std::max<int64_t>(c->nnz, 1) * sizeof(double), st);
  {
    Bracket b(c, st, "jacobian_columns");
    if (c->f64)
      launch_jcol<double>(c->conv_variant, c->d_jcwork, c->jcrange.data(), (int)c->jcrange.size(), c->d_srcs,
                          c->d_imgs, (const double*)c->d_dbuf, (double*)c->d_jbuf, c->Kmax, st);
    else if (c->jcol_fft)
      launch_jcol_fft_all(c, st);
    else
      launch_jcol<float>(c->conv_variant, c->d_jcwork, c->jcrange.data(), (int)c->jcrange.size(), c->d_srcs,
                         c->d_imgs, (const float*)c->d_dbuf, (float*)c->d_jbuf, c->Kmax, st);
  }
  Bracket b(c, st, "jtwj_gram");
  if (c->f64)
    launch_gram<double>(c->d_jwork, c->gram_ranges.data(), (int)c->gram_ranges.size(), c->d_jt_src, c->d_srcs,
                        c->d_imgs, (const double*)c->d_dbuf, (const double*)c->d_jbuf, c->gplan, c->d_vals,
                        c->d_status, st, c->have_fj ? &c->fj : nullptr);
  else
    launch_gram<float>(c->d_jwork, c->gram_ranges.data(), (int)c->gram_ranges.size(), c->d_jt_src, c->d_srcs,
                       c->d_imgs, (const float*)c->d_dbuf, (const float*)c->d_jbuf, c->gplan, c->d_vals,
                       c->d_status, st, c->have_fj ? &c->fj : nullptr);
  return AP_OK;
}

int solve_any(ap_ctx* c, double* lambda, double* delta, cudaStream_t st) {
  {
    Bracket b(c, st, "lm_solve");
    launch_lm_solve(c->n_groups, c->sp, c->d_vals, c->d_jtwr, lambda, delta, c->d_status, st, c->any_dense,
                    c->any_pcg, c->max_dense_n, c->max_pcg_n);
  }
  if (c->any_grid || c->dl.n_cluster_groups > 0) {
    Bracket b(c, st, "lm_solve_dist");
    const int e = launch_pcg_dist(c->h_groups.data(), c->n_groups, c->sp, c->d_vals, c->d_jtwr, lambda, delta,
                                  c->dl, c->d_status, st);
    if (e) return fail(c, AP_ERR_CUDA, std::string("distributed PCG launch: ") + cudaGetErrorString((cudaError_t)e));
  }
  return AP_OK;
}

// one LM iteration on the context's theta / lambda buffers.  The trial's
// forward state (source records, w r) goes to separate buffers; an accepted
// group copies it over its current state, a rejecting group keeps its own,
// so after every iteration each group's current records, w r and chi^2 are in
// place (d_fwd_valid, cleared by every other evaluation) and the next
// iteration's forward launches at theta return at once: the model is
// evaluated once per iteration, at the trial point.
int lm_iteration(ap_ctx* c, cudaStream_t st) {
  // (with a live PSF theta is evaluated in full: its columns need the galaxy
  // layer at theta, which the trial evaluation overwrites)
  int rc = normal_eq_any(c, c->d_theta, c->d_jtwr, st, c->n_live > 0 ? nullptr : c->d_fwd_valid);
  if (rc) return rc;
  rc = solve_any(c, c->d_lambda, c->d_delta, st);
  if (rc) return rc;
  {
    Bracket b(c, st, "lm_trial");
    launch_trial(c->d_theta, c->d_delta, c->d_lo, c->d_hi, c->d_trial, c->n_params, st);
  }
  rc = eval_any(c, c->d_trial, c->d_chi2_trial, nullptr, nullptr, false, st, nullptr, true);
  if (rc) return rc;
  {
    Bracket b(c, st, "lm_accept");
    launch_accept_groups(c->d_chi2, c->d_chi2_trial, c->d_lambda, c->d_chi2_state, c->d_log, c->d_accepted,
                         c->d_fwd_valid, c->n_groups, st);
    launch_accept_params(c->d_param_group, c->n_params, c->d_accepted, c->d_theta, c->d_trial, st);
    launch_accept_state(c->d_state_chunks, c->n_state_chunks, c->d_accepted, st);
  }
  return AP_OK;
}

// Evaluations outside the LM iteration overwrite the forward buffers: the
// next LM iteration must evaluate every group at theta.
int drop_lm_reuse(ap_ctx* c, cudaStream_t st) {
  CUDA_TRY(c, cudaMemsetAsync(c->d_fwd_valid, 0, (size_t)std::max(c->n_groups, 1) * sizeof(int), st));
  return AP_OK;
}

// The adaptive-integration plan: every profile source with a non-empty box
// gets its box's samples (row-major) and runs of ADAPT_THREADS of them; the
// deep pass's list can hold every sample.
int build_adaptive(ap_ctx* c) {
  if (c->have_adapt) return AP_OK;
  for (int s = 0; s < c->n_src; ++s)
    if (c->h_srcs[s].type == AP_PSF_STAR)
      return fail(c, AP_ERR_ARG, "adaptive integration covers the analytic profiles: the problem has a PSF star");
  std::vector<int64_t> aoff(c->n_src, -1);
  std::vector<int> asrc, blk_ptr{0};
  std::vector<AdaptBlock> blocks;
  int64_t tot = 0;
  for (int s = 0; s < c->n_src; ++s) {
    const SourceDev& m = c->h_srcs[s];
    if (m.type > AP_MOFFAT) continue;
    const int n = (m.box[1] - m.box[0]) * (m.box[3] - m.box[2]);
    if (n <= 0) continue;
    aoff[s] = tot;
    asrc.push_back(s);
    for (int l0 = 0; l0 < n; l0 += ADAPT_THREADS) blocks.push_back(AdaptBlock{s, l0});
    blk_ptr.push_back((int)blocks.size());
    tot += n;
  }
  const size_t tsz = c->f64 ? sizeof(double) : sizeof(float);
  AdaptPlan& ap = c->adapt;
  int rc;
  AdaptBlock* d_blocks;
  int *d_asrc, *d_blk_ptr;
  int64_t* d_aoff;
  if ((rc = upload(c, &d_blocks, blocks)) || (rc = upload(c, &d_asrc, asrc)) || (rc = upload(c, &d_blk_ptr, blk_ptr)) ||
      (rc = upload(c, &d_aoff, aoff)))
    return rc;
  if ((rc = dev_alloc(c, (void**)&ap.part, std::max<size_t>(blocks.size(), 1) * sizeof(double))) ||
      (rc = dev_alloc(c, &ap.ebud, (size_t)std::max(c->n_src, 1) * sizeof(double))) ||
      (rc = dev_alloc(c, (void**)&ap.list, (size_t)std::max<int64_t>(tot, 1) * sizeof(int2))) ||
      (rc = dev_alloc(c, (void**)&ap.n_list, sizeof(int))) ||
      (rc = dev_alloc(c, (void**)&ap.counts, ADAPT_COUNTS * sizeof(unsigned long long))) ||
      (rc = dev_alloc(c, (void**)&ap.level, (size_t)std::max<int64_t>(tot, 1))) ||
      (rc = dev_alloc(c, (void**)&ap.refbits, (size_t)std::max<int64_t>(tot, 1) * sizeof(uint32_t))) ||
      (rc = dev_alloc(c, &c->d_av0, (size_t)std::max<int64_t>(tot, 1) * tsz)) ||
      (rc = dev_alloc(c, &c->d_av, (size_t)std::max<int64_t>(tot, 1) * tsz)))
    return rc;
  int sms = 0;
  CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device));
  ap.blocks = d_blocks;
  ap.n_blocks = (int)blocks.size();
  ap.asrc = d_asrc;
  ap.n_asrc = (int)asrc.size();
  ap.blk_ptr = d_blk_ptr;
  ap.aoff = d_aoff;
  ap.deep_blocks = std::max(sms, 1) * 8;
  c->n_asamples = tot;
  c->h_aoff = aoff;
  c->have_adapt = true;
  return AP_OK;
}

// The shift plan: every convolved profile source with a non-empty sampling
// box keeps its box's samples at soff[s]; blocks of ADAPT_THREADS box pixels.
int build_shift(ap_ctx* c) {
  if (c->have_shift) return AP_OK;
  std::vector<int64_t> soff(c->n_src, -1);
  std::vector<AdaptBlock> blocks;
  int64_t tot = 0;
  for (int s = 0; s < c->n_src; ++s) {
    const SourceDev& m = c->h_srcs[s];
    if (!m.conv || m.type > AP_MOFFAT) continue;
    const int n = (m.box[1] - m.box[0]) * (m.box[3] - m.box[2]);
    if (n <= 0) continue;
    soff[s] = tot;
    for (int l0 = 0; l0 < n; l0 += ADAPT_THREADS) blocks.push_back(AdaptBlock{s, l0});
    tot += n;
  }
  const size_t tsz = c->f64 ? sizeof(double) : sizeof(float);
  const size_t par_bytes = c->f64 ? sizeof(SrcPar<double>) : sizeof(SrcPar<float>);
  ShiftPlan& sp = c->shift;
  AdaptBlock* d_blocks;
  int64_t* d_soff;
  int rc;
  if ((rc = upload(c, &d_blocks, blocks)) || (rc = upload(c, &d_soff, soff)) ||
      (rc = dev_alloc(c, &sp.snap, (size_t)std::max(c->n_src, 1) * par_bytes)) ||
      (rc = dev_alloc(c, &sp.shift, (size_t)std::max(c->n_src, 1) * 2 * tsz)) ||
      (rc = dev_alloc(c, &sp.R, (size_t)std::max<int64_t>(tot, 1) * tsz)) ||
      (rc = dev_alloc(c, &sp.S, (size_t)std::max<int64_t>(tot, 1) * tsz)))
    return rc;
  sp.blocks = d_blocks;
  sp.n_blocks = (int)blocks.size();
  sp.soff = d_soff;
  c->have_shift = true;
  return AP_OK;
}

template <typename T>
void eval_shifted(ap_ctx* c, const double* theta, int method, double* chi2_out, bool model_out, cudaStream_t st) {
  SrcPar<T>* par = (SrcPar<T>*)c->d_par;
  {
    Bracket b(c, st, "prepare");
    launch_prepare<T>(c->d_srcs, c->d_imgs, c->n_src, theta, par, c->d_bn_memo, nullptr, c->d_status, st);
  }
  if (c->n_live > 0) {
    Bracket b(c, st, "live_psf");
    launch_live_psf<T>(c->opt.quad_order, c->d_live_imgs, c->n_live, c->d_srcs, c->d_imgs, theta, c->d_status, st);
  }
  {
    Bracket b(c, st, "render_shifted");
    launch_shifted_render<T>(c->opt.quad_order, method, c->shift, c->d_rwork, c->n_rwork, c->d_tile_src, c->d_srcs,
                             par, c->d_imgs, c->n_src, st);
  }
  {
    Bracket b(c, st, "forward_conv_chi2");
    launch_forward_conv<T>(c->conv_variant, c->d_fwork, c->frange.data(), (int)c->frange.size(), c->d_imgs,
                           c->d_chi2_partial, model_out ? c->d_model_ptrs : nullptr, nullptr, 0, c->d_status,
                           c->Kmax, st);
  }
  if (chi2_out) {
    Bracket b(c, st, "chi2_gather");
    launch_sum_groups(c->d_chi2_partial, c->d_grp_ptr, c->d_grp_idx, c->n_groups, chi2_out, 1.0, nullptr, nullptr,
                      st);
  }
}

template <typename T>
void eval_adaptive(ap_ctx* c, const double* theta, double tol, double* chi2_out, bool model_out, cudaStream_t st) {
  SrcPar<T>* par = (SrcPar<T>*)c->d_par;
  {
    Bracket b(c, st, "prepare");
    launch_prepare<T>(c->d_srcs, c->d_imgs, c->n_src, theta, par, c->d_bn_memo, nullptr, c->d_status, st);
  }
  if (c->n_live > 0) {
    Bracket b(c, st, "live_psf");
    launch_live_psf<T>(c->opt.quad_order, c->d_live_imgs, c->n_live, c->d_srcs, c->d_imgs, theta, c->d_status, st);
  }
  {
    Bracket b(c, st, "adaptive_sampling");
    launch_adaptive<T>(c->adapt, c->d_srcs, par, tol, (T*)c->d_av0, (T*)c->d_av, st);
  }
  {
    Bracket b(c, st, "render_samples");
    launch_render_samples<T>(c->d_rwork, c->n_rwork, c->d_tile_src, c->d_srcs, par, c->d_imgs, c->adapt.aoff,
                             (const T*)c->d_av, st);
  }
  {
    Bracket b(c, st, "forward_conv_chi2");
    launch_forward_conv<T>(c->conv_variant, c->d_fwork, c->frange.data(), (int)c->frange.size(), c->d_imgs,
                           c->d_chi2_partial, model_out ? c->d_model_ptrs : nullptr, nullptr, 0, c->d_status,
                           c->Kmax, st);
  }
  if (chi2_out) {
    Bracket b(c, st, "chi2_gather");
    launch_sum_groups(c->d_chi2_partial, c->d_grp_ptr, c->d_grp_idx, c->n_groups, chi2_out, 1.0, nullptr, nullptr,
                      st);
  }
}

// n_iter iterations from the context's theta / lambda (graph replay, or the
// bracketed launch sequence in timing mode), then the state out to the
// caller's buffers
int lm_run(ap_ctx* c, double* theta, double* lambda, double* chi2, int n_iter, double* log_host, cudaStream_t st) {
  const size_t P = (size_t)c->n_params, G = (size_t)c->n_groups;
  if (c->timing) {
    // timed mode: the same launch sequence without the graph, every kernel
    // bracketed by events
    for (int it = 0; it < n_iter; ++it) {
      int rc = lm_iteration(c, st);
      if (rc) return rc;
      if (log_host)
        CUDA_TRY(c, cudaMemcpyAsync(log_host + (size_t)it * G * 4, c->d_log, G * 4 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
    }
  } else {
    if (!c->lm_exec) {
      // capture one iteration on a private stream; the graph holds only
      // device pointers owned by the context
      cudaStream_t cs;
      CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(c, AP_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
      }
      int rc = lm_iteration(c, cs);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : fail(c, AP_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
      }
      e = cudaGraphInstantiate(&c->lm_exec, g, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(c, AP_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
      c->lm_graph = g;
    }
    for (int it = 0; it < n_iter; ++it) {
      CUDA_TRY(c, cudaGraphLaunch(c->lm_exec, st));
      if (log_host)
        CUDA_TRY(c, cudaMemcpyAsync(log_host + (size_t)it * G * 4, c->d_log, G * 4 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
    }
  }
  c->iterations += n_iter;
  if (theta) CUDA_TRY(c, cudaMemcpyAsync(theta, c->d_theta, P * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (lambda) CUDA_TRY(c, cudaMemcpyAsync(lambda, c->d_lambda, G * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (chi2) {
    if (n_iter > 0) {
      CUDA_TRY(c, cudaMemcpyAsync(chi2, c->d_chi2_state, G * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      int rc = eval_any(c, c->d_theta, chi2, nullptr, nullptr, false, st);
      if (rc) return rc;
      if ((rc = drop_lm_reuse(c, st))) return rc;
    }
  }
  if (log_host) CUDA_TRY(c, cudaStreamSynchronize(st));
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* ap_strerror(int code) {
  switch (code) {
    case AP_OK: return "ok";
    case AP_ERR_ARG: return "invalid argument";
    case AP_ERR_CUDA: return "CUDA error";
    case AP_ERR_NOT_SPD: return "damped normal matrix not positive definite";
    case AP_ERR_NONFINITE: return "non-finite or non-positive input";
    case AP_ERR_TIMEOUT: return "bounded device loop gave up";
    case AP_ERR_STATE: return "no problem set";
    case AP_ERR_NOMEM: return "device allocation failed";
    default: return "unknown status";
  }
}

int ap_create(ap_ctx** out, const ap_options* opt) {
  if (!out || !opt) return AP_ERR_ARG;
  *out = nullptr;
  if (opt->precision != AP_PREC_MIXED && opt->precision != AP_PREC_F64) return AP_ERR_ARG;
  if (!(opt->quad_order == 1 || opt->quad_order == 3 || opt->quad_order == 5 || opt->quad_order == 7))
    return AP_ERR_ARG;
  if (opt->jcol_mode < AP_JCOL_AUTO || opt->jcol_mode > AP_JCOL_FFT) return AP_ERR_ARG;
  if (opt->conv_variant < 0 || opt->conv_variant > N_CONV_VARIANTS) return AP_ERR_ARG;
  if (opt->gram_tc_min < 0) return AP_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || opt->device < 0 || opt->device >= ndev) return AP_ERR_CUDA;
  if (cudaSetDevice(opt->device) != cudaSuccess) return AP_ERR_CUDA;
  ap_ctx* c = new ap_ctx();
  c->opt = *opt;
  c->f64 = opt->precision == AP_PREC_F64;
  upload_gl_rule(opt->quad_order);
  bool ok = cudaEventCreateWithFlags(&c->fj.fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < N_AUX_STREAMS && ok; ++k)
    ok = cudaStreamCreateWithFlags(&c->fj.aux[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->fj.join[k], cudaEventDisableTiming) == cudaSuccess;
  c->have_fj = ok;
  if (!ok) cudaGetLastError();   // fall back to one stream
  *out = c;
  return AP_OK;
}

void ap_destroy(ap_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->opt.device);
  free_problem(c);
  for (auto& t : c->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->fj.fork) cudaEventDestroy(c->fj.fork);
  for (int k = 0; k < N_AUX_STREAMS; ++k) {
    if (c->fj.aux[k]) cudaStreamDestroy(c->fj.aux[k]);
    if (c->fj.join[k]) cudaEventDestroy(c->fj.join[k]);
  }
  delete c;
}

const char* ap_get_error(ap_ctx* c) { return c ? c->err.c_str() : ""; }

// The Gram's column blocking per run of tiles (sorted by column count): the
// float path sends tiles of tc_min .. min(tc_max, gram_tc_max_cols()) columns
// to the tcgen05 kernel (in the form for up to 32, 64 or 128 columns) and the
// others to the warp-MMA kernel (column blocks of up to 96); the float64 path
// blocks by 32.
std::vector<GramRange> gram_ranges_for(const std::vector<int>& tile_ncol, bool f64, int tc_min,
                                       int tc_max = 1 << 30) {
  std::vector<GramRange> out;
  for (size_t t = 0; t < tile_ncol.size(); ++t) {
    GramRange gr{(int)t, (int)t + 1, 0, 0, 0};
    if (f64) gram_blocking<double>(tile_ncol[t], &gr.cb, &gr.two);
    else if (tile_ncol[t] >= tc_min && tile_ncol[t] <= std::min(tc_max, gram_tc_max_cols()))
      gr.tc = gram_tc_kind(tile_ncol[t]);
    else gram_blocking<float>(tile_ncol[t], &gr.cb, &gr.two);
    if (!out.empty() && out.back().cb == gr.cb && out.back().two == gr.two && out.back().tc == gr.tc)
      out.back().t1++;
    else
      out.push_back(gr);
  }
  return out;
}

int ap_set_problem(ap_ctx* c, const ap_image_desc* imgs, int n_img, const ap_source_desc* srcs, int n_src,
                   int n_params, void* stream) {
  if (!c) return AP_ERR_ARG;
  cudaSetDevice(c->opt.device);
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(c, cudaStreamSynchronize(st));
  free_problem(c);
  c->err.clear();
  if (n_img <= 0 || !imgs) return fail(c, AP_ERR_ARG, "need at least one image");
  if (n_src < 0 || (n_src > 0 && !srcs)) return fail(c, AP_ERR_ARG, "bad source array");
  if (n_params < 0) return fail(c, AP_ERR_ARG, "n_params < 0");
  const bool f64 = c->f64;
  const size_t tsz = f64 ? sizeof(double) : sizeof(float);
  const int Q = c->opt.quad_order;
  (void)Q;

  // ---- images ----
  std::vector<ImageDev> I(n_img);
  if (!c->f64 && !configure_fft()) return fail(c, AP_ERR_CUDA, "FFT kernels cannot get their shared memory");
  int n_groups = 0;
  int Kmax = 1;
  for (int i = 0; i < n_img; ++i) {
    const ap_image_desc& d = imgs[i];
    ImageDev& m = I[i];
    std::memset(&m, 0, sizeof(m));
    if (d.H < 1 || d.W < 1 || (int64_t)d.H * d.W > (int64_t)1 << 31)
      return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": bad size");
    if (!d.data_dev || !d.variance_dev) return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": data/variance NULL");
    if (d.group < 0) return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": negative group");
    const double det = d.A[0] * d.A[3] - d.A[1] * d.A[2];
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det))
      return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": singular pixel-scale matrix");
    m.H = d.H;
    m.W = d.W;
    for (int k = 0; k < 4; ++k) m.A[k] = d.A[k];
    m.origin[0] = d.origin[0];
    m.origin[1] = d.origin[1];
    m.Ainv[0] = d.A[3] / det;
    m.Ainv[1] = -d.A[1] / det;
    m.Ainv[2] = -d.A[2] / det;
    m.Ainv[3] = d.A[0] / det;
    m.area = std::fabs(det);
    m.hx = 0.5 * (d.A[0] * d.W + d.A[1] * d.H);
    m.hy = 0.5 * (d.A[2] * d.W + d.A[3] * d.H);
    m.data = d.data_dev;
    m.var = d.variance_dev;
    m.mask = d.mask_dev;
    m.group = d.group;
    m.live_src = -1;
    if (d.psf_live) {
      for (int k = 0; k < 2; ++k)
        if (d.psf_pidx[k] < -1 || d.psf_pidx[k] >= n_params)
          return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": live PSF theta index out of range");
    }
    if (d.psf_dev || d.psf_live) {
      if (d.K < 1 || d.K % 2 == 0 || d.K > 255)
        return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": PSF size must be odd, 1..255");
      m.K = d.K;
      m.h = (d.K - 1) / 2;
      m.K4 = (d.K + 3) & ~3;
      Kmax = std::max(Kmax, d.K);
    }
    m.Hp = m.H + 2 * m.h;
    m.Wp = m.W + 2 * m.h;
    n_groups = std::max(n_groups, d.group + 1);
  }

  // ---- sources ----
  std::vector<SourceDev> S(n_src);
  for (int s = 0; s < n_src; ++s) {
    const ap_source_desc& d = srcs[s];
    SourceDev& m = S[s];
    std::memset(&m, 0, sizeof(m));
    if (d.type < 0 || d.type > AP_PSF_STAR) return fail(c, AP_ERR_ARG, "source " + std::to_string(s) + ": bad type");
    if (d.image < 0 || d.image >= n_img) return fail(c, AP_ERR_ARG, "source " + std::to_string(s) + ": bad image");
    m.type = d.type;
    m.image = d.image;
    m.nslot = SLOTS_OF[d.type];
    const ImageDev& im = I[d.image];
    if (d.type == AP_PSF_STAR && im.K <= 0)
      return fail(c, AP_ERR_ARG, "source " + std::to_string(s) + ": a PSF star needs an image with a PSF");
    m.conv = (d.psf_convolve && im.K > 0 && d.type != AP_PSF_STAR) ? 1 : 0;
    for (int k = 0; k < MAX_SLOTS; ++k) {
      m.pidx[k] = k < m.nslot ? d.pidx[k] : -1;
      m.pfix[k] = d.pfix[k];
      if (m.pidx[k] >= n_params || m.pidx[k] < -1)
        return fail(c, AP_ERR_ARG, "source " + std::to_string(s) + ": theta index out of range");
    }
    int x0 = std::max(d.win[0], 0), x1 = std::min(d.win[1], im.W);
    int y0 = std::max(d.win[2], 0), y1 = std::min(d.win[3], im.H);
    if (m.conv) {
      const int h = im.h;
      m.box[0] = std::max(y0 - h, -h);
      m.box[1] = std::min(y1 + h, im.H + h);
      m.box[2] = std::max(x0 - h, -h);
      m.box[3] = std::min(x1 + h, im.W + h);
    } else {
      m.box[0] = y0;
      m.box[1] = y1;
      m.box[2] = x0;
      m.box[3] = x1;
    }
    if (x0 >= x1 || y0 >= y1) m.box[0] = m.box[1] = m.box[2] = m.box[3] = 0;  // empty
    m.d_off = -1;
  }
  for (int s = 0; s < n_src; ++s)
    if (S[s].type == AP_PSF_STAR && imgs[S[s].image].psf_live)
      return fail(c, AP_ERR_ARG, "source " + std::to_string(s) + ": a PSF star needs a fixed PSF image");
  // a live PSF becomes an internal source of its image (slots n, Rd, the
  // whole image as its box): it joins the gradient, the Jacobian tiles and
  // J^T W J like a whole-image sky
  const int n_src_user = n_src;
  std::vector<int> live_imgs;
  for (int i = 0; i < n_img; ++i) {
    if (!imgs[i].psf_live) continue;
    SourceDev m;
    std::memset(&m, 0, sizeof(m));
    m.type = AP_LIVE_PSF_SRC;
    m.image = i;
    m.nslot = 2;
    m.conv = 0;
    for (int k = 0; k < MAX_SLOTS; ++k) {
      m.pidx[k] = k < 2 ? imgs[i].psf_pidx[k] : -1;
      m.pfix[k] = k < 2 ? imgs[i].psf_pfix[k] : 0.0;
    }
    m.box[0] = 0;
    m.box[1] = I[i].H;
    m.box[2] = 0;
    m.box[3] = I[i].W;
    m.d_off = -1;
    I[i].live_src = (int)S.size();
    S.push_back(m);
    live_imgs.push_back(i);
  }
  n_src = (int)S.size();
  for (int s = 0; s < n_src; ++s)
    if (S[s].conv) I[S[s].image].has_gal = 1;

  // ---- render tiles (galaxy layer + unconvolved layer per image) ----
  std::vector<TileWork> rwork;
  std::vector<int> tile_src;
  {
    struct PlaneTiles { int img, plane, r0, c0, nr, nc; std::vector<std::vector<int>> lists; };
    std::vector<PlaneTiles> planes;
    std::vector<int> plane_of(2 * n_img, -1);
    for (int i = 0; i < n_img; ++i) {
      const ImageDev& m = I[i];
      if (m.has_gal) {
        PlaneTiles p{i, 0, -m.h, -m.h, (m.Hp + TILE - 1) / TILE, (m.Wp + TILE - 1) / TILE, {}};
        p.lists.resize((size_t)p.nr * p.nc);
        plane_of[2 * i] = (int)planes.size();
        planes.push_back(std::move(p));
      }
      PlaneTiles u{i, 1, 0, 0, (m.H + TILE - 1) / TILE, (m.W + TILE - 1) / TILE, {}};
      u.lists.resize((size_t)u.nr * u.nc);
      plane_of[2 * i + 1] = (int)planes.size();
      planes.push_back(std::move(u));
    }
    for (int s = 0; s < n_src; ++s) {
      const SourceDev& m = S[s];
      if (m.box[0] >= m.box[1] || m.box[2] >= m.box[3]) continue;
      PlaneTiles& p = planes[plane_of[2 * m.image + (m.conv ? 0 : 1)]];
      const int tr0 = (m.box[0] - p.r0) / TILE, tr1 = (m.box[1] - 1 - p.r0) / TILE;
      const int tc0 = (m.box[2] - p.c0) / TILE, tc1 = (m.box[3] - 1 - p.c0) / TILE;
      for (int tr = tr0; tr <= tr1; ++tr)
        for (int tc = tc0; tc <= tc1; ++tc) p.lists[(size_t)tr * p.nc + tc].push_back(s);
    }
    for (auto& p : planes)
      for (int tr = 0; tr < p.nr; ++tr)
        for (int tc = 0; tc < p.nc; ++tc) {
          auto& L = p.lists[(size_t)tr * p.nc + tc];
          TileWork w{p.img, p.plane, p.r0 + tr * TILE, p.c0 + tc * TILE, (int)tile_src.size(), 0};
          tile_src.insert(tile_src.end(), L.begin(), L.end());
          w.e1 = (int)tile_src.size();
          rwork.push_back(w);
        }
    // heaviest tiles first
    std::stable_sort(rwork.begin(), rwork.end(),
                     [](const TileWork& a, const TileWork& b) { return (a.e1 - a.e0) > (b.e1 - b.e0); });
  }
  if ((int64_t)tile_src.size() > ((int64_t)1 << 31) - 1) return fail(c, AP_ERR_ARG, "tile list too large");

  // gradient contributions: theta index -> (entry, slot) of the adjoint partials
  std::vector<int64_t> gc_ptr(n_params + 1, 0), gc_idx;
  {
    std::vector<std::pair<int, int64_t>> pairs;
    for (const auto& w : rwork)
      for (int e = w.e0; e < w.e1; ++e) {
        const SourceDev& m = S[tile_src[e]];
        for (int k = 0; k < m.nslot; ++k)
          if (m.pidx[k] >= 0) pairs.emplace_back(m.pidx[k], (int64_t)e * MAX_SLOTS + k);
      }
    std::sort(pairs.begin(), pairs.end());
    gc_idx.resize(pairs.size());
    for (size_t k = 0; k < pairs.size(); ++k) {
      gc_ptr[pairs[k].first + 1]++;
      gc_idx[k] = pairs[k].second;
    }
    for (int p = 0; p < n_params; ++p) gc_ptr[p + 1] += gc_ptr[p];
  }

  // ---- correlation tiles: one plan per tile variant; work items sorted by
  // the image's PSF chunk count so each run shares one kernel instantiation ----
  std::vector<ConvWork> v_f[N_CONV_VARIANTS], v_a[N_CONV_VARIANTS];
  std::vector<int> v_gp[N_CONV_VARIANTS], v_gi[N_CONV_VARIANTS];
  std::vector<ConvRange> v_fr[N_CONV_VARIANTS], v_ar[N_CONV_VARIANTS];
  std::vector<int> img_nc(n_img, 0);
  for (int i = 0; i < n_img; ++i) img_nc[i] = I[i].has_gal ? conv_nc_of(I[i].K4, f64 ? 1 : 0) : 0;
  auto make_ranges = [&](std::vector<ConvWork>& wl, std::vector<ConvRange>& rg) {
    std::stable_sort(wl.begin(), wl.end(),
                     [&](const ConvWork& a, const ConvWork& b) { return img_nc[a.image] < img_nc[b.image]; });
    for (int k = 0; k < (int)wl.size(); ++k) {
      const int nc = img_nc[wl[k].image];
      if (rg.empty() || rg.back().nc != nc) rg.push_back(ConvRange{nc, k, 0});
      rg.back().count++;
    }
  };
  size_t max_nf = 1;
  for (int v = 0; v < N_CONV_VARIANTS; ++v) {
    const int TW = conv_tile_w(v), TH = conv_tile_h(v);
    for (int i = 0; i < n_img; ++i) {
      const ImageDev& m = I[i];
      for (int r = 0; r < m.H; r += TH)
        for (int cc = 0; cc < m.W; cc += TW) v_f[v].push_back(ConvWork{i, r, cc});
      if (m.has_gal)
        for (int r = 0; r < m.Hp; r += TH)
          for (int cc = 0; cc < m.Wp; cc += TW) v_a[v].push_back(ConvWork{i, r, cc});
    }
    make_ranges(v_f[v], v_fr[v]);
    make_ranges(v_a[v], v_ar[v]);
    std::vector<std::vector<int>> group_items(n_groups);
    for (int k = 0; k < (int)v_f[v].size(); ++k) group_items[I[v_f[v][k].image].group].push_back(k);
    v_gp[v].assign(n_groups + 1, 0);
    for (int g = 0; g < n_groups; ++g) {
      v_gi[v].insert(v_gi[v].end(), group_items[g].begin(), group_items[g].end());
      v_gp[v][g + 1] = (int)v_gi[v].size();
    }
    max_nf = std::max(max_nf, v_f[v].size());
  }

  // ---- derivative images and Jacobian tiles ----
  int64_t dbuf_elems = 0;
  int64_t jbuf_elems = 0;
  for (auto& m : S) {
    bool any_free = false;
    for (int k = 0; k < m.nslot; ++k) any_free |= m.pidx[k] >= 0;
    const int64_t area = (int64_t)(m.box[1] - m.box[0]) * (m.box[3] - m.box[2]);
    m.j_off = -1;
    m.sup[0] = m.sup[1] = m.sup[2] = m.sup[3] = 0;
    if (any_free && area > 0) {
      m.d_off = dbuf_elems;
      dbuf_elems += area * m.nslot;
      const ImageDev& im = I[m.image];
      const int hh = m.conv ? im.h : 0;
      m.sup[0] = std::max(m.box[0] - hh, 0);
      m.sup[1] = std::min(m.box[1] + hh, im.H);
      m.sup[2] = std::max(m.box[2] - hh, 0);
      m.sup[3] = std::min(m.box[3] + hh, im.W);
      if (m.sup[0] >= m.sup[1] || m.sup[2] >= m.sup[3]) m.sup[0] = m.sup[1] = m.sup[2] = m.sup[3] = 0;
      const int64_t sarea = (int64_t)(m.sup[1] - m.sup[0]) * (m.sup[3] - m.sup[2]);
      if (m.conv && sarea > 0) {
        m.j_off = jbuf_elems;
        jbuf_elems += sarea * m.nslot;
      }
    }
  }
  std::vector<TileWork> jwork;
  std::vector<int> jt_src, tile_ncol;
  int gram_cols = 4;
  std::vector<std::vector<int>> rows_of(n_params);
  {
    std::set<std::pair<int, int>> src_pairs;
    gram_cols = 4;
    for (int i = 0; i < n_img; ++i) {
      const ImageDev& m = I[i];
      const int nr = (m.H + TILE - 1) / TILE, nc = (m.W + TILE - 1) / TILE;
      std::vector<std::vector<int>> lists((size_t)nr * nc);
      for (int s = 0; s < n_src; ++s) {
        const SourceDev& sd = S[s];
        if (sd.image != i || sd.d_off < 0) continue;
        const int r0 = sd.sup[0], r1 = sd.sup[1], c0 = sd.sup[2], c1 = sd.sup[3];
        if (r0 >= r1 || c0 >= c1) continue;
        for (int tr = r0 / TILE; tr <= (r1 - 1) / TILE; ++tr)
          for (int tc = c0 / TILE; tc <= (c1 - 1) / TILE; ++tc) lists[(size_t)tr * nc + tc].push_back(s);
      }
      for (int tr = 0; tr < nr; ++tr)
        for (int tc = 0; tc < nc; ++tc) {
          auto& L = lists[(size_t)tr * nc + tc];
          if (L.empty()) continue;
          int ncol = 0;
          for (int s : L)
            for (int k = 0; k < S[s].nslot; ++k) ncol += S[s].pidx[k] >= 0;

          gram_cols = std::max(gram_cols, ncol);
          TileWork w{i, 1, tr * TILE, tc * TILE, (int)jt_src.size(), 0};
          jt_src.insert(jt_src.end(), L.begin(), L.end());
          w.e1 = (int)jt_src.size();
          jwork.push_back(w);
          for (size_t a = 0; a < L.size(); ++a)
            for (size_t b = a; b < L.size(); ++b) src_pairs.insert({L[a], L[b]});
        }
    }
    for (auto& pr : src_pairs) {
      const SourceDev& A = S[pr.first];
      const SourceDev& B = S[pr.second];
      for (int k = 0; k < A.nslot; ++k) {
        if (A.pidx[k] < 0) continue;
        for (int l = 0; l < B.nslot; ++l) {
          if (B.pidx[l] < 0) continue;
          rows_of[A.pidx[k]].push_back(B.pidx[l]);
          rows_of[B.pidx[l]].push_back(A.pidx[k]);
        }
      }
    }
    // tiles by free-column class (largest first), in image order within a
    // class: the Gram launches one column blocking per run of tiles, and
    // tiles that run side by side are neighbours sharing column images (in
    // the L2, and in the address translation caches).  A class is 16 columns
    // wide in the float path (its column blocks and tensor-core thresholds
    // are multiples of 16), 4 in the float64 path (blocks of 4 up to 32)
    std::vector<int> ncol_of(jwork.size());
    for (size_t t = 0; t < jwork.size(); ++t) {
      int nc = 0;
      for (int e = jwork[t].e0; e < jwork[t].e1; ++e)
        for (int k = 0; k < S[jt_src[e]].nslot; ++k) nc += S[jt_src[e]].pidx[k] >= 0;
      ncol_of[t] = nc;
    }
    std::vector<size_t> order(jwork.size());
    std::iota(order.begin(), order.end(), 0);
    auto cls = [&](size_t t) {
      const int nc = ncol_of[t];
      return f64 ? std::min((nc + 3) / 4, 9) : std::min((nc + 15) / 16, 9);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cls(a) > cls(b); });
    std::vector<TileWork> sorted(jwork.size());
    std::vector<int> sorted_nc(jwork.size());
    for (size_t t = 0; t < order.size(); ++t) {
      sorted[t] = jwork[order[t]];
      sorted_nc[t] = ncol_of[order[t]];
    }
    jwork.swap(sorted);
    tile_ncol.swap(sorted_nc);
  }
  std::vector<int64_t> row_ptr(n_params + 1, 0);
  std::vector<int32_t> col_idx;
  for (int p = 0; p < n_params; ++p) {
    auto& r = rows_of[p];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    col_idx.insert(col_idx.end(), r.begin(), r.end());
    row_ptr[p + 1] = (int64_t)col_idx.size();
    std::vector<int>().swap(r);
  }

  // ---- J^T W J plan: source pairs per tile, scratch blocks, CSR positions ----
  std::vector<int64_t> g_tab0(jwork.size() + 1, 0), g_tab, g_col_ptr;
  std::vector<GramCol> g_cols;
  std::vector<int> g_tabs;
  std::vector<GramPair> g_pairs;
  std::vector<GramRange> g_ranges;
  int g_n_light = 0;
  std::vector<int64_t> g_pos;
  int64_t g_scr = 0;
  {
    auto free_params = [&](int s, int* out) {
      int m = 0;
      for (int k = 0; k < S[s].nslot; ++k)
        if (S[s].pidx[k] >= 0) out[m++] = S[s].pidx[k];
      return m;
    };
    std::unordered_map<uint64_t, int> pid;
    std::vector<int> pA, pB, rank_of;
    g_tab.reserve(jwork.size() * 16);
    for (size_t t = 0; t < jwork.size(); ++t) {
      const TileWork& w = jwork[t];
      g_tab0[t] = (int64_t)g_tab.size();
      for (int a = w.e0; a < w.e1; ++a)
        for (int b = a; b < w.e1; ++b) {
          const uint64_t key = ((uint64_t)(uint32_t)jt_src[a] << 32) | (uint32_t)jt_src[b];
          auto it = pid.find(key);
          int id;
          if (it == pid.end()) {
            id = (int)g_pairs.size();
            pid.emplace(key, id);
            GramPair gp{};
            int tmp[MAX_SLOTS];
            gp.ma = free_params(jt_src[a], tmp);
            gp.mb = free_params(jt_src[b], tmp);
            g_pairs.push_back(gp);
            pA.push_back(jt_src[a]);
            pB.push_back(jt_src[b]);
          } else {
            id = it->second;
          }
          g_tab.push_back(id);
          rank_of.push_back(g_pairs[id].cnt++);
        }
    }
    g_tab0[jwork.size()] = (int64_t)g_tab.size();
    // float path: every tile's free columns in (source, slot) order, as the
    // tensor-core tile Gram reads them (it then skips building the list)
    if (!f64) {
      g_col_ptr.assign(jwork.size() + 1, 0);
      for (size_t t = 0; t < jwork.size(); ++t) {
        const TileWork& w = jwork[t];
        for (int e = w.e0; e < w.e1; ++e) {
          const SourceDev& sd = S[jt_src[e]];
          int nf = 0;
          for (int k = 0; k < sd.nslot; ++k) nf += sd.pidx[k] >= 0;
          const int* bx = sd.conv ? sd.sup : sd.box;
          const int bw = bx[3] - bx[2];
          const int64_t area = (int64_t)(bx[1] - bx[0]) * bw;
          auto clampt = [](int v) { return (uint32_t)(v < 0 ? 0 : (v > TILE ? TILE : v)); };
          const uint32_t bounds = clampt(bx[0] - w.r0) | (clampt(bx[1] - w.r0) << 8) | (clampt(bx[2] - w.c0) << 16) |
                                  (clampt(bx[3] - w.c0) << 24);
          const int off0 = (w.r0 - bx[0]) * bw + (w.c0 - bx[2]);
          const int64_t base = sd.conv ? sd.j_off : sd.d_off;
          int f = 0;
          for (int k = 0; k < sd.nslot; ++k) {
            if (sd.pidx[k] < 0) continue;
            g_cols.push_back(GramCol{base + k * area, off0, bw, bounds,
                                     ((e - w.e0) << 8) | (f << 4) | nf | (sd.conv ? GRAM_COL_CONV : 0)});
            ++f;
          }
        }
        g_col_ptr[t + 1] = (int64_t)g_cols.size();
      }
    }
    // light pairs first (tile-major blocks), heavy pairs after (entry-major)
    std::vector<int> new_id(g_pairs.size());
    {
      std::vector<GramPair> light, heavy;
      std::vector<int> lA, lB, hA, hB;
      for (size_t q = 0; q < g_pairs.size(); ++q) {
        const bool hv = g_pairs[q].cnt > GRAM_HEAVY_TILES;
        new_id[q] = (int)(hv ? heavy.size() : light.size());
        (hv ? heavy : light).push_back(g_pairs[q]);
        (hv ? hA : lA).push_back(pA[q]);
        (hv ? hB : lB).push_back(pB[q]);
      }
      g_n_light = (int)light.size();
      for (size_t q = 0; q < g_pairs.size(); ++q)
        if (g_pairs[q].cnt > GRAM_HEAVY_TILES) new_id[q] += g_n_light;
      light.insert(light.end(), heavy.begin(), heavy.end());
      lA.insert(lA.end(), hA.begin(), hA.end());
      lB.insert(lB.end(), hB.begin(), hB.end());
      g_pairs.swap(light);
      pA.swap(lA);
      pB.swap(lB);
    }
    for (auto& gp : g_pairs) {
      gp.base = g_scr;
      g_scr += (int64_t)gp.cnt * gp.ma * gp.mb;
    }
    g_tabs.resize(g_tab.size());
    for (size_t k = 0; k < g_tab.size(); ++k) {
      const int id = new_id[g_tab[k]];
      const GramPair& gp = g_pairs[id];
      const bool hv = id >= g_n_light;
      g_tab[k] = gp.base + (int64_t)rank_of[k] * (hv ? 1 : gp.ma * gp.mb);
      g_tabs[k] = hv ? gp.cnt : 1;
    }
    std::vector<int>().swap(rank_of);
    // column blocking per run of tiles (the tiles are sorted by column count);
    // the float path's threshold between the warp-MMA and the tcgen05 kernel
    // is chosen by timing once the plans are on the device
    g_ranges = gram_ranges_for(tile_ncol, f64, GRAM_TC_MIN_DEFAULT);
    c->h_tile_ncol = tile_ncol;
    // CSR positions of every block entry and its mirror; entries below the
    // diagonal of a source's own block are left out (their mirror is there)
    auto find = [&](int r, int cc) -> int64_t {
      auto first = col_idx.begin() + row_ptr[r], last = col_idx.begin() + row_ptr[r + 1];
      auto it = std::lower_bound(first, last, cc);
      return (it != last && *it == cc) ? (int64_t)(it - col_idx.begin()) : -2;
    };
    std::vector<uint8_t> hits(col_idx.size(), 0);
    for (size_t q = 0; q < g_pairs.size(); ++q) {
      GramPair& gp = g_pairs[q];
      gp.pos = (int64_t)g_pos.size();
      int fa[MAX_SLOTS], fb[MAX_SLOTS];
      free_params(pA[q], fa);
      free_params(pB[q], fb);
      for (int a = 0; a < gp.ma; ++a)
        for (int b = 0; b < gp.mb; ++b) {
          int64_t ab = -1, ba = -1;
          if (!(pA[q] == pB[q] && b < a)) {
            ab = find(fa[a], fb[b]);
            if (!(pA[q] == pB[q] && a == b)) ba = find(fb[b], fa[a]);
          }
          if (ab == -2 || ba == -2) return fail(c, AP_ERR_ARG, "internal: J^T W J entry outside its sparsity pattern");
          for (int64_t e : {ab, ba})
            if (e >= 0 && hits[e] < 255) ++hits[e];
          g_pos.push_back(ab);
          g_pos.push_back(ba);
        }
    }
    for (auto& gp : g_pairs) {
      gp.excl = 1;
      for (int64_t k = gp.pos; k < gp.pos + 2 * (int64_t)gp.ma * gp.mb; ++k)
        if (g_pos[k] >= 0 && hits[g_pos[k]] > 1) gp.excl = 0;
    }
  }

  // ---- parameter groups ----
  std::vector<int> param_group(n_params, -1), owner(n_params, -1);
  for (int s = 0; s < n_src; ++s)
    for (int k = 0; k < S[s].nslot; ++k) {
      const int p = S[s].pidx[k];
      if (p >= 0 && param_group[p] < 0) {
        param_group[p] = I[S[s].image].group;
        owner[p] = s;
      }
    }
  // objects: the sources that share parameters (union of sources through
  // their common theta indices); a group lists its parameters object by
  // object (objects in the order of their first parameter, theta order
  // within), so that each object's parameters form preconditioner blocks
  std::vector<int> uf(n_src);
  for (int s = 0; s < n_src; ++s) uf[s] = s;
  auto root = [&](int s) {
    while (uf[s] != s) s = uf[s] = uf[uf[s]];
    return s;
  };
  {
    std::vector<int> first_src(n_params, -1);
    for (int s = 0; s < n_src; ++s)
      for (int k = 0; k < S[s].nslot; ++k) {
        const int p = S[s].pidx[k];
        if (p < 0) continue;
        if (first_src[p] < 0) first_src[p] = s;
        else uf[root(s)] = root(first_src[p]);
      }
  }
  std::vector<int> obj_of(n_params, -1), obj_rank(n_src, -1);
  int n_obj = 0;
  for (int p = 0; p < n_params; ++p)
    if (owner[p] >= 0) {
      const int o = root(owner[p]);
      if (obj_rank[o] < 0) obj_rank[o] = n_obj++;
      obj_of[p] = obj_rank[o];
    }
  std::vector<std::vector<int>> gplist(n_groups);
  for (int p = 0; p < n_params; ++p)
    if (param_group[p] >= 0) gplist[param_group[p]].push_back(p);
  for (auto& l : gplist)
    std::stable_sort(l.begin(), l.end(), [&](int a, int b) { return obj_of[a] < obj_of[b]; });
  std::vector<GroupDev> groups(n_groups);
  std::vector<int> gparams, plocal(n_params, -1), blk_ptr;
  int max_dense = 1, max_pcg = 1, any_dense = 0, any_pcg = 0, any_grid = 0;
  std::vector<int> cluster_groups;
  int64_t nblk_total = 0;
  int groups_pcg = 0;
  for (int g = 0; g < n_groups; ++g) {
    GroupDev G{};
    G.n = (int)gplist[g].size();
    G.p0 = (int)gparams.size();
    G.dense = G.n <= 64 ? 1 : 0;
    groups_pcg += G.dense != 1;
    G.b0 = (int)blk_ptr.size();
    for (int k = 0; k < G.n; ++k) {
      plocal[gplist[g][k]] = k;
      gparams.push_back(gplist[g][k]);
    }
    // preconditioner blocks: the parameters of one object, <= PCG_BLK
    int nb = 0;
    for (int k = 0; k < G.n;) {
      int e = k + 1;
      while (e < G.n && e - k < PCG_BLK && obj_of[gplist[g][e]] == obj_of[gplist[g][k]]) ++e;
      blk_ptr.push_back(k);
      ++nb;
      k = e;
    }
    blk_ptr.push_back(G.n);  // closing pointer of this group's list
    G.nblk = nb;
    nblk_total += nb;
    groups[g] = G;
  }
  // solve plans: group-local column of every CSR entry, diagonal positions,
  // and the CSR positions of every preconditioner block's entries
  std::vector<int32_t> lcol(col_idx.size());
  std::vector<int64_t> dpos(n_params, -1);
  for (int p = 0; p < n_params; ++p)
    for (int64_t e = row_ptr[p]; e < row_ptr[p + 1]; ++e) {
      lcol[e] = plocal[col_idx[e]];
      if (col_idx[e] == p) dpos[p] = e;
    }
  std::vector<int64_t> bpos(blk_ptr.size() * PCG_BLK2, -1);
  for (int g = 0; g < n_groups; ++g) {
    const GroupDev& G = groups[g];
    for (int b = 0; b < G.nblk; ++b) {
      const int s0 = blk_ptr[G.b0 + b], m = blk_ptr[G.b0 + b + 1] - s0;
      for (int a = 0; a < m; ++a) {
        const int pr = gparams[G.p0 + s0 + a];
        for (int cc = 0; cc < m; ++cc) {
          const int pc = gparams[G.p0 + s0 + cc];
          auto first = col_idx.begin() + row_ptr[pr], last = col_idx.begin() + row_ptr[pr + 1];
          auto it = std::lower_bound(first, last, pc);
          if (it != last && *it == pc) bpos[(size_t)(G.b0 + b) * PCG_BLK2 + a * PCG_BLK + cc] = it - col_idx.begin();
        }
      }
    }
  }
  // SpMV chunks, row-contiguous in group order: rows of up to DIST_WARP_ROW
  // entries in thread chunks of DIST_CHUNK, longer rows in warp chunks of at
  // least DIST_WCHUNK (at most DIST_MAX_PARTS partials per row even for the
  // sky's dense rows)
  std::vector<int64_t> ch_e0, ch_e1;
  std::vector<int> ch_row(gparams.size() + 1, 0), ch_lrow, ch_warp;
  for (int g = 0; g < n_groups; ++g) {
    const GroupDev& G = groups[g];
    for (int i = 0; i < G.n; ++i) {
      const int pr = gparams[G.p0 + i];
      const int64_t len = row_ptr[pr + 1] - row_ptr[pr];
      // long rows: warp chunks of DIST_WCHUNK entries, longer ones for rows
      // so long that they would exceed DIST_MAX_PARTS partials
      const int step = len <= DIST_WARP_ROW ? DIST_CHUNK
                                            : (int)std::max<int64_t>(DIST_WCHUNK, (len + DIST_MAX_PARTS - 1) / DIST_MAX_PARTS);
      for (int64_t e = row_ptr[pr]; e < row_ptr[pr + 1]; e += step) {
        ch_e0.push_back(e);
        ch_e1.push_back(std::min<int64_t>(e + step, row_ptr[pr + 1]));
        ch_lrow.push_back(i);
        ch_warp.push_back(len > DIST_WARP_ROW);
      }
      ch_row[G.p0 + i + 1] = (int)ch_e0.size();
    }
  }
  // Solver of each group.  Up to 64 parameters: dense Cholesky in one CTA.
  // Larger groups use block-Jacobi PCG, whose cost is the float64 SpMV of the
  // group's J^T W J block.  With enough such groups to fill the GPU, each
  // runs in one CTA on one SM's float64 pipe (one-CTA PCG, up to
  // PCG_ONE_CTA_MAX parameters).  Otherwise a group is spread over the CTAs
  // of a thread-block cluster (up to CLUSTER_N_MAX parameters and
  // CLUSTER_NNZ_MAX entries, with its state in shared memory), or else over
  // every SM (cooperative grid-wide launch).
  std::vector<int> dist_own_blk, dist_own_ptr(n_groups, 0), dist_owner(ch_e0.size(), 0), dist_dst(ch_e0.size(), 0);
  std::vector<int> dist_loff(blk_ptr.size(), 0);
  std::vector<int> dist_tlist, dist_tptr(n_groups + 1, 0), dist_wlist, dist_wptr(n_groups + 1, 0);
  DistLaunch dl;
  {
    int sms = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->opt.device));
    const int cs = cluster_pcg_size(c->opt.device, CLUSTER_SMEM_MAX);
    const bool fill = (int64_t)groups_pcg * 8 > 2 * (int64_t)sms;
    std::vector<int64_t> gnnz(n_groups, 0);
    for (int p = 0; p < n_params; ++p)
      if (param_group[p] >= 0) gnnz[param_group[p]] += row_ptr[p + 1] - row_ptr[p];
    for (int g = 0; g < n_groups; ++g) {
      GroupDev& G = groups[g];
      if (G.dense == 1) continue;
      if (fill && G.n <= PCG_ONE_CTA_MAX) G.dense = 0;
      else if (cs > 0 && gnnz[g] <= CLUSTER_NNZ_MAX && G.n <= CLUSTER_N_MAX) G.dense = 3;
      else G.dense = 2;
    }
    // contiguous runs of blocks per CTA, balanced by rows; the CTA's
    // extents; chunk owners and partial offsets; packed block-inverse offsets
    auto partition = [&](int g, int nct, DistSmem& ext, bool cluster) {
      const GroupDev& G = groups[g];
      const int* bp = blk_ptr.data() + G.b0;
      dist_own_ptr[g] = (int)dist_own_blk.size();
      const size_t base = dist_own_blk.size();
      dist_own_blk.resize(base + nct + 1);
      int b = 0;
      for (int k = 0; k <= nct; ++k) {
        const int64_t target = (int64_t)G.n * k / nct;
        while (b < G.nblk && bp[b] < target) ++b;
        dist_own_blk[base + k] = k == nct ? G.nblk : b;
      }
      for (int k = 0; k < nct; ++k) {
        const int bb0 = dist_own_blk[base + k], bb1 = dist_own_blk[base + k + 1];
        const int r0 = bp[bb0], r1 = bp[bb1];
        int lo_ = 0;
        for (int q = bb0; q < bb1; ++q) {
          dist_loff[G.b0 + q] = lo_;
          const int m = bp[q + 1] - bp[q];
          lo_ += m * m;
        }
        const int c0 = ch_row[G.p0 + r0], c1 = ch_row[G.p0 + r1];
        for (int ch = c0; ch < c1; ++ch) {
          dist_owner[ch] = k;
          dist_dst[ch] = ch - c0;
        }
        ext.nr = std::max(ext.nr, r1 - r0);
        ext.nb = std::max(ext.nb, lo_);
        ext.np = std::max(ext.np, cluster ? c1 - c0 : 0);
        ext.nu = std::max(ext.nu, cluster ? G.n : r1 - r0);
      }
    };
    // cluster groups: shrink to what fits CLUSTER_SMEM_MAX (the largest go grid-wide)
    for (;;) {
      DistSmem ext{};
      int biggest = -1;
      dist_own_blk.clear();
      for (int g = 0; g < n_groups; ++g)
        if (groups[g].dense == 3) {
          partition(g, cs, ext, true);
          if (biggest < 0 || groups[g].n > groups[biggest].n) biggest = g;
        }
      if (biggest < 0 || dist_smem_bytes(ext, cs, true) <= CLUSTER_SMEM_MAX) {
        dl.cluster_sz = ext;
        break;
      }
      groups[biggest].dense = 2;
    }
    // grid groups: two CTAs per SM if they fit, else one
    bool any_g = false;
    for (int g = 0; g < n_groups; ++g) any_g |= groups[g].dense == 2;
    if (any_g) {
      const size_t keep = dist_own_blk.size();
      for (int nct = 2 * sms; nct >= sms; nct -= sms) {
        DistSmem ext{};
        dist_own_blk.resize(keep);
        for (int g = 0; g < n_groups; ++g)
          if (groups[g].dense == 2) partition(g, nct, ext, false);
        const int fit = grid_pcg_blocks(c->opt.device, dist_smem_bytes(ext, nct, false));
        if (fit >= nct) {
          dl.grid_blocks = nct;
          dl.grid_sz = ext;
          break;
        }
      }
      if (dl.grid_blocks == 0) return fail(c, AP_ERR_CUDA, "grid-wide PCG cannot be made co-resident");
    }
    dl.cluster_size = cs;
    for (int g = 0; g < n_groups; ++g) {
      GroupDev& G = groups[g];
      if (G.dense == 1) { any_dense = 1; max_dense = std::max(max_dense, G.n); }
      if (G.dense == 0) { any_pcg = 1; max_pcg = std::max(max_pcg, G.n); }
      if (G.dense == 2) any_grid = 1;
      if (G.dense == 3) cluster_groups.push_back(g);
      for (int ch = ch_row[G.p0]; ch < ch_row[G.p0 + G.n]; ++ch)
        (ch_warp[ch] ? dist_wlist : dist_tlist).push_back(ch);
      dist_tptr[g + 1] = (int)dist_tlist.size();
      dist_wptr[g + 1] = (int)dist_wlist.size();
    }
    dl.n_cluster_groups = (int)cluster_groups.size();
  }
  std::vector<double> lo, hi;
  param_bounds(S, n_params, lo, hi);

  // ---- device allocation and upload ----
  int rc;
  for (int i = 0; i < n_img; ++i) {
    ImageDev& m = I[i];
    if (m.has_gal) {
      if ((rc = dev_alloc(c, &m.gal, (size_t)m.Hp * m.Wp * tsz))) return rc;
      if ((rc = dev_alloc(c, &m.adj, (size_t)m.Hp * m.Wp * tsz))) return rc;
    }
    if (m.live_src >= 0) {
      if ((rc = dev_alloc(c, &m.live_cols, (size_t)2 * m.H * m.W * tsz))) return rc;
      if ((rc = dev_alloc(c, &m.dpsf_flip, (size_t)4 * m.K * m.K4 * tsz))) return rc;
    }
    if (m.K > 0) {
      // (every image with a PSF: the convolution and the PSF stars read it)
      // normalised PSF (float64 sum), padded rows of K4, plain and flipped
      // (a live PSF starts as a centred delta: every evaluation renders it)
      std::vector<float> hp((size_t)m.K * m.K, 0.0f);
      if (imgs[i].psf_live)
        hp[(size_t)m.h * m.K + m.h] = 1.0f;
      else
        CUDA_TRY(c, cudaMemcpy(hp.data(), imgs[i].psf_dev, hp.size() * sizeof(float), cudaMemcpyDeviceToHost));
      double sum = 0.0;
      for (float v : hp) {
        if (!std::isfinite(v)) return fail(c, AP_ERR_NONFINITE, "image " + std::to_string(i) + ": non-finite PSF");
        sum += v;
      }
      if (!(sum > 0.0)) return fail(c, AP_ERR_ARG, "image " + std::to_string(i) + ": PSF sums to <= 0");
      std::vector<double> pn((size_t)m.K * m.K4, 0.0), pf((size_t)m.K * m.K4, 0.0);
      for (int ty = 0; ty < m.K; ++ty)
        for (int tx = 0; tx < m.K; ++tx) {
          const double v = hp[(size_t)ty * m.K + tx] / sum;
          pn[(size_t)ty * m.K4 + tx] = v;
          pf[(size_t)(m.K - 1 - ty) * m.K4 + (m.K - 1 - tx)] = v;
        }
      if ((rc = dev_alloc(c, &m.psf_norm, pn.size() * tsz))) return rc;
      if ((rc = dev_alloc(c, &m.psf_flip, pf.size() * tsz))) return rc;
      if (f64) {
        CUDA_TRY(c, cudaMemcpy(m.psf_norm, pn.data(), pn.size() * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(m.psf_flip, pf.data(), pf.size() * 8, cudaMemcpyHostToDevice));
      } else {
        std::vector<float> a(pn.begin(), pn.end()), b(pf.begin(), pf.end());
        CUDA_TRY(c, cudaMemcpy(m.psf_norm, a.data(), a.size() * 4, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(m.psf_flip, b.data(), b.size() * 4, cudaMemcpyHostToDevice));
        // spectra of the padded PSF for the FFT mode of the Jacobian columns
        // (none for a live PSF: the direct mode convolves with the current one)
        for (int N : {64, 128}) {
          if (m.K > (N == 64 ? FFT_MAX_K64 : FFT_MAX_K128) || imgs[i].psf_live) continue;
          float2*& tw = N == 64 ? c->d_tw64 : c->d_tw128;
          if (!tw && (rc = upload(c, &tw, fft_twiddles(N)))) return rc;
          float2* spec;
          if ((rc = dev_alloc(c, (void**)&spec, (size_t)N * N * sizeof(float2)))) return rc;
          launch_psf_spectrum(N, (const float*)m.psf_norm, m.K, m.K4, tw, spec, 0);
          CUDA_TRY(c, cudaGetLastError());
          (N == 64 ? m.spec64 : m.spec128) = spec;
        }
      }
    }
    if ((rc = dev_alloc(c, &m.unc, (size_t)m.H * m.W * tsz))) return rc;
    if ((rc = dev_alloc(c, &m.wr, (size_t)m.H * m.W * tsz))) return rc;
    if ((rc = dev_alloc(c, &m.wr_trial, (size_t)m.H * m.W * tsz))) return rc;
  }
  if ((rc = upload(c, &c->d_live_imgs, live_imgs))) return rc;
  c->n_live = (int)live_imgs.size();
  c->n_src_user = n_src_user;
  c->max_live_tiles = 0;
  for (int i : live_imgs)
    c->max_live_tiles = std::max(c->max_live_tiles, ((I[i].H + 15) / 16) * ((I[i].W + 15) / 16));
  if ((rc = upload(c, &c->d_imgs, I))) return rc;
  if ((rc = upload(c, &c->d_srcs, S))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_bn_memo, (size_t)std::max(n_src, 1) * 8 * sizeof(double)))) return rc;
  CUDA_TRY(c, cudaMemset(c->d_bn_memo, 0xff, (size_t)std::max(n_src, 1) * 8 * sizeof(double)));   // NaN: no entry
  const size_t par_bytes = f64 ? sizeof(SrcPar<double>) : sizeof(SrcPar<float>);
  if ((rc = dev_alloc(c, &c->d_par, (size_t)std::max(n_src, 1) * par_bytes))) return rc;
  if ((rc = dev_alloc(c, &c->d_par_trial, (size_t)std::max(n_src, 1) * par_bytes))) return rc;
  {
    // what an accepted group copies from its trial state: each source's
    // record, then each image's w r in runs of STATE_CHUNK_WORDS words
    static_assert(sizeof(SrcPar<float>) % 4 == 0 && sizeof(SrcPar<double>) % 4 == 0, "records of whole words");
    std::vector<StateChunk> ch;
    for (int s = 0; s < n_src; ++s)
      ch.push_back(StateChunk{(const uint32_t*)((const char*)c->d_par_trial + s * par_bytes),
                              (uint32_t*)((char*)c->d_par + s * par_bytes), (int)(par_bytes / 4),
                              I[S[s].image].group});
    for (const auto& m : I) {
      const int64_t words = (int64_t)m.H * m.W * (int64_t)tsz / 4;
      for (int64_t w0 = 0; w0 < words; w0 += STATE_CHUNK_WORDS)
        ch.push_back(StateChunk{(const uint32_t*)m.wr_trial + w0, (uint32_t*)m.wr + w0,
                                (int)std::min<int64_t>(STATE_CHUNK_WORDS, words - w0), m.group});
    }
    c->n_state_chunks = (int)ch.size();
    if ((rc = upload(c, &c->d_state_chunks, ch))) return rc;
  }
  if ((rc = upload(c, &c->d_rwork, rwork))) return rc;
  if ((rc = upload(c, &c->d_tile_src, tile_src))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_grad_partial, std::max<size_t>(tile_src.size(), 1) * MAX_SLOTS * sizeof(double))))
    return rc;
  if ((rc = upload(c, &c->d_gc_ptr, gc_ptr))) return rc;
  if ((rc = upload(c, &c->d_gc_idx, gc_idx))) return rc;
  for (int v = 0; v < N_CONV_VARIANTS; ++v) {
    if ((rc = upload(c, &c->v_fwork[v], v_f[v]))) return rc;
    if ((rc = upload(c, &c->v_awork[v], v_a[v]))) return rc;
    if ((rc = upload(c, &c->v_grp_ptr[v], v_gp[v]))) return rc;
    if ((rc = upload(c, &c->v_grp_idx[v], v_gi[v]))) return rc;
    c->v_nf[v] = (int)v_f[v].size();
    c->v_na[v] = (int)v_a[v].size();
    c->v_frange[v] = v_fr[v];
    c->v_arange[v] = v_ar[v];
  }
  if ((rc = dev_alloc(c, (void**)&c->d_chi2_partial, max_nf * sizeof(double)))) return rc;
  if ((rc = upload(c, &c->d_jwork, jwork))) return rc;
  if ((rc = upload(c, &c->d_jt_src, jt_src))) return rc;
  {
    const int64_t *d_t0, *d_tab, *d_pos;
    const int* d_tabs;
    const GramPair* d_gp;
    if ((rc = upload(c, &d_t0, g_tab0))) return rc;
    if ((rc = upload(c, &d_tab, g_tab))) return rc;
    if ((rc = upload(c, &d_tabs, g_tabs))) return rc;
    if ((rc = upload(c, &d_pos, g_pos))) return rc;
    if ((rc = upload(c, &d_gp, g_pairs))) return rc;
    double* d_scr;
    if ((rc = dev_alloc(c, (void**)&d_scr, (size_t)std::max<int64_t>(g_scr, 1) * sizeof(double)))) return rc;
    // work list of the heavy-pair reduction: one item per stored entry, the
    // entries spanning more than GRAM_CTA_TILES tiles first (a CTA each)
    std::vector<int> items, warp_items;
    for (int q = g_n_light; q < (int)g_pairs.size(); ++q) {
      const GramPair& gp = g_pairs[q];
      for (int e = 0; e < gp.ma * gp.mb; ++e)
        if (g_pos[gp.pos + 2 * e] >= 0)
          (gp.cnt > GRAM_CTA_TILES ? items : warp_items).push_back(((q - g_n_light) << 6) | e);
    }
    const int n_heavy_cta = (int)items.size();
    items.insert(items.end(), warp_items.begin(), warp_items.end());
    const int* d_items;
    if ((rc = upload(c, &d_items, items))) return rc;
    const int64_t* d_col_ptr = nullptr;
    const GramCol* d_cols = nullptr;
    if (!f64) {
      if ((rc = upload(c, &d_col_ptr, g_col_ptr))) return rc;
      if ((rc = upload(c, &d_cols, g_cols))) return rc;
    }
    std::vector<GramCol>().swap(g_cols);
    c->gplan = GramPlan{d_t0, d_tab, d_tabs, d_scr, d_gp, d_pos, g_n_light, (int)g_pairs.size() - g_n_light,
                        d_items, (int)items.size(), n_heavy_cta, d_col_ptr, d_cols};
    c->gram_ranges = g_ranges;
  }
  if ((rc = dev_alloc(c, &c->d_dbuf, (size_t)std::max<int64_t>(dbuf_elems, 1) * tsz))) return rc;
  if ((rc = dev_alloc(c, &c->d_jbuf, (size_t)std::max<int64_t>(jbuf_elems, 1) * tsz))) return rc;
  if ((rc = upload(c, &c->d_row_ptr, row_ptr))) return rc;
  if ((rc = upload(c, &c->d_col_idx, col_idx))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_vals, std::max<size_t>(col_idx.size(), 1) * sizeof(double)))) return rc;
  if ((rc = upload(c, &c->d_groups, groups))) return rc;
  if ((rc = upload(c, &c->d_gparams, gparams))) return rc;
  if ((rc = upload(c, &c->d_plocal, plocal))) return rc;
  if ((rc = upload(c, &c->d_blk_ptr, blk_ptr))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_work, std::max<size_t>(gparams.size(), 1) * 6 * sizeof(double)))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_blk_work, (size_t)std::max<int64_t>(nblk_total + n_groups, 1) * PCG_BLK2 * sizeof(double))))
    return rc;
  if ((rc = upload(c, &c->d_param_group, param_group))) return rc;
  if ((rc = upload(c, &c->d_lo, lo))) return rc;
  if ((rc = upload(c, &c->d_hi, hi))) return rc;
  const size_t P = (size_t)std::max(n_params, 1), G = (size_t)std::max(n_groups, 1);
  double** vecs[] = {&c->d_theta, &c->d_trial, &c->d_delta, &c->d_jtwr, &c->d_grad};
  for (double** v : vecs)
    if ((rc = dev_alloc(c, (void**)v, P * sizeof(double)))) return rc;
  double** gv[] = {&c->d_chi2, &c->d_chi2_trial, &c->d_chi2_state, &c->d_lambda};
  for (double** v : gv)
    if ((rc = dev_alloc(c, (void**)v, G * sizeof(double)))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_accepted, G * sizeof(int)))) return rc;
  CUDA_TRY(c, cudaMemset(c->d_accepted, 0, G * sizeof(int)));
  if ((rc = dev_alloc(c, (void**)&c->d_fwd_valid, G * sizeof(int)))) return rc;
  CUDA_TRY(c, cudaMemset(c->d_fwd_valid, 0, G * sizeof(int)));
  if ((rc = dev_alloc(c, (void**)&c->d_cg_iters, G * sizeof(int)))) return rc;
  CUDA_TRY(c, cudaMemset(c->d_cg_iters, 0, G * sizeof(int)));
  c->dl = dl;
  {
    SolvePlan& sp = c->sp;
    int32_t* d_lcol;
    int64_t* d_dpos;
    int64_t* d_bpos;
    if ((rc = upload(c, &d_lcol, lcol))) return rc;
    if ((rc = upload(c, &d_dpos, dpos))) return rc;
    if ((rc = upload(c, &d_bpos, bpos))) return rc;
    if ((rc = dev_alloc(c, (void**)&sp.part, 8 * (size_t)std::max(dl.grid_blocks, 1) * sizeof(double)))) return rc;
    sp.groups = c->d_groups;
    sp.gparams = c->d_gparams;
    sp.plocal = c->d_plocal;
    sp.blk_ptr = c->d_blk_ptr;
    sp.row_ptr = c->d_row_ptr;
    sp.col_idx = c->d_col_idx;
    sp.lcol = d_lcol;
    sp.dpos = d_dpos;
    sp.bpos = d_bpos;
    sp.work = c->d_work;
    sp.blk_work = c->d_blk_work;
    sp.iters = c->d_cg_iters;
    int64_t* d_ch0;
    int64_t* d_ch1;
    int* d_chr;
    int* d_clg;
    if ((rc = upload(c, &d_ch0, ch_e0))) return rc;
    if ((rc = upload(c, &d_ch1, ch_e1))) return rc;
    if ((rc = upload(c, &d_chr, ch_row))) return rc;
    if ((rc = upload(c, &d_clg, cluster_groups))) return rc;
    if ((rc = dev_alloc(c, (void**)&sp.ch_part, std::max<size_t>(ch_e0.size(), 1) * sizeof(double)))) return rc;
    sp.ch_e0 = d_ch0;
    sp.ch_e1 = d_ch1;
    sp.ch_row = d_chr;
    sp.cluster_groups = d_clg;
    DistPlan& dp = sp.dist;
    const int *d_lrow, *d_tl, *d_tp, *d_wl, *d_wp, *d_own, *d_dst, *d_ob, *d_op, *d_loff;
    if ((rc = upload(c, &d_lrow, ch_lrow))) return rc;
    if ((rc = upload(c, &d_tl, dist_tlist))) return rc;
    if ((rc = upload(c, &d_tp, dist_tptr))) return rc;
    if ((rc = upload(c, &d_wl, dist_wlist))) return rc;
    if ((rc = upload(c, &d_wp, dist_wptr))) return rc;
    if ((rc = upload(c, &d_own, dist_owner))) return rc;
    if ((rc = upload(c, &d_dst, dist_dst))) return rc;
    if ((rc = upload(c, &d_ob, dist_own_blk))) return rc;
    if ((rc = upload(c, &d_op, dist_own_ptr))) return rc;
    if ((rc = upload(c, &d_loff, dist_loff))) return rc;
    dp = DistPlan{d_ch0, d_ch1, d_lrow, d_chr, d_tl, d_tp, d_wl, d_wp, d_own, d_dst, d_ob, d_op, d_loff, d_lcol,
                  sp.ch_part};
  }

  if ((rc = dev_alloc(c, (void**)&c->d_log, G * 4 * sizeof(double)))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_status, sizeof(int)))) return rc;
  if ((rc = dev_alloc(c, (void**)&c->d_model_ptrs, (size_t)n_img * sizeof(void*)))) return rc;
  CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));

  int vok[N_CONV_VARIANTS] = {};
  if (f64) {
    configure_conv<double>(Kmax, vok);
    configure_gram<double>(0);

  } else {
    configure_conv<float>(Kmax, vok);
    configure_gram<float>(0);
    configure_gram_tc();

  }
  configure_solve();
  if (!live_imgs.empty() && !configure_live(Kmax, f64 ? 1 : 0))
    return fail(c, AP_ERR_ARG, "the live PSF's column kernel does not fit the PSF size in shared memory");
  c->Kmax = Kmax;
  c->max_dense_n = max_dense;
  c->max_pcg_n = max_pcg;
  CUDA_TRY(c, cudaGetLastError());
  // zero the scratch layers once (the autotuner runs on them)
  for (auto& m : I) {
    if (m.gal) CUDA_TRY(c, cudaMemset(m.gal, 0, (size_t)m.Hp * m.Wp * tsz));
    if (m.adj) CUDA_TRY(c, cudaMemset(m.adj, 0, (size_t)m.Hp * m.Wp * tsz));
    CUDA_TRY(c, cudaMemset(m.unc, 0, (size_t)m.H * m.W * tsz));
    CUDA_TRY(c, cudaMemset(m.wr, 0, (size_t)m.H * m.W * tsz));
    CUDA_TRY(c, cudaMemset(m.wr_trial, 0, (size_t)m.H * m.W * tsz));
  }
  c->d_imgs = c->d_imgs;  // (uploaded above)
  // ---- autotune the correlation tile shape: time forward + adjoint of every
  // fitting variant on this problem's images, keep the fastest ----
  int variant = -1;
  for (int v = 0; v < N_CONV_VARIANTS; ++v) c->conv_ms[v] = -1.0;
  if (c->opt.conv_variant > 0) {
    variant = c->opt.conv_variant - 1;
    if (variant >= N_CONV_VARIANTS) return fail(c, AP_ERR_ARG, "no such convolution tile variant");
    if (!vok[variant]) return fail(c, AP_ERR_ARG, "the forced convolution tile variant does not fit the PSF");
  } else if (c->opt.tile_w > 0 || c->opt.tile_h > 0) {
    for (int v = 0; v < N_CONV_VARIANTS; ++v)
      if (vok[v] && conv_tile_w(v) == c->opt.tile_w && conv_tile_h(v) == c->opt.tile_h) variant = v;
    if (variant < 0) return fail(c, AP_ERR_ARG, "no convolution tile variant of the requested shape");
  } else {
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    double best = 1e300;
    for (int v = 0; v < N_CONV_VARIANTS; ++v) {
      c->conv_ms[v] = -1.0;
      if (!vok[v]) continue;
      double tot = 0.0;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        const auto& fr = c->v_frange[v];
        const auto& ar = c->v_arange[v];
        if (f64) {
          launch_forward_conv<double>(v, c->v_fwork[v], fr.data(), (int)fr.size(), c->d_imgs, c->d_chi2_partial, nullptr,
                                      nullptr, 0, c->d_status, Kmax, st);
          launch_adjoint_conv<double>(v, c->v_awork[v], ar.data(), (int)ar.size(), c->d_imgs, Kmax, st);
        } else {
          launch_forward_conv<float>(v, c->v_fwork[v], fr.data(), (int)fr.size(), c->d_imgs, c->d_chi2_partial, nullptr,
                                     nullptr, 0, c->d_status, Kmax, st);
          launch_adjoint_conv<float>(v, c->v_awork[v], ar.data(), (int)ar.size(), c->d_imgs, Kmax, st);
        }
        cudaEventRecord(e1, st);
        CUDA_TRY(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;   // first repetition warms up
      }
      c->conv_ms[v] = tot / 3.0;
      if (tot < best) { best = tot; variant = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
    if (variant < 0) return fail(c, AP_ERR_ARG, "no convolution tile variant fits the PSF size in shared memory");
  }
  c->conv_variant = variant;
  c->d_fwork = c->v_fwork[variant];
  c->n_fwork = c->v_nf[variant];
  c->d_awork = c->v_awork[variant];
  c->n_awork = c->v_na[variant];
  c->d_grp_ptr = c->v_grp_ptr[variant];
  c->d_grp_idx = c->v_grp_idx[variant];
  c->frange = c->v_frange[variant];
  c->arange = c->v_arange[variant];
  {
    const int TW = conv_tile_w(variant), TH = conv_tile_h(variant);
    std::vector<JcolWork> jc;
    for (int s = 0; s < n_src; ++s) {
      const SourceDev& m = S[s];
      if (m.j_off < 0) continue;
      for (int r = m.sup[0]; r < m.sup[1]; r += TH)
        for (int cc = m.sup[2]; cc < m.sup[3]; cc += TW) jc.push_back(JcolWork{s, r, cc});
    }
    std::stable_sort(jc.begin(), jc.end(), [&](const JcolWork& a, const JcolWork& b) {
      return img_nc[S[a.src].image] < img_nc[S[b.src].image];
    });
    c->jcrange.clear();
    for (int k = 0; k < (int)jc.size(); ++k) {
      const int nc = img_nc[S[jc[k].src].image];
      if (c->jcrange.empty() || c->jcrange.back().nc != nc) c->jcrange.push_back(ConvRange{nc, k, 0});
      c->jcrange.back().count++;
    }
    if ((rc = upload(c, &c->d_jcwork, jc))) return rc;
    c->n_jcwork = (int)jc.size();
  }
  // FFT mode of the Jacobian columns: one work item per source, free slot
  // and output block; kept when it beats the direct correlation on this
  // problem (timed here, derivative buffer zeroed)
  if (!f64 && c->n_jcwork > 0) {
    std::vector<JcolFftWork> jf[2];
    bool all = true;
    for (int s = 0; s < n_src; ++s) {
      const SourceDev& m = S[s];
      if (m.j_off < 0) continue;
      const ImageDev& im = I[m.image];
      if (!im.spec64 && !im.spec128) { all = false; continue; }
      // block size with the smaller estimated cost: blocks x N^2 log2 N
      int N = 0;
      double best_cost = 0.0;
      for (int n : {64, 128}) {
        if (!(n == 64 ? im.spec64 : im.spec128)) continue;
        const int Bn = n - im.K + 1;
        const double nb = (double)((m.sup[1] - m.sup[0] + Bn - 1) / Bn) * ((m.sup[3] - m.sup[2] + Bn - 1) / Bn);
        const double cost = nb * n * n * (n == 64 ? 6.0 : 7.0);
        if (N == 0 || cost < best_cost) { N = n; best_cost = cost; }
      }
      const int B = N - im.K + 1;
      int fs[MAX_SLOTS], nf = 0;
      for (int k = 0; k < m.nslot; ++k)
        if (m.pidx[k] >= 0) fs[nf++] = k;
      for (int a = 0; a < nf; ++a)
        for (int r = m.sup[0]; r < m.sup[1]; r += B)
          for (int cc = m.sup[2]; cc < m.sup[3]; cc += B)
            jf[N == 128].push_back(JcolFftWork{s, fs[a], r - m.box[0], cc - m.box[2]});
    }
    if (all) {
      c->n_jf64 = (int)jf[0].size();
      c->n_jf128 = (int)jf[1].size();
      jf[0].insert(jf[0].end(), jf[1].begin(), jf[1].end());
      if ((rc = upload(c, &c->d_jfwork, jf[0]))) return rc;
      CUDA_TRY(c, cudaMemset(c->d_dbuf, 0, (size_t)std::max<int64_t>(dbuf_elems, 1) * tsz));
      cudaEvent_t e0, e1;
      CUDA_TRY(c, cudaEventCreate(&e0));
      CUDA_TRY(c, cudaEventCreate(&e1));
      double t[2] = {0.0, 0.0};
      for (int rep = 0; rep < 4; ++rep)
        for (int mode = 0; mode < 2; ++mode) {
          cudaEventRecord(e0, st);
          if (mode == 0)
            launch_jcol<float>(variant, c->d_jcwork, c->jcrange.data(), (int)c->jcrange.size(), c->d_srcs, c->d_imgs,
                               (const float*)c->d_dbuf, (float*)c->d_jbuf, Kmax, st);
          else
            launch_jcol_fft_all(c, st);
          cudaEventRecord(e1, st);
          CUDA_TRY(c, cudaEventSynchronize(e1));
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) t[mode] += ms / 3.0;
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      CUDA_TRY(c, cudaGetLastError());
      c->jcol_ms_direct = t[0];
      c->jcol_ms_fft = t[1];
      c->jcol_fft = c->opt.jcol_mode == AP_JCOL_FFT || (c->opt.jcol_mode == AP_JCOL_AUTO && t[1] < t[0]);
    }
  }
  // the Gram's tcgen05 threshold: tiles with few columns cost the tensor-core
  // kernel its per-tile hand-overs for little work, so both kernels are timed
  // on this problem's tiles for a few thresholds and the fastest kept
  // a forced threshold starts a 16-column class (tiles are grouped by class)
  c->gram_tc_min = c->opt.gram_tc_min > 0 ? (c->opt.gram_tc_min + 14) / 16 * 16 + 1 : GRAM_TC_MIN_DEFAULT;
  c->gram_tc_max = gram_tc_max_cols();
  if (c->opt.gram_tc_min > 0 && !f64) c->gram_ranges = gram_ranges_for(c->h_tile_ncol, false, c->gram_tc_min);
  if (!f64 && !c->h_tile_ncol.empty() && c->opt.gram_tc_min <= 0) {
    // (tc_min, tc_max): the tensor-core kernel for tiles of tc_min .. tc_max
    // columns; the 128-column form runs fewer CTAs per SM, so the warp-MMA
    // kernel may serve tiles past 64 columns better
    const int none = gram_tc_max_cols() + 1;
    const int cands[][2] = {{1, 128}, {33, 128}, {49, 128}, {65, 128}, {97, 128}, {1, 64}, {33, 64}, {49, 64},
                            {none, 128}};
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    double best = 1e300;
    for (const auto& cd : cands) {
      const std::vector<GramRange> rg = gram_ranges_for(c->h_tile_ncol, false, cd[0], cd[1]);
      double tot = 0.0;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        launch_gram<float>(c->d_jwork, rg.data(), (int)rg.size(), c->d_jt_src, c->d_srcs, c->d_imgs,
                           (const float*)c->d_dbuf, (const float*)c->d_jbuf, c->gplan, c->d_vals, c->d_status, st,
                           c->have_fj ? &c->fj : nullptr);
        cudaEventRecord(e1, st);
        CUDA_TRY(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;
      }
      if (tot < best) {
        best = tot;
        c->gram_tc_min = cd[0];
        c->gram_tc_max = cd[1];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
    c->gram_ranges = gram_ranges_for(c->h_tile_ncol, false, c->gram_tc_min, c->gram_tc_max);
  }

  c->h_imgs = I;
  c->h_srcs = S;
  c->n_img = n_img;
  c->n_src = n_src;
  c->n_params = n_params;
  c->n_groups = n_groups;
  c->n_rwork = (int)rwork.size();
  c->n_tile_entries = (int64_t)tile_src.size();
  c->n_jwork = (int)jwork.size();
  c->dbuf_elems = dbuf_elems;
  c->jbuf_elems = jbuf_elems;
  c->h_row_ptr = row_ptr;
  c->h_col_idx = col_idx;
  c->nnz = (int64_t)col_idx.size();
  c->h_param_group = param_group;
  c->max_dense_n = max_dense;
  c->any_dense = any_dense;
  c->any_pcg = any_pcg;
  c->any_grid = any_grid;
  c->h_groups = groups;
  c->Kmax = Kmax;
  c->iterations = 0;
  c->have_problem = true;
  return AP_OK;
}

int ap_get_layout(ap_ctx* c, int* n_groups, int* param_group_host) {
  if (!c) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  if (n_groups) *n_groups = c->n_groups;
  if (param_group_host) std::copy(c->h_param_group.begin(), c->h_param_group.end(), param_group_host);
  return AP_OK;
}

int ap_get_adaptive_layout(ap_ctx* c, int64_t* n_samples, int64_t* offsets_host) {
  if (!c) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaSetDevice(c->opt.device);
  int rc = build_adaptive(c);
  if (rc) return rc;
  if (n_samples) *n_samples = c->n_asamples;
  if (offsets_host) std::copy(c->h_aoff.begin(), c->h_aoff.begin() + c->n_src_user, offsets_host);
  return AP_OK;
}

int ap_eval_adaptive(ap_ctx* c, const double* theta, double tol, double* chi2, void* const* model_dev,
                     uint8_t* levels_dev, int64_t* counts_host, void* stream) {
  if (!c || !theta || !(tol >= 0.0) || !std::isfinite(tol)) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaSetDevice(c->opt.device);
  int rc = build_adaptive(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (model_dev) launch_store_ptrs(model_dev, c->n_img, c->d_model_ptrs, st);
  CUDA_TRY(c, cudaMemsetAsync(c->adapt.n_list, 0, sizeof(int), st));
  CUDA_TRY(c, cudaMemsetAsync(c->adapt.counts, 0, ADAPT_COUNTS * sizeof(unsigned long long), st));
  if (c->f64)
    eval_adaptive<double>(c, theta, tol, chi2, model_dev != nullptr, st);
  else
    eval_adaptive<float>(c, theta, tol, chi2, model_dev != nullptr, st);
  if (levels_dev && c->n_asamples > 0)
    CUDA_TRY(c, cudaMemcpyAsync(levels_dev, c->adapt.level, (size_t)c->n_asamples, cudaMemcpyDeviceToDevice, st));
  if ((rc = drop_lm_reuse(c, st))) return rc;
  if (counts_host) {
    unsigned long long h[ADAPT_COUNTS];
    CUDA_TRY(c, cudaMemcpyAsync(h, c->adapt.counts, sizeof(h), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    for (int k = 0; k < ADAPT_COUNTS; ++k) counts_host[k] = (int64_t)h[k];
  }
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

int ap_eval_shifted(ap_ctx* c, const double* theta, int method, double* chi2, void* const* model_dev, void* stream) {
  if (!c || !theta) return AP_ERR_ARG;
  if (method != AP_SHIFT_LANCZOS3 && method != AP_SHIFT_BILINEAR) return fail(c, AP_ERR_ARG, "unknown shift method");
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaSetDevice(c->opt.device);
  int rc = build_shift(c);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (model_dev) launch_store_ptrs(model_dev, c->n_img, c->d_model_ptrs, st);
  if (c->f64)
    eval_shifted<double>(c, theta, method, chi2, model_dev != nullptr, st);
  else
    eval_shifted<float>(c, theta, method, chi2, model_dev != nullptr, st);
  if ((rc = drop_lm_reuse(c, st))) return rc;
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

int ap_render(ap_ctx* c, const double* theta, void* const* model_dev, void* stream) {
  if (!c || !theta || !model_dev) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaSetDevice(c->opt.device);
  cudaStream_t st = (cudaStream_t)stream;
  launch_store_ptrs(model_dev, c->n_img, c->d_model_ptrs, st);
  int rc = eval_any(c, theta, nullptr, nullptr, c->d_model_ptrs, false, st);
  if (rc) return rc;
  if ((rc = drop_lm_reuse(c, st))) return rc;
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

int ap_eval(ap_ctx* c, const double* theta, double* chi2, double* grad, void* stream) {
  if (!c || !theta || !chi2) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = eval_any(c, theta, chi2, grad, nullptr, false, st);
  if (rc) return rc;
  if ((rc = drop_lm_reuse(c, st))) return rc;
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

int ap_normal_eq(ap_ctx* c, const double* theta, double* jtwr, void* stream) {
  if (!c || !theta || !jtwr) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = normal_eq_any(c, theta, c->d_jtwr, st);
  if (rc) return rc;
  if ((rc = drop_lm_reuse(c, st))) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(jtwr, c->d_jtwr, (size_t)c->n_params * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

int ap_get_jtwj_nnz(ap_ctx* c, int64_t* nnz) {
  if (!c || !nnz) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  *nnz = c->nnz;
  return AP_OK;
}

int ap_get_jtwj_structure(ap_ctx* c, int64_t* row_ptr, int32_t* col_idx) {
  if (!c || !row_ptr || !col_idx) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  std::copy(c->h_row_ptr.begin(), c->h_row_ptr.end(), row_ptr);
  std::copy(c->h_col_idx.begin(), c->h_col_idx.end(), col_idx);
  return AP_OK;
}

int ap_copy_jtwj(ap_ctx* c, double* values, void* stream) {
  if (!c || !values) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  if (c->nnz > 0)
    CUDA_TRY(c, cudaMemcpyAsync(values, c->d_vals, (size_t)c->nnz * sizeof(double), cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
  return AP_OK;
}

int ap_lm_solve(ap_ctx* c, double* lambda, double* delta, void* stream) {
  if (!c || !lambda || !delta) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(c, cudaMemsetAsync(delta, 0, (size_t)c->n_params * sizeof(double), st));
  int rc = solve_any(c, lambda, delta, st);
  if (rc) return rc;
  CUDA_TRY(c, cudaGetLastError());
  return AP_OK;
}

int ap_lm_iterate(ap_ctx* c, double* theta, double* lambda, double* chi2, int n_iter, double* log_host,
                  void* stream) {
  if (!c || !theta || !lambda || n_iter < 0) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  cudaSetDevice(c->opt.device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)c->n_params, G = (size_t)c->n_groups;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_theta, theta, P * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_lambda, lambda, G * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(c, cudaMemsetAsync(c->d_delta, 0, P * sizeof(double), st));
  // a new starting point (and possibly new image data): the first iteration
  // evaluates every group at theta
  int rc = drop_lm_reuse(c, st);
  if (rc) return rc;
  c->lm_started = true;
  return lm_run(c, theta, lambda, chi2, n_iter, log_host, st);
}

int ap_lm_continue(ap_ctx* c, double* theta, double* lambda, double* chi2, int n_iter, double* log_host,
                   void* stream) {
  if (!c || n_iter < 0) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  if (!c->lm_started) return fail(c, AP_ERR_STATE, "no fit to continue: call ap_lm_iterate first");
  cudaSetDevice(c->opt.device);
  return lm_run(c, theta, lambda, chi2, n_iter, log_host, (cudaStream_t)stream);
}

int ap_get_status(ap_ctx* c, int* status, void* stream) {
  if (!c || !status) return AP_ERR_ARG;
  if (!c->have_problem) { *status = AP_OK; return AP_OK; }
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(c, cudaStreamSynchronize(st));
  CUDA_TRY(c, cudaMemcpy(status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
  return AP_OK;
}

int ap_get_state(ap_ctx* c, double* chi2_host, int64_t* iterations_host, int* cg_iters_host) {
  if (!c) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_STATE, "no problem set");
  if (cg_iters_host)
    CUDA_TRY(c, cudaMemcpy(cg_iters_host, c->d_cg_iters, (size_t)c->n_groups * sizeof(int), cudaMemcpyDeviceToHost));
  if (chi2_host) CUDA_TRY(c, cudaMemcpy(chi2_host, c->d_chi2_state, (size_t)c->n_groups * sizeof(double), cudaMemcpyDeviceToHost));
  if (iterations_host) *iterations_host = c->iterations;
  return AP_OK;
}

int ap_get_jcol_mode(ap_ctx* c, int* mode, double* ms_direct, double* ms_fft, int* fft_blocks_64,
                     int* fft_blocks_128) {
  if (!c) return AP_ERR_ARG;
  if (!c->have_problem) return fail(c, AP_ERR_ARG, "no problem set");
  if (mode) *mode = c->jcol_fft ? AP_JCOL_FFT : AP_JCOL_DIRECT;
  if (ms_direct) *ms_direct = c->jcol_ms_direct;
  if (ms_fft) *ms_fft = c->jcol_ms_fft;
  if (fft_blocks_64) *fft_blocks_64 = c->n_jf64;
  if (fft_blocks_128) *fft_blocks_128 = c->n_jf128;
  return AP_OK;
}

int ap_get_conv_variant(ap_ctx* c, int* variant, int* n_variants, int* shape_host, double* ms_host) {
  if (!c) return AP_ERR_ARG;
  if (variant) *variant = c->have_problem ? c->conv_variant : -1;
  if (n_variants) *n_variants = N_CONV_VARIANTS;
  for (int v = 0; v < N_CONV_VARIANTS; ++v) {
    if (shape_host) {
      shape_host[3 * v] = conv_tile_w(v);
      shape_host[3 * v + 1] = conv_tile_h(v);
      shape_host[3 * v + 2] = conv_threads(v);
    }
    if (ms_host) ms_host[v] = c->have_problem ? c->conv_ms[v] : -1.0;
  }
  return AP_OK;
}

int ap_get_launch_count(ap_ctx* c, int* per_it, int* per_eval) {
  if (!c) return AP_ERR_ARG;
  if (per_eval) *per_eval = c->launches_last_eval;
  if (per_it) {
    *per_it = 0;
    if (c->lm_graph) {
      size_t n = 0;
      CUDA_TRY(c, cudaGraphGetNodes(c->lm_graph, nullptr, &n));
      std::vector<cudaGraphNode_t> nodes(n);
      if (n) CUDA_TRY(c, cudaGraphGetNodes(c->lm_graph, nodes.data(), &n));
      int k = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
      }
      *per_it = k;
    }
  }
  return AP_OK;
}

int ap_set_timing(ap_ctx* c, int on) {
  if (!c) return AP_ERR_ARG;
  c->timing = on != 0;
  return AP_OK;
}

int ap_get_timing(ap_ctx* c, char* names, int size, double* ms, int* counts, int max_kernels, int* n_kernels) {
  if (!c) return AP_ERR_ARG;
  for (auto& t : c->pending) {
    cudaEventSynchronize(t.b);
    float v = 0.f;
    cudaEventElapsedTime(&v, t.a, t.b);
    size_t k = 0;
    while (k < c->stats.names.size() && c->stats.names[k] != t.name) ++k;
    if (k == c->stats.names.size()) {
      c->stats.names.push_back(t.name);
      c->stats.total_ms.push_back(0.0);
      c->stats.count.push_back(0);
    }
    c->stats.total_ms[k] += v;
    c->stats.count[k] += 1;
    c->event_pool.push_back(t.a);
    c->event_pool.push_back(t.b);
  }
  c->pending.clear();
  std::string joined;
  int n = 0;
  for (size_t k = 0; k < c->stats.names.size(); ++k) {
    if ((int)k < max_kernels && ms) ms[k] = c->stats.total_ms[k] / std::max<long>(c->stats.count[k], 1);
    if ((int)k < max_kernels && counts) counts[k] = (int)c->stats.count[k];
    if (k) joined += ";";
    joined += c->stats.names[k];
    ++n;
  }
  if (names && size > 0) {
    std::strncpy(names, joined.c_str(), (size_t)size - 1);
    names[size - 1] = 0;
  }
  if (n_kernels) *n_kernels = n;
  c->stats = TimingStats{};
  return AP_OK;
}

}  // extern "C"
