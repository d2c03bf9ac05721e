// J^T W J tile Grams on the fifth-generation tensor cores (tcgen05), float
// path (Sec. "Optimization methods": the Gauss-Newton matrix of LM).
//
// Pass 1 of the two-pass J^T W J (see ap_gram.cu) for tiles of up to 128
// free columns.  A CTA owns a run of 16 x 16 image tiles (persistent,
// grid-stride).  For one tile it reads the tile's column list (planned on the
// host: where each column image lies and which source pair block its
// entries go to) and streams the sqrt(w)-scaled Jacobian columns
// through shared memory in chunks of 32 pixels: every thread loads its pixel
// of some columns (coalesced rows of the column images), splits each value
// into a TF32 head and a TF32 tail and stores both, K-major with the 128-byte
// swizzle, into a double-buffered stage.  One thread issues the MMAs of a
// chunk -- head x tail + tail x head + head x head (3xTF32, the small terms
// first; the tail x tail term is below float32 rounding) -- and commits them
// to the stage's mbarrier, so the loads of the next chunks overlap the MMAs
// of this one.  Each MMA step rounds its float32 accumulator, so the tile's
// 256 pixels are summed in four segments of 64 pixels (two chunks) -- the
// float32 sums of the warp-MMA path -- and the segments joined outside the
// MMA: the 32-column form keeps four accumulators in tensor memory and the
// epilogue adds them in float64; the 64- and 128-column forms keep two, a
// running sum (segment 0) and a segment accumulator, and the producer warps
// add each finished segment into the running sum (tcgen05.ld, float32 add,
// tcgen05.st) before the MMAs of the next one begin, the epilogue adding the
// last in float64.  At the end of the tile the accumulators are read back
// (tcgen05.ld) and each entry stored into its source pair's scratch block
// exactly as the warp-MMA path does.
//
// The MMA is M = 128 (rows past C unused) by N = C rounded up to 16.  Three
// forms by the column capacity CMAX (32, 64, 128), taking 128, 128 and 256
// tensor-memory columns: three, three and two CTAs share an SM.  Each
// producer warp holds CMAX / 8 columns of a chunk in registers and keeps the
// two next chunks (the 128-column form: the next one) in flight while one is
// stored (the loads are latency-bound).  Rows and columns past C hold stale values of earlier
// tiles; they only reach accumulator rows and columns that are never read.
//
// Every wait on an mbarrier is bounded: past the bound the kernel raises
// AP_ERR_TIMEOUT in the status word, stops taking tiles and still frees its
// tensor memory before returning.
#include <cuda_runtime.h>

#include <algorithm>

#include "ap_internal.cuh"

namespace ap {

namespace {

constexpr int TC_PRODUCERS = 256;                   // 8 producer / epilogue warps
constexpr int TC_THREADS = TC_PRODUCERS + 32;       // + the warp that issues the MMAs
constexpr int TC_CHUNK = 32;                        // pixels per chunk: one 128-byte row of TF32
constexpr int TC_NCHUNK = TILE_THREADS / TC_CHUNK;  // 8 chunks per tile
constexpr int TC_M = 128;                           // MMA rows (columns of the tile, past C unused)
constexpr int TC_SEG = 4;                           // accumulators: 64-pixel segments of the tile
constexpr uint32_t TC_WAIT_LIMIT = 1u << 20;        // mbarrier polls before giving up
constexpr int TC_MAX_SRC = 256;                     // sources reaching one tile (more: the warp-MMA kernel)

struct TcCol {           // one free column of the tile
  const float* base;     // the column image (its box, row pitch bw)
  int off0;              // offset of the tile's pixel (0, 0) in it (may lie outside the box)
  int bw;                // box width = row pitch
  uint32_t bounds;       // the box in tile coordinates, clamped to 0..16: rows [b0, b1), columns [b2, b3), a byte each
  int info;              // (local source << 8) | (free slot << 4) | free slots of that source
};

template <int CMAX>
struct TcSmem {
  static_assert(CMAX == 32 || CMAX == 64 || CMAX == 128, "column capacity");
  // How the four 64-pixel segments are joined:
  //  SEG4 (32 columns): four tensor-memory accumulators, added in the epilogue;
  //  SUM_SMEM (64): two tensor-memory accumulators taking the segments in
  //    turn, each finished one added into a float32 running sum in shared
  //    memory by the producer warps while the MMAs of the next one run;
  //  SUM_TMEM (128): a running sum and a segment accumulator in tensor
  //    memory, the segment added into the sum (tcgen05.ld / st) before the
  //    MMAs of the next one.
  static constexpr bool SEG4 = CMAX == 32, SUM_SMEM = CMAX == 64, SUM_TMEM = CMAX == 128;
  static constexpr int NACC = SEG4 ? TC_SEG : 2;     // tensor-memory accumulators, accumulator k at column k * CMAX
  static constexpr int TMEM_COLS = NACC * CMAX;      // 128, 128, 256
  // stages hold CMAX rows (the 32-column form: 128); the M = 128 operand
  // reads of the 64-column form run on past its 64 rows into the next
  // operand or the arrays behind the stages (at least 8 KB, all in this
  // CTA's shared memory) and fill accumulator rows that are never read
  static constexpr int ROWS = SUM_SMEM ? 64 : TC_M;
  static constexpr int OPERAND = ROWS * 128;         // bytes of one operand (head or tail) of one stage
  static constexpr int STAGE = 2 * OPERAND;          // head + tail
  static constexpr int DATA = 2 * STAGE;             // two stages
  static constexpr int COLS = DATA;                  // TcCol[TC_M]
  static constexpr int SW = COLS + TC_M * (int)sizeof(TcCol);   // float sw[256]
  static constexpr int SUMLD = CMAX + 1;                        // running sum: float [CMAX][CMAX + 1]
  static constexpr int SUM = (SW + TILE_THREADS * 4 + 15) / 16 * 16;
  static constexpr int MISC = SUM + (SUM_SMEM ? (CMAX * SUMLD * 4 + 15) / 16 * 16 : 0);
  static_assert(!SUM_SMEM || MISC - DATA >= TC_M * 128 - OPERAND, "operand reads past the stages stay inside");
  // CTAs per SM: as many as the tensor memory holds, at most three (registers)
  static constexpr int MIN_CTAS = 512 / TMEM_COLS < 3 ? 512 / TMEM_COLS : 3;
  // ten mbarriers, tensor-memory address, flags, stage column counts; a
  // form with fewer CTAs per SM asks for more, so that no more CTAs share an
  // SM than its tensor memory holds (a CTA past that would wait in its
  // allocation)
  static constexpr int NEED = MISC + 96;
  static constexpr int FLOOR = MIN_CTAS == 2 ? 80 * 1024 : 0;
  static constexpr int BYTES = NEED > FLOOR ? NEED : FLOOR;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// K-major operand with the 128-byte swizzle: row m of 32 TF32 values is 128
// bytes; rows come in atoms of 8 (1024 bytes) and the 16-byte chunk j of row
// m sits at chunk j ^ (m & 7).
__device__ __forceinline__ uint32_t sw128_offset(int m, int k) {
  return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((((k >> 2) ^ (m & 7)) << 4) | ((k & 3) << 2)));
}

// shared-memory matrix descriptor: start address, leading offset (unused by
// swizzled K-major layouts), stride 1024 bytes between 8-row atoms, the
// descriptor version of this architecture, 128-byte swizzle
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::tf32: float32 accumulator, TF32 A and B,
// both K-major, N and M
__device__ __forceinline__ uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive accumulator columns of this warp's 32 lanes (the caller
// waits with tmem_wait_ld before reading them)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&r)[4]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r[0]), "r"(r[1]),
               "r"(r[2]), "r"(r[3])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// the same store as the warp-MMA path: entry (ca <= cb) into its source
// pair's block (pairs of the tile's L sources numbered row-major over a <= b)
__device__ __forceinline__ void tc_store(double g, int ia, int ib, int L, const int64_t* __restrict__ tab,
                                         const int* __restrict__ tabs, double* __restrict__ scr) {
  const int la = ia >> 8, fa = (ia >> 4) & 15;
  const int lb = ib >> 8, fb = (ib >> 4) & 15, mb = ib & 15;
  const int pidx = la * L - (la * (la - 1)) / 2 + (lb - la);
  scr[tab[pidx] + (int64_t)(fa * mb + fb) * tabs[pidx]] = g;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// named barrier of the producer warps only (the MMA warp runs on its own)
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(TC_PRODUCERS) : "memory"); }

template <int CMAX>
__global__ void __launch_bounds__(TC_THREADS, TcSmem<CMAX>::MIN_CTAS) gram_tc_kernel(
    const TileWork* __restrict__ work, const int64_t* __restrict__ col_ptr, const GramCol* __restrict__ gcols,
    const ImageDev* __restrict__ imgs, const float* __restrict__ dbuf, const float* __restrict__ jbuf,
    const int64_t* __restrict__ tab0, const int64_t* __restrict__ tab_all, const int* __restrict__ tabs_all,
    double* __restrict__ scr, int t_first, int t_end, int* __restrict__ status) {
  using S = TcSmem<CMAX>;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment of the swizzled operands
  // (offset from the shared-window address, so that the pointer keeps its
  // shared address space and its accesses compile to shared-memory ones)
  unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  TcCol* cols = reinterpret_cast<TcCol*>(sm + S::COLS);
  float* sw = reinterpret_cast<float*>(sm + S::SW);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + S::MISC);        // [2]: a stage was filled (8 producer warps)
  uint64_t* empty = full + 2;                                          // [2]: its MMAs completed (commit)
  uint64_t* acc_full = full + 4;                                       // the tile's accumulator is complete (commit)
  uint64_t* acc_empty = full + 5;                                      // the accumulator was read (8 producer warps)
  // [2] per accumulator (SUM_SMEM; SUM_TMEM uses the first): a segment in
  // it is complete (commit), it was added to the running sum (8 warps).
  // Every waiter of a barrier is at most one phase behind it: a barrier
  // that completed twice since would look as if it had not.
  uint64_t* seg_full = full + 6;
  uint64_t* seg_empty = full + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + S::MISC + 80);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::MISC + 84);
  int* stage_cols = reinterpret_cast<int*>(sm + S::MISC + 88);        // [2]: C of the chunk in each stage

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[k])), "r"(TC_PRODUCERS / 32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[k])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(acc_full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(acc_empty)), "r"(TC_PRODUCERS / 32) : "memory");
    for (int k = 0; k < 2; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&seg_full[k])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&seg_empty[k])), "r"(TC_PRODUCERS / 32)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t base_addr = smem_u32(sm);

  if (warp == TC_PRODUCERS / 32) {
    // ================= MMA warp: one thread issues every MMA =================
    if (lane == 0) {
      uint32_t g = 0;   // chunks consumed by this CTA
      int t_local = 0;
      for (int tile = t_first + blockIdx.x; tile < t_end && !*abort_flag; tile += gridDim.x, ++t_local) {
        // the previous tile's accumulator must have been read
        if (t_local > 0 && !mbar_wait(smem_u32(acc_empty), (t_local - 1) & 1)) {
          atomicCAS(status, 0, AP_ERR_TIMEOUT);
          *abort_flag = 1;
          break;
        }
        fence_after_sync();
        for (int ch = 0; ch < TC_NCHUNK; ++ch, ++g) {
          const int st = g & 1;
          if (!mbar_wait(smem_u32(&full[st]), (g >> 1) & 1)) {
            atomicCAS(status, 0, AP_ERR_TIMEOUT);
            *abort_flag = 1;
            break;
          }
          fence_after_sync();
          const int C = stage_cols[st];
          const uint32_t id = tf32_idesc(TC_M, C <= 16 ? 16 : ((C + 15) & ~15));
          if (!S::SEG4 && (ch == 4 || ch == 6)) {
            // the accumulator is free once the segment it last held was
            // added to the running sum: SUM_SMEM accumulator ch / 2 & 1 (one
            // release per tile each), SUM_TMEM the segment one (two per tile)
            const bool ok = S::SUM_SMEM ? mbar_wait(smem_u32(&seg_empty[(ch >> 1) & 1]), t_local & 1)
                                        : mbar_wait(smem_u32(&seg_empty[0]), (2 * t_local + (ch == 6)) & 1);
            if (!ok) {
              atomicCAS(status, 0, AP_ERR_TIMEOUT);
              *abort_flag = 1;
              break;
            }
            fence_after_sync();
          }
          // the chunk's accumulator: its segment (SEG4), the segments in turn
          // (SUM_SMEM), the running sum for segment 0 and the segment
          // accumulator after it (SUM_TMEM)
          const int acc = S::SEG4 ? (ch >> 1) : S::SUM_SMEM ? ((ch >> 1) & 1) : (ch >= 2 ? 1 : 0);
          const uint32_t d = tmem + (uint32_t)(acc * CMAX);
          const uint32_t a_hi = base_addr + st * S::STAGE, a_lo = a_hi + S::OPERAND;
#pragma unroll
          for (int kk = 0; kk < TC_CHUNK / 8; ++kk) {
            const uint32_t kb = kk * 32;   // 8 TF32 values per MMA step
            const uint64_t h = sw128_desc(a_hi + kb), l = sw128_desc(a_lo + kb);
            mma_tf32(d, h, l, id, ((ch & 1) || kk > 0) ? 1u : 0u);   // a segment starts afresh
            mma_tf32(d, l, h, id, 1u);
            mma_tf32(d, h, h, id, 1u);
          }
          mma_commit(smem_u32(&empty[st]));     // the stage may be refilled once these complete
          // a segment is complete: SUM_SMEM in accumulator ch / 2 & 1 (chunks
          // 1 and 5: accumulator 0, chunk 3: 1), SUM_TMEM (chunks 3 and 5)
          if (S::SUM_SMEM && (ch & 1) && ch < 7) mma_commit(smem_u32(&seg_full[(ch >> 1) & 1]));
          if (S::SUM_TMEM && (ch == 3 || ch == 5)) mma_commit(smem_u32(&seg_full[0]));
          if (ch == TC_NCHUNK - 1) mma_commit(smem_u32(acc_full));
        }
      }
    }
    __syncwarp();
  } else {
    // ============ producer warps: columns in, accumulator out ============
    // Every producer warp runs the same sequence of named barriers whatever
    // happens: a warp that met a timeout (or sees another's) only skips its
    // waits, stores and arrivals (dead), it never leaves the loop early.
    uint32_t g = 0;   // chunks filled by this CTA
    int t_local = 0;
    bool dead = false;
    for (int tile = t_first + blockIdx.x; tile < t_end; tile += gridDim.x, ++t_local) {
      const TileWork w = work[tile];
      const int H = imgs[w.image].H, W = imgs[w.image].W;
      const float* var = imgs[w.image].var;
      const uint8_t* mask = imgs[w.image].mask;
      const int L = w.e1 - w.e0;
      // the tile's columns, planned on the host
      const int64_t c0 = col_ptr[tile];
      const int C = (int)(col_ptr[tile + 1] - c0);
      const bool fits = C <= CMAX && L <= TC_MAX_SRC;
      if (!fits && tid == 0) atomicCAS(status, 0, AP_ERR_ARG);
      const int Cu = fits ? C : 0;   // a tile that does not fit is reduced to no columns
      producers_sync();   // the previous tile's epilogue no longer reads cols
      if (tid < Cu) {
        const GramCol gc = gcols[c0 + tid];
        TcCol col;
        col.base = ((gc.info & GRAM_COL_CONV) ? jbuf : dbuf) + gc.off;
        col.off0 = gc.off0;
        col.bw = gc.bw;
        col.bounds = gc.bounds;
        col.info = gc.info & ~GRAM_COL_CONV;
        cols[tid] = col;
      }
      {
        // sqrt(w) of the thread's pixel (float32, correctly rounded division and root)
        const int i = w.r0 + tid / TILE, j = w.c0 + tid % TILE;
        float sv = 0.f;
        if (i < H && j < W) {
          const size_t o = (size_t)i * W + j;
          const float v = var[o];
          if ((mask == nullptr || mask[o] == 0) && v > 0.f && isfinite(v)) sv = 1.0f / sqrtf(v);
        }
        sw[tid] = sv;
      }
      producers_sync();
      dead = dead || *abort_flag;
      constexpr int MAXU = CMAX / (TC_PRODUCERS / 32);
      auto load_chunk = [&](int ch, float (&dst)[MAXU]) {
        const int p = ch * TC_CHUNK + lane;
        const int pi = p / TILE, pj = p % TILE;
#pragma unroll
        for (int u = 0; u < MAXU; ++u) {
          const int m = warp + u * (TC_PRODUCERS / 32);
          float v = 0.f;
          if (m < Cu) {
            const TcCol& cl = cols[m];
            const uint32_t b = cl.bounds;
            if (pi >= (int)(b & 255u) && pi < (int)((b >> 8) & 255u) && pj >= (int)((b >> 16) & 255u) &&
                pj < (int)(b >> 24))
              v = __ldg(cl.base + (cl.off0 + pi * cl.bw + pj));
          }
          dst[u] = v;
        }
      };
      // chunk ch into its stage: wait until the MMAs that last read the
      // stage have completed, split into head and tail, store, arrive
      auto store_chunk = [&](int ch, const float (&cur)[MAXU]) {
        const uint32_t gc = g + ch;
        const int st = gc & 1;
        int ok = 1;
        if (lane == 0 && gc >= 2 && !dead) ok = mbar_wait(smem_u32(&empty[st]), ((gc >> 1) - 1) & 1) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) {
            atomicCAS(status, 0, AP_ERR_TIMEOUT);
            *abort_flag = 1;
          }
          dead = true;
        }
        if (dead) return;
        unsigned char* hi = sm + st * S::STAGE;
        unsigned char* lo = hi + S::OPERAND;
        const float s = sw[ch * TC_CHUNK + lane];
#pragma unroll
        for (int u = 0; u < MAXU; ++u) {
          const int m = warp + u * (TC_PRODUCERS / 32);
          if (m < Cu) {
            const float x = cur[u] * s;
            const uint32_t h = tf32_rna(x);
            const uint32_t t = tf32_rna(x - __uint_as_float(h));
            const uint32_t off = sw128_offset(m, lane);
            *reinterpret_cast<uint32_t*>(hi + off) = h;
            *reinterpret_cast<uint32_t*>(lo + off) = t;
          }
        }
        if (tid == 0) stage_cols[st] = Cu;
        // the stores are read by the tensor cores (async proxy), then the
        // warp's arrival releases them to the MMA warp
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[st]));
      };
      // accumulator lanes and columns of this warp (tcgen05.ld / st reach
      // the lane quarter w % 4; the columns are split between warps 0-3 and
      // 4-7); warp-uniform
      const int q = warp & 3, half = warp >> 2;
      const int N = Cu <= 16 ? 16 : ((Cu + 15) & ~15);
      const int nh = ((N / 16) + 1) / 2 * 16;   // columns of the first half (a multiple of 16)
      const int n0 = half ? nh : 0, n1 = half ? N : nh;
      const bool mine = n0 < Cu && 32 * q < Cu;   // else nothing this warp reads or stores
      const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
      float* sumr = reinterpret_cast<float*>(sm + S::SUM) + (32 * q + lane) * S::SUMLD;   // this thread's row
      // SUM_SMEM: add segment j (accumulator a = j & 1; the first one
      // copied) into the running sum in shared memory, each thread its own
      // row and columns; segments 0 and 1 then release their accumulator.
      // SUM_TMEM: add the segment accumulator into the running sum in tensor
      // memory and release it (a = 0).  k is the phase of seg_full[a] that
      // completes the segment.
      auto drain = [&](int j, int a, uint32_t k, bool release) {
        int ok = 1;
        if (lane == 0 && !dead) ok = mbar_wait(smem_u32(&seg_full[a]), k & 1) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) {
            atomicCAS(status, 0, AP_ERR_TIMEOUT);
            *abort_flag = 1;
          }
          dead = true;
        }
        if (dead) return;
        fence_after_sync();
        if (mine) {
          if constexpr (S::SUM_SMEM) {
#pragma unroll 1
            for (int cb0 = n0; cb0 < n1 && cb0 < Cu; cb0 += 8) {
              uint32_t a[8];
              tmem_ld8(tq + (uint32_t)((j & 1) * CMAX + cb0), a);
              tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 8; ++u) sumr[cb0 + u] = (j == 0 ? 0.f : sumr[cb0 + u]) + __uint_as_float(a[u]);
            }
          } else {
#pragma unroll 1
            for (int cb0 = n0; cb0 < n1 && cb0 < Cu; cb0 += 4) {
              uint32_t a[4], b[4];
              tmem_ld4(tq + (uint32_t)cb0, a);
              tmem_ld4(tq + (uint32_t)(CMAX + cb0), b);
              tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 4; ++u) a[u] = __float_as_uint(__uint_as_float(a[u]) + __uint_as_float(b[u]));
              tmem_st4(tq + (uint32_t)cb0, a);
            }
            tmem_wait_st();
          }
        }
        if (!release) return;
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&seg_empty[a]));
      };
      // ---- chunks of 32 pixels (two image rows of the tile), warp w holding
      // columns w, w + 8, ...: the values of the two next chunks (the next
      // one in the 128-column form) are in flight into registers while chunk
      // ch is stored
      if constexpr (CMAX <= 64) {
        float buf[3][MAXU];
        load_chunk(0, buf[0]);
        load_chunk(1, buf[1]);
#pragma unroll
        for (int ch = 0; ch < TC_NCHUNK; ++ch) {
          if (ch + 2 < TC_NCHUNK) load_chunk(ch + 2, buf[(ch + 2) % 3]);
          store_chunk(ch, buf[ch % 3]);
          // segment j = chunks 2j, 2j + 1 is complete once the stage of
          // chunk 2j + 3 was free (its MMAs are done): no wait
          if (S::SUM_SMEM && (ch & 1) && ch >= 3) {
            const int j = (ch - 3) / 2, a = j & 1;
            drain(j, a, a == 0 ? 2 * t_local + (j == 2) : t_local, j < 2);
          }
        }
      } else {   // 128 columns: one chunk ahead (registers)
        float buf[2][MAXU];
        load_chunk(0, buf[0]);
#pragma unroll
        for (int ch = 0; ch < TC_NCHUNK; ++ch) {
          if (ch + 1 < TC_NCHUNK) load_chunk(ch + 1, buf[(ch + 1) % 2]);
          store_chunk(ch, buf[ch % 2]);
          // segments 1 and 2 into the running sum once chunks 5 and 7 are
          // stored (the MMAs of the segment are then done): the MMAs of the
          // next segment find both of its chunks ready
          if (ch == 5 || ch == 7) drain(0, 0, 2 * t_local + (ch == 7), true);
        }
      }
      g += TC_NCHUNK;
      // ---- epilogue: the accumulator is complete after the tile's last commit
      int ok = 1;
      if (lane == 0 && !dead) ok = mbar_wait(smem_u32(acc_full), t_local & 1) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) {
          atomicCAS(status, 0, AP_ERR_TIMEOUT);
          *abort_flag = 1;
        }
        dead = true;
      }
      if (dead) continue;
      fence_after_sync();
      // an entry is the float64 sum of the four segments (SEG4), of the
      // running sum and the last segment (accumulator 1) otherwise
      const int64_t* tab = tab_all + tab0[tile];
      const int* tabs = tabs_all + tab0[tile];
      const int ca = 32 * q + lane;
      constexpr int NLD = S::SEG4 ? TC_SEG : 2;
      if (mine) {
        for (int cb0 = n0; cb0 < n1 && cb0 < Cu; cb0 += 8) {
          uint32_t r[NLD][8];
#pragma unroll
          for (int k = 0; k < NLD; ++k) tmem_ld8(tq + (uint32_t)(k * CMAX + cb0), r[k]);
          tmem_wait_ld();
          if (ca < Cu) {
            const int ia = cols[ca].info;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int cb = cb0 + u;
              if (cb < Cu && cb >= ca) {
                double val;
                if constexpr (S::SEG4)
                  val = ((double)__uint_as_float(r[0][u]) + (double)__uint_as_float(r[1][u])) +
                        ((double)__uint_as_float(r[NLD - 2][u]) + (double)__uint_as_float(r[NLD - 1][u]));
                else if constexpr (S::SUM_SMEM)
                  val = (double)sumr[cb] + (double)__uint_as_float(r[1][u]);
                else
                  val = (double)__uint_as_float(r[0][u]) + (double)__uint_as_float(r[1][u]);
                tc_store(val, ia, cols[cb].info, L, tab, tabs, scr);
              }
            }
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(acc_empty));
    }
  }
  // free the tensor memory on every path (the next kernel on this SM needs it)
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
  }
}

// CTAs of the kernel one SM holds: shared memory (with the per-block
// reservation), registers, threads and the 512 tensor-memory columns
template <int CMAX>
int tc_blocks_per_sm() {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, gram_tc_kernel<CMAX>) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int per_block = TcSmem<CMAX>::BYTES + 1024 + (int)fa.sharedSizeBytes + reserved;
  int n = smem_sm / per_block;
  n = std::min(n, regs_sm / std::max(1, fa.numRegs * TC_THREADS));
  n = std::min(n, thr_sm / TC_THREADS);
  n = std::min(n, 512 / TcSmem<CMAX>::TMEM_COLS);
  return std::max(n, 1);
}

template <int CMAX>
void launch_tc(const TileWork* work, int t0, int t1, const ImageDev* imgs,
               const float* dbuf, const float* jbuf, const GramPlan& gp, int* status, cudaStream_t st, int sms) {
  const int grid = std::max(1, std::min(t1 - t0, sms * tc_blocks_per_sm<CMAX>()));
  gram_tc_kernel<CMAX><<<grid, TC_THREADS, TcSmem<CMAX>::BYTES + 1024, st>>>(
      work, gp.col_ptr, gp.cols, imgs, dbuf, jbuf, gp.tab0, gp.tab, gp.tabs, gp.scr, t0, t1, status);
}

}  // namespace

int gram_tc_max_cols() { return 128; }

int gram_tc_kind(int cols) { return cols <= 32 ? 1 : cols <= 64 ? 2 : 3; }

void configure_gram_tc() {
  cudaFuncSetAttribute(gram_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<32>::BYTES + 1024);
  cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<64>::BYTES + 1024);
  cudaFuncSetAttribute(gram_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<128>::BYTES + 1024);
  cudaGetLastError();
}

void launch_gram_tc(int kind, const TileWork* work, int t0, int t1, const int* jt_src, const SourceDev* srcs,
                    const ImageDev* imgs, const float* dbuf, const float* jbuf, const GramPlan& gp, int* status,
                    cudaStream_t st) {
  if (t1 <= t0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (kind == 1) launch_tc<32>(work, t0, t1, imgs, dbuf, jbuf, gp, status, st, sms);
  else if (kind == 2) launch_tc<64>(work, t0, t1, imgs, dbuf, jbuf, gp, status, st, sms);
  else launch_tc<128>(work, t0, t1, imgs, dbuf, jbuf, gp, status, st, sms);
}

}  // namespace ap
