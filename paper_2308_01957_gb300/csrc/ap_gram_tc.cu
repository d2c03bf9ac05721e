// J^T W J tile Grams on the fifth-generation tensor cores (tcgen05), float
// path (Sec. "Optimization methods": the Gauss-Newton matrix of LM).
//
// Pass 1 of the two-pass J^T W J (see ap_gram.cu) for tiles of up to 256
// free columns.  A CTA owns a run of 16 x 16 image tiles (persistent,
// grid-stride).  For one tile it streams the sqrt(w)-scaled Jacobian columns
// through shared memory in chunks of 32 pixels: every thread loads its pixel
// of some columns (coalesced rows of the column images), splits each value
// into a TF32 head and a TF32 tail and stores both, K-major with the 128-byte
// swizzle, into a double-buffered stage.  One thread issues the MMAs of a
// chunk -- head x head + head x tail + tail x head (3xTF32; the tail x tail
// term is below float32 rounding) -- accumulating the tile's C x C Gram in
// tensor memory, and commits them to the stage's mbarrier, so the loads of
// the next chunk overlap the MMAs of this one.  At the end of the tile the
// accumulator is read back (tcgen05.ld) and each entry stored into its
// source pair's scratch block exactly as the warp-MMA path does.
//
// Columns are cut into blocks of 128 (the MMA's M): NB = 1 block (C <= 128,
// one 128 x N accumulator, N = C rounded up to 16) or NB = 2 blocks
// (C <= 256: block pairs (0,0), (0,1), (1,1), three 128 x N accumulators).
// Rows and columns past C hold stale values of earlier tiles; they only reach
// accumulator rows and columns that are never read.
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
constexpr int TC_BLOCK = 128;                       // columns per block (MMA M)
constexpr uint32_t TC_WAIT_LIMIT = 1u << 20;        // mbarrier polls before giving up
constexpr int TC_MAX_SRC = 256;                     // sources reaching one tile (more: the warp-MMA kernel)

struct TcCol {           // one free column of the tile
  const float* base;     // the column image (its box, row pitch bw)
  int off0;              // offset of the tile's pixel (0, 0) in it (may lie outside the box)
  int bw;                // box width = row pitch
  uint32_t bounds;       // the box in tile coordinates, clamped to 0..16: rows [b0, b1), columns [b2, b3), a byte each
  int info;              // (local source << 8) | (free slot << 4) | free slots of that source
};

template <int NB>
struct TcSmem {
  static constexpr int ROWS = NB * TC_BLOCK;
  static constexpr int OPERAND = ROWS * 128;         // bytes of one operand (head or tail) of one stage
  static constexpr int STAGE = 2 * OPERAND;          // head + tail
  static constexpr int DATA = 2 * STAGE;             // two stages
  static constexpr int COLS = DATA;                  // TcCol[ROWS]
  static constexpr int SW = COLS + ROWS * (int)sizeof(TcCol);   // float sw[256]
  static constexpr int NFREE = SW + TILE_THREADS * 4;           // int nfree[TC_MAX_SRC + 1] (exclusive scan)
  static constexpr int MISC = (NFREE + (TC_MAX_SRC + 1) * 4 + 15) / 16 * 16;
  static constexpr int BYTES = MISC + 64;            // mbarriers, tensor-memory address, flags, stage column counts
  static constexpr int TMEM_COLS = NB == 1 ? 128 : 512;
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

// 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

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

template <int NB>
__global__ void __launch_bounds__(TC_THREADS, NB == 1 ? 3 : 1) gram_tc_kernel(
    const TileWork* __restrict__ work, const int* __restrict__ jt_src, const SourceDev* __restrict__ srcs,
    const ImageDev* __restrict__ imgs, const float* __restrict__ dbuf, const float* __restrict__ jbuf,
    const int64_t* __restrict__ tab0, const int64_t* __restrict__ tab_all, const int* __restrict__ tabs_all,
    double* __restrict__ scr, int t_first, int t_end, int* __restrict__ status) {
  using S = TcSmem<NB>;
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment of the swizzled operands
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TcCol* cols = reinterpret_cast<TcCol*>(sm + S::COLS);
  float* sw = reinterpret_cast<float*>(sm + S::SW);
  int* nfree = reinterpret_cast<int*>(sm + S::NFREE);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + S::MISC);        // [2]: a stage was filled (8 producer warps)
  uint64_t* empty = full + 2;                                          // [2]: its MMAs completed (commit)
  uint64_t* acc_full = full + 4;                                       // the tile's accumulator is complete (commit)
  uint64_t* acc_empty = full + 5;                                      // the accumulator was read (8 producer warps)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + S::MISC + 48);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::MISC + 52);
  int* stage_cols = reinterpret_cast<int*>(sm + S::MISC + 56);        // [2]: C of the chunk in each stage

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[k])), "r"(TC_PRODUCERS / 32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[k])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(acc_full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(acc_empty)), "r"(TC_PRODUCERS / 32) : "memory");
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
          const int npad = C <= 16 ? 16 : ((C + 15) & ~15);
          const uint32_t a_hi = base_addr + st * S::STAGE, a_lo = a_hi + S::OPERAND;
#pragma unroll
          for (int kk = 0; kk < TC_CHUNK / 8; ++kk) {
            const uint32_t kb = kk * 32;   // 8 TF32 values per MMA step
            for (int pr = 0; pr < (NB == 1 ? 1 : 3); ++pr) {
              const int I = NB == 1 ? 0 : (pr == 2 ? 1 : 0);
              const int J = NB == 1 ? 0 : (pr == 0 ? 0 : 1);
              const int N = NB == 1 ? npad : (J == 0 ? TC_BLOCK : (C - TC_BLOCK <= 16 ? 16 : ((C - TC_BLOCK + 15) & ~15)));
              const uint32_t id = tf32_idesc(TC_BLOCK, N);
              const uint32_t d = tmem + pr * TC_BLOCK;
              const uint64_t ah = sw128_desc(a_hi + I * TC_BLOCK * 128 + kb);
              const uint64_t al = sw128_desc(a_lo + I * TC_BLOCK * 128 + kb);
              const uint64_t bh = sw128_desc(a_hi + J * TC_BLOCK * 128 + kb);
              const uint64_t bl = sw128_desc(a_lo + J * TC_BLOCK * 128 + kb);
              mma_tf32(d, ah, bh, id, (ch > 0 || kk > 0) ? 1u : 0u);
              mma_tf32(d, ah, bl, id, 1u);
              mma_tf32(d, al, bh, id, 1u);
            }
          }
          mma_commit(smem_u32(&empty[st]));     // the stage may be refilled once these complete
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
      const int L = w.e1 - w.e0 <= TC_MAX_SRC ? w.e1 - w.e0 : 0;   // more sources: reported below
      producers_sync();   // the previous tile's epilogue no longer reads cols
      for (int e = tid; e < L; e += TC_PRODUCERS) {
        const SourceDev& sd = srcs[jt_src[w.e0 + e]];
        int nf = 0;
#pragma unroll
        for (int k = 0; k < MAX_SLOTS; ++k) nf += (k < sd.nslot && sd.pidx[k] >= 0);
        nfree[e + 1] = nf;
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
      if (warp == 0) {
        // exclusive scan of the free-column counts (one warp, 32 at a time)
        int run = 0;
        if (lane == 0) nfree[0] = 0;
        for (int e0 = 0; e0 < L; e0 += 32) {
          int v = e0 + lane < L ? nfree[e0 + lane + 1] : 0;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
          }
          if (e0 + lane < L) nfree[e0 + lane + 1] = run + v;
          run += __shfl_sync(0xffffffffu, v, 31);
        }
      }
      producers_sync();
      const int C = L > 0 ? nfree[L] : 0;
      const bool fits = C <= NB * TC_BLOCK && w.e1 - w.e0 <= TC_MAX_SRC;
      if (!fits && tid == 0) atomicCAS(status, 0, AP_ERR_ARG);
      const int Cu = fits ? C : 0;   // a tile that does not fit is reduced to no columns
      for (int e = tid; e < L && fits; e += TC_PRODUCERS) {
        const SourceDev& sd = srcs[jt_src[w.e0 + e]];
        const int* bx = sd.conv ? sd.sup : sd.box;
        const int64_t area = (int64_t)(bx[1] - bx[0]) * (bx[3] - bx[2]);
        const float* b0 = sd.conv ? jbuf + sd.j_off : dbuf + sd.d_off;
        const int nf = nfree[e + 1] - nfree[e];
        const int bw = bx[3] - bx[2];
        auto clampt = [](int v) { return (uint32_t)(v < 0 ? 0 : (v > TILE ? TILE : v)); };
        const uint32_t bounds = clampt(bx[0] - w.r0) | (clampt(bx[1] - w.r0) << 8) | (clampt(bx[2] - w.c0) << 16) |
                                (clampt(bx[3] - w.c0) << 24);
        const int off0 = (w.r0 - bx[0]) * bw + (w.c0 - bx[2]);
        int m = nfree[e], f = 0;
        for (int k = 0; k < MAX_SLOTS; ++k) {
          if (k >= sd.nslot || sd.pidx[k] < 0) continue;
          TcCol col;
          col.base = b0 + k * area;
          col.off0 = off0;
          col.bw = bw;
          col.bounds = bounds;
          col.info = (e << 8) | (f << 4) | nf;
          cols[m] = col;
          ++m;
          ++f;
        }
      }
      producers_sync();
      dead = dead || *abort_flag;
      // ---- chunks of 32 pixels (two image rows of the tile); the values of
      // chunk ch + 1 are loaded into registers while chunk ch is stored
      // (warp w holds columns w, w + 8, ...)
      constexpr int MAXU = NB * TC_BLOCK / (TC_PRODUCERS / 32);
      float cur[MAXU], nxt[MAXU];
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
      load_chunk(0, cur);
      for (int ch = 0; ch < TC_NCHUNK; ++ch, ++g) {
        const int st = g & 1;
        if (ch + 1 < TC_NCHUNK) load_chunk(ch + 1, nxt);
        // the stage is free once the MMAs that last read it have completed
        int ok = 1;
        if (lane == 0 && g >= 2 && !dead) ok = mbar_wait(smem_u32(&empty[st]), ((g >> 1) - 1) & 1) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) {
            atomicCAS(status, 0, AP_ERR_TIMEOUT);
            *abort_flag = 1;
          }
          dead = true;
        }
        if (dead) continue;
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
#pragma unroll
        for (int u = 0; u < MAXU; ++u) cur[u] = nxt[u];
        if (tid == 0) stage_cols[st] = Cu;
        // the stores are read by the tensor cores (async proxy), then the
        // warp's arrival releases them to the MMA warp
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&full[st]));
      }
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
      // warp w reads lanes 32 (w % 4) .. +31 of every accumulator, the columns
      // split between warps 0-3 and 4-7
      const int64_t* tab = tab_all + tab0[tile];
      const int* tabs = tabs_all + tab0[tile];
      const int q = warp & 3, half = warp >> 2;
      const int npad = Cu <= 16 ? 16 : ((Cu + 15) & ~15);
      for (int pr = 0; pr < (NB == 1 ? 1 : 3); ++pr) {
        const int I = NB == 1 ? 0 : (pr == 2 ? 1 : 0);
        const int J = NB == 1 ? 0 : (pr == 0 ? 0 : 1);
        const int N = NB == 1 ? npad : (J == 0 ? TC_BLOCK : (Cu - TC_BLOCK <= 16 ? 16 : ((Cu - TC_BLOCK + 15) & ~15)));
        const int ca = I * TC_BLOCK + 32 * q + lane;
        const int nh = ((N / 16) + 1) / 2 * 16;   // columns of the first half (a multiple of 16)
        const int n0 = half ? nh : 0, n1 = half ? N : nh;
        if (J * TC_BLOCK + n0 >= Cu || I * TC_BLOCK + 32 * q >= Cu) continue;   // nothing this warp stores
        for (int cb0 = n0; cb0 < n1 && J * TC_BLOCK + cb0 < Cu; cb0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(pr * TC_BLOCK + cb0), v);
          if (ca < Cu) {
            const int ia = cols[ca].info;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int cb = J * TC_BLOCK + cb0 + u;
              if (cb < Cu && cb >= ca) tc_store((double)v[u], ia, cols[cb].info, L, tab, tabs, scr);
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
template <int NB>
int tc_blocks_per_sm() {
  int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, thr_sm = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, gram_tc_kernel<NB>) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int per_block = TcSmem<NB>::BYTES + 1024 + (int)fa.sharedSizeBytes + reserved;
  int n = smem_sm / per_block;
  n = std::min(n, regs_sm / std::max(1, fa.numRegs * TC_THREADS));
  n = std::min(n, thr_sm / TC_THREADS);
  n = std::min(n, 512 / TcSmem<NB>::TMEM_COLS);
  return std::max(n, 1);
}

}  // namespace

int gram_tc_max_cols() { return 2 * TC_BLOCK; }

int gram_tc_blocks(int cols) { return cols <= TC_BLOCK ? 1 : 2; }

void configure_gram_tc() {
  cudaFuncSetAttribute(gram_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<1>::BYTES + 1024);
  cudaFuncSetAttribute(gram_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<2>::BYTES + 1024);
  cudaGetLastError();
}

void launch_gram_tc(int nb, const TileWork* work, int t0, int t1, const int* jt_src, const SourceDev* srcs,
                    const ImageDev* imgs, const float* dbuf, const float* jbuf, const GramPlan& gp, int* status,
                    cudaStream_t st) {
  if (t1 <= t0) return;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = nb == 1 ? tc_blocks_per_sm<1>() : tc_blocks_per_sm<2>();
  const int grid = std::max(1, std::min(t1 - t0, sms * std::max(per_sm, 1)));
  if (nb == 1)
    gram_tc_kernel<1><<<grid, TC_THREADS, TcSmem<1>::BYTES + 1024, st>>>(
        work, jt_src, srcs, imgs, dbuf, jbuf, gp.tab0, gp.tab, gp.tabs, gp.scr, t0, t1, status);
  else
    gram_tc_kernel<2><<<grid, TC_THREADS, TcSmem<2>::BYTES + 1024, st>>>(
        work, jt_src, srcs, imgs, dbuf, jbuf, gp.tab0, gp.tab, gp.tabs, gp.scr, t0, t1, status);
}

}  // namespace ap
