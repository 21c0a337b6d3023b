// Multi-right-hand-side Vanka local products on the 5th-generation tensor cores (a6'' of the hot path):
// Y_T = J_T^{-1} T_T for every cell T of a level and a 32-column block T_T of gathered residuals
// (Eq. LocVanka applied to 32 right-hand sides that share the cell inverses of Sec. 4.3).
//
// One persistent CTA per SM walks its cells in a warp-specialised pipeline:
//   warp 0      streams the cell's stored BF16 inverse into shared memory with TMA
//               (cp.async.bulk.tensor, one 64-row box per 64 stored rows, two-stage ring);
//   warp 1      allocates the tensor memory and issues tcgen05.mma (one elected thread):
//               D[128 rows][64 cols] += Inv[rows][16 k] x B[16 k][64 cols] over the contraction, FP32
//               accumulators in TMEM (two accumulator sets, so the epilogue of one cell overlaps the
//               products of the next);
//   warps 2-13  gather the 32 residual columns of the cell's DoFs (one 128-byte line per DoF of the
//               interleaved [N][32] block, each value already split into BF16 hi + lo parts by the
//               kernel that wrote it: t = hi + lo to about 2^-16 relative, so the only rounding of
//               note is the stored inverse's) and write them as the B operand: columns 0-31 hi,
//               32-63 lo; the loads of the next cell are in flight while the current one is written
//               (twelve warps, two 8-row chunks each: 262 us per 16,128-cell sweep against 324 us
//               with eight warps and three chunks each; sixteen warps: 263 us);
//   warps 14-17 read the accumulators back with tcgen05.ld (one TMEM lane per output row), add the
//               hi and lo halves and store Y in FP32, coalesced through a swizzled staging tile.
//
// Operand layouts. The inverse is stored column-major (element (i, j) at j*ld + i). TMA box b copies rows
// 64b..64b+63 (128 bytes) of every column j into shared memory with the 128-byte swizzle: box b holds
// RJ rows (one per column j, rows past n zero) of 64 i-values, in 8-row atoms of 1024 bytes. The same
// bytes serve both products:
//   forward  Inv   (M = i, K = j): MN-major A, 128B swizzle; MN atoms of 64 i one box apart (LBO),
//            8-row K groups 1024 B apart (SBO); a 16-wide K step moves two atoms;
//   adjoint  Inv^T (M = j, K = i): K-major A, 128B swizzle; 8-row M groups 1024 B apart (SBO); a
//            16-wide K step moves 32 bytes inside the 128-byte row, four steps per box.
// Output tiles of 128 rows start at rows 0 and 64 (the second only for ld > 128; its rows below 128
// repeat tile 0 and are skipped in the epilogue), for i in the forward and j in the adjoint product.
// B (gathered columns, written by the gather warps): K-major without swizzle, core matrices of 8 columns x 16
// bytes, core (n-group g, k-chunk q) at q*1024 + g*128. Rows past n of B and of every box stay zero
// (written once), so the padded contraction adds nothing.
//
// Every wait on an mbarrier gives up after a bounded number of polls, sets the level's error word and
// lets the CTA finish (after waiting, again bounded, for its own copies and products in flight), so a
// lost arrival shows up as STM_ERR_CUDA at the next synchronising call instead of a hung GPU.
#include <cuda.h>

#include <cstdint>

#include "internal.h"

namespace stm {
namespace {

constexpr int kNR = 32;             // right-hand sides per multi-vector
constexpr int kThreads = 18 * 32;   // roles: TMA, MMA, 12 gather warps, 4 epilogue warps
constexpr int kGatherWarps = 12;
constexpr int kGatherRounds = (24 + kGatherWarps - 1) / kGatherWarps;  // 8-row chunks per warp (ld <= 192)
constexpr int kEpiWarp0 = 2 + kGatherWarps;
constexpr int kStages = 2;          // inverse and B stages
constexpr int kTmemCols = 256;      // 2 accumulator sets x 2 output tiles x 64 columns
constexpr uint64_t kWaitNs = 1000000000ull;  // one second per wait at most

struct TcGeom {
  int n, ld;          // local size, stored rows per column (multiple of 8, at most 192)
  int KS;             // 16-wide contraction steps: ceil(n / 16)
  int MT;             // output tiles of 128 rows: 1 (ld <= 128) or 2
  int RJ;             // rows (columns j of the inverse) of one box in shared memory: 128 or 192
  int BOXB;           // bytes of one box: RJ * 128
  int NB;             // boxes TMA fills per cell: ceil(ld / 64)
  unsigned a_bytes;   // boxes allocated per stage (2 or 3, zero beyond NB) x BOXB
  unsigned b_bytes;   // KS * 2048 (16 k x 64 columns x 2 B per step)
  unsigned tx_bytes;  // bytes TMA delivers per cell: NB * 64 * n * 2 (out-of-range rows count, as zeros)
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity, for at most kWaitNs of wall time; false (and the error
// word set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255u) == 0 && global_ns() - t0 > kWaitNs) break;
  }
  atomicOr(err, code);
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of tcgen05 (no swizzle): start, leading-dimension byte offset
// (between core matrices adjacent along K), stride-dimension byte offset (adjacent along M/N), all in
// 16-byte units, and the fixed descriptor version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t start, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((start >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// The same with the 128-byte swizzle (layout type 2 in bits 61-63); atoms must start on 1024-byte boundaries.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t start, uint32_t lbo, uint32_t sbo) {
  return sdesc(start, lbo, sbo) | (2ull << 61);
}
// Instruction descriptor of tcgen05.mma kind::f16: D in FP32, A and B in BF16, A MN-major (a_mn) or
// K-major, B K-major, N columns, M rows.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct SmemLayout {
  uint32_t a[kStages], b[kStages], stage;  // byte offsets from the 1024-aligned base
  uint32_t bars;                           // 12 mbarriers
  uint32_t tmem_slot;
  uint32_t total;
};
__host__ __device__ inline SmemLayout smem_layout(const TcGeom& g) {
  SmemLayout s;
  uint32_t off = 0;
  for (int i = 0; i < kStages; ++i) {
    s.a[i] = off;
    off += (g.a_bytes + 1023u) & ~1023u;
  }
  for (int i = 0; i < kStages; ++i) {
    s.b[i] = off;
    off += (g.b_bytes + 1023u) & ~1023u;
  }
  s.stage = off;
  off += 4 * 32 * 128;  // epilogue staging: 4 warps x 32 rows x 32 floats
  s.bars = off;
  off += 12 * 8;
  s.tmem_slot = off;
  off += 16;
  s.total = off;
  return s;
}

// Barrier indices
enum { FULL_A = 0, EMPTY_A = 2, FULL_B = 4, EMPTY_B = 6, TM_FULL = 8, TM_EMPTY = 10 };

// FUSED = false: 32 forward columns, Y = Inv T. FUSED = true: columns 0-15 forward (Y = Inv T), columns
// 16-31 adjoint (Y = Inv^T T) from the same inverse tile: B holds [forward hi | forward lo | adjoint hi |
// adjoint lo] (16 columns each); per output tile one MMA chain reads the tile as Inv (MN-major A) against
// B columns 0-31 and one reads it as Inv^T (K-major A) against B columns 32-63.
template <bool FUSED>
__global__ void __launch_bounds__(kThreads, 1) k_vanka_mrhs_tc5(const __grid_constant__ CUtensorMap inv_map,
                                                                 const int* __restrict__ idx,
                                                                 const uint32_t* __restrict__ T16,
                                                                 float* __restrict__ Y, int ncells, TcGeom g,
                                                                 int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const SmemLayout L = smem_layout(g);
  const uint32_t sbase = saddr(base);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto bar = [&](int i) -> uint32_t { return sbase + L.bars + 8u * (uint32_t)i; };

  // zero both A and B stages once: rows past n in every chunk and chunks past ld/8 are never written
  // again and must read as zero in the padded contraction
  {
    uint4* z = reinterpret_cast<uint4*>(base);
    const uint32_t words = L.stage / 16u;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_async_smem();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar(FULL_A + s), 1);
      mbar_init(bar(EMPTY_A + s), 1);
      mbar_init(bar(FULL_B + s), kGatherWarps);
      mbar_init(bar(EMPTY_B + s), 1);
      mbar_init(bar(TM_FULL + s), 1);
      mbar_init(bar(TM_EMPTY + s), 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + L.tmem_slot),
                 "r"((uint32_t)kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(base + L.tmem_slot);

  if (warp == 0) {
    // ---- TMA producer -------------------------------------------------------------------------
    if (lane == 0) {
      int it = 0, last_c[kStages] = {-1, -1};
      bool ok = true;
      for (int c = blockIdx.x; c < ncells && ok; c += gridDim.x, ++it) {
        const int s = it & 1;
        const uint32_t u = (uint32_t)(it >> 1) & 1u;
        ok = mbar_wait(bar(EMPTY_A + s), u ^ 1u, err, 1);
        if (!ok) break;
        mbar_expect_tx(bar(FULL_A + s), g.tx_bytes);
        for (int b = 0; b < g.NB; ++b)
          tma_load_3d(sbase + L.a[s] + (uint32_t)b * (uint32_t)g.BOXB, &inv_map, 64 * b, 0, c, bar(FULL_A + s));
        last_c[s] = it;
      }
      // the copies of the last two cells must have landed before the CTA may finish
      for (int s = 0; s < kStages; ++s)
        if (last_c[s] >= 0) mbar_wait(bar(FULL_A + s), (uint32_t)(last_c[s] >> 1) & 1u, err, 16);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ---------------------------------------------------------------------------
    if (lane == 0) {
      const uint32_t id = idesc_bf16(128, 64, true);
      const uint32_t id_f = idesc_bf16(128, 32, true), id_a = idesc_bf16(128, 32, false);
      int it = 0, last = -1;
      for (int c = blockIdx.x; c < ncells; c += gridDim.x, ++it) {
        const int s = it & 1;
        const uint32_t u = (uint32_t)(it >> 1) & 1u;
        if (!mbar_wait(bar(FULL_A + s), u, err, 2)) break;
        if (!mbar_wait(bar(FULL_B + s), u, err, 2)) break;
        if (!mbar_wait(bar(TM_EMPTY + s), u ^ 1u, err, 2)) break;
        tc_fence_after();
        const uint32_t a0 = sbase + L.a[s], b0 = sbase + L.b[s];
        for (int t = 0; t < g.MT; ++t) {
          const uint32_t d = tmem + (uint32_t)(s * 128 + t * 64);
          // forward: Inv rows i = 64t .. 64t + 127 = boxes t, t + 1; K = j in whole 8-row atoms
          const uint32_t af = a0 + (uint32_t)t * (uint32_t)g.BOXB;
          for (int ks = 0; ks < g.KS; ++ks) {
            const uint64_t ad = sdesc_sw128(af + (uint32_t)ks * 2048u, (uint32_t)g.BOXB, 1024u);
            const uint64_t bd = sdesc(b0 + (uint32_t)ks * 2048u, 1024u, 128u);
            if (!FUSED) mma_bf16(d, ad, bd, id, ks > 0 ? 1u : 0u);
            else mma_bf16(d, ad, bd, id_f, ks > 0 ? 1u : 0u);
          }
          if (FUSED) {
            // adjoint: Inv^T rows j = 64t .. 64t + 127 of every box, K = i: 32 bytes per step inside a box
            for (int ks = 0; ks < g.KS; ++ks) {
              const uint32_t aj = a0 + (uint32_t)(ks >> 2) * (uint32_t)g.BOXB + (uint32_t)t * 64u * 128u +
                                  (uint32_t)(ks & 3) * 32u;
              const uint64_t ad = sdesc_sw128(aj, 16u, 1024u);
              const uint64_t bd = sdesc(b0 + (uint32_t)ks * 2048u + 512u, 1024u, 128u);
              mma_bf16(d + 32u, ad, bd, id_a, ks > 0 ? 1u : 0u);
            }
          }
        }
        mma_commit(bar(EMPTY_A + s));
        mma_commit(bar(EMPTY_B + s));
        mma_commit(bar(TM_FULL + s));
        last = it;
      }
      // products in flight must be complete before the tensor memory is released
      if (last >= 0) mbar_wait(bar(TM_FULL + (last & 1)), (uint32_t)(last >> 1) & 1u, err, 32);
    }
  } else if (warp < kEpiWarp0) {
    // ---- gather: 32 packed columns per local DoF -> BF16 hi (B columns 0-31) + lo (32-63) ---------
    const int gw = warp - 2;
    const int nchunks = 2 * g.KS;  // 8-row k-chunks of the B tile
    uint32_t cur[kGatherRounds][8], nxt[kGatherRounds][8];
    auto load_cell = [&](int c, uint32_t (*v)[8]) {
      const int* ic = idx + (long long)c * g.n;
#pragma unroll
      for (int r = 0; r < kGatherRounds; ++r) {
        const int q = gw + r * kGatherWarps;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int k = 8 * q + kk;
          v[r][kk] = (q < nchunks && k < g.n) ? __ldg(T16 + (long long)__ldg(ic + k) * kNR + lane) : 0u;
        }
      }
    };
    if (blockIdx.x < ncells) load_cell(blockIdx.x, cur);
    int it = 0;
    for (int c = blockIdx.x; c < ncells; c += gridDim.x, ++it) {
      const int s = it & 1;
      const uint32_t u = (uint32_t)(it >> 1) & 1u;
      if (c + (int)gridDim.x < ncells) load_cell(c + gridDim.x, nxt);  // next cell's loads in flight
      if (!__all_sync(0xffffffffu, mbar_wait(bar(EMPTY_B + s), u ^ 1u, err, 4))) break;
      unsigned char* bs = base + L.b[s];
#pragma unroll
      for (int r = 0; r < kGatherRounds; ++r) {
        const int q = gw + r * kGatherWarps;
        if (q >= nchunks) continue;
        // 8 consecutive k of this lane's column: hi halves into one 16-byte row, lo halves into another
        const uint4 H = make_uint4(__byte_perm(cur[r][0], cur[r][1], 0x5410), __byte_perm(cur[r][2], cur[r][3], 0x5410),
                                   __byte_perm(cur[r][4], cur[r][5], 0x5410), __byte_perm(cur[r][6], cur[r][7], 0x5410));
        const uint4 Lo = make_uint4(__byte_perm(cur[r][0], cur[r][1], 0x7632), __byte_perm(cur[r][2], cur[r][3], 0x7632),
                                    __byte_perm(cur[r][4], cur[r][5], 0x7632), __byte_perm(cur[r][6], cur[r][7], 0x7632));
        // B column of this lane's hi and lo parts; core matrix (n-group, k-chunk q) at q*1024 + group*128,
        // row (n % 8) at 16 * (n % 8)
        const int nh = FUSED ? (lane < 16 ? lane : 16 + lane) : lane;
        const int nl = FUSED ? (lane < 16 ? 16 + lane : 32 + lane) : 32 + lane;
        *reinterpret_cast<uint4*>(bs + q * 1024 + (nh >> 3) * 128 + (nh & 7) * 16) = H;
        *reinterpret_cast<uint4*>(bs + q * 1024 + (nl >> 3) * 128 + (nl & 7) * 16) = Lo;
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(FULL_B + s));
#pragma unroll
      for (int r = 0; r < kGatherRounds; ++r)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) cur[r][kk] = nxt[r][kk];
    }
  } else {
    // ---- epilogue: TMEM -> FP32 Y[c][row][32] ----------------------------------------------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    float* stg = reinterpret_cast<float*>(base + L.stage) + (warp - kEpiWarp0) * 32 * 32;
    const uint32_t stg_s = saddr(stg);
    int it = 0;
    for (int c = blockIdx.x; c < ncells; c += gridDim.x, ++it) {
      const int s = it & 1;
      const uint32_t u = (uint32_t)(it >> 1) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(bar(TM_FULL + s), u, err, 8))) break;
      tc_fence_after();
      for (int t = 0; t < g.MT; ++t) {
        const int row0 = 64 * t + 32 * q;  // first output row of this warp
        if (t == 1 && row0 + 31 < 128) continue;                  // rows already written by tile 0
        if (row0 >= g.n) continue;
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * 128 + t * 64);
        float hi[32], lo[32];
        tmem_ld32(ta, hi);
        tmem_ld32(ta + 32u, lo);
        tmem_wait_ld();
        if (FUSED) {
          // accumulator columns: 0-15 forward hi, 16-31 forward lo, 32-47 adjoint hi, 48-63 adjoint lo;
          // regroup as hi = [forward hi | adjoint hi], lo = [forward lo | adjoint lo]
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float fl = hi[16 + k];
            hi[16 + k] = lo[k];
            lo[k] = fl;
          }
        }
        // own row into the staging tile, 16-byte chunks XOR-swizzled by row
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const float4 w = make_float4(hi[4 * ch] + lo[4 * ch], hi[4 * ch + 1] + lo[4 * ch + 1],
                                       hi[4 * ch + 2] + lo[4 * ch + 2], hi[4 * ch + 3] + lo[4 * ch + 3]);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(stg_s + lane * 128 + ((ch ^ (lane & 7)) * 16)),
                       "f"(w.x), "f"(w.y), "f"(w.z), "f"(w.w)
                       : "memory");
        }
        __syncwarp();
        // 4 rows x 128 B per store instruction
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = 4 * i + (lane >> 3), ch = lane & 7;
          float4 w;
          asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                       : "=f"(w.x), "=f"(w.y), "=f"(w.z), "=f"(w.w)
                       : "r"(stg_s + r * 128 + ((ch ^ (r & 7)) * 16))
                       : "memory");
          const int row = row0 + r;
          if (row < g.n && (t == 0 || row >= 128))
            *reinterpret_cast<float4*>(Y + ((long long)c * g.n + row) * kNR + 4 * ch) = w;
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(TM_EMPTY + s));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  __syncwarp();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTmemCols)
                 : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

stm_status encode_fn(EncodeTiledFn* out) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return STM_ERR_CUDA;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = fn;
  return STM_OK;
}

TcGeom tc_geom(int n, int ld) {
  TcGeom g;
  g.n = n;
  g.ld = ld;
  g.KS = (n + 15) / 16;
  g.MT = ld > 128 ? 2 : 1;
  g.RJ = g.MT == 2 ? 192 : 128;
  g.BOXB = g.RJ * 128;
  g.NB = (ld + 63) / 64;
  g.a_bytes = (unsigned)((g.MT == 2 ? 3 : 2) * g.BOXB);
  g.b_bytes = (unsigned)(g.KS * 2048);
  g.tx_bytes = (unsigned)(g.NB * 64 * n * 2);
  return g;
}


// Self-test of the bounded wait: one thread waits for a phase of an mbarrier that nothing arrives on.
// The wait gives up after kWaitNs, sets the error word and the kernel returns normally.
__global__ void k_bounded_wait_selftest(int* err) {
  __shared__ uint64_t never;
  if (threadIdx.x == 0) {
    mbar_init(saddr(&never), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(saddr(&never), 0u, err, 128);
  }
}

}  // namespace

// The tensor-core path applies when the stored BF16 columns are whole 16-byte units (TMA strides) and
// the cell fits two 128-row output tiles.
bool mrhs_tc_supported(int n, int ld) { return ld % 8 == 0 && ld <= 192 && n <= ld && n >= 1; }
bool mrhs_tc_fused_supported(int n, int ld) { return mrhs_tc_supported(n, ld); }

stm_status mrhs_tc_apply(const Level& L, int ld, const uint32_t* T16, float* Y, int* err, cudaStream_t s, bool fused) {
  if (!mrhs_tc_supported(L.n, ld) || (fused && !mrhs_tc_fused_supported(L.n, ld))) {
    set_error("multi-RHS tensor-core product: unsupported local size");
    return STM_ERR_INVALID_ARG;
  }
  if (L.C == 0) return STM_OK;
  EncodeTiledFn enc = nullptr;
  STM_TRY(encode_fn(&enc));
  // the level's BF16 inverses as a 3-D tensor [C][n columns][ld rows], box = 64 rows x n columns
  alignas(64) CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)L.n, (cuuint64_t)L.C};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * L.n * 2};
  const cuuint32_t box[3] = {64, (cuuint32_t)L.n, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, L.inv, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed for the cell inverses (code " + std::to_string((int)r) + ")");
    return STM_ERR_CUDA;
  }
  const TcGeom g = tc_geom(L.n, ld);
  const SmemLayout sl = smem_layout(g);
  const int smem = (int)sl.total + 1024;
  const int blocks = std::min(L.C, sm_count());
  if (fused) {
    STM_CUDA(cudaFuncSetAttribute(k_vanka_mrhs_tc5<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_vanka_mrhs_tc5<true><<<blocks, kThreads, smem, s>>>(map, L.idx, T16, Y, L.C, g, err);
  } else {
    STM_CUDA(cudaFuncSetAttribute(k_vanka_mrhs_tc5<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_vanka_mrhs_tc5<false><<<blocks, kThreads, smem, s>>>(map, L.idx, T16, Y, L.C, g, err);
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status bounded_wait_selftest(int* err, cudaStream_t s) {
  k_bounded_wait_selftest<<<1, 32, 0, s>>>(err);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

}  // namespace stm
