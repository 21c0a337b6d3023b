// Direct coarse solve of Algorithm 1 (d_1 = J_1^{-1} r_1, or J_1^{-T} r_1 in the adjoint V-cycle) through
// the block LU factors of J_1 in x-slab order (kernels_factor.cu), for coarse levels too large for the
// dense explicit inverse to pay (3D: 18,000 DoFs, 2.6 GB as a dense inverse).
//
// In slab order J_1 is block tridiagonal; with S_b the Schur complements and A_{b,c} its blocks,
//   J_1 = L U,  L: diagonal S_b, sub-diagonal A_{b,b-1};  U: unit diagonal, super-diagonal W_b = S_b^{-1} A_{b,b+1}.
// Forward solve  J_1 x = r:   z_b = S_b^{-1} r_b (all slabs at once);  y_b = z_b - G_b y_{b-1}, G_b = S_b^{-1} A_{b,b-1};
//                              x_b = y_b - W_b x_{b+1}.
// Transposed     J_1^T x = r: w_b = r_b - P_b w_{b-1}, P_b = W_{b-1}^T;  s_b = S_b^{-T} w_b (all slabs);
//                              x_b = s_b - Q_b x_{b+1}, Q_b = S_b^{-T} A_{b+1,b}^T.
// Every matrix is stored row-major per block, so each product is a warp-per-row dot product over
// contiguous rows. One cooperative kernel runs the three phases. Instead of a grid-wide barrier between
// the dependent slab steps (2 (nx - 1) of them), every finished row bumps a per-slab, per-phase counter
// with release semantics and a warp starts a row once the counters of the slabs it reads are complete
// (acquire): a step waits only for the rows it needs, about a microsecond, where a grid-wide barrier cost
// about ten. While it waits, a warp has already prefetched its next row into L2. Every wait gives up after
// one second of wall time, sets the hierarchy's error word and lets the kernel finish. The counters are
// cleared at the end for the next launch. A 32-column variant (interleaved [N][32] multi-vectors, lane =
// column) serves the multi-RHS V-cycle.
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace stm {
namespace {

constexpr unsigned long long kFlagWaitNs = 1000000000ull;

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct SlabView {
  int nx;
  long long n;
  const long long* off;   // [nx + 1] first permuted row of every slab
  const long long* pos;   // [6][nx] block offsets in store: Sinv, G, W, Sinvt, P, Q (-1: absent)
  const int* rowslab;     // [n] slab of every permuted row
  const int* perm;        // [n] permuted position of every row of J_1
  const double* store;
  unsigned* cnt;          // [3][nx] finished rows per phase and slab (zero between launches)
  int* err;
};

enum { M_SINV = 0, M_G = 1, M_W = 2, M_SINVT = 3, M_P = 4, M_Q = 5 };

// Lane 0 waits until the counter reaches target (acquire), then the warp proceeds; false on timeout.
__device__ bool wait_count(const unsigned* c, unsigned target, int lane, int* err) {
  int ok = 1;
  if (lane == 0 && ld_acquire(c) < target) {
    const unsigned long long t0 = global_ns();
    while (ld_acquire(c) < target) {
      if (global_ns() - t0 > kFlagWaitNs) {
        atomicOr(err, 64);
        ok = 0;
        break;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// sum_k M[row][k] x[k] over a warp (NR = 1: lanes split k, butterfly sum; NR = 32: lane = column)
template <int NR>
__device__ __forceinline__ double row_product(const double* __restrict__ m, const double* x, long long nc, int lane) {
  // x was written by other warps during this launch: read it from L2 (never from a stale L1 line)
  double acc = 0.0;
  if (NR == 1) {
    for (long long k = lane; k < nc; k += 32) acc = fma(__ldg(m + k), __ldcg(x + k), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  } else {
    for (long long k = 0; k < nc; ++k) acc = fma(__ldg(m + k), __ldcg(x + k * 32 + lane), acc);
  }
  return acc;
}

__device__ __forceinline__ void prefetch_row(const double* m, long long nc, int lane) {
  const char* row = reinterpret_cast<const char*>(m);
  for (long long o = (long long)lane * 128; o < nc * 8; o += 32 * 128) prefetch_l2(row + o);
}

template <int NR>
__global__ void __launch_bounds__(256) k_coarse_slab(SlabView S, const double* __restrict__ r, double* __restrict__ d,
                                                     double* __restrict__ u, double* __restrict__ v, int transpose) {
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  const int nx = S.nx;
  auto mat = [&](int kind, int b) -> const double* { return S.store + S.pos[kind * nx + b]; };
  auto rows = [&](int b) -> unsigned { return (unsigned)(S.off[b + 1] - S.off[b]); };
  unsigned* c_batch = S.cnt;           // batched phase: z_b (forward) / s_b (transposed)
  unsigned* c_up = S.cnt + nx;         // chain over increasing b: y_b (forward) / w_b (transposed)
  unsigned* c_down = S.cnt + 2 * nx;   // chain over decreasing b: x_b
  bool ok = true;
  // gather into slab order
  for (long long e = gt; e < S.n * NR; e += nt) {
    const long long i = e / NR;
    u[(long long)S.perm[i] * NR + (e - i * NR)] = r[e];
  }
  grid.sync();

  // batched phase: row `row` of out = M_b(row) in_b; rows across all slabs; with wait_up, a row of
  // slab b waits for slab b of the increasing chain first (transposed solve)
  auto batched = [&](int kind, const double* in, double* out, bool wait_up) {
    for (long long row = gw; row < S.n && ok; row += nw) {
      const int b = S.rowslab[row];
      const long long nb = S.off[b + 1] - S.off[b], c0 = S.off[b];
      if (wait_up && !wait_count(c_up + b, rows(b), lane, S.err)) {
        ok = false;
        break;
      }
      const double acc = row_product<NR>(mat(kind, b) + (row - c0) * nb, in + c0 * NR, nb, lane);
      if (NR == 1) {
        if (lane == 0) out[row] = acc;
      } else {
        out[row * 32 + lane] = acc;
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) red_release_add(c_batch + b, 1u);
    }
  };
  // one step of a chain: rows of slab b: vec_b -= M_b vec_c, after slab c of this chain and slab b of
  // the phase that wrote vec_b are complete
  auto chain_row = [&](int kind, int b, int c, double* vec, unsigned* c_own, const unsigned* c_prev_b,
                       unsigned target_prev_b) {
    const long long nb = S.off[b + 1] - S.off[b], nc = S.off[c + 1] - S.off[c];
    for (long long rr = gw; rr < nb && ok; rr += nw) {
      const double* m = mat(kind, b) + rr * nc;
      prefetch_row(m, nc, lane);
      if ((c_prev_b && !wait_count(c_prev_b + b, target_prev_b, lane, S.err)) ||
          !wait_count(c_own + c, rows(c), lane, S.err)) {
        ok = false;
        break;
      }
      const double acc = row_product<NR>(m, vec + S.off[c] * NR, nc, lane);
      const long long row = S.off[b] + rr;
      if (NR == 1) {
        if (lane == 0) vec[row] = __ldcg(vec + row) - acc;
      } else {
        vec[row * 32 + lane] = __ldcg(vec + row * 32 + lane) - acc;
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) red_release_add(c_own + b, 1u);
    }
  };

  if (!transpose) {
    batched(M_SINV, u, v, false);
    // y_0 = z_0: slab 0 of the increasing chain is complete once its batched rows are
    if (gw == 0 && ok && wait_count(c_batch, rows(0), lane, S.err) && lane == 0) red_release_add(c_up, rows(0));
    for (int b = 1; b < nx && ok; ++b) chain_row(M_G, b, b - 1, v, c_up, c_batch, rows(b));
    // x_{nx-1} = y_{nx-1}
    if (gw == 0 && ok && wait_count(c_up + nx - 1, rows(nx - 1), lane, S.err) && lane == 0)
      red_release_add(c_down + nx - 1, rows(nx - 1));
    for (int b = nx - 2; b >= 0 && ok; --b) chain_row(M_W, b, b + 1, v, c_down, c_up, rows(b));
  } else {
    // w_0 = r_0 (gathered before the barrier)
    if (gw == 0 && lane == 0) red_release_add(c_up, rows(0));
    for (int b = 1; b < nx && ok; ++b) chain_row(M_P, b, b - 1, u, c_up, nullptr, 0u);
    batched(M_SINVT, u, v, true);
    if (gw == 0 && ok && wait_count(c_batch + nx - 1, rows(nx - 1), lane, S.err) && lane == 0)
      red_release_add(c_down + nx - 1, rows(nx - 1));
    for (int b = nx - 2; b >= 0 && ok; --b) chain_row(M_Q, b, b + 1, v, c_down, c_batch, rows(b));
  }
  grid.sync();
  // back to the row order of J_1; clear the counters for the next launch
  for (long long e = gt; e < S.n * NR; e += nt) {
    const long long i = e / NR;
    d[e] = v[(long long)S.perm[i] * NR + (e - i * NR)];
  }
  for (long long e = gt; e < 3LL * nx; e += nt) S.cnt[e] = 0u;
}

template <int NR>
stm_status launch_slab(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s) {
  static int occ = 0;
  if (!occ) {
    STM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_coarse_slab<NR>, 256, 0));
    if (occ < 1) {
      set_error("coarse slab solve: kernel does not fit on an SM");
      return STM_ERR_CUDA;
    }
  }
  SlabView S;
  S.nx = H.cs_nx;
  S.n = H.N0;
  S.off = H.cs_off;
  S.pos = H.cs_pos;
  S.rowslab = H.cs_rowslab;
  S.perm = H.cs_perm;
  S.store = H.cs_store;
  S.cnt = H.cs_cnt;
  S.err = H.dkerr;
  double* u = NR == 1 ? H.cs_u : H.cs_mu;
  double* v = NR == 1 ? H.cs_v : H.cs_mv;
  cudaLaunchConfig_t cfg = {};
  // co-resident CTAs (cooperative launch): rows wait on rows that other CTAs compute
  cfg.gridDim = dim3((unsigned)(std::min(occ, 2) * sm_count()));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  STM_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_slab<NR>, S, r, d, u, v, transpose));
  note_launch();
  return STM_OK;
}

}  // namespace

stm_status coarse_slab_apply(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s) {
  return launch_slab<1>(H, r, d, transpose, s);
}

stm_status coarse_slab_apply_multi(Hierarchy& H, const double* R, double* D, cudaStream_t s) {
  if (!H.cs_mu) {
    STM_CUDA(cudaMalloc(&H.cs_mu, sizeof(double) * 32 * (size_t)H.N0));
    STM_CUDA(cudaMalloc(&H.cs_mv, sizeof(double) * 32 * (size_t)H.N0));
  }
  return launch_slab<32>(H, R, D, 0, s);
}

}  // namespace stm
