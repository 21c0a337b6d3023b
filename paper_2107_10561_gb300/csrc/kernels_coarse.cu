// Direct coarse solve of Algorithm 1 (d_1 = J_1^{-1} r_1, or J_1^{-T} r_1 in the adjoint V-cycle) through
// the twisted block factors of J_1 in x-slab order (kernels_factor.cu), for coarse levels too large for
// the dense explicit inverse to pay (3D: 18,000 DoFs, 2.6 GB as a dense inverse).
//
// In slab order J_1 is block tridiagonal. Its slabs are eliminated from both ends towards the twist
// slab t; with Sinv_b the inverse Schur complements, the solve of J_1 x = r is
//   z_b = Sinv_b r_b                                         (all slabs at once)
//   y_b = z_b - Lo_b y_{b-1},  b = 1 .. t-1   together with  y_b = z_b - Up_b y_{b+1},  b = nx-2 .. t+1
//   x_t = z_t - Lo_t y_{t-1} - Up_t y_{t+1}
//   x_b = y_b - Bk_b x_{b+1},  b = t-1 .. 0   together with  x_b = y_b - Bk_b x_{b-1},  b = t+1 .. nx-1
// (Lo_b = Sinv_b A_{b,b-1}, Up_b = Sinv_b A_{b,b+1}, Bk_b the back-substitution block). J_1^T has its
// own blocks of the same shapes (kinds 4..7), so both directions run the same kernel. Every block is
// stored row-major, so each product is a warp-per-row dot product over contiguous rows. The dependent
// steps (about nx instead of the 2 (nx - 1) of a one-sided block LU, each step working on the two slabs
// at the ends of the chains) run inside one cooperative kernel with a grid-wide barrier between steps
// (the barrier also orders the vector written in one step before its reads in the next); before a
// step's barrier every thread prefetches into L2 a share of the blocks the next step reads.
// Measured on the 18,000-DoF 3D coarse level (16 slabs): 290 us per solve, against 347 us with the
// one-sided factors and 560 us for the explicit inverse. With four loads per lane in flight (312 us)
// the barriers with the gather and scatter took about 57 us, the batched products z_b about 72 us and
// each dependent step about 11 us: a row's dot product waits on memory round trips, so eight
// independent loads per lane are issued before the first FMA (sixteen: 317 us). Slower variants:
//   - per-slab completion counters polled by the waiting warps instead of the barriers: 555 us;
//   - four FMA chains per lane: 413 us one-sided, 329 us twisted;
//   - one 16-warp CTA per SM: 421 us;
//   - requesting the blocks two steps ahead at the start of each step: 473 us;
//   - no L2 requests at all: 315 us.
// A 32-column variant (interleaved [N][32] multi-vectors, lane = column) serves the multi-RHS V-cycle.
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace stm {
namespace {

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

struct SlabView {
  int nx, t;
  long long n;
  const long long* off;   // [nx + 1] first permuted row of every slab
  const long long* pos;   // [8][nx] block offsets in store (-1: absent)
  const int* rowslab;     // [n] slab of every permuted row
  const int* perm;        // [n] permuted position of every row of J_1
  const double* store;
};

enum { K_INV = 0, K_LO = 1, K_UP = 2, K_BACK = 3 };

// One product task of a step: rows of slab b, y_b (-)= M x_c (M: nb x nc, row-major).
struct Task {
  const double* M;
  long long r0, nb, c0, nc;
};

__device__ __forceinline__ Task make_task(const SlabView& S, int kind, int b, int c) {
  Task k;
  k.M = S.store + S.pos[kind * S.nx + b];
  k.r0 = S.off[b];
  k.nb = S.off[b + 1] - k.r0;
  k.c0 = S.off[c];
  k.nc = S.off[c + 1] - k.c0;
  return k;
}
__device__ __forceinline__ Task no_task() {
  Task k;
  k.M = nullptr;
  k.r0 = k.nb = k.c0 = k.nc = 0;
  return k;
}

// Dot product of one stored row m[0 .. nc) with the vector x (slab part starting at x). NR = 1: lanes
// stride the row, result in every lane; NR = 32: lane = column of interleaved 32-column vectors.
template <int NR>
__device__ __forceinline__ double row_dot(const double* m, long long nc, const double* x, int lane) {
  if (NR == 1) {
    // 8 independent loads of the row and of x per lane are in flight before the first FMA waits
    constexpr int UR = 8;
    double a[UR];
#pragma unroll
    for (int q = 0; q < UR; ++q) a[q] = 0.0;
    long long k = lane;
    for (; k + 32 * (UR - 1) < nc; k += 32 * UR) {
      double mv[UR], xv[UR];
#pragma unroll
      for (int q = 0; q < UR; ++q) {
        mv[q] = __ldg(m + k + 32 * q);
        xv[q] = x[k + 32 * q];
      }
#pragma unroll
      for (int q = 0; q < UR; ++q) a[q] = fma(mv[q], xv[q], a[q]);
    }
    for (; k < nc; k += 32) a[0] = fma(__ldg(m + k), x[k], a[0]);
#pragma unroll
    for (int q = 1; q < UR; ++q) a[0] += a[q];
    double acc = a[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
  } else {
    double a0 = 0.0, a1 = 0.0;
    long long k = 0;
    for (; k + 1 < nc; k += 2) {
      a0 = fma(__ldg(m + k), x[k * 32 + lane], a0);
      a1 = fma(__ldg(m + k + 1), x[(k + 1) * 32 + lane], a1);
    }
    if (k < nc) a0 = fma(__ldg(m + k), x[k * 32 + lane], a0);
    return a0 + a1;
  }
}

// y_{b} -= M x_c for the rows of up to two tasks (warps stride the concatenated rows of both).
template <int NR>
__device__ __forceinline__ void pair_step(const Task& A, const Task& B, double* v, long long gw, long long nw,
                                          int lane) {
  const long long tot = A.nb + B.nb;
  for (long long rr = gw; rr < tot; rr += nw) {
    const Task& T = rr < A.nb ? A : B;
    const long long r = rr < A.nb ? rr : rr - A.nb;
    const double acc = row_dot<NR>(T.M + r * T.nc, T.nc, v + T.c0 * NR, lane);
    if (NR == 1) {
      if (lane == 0) v[T.r0 + r] -= acc;
    } else {
      v[(T.r0 + r) * 32 + lane] -= acc;
    }
  }
}

// Every thread of the grid prefetches a share of the 128-byte lines of the task's block into L2.
__device__ __forceinline__ void task_prefetch(const Task& T, long long gt, long long nt) {
  if (!T.M) return;
  const char* p = reinterpret_cast<const char*>(T.M);
  const long long bytes = T.nb * T.nc * 8;
  for (long long o = gt * 128; o < bytes; o += nt * 128) prefetch_l2(p + o);
}

// Chain tasks of step s (1-based) of the forward elimination and of the back substitution.
__device__ __forceinline__ void chain_tasks(const SlabView& S, int base, int s, Task& A, Task& B) {
  const int t = S.t, nx = S.nx;
  A = s <= t - 1 ? make_task(S, base + K_LO, s, s - 1) : no_task();
  B = nx - 1 - s >= t + 1 ? make_task(S, base + K_UP, nx - 1 - s, nx - s) : no_task();
}
__device__ __forceinline__ void back_tasks(const SlabView& S, int base, int s, Task& A, Task& B) {
  const int t = S.t, nx = S.nx;
  A = t - s >= 0 ? make_task(S, base + K_BACK, t - s, t - s + 1) : no_task();
  B = t + s <= nx - 1 ? make_task(S, base + K_BACK, t + s, t + s - 1) : no_task();
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
  const int nx = S.nx, t = S.t;
  const int base = transpose ? 4 : 0;
  const int nchain = max(t - 1, nx - 2 - t), nback = max(t, nx - 1 - t);
  // gather into slab order
  for (long long e = gt; e < S.n * NR; e += nt) {
    const long long i = e / NR;
    u[(long long)S.perm[i] * NR + (e - i * NR)] = r[e];
  }
  grid.sync();
  // z_b = Sinv_b r_b for every slab: every warp takes rows across all slabs
  for (long long row = gw; row < S.n; row += nw) {
    const int b = S.rowslab[row];
    const long long c0 = S.off[b], nb = S.off[b + 1] - c0;
    const double acc = row_dot<NR>(S.store + S.pos[(base + K_INV) * nx + b] + (row - c0) * nb, nb, u + c0 * NR, lane);
    if (NR == 1) {
      if (lane == 0) v[row] = acc;
    } else {
      v[row * 32 + lane] = acc;
    }
  }
  Task A, B;
  if (nchain >= 1) {
    chain_tasks(S, base, 1, A, B);
    task_prefetch(A, gt, nt);
    task_prefetch(B, gt, nt);
  }
  grid.sync();
  // the two elimination chains, one step of each per barrier
  for (int s = 1; s <= nchain; ++s) {
    chain_tasks(S, base, s, A, B);
    pair_step<NR>(A, B, v, gw, nw, lane);
    Task nA, nB;
    if (s < nchain) {
      chain_tasks(S, base, s + 1, nA, nB);
    } else {
      nA = t >= 1 ? make_task(S, base + K_LO, t, t - 1) : no_task();
      nB = t + 1 < nx ? make_task(S, base + K_UP, t, t + 1) : no_task();
    }
    task_prefetch(nA, gt, nt);
    task_prefetch(nB, gt, nt);
    grid.sync();
  }
  // the twist slab: x_t = z_t - Lo_t y_{t-1} - Up_t y_{t+1}
  {
    const Task lo = t >= 1 ? make_task(S, base + K_LO, t, t - 1) : no_task();
    const Task up = t + 1 < nx ? make_task(S, base + K_UP, t, t + 1) : no_task();
    const long long r0 = S.off[t], nb = S.off[t + 1] - r0;
    for (long long rr = gw; rr < nb; rr += nw) {
      double acc = 0.0;
      if (lo.M) acc += row_dot<NR>(lo.M + rr * lo.nc, lo.nc, v + lo.c0 * NR, lane);
      if (up.M) acc += row_dot<NR>(up.M + rr * up.nc, up.nc, v + up.c0 * NR, lane);
      if (NR == 1) {
        if (lane == 0) v[r0 + rr] -= acc;
      } else {
        v[(r0 + rr) * 32 + lane] -= acc;
      }
    }
    if (nback >= 1) {
      back_tasks(S, base, 1, A, B);
      task_prefetch(A, gt, nt);
      task_prefetch(B, gt, nt);
    }
    grid.sync();
  }
  // back substitution away from the twist, both directions per barrier
  for (int s = 1; s <= nback; ++s) {
    back_tasks(S, base, s, A, B);
    pair_step<NR>(A, B, v, gw, nw, lane);
    if (s < nback) {
      Task nA, nB;
      back_tasks(S, base, s + 1, nA, nB);
      task_prefetch(nA, gt, nt);
      task_prefetch(nB, gt, nt);
    }
    grid.sync();
  }
  // back to the row order of J_1
  for (long long e = gt; e < S.n * NR; e += nt) {
    const long long i = e / NR;
    d[e] = v[(long long)S.perm[i] * NR + (e - i * NR)];
  }
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
  S.t = H.cs_t;
  S.n = H.N0;
  S.off = H.cs_off;
  S.pos = H.cs_pos;
  S.rowslab = H.cs_rowslab;
  S.perm = H.cs_perm;
  S.store = H.cs_store;
  double* u = NR == 1 ? H.cs_u : H.cs_mu;
  double* v = NR == 1 ? H.cs_v : H.cs_mv;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(std::min(occ, 4) * sm_count()));
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
