// Cell-based space-time Vanka smoother (Sec. 4.2, Eq. LocVanka, damping of Sec. 5.3).
//
// Local step for cell T: y_T = J_T^{-1} t_T with t = r - J d gathered over all (k+1) time nodes
// of the cell's DoFs. The inverses are the dominant HBM stream of the whole solve. Each cell's
// inverse is stored column-major with its rows padded to a multiple of the vector width, so a
// thread owns a fixed chunk of V consecutive rows and walks the columns with aligned 16/8/4-byte
// vector loads: consecutive threads read consecutive memory, every load is fully used, no
// per-element reductions. Small cells are packed several per CTA to keep enough loads in flight.
// Shared DoFs are combined in a second, deterministic pass:
//   additive : d_i += omega / m_i * sum over the owners of i of y_T[alpha]
//   overwrite: d_i += omega * y_Tlast[alpha] (highest-index owning cell, "last update wins")
//   coloured : cells of one colour share no DoF, so y is scattered directly (d_T += omega y_T).
#include "internal.h"

namespace stm {

template <typename S> struct Acc { using T = float; };
template <> struct Acc<double> { using T = double; };

static int storage_size(int prec) { return prec == STM_F64 ? 8 : prec == STM_F32 ? 4 : 2; }

InvLayout inv_layout(int n, int prec) {
  const int s = storage_size(prec);
  for (int vb = 16; vb >= 4; vb /= 2) {
    const int V = vb / s;
    if (V < 1) break;
    const int ld = (n + V - 1) / V * V;
    if (vb == 4 || ld * 100 <= n * 106) return InvLayout{ld, vb};
  }
  return InvLayout{n, s};
}

// Thread geometry of the forward kernel for one level.
struct VGeom {
  int n, ld, LDV, Q, T, P;
};

static VGeom vanka_geometry(int n, InvLayout lay, int prec) {
  VGeom g;
  g.n = n;
  g.ld = lay.ld;
  g.LDV = lay.ld / (lay.vb / storage_size(prec));
  if (g.LDV >= 64) {
    g.Q = std::max(1, 256 / g.LDV);
  } else {
    g.Q = std::max(1, 32 / g.LDV);
  }
  g.T = g.LDV * g.Q;
  g.P = std::max(1, 256 / g.T);
  return g;
}

// Raw vector loads (VB bytes as 32-bit words) and their conversion to the accumulation type.
template <int VB> struct Raw { unsigned w[VB / 4]; };
template <int VB> __device__ __forceinline__ Raw<VB> ld_raw(const void* p);
template <> __device__ __forceinline__ Raw<16> ld_raw<16>(const void* p) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
  return Raw<16>{{v.x, v.y, v.z, v.w}};
}
template <> __device__ __forceinline__ Raw<8> ld_raw<8>(const void* p) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  return Raw<8>{{v.x, v.y}};
}
template <> __device__ __forceinline__ Raw<4> ld_raw<4>(const void* p) {
  return Raw<4>{{__ldg(reinterpret_cast<const unsigned*>(p))}};
}
template <typename S, int VB> struct Conv;
template <int VB> struct Conv<double, VB> {
  static constexpr int V = VB / 8;
  __device__ static void run(const Raw<VB>& r, double* o) {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = __hiloint2double((int)r.w[2 * v + 1], (int)r.w[2 * v]);
  }
};
template <int VB> struct Conv<float, VB> {
  static constexpr int V = VB / 4;
  __device__ static void run(const Raw<VB>& r, float* o) {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = __uint_as_float(r.w[v]);
  }
};
template <int VB> struct Conv<__nv_bfloat16, VB> {
  static constexpr int V = VB / 2;
  __device__ static void run(const Raw<VB>& r, float* o) {
#pragma unroll
    for (int v = 0; v < VB / 4; ++v) {
      o[2 * v] = __uint_as_float(r.w[v] << 16);
      o[2 * v + 1] = __uint_as_float(r.w[v] & 0xffff0000u);
    }
  }
};

// Forward local solves y_T = Inv_T t_T for the cells of `cell_list` (all cells if NULL).
// CTA = P cell slots of T threads; thread (rc, cg) of a slot accumulates rows rc*V..rc*V+V-1 over
// the columns j = cg (mod Q); the Q partial sums of a row are added through shared memory.
template <typename S, int VB>
__global__ void __launch_bounds__(256, sizeof(S) == 2 ? 5 : 4) k_vanka_local(const S* __restrict__ inv, const int* __restrict__ idx,
                                                     const double* __restrict__ t, double* __restrict__ Y,
                                                     const int* __restrict__ cell_list, int ncells, VGeom g,
                                                     double* __restrict__ d_scatter, double omega) {
  using A = typename Acc<S>::T;
  using CV = Conv<S, VB>;
  constexpr int V = CV::V;
  constexpr int UB = VB == 16 ? 4 : 8;  // column loads issued before their FMAs
  extern __shared__ double smd[];
  A* tl = reinterpret_cast<A*>(smd);      // [P][n]
  A* part = tl + g.P * g.n;               // [P][Q][ld]
  const int slot = threadIdx.x / g.T;
  const int lt = threadIdx.x - slot * g.T;
  const int rc = lt % g.LDV, cg = lt / g.LDV;
  for (int base = blockIdx.x * g.P; base < ncells; base += gridDim.x * g.P) {
    const int ci = base + slot;
    const bool has = slot < g.P && ci < ncells;
    const int c = has ? (cell_list ? cell_list[ci] : ci) : 0;
    const int* ic = idx + (long long)c * g.n;
    __syncthreads();
    if (has)
      for (int i = lt; i < g.n; i += g.T) tl[slot * g.n + i] = (A)t[ic[i]];
    __syncthreads();
    if (has) {
      A acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0;
      const S* M = inv + (size_t)c * g.n * g.ld + rc * V;
      const A* tc = tl + slot * g.n;
      for (int j0 = cg; j0 < g.n; j0 += UB * g.Q) {
        Raw<VB> raw[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int j = j0 + u * g.Q;
          if (j < g.n) raw[u] = ld_raw<VB>(M + (size_t)j * g.ld);
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int j = j0 + u * g.Q;
          if (j < g.n) {
            A e[V];
            CV::run(raw[u], e);
            const A tj = tc[j];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += e[v] * tj;
          }
        }
      }
      A* pp = part + (slot * g.Q + cg) * g.ld + rc * V;
#pragma unroll
      for (int v = 0; v < V; ++v) pp[v] = acc[v];
    }
    __syncthreads();
    if (has)
      for (int i = lt; i < g.n; i += g.T) {
        A y = 0;
        for (int q = 0; q < g.Q; ++q) y += part[(slot * g.Q + q) * g.ld + i];
        if (d_scatter) d_scatter[ic[i]] += omega * (double)y;
        else Y[(long long)c * g.n + i] = (double)y;
      }
  }
}

// Small cells (n <= 64 and at most 32 vector chunks per column): one warp per cell and no CTA
// barriers. Lane (rc, cg) = (lane % LDV, lane / LDV) owns rows rc*V..rc*V+V-1 and the columns
// j = cg (mod Q); t_T sits in the warp's own shared slice; the Q partial sums of a row meet through
// shuffles. The next cell's DoF ids are loaded before the current inverse is streamed and its t
// values right after, so the gather latency overlaps the stream and the epilogue.
template <typename S, int VB>
__global__ void __launch_bounds__(256, 4) k_vanka_warp(const S* __restrict__ inv, const int* __restrict__ idx,
                                                    const double* __restrict__ t, double* __restrict__ Y,
                                                    const int* __restrict__ cell_list, int ncells, int n, int ld,
                                                    int LDV, int Q, double* __restrict__ d_scatter, double omega) {
  using A = typename Acc<S>::T;
  using CV = Conv<S, VB>;
  constexpr int V = CV::V;
  constexpr int UB = VB == 4 ? 12 : 6;  // column loads in flight per lane
  __shared__ A tsh[8][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int rc = lane % LDV, cg = lane / LDV;
  const int jstart = cg < Q ? cg : n;  // lanes beyond Q*LDV stream nothing
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  A* tl = tsh[wid];
  long long ci = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (ci >= ncells) return;  // warp-uniform
  int c = cell_list ? cell_list[ci] : (int)ci;
  A ta = lane < n ? (A)t[idx[(long long)c * n + lane]] : A(0);
  A tb = lane + 32 < n ? (A)t[idx[(long long)c * n + lane + 32]] : A(0);
  for (; ci < ncells; ci += nwarps) {
    __syncwarp();
    tl[lane] = ta;
    tl[lane + 32] = tb;
    __syncwarp();
    const long long cin = ci + nwarps;
    const bool has_next = cin < ncells;
    const int cn = has_next ? (cell_list ? cell_list[cin] : (int)cin) : 0;
    const int ia = (has_next && lane < n) ? idx[(long long)cn * n + lane] : -1;
    const int ib = (has_next && lane + 32 < n) ? idx[(long long)cn * n + lane + 32] : -1;
    A acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0;
    const S* M = inv + (size_t)c * n * ld + rc * V;
    for (int j0 = jstart; j0 < n; j0 += UB * Q) {
      Raw<VB> raw[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = j0 + u * Q;
        if (j < n) raw[u] = ld_raw<VB>(M + (size_t)j * ld);
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = j0 + u * Q;
        if (j < n) {
          A e[V];
          CV::run(raw[u], e);
          const A tj = tl[j];
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] += e[v] * tj;
        }
      }
    }
    // next cell's t (its ids have arrived during the stream)
    ta = ia >= 0 ? (A)t[ia] : A(0);
    tb = ib >= 0 ? (A)t[ib] : A(0);
    // lanes cg = 0 collect the Q partial sums of their rows
    for (int off = (Q >> 1) * LDV; off >= LDV; off >>= 1)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] += __shfl_down_sync(0xffffffffu, acc[v], off);
    if (cg == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int row = rc * V + v;
        if (row < n) {
          if (d_scatter) d_scatter[idx[(long long)c * n + row]] += omega * (double)acc[v];
          else Y[(long long)c * n + row] = (double)acc[v];
        }
      }
    }
    c = cn;
  }
}

// Transposed local solves y_T = Inv_T^T t_T (adjoint smoother). Column j of the stored inverse is
// contiguous, and (Inv^T t)_j is that column dotted with t_T, so one thread per column streams it
// with VB-byte vector loads against t_T in shared memory: no cross-thread sums. A cell takes T
// threads (n rounded up to a warp), a CTA P cells.
template <typename S, int VB>
__global__ void __launch_bounds__(256) k_vanka_local_t(const S* __restrict__ inv, const int* __restrict__ idx,
                                                       const double* __restrict__ t, double* __restrict__ Y,
                                                       const int* __restrict__ cell_list, int ncells, int n, int ld,
                                                       int T, int P, double* __restrict__ d_scatter, double omega) {
  using A = typename Acc<S>::T;
  using CV = Conv<S, VB>;
  constexpr int V = CV::V;
  extern __shared__ double smd[];
  A* tl = reinterpret_cast<A*>(smd);  // [P][ld], rows n..ld-1 zero like the stored padding
  const int slot = threadIdx.x / T, j = threadIdx.x - slot * T;
  for (int base = blockIdx.x * P; base < ncells; base += gridDim.x * P) {
    const int ci = base + slot;
    const bool has = slot < P && ci < ncells;
    const int c = has ? (cell_list ? cell_list[ci] : ci) : 0;
    const int* ic = idx + (long long)c * n;
    __syncthreads();
    if (has)
      for (int i = j; i < ld; i += T) tl[slot * ld + i] = i < n ? (A)t[ic[i]] : A(0);
    __syncthreads();
    if (has && j < n) {
      const S* col = inv + (size_t)c * n * ld + (size_t)j * ld;
      const A* tc = tl + slot * ld;
      A acc = 0;
#pragma unroll 8
      for (int i0 = 0; i0 < ld; i0 += V) {
        A e[V];
        CV::run(ld_raw<VB>(col + i0), e);
#pragma unroll
        for (int v = 0; v < V; ++v) acc += e[v] * tc[i0 + v];
      }
      if (d_scatter) d_scatter[ic[j]] += omega * (double)acc;
      else Y[(long long)c * n + j] = (double)acc;
    }
  }
}

// Second pass of the additive / overwrite variants (one thread per global DoF). A DoF has at most
// 2^d owners (the cells around a vertex), so all owner positions are loaded first and then all Y
// entries, two dependent loads in all instead of two per owner; the sum still runs in owner order.
// With d32 non-null the new d is also stored rounded to FP32 there (the next FP32 defect reads it).
template <int MAXO>
__global__ void k_vanka_gather(double* __restrict__ d, float* __restrict__ d32, const double* __restrict__ Y,
                               const int* __restrict__ own_ptr, const int* __restrict__ own_pos,
                               const int* __restrict__ last_owner, const double* __restrict__ wmult,
                               long long N, double omega, int overwrite) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    if (overwrite) {
      const double nd = d[i] + omega * Y[last_owner[i]];
      d[i] = nd;
      if (d32) d32[i] = __double2float_rn(nd);
    } else {
      const int p0 = own_ptr[i], p1 = own_ptr[i + 1];
      int pos[MAXO];
#pragma unroll
      for (int k = 0; k < MAXO; ++k) pos[k] = p0 + k < p1 ? __ldg(own_pos + p0 + k) : -1;
      double y[MAXO];
#pragma unroll
      for (int k = 0; k < MAXO; ++k) y[k] = pos[k] >= 0 ? Y[pos[k]] : 0.0;
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < MAXO; ++k)
        if (pos[k] >= 0) s += y[k];
      for (int p = p0 + MAXO; p < p1; ++p) s += Y[own_pos[p]];
      const double nd = d[i] + omega * wmult[i] * s;
      d[i] = nd;
      if (d32) d32[i] = __double2float_rn(nd);
    }
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename S, int VB>
static void launch_warp(const Level& L, const void* inv, const VGeom& g, const double* t, const int* cells, int nc,
                        double* scatter, double omega, cudaStream_t s) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_vanka_warp<S, VB>, 256, 0);
    if (per_sm <= 0) per_sm = 1;
  }
  int Q = 1;
  while (2 * Q * g.LDV <= 32) Q *= 2;
  // one warp per cell in rounds of the resident warps: as few warps as give the same number of rounds,
  // so that every warp streams the same number of cells and none idles through a last partial round
  const long long maxw = 8LL * sm_count() * per_sm;
  const long long rounds = std::max(1LL, ((long long)nc + maxw - 1) / maxw);
  const long long warps = ((long long)nc + rounds - 1) / rounds;
  const int blocks = (int)std::max(1LL, (warps + 7) / 8);
  k_vanka_warp<S, VB><<<blocks, 256, 0, s>>>((const S*)inv, L.idx, t, L.Y, cells, nc, g.n, g.ld, g.LDV, Q, scatter,
                                            omega);
}

// Cells per CTA for the block-per-cells kernel. All resident CTAs run rounds of P cells in lockstep
// with the memory system, so the launch takes ceil(rounds) rounds with rounds = ncells / (P x resident
// CTAs): among the P that keep at least 85 % of the largest resident thread count, take the one whose
// rounds come closest below a whole number (3D dG(1), 16,128 cells: P = 11 at five CTAs per SM gives
// 1.93 rounds, against 2.41 at four). Cached per (n, cells) of a level.
template <typename S, int VB>
static void launch_local_fwd(const Level& L, const void* inv, VGeom g, const double* t, const int* cells, int nc,
                             double* scatter, double omega, cudaStream_t s) {
  using A = typename Acc<S>::T;
  struct Pick { int n, nc, P, blocks; };
  static std::vector<Pick> memo;
  auto smem_of = [&](int P) { return sizeof(A) * ((size_t)P * g.n + (size_t)P * g.Q * g.ld) + 16; };
  int P = g.P, blocks = 0;
  bool found = false;
  for (const Pick& m : memo)
    if (m.n == g.n && m.nc == nc) { P = m.P; blocks = m.blocks; found = true; break; }
  if (!found) {
    const int pmax = std::max(1, 256 / g.T);
    std::vector<int> occ(pmax + 1, 0);
    int best_threads = 0;
    for (int p = 1; p <= pmax; ++p) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[p], k_vanka_local<S, VB>, g.T * p, smem_of(p)) != cudaSuccess)
        occ[p] = 0;
      best_threads = std::max(best_threads, occ[p] * g.T * p);
    }
    double best_eff = -1.0;
    for (int p = 1; p <= pmax; ++p) {
      if (occ[p] <= 0 || occ[p] * g.T * p * 100 < best_threads * 85) continue;
      const double slots = (double)occ[p] * sm_count();
      const double rounds = std::max(1.0, (double)((nc + p - 1) / p) / slots);
      const double eff = rounds / std::ceil(rounds);
      if (eff > best_eff + 1e-9 || (eff > best_eff - 1e-9 && p == g.P)) {
        best_eff = eff;
        P = p;
        blocks = (int)std::max(1.0, std::min(slots, (double)((nc + p - 1) / p)));
      }
    }
    if (blocks <= 0) {  // no occupancy answer: the default geometry, one CTA per group up to 8 per SM
      P = g.P;
      blocks = std::min((nc + P - 1) / P, sm_count() * 8);
    }
    memo.push_back(Pick{g.n, nc, P, blocks});
  }
  g.P = P;
  k_vanka_local<S, VB><<<blocks, g.T * P, smem_of(P), s>>>((const S*)inv, L.idx, t, L.Y, cells, nc, g, scatter,
                                                          omega);
}

template <typename S>
static void launch_fwd(const Level& L, const void* inv, int vb, const VGeom& g, const double* t, const int* cells,
                       int nc, double* scatter, double omega, cudaStream_t s) {
  using A = typename Acc<S>::T;
  if (g.n <= 64 && g.LDV <= 32) {
    if (vb == 16) launch_warp<S, 16>(L, inv, g, t, cells, nc, scatter, omega, s);
    else if (vb == 8 || sizeof(S) == 8) launch_warp<S, 8>(L, inv, g, t, cells, nc, scatter, omega, s);
    else if constexpr (sizeof(S) < 8) launch_warp<S, 4>(L, inv, g, t, cells, nc, scatter, omega, s);
    return;
  }
  if (vb == 16) {
    launch_local_fwd<S, 16>(L, inv, g, t, cells, nc, scatter, omega, s);
  } else if (vb == 8 || sizeof(S) == 8) {
    launch_local_fwd<S, 8>(L, inv, g, t, cells, nc, scatter, omega, s);
  } else if constexpr (sizeof(S) < 8) {
    launch_local_fwd<S, 4>(L, inv, g, t, cells, nc, scatter, omega, s);
  }
}

static stm_status launch_local(Hierarchy& H, Level& L, int level, const double* t, const int* cells, int nc,
                               int transpose, double* scatter, cudaStream_t s) {
  if (nc <= 0) return STM_OK;
  const int prec = H.p.inv_precision;
  const InvLayout lay = inv_layout(L.n, prec);
  ProfScope ps(&H, STM_KCLASS_VANKA_LOCAL, s, (double)nc * ((double)L.n * L.n * storage_size(prec) + 20.0 * L.n),
               level);
  const double omega = H.p.omega;
  if (!transpose) {
    const VGeom g = vanka_geometry(L.n, lay, prec);
    if (prec == STM_F64) launch_fwd<double>(L, L.inv, lay.vb, g, t, cells, nc, scatter, omega, s);
    else if (prec == STM_F32) launch_fwd<float>(L, L.inv, lay.vb, g, t, cells, nc, scatter, omega, s);
    else launch_fwd<__nv_bfloat16>(L, L.inv, lay.vb, g, t, cells, nc, scatter, omega, s);
  } else {
    const int T = (L.n + 31) / 32 * 32;
    const int P = std::max(1, 256 / T);
    const int blocks = std::min((nc + P - 1) / P, sm_count() * 8);
    if (prec == STM_F64) {
      const size_t smem = sizeof(double) * (size_t)P * lay.ld + 16;
      if (lay.vb == 16)
        k_vanka_local_t<double, 16><<<blocks, T * P, smem, s>>>((const double*)L.inv, L.idx, t, L.Y, cells, nc, L.n,
                                                                lay.ld, T, P, scatter, omega);
      else
        k_vanka_local_t<double, 8><<<blocks, T * P, smem, s>>>((const double*)L.inv, L.idx, t, L.Y, cells, nc, L.n,
                                                               lay.ld, T, P, scatter, omega);
    } else if (prec == STM_F32) {
      const size_t smem = sizeof(float) * (size_t)P * lay.ld + 16;
      if (lay.vb == 16)
        k_vanka_local_t<float, 16><<<blocks, T * P, smem, s>>>((const float*)L.inv, L.idx, t, L.Y, cells, nc, L.n,
                                                               lay.ld, T, P, scatter, omega);
      else if (lay.vb == 8)
        k_vanka_local_t<float, 8><<<blocks, T * P, smem, s>>>((const float*)L.inv, L.idx, t, L.Y, cells, nc, L.n,
                                                              lay.ld, T, P, scatter, omega);
      else
        k_vanka_local_t<float, 4><<<blocks, T * P, smem, s>>>((const float*)L.inv, L.idx, t, L.Y, cells, nc, L.n,
                                                              lay.ld, T, P, scatter, omega);
    } else {
      const size_t smem = sizeof(float) * (size_t)P * lay.ld + 16;
      const __nv_bfloat16* iv = (const __nv_bfloat16*)L.inv;
      if (lay.vb == 16)
        k_vanka_local_t<__nv_bfloat16, 16><<<blocks, T * P, smem, s>>>(iv, L.idx, t, L.Y, cells, nc, L.n, lay.ld, T,
                                                                       P, scatter, omega);
      else if (lay.vb == 8)
        k_vanka_local_t<__nv_bfloat16, 8><<<blocks, T * P, smem, s>>>(iv, L.idx, t, L.Y, cells, nc, L.n, lay.ld, T,
                                                                      P, scatter, omega);
      else
        k_vanka_local_t<__nv_bfloat16, 4><<<blocks, T * P, smem, s>>>(iv, L.idx, t, L.Y, cells, nc, L.n, lay.ld, T,
                                                                      P, scatter, omega);
    }
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status vanka_step(Hierarchy& H, int g, const double* r, double* d, int transpose, bool d_is_zero,
                      cudaStream_t s, bool d32_current) {
  Level& L = H.L[g];
  const double omega = H.p.omega;
  if (H.p.smoother == STM_VANKA_COLOURED) {
    for (int col = 0; col < (1 << L.dim); ++col) {
      const int nc = L.colour_off[col + 1] - L.colour_off[col];
      const double* t = r;
      if (!(d_is_zero && col == 0)) {
        // the colour's local solves read t only at the DoFs of its cells: with FP64 defects only
        // those velocity rows (and the pressure rows) are formed
        stm_status st = H.p.defect_precision == STM_F32 ? smoother_defect(H, g, d, r, L.t, transpose, s)
                                                         : jacobian_defect_colour(H, g, col, d, r, L.t, transpose, s);
        if (st != STM_OK) return st;
        t = L.t;
      }
      stm_status st = launch_local(H, L, g, t, L.colour_cells + L.colour_off[col], nc, transpose, d, s);
      if (st != STM_OK) return st;
    }
    return STM_OK;
  }
  const double* t = r;
  if (!d_is_zero) {
    stm_status st = smoother_defect(H, g, d, r, L.t, transpose, s, d32_current);
    if (st != STM_OK) return st;
    t = L.t;
  }
  stm_status st = launch_local(H, L, g, t, nullptr, L.C, transpose, nullptr, s);
  if (st != STM_OK) return st;
  const int blocks = (int)std::min<long long>((L.N + 255) / 256, sm_count() * 16LL);
  ProfScope ps(&H, STM_KCLASS_VANKA_COMBINE, s, 0.0, g);
  const int ow = H.p.smoother == STM_VANKA_PAPER_OVERWRITE;
  float* d32 = H.p.defect_precision == STM_F32 ? L.x32 : nullptr;
  if (L.dim == 2)
    k_vanka_gather<4><<<blocks, 256, 0, s>>>(d, d32, L.Y, L.own_ptr, L.own_pos, L.last_owner, L.wmult, L.N, omega, ow);
  else
    k_vanka_gather<8><<<blocks, 256, 0, s>>>(d, d32, L.Y, L.own_ptr, L.own_pos, L.last_owner, L.wmult, L.N, omega, ow);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

}  // namespace stm
