// Structured product with the slab Jacobian J_g or its transpose: y = J x, y = b - J x or y += J x,
// in FP64, or over FP32 copies of the values for the V-cycle's defects (FP32 products and sums, x
// rounded to FP32 in a pass of its own, b and y in FP64).
//
// Every velocity row (a, l, i) of J couples node i with the same neighbour list nbr(i) in every
// (time b, component m) block, plus the pressures of the cells around i at time a (Problem 3.1,
// Eq. newton_system_matrix_dG_1 with a diagonal time mass); a pressure row (a, cell, q) holds the
// velocities of its cell at time a. The pattern is structurally symmetric, so J^T uses the same
// structure with permuted values.
// The values are copied once per assembly into two layouts built for this product:
//   - node blocks: the K*d velocity rows of node i share one column structure, so position p of the
//     node holds those rows' K*d values contiguously; VL lanes per node walk consecutive positions
//     (one contiguous run), load each x entry once for all K*d rows, and combine the K*d partial
//     sums through a reduce-scatter butterfly (few FP64 adds); nodes are ordered by neighbour
//     count so that the groups of one warp run equal trip counts;
//   - warp-transposed pressure rows: one lane per row, entry t of 32 consecutive rows contiguous.
// Column indices are never read. In FP64, issue slots of the FP64 pipe are the limit (one FP64 warp
// instruction every 16 cycles per SM); results equal the plain CSR product up to FP64 summation
// order. In FP32 the arithmetic is cheap and the loads in flight per SM set the pace.
#include "internal.h"

namespace stm {

__host__ __device__ constexpr int pow2ceil(int v) { return v <= 1 ? 1 : 2 * pow2ceil((v + 1) / 2); }

// Reduce-scatter over the VL lanes of a group: on entry every lane holds NA partial sums; each halving
// step trades half of the accumulators still held with the partner lane. With NA <= VL, acc[0] of lane
// L ends as the full group sum of accumulator scatter_index(L) (NA - 1 + the remaining log2(VL/NA)
// adds instead of NA * log2(VL)); with NA > VL, acc[0 .. NA/VL - 1] of lane L end as the full sums of
// accumulators scatter_index(L) + 0 .. NA/VL - 1 (NA (1 - 1/VL) adds).
template <int VL, int NA, typename T>
__device__ __forceinline__ void reduce_scatter(T* acc, int lane) {
  int cnt = NA;
#pragma unroll
  for (int off = VL / 2; off >= 1; off >>= 1) {
    if (cnt > 1) {
      const int half = cnt / 2;
      const bool upper = (lane & off) != 0;
#pragma unroll
      for (int k = 0; k < NA / 2; ++k) {
        if (k < half) {
          const T send = upper ? acc[k] : acc[k + half];
          const T keep = upper ? acc[k + half] : acc[k];
          acc[k] = keep + __shfl_xor_sync(0xffffffffu, send, off, VL);
        }
      }
      cnt = half;
    } else {
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], off, VL);
    }
  }
}
template <int VL, int NA>
__device__ __forceinline__ int scatter_index(int lane, int* writer_mask) {
  int cnt = NA, k = 0, wm = 0;
#pragma unroll
  for (int off = VL / 2; off >= 1; off >>= 1) {
    if (cnt > 1) {
      const int half = cnt / 2;
      if (lane & off) k += half;
      cnt = half;
    } else {
      wm |= off;
    }
  }
  *writer_mask = wm;
  return k;
}

// ---------------------------------------------------------------------------------------------
// Node-block copy of the velocity rows and the forward product that reads it
// ---------------------------------------------------------------------------------------------
// One warp per node: CSR position pos of velocity row (a, l) -> node-block position p:
//   pos < (a+1) d nn                 : p = pos                        (velocity blocks b <= a)
//   next n_p nc entries (pressure)   : p = K d nn + (pos - (a+1) d nn)
//   beyond                           : p = pos - n_p nc               (velocity blocks b > a)
__global__ void k_build_nodeblock(const long long* __restrict__ rowptr, const double* __restrict__ val,
                                  const int* __restrict__ nbr_ptr, const int* __restrict__ ncell,
                                  const long long* __restrict__ nbase, double* __restrict__ nval, long long block,
                                  int R, int K, int D, int NP) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int KD = K * D;
  for (long long i = warp; i < R; i += nwarps) {
    const int nn = nbr_ptr[i + 1] - nbr_ptr[i], nc = ncell[i];
    const int len = KD * nn + NP * nc;
    for (int a = 0; a < K; ++a)
      for (int l = 0; l < D; ++l) {
        const long long rb = rowptr[a * block + (long long)l * R + i];
        for (int pos = lane; pos < len; pos += 32) {
          const int lim = (a + 1) * D * nn;
          int p;
          if (pos < lim) p = pos;
          else if (pos < lim + NP * nc) p = KD * nn + (pos - lim);
          else p = pos - NP * nc;
          nval[nbase[i] + (long long)p * KD + a * D + l] = val[rb + pos];
        }
      }
  }
}

// One thread per pressure row pr = (a*C + c)*n_p + q: its d*nv CSR entries (ordered m*nv + j, the
// cell's nodes in ascending id) go to the warp-transposed copy.
__global__ void k_build_pval(const long long* __restrict__ rowptr, const double* __restrict__ val,
                             double* __restrict__ pvalT, long long block, int R, int C, int K, int D, int NP, int nv) {
  const long long npr = (long long)K * C * NP;
  const int dnv = D * nv;
  for (long long pr = blockIdx.x * (long long)blockDim.x + threadIdx.x; pr < npr;
       pr += (long long)gridDim.x * blockDim.x) {
    const long long a = pr / ((long long)C * NP);
    const long long row = a * block + (long long)D * R + (pr - a * C * NP);
    const double* v = val + rowptr[row];
    double* o = pvalT + ((pr >> 5) * dnv) * 32 + (pr & 31);
    for (int t = 0; t < dnv; ++t) o[(long long)t * 32] = v[t];
  }
}

stm_status build_nodeblock(Level& L, cudaStream_t s) { return build_nodeblock_from(L, L.val, L.nval, L.pvalT, s); }

stm_status build_nodeblock_from(const Level& L, const double* val, double* nval, double* pvalT, cudaStream_t s) {
  const int blocks = (int)std::min<long long>(((long long)L.R * 32 + 255) / 256, sm_count() * 8LL);
  k_build_nodeblock<<<blocks, 256, 0, s>>>(L.rowptr, val, L.nbr_ptr, L.ncell, L.nbase, nval, L.block, L.R, L.K,
                                           L.dim, L.np);
  note_launch();
  STM_CUDA(cudaGetLastError());
  const long long npr = (long long)L.K * L.C * L.np;
  const int pblocks = (int)std::min<long long>((npr + 255) / 256, sm_count() * 8LL);
  k_build_pval<<<std::max(pblocks, 1), 256, 0, s>>>(L.rowptr, val, pvalT, L.block, L.R, L.C, L.K, L.dim, L.np,
                                                    L.nv);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// Loads the K*d values of one node-block position (FP64: one by one; FP32 with K*d even: as float2,
// the position starts on an 8-byte boundary since every node block holds a multiple of K*d values).
template <int KD>
__device__ __forceinline__ void load_position(const double* v, double* out) {
#pragma unroll
  for (int r = 0; r < KD; ++r) out[r] = __ldcs(v + r);
}
template <int KD>
__device__ __forceinline__ void load_position(const float* v, float* out) {
  if constexpr (KD % 2 == 0) {
#pragma unroll
    for (int r = 0; r < KD; r += 2) {
      const float2 w = __ldcs(reinterpret_cast<const float2*>(v + r));
      out[r] = w.x;
      out[r + 1] = w.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < KD; ++r) out[r] = __ldcs(v + r);
  }
}

// VL lanes per node walk the node's positions; each position's K*d row values are contiguous, so VL
// consecutive positions are one contiguous run of VL*K*d values (whole lines even for VL = 4) and
// all lanes stay busy; the K*d partial sums go through the reduce-scatter butterfly (few adds).
// TV is the value and arithmetic type: double (the FP64 product), or float (FP32 copies of the
// values, FP32 products and sums; x and b are read in FP64 and y is written in FP64).
template <typename TV, int VL, int K, int D>
__global__ void __launch_bounds__(256, ((sizeof(TV) == 4 && VL > 8) || K < 3) ? 4 : 3) k_spmv_nodeblock(
    const TV* __restrict__ nval, const TV* __restrict__ pvalT,
    const long long* __restrict__ nbase, const int* __restrict__ nbr_ptr, const int* __restrict__ nbr,
    const int* __restrict__ ncell, const int* __restrict__ node_cells, const int* __restrict__ cell_nodes,
    const int* __restrict__ job_nodes, long long block, int R, int C, int nv, const TV* __restrict__ x,
    const double* __restrict__ b, double* __restrict__ y, int mode, int vpc) {
  constexpr int GPW = 32 / VL;
  constexpr int KD = K * D;
  constexpr int NP = D + 1;
  constexpr int MAXC = 1 << D;
  constexpr int NAV = pow2ceil(KD);
  static_assert(NAV <= VL || VL >= 4, "group too small");
  const int lane = threadIdx.x & (VL - 1);
  const int gw = (threadIdx.x & 31) / VL;
  const int wslot = threadIdx.x >> 5, nslot = blockDim.x >> 5;
  int wmask_v;
  constexpr int NAV_R = NAV < VL ? NAV : VL;
  const int kv = scatter_index<VL, NAV_R>(lane, &wmask_v);
  // vpc < 8: the first vpc warps of every CTA take the velocity rows node by node, the others the
  // pressure rows, so the two kinds of work (FP64-heavy, load-heavy) run side by side on every SM and
  // their latency chains overlap; vpc = 8: every warp takes velocity groups, then pressure rows
  const bool both = vpc >= nslot;
  if (both || wslot < vpc) {
  const int vs = both ? nslot : vpc;
  const long long vw = (long long)blockIdx.x * vs + wslot, nvw = (long long)gridDim.x * vs;
  for (long long wb = vw * GPW; wb < R; wb += nvw * GPW) {
    const long long job = wb + gw;
    const bool ok = job < R;
    const int i = ok ? job_nodes[job] : 0;
    TV acc[NAV];
#pragma unroll
    for (int r = 0; r < NAV; ++r) acc[r] = TV(0);
    if (ok) {
      const int p0 = nbr_ptr[i], nn = nbr_ptr[i + 1] - p0, nc = ncell[i];
      const TV* blk = nval + nbase[i];
      const int npv = KD * nn;
      int j = lane, bm = 0;
      while (j >= nn) { j -= nn; ++bm; }
      if constexpr (sizeof(TV) == 8) {
        for (int p = lane; p < npv; p += VL) {
          const int bb = bm / D, m = bm - bb * D;
          const TV xv = __ldg(x + bb * block + (long long)m * R + nbr[p0 + j]);
          TV vv[KD];
          load_position<KD>(blk + (long long)p * KD, vv);
#pragma unroll
          for (int r = 0; r < KD; ++r) acc[r] += vv[r] * xv;
          j += VL;
          while (j >= nn) { j -= nn; ++bm; }
        }
      } else {
        // FP32 values: half the bytes per position, so U positions per step keep U position loads
        // in flight per lane before the first FMA waits; positions past the end read nothing.
        // U = 3 on the large-level classes (80 registers); U = 2 keeps 64 registers and more warps
        // for the 16- and 32-lane classes of smaller levels (measured per level)
        constexpr int U = VL <= 8 ? 3 : 2;
        int jk[U], bk[U];
        jk[0] = j;
        bk[0] = bm;
#pragma unroll
        for (int k = 1; k < U; ++k) {
          jk[k] = jk[k - 1] + VL;
          bk[k] = bk[k - 1];
          while (jk[k] >= nn) { jk[k] -= nn; ++bk[k]; }
        }
        for (int p = lane; p < npv; p += U * VL) {
          TV v[U][KD], xk[U];
#pragma unroll
          for (int k = 0; k < U; ++k) {
#pragma unroll
            for (int r = 0; r < KD; ++r) v[k][r] = TV(0);
            xk[k] = TV(0);
            if (k == 0 || p + k * VL < npv) load_position<KD>(blk + (long long)(p + k * VL) * KD, v[k]);
          }
#pragma unroll
          for (int k = 0; k < U; ++k)
            if (k == 0 || p + k * VL < npv) {
              const int bb = bk[k] / D, m = bk[k] - bb * D;
              xk[k] = __ldg(x + bb * block + (long long)m * R + nbr[p0 + jk[k]]);
            }
#pragma unroll
          for (int k = 0; k < U; ++k)
#pragma unroll
            for (int r = 0; r < KD; ++r) acc[r] += v[k][r] * xk[k];
#pragma unroll
          for (int k = 0; k < U; ++k) {
            jk[k] += U * VL;
            while (jk[k] >= nn) { jk[k] -= nn; ++bk[k]; }
          }
        }
      }
      for (int tq = lane; tq < NP * nc; tq += VL) {
        const int ci = tq / NP, q = tq - ci * NP;
        const long long pc = (long long)D * R + (long long)node_cells[(long long)i * MAXC + ci] * NP + q;
        const TV* v = blk + (long long)(npv + tq) * KD;
#pragma unroll
        for (int a = 0; a < K; ++a) {
          const TV xp = __ldg(x + a * block + pc);
#pragma unroll
          for (int l = 0; l < D; ++l) acc[a * D + l] += __ldcs(v + a * D + l) * xp;
        }
      }
    }
    if constexpr (NAV <= VL) {
      reduce_scatter<VL, NAV>(acc, lane);
      if (ok && kv < KD && (lane & wmask_v) == 0) {
        const int a = kv / D, l = kv - a * D;
        const long long row = a * block + (long long)l * R + i;
        const double sum = (double)acc[0];
        if (mode == 0) y[row] = sum;
        else if (mode == 1) y[row] = b[row] - sum;
        else y[row] += sum;
      }
    } else {
      // more accumulators than lanes: plain butterfly sums, lane 0 writes all rows
#pragma unroll
      for (int r = 0; r < NAV; ++r)
#pragma unroll
        for (int off = VL / 2; off > 0; off >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off, VL);
      if (ok && lane == 0)
#pragma unroll
        for (int r = 0; r < KD; ++r) {
          const int a = r / D, l = r - a * D;
          const long long row = a * block + (long long)l * R + i;
          const double sum = (double)acc[r];
          if (mode == 0) y[row] = sum;
          else if (mode == 1) y[row] = b[row] - sum;
          else y[row] += sum;
        }
    }
  }
  }
  if (both || wslot >= vpc) {
    // Pressure rows: one lane per row pr = (a*C + c)*n_p + q over the warp-transposed copy, so entry
    // t of 32 consecutive rows is one contiguous 256-byte load; all lanes busy, no cross-lane sums.
    constexpr int NV = D == 2 ? 9 : 27;
    const int pslots = both ? nslot : nslot - vpc;
    const long long tid_g = ((long long)blockIdx.x * pslots + (both ? wslot : wslot - vpc)) * 32 + (threadIdx.x & 31);
    const long long nthreads = (long long)gridDim.x * pslots * 32;
    const long long npr = (long long)K * C * NP;
    for (long long pr = tid_g; pr < npr; pr += nthreads) {
      const int a = (int)(pr / ((long long)C * NP));
      const long long cq = pr - (long long)a * C * NP;
      const long long c = cq / NP;
      const long long row = a * block + (long long)D * R + cq;
      const TV* vr = pvalT + ((pr >> 5) * (D * NV)) * 32 + (pr & 31);
      const int* cn = cell_nodes + c * NV;
      const TV* xa = x + a * block;
      TV s = TV(0);
#pragma unroll
      for (int m = 0; m < D; ++m) {
#pragma unroll 9
        for (int jj = 0; jj < NV; ++jj)
          s += __ldcs(vr + (m * NV + jj) * 32) * __ldg(xa + (long long)m * R + __ldg(cn + jj));
      }
      const double sum = (double)s;
      if (mode == 0) y[row] = sum;
      else if (mode == 1) y[row] = b[row] - sum;
      else y[row] += sum;
    }
  }
}

// FP64 product with work handed out at run time. The work is cut into units: velocity units of GPW
// nodes (one group of VL lanes per node; job order reversed, so the nodes with most neighbours come
// first) followed by pressure units of 32 rows (one lane per row). A persistent grid of the resident
// CTA count takes units from one device counter (lane 0 of a warp fetches, the warp shares it), so every
// SM stays busy to the last unit and the end of the launch waits for one unit at most; the last CTA to
// finish resets the counter for the next launch (launches on one hierarchy are serialised). The group
// sums go through the reduce-scatter above: with more accumulators than lanes (2D), each lane ends with
// K*d/VL row sums (6 FP64 adds per node with VL = 4, K*d = 6), so the FP64 pipe spends its issue slots
// on the 2 nnz FMAs.
template <int VL, int K, int D, int U>
__global__ void __launch_bounds__(256) k_spmv_nb_dyn(
    const double* __restrict__ nval, const double* __restrict__ pvalT, const long long* __restrict__ nbase,
    const int* __restrict__ nbr_ptr, const int* __restrict__ nbr, const int* __restrict__ ncell,
    const int* __restrict__ node_cells, const int* __restrict__ cell_nodes, const int* __restrict__ job_nodes,
    long long block, int R, int C, const double* __restrict__ x, const double* __restrict__ b,
    double* __restrict__ y, int mode, unsigned* __restrict__ work, unsigned nvu, unsigned ntot, int njobs) {
  constexpr int GPW = 32 / VL;
  constexpr int KD = K * D;
  constexpr int NP = D + 1;
  constexpr int MAXC = 1 << D;
  constexpr int NV = D == 2 ? 9 : 27;
  constexpr int NAV = pow2ceil(KD);
  constexpr int HOLD = NAV > VL ? NAV / VL : 1;  // row sums each lane holds after the reduce-scatter
  constexpr int NAV_R = NAV < VL ? NAV : VL;
  const int lw = threadIdx.x & 31;
  const int lane = lw & (VL - 1);
  const int gw = lw / VL;
  int wmask_v;
  const int kv = NAV > VL ? scatter_index<VL, NAV>(lane, &wmask_v) : scatter_index<VL, NAV_R>(lane, &wmask_v);
  for (;;) {
    unsigned u = 0;
    if (lw == 0) u = atomicAdd(work, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= ntot) break;
    if (u < nvu) {
      const long long job = (long long)(nvu - 1 - u) * GPW + gw;
      const bool ok = job < njobs;
      const int i = ok ? job_nodes[job] : 0;
      double acc[NAV];
#pragma unroll
      for (int r = 0; r < NAV; ++r) acc[r] = 0.0;
      if (ok) {
        const int p0 = nbr_ptr[i], nn = nbr_ptr[i + 1] - p0, nc = ncell[i];
        const double* blk = nval + nbase[i];
        const int npv = KD * nn;
        // U positions per step: the loads of all U are issued before the first FMA waits (U = 1 is used:
        // two positions per step measured 93.2 against 89.4 us on the finest 2D dG(2) level and 567
        // against 564 us on the finest 3D dG(1) level, with fewer resident warps at 64-80 registers)
        int jk[U], bk[U];
        jk[0] = lane;
        bk[0] = 0;
        while (jk[0] >= nn) { jk[0] -= nn; ++bk[0]; }
#pragma unroll
        for (int k = 1; k < U; ++k) {
          jk[k] = jk[k - 1] + VL;
          bk[k] = bk[k - 1];
          while (jk[k] >= nn) { jk[k] -= nn; ++bk[k]; }
        }
        for (int p = lane; p < npv; p += U * VL) {
          double vv[U][KD], xk[U];
#pragma unroll
          for (int k = 0; k < U; ++k) {
            const bool live = k == 0 || p + k * VL < npv;
            const int bb = bk[k] / D, m = bk[k] - bb * D;
            xk[k] = live ? __ldg(x + bb * block + (long long)m * R + nbr[p0 + jk[k]]) : 0.0;
            if (live) load_position<KD>(blk + (long long)(p + k * VL) * KD, vv[k]);
            else
#pragma unroll
              for (int r = 0; r < KD; ++r) vv[k][r] = 0.0;
          }
#pragma unroll
          for (int k = 0; k < U; ++k)
#pragma unroll
            for (int r = 0; r < KD; ++r) acc[r] = fma(vv[k][r], xk[k], acc[r]);
#pragma unroll
          for (int k = 0; k < U; ++k) {
            jk[k] += U * VL;
            while (jk[k] >= nn) { jk[k] -= nn; ++bk[k]; }
          }
        }
        for (int tq = lane; tq < NP * nc; tq += VL) {
          const int ci = tq / NP, q = tq - ci * NP;
          const long long pc = (long long)D * R + (long long)node_cells[(long long)i * MAXC + ci] * NP + q;
          const double* v = blk + (long long)(npv + tq) * KD;
#pragma unroll
          for (int a = 0; a < K; ++a) {
            const double xp = __ldg(x + a * block + pc);
#pragma unroll
            for (int l = 0; l < D; ++l) acc[a * D + l] = fma(__ldcs(v + a * D + l), xp, acc[a * D + l]);
          }
        }
      }
      reduce_scatter<VL, NAV>(acc, lane);
      if (ok && (lane & wmask_v) == 0) {
#pragma unroll
        for (int h = 0; h < HOLD; ++h) {
          const int rr = kv + h;
          if (rr < KD) {
            const int a = rr / D, l = rr - a * D;
            const long long row = a * block + (long long)l * R + i;
            if (mode == 0) y[row] = acc[h];
            else if (mode == 1) y[row] = b[row] - acc[h];
            else y[row] += acc[h];
          }
        }
      }
    } else {
      // pressure rows pr = (a*C + c)*n_p + q: one lane per row over the warp-transposed copy
      const long long pr = (long long)(u - nvu) * 32 + lw;
      const long long npr = (long long)K * C * NP;
      if (pr < npr) {
        const int a = (int)(pr / ((long long)C * NP));
        const long long cq = pr - (long long)a * C * NP;
        const long long c = cq / NP;
        const long long row = a * block + (long long)D * R + cq;
        const double* vr = pvalT + ((pr >> 5) * (D * NV)) * 32 + (pr & 31);
        const int* cn = cell_nodes + c * NV;
        const double* xa = x + a * block;
        // three accumulators: three independent FMA chains per lane
        double s3[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int m = 0; m < D; ++m) {
#pragma unroll 9
          for (int jj = 0; jj < NV; ++jj)
            s3[jj % 3] = fma(__ldcs(vr + (m * NV + jj) * 32), __ldg(xa + (long long)m * R + __ldg(cn + jj)), s3[jj % 3]);
        }
        const double sacc = (s3[0] + s3[1]) + s3[2];
        if (mode == 0) y[row] = sacc;
        else if (mode == 1) y[row] = b[row] - sacc;
        else y[row] += sacc;
      }
    }
  }
  // the last CTA to finish resets the counter: every warp has fetched a unit past the end by then
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
      work[0] = 0u;
      work[1] = 0u;
      __threadfence();
    }
  }
}

static int sms_count();

template <typename TV, int VL, int K, int D>
static void launch_nodeblock(const Level& L, const TV* nval, const TV* pvalT, const TV* x, const double* b,
                             double* y, int mode, cudaStream_t s) {
  constexpr int GPW = 32 / VL;
  const long long npr = (long long)K * L.C * (D + 1);
  const long long need_v = (L.R + GPW - 1) / GPW, need_p = (npr + 31) / 32;
  int vpc;
  long long blocks;
  if (D == 2 && VL == 4) {
    // large 2D levels (velocity rows ~96% of the entries): every warp takes velocity groups, then
    // pressure rows, over a grid of up to 4 CTAs per SM. Where only 3 fit (80 registers) the last
    // quarter of the CTAs fills in as others retire; measured faster than a grid of the resident
    // count, twice it, or one unit per warp (FP64 98 against 107 us, FP32 56 against 62-69 us)
    vpc = 8;
    blocks = std::min<long long>(std::max((long long)L.R * VL, npr), (long long)sms_count() * 4 * 256);
    blocks = std::max<long long>(1, (blocks + 255) / 256);
  } else {
    // 3D and small 2D levels: one unit per warp (a group of GPW nodes, or 32 pressure rows), the two
    // kinds mixed in every CTA in proportion to their counts; CTAs are handed out as others retire
    vpc = (int)std::min<long long>(7, std::max<long long>(1, (8 * need_v + (need_v + need_p) / 2) / (need_v + need_p)));
    blocks = std::max<long long>(1, std::max((need_v + vpc - 1) / vpc, (need_p + (8 - vpc) - 1) / (8 - vpc)));
  }
  k_spmv_nodeblock<TV, VL, K, D><<<(int)blocks, 256, 0, s>>>(nval, pvalT, L.nbase, L.nbr_ptr, L.nbr, L.ncell,
                                                             L.node_cells, L.cell_nodes, L.job_nodes, L.block, L.R,
                                                             L.C, L.nv, x, b, y, mode, vpc);
}

template <typename TV>
static stm_status spmv_nodeblock_t(const Level& L, const TV* nval, const TV* pvalT, const TV* x, const double* b,
                                   double* y, int mode, cudaStream_t s) {
  // short groups (4 lanes in 2D, 8 in 3D) need at least ~1024 resident threads per SM to keep
  // enough loads in flight; smaller levels use 16 lanes per node
  const long long per_sm_threads = 1024;
  int cls = 0;  // 0: 4 (2D) / 8 (3D) lanes per node, 100: 16 lanes, 200: 32 lanes
  if ((long long)L.R * (L.dim == 2 ? 4 : 8) < (long long)sms_count() * per_sm_threads) cls = 100;
  if ((long long)L.R * 16 < (long long)sms_count() * per_sm_threads / 4) cls = 200;
  switch (L.dim * 10 + L.K + cls) {
    case 21: launch_nodeblock<TV, 4, 1, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 22: launch_nodeblock<TV, 4, 2, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 23: launch_nodeblock<TV, 4, 3, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 31: launch_nodeblock<TV, 8, 1, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 32: launch_nodeblock<TV, 8, 2, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 33: launch_nodeblock<TV, 8, 3, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 121: launch_nodeblock<TV, 16, 1, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 122: launch_nodeblock<TV, 16, 2, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 123: launch_nodeblock<TV, 16, 3, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 131: launch_nodeblock<TV, 16, 1, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 132: launch_nodeblock<TV, 16, 2, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 133: launch_nodeblock<TV, 16, 3, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 221: launch_nodeblock<TV, 32, 1, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 222: launch_nodeblock<TV, 32, 2, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 223: launch_nodeblock<TV, 32, 3, 2>(L, nval, pvalT, x, b, y, mode, s); break;
    case 231: launch_nodeblock<TV, 32, 1, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 232: launch_nodeblock<TV, 32, 2, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    case 233: launch_nodeblock<TV, 32, 3, 3>(L, nval, pvalT, x, b, y, mode, s); break;
    default:
      set_error("node-block SpMV: unsupported (dim, k)");
      return STM_ERR_INVALID_ARG;
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

template <int VL, int K, int D, int U>
static stm_status launch_nb_dyn(const Level& L, const double* nval, const double* pvalT, const double* x,
                                const double* b, double* y, int mode, cudaStream_t s, const int* jobs, int njobs) {
  constexpr int GPW = 32 / VL;
  static int occ = 0;  // resident CTAs per SM of this instantiation
  if (!occ) {
    STM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_nb_dyn<VL, K, D, U>, 256, 0));
    if (occ < 1) occ = 1;
  }
  const long long npr = (long long)K * L.C * (D + 1);
  const unsigned nvu = (unsigned)((njobs + GPW - 1) / GPW);
  const unsigned ntot = nvu + (unsigned)((npr + 31) / 32);
  const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)occ * sms_count(), (ntot + 7) / 8));
  k_spmv_nb_dyn<VL, K, D, U><<<blocks, 256, 0, s>>>(nval, pvalT, L.nbase, L.nbr_ptr, L.nbr, L.ncell, L.node_cells,
                                                 L.cell_nodes, jobs, L.block, L.R, L.C, x, b, y, mode,
                                                 L.spmv_work, nvu, ntot, njobs);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status spmv_nodeblock(const Level& L, const double* nval, const double* pvalT, const double* x, const double* b,
                          double* y, int mode, cudaStream_t s, const int* jobs, int njobs) {
  if (!jobs) {
    jobs = L.job_nodes;
    njobs = L.R;
  }
  // lanes per node as for the static product: short groups on large levels, 16 / 32 on small ones
  const long long per_sm_threads = 1024;
  int cls = 0;
  if ((long long)L.R * (L.dim == 2 ? 4 : 8) < (long long)sms_count() * per_sm_threads) cls = 100;
  if ((long long)L.R * 16 < (long long)sms_count() * per_sm_threads / 4) cls = 200;
  switch (L.dim * 10 + L.K + cls) {
    case 21: return launch_nb_dyn<4, 1, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 22: return launch_nb_dyn<4, 2, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 23: return launch_nb_dyn<4, 3, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 31: return launch_nb_dyn<8, 1, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 32: return launch_nb_dyn<8, 2, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 33: return launch_nb_dyn<8, 3, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 121: return launch_nb_dyn<16, 1, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 122: return launch_nb_dyn<16, 2, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 123: return launch_nb_dyn<16, 3, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 131: return launch_nb_dyn<16, 1, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 132: return launch_nb_dyn<16, 2, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 133: return launch_nb_dyn<16, 3, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 221: return launch_nb_dyn<32, 1, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 222: return launch_nb_dyn<32, 2, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 223: return launch_nb_dyn<32, 3, 2, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 231: return launch_nb_dyn<32, 1, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 232: return launch_nb_dyn<32, 2, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    case 233: return launch_nb_dyn<32, 3, 3, 1>(L, nval, pvalT, x, b, y, mode, s, jobs, njobs);
    default:
      set_error("node-block SpMV: unsupported (dim, k)");
      return STM_ERR_INVALID_ARG;
  }
}

// FP32 copy of an FP64 array (round to nearest)
__global__ void k_round_f32(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

static stm_status round_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  if (n <= 0) return STM_OK;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)sms_count() * 8));
  k_round_f32<<<blocks, 256, 0, s>>>(src, dst, n);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status build_values_f32(Level& L, int transpose, cudaStream_t s) {
  const double* nv = transpose ? L.nvalJT : L.nval;
  const double* pv = transpose ? L.pvalJT : L.pvalT;
  float*& n32 = transpose ? L.nvalJT32 : L.nval32;
  float*& p32 = transpose ? L.pvalJT32 : L.pval32;
  if (!nv) {
    set_error("FP32 defect copies: the FP64 node-block values are not built");
    return STM_ERR_STATE;
  }
  if (!n32) STM_CUDA(cudaMalloc((void**)&n32, sizeof(float) * std::max<long long>(1, L.nval_len)));
  if (!p32) STM_CUDA(cudaMalloc((void**)&p32, sizeof(float) * std::max<long long>(1, L.pval_len)));
  if (!L.x32) STM_CUDA(cudaMalloc((void**)&L.x32, sizeof(float) * std::max<long long>(1, L.N)));
  STM_TRY(round_f32(nv, n32, L.nval_len, s));
  if (pv) STM_TRY(round_f32(pv, p32, L.pval_len, s));
  return STM_OK;
}

// y = b - J x (or J^T x) over the FP32 copies: x is rounded to FP32 once (one pass over N, or by the
// kernel that wrote x), so the product gathers 4-byte entries and converts nothing
stm_status defect_f32(Hierarchy& H, int g, int transpose, const double* x, const double* b, double* y,
                      cudaStream_t s, bool x32_current) {
  Level& L = H.L[g];
  const float* nv = transpose ? L.nvalJT32 : L.nval32;
  const float* pv = transpose ? L.pvalJT32 : L.pval32;
  if (!nv || !pv || !L.x32) {
    set_error("FP32 defect copies missing: assemble the Jacobian first");
    return STM_ERR_STATE;
  }
  if (!x32_current) {
    ProfScope ps(&H, STM_KCLASS_ROUND_F32, s, 12.0 * (double)L.N, g);
    STM_TRY(round_f32(x, L.x32, L.N, s));
  }
  ProfScope ps(&H, STM_KCLASS_DEFECT_F32, s, 4.0 * (double)L.nnz + 20.0 * (double)L.N, g);
  return spmv_nodeblock_t<float>(L, nv, pv, L.x32, b, y, 1, s);
}

static int sms_count() { return sm_count(); }

}  // namespace stm
