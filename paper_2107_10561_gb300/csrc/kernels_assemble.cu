// Assembly of the slab Jacobian J_g on the GPU (FP64).
//
// J_g = sum_T R_T^T E_T R_T with the element blocks of Problem 3.1 linearised as in Eq. linNewEq:
//   velocity-velocity (a,l,i; b,m,j): D_ab M_ij d_lm + Mt_ab A_l,ij d_lm + sum_c T_abc N(w^c)_lm,ij
//   velocity-pressure (a,l,i; a,q)  : Mt_aa Bc_l,iq    pressure-velocity (a,q; a,m,j): Mt_aa Br_m,qj
// with A the diffusion + Nitsche operator (Eqs. Def:Ah, Def:B_GamD) and
//   N(w)_lm,ij = ((w . grad) phi_j d_lm + phi_j d_m w_l, phi_i).
// Cells are processed colour by colour (cells of one colour share no node), so every CSR entry
// is updated by at most one thread at a time: no atomics, bitwise reproducible.
#include "internal.h"

namespace stm {

// ---------------------------------------------------------------------------------------------
// CSR column indices from the structured pattern
// ---------------------------------------------------------------------------------------------
__global__ void k_fill_colidx(const long long* __restrict__ rowptr, int* __restrict__ colidx,
                              const int* __restrict__ nbr_ptr, const int* __restrict__ nbr,
                              const int* __restrict__ node_cells, const int* __restrict__ cell_nodes,
                              long long N, long long block, int R, int d, int K, int nv, int np,
                              int maxc) {
  const long long warps = (long long)gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  for (long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; row < N; row += warps) {
    const int a = (int)(row / block);
    const long long r = row - a * block;
    const long long base = rowptr[row];
    const int len = (int)(rowptr[row + 1] - base);
    if (r < (long long)d * R) {
      const int node = (int)(r % R);
      const int p0 = nbr_ptr[node];
      const int nn = nbr_ptr[node + 1] - p0;
      int nc = 0;
      while (nc < maxc && node_cells[(long long)node * maxc + nc] >= 0) ++nc;
      for (int p = lane; p < len; p += 32) {
        // columns per time block b: d*nn velocity, plus n_p*nc pressure when b == a
        int off = p, b = 0;
        for (; b < K; ++b) {
          const int sz = d * nn + (b == a ? np * nc : 0);
          if (off < sz) break;
          off -= sz;
        }
        long long col;
        if (off < d * nn) {
          const int m = off / nn, j = off - m * nn;
          col = b * block + (long long)m * R + nbr[p0 + j];
        } else {
          const int t = off - d * nn;
          const int ci = t / np, q = t - ci * np;
          col = a * block + (long long)d * R + (long long)node_cells[(long long)node * maxc + ci] * np + q;
        }
        colidx[base + p] = (int)col;
      }
    } else {
      const long long pr = r - (long long)d * R;
      const int c = (int)(pr / np);
      for (int p = lane; p < len; p += 32) {
        const int m = p / nv, j = p - m * nv;
        colidx[base + p] = (int)(a * block + (long long)m * R + cell_nodes[c * nv + j]);
      }
    }
  }
}

stm_status launch_fill_colidx(Level& L, const int* nbr_ptr, const int* nbr, const int* node_cells,
                              cudaStream_t s) {
  const int threads = 256;
  long long warps_needed = L.N;
  int blocks = (int)std::min<long long>((warps_needed + 7) / 8, sm_count() * 64LL);
  k_fill_colidx<<<blocks, threads, 0, s>>>(L.rowptr, L.colidx, nbr_ptr, nbr, node_cells, L.cell_nodes,
                                           L.N, L.block, L.R, L.dim, L.K, L.nv, L.np, 1 << L.dim); note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Linearisation point on every level (injection: coarse nodes are fine nodes)
// ---------------------------------------------------------------------------------------------
__global__ void k_inject(const double* __restrict__ X, double* __restrict__ wnod,
                         const int* __restrict__ inj, int R, int K, int d, long long blockF, int RF) {
  const long long total = (long long)K * d * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(e % R);
    const int al = (int)(e / R);  // a * d + l
    const int a = al / d, l = al - a * d;
    wnod[e] = X[a * blockF + (long long)l * RF + inj[node]];
  }
}

stm_status inject_level(const Hierarchy& H, int g, const double* X, double* wnod, cudaStream_t s) {
  const Level& F = H.L.back();
  const Level& L = H.L[g];
  long long total = (long long)L.K * L.dim * L.R;
  int blocks = (int)std::min<long long>((total + 255) / 256, sm_count() * 16LL);
  k_inject<<<std::max(blocks, 1), 256, 0, s>>>(X, wnod, L.inj, L.R, L.K, L.dim, F.block, F.R);
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status inject_linearisation(Hierarchy& H, const double* X, cudaStream_t s) {
  const Level& F = H.L.back();
  for (Level& L : H.L) {
    long long total = (long long)L.K * L.dim * L.R;
    int blocks = (int)std::min<long long>((total + 255) / 256, sm_count() * 16LL);
    k_inject<<<blocks, 256, 0, s>>>(X, L.wnod, L.inj, L.R, L.K, L.dim, F.block, F.R); note_launch();
    STM_CUDA(cudaGetLastError());
  }
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Element assembly
// ---------------------------------------------------------------------------------------------
struct AsmConst {
  double Mt[3][3], D[3][3], T[3][3][3];
  double nu, g1, g2, hT;
};

__global__ void __launch_bounds__(256) k_assemble(
    const int* __restrict__ cells, int ncells, const int* __restrict__ idx,
    const int* __restrict__ cell_nodes, const unsigned char* __restrict__ bmask,
    const unsigned char* __restrict__ rank, const unsigned char* __restrict__ cellrank,
    const int* __restrict__ nn, const int* __restrict__ ncell, const long long* __restrict__ rowptr,
    double* __restrict__ val, const double* __restrict__ wnod, const double* __restrict__ ref,
    RefOffsets ro, AsmConst ac, int d, int K, int R, int n, int nt) {
  extern __shared__ double sm[];
  const int nv = ro.nv, np = ro.np, nq = ro.nq;
  double* wq = sm;                       // [K][nq][d]
  double* gw = wq + K * nq * d;          // [K][nq][d][d]
  const double* W = ref + ro.W;
  const double* phi = ref + ro.phi;
  const double* gphi = ref + ro.gphi;
  const double* Mm = ref + ro.M;
  const double* Ks = ref + ro.Kst;
  const double* Div = ref + ro.Div;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x) {
    const int c = cells[ci];
    const int* cn = cell_nodes + (long long)c * nv;
    const unsigned mask = bmask[c];
    __syncthreads();
    // linearisation velocity and its gradient at the quadrature points, per time node
    for (int e = threadIdx.x; e < K * nq * d; e += blockDim.x) {
      const int l = e % d, q = (e / d) % nq, cc = e / (d * nq);
      const double* wl = wnod + ((long long)cc * d + l) * R;
      double v = 0.0;
      double g[3] = {0.0, 0.0, 0.0};
      for (int s = 0; s < nv; ++s) {
        const double ws = wl[cn[s]];
        v += phi[q * nv + s] * ws;
        for (int m = 0; m < d; ++m) g[m] += gphi[(q * nv + s) * d + m] * ws;
      }
      wq[(cc * nq + q) * d + l] = v;
      for (int m = 0; m < d; ++m) gw[((cc * nq + q) * d + l) * d + m] = g[m];
    }
    __syncthreads();
    // velocity-velocity blocks: one (i, j) pair per thread iteration
    for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) {
      const int i = e / nv, j = e - i * nv;
      double t1[3], t2[3][9];
      for (int cc = 0; cc < K; ++cc) {
        t1[cc] = 0.0;
        for (int lm = 0; lm < d * d; ++lm) t2[cc][lm] = 0.0;
      }
      for (int q = 0; q < nq; ++q) {
        const double u = W[q] * phi[q * nv + i];
        const double uj = u * phi[q * nv + j];
        const double* gj = gphi + (q * nv + j) * d;
        for (int cc = 0; cc < K; ++cc) {
          const double* wv = wq + (cc * nq + q) * d;
          double adv = 0.0;
          for (int m = 0; m < d; ++m) adv += wv[m] * gj[m];
          t1[cc] += u * adv;
          const double* gv = gw + (cc * nq + q) * d * d;
          for (int lm = 0; lm < d * d; ++lm) t2[cc][lm] += uj * gv[lm];
        }
      }
      // diffusion + Nitsche part (identical for all components except the gamma2 normal term)
      double base = ac.nu * Ks[i * nv + j];
      double g2axis[3] = {0.0, 0.0, 0.0};
      for (int f = 0; f < 2 * d; ++f) {
        if (!(mask & (1u << f))) continue;
        const double* F = ref + ro.face0 + f * ro.face_stride;
        base += -ac.nu * F[ro.fG + i * nv + j] - ac.nu * F[ro.fG + j * nv + i] +
                ac.g1 * ac.nu / ac.hT * F[ro.fS + i * nv + j];
        g2axis[f / 2] += ac.g2 / ac.hT * F[ro.fS + i * nv + j];
      }
      const int node_i = cn[i];
      const int nni = nn[node_i], nci = ncell[node_i];
      const int rk = rank[((long long)c * nv + i) * nv + j];
      for (int a = 0; a < K; ++a)
        for (int l = 0; l < d; ++l) {
          const long long row = idx[(long long)c * n + a * nt + l * nv + i];
          const long long rb = rowptr[row];
          for (int b = 0; b < K; ++b) {
            double t1ab = 0.0, t2ab[9];
            for (int lm = 0; lm < d * d; ++lm) t2ab[lm] = 0.0;
            for (int cc = 0; cc < K; ++cc) {
              const double tc = ac.T[a][b][cc];
              t1ab += tc * t1[cc];
              for (int lm = 0; lm < d * d; ++lm) t2ab[lm] += tc * t2[cc][lm];
            }
            const long long pb = rb + (long long)b * d * nni + (b > a ? np * nci : 0) + rk;
            for (int m = 0; m < d; ++m) {
              double v = t2ab[l * d + m];
              if (m == l) v += ac.D[a][b] * Mm[i * nv + j] + ac.Mt[a][b] * (base + g2axis[l]) + t1ab;
              val[pb + (long long)m * nni] += v;
            }
          }
        }
    }
    // pressure couplings (time-diagonal because the Radau-Lagrange time mass is diagonal)
    for (int e = threadIdx.x; e < K * d * nv * np; e += blockDim.x) {
      const int q = e % np, i = (e / np) % nv, l = (e / (np * nv)) % d, a = e / (np * nv * d);
      double bc = -Div[(l * np + q) * nv + i];
      for (int f = 2 * l; f < 2 * l + 2; ++f)
        if (mask & (1u << f)) bc += (2.0 * (f & 1) - 1.0) * ref[ro.face0 + f * ro.face_stride + ro.fPf + q * nv + i];
      const int node_i = cn[i];
      const int nni = nn[node_i];
      const long long row = idx[(long long)c * n + a * nt + l * nv + i];
      const long long pos = rowptr[row] + (long long)a * d * nni + (long long)d * nni +
                            (long long)cellrank[(long long)c * nv + i] * np + q;
      val[pos] += ac.Mt[a][a] * bc;
      // pressure row (a, q) against velocity (a, l, i): Br_l,qi
      double br = Div[(l * np + q) * nv + i];
      for (int f = 2 * l; f < 2 * l + 2; ++f)
        if (mask & (1u << f)) br -= (2.0 * (f & 1) - 1.0) * ref[ro.face0 + f * ro.face_stride + ro.fPf + q * nv + i];
      const long long prow = idx[(long long)c * n + a * nt + d * nv + q];
      val[rowptr[prow] + (long long)l * nv + i] += ac.Mt[a][a] * br;
    }
  }
}

stm_status assemble_level(Hierarchy& H, int g, double nu, cudaStream_t s) {
  Level& L = H.L[g];
  STM_CUDA(cudaMemsetAsync(L.val, 0, sizeof(double) * L.nnz, s));
  AsmConst ac;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      ac.Mt[a][b] = H.Mt[a][b];
      ac.D[a][b] = H.D[a][b];
      for (int c = 0; c < 3; ++c) ac.T[a][b][c] = H.T[a][b][c];
    }
  ac.nu = nu;
  ac.g1 = H.p.gamma1;
  ac.g2 = H.p.gamma2;
  ac.hT = L.hT;
  const size_t smem = sizeof(double) * (size_t)L.K * L.ro.nq * L.dim * (1 + L.dim);
  if (smem > 48 * 1024) STM_CUDA(cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int col = 0; col < (1 << L.dim); ++col) {
    const int nc = L.colour_off[col + 1] - L.colour_off[col];
    if (nc == 0) continue;
    const int blocks = std::min(nc, sm_count() * 8);
    k_assemble<<<blocks, 256, smem, s>>>(L.colour_cells + L.colour_off[col], nc, L.idx, L.cell_nodes,
                                         L.bmask, L.rank, L.cellrank, L.nn, L.ncell, L.rowptr, L.val,
                                         L.wnod, L.ref, L.ro, ac, L.dim, L.K, L.R, L.n, L.nt); note_launch();
    STM_CUDA(cudaGetLastError());
  }
  if (L.valT) {
    cudaFree(L.valT);
    L.valT = nullptr;
  }
  if (L.nvalJT) {
    cudaFree(L.nvalJT);
    L.nvalJT = nullptr;
  }
  if (L.pvalJT) {
    cudaFree(L.pvalJT);
    L.pvalJT = nullptr;
  }
  STM_TRY(build_nodeblock(L, s));
  // FP32 defect copies follow the new values (J^T's are rebuilt with J^T)
  if (H.p.defect_precision == STM_F32) STM_TRY(build_values_f32(L, 0, s));
  return STM_OK;
}

}  // namespace stm
