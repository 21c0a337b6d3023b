// Right-hand sides, functional weights and the viscosity derivative of J (adjoint / gradient path).
//
// With the linearisation point w fixed, one Newton step from w solves J(w; nu) X = b(U, nu) + c(w, w):
//   b(U, nu) = int_{I_n} B_GamD(g, (psi, xi)) dt + <v(t_{n-1}^-), psi(t_{n-1}^+)>   (Problem 3.1,
//   Eqs. Def:Lh, Def:B_GamD; f = 0), with the inflow data g = U g_1 on x = 0 (zero on walls and
//   obstacle) and the previous-slab state U g_1 e_x (Poiseuille field, exact in Q2), or, for time
//   marching, the discrete velocity of the previous slab's last time node (right Radau: t_{n-1});
//   c(w, w) = sum_{b,c} T_abc <(w^c . grad) w^b, psi>, the convection term at w (J(w) w - A(w) w).
// The drag-like functional is J(X) = int_{I_n} int_wake v_1 dx dt = j . X.
// b is linear in U and affine in nu; J is affine in nu with dJ/dnu = Mt (x) (K - G - G^T + gamma1/h S)
// per velocity component (diffusion and its Nitsche terms). Cells are processed colour by colour so
// that every scatter-add is race free and bitwise reproducible.
#include "internal.h"

namespace stm {

struct VecConst {
  double Mt[3], chi0[3], tint[3];  // Mt_aa, chi_a(0), int_{I_n} chi_a dt
  double T[3][3][3];
  double nu, g1, g2, hT, U;
  double H, L2;                    // channel height (y) and depth (z)
  double h[3];
  int wake_lo[3], wake_hi[3];      // functional region in this level's cell units
};

enum { VEC_RHS = 0, VEC_RHS_DU = 1, VEC_RHS_DNU = 2, VEC_FUNCTIONAL = 3 };

__device__ __forceinline__ double inflow_profile(int d, double y, double z, const VecConst& vc) {
  const double gy = 4.0 * y * (vc.H - y) / (vc.H * vc.H);
  if (d == 2) return gy;
  return gy * 4.0 * z * (vc.L2 - z) / (vc.L2 * vc.L2);
}

__global__ void __launch_bounds__(256) k_cellvec(const int* __restrict__ cells, int ncells, int mode,
                                                 const int* __restrict__ idx, const int* __restrict__ cell_nodes,
                                                 const int* __restrict__ cell_xyz, const unsigned char* __restrict__ bmask,
                                                 const double* __restrict__ wnod, const double* __restrict__ ref,
                                                 RefOffsets ro, VecConst vc, int d, int K, int R, int n, int nt,
                                                 const double* __restrict__ vprev, double* __restrict__ out) {
  extern __shared__ double sm[];
  const int nv = ro.nv, np = ro.np, nq = ro.nq;
  double* wq = sm;                // [K][nq][d]
  double* gw = wq + K * nq * d;   // [K][nq][d][d]
  double* pq = gw + K * nq * d * d;  // [nq][d] previous-slab velocity at the quadrature points
  const double* W = ref + ro.W;
  const double* phi = ref + ro.phi;
  const double* gphi = ref + ro.gphi;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x) {
    const int c = cells[ci];
    const int* cn = cell_nodes + (long long)c * nv;
    const int* xyz = cell_xyz + 3 * c;
    const double o[3] = {xyz[0] * vc.h[0], xyz[1] * vc.h[1], xyz[2] * vc.h[2]};
    const bool inflow = (bmask[c] & 1u) && xyz[0] == 0;
    bool in_wake = true;
    for (int m = 0; m < d; ++m) in_wake = in_wake && xyz[m] >= vc.wake_lo[m] && xyz[m] < vc.wake_hi[m];
    __syncthreads();
    if (mode == VEC_RHS) {
      for (int e = threadIdx.x; e < K * nq * d; e += blockDim.x) {
        const int l = e % d, q = (e / d) % nq, cc = e / (d * nq);
        const double* wl = wnod + ((long long)cc * d + l) * R;
        double v = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int s = 0; s < nv; ++s) {
          const double ws = wl[cn[s]];
          v += phi[q * nv + s] * ws;
          for (int m = 0; m < d; ++m) g[m] += gphi[(q * nv + s) * d + m] * ws;
        }
        wq[(cc * nq + q) * d + l] = v;
        for (int m = 0; m < d; ++m) gw[((cc * nq + q) * d + l) * d + m] = g[m];
      }
      if (vprev)
        for (int e = threadIdx.x; e < nq * d; e += blockDim.x) {
          const int l = e % d, q = e / d;
          const double* vl = vprev + (long long)l * R;
          double v = 0.0;
          for (int s2 = 0; s2 < nv; ++s2) v += phi[q * nv + s2] * vl[cn[s2]];
          pq[q * d + l] = v;
        }
    }
    __syncthreads();
    for (int al = threadIdx.x; al < n; al += blockDim.x) {
      const int a = al / nt, r = al - a * nt;
      double v = 0.0;
      if (r < d * nv) {
        const int l = r / nv, i = r - l * nv;
        if (mode == VEC_FUNCTIONAL) {
          if (l == 0 && in_wake) {
            double s = 0.0;
            for (int q = 0; q < nq; ++q) s += W[q] * phi[q * nv + i];
            v = vc.tint[a] * s;
          }
        } else {
          if (l == 0 && inflow) {
            double s_n = 0.0, s_p = 0.0;
            for (int qf = 0; qf < ro.nqf; ++qf) {
              const double y = o[1] + vc.h[1] * ref[ro.XF + qf * d + 1];
              const double z = d == 3 ? o[2] + vc.h[2] * ref[ro.XF + qf * d + 2] : 0.0;
              const double gq = inflow_profile(d, y, z, vc) * ref[ro.WF + qf];
              s_n += gq * ref[ro.gnF + qf * nv + i];
              s_p += gq * ref[ro.phiF + qf * nv + i];
            }
            if (mode == VEC_RHS_DNU) v += vc.U * vc.tint[a] * (-s_n + vc.g1 / vc.hT * s_p);
            else v += (mode == VEC_RHS ? vc.U : 1.0) * vc.tint[a] * (-vc.nu * s_n + (vc.g1 * vc.nu + vc.g2) / vc.hT * s_p);
          }
          if (mode == VEC_RHS && vprev) {
            // <v_h(t_{n-1}^-), psi(t_{n-1}^+)> with the discrete previous-slab velocity
            double s = 0.0;
            for (int q = 0; q < nq; ++q) s += W[q] * phi[q * nv + i] * pq[q * d + l];
            v += vc.chi0[a] * s;
          } else if (l == 0 && mode != VEC_RHS_DNU) {
            double s = 0.0;
            for (int q = 0; q < nq; ++q) {
              const double y = o[1] + vc.h[1] * ref[ro.Xq + q * d + 1];
              const double z = d == 3 ? o[2] + vc.h[2] * ref[ro.Xq + q * d + 2] : 0.0;
              s += W[q] * inflow_profile(d, y, z, vc) * phi[q * nv + i];
            }
            v += (mode == VEC_RHS ? vc.U : 1.0) * vc.chi0[a] * s;
          }
          if (mode == VEC_RHS) {
            double s = 0.0;
            for (int b = 0; b < K; ++b)
              for (int cc = 0; cc < K; ++cc) {
                const double tabc = vc.T[a][b][cc];
                if (tabc == 0.0) continue;
                double sq = 0.0;
                for (int q = 0; q < nq; ++q) {
                  double adv = 0.0;
                  for (int m = 0; m < d; ++m) adv += wq[(cc * nq + q) * d + m] * gw[((b * nq + q) * d + l) * d + m];
                  sq += W[q] * phi[q * nv + i] * adv;
                }
                s += tabc * sq;
              }
            v += s;
          }
        }
      } else if (inflow && (mode == VEC_RHS || mode == VEC_RHS_DU)) {
        const int q = r - d * nv;
        double s = 0.0;
        for (int qf = 0; qf < ro.nqf; ++qf) {
          const double y = o[1] + vc.h[1] * ref[ro.XF + qf * d + 1];
          const double z = d == 3 ? o[2] + vc.h[2] * ref[ro.XF + qf * d + 2] : 0.0;
          s += inflow_profile(d, y, z, vc) * ref[ro.WF + qf] * ref[ro.xiF + qf * np + q];
        }
        v = (mode == VEC_RHS ? vc.U : 1.0) * vc.tint[a] * s;
      }
      if (v != 0.0) out[idx[(long long)c * n + al]] += v;
    }
  }
}

// y += (dJ/dnu) x over the cells of one colour: velocity rows only, time-diagonal (Mt diagonal).
__global__ void __launch_bounds__(256) k_dnu_apply(const int* __restrict__ cells, int ncells,
                                                   const int* __restrict__ idx, const unsigned char* __restrict__ bmask,
                                                   const double* __restrict__ ref, RefOffsets ro, VecConst vc, int d,
                                                   int K, int n, int nt, const double* __restrict__ x,
                                                   double* __restrict__ y) {
  const int nv = ro.nv;
  for (int ci = blockIdx.x; ci < ncells; ci += gridDim.x) {
    const int c = cells[ci];
    const unsigned mask = bmask[c];
    const int* ic = idx + (long long)c * n;
    for (int e = threadIdx.x; e < K * d * nv; e += blockDim.x) {
      const int i = e % nv, l = (e / nv) % d, a = e / (nv * d);
      const int* xr = ic + a * nt + l * nv;
      double s = 0.0;
      for (int j = 0; j < nv; ++j) {
        double aij = ref[ro.Kst + i * nv + j];
        for (int f = 0; f < 2 * d; ++f) {
          if (!(mask & (1u << f))) continue;
          const double* F = ref + ro.face0 + f * ro.face_stride;
          aij += -F[ro.fG + i * nv + j] - F[ro.fG + j * nv + i] + vc.g1 / vc.hT * F[ro.fS + i * nv + j];
        }
        s += aij * x[xr[j]];
      }
      y[xr[i]] += vc.Mt[a] * s;
    }
  }
}

static VecConst make_vc(const Hierarchy& H, const Level& L, double U, double nu) {
  VecConst vc{};
  const int K = L.K;
  double s[3];
  // chi_a(0): D_ab = int chi_b' chi_a + chi_b(0) chi_a(0) and sum_b chi_b = 1 give sum_b D_ab = chi_a(0)
  for (int a = 0; a < 3; ++a) {
    vc.Mt[a] = a < K ? H.Mt[a][a] : 0.0;
    double rs = 0.0, ts = 0.0;
    for (int b = 0; b < K && a < K; ++b) {
      rs += H.D[a][b];
      ts += H.Mt[a][b];
    }
    vc.chi0[a] = rs;
    vc.tint[a] = ts;
    s[a] = 0.0;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) vc.T[a][b][c] = H.T[a][b][c];
  }
  (void)s;
  vc.nu = nu;
  vc.g1 = H.p.gamma1;
  vc.g2 = H.p.gamma2;
  vc.hT = L.hT;
  vc.U = U;
  vc.H = H.p.length[1];
  vc.L2 = H.p.dim == 3 ? H.p.length[2] : 1.0;
  for (int m = 0; m < 3; ++m) vc.h[m] = L.h[m];
  return vc;
}

stm_status assemble_cellvec(Hierarchy& H, int mode, double U, double nu, const int* wake_lo, const int* wake_hi,
                            double* out, cudaStream_t s, const double* vprev, const double* wnod) {
  Level& L = H.L.back();
  VecConst vc = make_vc(H, L, U, nu);
  const int f = 1 << ((int)H.L.size() - 1);
  for (int m = 0; m < 3; ++m) {
    vc.wake_lo[m] = wake_lo ? wake_lo[m] * f : 0;
    vc.wake_hi[m] = wake_hi ? wake_hi[m] * f : 0;
    if (m >= L.dim) {
      vc.wake_lo[m] = 0;
      vc.wake_hi[m] = 1;
    }
  }
  STM_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * L.N, s));
  const size_t smem = sizeof(double) * ((size_t)L.K * L.ro.nq * L.dim * (1 + L.dim) + (size_t)L.ro.nq * L.dim);
  if (smem > 48 * 1024) STM_CUDA(cudaFuncSetAttribute(k_cellvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int col = 0; col < (1 << L.dim); ++col) {
    const int nc = L.colour_off[col + 1] - L.colour_off[col];
    if (!nc) continue;
    k_cellvec<<<std::min(nc, sm_count() * 8), 256, smem, s>>>(L.colour_cells + L.colour_off[col], nc, mode, L.idx,
                                                       L.cell_nodes, L.cell_xyz, L.bmask, wnod ? wnod : L.wnod, L.ref, L.ro, vc,
                                                       L.dim, L.K, L.R, L.n, L.nt, mode == 0 ? vprev : nullptr,
                                                       out);
    note_launch();
    STM_CUDA(cudaGetLastError());
  }
  return STM_OK;
}

stm_status dnu_apply(Hierarchy& H, const double* x, double* y, cudaStream_t s) {
  Level& L = H.L.back();
  const VecConst vc = make_vc(H, L, 0.0, H.p.nu);
  STM_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * L.N, s));
  for (int col = 0; col < (1 << L.dim); ++col) {
    const int nc = L.colour_off[col + 1] - L.colour_off[col];
    if (!nc) continue;
    k_dnu_apply<<<std::min(nc, sm_count() * 8), 256, 0, s>>>(L.colour_cells + L.colour_off[col], nc, L.idx, L.bmask, L.ref,
                                                      L.ro, vc, L.dim, L.K, L.n, L.nt, x, y);
    note_launch();
    STM_CUDA(cudaGetLastError());
  }
  return STM_OK;
}

}  // namespace stm
