// Intergrid transfers of the V-cycle (Algorithm 1: c_g = P d_{g-1} added to d_g, r_{g-1} = P^T t_g),
// applied from the mesh structure instead of an assembled P.
//
// P interpolates the coarse Q2/P1disc function on the fine level (Sec. 4.4: nested meshes, so the
// coarse space is contained in the fine one). For the velocity, the fine nodal value is the coarse
// Q2 interpolant at that node: one list of (coarse node, weight) per fine node, the same for all
// K*d (time node, component) blocks, so it is read once and applied to all of them. For the
// pressure, a fine cell's Legendre P1 coefficients follow from its parent's (child position o_m):
//   c0' = c0 + sum_m sqrt(3) (o_m - 1/2) c_m,    c_m' = c_m / 2.
// The restriction applies P^T with the transposed node lists and the 2^d children of each coarse
// cell. A group of lanes per node splits its list (so the chains of dependent loads stay short),
// one thread per cell; no atomics.
#include "internal.h"

namespace stm {

static int sm_count_tr() { return sm_count(); }

struct TransferGeom {
  long long fblock, cblock;  // DoFs per time node on the fine / coarse level
  int fR, cR, fC, cC;        // velocity nodes and cells
};

// fine += P coarse. Velocity: G lanes per fine node share its (coarse node, weight) list and meet
// through shuffles (short dependent-load chains); then one thread per fine cell for the pressure.
// The velocity range is padded to whole warps so that every warp is entirely in one part.
template <int K, int D, int G>
__global__ void k_prolong(const int* __restrict__ vptr, const int* __restrict__ vnode, const double* __restrict__ vw,
                          const int* __restrict__ parent, const unsigned char* __restrict__ bits, TransferGeom g,
                          const double* __restrict__ xc, double* __restrict__ yf, float* __restrict__ yf32) {
  constexpr int NP = D + 1;
  const double s3 = 1.7320508075688772;  // sqrt(3), P1 Legendre normalisation
  const long long vthreads = ((long long)g.fR * G + 31) / 32 * 32;
  const long long items = vthreads + g.fC;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    if (it < vthreads) {
      const long long nd = it / G;
      const int gl = (int)(it % G);
      double acc[K * D];
#pragma unroll
      for (int r = 0; r < K * D; ++r) acc[r] = 0.0;
      if (nd < g.fR)
        for (int e = vptr[nd] + gl; e < vptr[nd + 1]; e += G) {
          const int cn = vnode[e];
          const double w = vw[e];
#pragma unroll
          for (int a = 0; a < K; ++a)
#pragma unroll
            for (int l = 0; l < D; ++l) acc[a * D + l] += w * __ldg(xc + a * g.cblock + (long long)l * g.cR + cn);
        }
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
        for (int r = 0; r < K * D; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off, G);
      if (nd < g.fR)
#pragma unroll
        for (int r = 0; r < K * D; ++r)
          if (r % G == gl) {
            const long long e = (r / D) * g.fblock + (long long)(r % D) * g.fR + nd;
            const double v = yf[e] + acc[r];
            yf[e] = v;
            if (yf32) yf32[e] = __double2float_rn(v);
          }
    } else {
      const int cf = (int)(it - vthreads);
      const int pc = parent[cf];
      const int b = bits[cf];
#pragma unroll
      for (int a = 0; a < K; ++a) {
        const double* c = xc + a * g.cblock + (long long)D * g.cR + (long long)pc * NP;
        const long long fo = a * g.fblock + (long long)D * g.fR + (long long)cf * NP;
        double* f = yf + fo;
        double c0 = c[0];
#pragma unroll
        for (int m = 0; m < D; ++m) c0 += s3 * ((double)((b >> m) & 1) - 0.5) * c[1 + m];
        f[0] += c0;
#pragma unroll
        for (int m = 0; m < D; ++m) f[1 + m] += 0.5 * c[1 + m];
        if (yf32)
#pragma unroll
          for (int q = 0; q < NP; ++q) yf32[fo + q] = __double2float_rn(f[q]);
      }
    }
  }
}

// coarse = P^T fine; G lanes per coarse node over its transposed list (up to 5^d entries), as above
template <int K, int D, int G>
__global__ void k_restrict(const int* __restrict__ cptr, const int* __restrict__ cnode, const double* __restrict__ cw,
                           const int* __restrict__ children, TransferGeom g, const double* __restrict__ tf,
                           double* __restrict__ rc) {
  constexpr int NP = D + 1;
  constexpr int NCH = 1 << D;
  const double s3 = 1.7320508075688772;
  const long long vthreads = ((long long)g.cR * G + 31) / 32 * 32;
  const long long items = vthreads + g.cC;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    if (it < vthreads) {
      const long long cn = it / G;
      const int gl = (int)(it % G);
      double acc[K * D];
#pragma unroll
      for (int r = 0; r < K * D; ++r) acc[r] = 0.0;
      if (cn < g.cR)
        for (int e = cptr[cn] + gl; e < cptr[cn + 1]; e += G) {
          const int nd = cnode[e];
          const double w = cw[e];
#pragma unroll
          for (int a = 0; a < K; ++a)
#pragma unroll
            for (int l = 0; l < D; ++l) acc[a * D + l] += w * __ldg(tf + a * g.fblock + (long long)l * g.fR + nd);
        }
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
        for (int r = 0; r < K * D; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off, G);
      if (cn < g.cR)
#pragma unroll
        for (int r = 0; r < K * D; ++r)
          if (r % G == gl) rc[(r / D) * g.cblock + (long long)(r % D) * g.cR + cn] = acc[r];
    } else {
      const int pc = (int)(it - vthreads);
#pragma unroll
      for (int a = 0; a < K; ++a) {
        double acc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) acc[q] = 0.0;
#pragma unroll
        for (int b = 0; b < NCH; ++b) {
          const int cf = children[(long long)pc * NCH + b];
          const double* f = tf + a * g.fblock + (long long)D * g.fR + (long long)cf * NP;
          const double f0 = __ldg(f);
          acc[0] += f0;
#pragma unroll
          for (int m = 0; m < D; ++m) acc[1 + m] += s3 * ((double)((b >> m) & 1) - 0.5) * f0 + 0.5 * __ldg(f + 1 + m);
        }
        double* c = rc + a * g.cblock + (long long)D * g.cR + (long long)pc * NP;
#pragma unroll
        for (int q = 0; q < NP; ++q) c[q] = acc[q];
      }
    }
  }
}

static TransferGeom geom(const Level& F, const Level& Cl) {
  return TransferGeom{F.block, Cl.block, F.R, Cl.R, F.C, Cl.C};
}

// Lanes per node: fine-node lists hold up to 3^d entries, coarse-node lists up to 5^d. Groups of
// lanes shorten the chains of dependent loads on the smaller levels; on large levels (at least
// many_nodes(d) nodes) one thread per node keeps the stores of consecutive nodes contiguous, which
// measured faster there. The 3D lists are longer, so the groups pay off up to larger levels.
constexpr long long many_nodes(int d) { return d == 2 ? 16384 : 65536; }

template <int K, int D, int G>
static void launch_prolong_g(const Level& F, const TransferGeom& g, const double* xc, double* yf, float* yf32,
                             cudaStream_t s) {
  const long long items = ((long long)g.fR * G + 31) / 32 * 32 + g.fC;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((items + 255) / 256, sm_count_tr() * 8LL));
  k_prolong<K, D, G><<<blocks, 256, 0, s>>>(F.tv_ptr, F.tv_node, F.tv_w, F.cparent, F.cbits, g, xc, yf, yf32);
}

template <int K, int D>
static void launch_prolong(const Level& F, const TransferGeom& g, const double* xc, double* yf, float* yf32,
                           cudaStream_t s) {
  if (g.fR >= many_nodes(D)) launch_prolong_g<K, D, 1>(F, g, xc, yf, yf32, s);
  else launch_prolong_g<K, D, D == 2 ? 4 : 8>(F, g, xc, yf, yf32, s);
}

template <int K, int D, int G>
static void launch_restrict_g(const Level& F, const TransferGeom& g, const double* tf, double* rc, cudaStream_t s) {
  const long long items = ((long long)g.cR * G + 31) / 32 * 32 + g.cC;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((items + 255) / 256, sm_count_tr() * 8LL));
  k_restrict<K, D, G><<<blocks, 256, 0, s>>>(F.tc_ptr, F.tc_node, F.tc_w, F.cchildren, g, tf, rc);
}

template <int K, int D>
static void launch_restrict(const Level& F, const TransferGeom& g, const double* tf, double* rc, cudaStream_t s) {
  if (g.cR >= many_nodes(D)) launch_restrict_g<K, D, 1>(F, g, tf, rc, s);
  else launch_restrict_g<K, D, D == 2 ? 8 : 16>(F, g, tf, rc, s);
}

stm_status transfer_prolong_add(const Level& F, const Level& Cl, const double* coarse, double* fine, cudaStream_t s,
                                float* fine32) {
  const TransferGeom g = geom(F, Cl);
  switch (F.dim * 10 + F.K) {
    case 21: launch_prolong<1, 2>(F, g, coarse, fine, fine32, s); break;
    case 22: launch_prolong<2, 2>(F, g, coarse, fine, fine32, s); break;
    case 23: launch_prolong<3, 2>(F, g, coarse, fine, fine32, s); break;
    case 31: launch_prolong<1, 3>(F, g, coarse, fine, fine32, s); break;
    case 32: launch_prolong<2, 3>(F, g, coarse, fine, fine32, s); break;
    case 33: launch_prolong<3, 3>(F, g, coarse, fine, fine32, s); break;
    default:
      set_error("prolongation: unsupported (dim, k)");
      return STM_ERR_INVALID_ARG;
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

stm_status transfer_restrict(const Level& F, const Level& Cl, const double* fine, double* coarse, cudaStream_t s) {
  const TransferGeom g = geom(F, Cl);
  switch (F.dim * 10 + F.K) {
    case 21: launch_restrict<1, 2>(F, g, fine, coarse, s); break;
    case 22: launch_restrict<2, 2>(F, g, fine, coarse, s); break;
    case 23: launch_restrict<3, 2>(F, g, fine, coarse, s); break;
    case 31: launch_restrict<1, 3>(F, g, fine, coarse, s); break;
    case 32: launch_restrict<2, 3>(F, g, fine, coarse, s); break;
    case 33: launch_restrict<3, 3>(F, g, fine, coarse, s); break;
    default:
      set_error("restriction: unsupported (dim, k)");
      return STM_ERR_INVALID_ARG;
  }
  note_launch();
  STM_CUDA(cudaGetLastError());
  return STM_OK;
}

}  // namespace stm
