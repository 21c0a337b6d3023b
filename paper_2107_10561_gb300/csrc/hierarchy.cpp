// Host-side set-up of the level hierarchy: numbering, cell->DoF maps, boundary masks, colours,
// multiplicities, CSR patterns of J_g, transfer matrices and reference tables. Integer work and
// small FP64 tables only; every per-cell or per-entry floating-point computation runs on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace stm {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* last_error_cstr() { return g_err.c_str(); }

stm_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? STM_ERR_OOM : STM_ERR_CUDA;
}

// ---------------------------------------------------------------------------------------------
// 1D polynomials and rules
// ---------------------------------------------------------------------------------------------
// Quadratic Lagrange polynomials on [0,1] with nodes 0, 1/2, 1.
static double q2v(int a, double x) {
  switch (a) {
    case 0: return 2.0 * (x - 0.5) * (x - 1.0);
    case 1: return -4.0 * x * (x - 1.0);
    default: return 2.0 * x * (x - 0.5);
  }
}
static double q2d(int a, double x) {
  switch (a) {
    case 0: return 4.0 * x - 3.0;
    case 1: return -8.0 * x + 4.0;
    default: return 4.0 * x - 1.0;
  }
}

// Gauss-Legendre points/weights on [0,1] (Newton iteration on the Legendre recurrence).
static void gauss01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Right Gauss-Radau points of [0,1] (end point included), closed forms for k <= 2.
static void radau_right(int k, double* s) {
  if (k == 0) {
    s[0] = 1.0;
  } else if (k == 1) {
    s[0] = 1.0 / 3.0;
    s[1] = 1.0;
  } else {
    s[0] = (4.0 - std::sqrt(6.0)) / 10.0;
    s[1] = (4.0 + std::sqrt(6.0)) / 10.0;
    s[2] = 1.0;
  }
}

// Temporal matrices of one slab (Problem 3.1 with the Lagrange basis at the Radau points):
// Mt_ab = tau int chi_a chi_b, D_ab = int chi_b' chi_a + chi_b(0) chi_a(0), T_abc = tau int chi_a chi_b chi_c.
void time_matrices(int k, double tau, double Mt[3][3], double D[3][3], double T[3][3][3]) {
  const int K = k + 1;
  double s[3];
  radau_right(k, s);
  auto lag = [&](int a, double t, double* der) {
    double v = 1.0, dv = 0.0;
    for (int b = 0; b < K; ++b) {
      if (b == a) continue;
      double f = (t - s[b]) / (s[a] - s[b]);
      dv = dv * f + v / (s[a] - s[b]);
      v *= f;
    }
    if (der) *der = dv;
    return v;
  };
  double gx[8], gw[8];
  const int nq = k + 3;
  gauss01(nq, gx, gw);
  std::memset(Mt, 0, sizeof(double) * 9);
  std::memset(D, 0, sizeof(double) * 9);
  std::memset(T, 0, sizeof(double) * 27);
  for (int q = 0; q < nq; ++q) {
    double v[3], dv[3];
    for (int a = 0; a < K; ++a) v[a] = lag(a, gx[q], &dv[a]);
    for (int a = 0; a < K; ++a)
      for (int b = 0; b < K; ++b) {
        Mt[a][b] += tau * gw[q] * v[a] * v[b];
        D[a][b] += gw[q] * dv[b] * v[a];
        for (int c = 0; c < K; ++c) T[a][b][c] += tau * gw[q] * v[a] * v[b] * v[c];
      }
  }
  double v0[3];
  for (int a = 0; a < K; ++a) v0[a] = lag(a, 0.0, nullptr);
  for (int a = 0; a < K; ++a)
    for (int b = 0; b < K; ++b) D[a][b] += v0[b] * v0[a];
}

// ---------------------------------------------------------------------------------------------
// Device upload helpers
// ---------------------------------------------------------------------------------------------
template <typename T>
static stm_status upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return STM_OK;
  STM_CUDA(cudaMalloc((void**)dst, sizeof(T) * src.size()));
  STM_CUDA(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return STM_OK;
}

// ---------------------------------------------------------------------------------------------
// Reference tables of a uniform level
// ---------------------------------------------------------------------------------------------
static void local_offsets(int dim, int i, int* o) {
  o[0] = i % 3;
  o[1] = (i / 3) % 3;
  o[2] = (dim == 3) ? (i / 9) : 0;
}

static stm_status build_reference(Level& L) {
  const int d = L.dim, nv = L.nv, np = L.np;
  int nq = 1;
  for (int m = 0; m < d; ++m) nq *= kQ1;
  RefOffsets o{};
  o.nq = nq;
  o.nv = nv;
  o.np = np;
  int off = 0;
  o.W = off; off += nq;
  o.phi = off; off += nq * nv;
  o.gphi = off; off += nq * nv * d;
  o.M = off; off += nv * nv;
  o.Kst = off; off += nv * nv;
  o.Div = off; off += d * np * nv;
  o.face0 = off;
  o.fS = 0;
  o.fG = nv * nv;
  o.fPf = 2 * nv * nv;
  o.face_stride = 2 * nv * nv + np * nv;
  off += 2 * d * o.face_stride;
  int nqf0 = 1;
  for (int m = 0; m < d - 1; ++m) nqf0 *= kQ1;
  o.Xq = off; off += nq * d;
  o.nqf = nqf0;
  o.XF = off; off += nqf0 * d;
  o.WF = off; off += nqf0;
  o.phiF = off; off += nqf0 * nv;
  o.gnF = off; off += nqf0 * nv;
  o.xiF = off; off += nqf0 * np;
  o.total = off;
  std::vector<double> ref(off, 0.0);
  double gx[kQ1], gw[kQ1];
  gauss01(kQ1, gx, gw);
  double vol = 1.0;
  for (int m = 0; m < d; ++m) vol *= L.h[m];
  // volume points (x fastest)
  std::vector<double> X(nq * 3, 0.0), Wq(nq);
  for (int q = 0; q < nq; ++q) {
    int qi[3] = {q % kQ1, (q / kQ1) % kQ1, q / (kQ1 * kQ1)};
    double w = 1.0;
    for (int m = 0; m < d; ++m) {
      X[q * 3 + m] = gx[qi[m]];
      w *= gw[qi[m]];
    }
    Wq[q] = w;
    ref[o.W + q] = w * vol;
  }
  auto basis = [&](const double* x, int i, double* val, double* grad) {
    int oi[3];
    local_offsets(d, i, oi);
    double v = 1.0;
    for (int m = 0; m < d; ++m) v *= q2v(oi[m], x[m]);
    *val = v;
    for (int mm = 0; mm < d; ++mm) {
      double g = 1.0;
      for (int m = 0; m < d; ++m) g *= (m == mm) ? q2d(oi[m], x[m]) : q2v(oi[m], x[m]);
      grad[mm] = g / L.h[mm];
    }
  };
  auto pbasis = [&](const double* x, int q) {
    return q == 0 ? 1.0 : std::sqrt(3.0) * (2.0 * x[q - 1] - 1.0);
  };
  std::vector<double> phi(nq * nv), gphi(nq * nv * 3);
  for (int q = 0; q < nq; ++q)
    for (int i = 0; i < nv; ++i) {
      double g[3];
      basis(&X[q * 3], i, &phi[q * nv + i], g);
      ref[o.phi + q * nv + i] = phi[q * nv + i];
      for (int m = 0; m < d; ++m) {
        gphi[(q * nv + i) * 3 + m] = g[m];
        ref[o.gphi + (q * nv + i) * d + m] = g[m];
      }
    }
  for (int i = 0; i < nv; ++i)
    for (int j = 0; j < nv; ++j) {
      double m_ = 0.0, k_ = 0.0;
      for (int q = 0; q < nq; ++q) {
        m_ += Wq[q] * vol * phi[q * nv + i] * phi[q * nv + j];
        double dot = 0.0;
        for (int m = 0; m < d; ++m) dot += gphi[(q * nv + i) * 3 + m] * gphi[(q * nv + j) * 3 + m];
        k_ += Wq[q] * vol * dot;
      }
      ref[o.M + i * nv + j] = m_;
      ref[o.Kst + i * nv + j] = k_;
    }
  for (int m = 0; m < d; ++m)
    for (int a = 0; a < np; ++a)
      for (int j = 0; j < nv; ++j) {
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += Wq[q] * vol * pbasis(&X[q * 3], a) * gphi[(q * nv + j) * 3 + m];
        ref[o.Div + (m * np + a) * nv + j] = s;
      }
  // faces f = 2*axis + side, outer normal (2 side - 1) e_axis
  int nqf = 1;
  for (int m = 0; m < d - 1; ++m) nqf *= kQ1;
  for (int f = 0; f < 2 * d; ++f) {
    const int ax = f / 2, side = f % 2;
    const double nrm = 2.0 * side - 1.0;
    double area = 1.0;
    for (int m = 0; m < d; ++m)
      if (m != ax) area *= L.h[m];
    double* S = &ref[o.face0 + f * o.face_stride + o.fS];
    double* G = &ref[o.face0 + f * o.face_stride + o.fG];
    double* Pf = &ref[o.face0 + f * o.face_stride + o.fPf];
    for (int qf = 0; qf < nqf; ++qf) {
      double x[3] = {0, 0, 0};
      double w = 1.0;
      int t = qf;
      for (int m = 0; m < d; ++m) {
        if (m == ax) {
          x[m] = side;
        } else {
          x[m] = gx[t % kQ1];
          w *= gw[t % kQ1];
          t /= kQ1;
        }
      }
      double pv[27], pg[27][3];
      for (int i = 0; i < nv; ++i) basis(x, i, &pv[i], pg[i]);
      for (int i = 0; i < nv; ++i)
        for (int j = 0; j < nv; ++j) {
          S[i * nv + j] += w * area * pv[i] * pv[j];
          G[i * nv + j] += w * area * nrm * pg[j][ax] * pv[i];
        }
      for (int a = 0; a < np; ++a)
        for (int i = 0; i < nv; ++i) Pf[a * nv + i] += w * area * pbasis(x, a) * pv[i];
    }
  }
  for (int q = 0; q < nq; ++q)
    for (int m = 0; m < d; ++m) ref[o.Xq + q * d + m] = X[q * 3 + m];
  {
    double area = 1.0;
    for (int m = 1; m < d; ++m) area *= L.h[m];
    for (int qf = 0; qf < o.nqf; ++qf) {
      double x[3] = {0.0, 0.0, 0.0};
      double w = 1.0;
      int t = qf;
      for (int m = 1; m < d; ++m) {
        x[m] = gx[t % kQ1];
        w *= gw[t % kQ1];
        t /= kQ1;
      }
      for (int m = 0; m < d; ++m) ref[o.XF + qf * d + m] = x[m];
      ref[o.WF + qf] = w * area;
      for (int i = 0; i < nv; ++i) {
        double v, g[3];
        basis(x, i, &v, g);
        ref[o.phiF + qf * nv + i] = v;
        ref[o.gnF + qf * nv + i] = -g[0];
      }
      for (int a = 0; a < np; ++a) ref[o.xiF + qf * np + a] = pbasis(x, a);
    }
  }
  L.ro = o;
  return upload(&L.ref, ref);
}

// ---------------------------------------------------------------------------------------------
// One level: numbering, maps, pattern
// ---------------------------------------------------------------------------------------------
static stm_status build_level(const stm_params& p, int g, Level& L, std::vector<int>* keep_nbr_ptr,
                              std::vector<int>* keep_nbr, std::vector<int>* keep_node_cells) {
  const int d = p.dim;
  L.dim = d;
  L.K = p.k + 1;
  const int f = 1 << g;
  for (int m = 0; m < 3; ++m) {
    L.cells[m] = (m < d) ? p.coarse_cells[m] * f : 1;
    L.h[m] = (m < d) ? p.length[m] / L.cells[m] : 1.0;
    L.lat[m] = (m < d) ? 2 * L.cells[m] + 1 : 1;
  }
  double hh = 0.0;
  for (int m = 0; m < d; ++m) hh += L.h[m] * L.h[m];
  L.hT = std::sqrt(hh);
  L.nv = (d == 2) ? 9 : 27;
  L.np = d + 1;
  L.nt = d * L.nv + L.np;
  L.n = L.K * L.nt;
  L.Cfull = (long long)L.cells[0] * L.cells[1] * L.cells[2];
  L.P_lat = (long long)L.lat[0] * L.lat[1] * L.lat[2];
  const int nx = L.cells[0], ny = L.cells[1];
  // active cells
  L.h_full_active.assign(L.Cfull, -1);
  L.h_cell_full.clear();
  L.h_cell_xyz.clear();
  for (long long c = 0; c < L.Cfull; ++c) {
    int xyz[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
    bool removed = true;
    for (int m = 0; m < d; ++m) {
      int lo = p.obstacle_lo[m] * f, hi = p.obstacle_hi[m] * f;
      removed = removed && xyz[m] >= lo && xyz[m] < hi;
    }
    if (!removed) {
      L.h_full_active[c] = (int)L.h_cell_full.size();
      L.h_cell_full.push_back((int)c);
      L.h_cell_xyz.insert(L.h_cell_xyz.end(), xyz, xyz + 3);
    }
  }
  L.C = (int)L.h_cell_full.size();
  const int C = L.C, nv = L.nv, np = L.np;
  // nodes
  std::vector<unsigned char> used(L.P_lat, 0);
  auto latidx = [&](int x, int y, int z) { return (long long)x + (long long)L.lat[0] * (y + (long long)L.lat[1] * z); };
  std::vector<long long> cl(C * (size_t)nv);
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < nv; ++i) {
      int o[3];
      local_offsets(d, i, o);
      const int* xyz = &L.h_cell_xyz[3 * c];
      long long li = latidx(2 * xyz[0] + o[0], 2 * xyz[1] + o[1], d == 3 ? 2 * xyz[2] + o[2] : 0);
      cl[(size_t)c * nv + i] = li;
      used[li] = 1;
    }
  L.h_lat_node.assign(L.P_lat, -1);
  L.h_node_lat.clear();
  for (long long li = 0; li < L.P_lat; ++li)
    if (used[li]) {
      L.h_lat_node[li] = (int)L.h_node_lat.size();
      L.h_node_lat.push_back((int)li);
    }
  L.R = (int)L.h_node_lat.size();
  const int R = L.R;
  L.S = np * C;
  L.block = (long long)d * R + L.S;
  L.N = L.K * L.block;
  L.h_cell_nodes.resize((size_t)C * nv);
  for (size_t e = 0; e < cl.size(); ++e) L.h_cell_nodes[e] = L.h_lat_node[cl[e]];
  // local -> global DoF map (Eq. locdofs)
  std::vector<int> idx((size_t)C * L.n);
  for (int c = 0; c < C; ++c)
    for (int a = 0; a < L.K; ++a) {
      for (int l = 0; l < d; ++l)
        for (int i = 0; i < nv; ++i)
          idx[(size_t)c * L.n + a * L.nt + l * nv + i] = (int)(a * L.block + (long long)l * R + L.h_cell_nodes[(size_t)c * nv + i]);
      for (int q = 0; q < np; ++q)
        idx[(size_t)c * L.n + a * L.nt + d * nv + q] = (int)(a * L.block + (long long)d * R + (long long)c * np + q);
    }
  // Dirichlet face mask
  std::vector<unsigned char> bmask(C, 0);
  for (int c = 0; c < C; ++c) {
    const int* xyz = &L.h_cell_xyz[3 * c];
    for (int m = 0; m < d; ++m)
      for (int s = 0; s < 2; ++s) {
        int nb[3] = {xyz[0], xyz[1], xyz[2]};
        nb[m] += s ? 1 : -1;
        bool outside = nb[m] < 0 || nb[m] >= L.cells[m];
        bool gd;
        if (outside) {
          gd = (m == 0) ? (s == 0) : true;  // inflow x=0 and walls; x=L is the outflow
        } else {
          long long nf = nb[0] + (long long)nx * (nb[1] + (long long)ny * nb[2]);
          gd = L.h_full_active[nf] < 0;  // face shared with a removed (obstacle) cell
        }
        if (gd) bmask[c] |= (unsigned char)(1u << (2 * m + s));
      }
  }
  // cells of each node (sorted by cell id) and neighbour lists
  std::vector<int> ncell(R, 0);
  for (size_t e = 0; e < L.h_cell_nodes.size(); ++e) ncell[L.h_cell_nodes[e]]++;
  const int maxc = 1 << d;
  std::vector<int> node_cells((size_t)R * maxc, -1);
  {
    std::vector<int> fill(R, 0);
    for (int c = 0; c < C; ++c)
      for (int i = 0; i < nv; ++i) {
        int nd = L.h_cell_nodes[(size_t)c * nv + i];
        node_cells[(size_t)nd * maxc + fill[nd]++] = c;
      }
  }
  std::vector<int> nbr_ptr(R + 1, 0), nbr;
  nbr.reserve((size_t)R * (d == 2 ? 25 : 125));
  {
    std::vector<int> tmp;
    for (int nd = 0; nd < R; ++nd) {
      tmp.clear();
      for (int t = 0; t < ncell[nd]; ++t) {
        int c = node_cells[(size_t)nd * maxc + t];
        for (int j = 0; j < nv; ++j) tmp.push_back(L.h_cell_nodes[(size_t)c * nv + j]);
      }
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      nbr.insert(nbr.end(), tmp.begin(), tmp.end());
      nbr_ptr[nd + 1] = (int)nbr.size();
    }
  }
  std::vector<int> nn(R);
  for (int nd = 0; nd < R; ++nd) nn[nd] = nbr_ptr[nd + 1] - nbr_ptr[nd];
  std::vector<unsigned char> rank((size_t)C * nv * nv), cellrank((size_t)C * nv);
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < nv; ++i) {
      int ni = L.h_cell_nodes[(size_t)c * nv + i];
      const int* b = &nbr[nbr_ptr[ni]];
      const int* e = &nbr[nbr_ptr[ni + 1] - 1] + 1;
      for (int j = 0; j < nv; ++j) {
        int nj = L.h_cell_nodes[(size_t)c * nv + j];
        rank[((size_t)c * nv + i) * nv + j] = (unsigned char)(std::lower_bound(b, e, nj) - b);
      }
      int r = 0;
      while (node_cells[(size_t)ni * maxc + r] != c) ++r;
      cellrank[(size_t)c * nv + i] = (unsigned char)r;
    }
  // CSR row pointers (row order = global DoF order)
  std::vector<long long> rowptr(L.N + 1, 0);
  {
    long long pos = 0, row = 0;
    for (int a = 0; a < L.K; ++a) {
      for (int l = 0; l < d; ++l)
        for (int nd = 0; nd < R; ++nd) {
          rowptr[row++] = pos;
          pos += (long long)L.K * d * nn[nd] + (long long)np * ncell[nd];
        }
      for (int c = 0; c < C; ++c)
        for (int q = 0; q < np; ++q) {
          rowptr[row++] = pos;
          pos += (long long)d * nv;
        }
    }
    rowptr[row] = pos;
    L.nnz = pos;
  }
  // multiplicities, owner lists (sorted by cell), colours
  std::vector<int> own_cnt(L.N, 0);
  for (size_t e = 0; e < idx.size(); ++e) own_cnt[idx[e]]++;
  std::vector<int> own_ptr(L.N + 1, 0);
  for (long long i = 0; i < L.N; ++i) own_ptr[i + 1] = own_ptr[i] + own_cnt[i];
  std::vector<int> own_pos(own_ptr[L.N]);
  {
    std::vector<int> fill(own_ptr.begin(), own_ptr.end() - 1);
    for (int c = 0; c < C; ++c)
      for (int al = 0; al < L.n; ++al) own_pos[fill[idx[(size_t)c * L.n + al]]++] = c * L.n + al;
  }
  std::vector<double> wmult(L.N);
  std::vector<int> last_owner(L.N);
  for (long long i = 0; i < L.N; ++i) {
    wmult[i] = 1.0 / own_cnt[i];
    last_owner[i] = own_pos[own_ptr[i + 1] - 1];
  }
  std::vector<int> colour_cells;
  colour_cells.reserve(C);
  for (int col = 0; col < (1 << d); ++col) {
    L.colour_off[col] = (int)colour_cells.size();
    for (int c = 0; c < C; ++c) {
      const int* xyz = &L.h_cell_xyz[3 * c];
      int cc = 0;
      for (int m = 0; m < d; ++m) cc |= (xyz[m] & 1) << m;
      if (cc == col) colour_cells.push_back(c);
    }
  }
  for (int col = (1 << d); col < 9; ++col) L.colour_off[col] = (int)colour_cells.size();

  std::vector<long long> nbase(R + 1, 0);
  for (int nd = 0; nd < R; ++nd)
    nbase[nd + 1] = nbase[nd] + (long long)(L.K * d) * ((long long)L.K * d * nn[nd] + (long long)np * ncell[nd]);
  STM_TRY(upload(&L.nbase, nbase));
  STM_CUDA(cudaMalloc((void**)&L.spmv_work, sizeof(unsigned) * 2));
  STM_CUDA(cudaMemset(L.spmv_work, 0, sizeof(unsigned) * 2));
  STM_CUDA(cudaMalloc((void**)&L.nval, sizeof(double) * nbase[R]));
  L.nval_len = nbase[R];
  {
    const long long prows = ((long long)L.K * C * np + 31) / 32 * 32;
    L.pval_len = prows * d * L.nv;
    STM_CUDA(cudaMalloc((void**)&L.pvalT, sizeof(double) * L.pval_len));
    STM_CUDA(cudaMemset(L.pvalT, 0, sizeof(double) * L.pval_len));
  }
  std::vector<int> job_nodes(R);
  std::iota(job_nodes.begin(), job_nodes.end(), 0);
  std::stable_sort(job_nodes.begin(), job_nodes.end(), [&](int a, int b) {
    return nn[a] != nn[b] ? nn[a] < nn[b] : ncell[a] < ncell[b];
  });
  STM_TRY(upload(&L.job_nodes, job_nodes));
  // per colour, the nodes touched by its cells, in job order: the coloured smoother's defect needs
  // only their velocity rows (and the pressure rows) before the local solves of that colour
  {
    std::vector<int> colour_jobs;
    std::vector<char> touched(R);
    for (int col = 0; col < (1 << d); ++col) {
      std::fill(touched.begin(), touched.end(), 0);
      for (int k = L.colour_off[col]; k < L.colour_off[col + 1]; ++k)
        for (int i = 0; i < nv; ++i) touched[L.h_cell_nodes[(size_t)colour_cells[k] * nv + i]] = 1;
      L.colour_job_off[col] = (int)colour_jobs.size();
      for (int nd : job_nodes)
        if (touched[nd]) colour_jobs.push_back(nd);
    }
    for (int col = (1 << d); col < 9; ++col) L.colour_job_off[col] = (int)colour_jobs.size();
    if (colour_jobs.empty()) colour_jobs.push_back(0);
    STM_TRY(upload(&L.colour_jobs, colour_jobs));
  }
  STM_TRY(upload(&L.idx, idx));
  STM_TRY(upload(&L.cell_nodes, L.h_cell_nodes));
  STM_TRY(upload(&L.cell_xyz, L.h_cell_xyz));
  STM_TRY(upload(&L.bmask, bmask));
  STM_TRY(upload(&L.rank, rank));
  STM_TRY(upload(&L.cellrank, cellrank));
  STM_TRY(upload(&L.nn, nn));
  STM_TRY(upload(&L.ncell, ncell));
  STM_TRY(upload(&L.rowptr, rowptr));
  STM_TRY(upload(&L.own_ptr, own_ptr));
  STM_TRY(upload(&L.own_pos, own_pos));
  STM_TRY(upload(&L.last_owner, last_owner));
  STM_TRY(upload(&L.wmult, wmult));
  STM_TRY(upload(&L.colour_cells, colour_cells));
  STM_CUDA(cudaMalloc((void**)&L.colidx, sizeof(int) * L.nnz));
  STM_CUDA(cudaMalloc((void**)&L.val, sizeof(double) * L.nnz));
  STM_CUDA(cudaMemset(L.val, 0, sizeof(double) * L.nnz));
  STM_CUDA(cudaMalloc((void**)&L.d, sizeof(double) * L.N));
  STM_CUDA(cudaMalloc((void**)&L.r, sizeof(double) * L.N));
  STM_CUDA(cudaMalloc((void**)&L.t, sizeof(double) * L.N));
  STM_CUDA(cudaMalloc((void**)&L.wnod, sizeof(double) * L.K * d * (size_t)R));
  STM_CUDA(cudaMalloc((void**)&L.Y, sizeof(double) * (size_t)C * L.n));
  *keep_nbr_ptr = std::move(nbr_ptr);
  *keep_nbr = std::move(nbr);
  *keep_node_cells = std::move(node_cells);
  return build_reference(L);
}

// Transfer P: level g-1 (coarse) -> level g (fine); interpolation of the coarse Q2/P1disc function.
static stm_status build_transfer(const Level& Cl, Level& F) {
  const int d = F.dim, nv = F.nv, np = F.np;
  // velocity: per fine node a list of (coarse node, weight)
  std::vector<int> vptr(F.R + 1, 0);
  std::vector<int> vcol;
  std::vector<double> vval;
  for (int nd = 0; nd < F.R; ++nd) {
    long long li = F.h_node_lat[nd];
    int fx[3] = {(int)(li % F.lat[0]), (int)((li / F.lat[0]) % F.lat[1]), (int)(li / ((long long)F.lat[0] * F.lat[1]))};
    // candidate coarse cells per axis with the reference coordinate in that cell
    int cand[3][2], ncand[3];
    double xi[3][2];
    for (int m = 0; m < 3; ++m) {
      ncand[m] = 0;
      if (m >= d) {
        cand[m][0] = 0;
        xi[m][0] = 0.0;
        ncand[m] = 1;
        continue;
      }
      int xf = fx[m];
      if (xf % 4 == 0) {
        int c1 = xf / 4 - 1, c2 = xf / 4;
        if (c1 >= 0) { cand[m][ncand[m]] = c1; xi[m][ncand[m]++] = 1.0; }
        if (c2 < Cl.cells[m]) { cand[m][ncand[m]] = c2; xi[m][ncand[m]++] = 0.0; }
      } else {
        int c = xf / 4;
        cand[m][0] = c;
        xi[m][0] = (xf - 4.0 * c) / 4.0;
        ncand[m] = 1;
      }
    }
    int best = -1;
    double bxi[3] = {0, 0, 0};
    for (int a0 = 0; a0 < ncand[0]; ++a0)
      for (int a1 = 0; a1 < ncand[1]; ++a1)
        for (int a2 = 0; a2 < ncand[2]; ++a2) {
          long long cf = cand[0][a0] + (long long)Cl.cells[0] * (cand[1][a1] + (long long)Cl.cells[1] * cand[2][a2]);
          int ca = Cl.h_full_active[cf];
          if (ca >= 0 && (best < 0 || ca < best)) {
            best = ca;
            bxi[0] = xi[0][a0];
            bxi[1] = xi[1][a1];
            bxi[2] = xi[2][a2];
          }
        }
    if (best < 0) {
      set_error("transfer: fine node outside every active coarse cell");
      return STM_ERR_INVALID_ARG;
    }
    for (int s = 0; s < nv; ++s) {
      int o[3];
      local_offsets(d, s, o);
      double w = 1.0;
      for (int m = 0; m < d; ++m) w *= q2v(o[m], bxi[m]);
      if (w != 0.0) {
        vcol.push_back(Cl.h_cell_nodes[(size_t)best * nv + s]);
        vval.push_back(w);
      }
    }
    vptr[nd + 1] = (int)vcol.size();
  }
  // assemble P over all (time, component) blocks and the pressure
  std::vector<long long> prow(F.N + 1, 0);
  std::vector<int> pcol;
  std::vector<double> pval;
  const double s3 = std::sqrt(3.0);
  long long row = 0;
  for (int a = 0; a < F.K; ++a) {
    for (int l = 0; l < d; ++l)
      for (int nd = 0; nd < F.R; ++nd) {
        for (int e = vptr[nd]; e < vptr[nd + 1]; ++e) {
          pcol.push_back((int)(a * Cl.block + (long long)l * Cl.R + vcol[e]));
          pval.push_back(vval[e]);
        }
        prow[++row] = (long long)pcol.size();
      }
    for (int c = 0; c < F.C; ++c) {
      const int* xyz = &F.h_cell_xyz[3 * c];
      int px[3] = {xyz[0] / 2, xyz[1] / 2, xyz[2] / 2};
      long long pf = px[0] + (long long)Cl.cells[0] * (px[1] + (long long)Cl.cells[1] * px[2]);
      int pc = Cl.h_full_active[pf];
      long long base = a * Cl.block + (long long)d * Cl.R + (long long)pc * np;
      // child map of the Legendre P1 coefficients: c0' = c0 + sum_m sqrt3 (o_m - 1/2) c_m, c_m' = c_m / 2
      pcol.push_back((int)base);
      pval.push_back(1.0);
      for (int m = 0; m < d; ++m) {
        pcol.push_back((int)(base + 1 + m));
        pval.push_back(s3 * ((xyz[m] - 2 * px[m]) - 0.5));
      }
      prow[++row] = (long long)pcol.size();
      for (int m = 0; m < d; ++m) {
        pcol.push_back((int)(base + 1 + m));
        pval.push_back(0.5);
        prow[++row] = (long long)pcol.size();
      }
    }
  }
  // transpose (restriction R = P^T)
  const long long Nc = Cl.N;
  std::vector<long long> trow(Nc + 1, 0);
  for (size_t e = 0; e < pcol.size(); ++e) trow[pcol[e] + 1]++;
  for (long long i = 0; i < Nc; ++i) trow[i + 1] += trow[i];
  std::vector<int> tcol(pcol.size());
  std::vector<double> tval(pcol.size());
  {
    std::vector<long long> fill(trow.begin(), trow.end() - 1);
    for (long long r = 0; r < F.N; ++r)
      for (long long e = prow[r]; e < prow[r + 1]; ++e) {
        long long dst = fill[pcol[e]]++;
        tcol[dst] = (int)r;
        tval[dst] = pval[e];
      }
  }
  // node lists and cell maps of the matrix-free transfers
  {
    std::vector<int> cptr(Cl.R + 1, 0);
    for (int e : vcol) cptr[e + 1]++;
    for (int i = 0; i < Cl.R; ++i) cptr[i + 1] += cptr[i];
    std::vector<int> cnode(vcol.size());
    std::vector<double> cw(vcol.size());
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int nd = 0; nd < F.R; ++nd)
      for (int e = vptr[nd]; e < vptr[nd + 1]; ++e) {
        const int dst = fill[vcol[e]]++;
        cnode[dst] = nd;
        cw[dst] = vval[e];
      }
    const int nch = 1 << d;
    std::vector<int> parent(F.C), children((size_t)Cl.C * nch, -1);
    std::vector<unsigned char> bits(F.C);
    for (int c = 0; c < F.C; ++c) {
      const int* xyz = &F.h_cell_xyz[3 * c];
      long long pf = xyz[0] / 2 + (long long)Cl.cells[0] * (xyz[1] / 2 + (long long)Cl.cells[1] * (xyz[2] / 2));
      int b = 0;
      for (int m = 0; m < d; ++m) b |= (xyz[m] & 1) << m;
      parent[c] = Cl.h_full_active[pf];
      bits[c] = (unsigned char)b;
      if (parent[c] < 0) {
        set_error("transfer: fine cell without an active parent");
        return STM_ERR_INVALID_ARG;
      }
      children[(size_t)parent[c] * nch + b] = c;
    }
    for (int v : children)
      if (v < 0) {
        set_error("transfer: active coarse cell with a removed child");
        return STM_ERR_INVALID_ARG;
      }
    STM_TRY(upload(&F.tv_ptr, vptr));
    STM_TRY(upload(&F.tv_node, vcol));
    STM_TRY(upload(&F.tv_w, vval));
    STM_TRY(upload(&F.tc_ptr, cptr));
    STM_TRY(upload(&F.tc_node, cnode));
    STM_TRY(upload(&F.tc_w, cw));
    STM_TRY(upload(&F.cparent, parent));
    STM_TRY(upload(&F.cbits, bits));
    STM_TRY(upload(&F.cchildren, children));
  }
  F.P_nnz = (long long)pcol.size();
  STM_TRY(upload(&F.P_rowptr, prow));
  STM_TRY(upload(&F.P_col, pcol));
  STM_TRY(upload(&F.P_val, pval));
  STM_TRY(upload(&F.Rt_rowptr, trow));
  STM_TRY(upload(&F.Rt_col, tcol));
  STM_TRY(upload(&F.Rt_val, tval));
  return STM_OK;
}

stm_status build_levels(Hierarchy& H) {
  const stm_params& p = H.p;
  const int G = p.n_levels;
  H.L.assign(G, Level());
  time_matrices(p.k, p.tau, H.Mt, H.D, H.T);
  for (int g = 0; g < G; ++g) {
    std::vector<int> nbr_ptr, nbr, node_cells;
    STM_TRY(build_level(p, g, H.L[g], &nbr_ptr, &nbr, &node_cells));
    Level& L = H.L[g];
    STM_TRY(upload(&L.nbr_ptr, nbr_ptr));
    STM_TRY(upload(&L.nbr, nbr));
    STM_TRY(upload(&L.node_cells, node_cells));
    stm_status st = launch_fill_colidx(L, L.nbr_ptr, L.nbr, L.node_cells, 0);
    STM_CUDA(cudaDeviceSynchronize());
    if (st != STM_OK) return st;
    if (g > 0) STM_TRY(build_transfer(H.L[g - 1], H.L[g]));
  }
  // injection maps: node of level g -> finest node at the same position
  const Level& Fl = H.L[G - 1];
  for (int g = 0; g < G; ++g) {
    Level& L = H.L[g];
    const int f = 1 << (G - 1 - g);
    std::vector<int> inj(L.R);
    for (int nd = 0; nd < L.R; ++nd) {
      long long li = L.h_node_lat[nd];
      long long x = li % L.lat[0], y = (li / L.lat[0]) % L.lat[1], z = li / ((long long)L.lat[0] * L.lat[1]);
      long long lf = x * f + (long long)Fl.lat[0] * (y * f + (long long)Fl.lat[1] * z * f);
      inj[nd] = Fl.h_lat_node[lf];
      if (inj[nd] < 0) {
        set_error("injection: coarse node missing on the finest level");
        return STM_ERR_INVALID_ARG;
      }
    }
    STM_TRY(upload(&L.inj, inj));
  }
  STM_CUDA(cudaMalloc((void**)&H.dflag, sizeof(int) * 4));
  STM_CUDA(cudaMemset(H.dflag, 0, sizeof(int) * 4));
  STM_CUDA(cudaMalloc((void**)&H.dkerr, sizeof(int)));
  STM_CUDA(cudaMemset(H.dkerr, 0, sizeof(int)));
  STM_CUDA(cudaMalloc((void**)&H.dbad, sizeof(long long) * 2));
  return STM_OK;
}

void free_hierarchy(Hierarchy& H) {
  clear_graphs(H);
  if (H.cap_stream) cudaStreamDestroy(H.cap_stream);
  H.cap_stream = nullptr;
  for (Level& L : H.L) {
    void* ptrs[] = {L.idx, L.cell_nodes, L.cell_xyz, L.bmask, L.rank, L.cellrank, L.nn, L.ncell, L.rowptr, L.nbr_ptr, L.nbr,
                    L.node_cells, L.job_nodes, L.nbase, L.spmv_work, L.nval, L.pvalT, L.nvalJT, L.pvalJT, L.nval32, L.pval32,
                    L.nvalJT32, L.pvalJT32, L.x32,
                    L.colidx, L.val, L.valT, L.ref, L.inj, L.wnod, L.inv, L.wmult, L.own_ptr,
                    L.own_pos, L.last_owner, L.colour_cells, L.colour_jobs, L.Y, L.P_rowptr, L.P_col, L.P_val,
                    L.Rt_rowptr, L.Rt_col, L.Rt_val, L.tv_ptr, L.tv_node, L.tv_w, L.tc_ptr, L.tc_node,
                    L.tc_w, L.cparent, L.cbits, L.cchildren, L.d, L.r, L.t, L.md, L.mr, L.mt, L.mY, L.mt16};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
  void* hp[] = {H.cinv, H.cinvT, H.dflag, H.dkerr, H.dbad, H.V, H.Z, H.w, H.hcol, H.part, H.yvec, H.bbuf, H.xbuf,
                H.nw_negF, H.nw_D, H.nw_Xt, H.nw_B, H.nw_Ft, H.ag_buf, H.ag_wnod,
                H.cs_off, H.cs_pos, H.cs_rowslab, H.cs_perm, H.cs_store, H.cs_u, H.cs_v, H.cs_mu, H.cs_mv,
                H.mV, H.mZ, H.mW, H.mB, H.mX, H.mh, H.mpart, H.mf, H.my};
  for (void* q : hp)
    if (q) cudaFree(q);
  for (ProfRec& r : H.prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : H.prof.pool) cudaEventDestroy(e);
  H.prof.recs.clear();
  H.prof.pool.clear();
  H.L.clear();
}

}  // namespace stm
