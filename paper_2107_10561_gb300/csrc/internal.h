// Internal data structures of libstm (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <map>
#include <tuple>
#include <cstdint>
#include <string>
#include <vector>

#include "stm.h"

namespace stm {
constexpr int STM_KCLASS_COUNT = 8;

constexpr int kMaxDim = 3;
constexpr int kQ1 = 4;  // Gauss points per direction (exact for every integrand of the forms)

// Thread-local error message and helpers -----------------------------------------------------
void set_error(const std::string& msg);
stm_status cuda_fail(cudaError_t e, const char* what);
#define STM_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::stm::cuda_fail(e_, #call);  \
  } while (0)

#ifndef STM_TRY
#define STM_TRY(x)               \
  do {                           \
    stm_status s_ = (x);         \
    if (s_ != STM_OK) return s_; \
  } while (0)
#endif

// Streaming multiprocessors of the current device (queried once per process)
int sm_count();

// BF16 bits of the value nearest to x (ties to even), rounded once from the FP64 bit fields: 8
// significant bits, exponent range of FP32. Zero, values below the BF16 normal range, overflow and
// non-finite values take the FP32 route (exact for zero, infinities and NaN).
__device__ __forceinline__ uint32_t bf16_bits_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 48) & 0x8000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126 || e > 127) {
    const uint32_t f = __float_as_uint((float)x);
    if ((f & 0x7F800000u) == 0x7F800000u) return (f >> 16) | ((f & 0xFFFFu) ? 0x40u : 0u);
    const uint32_t lsb = (f >> 16) & 1u;
    return (f + 0x7FFFu + lsb) >> 16;
  }
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;  // 52 stored bits, 7 are kept
  uint32_t r = sign | ((uint32_t)(e + 127) << 7) | (uint32_t)(mant >> 45);
  const unsigned long long rest = mant & ((1ull << 45) - 1);
  const unsigned long long half = 1ull << 44;
  if (rest > half || (rest == half && (r & 1u))) ++r;  // a carry moves into the exponent as it should
  return r;
}
__device__ __forceinline__ double bf16_bits_to_double(uint32_t h) { return (double)__uint_as_float(h << 16); }

// x = hi + lo + (rounding of lo) with hi = the BF16 value nearest to x and lo = the BF16 value nearest to
// x - hi (which FP64 holds exactly), both taken from the FP64 bit fields with integer operations only:
// no FP64 pipe instructions in the common case. Out-of-range exponents (x or lo outside the BF16
// normal range, zero, non-finite) take the bf16_bits_rn route above.
__device__ __forceinline__ void bf16_split_rn(double x, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 48) & 0x8000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -74 || e > 127) {
    hi = bf16_bits_rn(x);
    lo = bf16_bits_rn(x - bf16_bits_to_double(hi));
    return;
  }
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  uint32_t h = sign | ((uint32_t)(e + 127) << 7) | (uint32_t)(mant >> 45);
  long long rem = (long long)(mant & ((1ull << 45) - 1));  // x - (truncated hi) in units of 2^(e - 52)
  const long long half = 1ll << 44;
  if (rem > half || (rem == half && (h & 1u))) {
    ++h;                    // rounded up (a carry moves into the exponent as it should)
    rem -= (1ll << 45);     // the remainder is now negative
  }
  hi = h;
  if (rem == 0) {
    lo = 0u;
    return;
  }
  const uint32_t ls = rem < 0 ? (sign ^ 0x8000u) : sign;
  const unsigned long long a = (unsigned long long)(rem < 0 ? -rem : rem);  // < 2^45
  const int p = 63 - __clzll((long long)a);                                  // leading bit, 0..44
  const int le = p + e - 52;                                                 // exponent of |x - hi|
  if (le < -126) {
    lo = bf16_bits_rn(x - bf16_bits_to_double(hi));
    return;
  }
  if (p <= 7) {
    lo = ls | ((uint32_t)(le + 127) << 7) | ((uint32_t)(a << (7 - p)) & 0x7Fu);
    return;
  }
  const int sh = p - 7;
  uint32_t l = ls | ((uint32_t)(le + 127) << 7) | ((uint32_t)(a >> sh) & 0x7Fu);
  const unsigned long long rest = a & ((1ull << sh) - 1), hl = 1ull << (sh - 1);
  if (rest > hl || (rest == hl && (l & 1u))) ++l;
  lo = l;
}

// Launch accounting and optional per-class CUDA-event timing --------------------------------
extern std::atomic<long long> g_launches;
inline void note_launch(long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

constexpr int kProfLevels = 17;  // slot 0: all levels, slot 1 + g: level g
struct ProfRec {
  cudaEvent_t a, b;
  int cls, level;
  double bytes;
};
struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  double total_ms[STM_KCLASS_COUNT][kProfLevels] = {};
  long long count[STM_KCLASS_COUNT][kProfLevels] = {};
  double bytes[STM_KCLASS_COUNT][kProfLevels] = {};
};

// Reference tables of a uniform level (all cells congruent): computed on the host --------------
// Layout of the packed device buffer `ref` (doubles):
//   W[nq]                       quadrature weight x |T|
//   phi[nq][nv]                 Q2 basis values
//   gphi[nq][nv][d]             physical gradients
//   M[nv][nv], Kst[nv][nv]      mass, stiffness
//   Div[d][np][nv]              (d_m phi_j, xi_q)
//   per face f in 0..2d-1:  S[nv][nv], G[nv][nv] (<grad phi_j . n, phi_i>), Pf[np][nv]
//   Xq[nq][d]                   reference coordinates of the volume points
//   inflow face x = 0 (face 0): nqf points XF[nqf][d], WF[nqf] (weight x |F|), phiF[nqf][nv],
//   gnF[nqf][nv] (grad phi . n with n = -e_x), xiF[nqf][np]
struct RefOffsets {
  int nq, nv, np;
  int W, phi, gphi, M, Kst, Div, face0, face_stride, fS, fG, fPf;
  int Xq, nqf, XF, WF, phiF, gnF, xiF;
  int total;
};

struct Level {
  // geometry and sizes
  int dim = 2, K = 2;         // K = k + 1 time nodes
  int cells[3] = {1, 1, 1};   // cells per axis (cells[2] = 1 in 2D)
  double h[3] = {1, 1, 1};
  double hT = 1;              // cell diameter (Nitsche h)
  int lat[3] = {1, 1, 1};     // lattice points per axis
  int C = 0, R = 0, S = 0, nv = 9, np = 3, nt = 0, n = 0;
  long long block = 0, N = 0, nnz = 0, P_lat = 0, Cfull = 0;

  // host copies needed for later set-up steps
  std::vector<int> h_cell_full;   // active cell -> full cell index
  std::vector<int> h_cell_xyz;    // [C][3]
  std::vector<int> h_node_lat;    // node -> lattice index
  std::vector<int> h_lat_node;    // lattice index -> node (-1: unused)
  std::vector<int> h_cell_nodes;  // [C][nv]
  std::vector<int> h_full_active; // full cell -> active index (-1: removed)

  // device data -----------------------------------------------------------------------------
  int* idx = nullptr;             // [C][n] global DoF of each local DoF
  int* cell_nodes = nullptr;      // [C][nv]
  int* cell_xyz = nullptr;        // [C][3] integer cell coordinates
  unsigned char* bmask = nullptr; // [C] bit f set: face f on Gamma_D
  unsigned char* rank = nullptr;  // [C][nv][nv] rank of node j in the neighbour list of node i
  unsigned char* cellrank = nullptr; // [C][nv] rank of the cell among the cells of node i
  int* nn = nullptr;              // [R] number of neighbour nodes
  int* nbr_ptr = nullptr;         // [R+1] neighbour lists (sorted node ids)
  int* nbr = nullptr;
  int* node_cells = nullptr;      // [R][2^d] cells containing each node, sorted, -1 padded
  int* job_nodes = nullptr;       // [R] node ids ordered by (neighbour count, cell count, id)
  // node-block copy of the velocity-row values of J (forward SpMV): for node i, positions
  // p = (b*d + m)*nn + j (velocity) then K*d*nn + ci*n_p + q (pressure of the node's cells), each
  // position holding the K*d row values (a*d + l) contiguously; block of node i starts at nbase[i]
  long long* nbase = nullptr;     // [R+1]
  double* nval = nullptr;
  // pressure rows pr = (a*C + c)*n_p + q of J, warp-transposed for the forward SpMV: entry
  // t = m*nv + j of row pr at pvalT[((pr/32)*d*nv + t)*32 + pr%32] (rows padded to a multiple of 32)
  double* pvalT = nullptr;
  double *nvalJT = nullptr, *pvalJT = nullptr;  // the same two copies for J^T (built with valT)
  unsigned* spmv_work = nullptr;  // [2] unit counter and finished-CTA count of the FP64 product (zeroed)
  // FP32 copies of nval/pvalT (and of nvalJT/pvalJT) in the same layout, for the V-cycle's defects
  // r - J_g d with defect_precision = STM_F32; null otherwise
  float *nval32 = nullptr, *pval32 = nullptr, *nvalJT32 = nullptr, *pvalJT32 = nullptr;
  float* x32 = nullptr;  // [N] the defect's d rounded to FP32
  long long nval_len = 0, pval_len = 0;          // entries of nval and pvalT
  int* ncell = nullptr;           // [R] number of cells containing the node
  long long* rowptr = nullptr;    // [N+1]
  int* colidx = nullptr;          // [nnz]
  double* val = nullptr;          // [nnz]
  double* valT = nullptr;         // [nnz] values of J^T on the same (symmetric) pattern, lazy
  long long* tpos = nullptr;      // not kept (transpose built on demand)
  double* ref = nullptr;          // packed reference tables
  RefOffsets ro{};
  int* inj = nullptr;             // [R] node -> finest-level node holding its linearisation value
  double* wnod = nullptr;         // [K][d][R] linearisation velocity at this level's nodes

  // smoother data (levels >= 1)
  void* inv = nullptr;            // [C][n*n] column-major per cell, storage precision
  double* wmult = nullptr;        // [N] 1/m_i
  int* own_ptr = nullptr;         // [N+1]
  int* own_pos = nullptr;         // [sum m_i] flat positions c*n + alpha
  int* last_owner = nullptr;      // [N] flat position of the highest-index owning cell
  int* colour_cells = nullptr;    // cells sorted by colour
  int colour_off[9] = {0};
  int* colour_jobs = nullptr;     // per colour, the nodes its cells touch, in job_nodes order
  int colour_job_off[9] = {0};
  double* Y = nullptr;            // [C][n] per-cell local corrections (scratch)

  // transfer from level g-1 (coarse) to this level: P [N x N_c], P^T [N_c x N]
  long long* P_rowptr = nullptr; int* P_col = nullptr; double* P_val = nullptr;
  long long P_nnz = 0;
  long long* Rt_rowptr = nullptr; int* Rt_col = nullptr; double* Rt_val = nullptr;
  // the same P without assembled blocks (single-right-hand-side V-cycle): the Q2 weights of a fine
  // node are shared by every time node and velocity component, so one list per node serves all
  // K*d blocks; the P1disc child map follows from the child's position bits in its parent
  int* tv_ptr = nullptr; int* tv_node = nullptr; double* tv_w = nullptr;  // [R+1] fine node -> coarse
  int* tc_ptr = nullptr; int* tc_node = nullptr; double* tc_w = nullptr;  // [R_c+1] coarse node -> fine
  int* cparent = nullptr;         // [C] coarse cell containing each fine cell
  unsigned char* cbits = nullptr; // [C] child position bits (bit m: upper half along axis m)
  int* cchildren = nullptr;       // [C_c][2^d] fine cells of each coarse cell, by position bits

  // work vectors of the V-cycle
  double *d = nullptr, *r = nullptr, *t = nullptr;
  // multi-right-hand-side work space ([N][32] interleaved; mY: [C*n][32]), allocated on first use
  double *md = nullptr, *mr = nullptr, *mt = nullptr, *mY = nullptr;
  uint32_t* mt16 = nullptr;       // [N][32] the smoothing step's residual block as packed BF16 (lo << 16 | hi)
};

struct Hierarchy {
  stm_params p{};
  std::vector<Level> L;
  double Mt[3][3] = {}, D[3][3] = {}, T[3][3][3] = {};
  bool assembled = false, factored = false;
  // coarse direct solver: explicit FP64 inverse of J_0, row-major [N0][N0]
  double* cinv = nullptr;
  long long N0 = 0;
  double* cinvT = nullptr;  // [N0][N0] its transpose, row-major (the adjoint coarse solve reads rows too)
  // coarse solve through the twisted block factors in x-slab order (large coarse levels; cinv is then
  // not formed): cs_nx slabs eliminated from both ends towards slab cs_t, row offsets cs_off [nx + 1],
  // block offsets cs_pos [8][nx] into cs_store (inverse, lower and upper chain blocks, back-substitution
  // block, for J_0 and for J_0^T), slab of every permuted row, permuted position of every row; work
  // vectors for one column and for 32 interleaved columns
  bool coarse_slab = false;
  int cs_nx = 0, cs_t = 0;
  long long *cs_off = nullptr, *cs_pos = nullptr;
  int *cs_rowslab = nullptr, *cs_perm = nullptr;
  double *cs_store = nullptr, *cs_u = nullptr, *cs_v = nullptr, *cs_mu = nullptr, *cs_mv = nullptr;
  int* dflag = nullptr;           // device flags: [0] singular flag, [1..2] bad cell (int64 split)
  int* dkerr = nullptr;           // device error word of the tensor-core pipelines (bounded waits)
  long long* dbad = nullptr;
  // FGMRES work space (finest level)
  int restart_cap = 0;
  double* V = nullptr;            // [(m+1)][N]
  double* Z = nullptr;            // [m][N]
  double* w = nullptr;            // [N]
  double* hcol = nullptr;         // [m+2] device Hessenberg column / scratch
  double* part = nullptr;         // partial sums of batched dots
  double* yvec = nullptr;         // [m]
  double* bbuf = nullptr;         // host-API staging for b and x
  double* xbuf = nullptr;
  // damped Newton (allocated on first use): -F, step D, trial iterate, b + c(X, X), trial's -F
  double *nw_negF = nullptr, *nw_D = nullptr, *nw_Xt = nullptr, *nw_B = nullptr, *nw_Ft = nullptr;
  // adjoint gradient and explicit-point load vector (allocated on first use): db/dU, db/dnu,
  // (dJ/dnu) X, lambda; nodal linearisation velocity of an explicit point
  double *ag_buf = nullptr, *ag_wnod = nullptr;
  // residual histories of the last single- and multi-right-hand-side solves (host)
  std::vector<double> hist;
  std::vector<double> mhist[32];
  int nblk_dot = 0;
  // multi-right-hand-side FGMRES work space ([.][N][32])
  int mrestart_cap = 0;
  double *mV = nullptr, *mZ = nullptr, *mW = nullptr, *mB = nullptr, *mX = nullptr, *mh = nullptr, *mpart = nullptr,
         *mf = nullptr, *my = nullptr;
  Profiler prof;
  // CUDA graphs of the V-cycle, one per (r, d, transpose) pointer triple; launched on the caller's
  // stream, captured on a private stream (the legacy default stream cannot be captured)
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  std::map<std::tuple<const double*, double*, int>, std::pair<cudaGraphExec_t, long long>> vgraphs;
};

// Records CUDA events around the launches made in its lifetime when profiling is on.
struct ProfScope {
  Hierarchy* H;
  int cls, level;
  cudaStream_t s;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(Hierarchy* H_, int cls_, cudaStream_t s_, double bytes_, int level_ = -1);
  ~ProfScope();
};

// Storage of the cell inverses: column-major per cell with leading dimension ld >= n, ld a
// multiple of the vector width used by the smoother (rows n..ld-1 are zero padding).
struct InvLayout {
  int ld;   // padded rows per column
  int vb;   // bytes per vector load (16, 8 or 4)
};
InvLayout inv_layout(int n, int prec);

// Host set-up (hierarchy.cpp)
stm_status build_levels(Hierarchy& H);
void free_hierarchy(Hierarchy& H);
void time_matrices(int k, double tau, double Mt[3][3], double D[3][3], double T[3][3][3]);

// Kernel launchers (kernels_*.cu) -----------------------------------------------------------
stm_status launch_fill_colidx(Level& Lv, const int* nbr_ptr, const int* nbr_idx,
                              const int* node_cells, cudaStream_t s);
stm_status inject_linearisation(Hierarchy& H, const double* X_fine, cudaStream_t s);
stm_status assemble_level(Hierarchy& H, int g, double nu, cudaStream_t s);
stm_status factor_level(Hierarchy& H, int g, cudaStream_t s);
stm_status factor_coarse(Hierarchy& H, cudaStream_t s);
stm_status ensure_transpose(Hierarchy& H, int g, cudaStream_t s);

// y = alpha*A x + beta_y*y (+ b): mode 0: y = A x; 1: y = b - A x; 2: y += A x
stm_status csr_apply(const long long* rowptr, const int* col, const double* val, long long nrows, long long nnz,
                     const double* x, const double* b, double* y, int mode, cudaStream_t s);
// Matrix-free transfers between level g-1 and level g (kernels_transfer.cu)
stm_status transfer_restrict(const Level& F, const Level& Cl, const double* fine, double* coarse, cudaStream_t s);
// fine += P coarse; with fine32 non-null the updated entries are also stored rounded to FP32 there
stm_status transfer_prolong_add(const Level& F, const Level& Cl, const double* coarse, double* fine, cudaStream_t s,
                                float* fine32 = nullptr);
stm_status spmv_nodeblock(const Level& L, const double* nval, const double* pvalT, const double* x, const double* b,
                          double* y, int mode, cudaStream_t s,
                          const int* jobs = nullptr, int njobs = -1);
stm_status build_nodeblock(Level& L, cudaStream_t s);
// node-block and warp-transposed pressure-row copies of any value array on J's pattern (J or J^T)
stm_status build_nodeblock_from(const Level& L, const double* val, double* nval, double* pvalT, cudaStream_t s);
// y = b - J_g x (transpose: J_g^T) over the FP32 copies of the values: x rounded to FP32 into L.x32
// (skipped when x32_current: the kernel that last wrote x stored it there rounded), FP32 products
// and sums, b and y in FP64
stm_status defect_f32(Hierarchy& H, int g, int transpose, const double* x, const double* b, double* y,
                      cudaStream_t s, bool x32_current = false);
// FP32 copies of J_g's (or J_g^T's) node-block arrays (allocated on first use, same layout)
stm_status build_values_f32(Level& L, int transpose, cudaStream_t s);
stm_status jacobian_apply(Hierarchy& H, int g, const double* x, const double* b, double* y,
                          int mode, int transpose, cudaStream_t s);
// y = b - J_g x (or J_g^T) in FP64 on the velocity rows of the nodes that the cells of one colour
// touch and on every pressure row; the other rows of y are left as they are
stm_status jacobian_defect_colour(Hierarchy& H, int g, int colour, const double* x, const double* b, double* y,
                                  int transpose, cudaStream_t s);
// the V-cycle's defect y = b - J_g x (or J_g^T): over the FP32 copies with defect_precision =
// STM_F32, else jacobian_apply in FP64
stm_status smoother_defect(Hierarchy& H, int g, const double* x, const double* b, double* y, int transpose,
                           cudaStream_t s, bool x32_current = false);
// one smoothing step; d32_current: L.x32 holds d rounded to FP32 (the V-cycle's own sequence). With
// FP32 defects the additive/overwrite combine stores the new d rounded to FP32 in L.x32 as well.
stm_status vanka_step(Hierarchy& H, int g, const double* r, double* d, int transpose,
                      bool d_is_zero, cudaStream_t s, bool d32_current = false);
stm_status coarse_apply(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s);
// the coarse solve through the slab block-LU factors (kernels_coarse.cu): one column, or 32 interleaved
stm_status coarse_slab_apply(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s);
stm_status coarse_slab_apply_multi(Hierarchy& H, const double* R, double* D, cudaStream_t s);
// wnod: nodal linearisation velocity [K][d][R] of the finest level to use instead of the stored one
stm_status assemble_cellvec(Hierarchy& H, int mode, double U, double nu, const int* wake_lo, const int* wake_hi,
                            double* out, cudaStream_t s, const double* vprev = nullptr, const double* wnod = nullptr);
// wnod = the velocity of the finest-level DoF vector X at the nodes of level g ([K][d][R_g])
stm_status inject_level(const Hierarchy& H, int g, const double* X, double* wnod, cudaStream_t s);
stm_status dnu_apply(Hierarchy& H, const double* x, double* y, cudaStream_t s);
// multi-right-hand-side path (kernels_multi.cu), multi-vectors interleaved [N][32]
stm_status multi_to_interleaved(const double* src, double* dst, long long N, int nrhs, cudaStream_t s);
stm_status multi_from_interleaved(const double* src, double* dst, long long N, int nrhs, cudaStream_t s);
// columns [col0, col0 + ncols) of an interleaved [N][32] block from / to a column-major [ncols][N] array
stm_status multi_columns_in(const double* src, double* dst, long long N, int ncols, int col0, cudaStream_t s);
stm_status multi_columns_out(const double* src, double* dst, long long N, int ncols, int col0, cudaStream_t s);
// columns split..31 use J^T (L.valT, which must exist when split < 32)
// T16 (mode 1 only, may be null): the result also as packed BF16 hi + lo parts (lo << 16 | hi)
stm_status spmm_structured(const Level& L, const double* X, const double* B, double* Y, int mode, cudaStream_t s,
                           int split = 32, uint32_t* T16 = nullptr);
stm_status ensure_multi(Hierarchy& H);
// split < 32: columns split..31 are adjoint columns (defect with J^T, local products with J_T^{-T});
// with split = 16 and BF16 inverses on the tensor cores both come from one pass over the inverses
stm_status vanka_step_multi(Hierarchy& H, int g, const double* R, double* Dm, bool d_is_zero, cudaStream_t s,
                            int split = 32);
// Y[c][i][32] (FP32) = J_c^{-1} T_c on the tcgen05 tensor cores, BF16 inverses of leading dimension ld
// (kernels_mrhs_tc.cu); err: device word set when a pipeline wait times out
// fused = true: columns 0-15 get Y = J^{-1} T, columns 16-31 Y = J^{-T} T from the same inverse tile
bool mrhs_tc_supported(int n, int ld);
stm_status bounded_wait_selftest(int* err, cudaStream_t s);  // error word bit 128 after ~1 s
bool mrhs_tc_fused_supported(int n, int ld);
// T16: the residual block as packed BF16 hi + lo parts (lo << 16 | hi), [N][32]
stm_status mrhs_tc_apply(const Level& L, int ld, const uint32_t* T16, float* Y, int* err, cudaStream_t s,
                         bool fused = false);
// reads and clears the device error word of the tensor-core kernels (synchronous)
stm_status check_kernel_error(Hierarchy& H, cudaStream_t s);
stm_status vcycle_multi(Hierarchy& H, const double* R_fine, double* D_fine, cudaStream_t s);
stm_status mdots(const double* V, int nv, const double* w, long long n, double* out, double* part, int nblk,
                 cudaStream_t s);
stm_status mupdate(const double* V, int nv, const double* h, double* w, long long n, double sign, cudaStream_t s);
stm_status mscale(double* y, const double* x, const double* f, long long n, cudaStream_t s);
stm_status madd_small(double* a, const double* b, int n, cudaStream_t s);
stm_status vcycle(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s);
// V-cycle through a cached CUDA graph (direct launches while profiling is on)
stm_status vcycle_graph(Hierarchy& H, const double* r, double* d, int transpose, cudaStream_t s);
void clear_graphs(Hierarchy& H);

// BLAS-1 style helpers on device vectors (kernels_krylov.cu)
stm_status vec_fill(double* x, double v, long long n, cudaStream_t s);
stm_status vec_copy(double* y, const double* x, long long n, cudaStream_t s);
stm_status vec_scale_to(double* y, const double* x, const double* scale_dev, int inv, long long n, cudaStream_t s);
stm_status batched_dots(const double* V, int nv, const double* w, long long n, double* out,
                        double* part, int nblk, cudaStream_t s);
stm_status batched_update(const double* V, int nv, const double* h, double* w, long long n,
                          cudaStream_t s);
stm_status gemv_accumulate(const double* Z, int nz, const double* y, double* x, long long n,
                           cudaStream_t s);
stm_status vec_axpby_dev(double* hacc, const double* h2, int n, cudaStream_t s);
stm_status vec_axpy(double* y, double a, const double* x, long long n, cudaStream_t s);  // y += a x
stm_status vec_norm_sq(const double* x, long long n, double* out, double* part, int nblk,
                       cudaStream_t s);

}  // namespace stm
