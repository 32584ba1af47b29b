// Host-callable launchers of the device kernels (one translation unit per
// family: spmv.cu, blas.cu, amg_setup.cu).
#pragma once
#include "common.cuh"

namespace scr {

// --------------------------------------------------------------- counters
struct LaunchCounter {
  long long launches = 0;
  long long spmv_bytes = 0;
  long long vcycles[3] = {0, 0, 0};  // V-cycles recorded into a graph, by hierarchy (A, Shat, mesh)
  long long fixed[2] = {0, 0};       // fixed-count A-solve steps recorded into a graph (intermediate, inner)
};
LaunchCounter& counters();

// Event-pair timing of one kernel class (selected by the matrix value
// pointer for SpMV, or the block operator) inside a profiling region.
struct KernelProfiler {
  bool active = false;
  int kclass = 0;
  const void* target = nullptr;  // SpMV: value array of the profiled matrix
  int cap = 0, used = 0;
  long long launches = 0;
  double bytes = 0, flops = 0;
  std::vector<cudaEvent_t> ev;  // 2 * cap
};
KernelProfiler& profiler();
// returns the pair index to close with prof_stop, or -1
int prof_start(int kclass, const void* key, cudaStream_t s);
void prof_stop(int idx, double bytes, double flops, cudaStream_t s);

// --------------------------------------------------------------- layouts
// standard BSR values (block after block, row-major) -> slab layout
template <typename TO>
void to_slab(const int* rp, const double* std_val, TO* slab_val, int nbr, int br, int bc,
             long long nnzb, cudaStream_t s);
// slab -> standard (export)
void from_slab(const int* rp, const double* slab_val, double* std_val, int nbr, int br, int bc,
               long long nnzb, cudaStream_t s);
void from_slab_f(const int* rp, const float* slab_val, double* std_val, int nbr, int br, int bc,
                 long long nnzb, cudaStream_t s);
// slab double -> slab float
void slab_to_float(const double* in, float* out, long long n, cudaStream_t s);
// slab float -> slab BF16 (round to nearest even); out holds n __nv_bfloat16
void slab_to_bf16(const float* in, void* out, long long n, cudaStream_t s);

// y_p = D x_p - C x_t in one pass (the last line of Algorithm 2); C 1x3
// blocks, D 1x1, nrhs interleaved right-hand sides (1 or kSpmmCols)
template <typename T>
void schur_combine(const DBsr<T>& C, const DBsr<T>& D, const T* xt, const T* xp, T* yp, int nrhs, cudaStream_t s);

// Validation of caller index arrays before any kernel indexes with them:
// sets *bad (device int, not cleared here) when a row pointer is out of
// [0, nnzb] or decreasing, or a column index is out of [0, nbc), unsorted or
// repeated within its row (solver.cu).
void check_bsr_indices(int nbr, int nbc, const int* rp, const int* col, long long nnzb, int* bad,
                       cudaStream_t s);

// --------------------------------------------------------------- SpMV
// Epilogues applied to the row sums acc of M x (scalar output index o,
// right-hand side h, flat index gi = o*nrhs + h):
enum class Epi : int {
  Set = 0,        // y = acc
  Axpby = 1,      // y = alpha*acc + beta*z
  Resid = 2,      // y = z - acc
  Jacobi = 3,     // y = xs + (z - acc) * dinv[o]
  ChebFirst = 4,  // r = (z - acc) dinv[o]; dout = alpha r; y = xs + dout   (x = xs)
  ChebStep = 5,   // r -= acc dinv[o]; dout = alpha x + beta r; xsol += dout (x = d)
  ScaledSub = 6,  // y = z - acc * dinv[o]
};
struct EpiArgs {
  Epi kind = Epi::Set;
  double alpha = 1.0, beta = 0.0;
  const void* z = nullptr;     // same precision as y
  const void* xs = nullptr;    // Jacobi / ChebFirst: current iterate
  const void* dinv = nullptr;  // inverse l1 row sums (Jacobi) or inverse diagonal (Chebyshev)
  void* r = nullptr;           // Chebyshev: preconditioned residual (in/out)
  void* dout = nullptr;        // Chebyshev: next direction
  void* xsol = nullptr;        // ChebStep: iterate updated in place
};

// y = epilogue(M x); M in slab layout; x and y of type XT; nrhs interleaved
// right-hand sides (1 or 3).
template <typename VT, typename XT>
void spmv(const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s);

// Block products with kSpmmCols interleaved right-hand sides (x[(j * bc +
// c) * kSpmmCols + h], y likewise), any block shape of the solver
// (spmm.cu); called by spmv for nrhs == kSpmmCols.
constexpr int kSpmmCols = 8;
template <typename VT, typename XT>
void spmm_launch(int G, const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s);

// build the sliced block-ELL copy of M (values converted to VT)
template <typename VT>
void build_sell(const DBsr<double>& M, DSell<VT>& S, DeviceArena& a, cudaStream_t s, int window);

// padded copy of M for 16-byte loads (see DBsr::vdesc), for 3x3 and 1x1
// blocks; sets M.vdesc / vcol / vval (arrays in a).  Leaves M unchanged for
// other shapes or when a padded array would exceed int32 indexing.
template <typename VT>
void build_vec(DBsr<VT>& M, DeviceArena& a, cudaStream_t s);

// forced kernel code for every product (0: per-matrix choice)
void set_forced_group(int code);
int forced_group();
// CTAs ahead for the L2 prefetch of the scalar-row products (0: off)
void set_l2_prefetch(int ctas);
// programmatic dependent launch of the product kernels (0: off)
void set_pdl(int on);
// print every autotune decision to stderr (0: quiet)
void set_tune_verbose(int v);
// write / read the autotune cache as text (throw std::invalid_argument)
void tune_save(const char* path);
void tune_load(const char* path);
// time the lane-group widths for products of M with nrhs right-hand sides
// and store the fastest in M.g; returns the chosen width
template <typename VT>
int autotune_spmv(DBsr<VT>& M, int nrhs, cudaStream_t s);

// Residual assembly of the VMS formulation on the GPU (residual.cu): the
// mesh and the (element, vertex) lists of every row live on the device;
// evaluate() writes R = [R_m (3 n_nodes) | R_p (n_p)] (raw, before the
// Dirichlet rows) for the state v, vhat, p, vdot, u (device pointers;
// vhat, vdot, u may be null for zero).
struct ResidualPhysics {
  double rho_f, mu_f, rho_s, mu_s, dt, c_m_solid, c_c_solid;
};
struct ResidualAssembler {
  int nn = 0, ne = 0, np = 0;
  ResidualPhysics ph{};
  double* d_xyz = nullptr;
  int *d_ien = nullptr, *d_pien = nullptr;
  unsigned char* d_etype = nullptr;
  int *d_vptr = nullptr, *d_vent = nullptr, *d_pptr = nullptr, *d_pent = nullptr;
  double* d_E = nullptr;
  void setup(int nn, int ne, int np, const double* xyz, const int* ien, const int* pien,
             const unsigned char* etype, const ResidualPhysics& ph, DeviceArena& a, cudaStream_t s);
  void evaluate(const double* v, const double* vhat, const double* p, const double* vd, const double* u,
                double* R, cudaStream_t s);
};

// Tangent assembly on the GPU (tangent.cu): the consistent tangent of the
// element residuals of ResidualAssembler (tau frozen at the state) written
// into the values of the patterns captured by setup() (A, B, C, D in that
// order; values in the standard block layout), with the velocity Dirichlet
// nodes d_dir (may be null) as identity rows of A.  cm = alpha_m, cf =
// alpha_f gamma dt, cu = cf^2 / alpha_m.
struct TangentAssembler {
  struct Pattern {
    int nbr = 0, nbc = 0, br = 1, bc = 1;
    long long nnzb = 0;
    int *rp = nullptr, *col = nullptr, *brow = nullptr;
    double* val = nullptr;
  };
  Pattern pat[4];
  double* E = nullptr;  // per-element tangents (256 values each)
  bool ready = false;
  void setup(const ResidualAssembler& ra, const DBsr<double>* const mats[4], DeviceArena& a, cudaStream_t s);
  void evaluate(const ResidualAssembler& ra, const unsigned char* d_dir, const double* v, const double* vhat,
                const double* p, const double* vd, double cm, double cf, double cu, cudaStream_t s);
};

// y = epilogue([[A, B], [C, D]] x) in FP64 (the outer operator calA); nrhs
// interleaved right-hand sides (1 or kSpmmCols)
void block_op(const DBsr<double>& A, const DBsr<double>& B, const DBsr<double>& C,
              const DBsr<double>& D, const double* x, double* y, const double* z, bool resid,
              cudaStream_t s, int nrhs = 1);

// --------------------------------------------------------------- BLAS-1
constexpr int kMaxBasis = 64;  // largest restart length + 1
struct ArnoldiState {           // device-resident Krylov scalars
  double H[(kMaxBasis + 1) * kMaxBasis];  // column-major, ld = kMaxBasis + 1
  double cs[kMaxBasis], sn[kMaxBasis], g[kMaxBasis + 1], y[kMaxBasis];
  double h1[kMaxBasis + 1], h2[kMaxBasis + 1];
  double beta, bnorm, rel, inv_hnext, nrm2;
  int breakdown;
};
struct Reducer {  // partial-sum scratch for deterministic two-stage reductions
  double* partial = nullptr;  // [nblk * kMaxBasis]
  int nblk = 0;
};
Reducer make_reducer(DeviceArena& a);

template <typename T>
void fill(T* x, T v, long long n, cudaStream_t s);
template <typename T>
void copy(const T* x, T* y, long long n, cudaStream_t s);
void cast_d2f(const double* x, float* y, long long n, cudaStream_t s);
void cast_f2d(const float* x, double* y, long long n, cudaStream_t s);
// y = a*x + b*y
void axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s);
// y += (c * dot[0]) a with dot a device scalar (rank-1 outlet term)
template <typename T>
void axpy_dev(const T* a, const double* dot, double c, T* y, long long n, cudaStream_t s);
// d += c a .* a
void add_scaled_squares(double* d, const double* a, double c, long long n, cudaStream_t s);
// b = -R, zero on the velocity rows of flagged nodes (mask per node, may be null)
void negate_masked(const double* R, const unsigned char* mask, double* b, long long nv3, long long n,
                   cudaStream_t s);
// Mesh motion inside the corrector (Sec. 3.5, steps 3-4), one thread per
// (fluid node f, component c), entries 3 f + c.
// g = follow_f ? un + (u - un) / af at node_of_f[f] : 0
void mesh_interface_data(const int* node_of_f, const unsigned char* follow, const double* u, const double* un,
                         double af, double* g, int nf, cudaStream_t s);
// b = g on Dirichlet mesh nodes, -b (b holds L_raw g on entry) elsewhere
void mesh_lift(const unsigned char* dir_m, const double* g, double* b, int nf, cudaStream_t s);
// vhat[node_of_f[f]] = vn + af (v1 - vn), v1 = (uh - uhn) / (gamma dt) + (gamma - 1) / gamma vn
void mesh_velocity(const int* node_of_f, const double* uh, const double* uhn, const double* vn, double af,
                   double gamma, double dt, double* vhat, int nf, cudaStream_t s);
// y = 1 ./ x
void reciprocal(const double* x, double* y, long long n, cudaStream_t s);
// k vectors of length n one after another <-> interleaved (entry i of vector c
// at i * k + c)
void interleave(const double* in, double* out, long long n, int k, bool to_interleaved, cudaStream_t s);
template <typename T>
void axpby_t(double a, const T* x, double b, T* y, long long n, cudaStream_t s);
// x[o*nrhs+h] = b[o*nrhs+h] * d[o]  (l1-Jacobi sweep from a zero iterate)
template <typename T>
void diag_scale(const T* b, const T* d, T* x, long long n, int nrhs, cudaStream_t s);
// Chebyshev start from a zero iterate: r = b d, dv = r / theta, x = dv
template <typename T>
void cheb_zero(const T* b, const T* d, T* r, T* dv, T* x, double inv_theta, long long n, int nrhs,
               cudaStream_t s);

// out = ||x||^2 (device scalar).  Vector kernels take T = double or float;
// FP32 vectors are summed per thread in FP32, across threads in FP64.
template <typename T>
void norm2(const T* x, long long n, double* out, const Reducer& r, cudaStream_t s);
// The Gram-Schmidt and update kernels take their count k from the host, or,
// with kp given (loops recorded in a CUDA graph), from the device as
// *kp + koff, with k then an upper bound of it.
// out[j] = V_j . w, j < k (V vectors of length n with stride ld)
template <typename T>
void multidot(const T* V, long long ld, int k, const T* w, long long n, double* out, const Reducer& r,
              cudaStream_t s, const int* kp = nullptr, int koff = 0);
// w -= sum_j V_j h[j]; then out[j] = V_j . w (second Gram-Schmidt pass)
template <typename T>
void cgs_update_dot(const T* V, long long ld, int k, const double* h, T* w, long long n, double* out,
                    const Reducer& r, cudaStream_t s, const int* kp = nullptr, int koff = 0);
// w -= sum_j V_j h[j]; then out = ||w||^2
template <typename T>
void cgs_update_norm(const T* V, long long ld, int k, const double* h, T* w, long long n, double* out,
                     const Reducer& r, cudaStream_t s, const int* kp = nullptr, int koff = 0);
// Arnoldi bookkeeping for column j (or *jp when jp is given): H(:,j) = h1 + h2,
// H(j+1,j) = sqrt(nrm2), Givens rotations, residual estimate
// st->rel = |g_{j+1}| / bnorm, copied to *host_rel (mapped host memory) when
// host_rel is not null.
void arnoldi_finalize(ArnoldiState* st, int j, double* host_rel, cudaStream_t s, const int* jp = nullptr);
// GMRES start: beta = sqrt(st->nrm2); g = beta e_1; bnorm set when first;
// writes beta/bnorm to *host_rel when it is not null
void arnoldi_start(ArnoldiState* st, int first, double* host_rel, cudaStream_t s);
// y = x * (*scale) with scale a device scalar
template <typename T>
void scale_by(const T* x, const double* scale, T* y, long long n, cudaStream_t s);
// y = x (times *sc when sc is not null); x is column *xj of X when xj is
// given, y column *yj + yoff of Y when yj is given (columns ld apart)
template <typename T>
void col_copy(const T* X, const int* xj, T* Y, const int* yj, int yoff, long long ld, const double* sc, long long n,
              cudaStream_t s);
// y = H^{-1} g (k x k upper triangle, k = *kp when kp is given), then
// x += sum_j y_j Z_j
template <typename T>
void gmres_update(ArnoldiState* st, int k, const T* Z, long long ld, T* x, long long n, cudaStream_t s,
                  const int* kp = nullptr);

// CG helpers: scalars on the device
struct CgState {
  double rz, rz_new, pq, alpha, beta, rr, bnorm2, rel;
};
void cg_step_x_r(CgState* st, const double* p, const double* q, double* x, double* r, long long n,
                 const Reducer& red, double* host_rel, cudaStream_t s);
void cg_dot_rz(CgState* st, const double* r, const double* z, long long n, const Reducer& red,
               int first, cudaStream_t s);
void cg_update_p(CgState* st, const double* z, double* p, long long n, cudaStream_t s);
void cg_alpha(CgState* st, const double* p, const double* q, long long n, const Reducer& red,
              cudaStream_t s);
void cg_start(CgState* st, const double* b, long long n, const Reducer& red, double* host_rel,
              cudaStream_t s);

// --------------------------------------------------------------- AMG set-up
// exclusive scan of n ints; returns the total (host sync)
long long exclusive_scan(const int* in, int* out, int n, DeviceArena& tmp, cudaStream_t s);

// sparse product C = A * B of slab matrices (deterministic); C allocated in arena
void spgemm(const DBsr<double>& A, const DBsr<double>& B, DBsr<double>& C, DeviceArena& arena,
            cudaStream_t s);
// C = alpha A + diag(rowscale) B with the scalar rows of B scaled by
// rowscale; rowscale == nullptr means C = alpha A - B
void spadd(const DBsr<double>& A, double alpha, const DBsr<double>& B, const double* rowscale,
           DBsr<double>& C, DeviceArena& arena, cudaStream_t s);
// out = diag(d)^{-1} M, sharing M's pattern
void scale_rows_inv(const DBsr<double>& M, const double* d, DBsr<double>& out, DeviceArena& a, cudaStream_t s);
// interpolation truncation: keep the blocks of each row whose norm is at
// least trunc * the row maximum, at most pmax of them (largest first, ties
// by smaller column), rescale each scalar row to its original sum
void truncate_rows(const DBsr<double>& P, double trunc, int pmax, DBsr<double>& out, DeviceArena& a,
                   cudaStream_t s);
// transpose (blocks transposed)
void transpose(const DBsr<double>& A, DBsr<double>& T, DeviceArena& arena, cudaStream_t s);
// scalar diagonal of A (n scalar rows); returns false if a diagonal entry is missing/zero
void diag_scalar(const DBsr<double>& A, double* d, int* bad, cudaStream_t s);
// 1 / a_ii per scalar row (0 where the diagonal is zero)
void inv_diag(const DBsr<double>& A, double* dinv, cudaStream_t s);
// 1.1 x the power-iteration estimate (iters steps) of rho(D^{-1} A), from
// the fixed start vector 1 + ((i * 2654435761) mod 2^32 mod 1000) / 1000
double power_lambda(const DBsr<double>& A, const double* dinv, int iters, cudaStream_t s);
// 1/ sum_j |a_ij| per scalar row
void l1_inv(const DBsr<double>& A, double* dinv, cudaStream_t s);
// v = the power-iteration start vector 1 + ((i * 2654435761) mod 2^32 mod
// 1000) / 1000, normalised; nrm: 2 doubles of scratch
void power_start_unit(double* v, long long n, const Reducer& red, double* nrm, cudaStream_t s);
// d_i = sum_j |a_ij| per scalar row (SIMPLEC's lumped diagonal)
void abs_rowsum(const DBsr<double>& A, double* d, cudaStream_t s);
// max_i sum_j |a_ij| / |a_ii| (device scalar)
void gershgorin(const DBsr<double>& A, const double* diag, double* out, cudaStream_t s);
// scale scalar rows of B by -omega(dev)/d_i : out rowscale[n]
void prolong_rowscale(const double* diag, const double* lambda, double* rowscale, int n,
                      cudaStream_t s);

struct Aggregation {
  int* agg = nullptr;    // per block row, -1 = none
  int* roots = nullptr;  // per aggregate: its root (the MIS-2 node that seeded it)
  int n_agg = 0;
};
// strength graph + MIS-2 aggregation of the block rows of A
Aggregation aggregate(const DBsr<double>& A, double theta, DeviceArena& arena, DeviceArena& tmp,
                      cudaStream_t s, int* mis_rounds);
// numeric re-set-up on unchanged patterns (amg_setup.cu): C = A B, C = alpha
// A + beta diag(rowscale) B (beta = 1, or -1 without rowscale), out =
// diag(d)^{-1} M values, O = the row-sum preserving truncation of P to O's
// kept columns, T = A^T; each writes the values of an output whose pattern
// a full set-up built
void spgemm_numeric(const DBsr<double>& A, const DBsr<double>& B, DBsr<double>& C, cudaStream_t s);
void spadd_numeric(const DBsr<double>& A, double alpha, const DBsr<double>& B, const double* rowscale,
                   DBsr<double>& C, cudaStream_t s);
void scale_rows_inv_values(const DBsr<double>& M, const double* d, double* out, cudaStream_t s);
void truncate_refill(const DBsr<double>& P, DBsr<double>& O, cudaStream_t s);
void transpose_numeric(const DBsr<double>& A, DBsr<double>& T, cudaStream_t s);
// the padded copy's values from M's slab values (same pattern)
template <typename VT>
void refresh_vec(DBsr<VT>& M, cudaStream_t s);
// tentative prolongator I_bs / sqrt(|a|)
void tentative(const int* agg, int nbr, int n_agg, int bs, DBsr<double>& P, DeviceArena& arena,
               DeviceArena& tmp, cudaStream_t s);
// dense copy (column-major n x n) and in-place Gauss-Jordan inverse
void to_dense(const DBsr<double>& A, double* dense, cudaStream_t s);
void dense_inverse(double* M, double* inv, int n, int* singular, cudaStream_t s);
// x[i*nrhs+h] = sum_j inv[i + j n] b[j*nrhs+h]
void dense_apply(const double* inv, const double* b, double* x, int n, int nrhs, cudaStream_t s);
void dense_apply_f(const float* inv, const float* b, float* x, int n, int nrhs, cudaStream_t s);

}  // namespace scr
