// Host drivers of the SCR-FGMRES + AMG path and the C ABI (scr_gb300.h).
//
// Outer level (Sec. 5.2.1): FGMRES(m) on calA x = b in FP64, classical
// Gram-Schmidt applied twice, Givens rotations, x_0 = 0, stop when the
// recurrence residual drops below rtol and the recomputed FP64 residual
// confirms it.  Preconditioner: Algorithm 1 of App. B (SCR) with
// Algorithm 2 for the Schur complement; the intermediate and inner solves
// are GMRES(m) with AMG V-cycles (P_A = P_I = AMG(A), P_S = AMG(Shat)).  The
// mesh-motion system (Sec. 5.2.2) uses CG + AMG.  Every arithmetic step runs
// in the kernels of spmv.cu / blas.cu / amg_setup.cu; the host only orders
// launches and reads one residual estimate per Krylov iteration (mapped
// host memory) to decide when to stop.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <functional>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>

#include "kernels.h"

namespace scr {

static thread_local std::string g_last_error;

void set_last_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void configure_pool(int device) {
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
}

using Clock = std::chrono::steady_clock;
static double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// ------------------------------------------------------------ host scalars
// Two doubles of mapped pinned memory per solver: the device writes the
// residual estimate there and the host reads it after a stream sync.
// Scalars the host reads after a stream synchronisation (Krylov residual
// estimates).  Mapped mode (default): the kernels write them straight into
// mapped pinned host memory.  Copy mode: the kernels write a device buffer,
// and fetch() queues a 16-byte copy into pinned host memory before the
// synchronisation.  Measured on the 616k-node tube: mapped 1070 ms per FP64
// step, copy 1074 ms.
int g_mapped_scalars = 1;
struct HostScalars {
  double* h = nullptr;
  double* d = nullptr;
  bool mapped = false;
  HostScalars() {
    mapped = g_mapped_scalars != 0;
    if (mapped) {
      SCR_CUDA(cudaHostAlloc(&h, 4 * sizeof(double), cudaHostAllocMapped));
      SCR_CUDA(cudaHostGetDevicePointer(&d, h, 0));
    } else {
      SCR_CUDA(cudaHostAlloc(&h, 4 * sizeof(double), cudaHostAllocDefault));
      SCR_CUDA(cudaMalloc(&d, 4 * sizeof(double)));
    }
  }
  ~HostScalars() {
    if (h) cudaFreeHost(h);
    if (d && !mapped) cudaFree(d);
  }
  void fetch(cudaStream_t s) {
    if (!mapped) SCR_CUDA(cudaMemcpyAsync(h, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  HostScalars(const HostScalars&) = delete;
  HostScalars& operator=(const HostScalars&) = delete;
};

// nesting depth of Krylov-loop captures in progress on this thread: inside
// one, V-cycles run as plain launches (recorded) and GMRES solves record
// their loops inline
static thread_local int g_capture_depth = 0;

// ------------------------------------------------------------ AMG hierarchy
struct Level {
  DBsr<double> A, P, R;
  // products of the build kept for a numeric re-set-up (refresh): the
  // tentative prolongator, A P_tent, the untruncated smoothed prolongator
  // and A P (their patterns are reused, their values recomputed)
  DBsr<double> Pt, T, Ps, AP;
  DBsr<float> Af, Pf, Rf;
  double* dinv = nullptr;   // l1-Jacobi: 1 / sum_j |a_ij|
  float* dinvf = nullptr;
  double* dd = nullptr;     // Chebyshev: 1 / a_ii
  float* ddf = nullptr;
  double lam = 0.0;         // Chebyshev interval [lam/30, lam]
  bool cheb_off = false;    // the Chebyshev guard switched this level to l1-Jacobi
  double *d0 = nullptr, *d1 = nullptr;
  float *d0f = nullptr, *d1f = nullptr;
  int* agg = nullptr;
  int* roots = nullptr;  // root block row of each aggregate
  int n_agg = 0;
  long long n = 0;  // scalar rows
  double *b = nullptr, *x = nullptr, *r = nullptr, *t = nullptr;
  float *bf = nullptr, *xf = nullptr, *rf = nullptr, *tf = nullptr;
};

template <typename T>
static const DBsr<T>& pick(const DBsr<double>& d, const DBsr<float>& f);
template <>
const DBsr<double>& pick<double>(const DBsr<double>& d, const DBsr<float>&) {
  return d;
}
template <>
const DBsr<float>& pick<float>(const DBsr<double>&, const DBsr<float>& f) {
  return f;
}

static DBsr<float> to_float_copy(const DBsr<double>& M, DeviceArena& a, cudaStream_t s) {
  DBsr<float> F;
  F.nbr = M.nbr;
  F.nbc = M.nbc;
  F.br = M.br;
  F.bc = M.bc;
  F.nnzb = M.nnzb;
  F.rp = M.rp;
  F.col = M.col;
  F.val = a.alloc<float>(M.nnzb * M.br * M.bc + 1);
  F.g = 0;
  slab_to_float(M.val, F.val, M.nnzb * M.br * M.bc, s);
  return F;
}

// BF16 copy of an FP32 matrix's values, used by its products from now on
static void add_bf16_copy(DBsr<float>& F, DeviceArena& a, cudaStream_t s) {
  if (F.nnzb == 0) return;
  const long long n = F.nnzb * F.br * F.bc;
  uint16_t* h = a.alloc<uint16_t>(n + 1);
  slab_to_bf16(F.val, h, n, s);
  F.hval = h;
}

// the timed choice of the product kernel (o.autotune) for products of M
// with nrhs right-hand sides
template <typename VT>
static void tune_product(DBsr<VT>& M, int nrhs, const scr_opts& o, DeviceArena& a, cudaStream_t s) {
  (void)a;
  if (o.autotune) autotune_spmv<VT>(M, nrhs, s);
}

struct GraphExecDeleter {
  void operator()(CUgraphExec_st* g) const {
    if (g) cudaGraphExecDestroy(g);
  }
};
using GraphExecPtr = std::unique_ptr<CUgraphExec_st, GraphExecDeleter>;

struct Hierarchy {
  int slot = 0;  // 0: A, 1: Shat, 2: mesh (the recorded V-cycle counters)
  int bs = 1, nrhs = 1, nu = 1;
  int smoother = SCR_SMOOTH_CHEB, degree = 3;
  double cheb_theta_inv = 0.0;
  bool f32 = false;
  std::vector<Level> lv;
  double* cinv = nullptr;
  float* cinvf = nullptr;
  int nc = 0;
  int vcycles = 0;
  int mis_rounds = 0;
  std::unique_ptr<DeviceArena> arena;
  // CUDA graph of one V-cycle from the staging vector gin to gout (captured
  // at the first V-cycle after set-up, replayed by every later one); the
  // library counters of one captured V-cycle are added at each replay
  bool use_graph = false, graph_failed = false;
  GraphExecPtr gexec;
  void *gin = nullptr, *gout = nullptr;
  size_t gsize = 0;  // element size the graph was captured for
  long long glaunches = 0, gbytes = 0;

  int n_levels() const { return (int)lv.size(); }

  void build(const DBsr<double>& A0, int bs_, int nrhs_, const scr_opts& o, bool use_f32, cudaStream_t s,
             const DBsr<float>* A0f = nullptr) {
    bs = bs_;
    nrhs = nrhs_;
    use_graph = o.cuda_graphs != 0;
    graph_failed = false;
    gexec.reset();
    gin = gout = nullptr;
    gsize = 0;
    nu = std::max(1, o.amg_nu);
    smoother = o.amg_smoother;
    degree = std::max(1, o.amg_degree);
    f32 = use_f32;
    lv.clear();
    arena.reset(new DeviceArena(s));
    DeviceArena& ar = *arena;
    DBsr<double> Al = A0;
    for (;;) {
      Level L;
      L.A = Al;
      L.n = (long long)Al.nbr * bs;
      L.dinv = ar.alloc<double>(L.n + 1);
      l1_inv(Al, L.dinv, s);
      const bool last = Al.nbr <= o.amg_coarse_size || (int)lv.size() + 1 >= o.amg_max_levels;
      if (!last) {
        DeviceArena tmp(s);
        auto t0 = Clock::now();
        Aggregation ag = aggregate(Al, o.amg_theta, ar, tmp, s, &mis_rounds);
        SCR_CUDA(cudaStreamSynchronize(s));
        const double t_agg = ms_since(t0);
        if (ag.n_agg > 0 && ag.n_agg < (int)(0.9 * Al.nbr)) {
          L.agg = ag.agg;
          L.roots = ag.roots;
          L.n_agg = ag.n_agg;
          DBsr<double> Pt, T, AP, Ac;
          t0 = Clock::now();
          tentative(ag.agg, Al.nbr, ag.n_agg, bs, Pt, ar, tmp, s);
          double* d = tmp.alloc<double>(L.n + 1);
          int* bad = tmp.alloc<int>(1);
          SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
          diag_scalar(Al, d, bad, s);
          double* lam = tmp.alloc<double>(1);
          gershgorin(Al, d, lam, s);
          double* rs = tmp.alloc<double>(L.n + 1);
          prolong_rowscale(d, lam, rs, (int)L.n, s);
          spgemm(Al, Pt, T, ar, s);
          L.Pt = Pt;
          L.T = T;
          if (o.amg_trunc > 0.0 || o.amg_pmax > 0) {
            DBsr<double> Ps;
            spadd(Pt, 1.0, T, rs, Ps, ar, s);
            truncate_rows(Ps, o.amg_trunc, o.amg_pmax, L.P, ar, s);
            L.Ps = Ps;
          } else {
            spadd(Pt, 1.0, T, rs, L.P, ar, s);
          }
          SCR_CUDA(cudaStreamSynchronize(s));
          const double t_p = ms_since(t0);
          t0 = Clock::now();
          transpose(L.P, L.R, ar, s);
          SCR_CUDA(cudaStreamSynchronize(s));
          const double t_tr = ms_since(t0);
          t0 = Clock::now();
          spgemm(Al, L.P, AP, ar, s);
          L.AP = AP;
          SCR_CUDA(cudaStreamSynchronize(s));
          const double t_ap = ms_since(t0);
          t0 = Clock::now();
          spgemm(L.R, AP, Ac, ar, s);
          SCR_CUDA(cudaStreamSynchronize(s));
          const double t_rap = ms_since(t0);
          if (o.verbose)
            fprintf(stderr,
                    "[amg bs=%d] level %zu: %d block rows, %lld blocks -> %d aggregates (%d MIS rounds); P %lld blocks,"
                    " AP %lld, Ac %lld | ms: agg %.2f P %.2f R %.2f AP %.2f RAP %.2f\n",
                    bs, lv.size(), Al.nbr, Al.nnzb, ag.n_agg, mis_rounds, L.P.nnzb, AP.nnzb, Ac.nnzb, t_agg, t_p,
                    t_tr, t_ap, t_rap);
          lv.push_back(L);
          Al = Ac;
          continue;
        }
      }
      lv.push_back(L);
      break;
    }
    // coarsest level: dense inverse
    Level& C = lv.back();
    nc = (int)C.n;
    auto tc0 = Clock::now();
    if (nc > 4096) throw CudaError{cudaErrorInvalidValue, "coarsest AMG level too large for a dense inverse"};
    {
      DeviceArena tmp(s);
      double* M = tmp.alloc<double>((size_t)nc * nc + 1);
      cinv = ar.alloc<double>((size_t)nc * nc + 1);
      int* sing = tmp.alloc<int>(1);
      SCR_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
      to_dense(C.A, M, s);
      dense_inverse(M, cinv, nc, sing, s);
      int hs = 0;
      SCR_CUDA(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      if (hs) throw CudaError{cudaErrorInvalidValue, "singular coarsest AMG operator"};
    }
    if (o.verbose)
      fprintf(stderr, "[amg bs=%d] coarsest level %zu: %d scalar rows, dense inverse %.2f ms\n", bs, lv.size() - 1,
              nc, ms_since(tc0));
    // work vectors and FP32 copies
    for (size_t l = 0; l < lv.size(); ++l) {
      Level& L = lv[l];
      const long long m = L.n * nrhs + 1;
      if (smoother == SCR_SMOOTH_CHEB && l + 1 < lv.size()) {
        L.dd = ar.alloc<double>(L.n + 1);
        inv_diag(L.A, L.dd, s);
        L.lam = power_lambda(L.A, L.dd, 20, s);
        L.cheb_off = cheb_guard_growth(L, s) > kChebGuardGrowth;
        if (o.verbose && L.cheb_off)
          fprintf(stderr, "[amg bs=%d] level %zu: Chebyshev guard -> l1-Jacobi\n", bs, l);
        if (f32) {
          L.ddf = ar.alloc<float>(L.n + 1);
          cast_d2f(L.dd, L.ddf, L.n, s);
          L.d0f = ar.alloc<float>(m);
          L.d1f = ar.alloc<float>(m);
        } else {
          L.d0 = ar.alloc<double>(m);
          L.d1 = ar.alloc<double>(m);
        }
      }
      if (!f32) {
        L.b = ar.alloc<double>(m);
        L.x = ar.alloc<double>(m);
        L.r = ar.alloc<double>(m);
        L.t = ar.alloc<double>(m);
      } else {
        L.Af = (l == 0 && A0f) ? *A0f : to_float_copy(L.A, ar, s);
        // the finest operator's 16-byte copy (Shat in FP32; A's comes with A0f)
        if (l == 0 && o.vec && !L.Af.vdesc) build_vec<float>(L.Af, ar, s);
        if (L.P.nbr) {
          L.Pf = to_float_copy(L.P, ar, s);
          L.Rf = to_float_copy(L.R, ar, s);
        }
        // coarse levels: products read BF16 values (FP32 vectors and sums);
        // the coarsest operator is only used through its dense inverse
        if (o.amg_coarse_bf16 && l >= 1 && l + 1 < lv.size()) {
          add_bf16_copy(L.Af, ar, s);
          add_bf16_copy(L.Pf, ar, s);
          add_bf16_copy(L.Rf, ar, s);
        }
        L.dinvf = ar.alloc<float>(L.n + 1);
        cast_d2f(L.dinv, L.dinvf, L.n, s);
        L.bf = ar.alloc<float>(m);
        L.xf = ar.alloc<float>(m);
        L.rf = ar.alloc<float>(m);
        L.tf = ar.alloc<float>(m);
      }
    }
    if (f32) {
      cinvf = ar.alloc<float>((size_t)nc * nc + 1);
      cast_d2f(cinv, cinvf, (long long)nc * nc, s);
    }
    // lane-group widths of the products on the two finest levels
    if (o.autotune) {
      for (size_t l = 0; l < lv.size() && l < 2; ++l) {
        Level& L = lv[l];
        if (L.n < 4096) continue;
        if (f32) {
          if (!(l == 0 && A0f)) tune_product<float>(L.Af, nrhs, o, ar, s);
          if (L.P.nbr) {
            tune_product<float>(L.Pf, nrhs, o, ar, s);
            tune_product<float>(L.Rf, nrhs, o, ar, s);
          }
        } else {
          if (l > 0 || A0.g == 0) tune_product<double>(L.A, nrhs, o, ar, s);
          if (L.P.nbr) {
            tune_product<double>(L.P, nrhs, o, ar, s);
            tune_product<double>(L.R, nrhs, o, ar, s);
          }
        }
      }
    }
    SCR_CUDA(cudaStreamSynchronize(s));
  }

  // New values on the patterns of the last build: A0 has the pattern of the
  // build's level-0 operator (its values may differ).  Every level's
  // operator, prolongator, restriction and smoother data are recomputed on
  // the stored patterns: the aggregates, the truncation's kept positions and
  // the sparse products' patterns are those of the build (a numeric
  // re-set-up); the V-cycle graph is recorded again at its next use.
  void refresh(const DBsr<double>& A0, const scr_opts& o, cudaStream_t s, const DBsr<float>* A0f = nullptr) {
    gexec.reset();
    graph_failed = false;
    gin = gout = nullptr;
    gsize = 0;
    const int nl = n_levels();
    if (nl == 0) return;
    lv[0].A.val = A0.val;
    lv[0].A.vdesc = A0.vdesc;
    lv[0].A.vval = A0.vval;
    for (int l = 0; l < nl; ++l) {
      Level& L = lv[l];
      l1_inv(L.A, L.dinv, s);
      if (l + 1 >= nl) break;
      DeviceArena tmp(s);
      double* d = tmp.alloc<double>(L.n + 1);
      int* bad = tmp.alloc<int>(1);
      SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      diag_scalar(L.A, d, bad, s);
      double* lam = tmp.alloc<double>(1);
      gershgorin(L.A, d, lam, s);
      double* rs = tmp.alloc<double>(L.n + 1);
      prolong_rowscale(d, lam, rs, (int)L.n, s);
      spgemm_numeric(L.A, L.Pt, L.T, s);
      if (L.Ps.nbr) {
        spadd_numeric(L.Pt, 1.0, L.T, rs, L.Ps, s);
        truncate_refill(L.Ps, L.P, s);
      } else {
        spadd_numeric(L.Pt, 1.0, L.T, rs, L.P, s);
      }
      transpose_numeric(L.P, L.R, s);
      spgemm_numeric(L.A, L.P, L.AP, s);
      spgemm_numeric(L.R, L.AP, lv[l + 1].A, s);
      SCR_CUDA(cudaStreamSynchronize(s));
    }
    // coarsest level: dense inverse
    {
      DeviceArena tmp(s);
      double* M = tmp.alloc<double>((size_t)nc * nc + 1);
      int* sing = tmp.alloc<int>(1);
      SCR_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
      to_dense(lv.back().A, M, s);
      dense_inverse(M, cinv, nc, sing, s);
      int hs = 0;
      SCR_CUDA(cudaMemcpyAsync(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      if (hs) throw CudaError{cudaErrorInvalidValue, "singular coarsest AMG operator"};
    }
    // smoother data and lower-precision copies, as in build
    for (int l = 0; l < nl; ++l) {
      Level& L = lv[l];
      if (smoother == SCR_SMOOTH_CHEB && l + 1 < nl) {
        inv_diag(L.A, L.dd, s);
        L.lam = power_lambda(L.A, L.dd, 20, s);
        L.cheb_off = cheb_guard_growth(L, s) > kChebGuardGrowth;
        if (f32) cast_d2f(L.dd, L.ddf, L.n, s);
      }
      if (f32) {
        if (!(l == 0 && A0f)) {
          slab_to_float(L.A.val, L.Af.val, L.A.nnzb * L.A.br * L.A.bc, s);
          if (L.Af.vdesc) refresh_vec<float>(L.Af, s);
        }
        if (L.P.nbr) {
          slab_to_float(L.P.val, L.Pf.val, L.P.nnzb * L.P.br * L.P.bc, s);
          slab_to_float(L.R.val, L.Rf.val, L.R.nnzb * L.R.br * L.R.bc, s);
        }
        if (L.Af.hval) slab_to_bf16(L.Af.val, const_cast<void*>(L.Af.hval), L.Af.nnzb * L.Af.br * L.Af.bc, s);
        if (L.Pf.hval) slab_to_bf16(L.Pf.val, const_cast<void*>(L.Pf.hval), L.Pf.nnzb * L.Pf.br * L.Pf.bc, s);
        if (L.Rf.hval) slab_to_bf16(L.Rf.val, const_cast<void*>(L.Rf.hval), L.Rf.nnzb * L.Rf.br * L.Rf.bc, s);
        cast_d2f(L.dinv, L.dinvf, L.n, s);
      }
    }
    if (f32) cast_d2f(cinv, cinvf, (long long)nc * nc, s);
    SCR_CUDA(cudaStreamSynchronize(s));
  }

  template <typename T>
  T* vb(Level& L) {
    if constexpr (sizeof(T) == 8) return L.b; else return L.bf;
  }
  template <typename T>
  T* vr(Level& L) {
    if constexpr (sizeof(T) == 8) return L.r; else return L.rf;
  }
  template <typename T>
  T* vt(Level& L) {
    if constexpr (sizeof(T) == 8) return L.t; else return L.tf;
  }
  template <typename T>
  T* vx(Level& L) {
    if constexpr (sizeof(T) == 8) return L.x; else return L.xf;
  }
  template <typename T>
  const T* dv(Level& L) {
    if constexpr (sizeof(T) == 8) return L.dinv; else return L.dinvf;
  }

  // Chebyshev guard: the smoother's error propagation run kChebGuardSweeps
  // times on the homogeneous problem (FP64, level operator and inverse
  // diagonal of the set-up) from the normalised power-iteration start
  // vector; returns ||e||.  A level whose error grows beyond
  // kChebGuardGrowth is smoothed by l1-Jacobi instead: nonsymmetric coarse
  // operators (Galerkin levels of Shat with a heavy, stiff wall) can have
  // eigenvalues of D^{-1}A off [lam/30, lam], where the polynomial amplifies.
  static constexpr int kChebGuardSweeps = 5;
  static constexpr double kChebGuardGrowth = 10.0;
  double cheb_guard_growth(Level& L, cudaStream_t s) {
    const long long n = L.n;
    DeviceArena tmp(s);
    Reducer red = make_reducer(tmp);
    double* e = tmp.alloc<double>(n + 1);
    double* out = tmp.alloc<double>(n + 1);
    double* r = tmp.alloc<double>(n + 1);
    double* d0 = tmp.alloc<double>(n + 1);
    double* d1 = tmp.alloc<double>(n + 1);
    double* zero = tmp.alloc<double>(n + 1);
    double* nrm = tmp.alloc<double>(2);
    fill<double>(zero, 0.0, n, s);
    power_start_unit(e, n, red, nrm, s);
    double inv_theta;
    std::vector<std::pair<double, double>> st;
    cheb_coeffs(L.lam, degree, &inv_theta, st);
    for (int k = 0; k < kChebGuardSweeps; ++k) {
      EpiArgs f;
      f.kind = Epi::ChebFirst;
      f.alpha = inv_theta;
      f.z = zero;
      f.xs = e;
      f.dinv = L.dd;
      f.r = r;
      f.dout = d0;
      spmv<double, double>(L.A, e, out, 1, f, s);
      double *a = d0, *b = d1;
      EpiArgs g;
      g.kind = Epi::ChebStep;
      g.dinv = L.dd;
      g.r = r;
      for (auto& ab : st) {
        g.alpha = ab.first;
        g.beta = ab.second;
        g.dout = b;
        g.xsol = out;
        spmv<double, double>(L.A, a, b, 1, g, s);
        std::swap(a, b);
      }
      std::swap(e, out);
    }
    norm2<double>(e, n, nrm, red, s);
    double h = 0.0;
    SCR_CUDA(cudaMemcpyAsync(&h, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    return std::sqrt(h);
  }

  // Chebyshev coefficients on [lam/30, lam]: 1/theta and (alpha_j, beta_j)
  static void cheb_coeffs(double lam, int degree, double* inv_theta, std::vector<std::pair<double, double>>& st) {
    const double lo = lam / 30.0, hi = lam;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    st.clear();
    for (int j = 1; j < degree; ++j) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      st.emplace_back(rn * rho, 2.0 * rn / delta);
      rho = rn;
    }
    *inv_theta = 1.0 / theta;
  }

  template <typename T>
  void cycle_cheb(int l, const T* b, T* out, cudaStream_t s) {
    Level& L = lv[l];
    const DBsr<T>& A = pick<T>(L.A, L.Af);
    const DBsr<T>& P = pick<T>(L.P, L.Pf);
    const DBsr<T>& R = pick<T>(L.R, L.Rf);
    const T* dd;
    T *d0, *d1;
    if constexpr (sizeof(T) == 8) {
      dd = L.dd;
      d0 = L.d0;
      d1 = L.d1;
    } else {
      dd = L.ddf;
      d0 = L.d0f;
      d1 = L.d1f;
    }
    double inv_theta;
    std::vector<std::pair<double, double>> st;
    cheb_coeffs(L.lam, degree, &inv_theta, st);
    T* r = vr<T>(L);
    T* cur = vt<T>(L);
    // pre-smoothing from zero
    cheb_zero<T>(b, dd, r, d0, cur, inv_theta, L.n, nrhs, s);
    EpiArgs e;
    e.kind = Epi::ChebStep;
    e.dinv = dd;
    e.r = r;
    for (auto& ab : st) {
      e.alpha = ab.first;
      e.beta = ab.second;
      e.dout = d1;
      e.xsol = cur;
      spmv<T, T>(A, d0, d1, nrhs, e, s);
      std::swap(d0, d1);
    }
    // coarse-grid correction
    EpiArgs res;
    res.kind = Epi::Resid;
    res.z = b;
    spmv<T, T>(A, cur, r, nrhs, res, s);
    Level& Lc = lv[l + 1];
    T* bc = vb<T>(Lc);
    spmv<T, T>(R, r, bc, nrhs, EpiArgs(), s);
    T* xc = vx<T>(Lc);
    cycle<T>(l + 1, bc, xc, s);
    EpiArgs pro;
    pro.kind = Epi::Axpby;
    pro.alpha = 1.0;
    pro.beta = 1.0;
    pro.z = cur;
    spmv<T, T>(P, xc, cur, nrhs, pro, s);
    // post-smoothing from cur, result in out
    EpiArgs f;
    f.kind = Epi::ChebFirst;
    f.alpha = inv_theta;
    f.z = b;
    f.xs = cur;
    f.dinv = dd;
    f.r = r;
    f.dout = d0;
    spmv<T, T>(A, cur, out, nrhs, f, s);
    for (auto& ab : st) {
      e.alpha = ab.first;
      e.beta = ab.second;
      e.dout = d1;
      e.xsol = out;
      spmv<T, T>(A, d0, d1, nrhs, e, s);
      std::swap(d0, d1);
    }
  }

  // out = V-cycle(b) at level l, starting from a zero iterate
  template <typename T>
  void cycle(int l, const T* b, T* out, cudaStream_t s) {
    Level& L = lv[l];
    if (l == n_levels() - 1) {
      if constexpr (sizeof(T) == 8) dense_apply(cinv, b, out, nc, nrhs, s);
      else dense_apply_f(cinvf, b, out, nc, nrhs, s);
      return;
    }
    if (smoother == SCR_SMOOTH_CHEB && !L.cheb_off) {
      cycle_cheb<T>(l, b, out, s);
      return;
    }
    const DBsr<T>& A = pick<T>(L.A, L.Af);
    const DBsr<T>& P = pick<T>(L.P, L.Pf);
    const DBsr<T>& R = pick<T>(L.R, L.Rf);
    const T* dinv = dv<T>(L);
    T* tb = vt<T>(L);
    // 2 nu - 1 out-of-place sweeps follow the first, so starting in the
    // scratch buffer leaves the result in out
    T* cur = tb;
    T* oth = out;
    diag_scale<T>(b, dinv, cur, L.n, nrhs, s);
    EpiArgs jac;
    jac.kind = Epi::Jacobi;
    jac.z = b;
    jac.dinv = dinv;
    for (int it = 1; it < nu; ++it) {
      jac.xs = cur;
      spmv<T, T>(A, cur, oth, nrhs, jac, s);
      std::swap(cur, oth);
    }
    EpiArgs res;
    res.kind = Epi::Resid;
    res.z = b;
    T* r = vr<T>(L);
    spmv<T, T>(A, cur, r, nrhs, res, s);
    Level& Lc = lv[l + 1];
    T* bc = vb<T>(Lc);
    spmv<T, T>(R, r, bc, nrhs, EpiArgs(), s);
    T* xc = vx<T>(Lc);
    cycle<T>(l + 1, bc, xc, s);
    EpiArgs pro;
    pro.kind = Epi::Axpby;
    pro.alpha = 1.0;
    pro.beta = 1.0;
    pro.z = cur;
    spmv<T, T>(P, xc, cur, nrhs, pro, s);
    for (int it = 0; it < nu; ++it) {
      jac.xs = cur;
      spmv<T, T>(A, cur, oth, nrhs, jac, s);
      std::swap(cur, oth);
    }
    if (cur != out) copy<T>(cur, out, L.n * nrhs, s);
  }

  // record one V-cycle (gin -> gout) as a CUDA graph; on any failure the
  // hierarchy keeps running V-cycles eagerly
  template <typename T>
  void capture(cudaStream_t s) {
    const long long n = lv[0].n * nrhs;
    T* in = arena->alloc<T>(n + 1);
    T* out = arena->alloc<T>(n + 1);
    fill<T>(in, (T)0, n, s);
    // an eager V-cycle first: kernels configured on first use are set up
    // outside the capture
    cycle<T>(0, in, out, s);
    SCR_CUDA(cudaStreamSynchronize(s));
    const long long l0 = counters().launches, b0 = counters().spmv_bytes;
    // recorded on a private stream (the caller's stream may be the legacy
    // default stream, which cannot be captured); replayed on the caller's
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        cycle<T>(0, in, out, cs);
      } catch (const CudaError&) {
        e = cudaErrorStreamCaptureInvalidated;
      }
      const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (cs) cudaStreamDestroy(cs);
    glaunches = counters().launches - l0;
    gbytes = counters().spmv_bytes - b0;
    counters().launches = l0;  // the captured work has not run yet
    counters().spmv_bytes = b0;
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || !ex) {
      cudaGetLastError();
      graph_failed = true;
      return;
    }
    gexec.reset(ex);
    gin = in;
    gout = out;
    gsize = sizeof(T);
  }

  template <typename T>
  void apply(const T* b, T* x, cudaStream_t s) {
    if (g_capture_depth > 0) {  // recorded into a graph: counted at each replay
      cycle<T>(0, b, x, s);
      counters().vcycles[slot]++;
      return;
    }
    ++vcycles;
    // the per-launch event profiler needs the launches themselves
    if (use_graph && !graph_failed && !profiler().active) {
      if (!gexec) capture<T>(s);
      if (gexec && gsize == sizeof(T)) {
        const long long n = lv[0].n * nrhs;
        copy<T>(b, static_cast<T*>(gin), n, s);
        SCR_CUDA(cudaGraphLaunch(gexec.get(), s));
        copy<T>(static_cast<const T*>(gout), x, n, s);
        counters().launches += glaunches;
        counters().spmv_bytes += gbytes;
        return;
      }
    }
    cycle<T>(0, b, x, s);
  }
};

// ------------------------------------------------------------ device loops
// A GMRES solve can be recorded into a CUDA graph with its control flow on
// the device (option graph_krylov): a WHILE node over the restart cycles
// holds a WHILE node over the Arnoldi steps (copy of v_j, preconditioner,
// operator, the Gram-Schmidt passes, the Givens update, v_{j+1}), then the
// solution update and an IF node with the restart.  One-thread kernels set
// each node's condition from the residual estimate on the device, with the
// same tests, in the same order, as the host-driven loop (Gmres::solve), so
// both run the same kernels on the same data.  Every Arnoldi step counts
// against the iteration cap and every cycle against a cycle cap, so each
// loop ends after at most maxit body runs whatever the estimates are.
struct KrylovLoop {
  int j;          // Arnoldi step inside the current cycle
  int iters;      // Arnoldi steps of the current solve
  int cycles;     // restart cycles of the current solve
  int nonfinite;  // 1 when an estimate was NaN or infinite
  double rel;     // last residual estimate
  // since the last reset (read back once per outer solve for the counters)
  long long tot_iters, tot_solves, tot_cycles, tot_restarts;
};

// streams that record conditional bodies, one per nesting depth, created
// before the outermost capture begins
constexpr int kMaxCaptureDepth = 8;
static thread_local cudaStream_t g_capture_streams[kMaxCaptureDepth + 1] = {};

__global__ void k_loop_begin(const ArnoldiState* __restrict__ st, KrylovLoop* L, cudaGraphConditionalHandle h_outer) {
  const double b = st->bnorm;
  L->j = 0;
  L->iters = 0;
  L->cycles = 0;
  L->nonfinite = isfinite(b) ? 0 : 1;
  L->rel = isfinite(b) ? 0.0 : b;
  L->tot_solves++;
  // b = 0 gives x = 0 and a NaN or infinite b stops at once, as on the host
  cudaGraphSetConditional(h_outer, (isfinite(b) && b > 0.0) ? 1u : 0u);
}
__global__ void k_loop_arm(KrylovLoop* L, cudaGraphConditionalHandle h_inner) {
  L->j = 0;
  L->tot_cycles++;
  cudaGraphSetConditional(h_inner, 1u);
}
__global__ void k_loop_next(const ArnoldiState* __restrict__ st, KrylovLoop* L, cudaGraphConditionalHandle h_inner,
                            double tol, int m, int maxit) {
  const int j = L->j + 1, it = L->iters + 1;
  L->j = j;
  L->iters = it;
  L->tot_iters++;
  const double r = st->rel;
  L->rel = r;
  const bool fin = isfinite(r);
  if (!fin) {  // the host loop returns here without the update: a zero count skips it
    L->nonfinite = 1;
    L->j = 0;
  }
  const bool go = fin && !(r <= tol) && st->breakdown == 0 && j < m && it < maxit;
  cudaGraphSetConditional(h_inner, go ? 1u : 0u);
}
__global__ void k_loop_after(const ArnoldiState* __restrict__ st, KrylovLoop* L, cudaGraphConditionalHandle h_outer,
                             cudaGraphConditionalHandle h_restart, double tol, int maxit) {
  const int c = L->cycles + 1;
  L->cycles = c;
  const double r = st->rel;
  const bool fin = isfinite(r);
  const bool done = !fin || r <= tol || st->breakdown != 0 || L->iters >= maxit || c >= maxit;
  if (!done) L->tot_restarts++;
  cudaGraphSetConditional(h_outer, done ? 0u : 1u);
  cudaGraphSetConditional(h_restart, done ? 0u : 1u);
}

// the graph being recorded on a capturing stream
static cudaGraph_t capturing_graph(cudaStream_t cs) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  SCR_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive || !g) throw CudaError{cudaErrorStreamCaptureInvalidated, "capture"};
  return g;
}

static cudaGraphConditionalHandle make_handle(cudaGraph_t g) {
  cudaGraphConditionalHandle hnd = 0;
  SCR_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 0, cudaGraphCondAssignDefault));
  return hnd;
}

// appends a conditional node (WHILE or IF, condition hnd) after the work
// recorded so far on the capturing stream cs, records its body with body(bs)
// on the stream of the next nesting depth, and continues cs after the node
template <class F>
static void record_conditional(cudaStream_t cs, cudaGraphConditionalHandle hnd, cudaGraphConditionalNodeType type,
                               F&& body) {
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  SCR_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &nd));
  if (cst != cudaStreamCaptureStatusActive || !g) throw CudaError{cudaErrorStreamCaptureInvalidated, "capture"};
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  SCR_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  SCR_CUDA(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  if (g_capture_depth >= kMaxCaptureDepth) throw CudaError{cudaErrorStreamCaptureUnsupported, "capture depth"};
  cudaStream_t bs = g_capture_streams[g_capture_depth];
  SCR_CUDA(cudaStreamBeginCaptureToGraph(bs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
  ++g_capture_depth;
  try {
    body(bs);
  } catch (...) {
    --g_capture_depth;
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(bs, &tmp);
    throw;
  }
  --g_capture_depth;
  cudaGraph_t out = nullptr;
  SCR_CUDA(cudaStreamEndCapture(bs, &out));
}

// records rec(cs) on a private stream and instantiates it; null when the
// capture or the instantiation fails (the caller then runs eagerly)
template <class F>
static cudaGraphExec_t capture_exec(F&& rec) {
  for (int d = 0; d <= kMaxCaptureDepth; ++d)
    if (!g_capture_streams[d] && cudaStreamCreateWithFlags(&g_capture_streams[d], cudaStreamNonBlocking) != cudaSuccess) {
      g_capture_streams[d] = nullptr;
      cudaGetLastError();
      return nullptr;
    }
  cudaStream_t cs = g_capture_streams[kMaxCaptureDepth];
  const LaunchCounter c0 = counters();
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  bool ok = true;
  ++g_capture_depth;
  try {
    rec(cs);
  } catch (const CudaError&) {
    ok = false;
  } catch (const std::exception&) {
    ok = false;
  }
  --g_capture_depth;
  counters() = c0;  // nothing has run yet
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaGraphExec_t ex = nullptr;
  if (ok && e == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ex;
}

static LaunchCounter diff(const LaunchCounter& a, const LaunchCounter& b) {
  LaunchCounter d;
  d.launches = a.launches - b.launches;
  d.spmv_bytes = a.spmv_bytes - b.spmv_bytes;
  for (int i = 0; i < 3; ++i) d.vcycles[i] = a.vcycles[i] - b.vcycles[i];
  for (int i = 0; i < 2; ++i) d.fixed[i] = a.fixed[i] - b.fixed[i];
  return d;
}

// ------------------------------------------------------------ GMRES
template <typename T>
struct Gmres {
  int m = 0;
  long long n = 0;
  T *V = nullptr, *Z = nullptr, *w = nullptr;
  ArnoldiState* st = nullptr;
  HostScalars hs;
  int syncs = 0;
  // device loop (emit): the loop's counters, the preconditioner's input and
  // output in the recorded Arnoldi step, and the library launches / modelled
  // bytes of one prologue, Arnoldi step, cycle end and restart (nested
  // loops excluded: they count their own)
  KrylovLoop* L = nullptr;
  T *pin = nullptr, *pout = nullptr;
  LaunchCounter sec[4];
  bool recorded = false;

  void init(DeviceArena& a, long long n_, int m_) {
    n = n_;
    m = std::max(1, std::min(m_, kMaxBasis - 1));
    V = a.alloc<T>((size_t)(m + 1) * n + 1);
    Z = a.alloc<T>((size_t)m * n + 1);
    w = a.alloc<T>(n + 1);
    st = a.alloc<ArnoldiState>(1);
    L = a.alloc<KrylovLoop>(1);
    pin = a.alloc<T>(n + 1);
    pout = a.alloc<T>(n + 1);
    SCR_CUDA(cudaMemsetAsync(L, 0, sizeof(KrylovLoop), a.stream()));
    recorded = false;
  }

  using OpS = std::function<void(const T*, T*, cudaStream_t)>;

  // records the solve of op x = b (x0 = 0, restarted every m steps, to tol
  // or maxit steps) into the graph being captured on cs
  void emit(cudaStream_t cs, const OpS& op, const OpS& pc, const T* b, T* x, double tol, int maxit,
            const Reducer& red) {
    const LaunchCounter c0 = counters();
    fill<T>(x, (T)0, n, cs);
    norm2<T>(b, n, &st->nrm2, red, cs);
    arnoldi_start(st, 1, nullptr, cs);
    scale_by<T>(b, &st->inv_hnext, V, n, cs);
    const cudaGraphConditionalHandle h_outer = make_handle(capturing_graph(cs));
    k_loop_begin<<<1, 1, 0, cs>>>(st, L, h_outer);
    SCR_LAUNCH();
    counters().launches++;
    sec[0] = diff(counters(), c0);
    record_conditional(cs, h_outer, cudaGraphCondTypeWhile, [&](cudaStream_t os) {
      const LaunchCounter c1 = counters();
      const cudaGraph_t go = capturing_graph(os);
      const cudaGraphConditionalHandle h_inner = make_handle(go), h_restart = make_handle(go);
      k_loop_arm<<<1, 1, 0, os>>>(L, h_inner);
      SCR_LAUNCH();
      counters().launches++;
      const LaunchCounter arm = diff(counters(), c1);
      record_conditional(os, h_inner, cudaGraphCondTypeWhile, [&](cudaStream_t is) {
        const LaunchCounter c2 = counters();
        col_copy<T>(V, &L->j, pin, nullptr, 0, n, nullptr, n, is);
        pc(pin, pout, is);
        col_copy<T>(pout, nullptr, Z, &L->j, 0, n, nullptr, n, is);
        op(pout, w, is);
        multidot<T>(V, n, m, w, n, st->h1, red, is, &L->j, 1);
        cgs_update_dot<T>(V, n, m, st->h1, w, n, st->h2, red, is, &L->j, 1);
        cgs_update_norm<T>(V, n, m, st->h2, w, n, &st->nrm2, red, is, &L->j, 1);
        arnoldi_finalize(st, 0, nullptr, is, &L->j);
        col_copy<T>(w, nullptr, V, &L->j, 1, n, &st->inv_hnext, n, is);
        k_loop_next<<<1, 1, 0, is>>>(st, L, h_inner, tol, m, maxit);
        SCR_LAUNCH();
        counters().launches++;
        sec[1] = diff(counters(), c2);
      });
      const LaunchCounter c3 = counters();
      gmres_update<T>(st, m, Z, n, x, n, os, &L->j);
      k_loop_after<<<1, 1, 0, os>>>(st, L, h_outer, h_restart, tol, maxit);
      SCR_LAUNCH();
      counters().launches++;
      sec[2] = diff(counters(), c3);
      sec[2].launches += arm.launches;  // k_loop_arm: no V-cycle, no product
      record_conditional(os, h_restart, cudaGraphCondTypeIf, [&](cudaStream_t rs) {
        const LaunchCounter c4 = counters();
        op(x, w, rs);
        axpby_t<T>(1.0, b, -1.0, w, n, rs);
        norm2<T>(w, n, &st->nrm2, red, rs);
        arnoldi_start(st, 0, nullptr, rs);
        scale_by<T>(w, &st->inv_hnext, V, n, rs);
        sec[3] = diff(counters(), c4);
      });
    });
    counters() = c0;  // counted from the loop's own counters when read back
    recorded = true;
  }

  // counters of the device loops since the last reset_loop: adds their
  // library launches and modelled bytes to the process counters, their
  // V-cycles and fixed-count A-solve steps to acc, and returns the Arnoldi
  // steps run
  long long collect(cudaStream_t s, LaunchCounter& acc) {
    if (!L || !recorded) return 0;
    KrylovLoop hL{};
    SCR_CUDA(cudaMemcpyAsync(&hL, L, sizeof hL, cudaMemcpyDeviceToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    const long long c[4] = {hL.tot_solves, hL.tot_iters, hL.tot_cycles, hL.tot_restarts};
    for (int i = 0; i < 4; ++i) {
      counters().launches += c[i] * sec[i].launches;
      counters().spmv_bytes += c[i] * sec[i].spmv_bytes;
      for (int k = 0; k < 3; ++k) acc.vcycles[k] += c[i] * sec[i].vcycles[k];
      for (int k = 0; k < 2; ++k) acc.fixed[k] += c[i] * sec[i].fixed[k];
    }
    return hL.tot_iters;
  }
  void reset_loop(cudaStream_t s) {
    if (L && recorded) SCR_CUDA(cudaMemsetAsync(L, 0, sizeof(KrylovLoop), s));
  }

  using Op = std::function<void(const T*, T*)>;

  // returns true when converged; iters/rel report the work done
  bool solve(const Op& op, const Op* pc, const T* b, T* x, double tol, int maxit, const Reducer& red,
             cudaStream_t s, int* iters, double* rel, const std::function<double(const T*)>* true_rel = nullptr) {
    fill<T>(x, (T)0, n, s);
    norm2<T>(b, n, &st->nrm2, red, s);
    arnoldi_start(st, 1, hs.d, s);
    hs.fetch(s);
    SCR_CUDA(cudaStreamSynchronize(s));
    ++syncs;
    *iters = 0;
    *rel = 0.0;
    if (!std::isfinite(hs.h[1])) {  // a NaN or infinite right-hand side: x = 0, not converged
      *rel = hs.h[1];
      return false;
    }
    if (!(hs.h[1] > 0.0)) return true;  // b = 0 -> x = 0
    scale_by<T>(b, &st->inv_hnext, V, n, s);
    for (;;) {
      int k = 0;
      bool breakdown = false;
      double r = 1.0;
      for (int j = 0; j < m; ++j) {
        T* vj = V + (size_t)j * n;
        T* zj = Z + (size_t)j * n;
        if (pc) (*pc)(vj, zj);
        else copy<T>(vj, zj, n, s);
        op(zj, w);
        multidot<T>(V, n, j + 1, w, n, st->h1, red, s);
        cgs_update_dot<T>(V, n, j + 1, st->h1, w, n, st->h2, red, s);
        cgs_update_norm<T>(V, n, j + 1, st->h2, w, n, &st->nrm2, red, s);
        arnoldi_finalize(st, j, hs.d, s);
        scale_by<T>(w, &st->inv_hnext, V + (size_t)(j + 1) * n, n, s);
        hs.fetch(s);
        SCR_CUDA(cudaStreamSynchronize(s));
        ++syncs;
        r = hs.h[0];
        breakdown = hs.h[1] != 0.0;
        ++*iters;
        k = j + 1;
        if (!std::isfinite(r)) {
          *rel = r;
          return false;
        }
        if (r <= tol || *iters >= maxit || breakdown) break;
      }
      gmres_update<T>(st, k, Z, n, x, n, s);
      *rel = r;
      if (r <= tol || breakdown) {
        if (!true_rel) return r <= tol || breakdown;
        const double tr = (*true_rel)(x);
        *rel = tr;
        if (tr <= tol) return true;
        if (*iters >= maxit) return false;
      } else if (*iters >= maxit) {
        return false;
      }
      // restart from the current residual r = b - op(x)
      op(x, w);
      axpby_t<T>(1.0, b, -1.0, w, n, s);
      norm2<T>(w, n, &st->nrm2, red, s);
      arnoldi_start(st, 0, hs.d, s);
      scale_by<T>(w, &st->inv_hnext, V, n, s);
    }
  }
};

}  // namespace scr

using namespace scr;

// ------------------------------------------------------------ context
struct scr_ctx {
  scr_opts o;
  cudaStream_t s = nullptr;
  int device = 0;
  std::unique_ptr<DeviceArena> mats;   // A, B, C, D, Shat and their FP32 copies
  std::unique_ptr<DeviceArena> work;   // Krylov workspaces
  std::unique_ptr<DeviceArena> mwork;  // mesh workspaces
  std::unique_ptr<DeviceArena> mmats;
  DBsr<double> A, B, C, D, Shat, L;
  DBsr<double> Bs, CBs;  // diag(A)^{-1} B and C diag(A)^{-1} B of Shat's set-up (kept for scr_update_values)
  DBsr<float> Af, Bf, Cf, Df;
  DSell<double> A_sell, Shat_sell, L_sell;
  DSell<float> Af_sell, Shatf_sell;
  Hierarchy hA, hS, hM;
  Reducer red, mred;
  int nv = 0, np = 0, nm = 0;
  bool have_block = false, have_mesh = false;
  // outer (FP64) and preconditioner workspaces (FP64 or FP32)
  Gmres<double> gOuter;
  Gmres<double> gA, gS, gI;
  Gmres<float> gAf, gSf, gIf;
  double *bvec = nullptr, *xvec = nullptr, *rvec = nullptr;
  double *yhat = nullptr, *rp2 = nullptr, *rv2 = nullptr, *xbar = nullptr, *xt = nullptr;
  double* dAinv = nullptr;  // 1 / diag(A) (SIMPLE upper factor; SIMPLEC: 1 / sum_j |a_ij|)
  float* dAinvf = nullptr;
  float *pr = nullptr, *py = nullptr, *yhatf = nullptr, *rp2f = nullptr, *rv2f = nullptr, *xbarf = nullptr,
        *xtf = nullptr;
  double *rr = nullptr, *rt = nullptr;  // fixed-count A solves (inner_vcycles, inter_vcycles)
  float *rrf = nullptr, *rtf = nullptr;
  // mesh CG
  double *mb = nullptr, *mx = nullptr, *mr = nullptr, *mz = nullptr, *mp = nullptr, *mq = nullptr;
  CgState* cg = nullptr;
  HostScalars mhs;
  scr_stats stats;
  int counters_outer = 0;
  // interleaved right-hand sides of the block solve (options.nrhs): every
  // vector of the block path holds k of them, entry i of right-hand side c
  // at i * k + c, and every product acts as M (x) I_k
  int k = 1;
  double* mstage = nullptr;  // k vectors one after another (multi-right-hand-side staging)
  // resistance outlets (scr_set_outlets): A acts as A + sum_j c_j a_j a_j^T
  int n_out = 0;                    // outlets in effect (from the last scr_setup)
  std::vector<double> out_c;
  int pend_n = 0, pend_len = 0;     // set by scr_set_outlets, used by the next scr_setup
  std::vector<double> pend_a, pend_c;
  double* out_a = nullptr;    // device, n_out x 3 n_v
  float* out_af = nullptr;    // FP32 copy (mixed precision)
  double* out_dot = nullptr;  // device, n_out scratch dots
  // residual assembly (scr_assembly_setup)
  ResidualAssembler ra;
  std::unique_ptr<DeviceArena> rmats;
  // tangent assembly (scr_assemble_tangent): patterns of the block system
  // captured from the set-up it first ran after, and its own re-set-ups
  TangentAssembler ta;
  std::unique_ptr<DeviceArena> tmats;
  bool tangent_setup = false;  // scr_setup called by scr_assemble_tangent
  bool have_residual = false;
  std::vector<unsigned char> dir_v;  // velocity Dirichlet flag per node (empty: none)
  scr_physics phys{};
  double* r_in = nullptr;  // host-path staging: v, vhat, p, vdot, u, R
  unsigned char* d_dir = nullptr;  // device copy of dir_v
  // mesh motion inside the corrector (scr_mesh_coupling): the fluid nodes'
  // mesh Laplacian without boundary conditions, their node numbers, the
  // Dirichlet and interface flags, and the loop's vectors
  std::unique_ptr<DeviceArena> cmats;
  bool have_coupling = false;
  int cpl_nf = 0, cpl_nn = 0;
  DBsr<double> Lraw;
  int* d_node_of_f = nullptr;
  unsigned char *d_dir_m = nullptr, *d_follow = nullptr;
  double *d_g = nullptr, *d_lift = nullptr, *d_uh = nullptr, *d_uhn = nullptr, *d_vhn = nullptr;
  double *d_un = nullptr, *d_vhat = nullptr;
  // batched form: member sizes and offsets inside the union system
  int nbatch = 0;
  std::vector<int> b_nv, b_np, b_vo, b_po;
  std::vector<double> b_rel;
  double* b_norms = nullptr;  // device, 2 per member
  // the preconditioner application as one CUDA graph (option graph_krylov):
  // recorded from pc_r to pc_y at its first use after a set-up (epoch), with
  // every inner GMRES as a device loop; the library launches, modelled bytes
  // and A solves of its straight-line part, added at each replay
  long long graph_epoch = 0, pc_epoch = -1;
  bool pc_failed = false;
  GraphExecPtr pc_exec;
  double *pc_r = nullptr, *pc_y = nullptr;
  LaunchCounter pc_sec;
  int pc_a_solves = 0;
  scr_ctx() {
    hS.slot = 1;
    hM.slot = 2;
  }
};

namespace {

void check_bsr(const scr_bsr* M, int br, int bc, int nbr, int nbc, const char* name) {
  if (!M) throw std::invalid_argument(std::string(name) + ": NULL matrix");
  if (M->br != br || M->bc != bc)
    throw std::invalid_argument(std::string(name) + ": wrong block size");
  if (M->nb_rows != nbr || M->nb_cols != nbc) throw std::invalid_argument(std::string(name) + ": wrong shape");
  if (M->nb_rows < 0 || M->nnzb < 0) throw std::invalid_argument(std::string(name) + ": negative size");
  if (!M->row_ptr || (M->nnzb > 0 && (!M->col_idx || !M->val)))
    throw std::invalid_argument(std::string(name) + ": NULL array");
}

__global__ void k_check_cols(int nbr, int nbc, const int* __restrict__ rp, const int* __restrict__ col,
                             long long nnzb, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  const int s = rp[i], e = rp[i + 1];
  if (s < 0 || e < s || e > nnzb) {
    atomicExch(bad, 1);
    return;
  }
  for (int t = s; t < e; ++t) {
    const int c = col[t];
    if (c < 0 || c >= nbc || (t > s && col[t - 1] >= c)) atomicExch(bad, 1);
  }
}


// copy a caller matrix to the device in slab layout (FP64)
DBsr<double> upload(const scr_bsr* M, int dev_ptr, DeviceArena& a, cudaStream_t s) {
  DBsr<double> D;
  D.nbr = M->nb_rows;
  D.nbc = M->nb_cols;
  D.br = M->br;
  D.bc = M->bc;
  D.nnzb = M->nnzb;
  const size_t nv = (size_t)M->nnzb * M->br * M->bc;
  D.rp = a.alloc<int>(M->nb_rows + 1);
  D.col = a.alloc<int>(M->nnzb + 1);
  D.val = a.alloc<double>(nv + 1);
  const cudaMemcpyKind k = dev_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  SCR_CUDA(cudaMemcpyAsync(D.rp, M->row_ptr, sizeof(int) * (M->nb_rows + 1), k, s));
  if (M->nnzb > 0) SCR_CUDA(cudaMemcpyAsync(D.col, M->col_idx, sizeof(int) * M->nnzb, k, s));
  DeviceArena tmp(s);
  // validate the index arrays before any kernel indexes with them
  int* bad = tmp.alloc<int>(1);
  SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (D.nbr > 0) {
    k_check_cols<<<ceil_div(D.nbr, 256), 256, 0, s>>>(D.nbr, D.nbc, D.rp, D.col, D.nnzb, bad);
    SCR_LAUNCH();
  }
  int hb = 0;
  SCR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  if (hb) throw std::invalid_argument("row_ptr/col_idx invalid (range, order or duplicates)");
  const double* src = M->val;
  if (!dev_ptr && nv > 0) {
    double* t = tmp.alloc<double>(nv);
    SCR_CUDA(cudaMemcpyAsync(t, M->val, sizeof(double) * nv, k, s));
    src = t;
  }
  if (nv > 0) to_slab<double>(D.rp, src, D.val, D.nbr, D.br, D.bc, D.nnzb, s);
  SCR_CUDA(cudaStreamSynchronize(s));
  return D;
}

DBsr<float> float_copy(const DBsr<double>& M, DeviceArena& a, cudaStream_t s) {
  DBsr<float> F;
  F.nbr = M.nbr;
  F.nbc = M.nbc;
  F.br = M.br;
  F.bc = M.bc;
  F.nnzb = M.nnzb;
  F.rp = M.rp;
  F.col = M.col;
  F.val = a.alloc<float>(M.nnzb * M.br * M.bc + 1);
  slab_to_float(M.val, F.val, M.nnzb * M.br * M.bc, s);
  return F;
}

template <typename F>
int guarded(F&& f) {
  try {
    f();
    return SCR_OK;
  } catch (const CudaError& e) {
    set_last_error("CUDA error %s in %s", cudaGetErrorString(e.err), e.where ? e.where : "?");
    cudaGetLastError();
    return e.err == cudaErrorInvalidValue ? SCR_INVALID_ARG : SCR_CUDA_ERROR;
  } catch (const std::invalid_argument& e) {
    set_last_error("%s", e.what());
    return SCR_INVALID_ARG;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return SCR_CUDA_ERROR;
  } catch (const std::exception& e) {
    set_last_error("%s", e.what());
    return SCR_CUDA_ERROR;
  }
}

// ---- the operators of the path, in precision T ----
template <typename T>
struct PcView {
  const DBsr<T>*A, *B, *C, *D, *Shat;
  Hierarchy *hA, *hS;
  Gmres<T>*gA, *gS, *gI;
  T *yhat, *rp2, *rv2, *xbar, *xt;
  T *rr, *rt;  // fixed-count A solves: residual and correction
  const T* dAinv;
  const T* out_a;  // outlet vectors in this precision (n_out x 3 n_v) or null
};

PcView<double> view64(scr_ctx* h) {
  return PcView<double>{&h->A, &h->B, &h->C, &h->D, &h->Shat, &h->hA, &h->hS, &h->gA, &h->gS, &h->gI,
                        h->yhat, h->rp2, h->rv2, h->xbar, h->xt, h->rr, h->rt, h->dAinv, h->out_a};
}
PcView<float> view32(scr_ctx* h) {
  return PcView<float>{&h->Af, &h->Bf, &h->Cf, &h->Df, &h->hS.lv[0].Af, &h->hA, &h->hS, &h->gAf, &h->gSf, &h->gIf,
                       h->yhatf, h->rp2f, h->rv2f, h->xbarf, h->xtf, h->rrf, h->rtf, h->dAinvf, h->out_af};
}

// runs the context's launches on another stream for its lifetime (the
// stream a Krylov-loop capture records on)
struct StreamSwap {
  scr_ctx* h;
  cudaStream_t old;
  StreamSwap(scr_ctx* h_, cudaStream_t s) : h(h_), old(h_->s) { h->s = s; }
  ~StreamSwap() { h->s = old; }
  StreamSwap(const StreamSwap&) = delete;
  StreamSwap& operator=(const StreamSwap&) = delete;
};

// one GMRES solve of the path: recorded as a device loop when a Krylov-loop
// capture is in progress (returns 0: its steps are counted on the device),
// else the host-driven loop (returns its steps)
template <typename T>
int gmres_run(scr_ctx* h, Gmres<T>* g, const typename Gmres<T>::OpS& op, const typename Gmres<T>::OpS& pc,
              const T* b, T* x, double tol, int maxit) {
  if (g_capture_depth > 0) {
    g->emit(h->s, op, pc, b, x, tol, maxit, h->red);
    return 0;
  }
  cudaStream_t s = h->s;
  typename Gmres<T>::Op o = [&](const T* a, T* y) { op(a, y, s); };
  typename Gmres<T>::Op p = [&](const T* a, T* y) { pc(a, y, s); };
  int it = 0;
  double rel = 0;
  g->solve(o, &p, b, x, tol, maxit, h->red, s, &it, &rel);
  return it;
}

// y += sign * sum_j c_j a_j (a_j^T x) on the velocity rows (the outlets'
// rank-1 terms of the momentum block; one dot and one update per outlet)
template <typename T>
void outlet_terms(scr_ctx* h, const T* a, const T* x, T* y, double sign) {
  const long long nv3 = 3LL * h->nv;
  for (int j = 0; j < h->n_out; ++j) {
    multidot<T>(a + j * nv3, 0, 1, x, nv3, h->out_dot + j, h->red, h->s);
    axpy_dev<T>(a + j * nv3, h->out_dot + j, sign * h->out_c[j], y, nv3, h->s);
  }
}

// the momentum block's action: y = A x (+ the outlet terms)
template <typename T>
void apply_A(scr_ctx* h, PcView<T>& v, const T* x, T* y) {
  spmv<T, T>(*v.A, x, y, h->k, EpiArgs(), h->s);
  if (h->n_out) outlet_terms<T>(h, v.out_a, x, y, 1.0);
}

// y = calA x, or y = z - calA x (resid), with the outlet terms, in FP64
void apply_calA(scr_ctx* h, const double* x, double* y, const double* z, bool resid) {
  block_op(h->A, h->B, h->C, h->D, x, y, z, resid, h->s, h->k);
  if (h->n_out) outlet_terms<double>(h, h->out_a, x, y, resid ? -1.0 : 1.0);
}

// A^{-1} b approximated by k steps of Richardson's iteration preconditioned
// by one V-cycle M, from x = 0: x_1 = M b, x_{i+1} = x_i + M (b - A x_i).
// A fixed linear operator (the same for every b) without host
// synchronisation; it replaces GMRES to a tolerance when the options ask for
// a fixed count (the outer FGMRES is flexible, and a fixed linear inner
// solve keeps the S operator of Algorithm 2 linear for the GMRES on S).
template <typename T>
void richardson_A(scr_ctx* h, PcView<T>& v, int k, const T* b, T* x) {
  cudaStream_t s = h->s;
  const long long n = 3LL * h->nv * h->k;
  v.hA->template apply<T>(b, x, s);
  for (int i = 1; i < k; ++i) {
    if (h->n_out) {
      apply_A<T>(h, v, x, v.rr);
      axpby_t<T>(1.0, b, -1.0, v.rr, n, s);
    } else {
      EpiArgs res;
      res.kind = Epi::Resid;
      res.z = b;
      spmv<T, T>(*v.A, x, v.rr, h->k, res, s);
    }
    v.hA->template apply<T>(v.rr, v.rt, s);
    axpby_t<T>(1.0, v.rt, 1.0, x, n, s);
  }
}

// an intermediate or inner A solve: GMRES + P_A to rtol (the paper), or k
// fixed V-cycle Richardson steps when k > 0; returns the iterations
template <typename T>
int solve_A(scr_ctx* h, PcView<T>& v, Gmres<T>* g, int k, double rtol, int maxit, const T* b, T* x) {
  if (k > 0) {
    richardson_A<T>(h, v, k, b, x);
    if (g_capture_depth > 0) {  // recorded: counted at each replay
      counters().fixed[g == v.gI ? 1 : 0] += k;
      return 0;
    }
    return k;
  }
  typename Gmres<T>::OpS opA = [&](const T* xx, T* y, cudaStream_t cs) {
    StreamSwap sw(h, cs);
    apply_A<T>(h, v, xx, y);
  };
  typename Gmres<T>::OpS pcA = [&](const T* bb, T* xx, cudaStream_t cs) { v.hA->template apply<T>(bb, xx, cs); };
  return gmres_run<T>(h, g, opA, pcA, b, x, rtol, maxit);
}

// Algorithm 2: y_p = D x_p - C A^{-1} (B x_p), A^{-1} by inner GMRES + P_I
// (or the fixed-count solve); D x_p - C x_t in one pass
template <typename T>
void apply_S(scr_ctx* h, PcView<T>& v, const T* xp, T* yp) {
  cudaStream_t s = h->s;
  spmv<T, T>(*v.B, xp, v.xbar, h->k, EpiArgs(), s);
  h->stats.i_iters += solve_A<T>(h, v, v.gI, h->o.inner_vcycles, h->o.rtol_I, h->o.max_I, v.xbar, v.xt);
  schur_combine<T>(*v.C, *v.D, v.xt, xp, yp, h->k, s);
}

// Algorithm 1: y = P_SCR^{-1} r
template <typename T>
void apply_pc(scr_ctx* h, PcView<T>& v, const T* r, T* y) {
  cudaStream_t s = h->s;
  const long long nv3 = 3LL * h->nv * h->k;
  const T* rv = r;
  const T* rp = r + nv3;
  T* yv = y;
  T* yp = y + nv3;
  typename Gmres<T>::OpS opS = [&](const T* x, T* o, cudaStream_t cs) {
    StreamSwap sw(h, cs);
    apply_S<T>(h, v, x, o);
  };
  typename Gmres<T>::OpS pcS = [&](const T* b, T* x, cudaStream_t cs) { v.hS->template apply<T>(b, x, cs); };
  const int kA = h->o.inter_vcycles;
  // 1. A yhat_v = r_v
  h->stats.a_iters += solve_A<T>(h, v, v.gA, kA, h->o.rtol_A, h->o.max_A, rv, v.yhat);
  h->stats.a_solves++;
  // 2. r_p <- r_p - C yhat_v
  EpiArgs e;
  e.kind = Epi::Axpby;
  e.alpha = -1.0;
  e.beta = 1.0;
  e.z = rp;
  spmv<T, T>(*v.C, v.yhat, v.rp2, h->k, e, s);
  // 3. S y_p = r_p
  h->stats.s_iters += gmres_run<T>(h, v.gS, opS, pcS, v.rp2, yp, h->o.rtol_S, h->o.max_S);
  // 4. r_v <- r_v - B y_p
  e.z = rv;
  spmv<T, T>(*v.B, yp, v.rv2, h->k, e, s);
  // 5. A y_v = r_v
  h->stats.a_iters += solve_A<T>(h, v, v.gA, kA, h->o.rtol_A, h->o.max_A, v.rv2, yv);
  h->stats.a_solves++;
}

// P_SIMPLE^{-1} r = U_SIMPLE^{-1} diag(A, Shat)^{-1} L^{-1} r (Sec. 5.2.1):
//   yhat_v = A^{-1} r_v (GMRES + P_A), y_p = Shat^{-1} (r_p - C yhat_v)
//   (GMRES + P_S on the explicit Shat, no inner level),
//   y_v = yhat_v - diag(A)^{-1} B y_p
template <typename T>
void apply_simple(scr_ctx* h, PcView<T>& v, const T* r, T* y) {
  cudaStream_t s = h->s;
  const long long nv3 = 3LL * h->nv * h->k;
  const T* rv = r;
  const T* rp = r + nv3;
  T* yv = y;
  T* yp = y + nv3;
  typename Gmres<T>::OpS opS = [&](const T* x, T* o, cudaStream_t cs) {
    spmv<T, T>(*v.Shat, x, o, h->k, EpiArgs(), cs);
  };
  typename Gmres<T>::OpS pcS = [&](const T* b, T* x, cudaStream_t cs) { v.hS->template apply<T>(b, x, cs); };
  h->stats.a_iters += solve_A<T>(h, v, v.gA, h->o.inter_vcycles, h->o.rtol_A, h->o.max_A, rv, v.yhat);
  h->stats.a_solves++;
  EpiArgs e;
  e.kind = Epi::Axpby;
  e.alpha = -1.0;
  e.beta = 1.0;
  e.z = rp;
  spmv<T, T>(*v.C, v.yhat, v.rp2, h->k, e, s);
  h->stats.s_iters += gmres_run<T>(h, v.gS, opS, pcS, v.rp2, yp, h->o.rtol_S, h->o.max_S);
  EpiArgs u;
  u.kind = Epi::ScaledSub;
  u.z = v.yhat;
  u.dinv = v.dAinv;
  spmv<T, T>(*v.B, yp, yv, h->k, u, s);
}

void apply_pc_direct(scr_ctx* h, const double* r, double* y) {
  const bool simple = h->o.precond == SCR_PC_SIMPLE || h->o.precond == SCR_PC_SIMPLEC;
  if (h->o.precision == SCR_MIXED) {
    const long long n = (3LL * h->nv + h->np) * h->k;
    cast_d2f(r, h->pr, n, h->s);
    PcView<float> v = view32(h);
    if (simple) apply_simple<float>(h, v, h->pr, h->py);
    else apply_pc<float>(h, v, h->pr, h->py);
    cast_f2d(h->py, y, n, h->s);
  } else {
    PcView<double> v = view64(h);
    if (simple) apply_simple<double>(h, v, r, y);
    else apply_pc<double>(h, v, r, y);
  }
}

// Largest block system (unknowns times right-hand sides) that graph_krylov
// = 2 runs with device loops.  Measured on one GB300 (set-up + solve, FP64 /
// mixed): 24,764 unknowns 57 -> 53 ms / 47 -> 42 ms and 16 members of the
// batch one after another 15.7 -> 15.1 s / 8.7 -> 7.8 s with device loops,
// 2,503,844 unknowns 1037 -> 1042 ms / 581 -> 589 ms: where each inner step
// takes milliseconds of GPU work the host waits cost less than the
// conditional nodes' relaunch of their bodies.
constexpr long long kDeviceLoopMaxUnknowns = 1000000;

// y = P^{-1} r (SCR, SIMPLE or SIMPLEC in the handle's precision).  With
// device loops (graph_krylov) the application is recorded once per set-up as
// a CUDA graph from pc_r to pc_y, every inner GMRES a device loop, and
// replayed between two copies; the library profiler, or a failed capture,
// runs it directly.
void apply_pc_any(scr_ctx* h, const double* r, double* y) {
  const long long n_all = (3LL * h->nv + h->np) * h->k;
  const bool loops = h->o.graph_krylov == 1 || (h->o.graph_krylov == 2 && n_all <= kDeviceLoopMaxUnknowns);
  if (loops && !profiler().active && h->pc_r) {
    if (h->pc_epoch != h->graph_epoch) {
      h->pc_epoch = h->graph_epoch;
      h->pc_exec.reset();
      h->pc_failed = false;
    }
    if (!h->pc_exec && !h->pc_failed) {
      const int a0 = h->stats.a_solves;
      LaunchCounter sec;
      cudaGraphExec_t ex = capture_exec([&](cudaStream_t cs) {
        StreamSwap sw(h, cs);
        const LaunchCounter c0 = counters();
        apply_pc_direct(h, h->pc_r, h->pc_y);
        sec = diff(counters(), c0);
      });
      h->pc_a_solves = h->stats.a_solves - a0;
      h->stats.a_solves = a0;
      h->pc_sec = sec;
      if (ex) h->pc_exec.reset(ex);
      else h->pc_failed = true;
    }
    if (h->pc_exec) {
      const long long n = (3LL * h->nv + h->np) * h->k;
      copy<double>(r, h->pc_r, n, h->s);
      SCR_CUDA(cudaGraphLaunch(h->pc_exec.get(), h->s));
      copy<double>(h->pc_y, y, n, h->s);
      counters().launches += h->pc_sec.launches;
      counters().spmv_bytes += h->pc_sec.spmv_bytes;
      h->hA.vcycles += (int)h->pc_sec.vcycles[0];
      h->hS.vcycles += (int)h->pc_sec.vcycles[1];
      h->stats.a_iters += (int)h->pc_sec.fixed[0];
      h->stats.i_iters += (int)h->pc_sec.fixed[1];
      h->stats.a_solves += h->pc_a_solves;
      h->stats.pc_graph_runs++;
      return;
    }
  }
  apply_pc_direct(h, r, y);
}

// adds the steps of the inner GMRES device loops run since the last
// reset_solve_stats to the solve counters (one read-back per loop)
void collect_loops(scr_ctx* h) {
  LaunchCounter acc;
  const long long a = h->gA.collect(h->s, acc) + h->gAf.collect(h->s, acc);
  const long long sI = h->gS.collect(h->s, acc) + h->gSf.collect(h->s, acc);
  const long long in = h->gI.collect(h->s, acc) + h->gIf.collect(h->s, acc);
  h->stats.a_iters += (int)(a + acc.fixed[0]);
  h->stats.s_iters += (int)sI;
  h->stats.i_iters += (int)(in + acc.fixed[1]);
  h->hA.vcycles += (int)acc.vcycles[0];
  h->hS.vcycles += (int)acc.vcycles[1];
}

double true_rel_block(scr_ctx* h, const double* b, const double* x) {
  const long long n = (3LL * h->nv + h->np) * h->k;
  apply_calA(h, x, h->rvec, b, true);
  ArnoldiState* st = h->gOuter.st;
  norm2<double>(h->rvec, n, &st->nrm2, h->red, h->s);
  double r2 = 0, b2 = 0;
  SCR_CUDA(cudaMemcpyAsync(&r2, &st->nrm2, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  norm2<double>(b, n, &st->nrm2, h->red, h->s);
  SCR_CUDA(cudaMemcpyAsync(&b2, &st->nrm2, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  SCR_CUDA(cudaStreamSynchronize(h->s));
  return b2 > 0 ? std::sqrt(r2 / b2) : std::sqrt(r2);
}

}  // namespace

// ------------------------------------------------------------ C ABI
extern "C" {

const char* scr_last_error(void) { return g_last_error.c_str(); }

int scr_default_opts(scr_opts* o) {
  if (!o) return SCR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  o->rtol = 1e-8;
  o->max_it = 200;
  o->restart = 30;
  o->rtol_A = o->rtol_S = o->rtol_I = 1e-3;
  o->max_A = o->max_S = o->max_I = 200;
  o->restart_inner = 30;
  o->precision = SCR_FP64;
  o->precond = 0;
  o->amg_theta = 0.08;
  o->amg_max_levels = 10;
  o->amg_coarse_size = 64;
  o->amg_nu = 1;
  o->amg_trunc = 0.3;
  o->amg_pmax = 5;
  o->autotune = 1;
  o->amg_smoother = SCR_SMOOTH_CHEB;
  o->amg_degree = 3;
  o->sell = 0;
  o->vec = 1;
  o->inner_vcycles = 0;
  o->inter_vcycles = 0;
  o->newton = 0;
  o->pdl = 1;
  o->tangent_resetup = 1;
  o->mapped_scalars = 1;
  o->l2_prefetch = 192;
  o->amg_coarse_bf16 = 1;
  o->cuda_graphs = 1;
  o->graph_krylov = 2;
  o->nrhs = 1;
  o->mm_rtol = 1e-8;
  o->mm_max_it = 500;
  o->verbose = 0;
  return SCR_OK;
}

int scr_create(scr_handle* out, const scr_opts* o, void* stream) {
  if (!out) {
    set_last_error("scr_create: NULL handle pointer");
    return SCR_INVALID_ARG;
  }
  *out = nullptr;
  return guarded([&] {
    scr_opts def;
    scr_default_opts(&def);
    const scr_opts& op = o ? *o : def;
    if (op.restart < 1 || op.restart >= kMaxBasis || op.restart_inner < 1 || op.restart_inner >= kMaxBasis)
      throw std::invalid_argument("restart lengths must lie in [1, 63]");
    if (op.precision != SCR_FP64 && op.precision != SCR_MIXED) throw std::invalid_argument("unknown precision");
    if (op.precond != SCR_PC_SCR && op.precond != SCR_PC_SIMPLE && op.precond != SCR_PC_SIMPLEC)
      throw std::invalid_argument("unknown preconditioner");
    if (op.amg_smoother != SCR_SMOOTH_L1 && op.amg_smoother != SCR_SMOOTH_CHEB)
      throw std::invalid_argument("unknown smoother");
    if (op.amg_degree < 1 || op.amg_degree > 16) throw std::invalid_argument("Chebyshev degree must lie in [1, 16]");
    if (op.l2_prefetch < 0) throw std::invalid_argument("l2_prefetch must be >= 0");
    if (op.vec != 0 && op.vec != 1) throw std::invalid_argument("vec must be 0 or 1");
    if (op.graph_krylov < 0 || op.graph_krylov > 2) throw std::invalid_argument("graph_krylov must be 0, 1 or 2");
    if (op.inner_vcycles < 0 || op.inner_vcycles > 64 || op.inter_vcycles < 0 || op.inter_vcycles > 64)
      throw std::invalid_argument("inner_vcycles and inter_vcycles must lie in [0, 64]");
    if (op.newton != 0 && op.newton != 1) throw std::invalid_argument("newton must be 0 or 1");
    if (op.pdl != 0 && op.pdl != 1) throw std::invalid_argument("pdl must be 0 or 1");
    if (op.tangent_resetup != 0 && op.tangent_resetup != 1)
      throw std::invalid_argument("tangent_resetup must be 0 or 1");
    if (op.nrhs != 1 && op.nrhs != kSpmmCols) throw std::invalid_argument("nrhs must be 1 or 8");
    if (op.amg_coarse_bf16 != 0 && op.amg_coarse_bf16 != 1) throw std::invalid_argument("amg_coarse_bf16 must be 0 or 1");
    if (op.mapped_scalars != 0 && op.mapped_scalars != 1) throw std::invalid_argument("mapped_scalars must be 0 or 1");
    g_mapped_scalars = op.mapped_scalars;
    std::unique_ptr<scr_ctx> h(new scr_ctx());
    h->o = op;
    set_forced_group(op.spmv_group);
    set_l2_prefetch(op.l2_prefetch);
    set_pdl(op.pdl);
    set_tune_verbose(op.verbose);
    h->s = static_cast<cudaStream_t>(stream);
    SCR_CUDA(cudaGetDevice(&h->device));
    configure_pool(h->device);
    h->work.reset(new DeviceArena(h->s));
    h->mwork.reset(new DeviceArena(h->s));
    h->red = make_reducer(*h->work);
    h->mred = make_reducer(*h->mwork);
    memset(&h->stats, 0, sizeof(h->stats));
    *out = h.release();
  });
}

int scr_destroy(scr_handle h) {
  if (!h) return SCR_OK;
  return guarded([&] {
    cudaStreamSynchronize(h->s);
    delete h;
  });
}

namespace {
// flag when the caller's pattern (rp, col) differs from the stored one
__global__ void k_pattern_differs(int nbr, long long nnzb, const int* __restrict__ rp, const int* __restrict__ col,
                                  const int* __restrict__ rp0, const int* __restrict__ col0, int* __restrict__ diff) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t <= nbr && rp[t] != rp0[t]) atomicExch(diff, 1);
  if (t < nnzb && col[t] != col0[t]) atomicExch(diff, 1);
}

// new values of a stored matrix with an unchanged pattern: checks the
// pattern against the stored one (SCR_INVALID_ARG when it differs) and
// writes the values into the stored slab array
void update_values(const scr_bsr* M, DBsr<double>& D, int dev, cudaStream_t s, const char* name) {
  if (M->nb_rows != D.nbr || M->nb_cols != D.nbc || M->br != D.br || M->bc != D.bc || M->nnzb != D.nnzb)
    throw std::invalid_argument(std::string(name) + ": sizes differ from the set-up's; call scr_setup");
  DeviceArena tmp(s);
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int* rp = M->row_ptr;
  const int* col = M->col_idx;
  const double* val = M->val;
  const size_t nv = (size_t)M->nnzb * M->br * M->bc;
  if (!dev) {
    int* r = tmp.alloc<int>(M->nb_rows + 1);
    int* c = tmp.alloc<int>(M->nnzb + 1);
    double* v = tmp.alloc<double>(nv + 1);
    SCR_CUDA(cudaMemcpyAsync(r, M->row_ptr, sizeof(int) * (M->nb_rows + 1), k, s));
    if (M->nnzb) SCR_CUDA(cudaMemcpyAsync(c, M->col_idx, sizeof(int) * M->nnzb, k, s));
    if (nv) SCR_CUDA(cudaMemcpyAsync(v, M->val, sizeof(double) * nv, k, s));
    rp = r;
    col = c;
    val = v;
  }
  int* diff = tmp.alloc<int>(1);
  SCR_CUDA(cudaMemsetAsync(diff, 0, sizeof(int), s));
  const long long n = std::max<long long>(M->nb_rows + 1, M->nnzb);
  k_pattern_differs<<<ceil_div(n, 256), 256, 0, s>>>(M->nb_rows, M->nnzb, rp, col, D.rp, D.col, diff);
  SCR_LAUNCH();
  int hd = 0;
  SCR_CUDA(cudaMemcpyAsync(&hd, diff, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  if (hd) throw std::invalid_argument(std::string(name) + ": pattern differs from the set-up's; call scr_setup");
  if (nv) to_slab<double>(D.rp, val, D.val, D.nbr, D.br, D.bc, D.nnzb, s);
  SCR_CUDA(cudaStreamSynchronize(s));
}
}  // namespace

int scr_update_values(scr_handle h, const scr_bsr* A, const scr_bsr* B, const scr_bsr* C, const scr_bsr* D,
                      int dev) {
  if (!h || !A || !B || !C || !D) return SCR_INVALID_ARG;
  if (!h->have_block || h->nbatch) {
    set_last_error("scr_update_values: needs a block set-up (scr_setup, not batched)");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    auto t0 = Clock::now();
    cudaStream_t s = h->s;
    SCR_CUDA(cudaStreamSynchronize(s));
    update_values(A, h->A, dev, s, "A");
    update_values(B, h->B, dev, s, "B");
    update_values(C, h->C, dev, s, "C");
    update_values(D, h->D, dev, s, "D");
    const int nv = h->nv;
    {
      // Shat = D - C diag(A)^{-1} B on its stored patterns (Sec. 5.2.1)
      DeviceArena tmp(s);
      double* d = tmp.alloc<double>(3LL * nv + 1);
      int* bad = tmp.alloc<int>(1);
      SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      diag_scalar(h->A, d, bad, s);
      int hb = 0;
      SCR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      if (hb) throw std::invalid_argument("A has a missing or zero diagonal entry");
      if (h->o.precond == SCR_PC_SIMPLEC) abs_rowsum(h->A, d, s);
      for (int j = 0; j < h->n_out; ++j) add_scaled_squares(d, h->out_a + 3LL * nv * j, h->out_c[j], 3LL * nv, s);
      if (h->n_out) reciprocal(d, h->dAinv, 3LL * nv, s);
      scale_rows_inv_values(h->B, d, h->Bs.val, s);
      spgemm_numeric(h->C, h->Bs, h->CBs, s);
      spadd_numeric(h->D, 1.0, h->CBs, nullptr, h->Shat, s);
      SCR_CUDA(cudaStreamSynchronize(s));
    }
    if (!h->n_out) {
      if (h->o.precond == SCR_PC_SIMPLEC) l1_inv(h->A, h->dAinv, s);
      else inv_diag(h->A, h->dAinv, s);
    }
    refresh_vec<double>(h->A, s);
    refresh_vec<double>(h->Shat, s);
    const bool f32 = h->o.precision == SCR_MIXED;
    if (f32) {
      slab_to_float(h->A.val, h->Af.val, h->A.nnzb * 9, s);
      slab_to_float(h->B.val, h->Bf.val, h->B.nnzb * 3, s);
      slab_to_float(h->C.val, h->Cf.val, h->C.nnzb * 3, s);
      slab_to_float(h->D.val, h->Df.val, h->D.nnzb, s);
      refresh_vec<float>(h->Af, s);
      cast_d2f(h->dAinv, h->dAinvf, 3LL * nv, s);
    }
    h->hA.refresh(h->A, h->o, s, f32 ? &h->Af : nullptr);
    h->hS.refresh(h->Shat, h->o, s);
    h->graph_epoch++;
    SCR_CUDA(cudaStreamSynchronize(s));
    h->stats.setup_ms = ms_since(t0);
  });
}

int scr_setup(scr_handle h, const scr_bsr* A, const scr_bsr* B, const scr_bsr* C, const scr_bsr* D, int dev) {
  if (!h) return SCR_INVALID_ARG;
  return guarded([&] {
    auto t0 = Clock::now();
    if (!A || !D) throw std::invalid_argument("NULL matrix");
    const int nv = A->nb_rows;
    const int np = D->nb_rows;
    check_bsr(A, 3, 3, nv, nv, "A");
    check_bsr(B, 3, 1, nv, np, "B");
    check_bsr(C, 1, 3, np, nv, "C");
    check_bsr(D, 1, 1, np, np, "D");
    cudaStream_t s = h->s;
    SCR_CUDA(cudaStreamSynchronize(s));
    h->have_block = false;
    h->nbatch = 0;
    if (!h->tangent_setup) h->ta.ready = false;  // new matrices: a new pattern for the tangent
    h->hA = Hierarchy();
    h->hS = Hierarchy();
    h->hS.slot = 1;
    h->work.reset();
    h->mats.reset(new DeviceArena(s));
    DeviceArena& a = *h->mats;
    h->nv = nv;
    h->np = np;
    h->k = h->o.nrhs;
    h->mstage = nullptr;
    h->n_out = 0;
    h->out_a = nullptr;
    h->out_af = nullptr;
    if (h->pend_n) {
      if (h->pend_len != 3 * nv) throw std::invalid_argument("outlet vectors must have 3 n_v entries");
      if (h->k != 1) throw std::invalid_argument("outlet terms take one right-hand side (nrhs = 1)");
      if (h->o.precond == SCR_PC_SIMPLEC) throw std::invalid_argument("SIMPLEC with outlet terms is not supported");
    }
    h->A = upload(A, dev, a, s);
    if (h->pend_n) {
      const long long len = (long long)h->pend_n * 3 * nv;
      h->out_a = a.alloc<double>(len + 1);
      SCR_CUDA(cudaMemcpyAsync(h->out_a, h->pend_a.data(), sizeof(double) * len, cudaMemcpyHostToDevice, s));
      h->out_dot = a.alloc<double>(h->pend_n);
      h->out_c = h->pend_c;
      h->n_out = h->pend_n;
    }
    h->B = upload(B, dev, a, s);
    h->C = upload(C, dev, a, s);
    h->D = upload(D, dev, a, s);
    if (h->o.verbose) fprintf(stderr, "[setup] upload %.2f ms\n", ms_since(t0));
    auto t1 = Clock::now();
    // Shat = D - C diag(A)^{-1} B  (Sec. 5.2.1)
    {
      DeviceArena tmp(s);
      double* d = tmp.alloc<double>(3LL * nv + 1);
      int* bad = tmp.alloc<int>(1);
      SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      diag_scalar(h->A, d, bad, s);
      int hb = 0;
      SCR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      if (hb) throw std::invalid_argument("A has a missing or zero diagonal entry");
      // SIMPLEC: the diagonal lumped from the absolute values of A's entries
      if (h->o.precond == SCR_PC_SIMPLEC) abs_rowsum(h->A, d, s);
      // outlets: diag(A + sum_j c_j a_j a_j^T) = diag(A) + sum_j c_j a_j .* a_j
      for (int j = 0; j < h->n_out; ++j) add_scaled_squares(d, h->out_a + 3LL * nv * j, h->out_c[j], 3LL * nv, s);
      if (h->n_out) {
        h->dAinv = a.alloc<double>(3LL * nv + 1);
        reciprocal(d, h->dAinv, 3LL * nv, s);
      }
      scale_rows_inv(h->B, d, h->Bs, a, s);
      spgemm(h->C, h->Bs, h->CBs, a, s);
      spadd(h->D, 1.0, h->CBs, nullptr, h->Shat, a, s);
      SCR_CUDA(cudaStreamSynchronize(s));
    }
    if (h->o.verbose) fprintf(stderr, "[setup] Shat %.2f ms (%lld entries)\n", ms_since(t1), h->Shat.nnzb);
    if (!h->n_out) {
      h->dAinv = a.alloc<double>(3LL * nv + 1);
      if (h->o.precond == SCR_PC_SIMPLEC) l1_inv(h->A, h->dAinv, s);  // 1 / sum_j |a_ij|
      else inv_diag(h->A, h->dAinv, s);
    }
    const bool f32 = h->o.precision == SCR_MIXED;
    if (h->o.sell) {
      build_sell<double>(h->A, h->A_sell, a, s, h->o.sell);
      h->A.sell = &h->A_sell;
      build_sell<double>(h->Shat, h->Shat_sell, a, s, h->o.sell);
      h->Shat.sell = &h->Shat_sell;
    }
    if (h->o.vec) {
      build_vec<double>(h->A, a, s);
      build_vec<double>(h->Shat, a, s);
    }
    tune_product<double>(h->A, 1, h->o, a, s);
    tune_product<double>(h->Shat, 1, h->o, a, s);
    if (f32) {
      h->Af = float_copy(h->A, a, s);
      if (h->o.vec) build_vec<float>(h->Af, a, s);
      h->Bf = float_copy(h->B, a, s);
      h->Cf = float_copy(h->C, a, s);
      h->Df = float_copy(h->D, a, s);
      if (h->o.sell) {
        build_sell<float>(h->A, h->Af_sell, a, s, h->o.sell);
        h->Af.sell = &h->Af_sell;
      }
      tune_product<float>(h->Af, 1, h->o, a, s);
    }
    if (h->o.verbose)
      fprintf(stderr, "[setup] lane groups: A %d, Shat %d, A(fp32) %d\n", h->A.g, h->Shat.g, h->Af.g);
    h->hA.build(h->A, 3, h->k, h->o, f32, s, f32 ? &h->Af : nullptr);
    h->hS.build(h->Shat, 1, h->k, h->o, f32, s);
    if (f32 && h->o.sell && h->hS.n_levels() > 0) {
      build_sell<float>(h->Shat, h->Shatf_sell, a, s, h->o.sell);
      h->hS.lv[0].Af.sell = &h->Shatf_sell;
    }
    // workspaces
    h->work.reset(new DeviceArena(s));
    DeviceArena& w = *h->work;
    h->red = make_reducer(w);
    const int k = h->k;
    const long long n = (3LL * nv + np) * k, nv3 = 3LL * nv * k;
    h->gOuter.init(w, n, h->o.restart);
    h->pc_r = w.alloc<double>(n + 1);
    h->pc_y = w.alloc<double>(n + 1);
    h->graph_epoch++;
    if (k > 1) h->mstage = w.alloc<double>(n + 1);
    h->bvec = w.alloc<double>(n + 1);
    h->xvec = w.alloc<double>(n + 1);
    h->rvec = w.alloc<double>(n + 1);
    if (f32) {
      h->dAinvf = w.alloc<float>(3LL * nv + 1);
      cast_d2f(h->dAinv, h->dAinvf, 3LL * nv, s);
      if (h->n_out) {
        h->out_af = w.alloc<float>((long long)h->n_out * 3 * nv + 1);
        cast_d2f(h->out_a, h->out_af, (long long)h->n_out * 3 * nv, s);
      }
      h->gAf.init(w, nv3, h->o.restart_inner);
      h->gSf.init(w, (long long)np * k, h->o.restart_inner);
      h->gIf.init(w, nv3, h->o.restart_inner);
      h->pr = w.alloc<float>(n + 1);
      h->py = w.alloc<float>(n + 1);
      h->yhatf = w.alloc<float>(nv3 + 1);
      h->rv2f = w.alloc<float>(nv3 + 1);
      h->xbarf = w.alloc<float>(nv3 + 1);
      h->xtf = w.alloc<float>(nv3 + 1);
      h->rrf = w.alloc<float>(nv3 + 1);
      h->rtf = w.alloc<float>(nv3 + 1);
      h->rp2f = w.alloc<float>((long long)np * k + 1);
    } else {
      h->gA.init(w, nv3, h->o.restart_inner);
      h->gS.init(w, (long long)np * k, h->o.restart_inner);
      h->gI.init(w, nv3, h->o.restart_inner);
      h->yhat = w.alloc<double>(nv3 + 1);
      h->rv2 = w.alloc<double>(nv3 + 1);
      h->xbar = w.alloc<double>(nv3 + 1);
      h->xt = w.alloc<double>(nv3 + 1);
      h->rr = w.alloc<double>(nv3 + 1);
      h->rt = w.alloc<double>(nv3 + 1);
      h->rp2 = w.alloc<double>((long long)np * k + 1);
    }
    SCR_CUDA(cudaStreamSynchronize(s));
    h->have_block = true;
    h->stats.levels_A = h->hA.n_levels();
    h->stats.levels_S = h->hS.n_levels();
    h->stats.setup_ms = ms_since(t0);
  });
}

static void reset_solve_stats(scr_ctx* h) {
  h->stats.outer_iters = h->stats.a_solves = h->stats.a_iters = h->stats.s_iters = h->stats.i_iters = 0;
  h->stats.pc_graph_runs = 0;
  h->hA.vcycles = h->hS.vcycles = 0;
  h->gA.reset_loop(h->s);
  h->gS.reset_loop(h->s);
  h->gI.reset_loop(h->s);
  h->gAf.reset_loop(h->s);
  h->gSf.reset_loop(h->s);
  h->gIf.reset_loop(h->s);
  h->gOuter.syncs = h->gA.syncs = h->gS.syncs = h->gI.syncs = 0;
  h->gAf.syncs = h->gSf.syncs = h->gIf.syncs = 0;
}

static int solve_impl(scr_ctx* h, const double* b, double* x, double rtol) {
  reset_solve_stats(h);
  Gmres<double>::Op op = [&](const double* xi, double* y) { apply_calA(h, xi, y, nullptr, false); };
  Gmres<double>::Op pc = [&](const double* r, double* y) { apply_pc_any(h, r, y); };
  std::function<double(const double*)> tr = [&](const double* xi) { return true_rel_block(h, b, xi); };
  int it = 0;
  double rel = 0;
  const bool ok = h->gOuter.solve(op, &pc, b, x, rtol, h->o.max_it, h->red, h->s, &it, &rel, &tr);
  collect_loops(h);
  h->stats.outer_iters = it;
  h->stats.rel_res = true_rel_block(h, b, x);
  h->stats.vcycles_A = h->hA.vcycles;
  h->stats.vcycles_S = h->hS.vcycles;
  h->stats.syncs = h->gOuter.syncs + h->gA.syncs + h->gS.syncs + h->gI.syncs + h->gAf.syncs + h->gSf.syncs +
                   h->gIf.syncs;
  if (!std::isfinite(h->stats.rel_res)) return SCR_NOT_CONVERGED;
  return (ok && h->stats.rel_res <= rtol) ? SCR_OK : SCR_NOT_CONVERGED;
}

int scr_solve(scr_handle h, const double* b, double* x, int dev) {
  if (!h || !b || !x) return SCR_INVALID_ARG;
  if (!h->have_block) {
    set_last_error("scr_solve before scr_setup");
    return SCR_INVALID_ARG;
  }
  if (h->k != 1) {
    set_last_error("scr_solve: the handle was set up for %d right-hand sides; use scr_solve_multi", h->k);
    return SCR_INVALID_ARG;
  }
  int status = SCR_OK;
  int rc = guarded([&] {
    auto t0 = Clock::now();
    const long long n = 3LL * h->nv + h->np;
    const double* bd = b;
    double* xd = x;
    if (!dev) {
      SCR_CUDA(cudaMemcpyAsync(h->bvec, b, sizeof(double) * n, cudaMemcpyHostToDevice, h->s));
      bd = h->bvec;
      xd = h->xvec;
    }
    status = solve_impl(h, bd, xd, h->o.rtol);
    if (!dev) SCR_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
    SCR_CUDA(cudaStreamSynchronize(h->s));
    h->stats.solve_ms = ms_since(t0);
  });
  if (rc != SCR_OK) return rc;
  if (status == SCR_NOT_CONVERGED)
    set_last_error("FGMRES stopped at %d iterations with relative residual %.3e", h->stats.outer_iters,
                   h->stats.rel_res);
  return status;
}

int scr_solve_multi(scr_handle h, const double* const* b, double* const* x, int dev, double* rel_res) {
  if (!h || !b || !x) return SCR_INVALID_ARG;
  if (!h->have_block) {
    set_last_error("scr_solve_multi before scr_setup");
    return SCR_INVALID_ARG;
  }
  const int k = h->k;
  for (int c = 0; c < k; ++c)
    if (!b[c] || !x[c]) {
      set_last_error("scr_solve_multi: NULL right-hand side or solution pointer");
      return SCR_INVALID_ARG;
    }
  int status = SCR_OK;
  int rc = guarded([&] {
    auto t0 = Clock::now();
    const long long n = 3LL * h->nv + h->np;
    cudaStream_t s = h->s;
    const cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    // right-hand sides one after another, their norms, then interleaved
    double* st = k > 1 ? h->mstage : h->bvec;
    for (int c = 0; c < k; ++c) SCR_CUDA(cudaMemcpyAsync(st + c * n, b[c], sizeof(double) * n, kin, s));
    std::vector<double> bn(k, 0.0), rn(k, 0.0);
    ArnoldiState* ast = h->gOuter.st;
    for (int c = 0; c < k; ++c) {
      norm2<double>(st + c * n, n, &ast->nrm2, h->red, s);
      SCR_CUDA(cudaMemcpyAsync(&bn[c], &ast->nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
    }
    if (k > 1) interleave(st, h->bvec, n, k, true, s);
    // the union tolerance rtol * min_c ||b_c|| / ||b|| bounds every
    // right-hand side's relative residual by rtol
    double b2 = 0.0, bmin = 0.0;
    for (int c = 0; c < k; ++c) {
      b2 += bn[c];
      if (bn[c] > 0.0 && (bmin == 0.0 || bn[c] < bmin)) bmin = bn[c];
    }
    const double rtol = b2 > 0.0 ? h->o.rtol * std::sqrt(bmin / b2) : h->o.rtol;
    status = solve_impl(h, h->bvec, h->xvec, rtol);
    // per right-hand side: FP64 residual norms, solutions out
    apply_calA(h, h->xvec, h->rvec, h->bvec, true);
    double* rs = k > 1 ? h->mstage : h->rvec;
    if (k > 1) interleave(h->rvec, rs, n, k, false, s);
    double worst = 0.0;
    for (int c = 0; c < k; ++c) {
      norm2<double>(rs + c * n, n, &ast->nrm2, h->red, s);
      SCR_CUDA(cudaMemcpyAsync(&rn[c], &ast->nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      const double rel = bn[c] > 0.0 ? std::sqrt(rn[c] / bn[c]) : std::sqrt(rn[c]);
      if (rel_res) rel_res[c] = rel;
      worst = std::max(worst, std::isfinite(rel) ? rel : 1e300);
    }
    double* xs = k > 1 ? h->mstage : h->xvec;
    if (k > 1) interleave(h->xvec, xs, n, k, false, s);
    for (int c = 0; c < k; ++c) SCR_CUDA(cudaMemcpyAsync(x[c], xs + c * n, sizeof(double) * n, kout, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    h->stats.rel_res = worst;
    status = worst <= h->o.rtol ? SCR_OK : SCR_NOT_CONVERGED;
    h->stats.solve_ms = ms_since(t0);
  });
  if (rc != SCR_OK) return rc;
  if (status == SCR_NOT_CONVERGED)
    set_last_error("multi-right-hand-side solve: a right-hand side did not reach the tolerance");
  return status;
}

// ------------------------------------------------------------ batched form
namespace {

__global__ void k_add_offset(int* __restrict__ a, long long n, int off) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) a[i] += off;
}

// Concatenate nb block matrices into one block-diagonal device matrix
// (standard value layout); row and column offsets in blocks.
struct UnionMatrix {
  int* rp = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  scr_bsr desc{};
};

UnionMatrix build_union(int nb, const scr_bsr* M, int br, int bc, const std::vector<int>& roff,
                        const std::vector<int>& coff, int nrows, int ncols, int dev, DeviceArena& a,
                        cudaStream_t s, const char* name) {
  UnionMatrix U;
  long long nnz = 0;
  for (int i = 0; i < nb; ++i) {
    check_bsr(&M[i], br, bc, M[i].nb_rows, M[i].nb_cols, name);
    nnz += M[i].nnzb;
  }
  if (nnz > 2147483647LL) throw std::invalid_argument("batched matrix exceeds int32 block indices");
  const int bs = br * bc;
  U.rp = a.alloc<int>(nrows + 1);
  U.col = a.alloc<int>(nnz + 1);
  U.val = a.alloc<double>(nnz * bs + 1);
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  long long off = 0;
  for (int i = 0; i < nb; ++i) {
    const scr_bsr& m = M[i];
    int first = 0, last = 0;
    SCR_CUDA(cudaMemcpyAsync(&first, m.row_ptr, sizeof(int), dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    SCR_CUDA(cudaMemcpyAsync(&last, m.row_ptr + m.nb_rows, sizeof(int),
                             dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    if (first != 0 || last != m.nnzb) throw std::invalid_argument(std::string(name) + ": row_ptr inconsistent");
    if (m.nb_rows > 0) {
      SCR_CUDA(cudaMemcpyAsync(U.rp + roff[i], m.row_ptr, sizeof(int) * m.nb_rows, k, s));
      k_add_offset<<<ceil_div(m.nb_rows, 256), 256, 0, s>>>(U.rp + roff[i], m.nb_rows, (int)off);
      SCR_LAUNCH();
    }
    if (m.nnzb > 0) {
      SCR_CUDA(cudaMemcpyAsync(U.col + off, m.col_idx, sizeof(int) * m.nnzb, k, s));
      k_add_offset<<<ceil_div(m.nnzb, 256), 256, 0, s>>>(U.col + off, m.nnzb, coff[i]);
      SCR_LAUNCH();
      SCR_CUDA(cudaMemcpyAsync(U.val + off * bs, m.val, sizeof(double) * m.nnzb * bs, k, s));
    }
    off += m.nnzb;
  }
  const int total = (int)nnz;
  SCR_CUDA(cudaMemcpyAsync(U.rp + nrows, &total, sizeof(int), cudaMemcpyHostToDevice, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  U.desc.nb_rows = nrows;
  U.desc.nb_cols = ncols;
  U.desc.br = br;
  U.desc.bc = bc;
  U.desc.nnzb = total;
  U.desc.row_ptr = U.rp;
  U.desc.col_idx = U.col;
  U.desc.val = U.val;
  return U;
}

}  // namespace

int scr_setup_batch(scr_handle h, int nb, const scr_bsr* A, const scr_bsr* B, const scr_bsr* C, const scr_bsr* D,
                    int dev) {
  if (!h || nb < 1 || !A || !B || !C || !D) {
    set_last_error("scr_setup_batch: NULL argument or nb < 1");
    return SCR_INVALID_ARG;
  }
  if (h->o.nrhs != 1) {
    set_last_error("scr_setup_batch: the batched form takes one right-hand side per member (nrhs = 1)");
    return SCR_INVALID_ARG;
  }
  std::vector<int> nv(nb), np(nb), vo(nb), po(nb);
  int NV = 0, NP = 0;
  for (int i = 0; i < nb; ++i) {
    nv[i] = A[i].nb_rows;
    np[i] = D[i].nb_rows;
    if (nv[i] < 0 || np[i] < 0) {
      set_last_error("scr_setup_batch: negative size");
      return SCR_INVALID_ARG;
    }
    vo[i] = NV;
    po[i] = NP;
    NV += nv[i];
    NP += np[i];
  }
  int rc = SCR_OK;
  DeviceArena tmp(h->s);
  UnionMatrix UA, UB, UC, UD;
  rc = guarded([&] {
    for (int i = 0; i < nb; ++i) {
      check_bsr(&A[i], 3, 3, nv[i], nv[i], "A");
      check_bsr(&B[i], 3, 1, nv[i], np[i], "B");
      check_bsr(&C[i], 1, 3, np[i], nv[i], "C");
      check_bsr(&D[i], 1, 1, np[i], np[i], "D");
    }
    UA = build_union(nb, A, 3, 3, vo, vo, NV, NV, dev, tmp, h->s, "A");
    UB = build_union(nb, B, 3, 1, vo, po, NV, NP, dev, tmp, h->s, "B");
    UC = build_union(nb, C, 1, 3, po, vo, NP, NV, dev, tmp, h->s, "C");
    UD = build_union(nb, D, 1, 1, po, po, NP, NP, dev, tmp, h->s, "D");
  });
  if (rc != SCR_OK) return rc;
  rc = scr_setup(h, &UA.desc, &UB.desc, &UC.desc, &UD.desc, 1);
  if (rc != SCR_OK) return rc;
  return guarded([&] {
    h->nbatch = nb;
    h->b_nv = nv;
    h->b_np = np;
    h->b_vo = vo;
    h->b_po = po;
    h->b_rel.assign(nb, 0.0);
    h->b_norms = h->work->alloc<double>(2LL * nb + 2);
    SCR_CUDA(cudaStreamSynchronize(h->s));
  });
}

namespace {

// out[2i] = ||v_i||^2, out[2i+1] = ||p_i||^2 of the union vector u, copied to host
std::vector<double> member_norms(scr_ctx* h, const double* u) {
  const int nb = h->nbatch;
  const long long NV3 = 3LL * h->nv;
  for (int i = 0; i < nb; ++i) {
    norm2<double>(u + 3LL * h->b_vo[i], 3LL * h->b_nv[i], h->b_norms + 2 * i, h->red, h->s);
    norm2<double>(u + NV3 + h->b_po[i], h->b_np[i], h->b_norms + 2 * i + 1, h->red, h->s);
  }
  std::vector<double> out(2 * nb);
  SCR_CUDA(cudaMemcpyAsync(out.data(), h->b_norms, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, h->s));
  SCR_CUDA(cudaStreamSynchronize(h->s));
  return out;
}

}  // namespace

int scr_solve_batch(scr_handle h, const double* const* b, double* const* x, int dev) {
  if (!h || !b || !x) return SCR_INVALID_ARG;
  if (!h->have_block || h->nbatch == 0) {
    set_last_error("scr_solve_batch before scr_setup_batch");
    return SCR_INVALID_ARG;
  }
  int status = SCR_OK;
  int rc = guarded([&] {
    auto t0 = Clock::now();
    const int nb = h->nbatch;
    const long long NV3 = 3LL * h->nv;
    const cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int i = 0; i < nb; ++i) {
      if (!b[i] || !x[i]) throw std::invalid_argument("scr_solve_batch: NULL member vector");
      const long long v3 = 3LL * h->b_nv[i];
      if (v3) SCR_CUDA(cudaMemcpyAsync(h->bvec + 3LL * h->b_vo[i], b[i], sizeof(double) * v3, kin, h->s));
      if (h->b_np[i])
        SCR_CUDA(cudaMemcpyAsync(h->bvec + NV3 + h->b_po[i], b[i] + v3, sizeof(double) * h->b_np[i], kin, h->s));
    }
    // every member's relative residual stays below rtol when the union's
    // does below rtol * min_i ||b_i|| / ||b||
    std::vector<double> bn = member_norms(h, h->bvec);
    double btot = 0.0, bmin = INFINITY;
    for (int i = 0; i < nb; ++i) {
      const double bi = bn[2 * i] + bn[2 * i + 1];
      btot += bi;
      if (bi > 0.0) bmin = std::min(bmin, std::sqrt(bi));
    }
    btot = std::sqrt(btot);
    const double rtol = (btot > 0.0 && std::isfinite(bmin)) ? h->o.rtol * bmin / btot : h->o.rtol;
    status = solve_impl(h, h->bvec, h->xvec, rtol);
    block_op(h->A, h->B, h->C, h->D, h->xvec, h->rvec, h->bvec, true, h->s);
    std::vector<double> rn = member_norms(h, h->rvec);
    for (int i = 0; i < nb; ++i) {
      const double bi = std::sqrt(bn[2 * i] + bn[2 * i + 1]);
      const double ri = std::sqrt(rn[2 * i] + rn[2 * i + 1]);
      h->b_rel[i] = bi > 0.0 ? ri / bi : ri;
      if (!(h->b_rel[i] <= h->o.rtol) && bi > 0.0) status = SCR_NOT_CONVERGED;
    }
    for (int i = 0; i < nb; ++i) {
      const long long v3 = 3LL * h->b_nv[i];
      if (v3) SCR_CUDA(cudaMemcpyAsync(x[i], h->xvec + 3LL * h->b_vo[i], sizeof(double) * v3, kout, h->s));
      if (h->b_np[i])
        SCR_CUDA(cudaMemcpyAsync(x[i] + v3, h->xvec + NV3 + h->b_po[i], sizeof(double) * h->b_np[i], kout, h->s));
    }
    SCR_CUDA(cudaStreamSynchronize(h->s));
    h->stats.solve_ms = ms_since(t0);
  });
  if (rc != SCR_OK) return rc;
  if (status == SCR_NOT_CONVERGED) set_last_error("batched solve: a member did not reach the tolerance");
  return status;
}

int scr_batch_residuals(scr_handle h, double* rel_res) {
  if (!h || !rel_res || h->nbatch == 0) return SCR_INVALID_ARG;
  for (int i = 0; i < h->nbatch; ++i) rel_res[i] = h->b_rel[i];
  return SCR_OK;
}

int scr_iters(scr_handle h, int* outer, int* inner_total) {
  if (!h) return SCR_INVALID_ARG;
  if (outer) *outer = h->stats.outer_iters;
  if (inner_total) *inner_total = h->stats.a_iters + h->stats.s_iters + h->stats.i_iters;
  return SCR_OK;
}

int scr_residual(scr_handle h, double* rel) {
  if (!h || !rel) return SCR_INVALID_ARG;
  *rel = h->stats.rel_res;
  return SCR_OK;
}

int scr_get_stats(scr_handle h, scr_stats* st) {
  if (!h || !st) return SCR_INVALID_ARG;
  *st = h->stats;
  const bool f32 = h->o.precision == SCR_MIXED;
  st->kernel_A = f32 ? h->Af.g : h->A.g;
  st->kernel_Shat = h->hS.n_levels() ? (f32 ? h->hS.lv[0].Af.g : h->hS.lv[0].A.g) : 0;
  if (forced_group() > 0) st->kernel_A = st->kernel_Shat = forced_group();
  st->kernel_launches = counters().launches;
  st->spmv_bytes = counters().spmv_bytes;
  st->levels_M = h->hM.n_levels();
  return SCR_OK;
}

int mm_setup(scr_handle h, const scr_bsr* L, int dev) {
  if (!h) return SCR_INVALID_ARG;
  return guarded([&] {
    auto t0 = Clock::now();
    if (!L) throw std::invalid_argument("L: NULL matrix");
    check_bsr(L, 1, 1, L->nb_rows, L->nb_rows, "L");
    cudaStream_t s = h->s;
    SCR_CUDA(cudaStreamSynchronize(s));
    h->have_mesh = false;
    h->hM = Hierarchy();
    h->hM.slot = 2;
    h->mwork.reset();
    h->mmats.reset(new DeviceArena(s));
    h->nm = L->nb_rows;
    h->L = upload(L, dev, *h->mmats, s);
    {
      DeviceArena tmp(s);
      double* d = tmp.alloc<double>(h->nm + 1);
      int* bad = tmp.alloc<int>(1);
      SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      diag_scalar(h->L, d, bad, s);
      int hb = 0;
      SCR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      if (hb) throw std::invalid_argument("L has a missing or zero diagonal entry");
    }
    scr_opts o = h->o;
    if (o.sell) {
      build_sell<double>(h->L, h->L_sell, *h->mmats, s, o.sell);
      h->L.sell = &h->L_sell;
    }
    tune_product<double>(h->L, 3, o, *h->mmats, s);
    h->hM.build(h->L, 1, 3, o, false, s);
    h->mwork.reset(new DeviceArena(s));
    DeviceArena& w = *h->mwork;
    h->mred = make_reducer(w);
    const long long n = 3LL * h->nm;
    h->mb = w.alloc<double>(n + 1);
    h->mx = w.alloc<double>(n + 1);
    h->mr = w.alloc<double>(n + 1);
    h->mz = w.alloc<double>(n + 1);
    h->mp = w.alloc<double>(n + 1);
    h->mq = w.alloc<double>(n + 1);
    h->cg = w.alloc<CgState>(1);
    SCR_CUDA(cudaStreamSynchronize(s));
    h->have_mesh = true;
    h->stats.levels_M = h->hM.n_levels();
    h->stats.mm_setup_ms = ms_since(t0);
  });
}

static double mesh_true_rel(scr_ctx* h, const double* g, const double* u);

// CG + AMG (Sec. 5.2.2) on (L kron I3) u = g, FP64.  The loop stops on the
// recursive residual r_k; before it reports convergence the true residual
// g - L u is recomputed, and where rounding has let the two drift apart the
// iteration restarts from the true residual (r = g - L u, z = M r, p = z) and
// goes on until the true residual meets mm_rtol or the iteration cap is hit.
// *rel is then the true relative residual.
static bool mesh_cg(scr_ctx* h, const double* g, double* u, int* iters, double* rel) {
  cudaStream_t s = h->s;
  const long long n = 3LL * h->nm;
  double* hr = h->mhs.h;
  fill<double>(u, 0.0, n, s);
  copy<double>(g, h->mr, n, s);
  cg_start(h->cg, g, n, h->mred, h->mhs.d, s);
  h->mhs.fetch(s);
  SCR_CUDA(cudaStreamSynchronize(s));
  *iters = 0;
  *rel = 0.0;
  if (!std::isfinite(hr[1])) {  // a NaN or infinite right-hand side: u = 0, not converged
    *rel = hr[1];
    return false;
  }
  if (!(hr[1] > 0.0)) return true;
  h->hM.apply<double>(h->mr, h->mz, s);
  cg_dot_rz(h->cg, h->mr, h->mz, n, h->mred, 1, s);
  copy<double>(h->mz, h->mp, n, s);
  EpiArgs set;
  for (int it = 1; it <= h->o.mm_max_it; ++it) {
    spmv<double, double>(h->L, h->mp, h->mq, 3, set, s);
    cg_alpha(h->cg, h->mp, h->mq, n, h->mred, s);
    cg_step_x_r(h->cg, h->mp, h->mq, u, h->mr, n, h->mred, h->mhs.d, s);
    h->mhs.fetch(s);
    SCR_CUDA(cudaStreamSynchronize(s));
    *iters = it;
    *rel = hr[0];
    if (!std::isfinite(*rel)) return false;
    if (*rel <= h->o.mm_rtol) {
      // confirm on the true residual (left in h->mq by mesh_true_rel)
      *rel = mesh_true_rel(h, g, u);
      if (*rel <= h->o.mm_rtol) return true;
      if (!std::isfinite(*rel)) return false;
      copy<double>(h->mq, h->mr, n, s);
      h->hM.apply<double>(h->mr, h->mz, s);
      cg_dot_rz(h->cg, h->mr, h->mz, n, h->mred, 1, s);
      copy<double>(h->mz, h->mp, n, s);
      continue;
    }
    h->hM.apply<double>(h->mr, h->mz, s);
    cg_dot_rz(h->cg, h->mr, h->mz, n, h->mred, 0, s);
    cg_update_p(h->cg, h->mz, h->mp, n, s);
  }
  return false;
}

static double mesh_true_rel(scr_ctx* h, const double* g, const double* u) {
  const long long n = 3LL * h->nm;
  EpiArgs res;
  res.kind = Epi::Resid;
  res.z = g;
  spmv<double, double>(h->L, u, h->mq, 3, res, h->s);
  norm2<double>(h->mq, n, &h->cg->rr, h->mred, h->s);
  double r2 = 0, b2 = 0;
  SCR_CUDA(cudaMemcpyAsync(&r2, &h->cg->rr, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  SCR_CUDA(cudaMemcpyAsync(&b2, &h->cg->bnorm2, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  SCR_CUDA(cudaStreamSynchronize(h->s));
  return b2 > 0 ? std::sqrt(r2 / b2) : std::sqrt(r2);
}

int mm_solve(scr_handle h, const double* g, double* u, int dev) {
  if (!h || !g || !u) return SCR_INVALID_ARG;
  if (!h->have_mesh) {
    set_last_error("mm_solve before mm_setup");
    return SCR_INVALID_ARG;
  }
  bool ok = false;
  int rc = guarded([&] {
    auto t0 = Clock::now();
    const long long n = 3LL * h->nm;
    const double* gd = g;
    double* ud = u;
    if (!dev) {
      SCR_CUDA(cudaMemcpyAsync(h->mb, g, sizeof(double) * n, cudaMemcpyHostToDevice, h->s));
      gd = h->mb;
      ud = h->mx;
    }
    h->hM.vcycles = 0;
    int it = 0;
    double rel = 0;
    ok = mesh_cg(h, gd, ud, &it, &rel);
    h->stats.mm_iters = it;
    h->stats.mm_rel_res = mesh_true_rel(h, gd, ud);
    h->stats.vcycles_M = h->hM.vcycles;
    if (!dev) SCR_CUDA(cudaMemcpyAsync(u, ud, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
    SCR_CUDA(cudaStreamSynchronize(h->s));
    h->stats.mm_solve_ms = ms_since(t0);
  });
  if (rc != SCR_OK) return rc;
  if (!ok) {
    set_last_error("mesh CG stopped at %d iterations, relative residual %.3e", h->stats.mm_iters,
                   h->stats.mm_rel_res);
    return SCR_NOT_CONVERGED;
  }
  return SCR_OK;
}

int mm_iters(scr_handle h, int* iters, double* rel) {
  if (!h) return SCR_INVALID_ARG;
  if (iters) *iters = h->stats.mm_iters;
  if (rel) *rel = h->stats.mm_rel_res;
  return SCR_OK;
}

int scr_apply_op(scr_handle h, const double* x, double* y) {
  if (h && h->k != 1) {
    set_last_error("this entry point takes one right-hand side (the handle has nrhs = %d)", h->k);
    return SCR_INVALID_ARG;
  }
  if (!h || !x || !y || !h->have_block) return SCR_INVALID_ARG;
  return guarded([&] {
    apply_calA(h, x, y, nullptr, false);
    SCR_CUDA(cudaStreamSynchronize(h->s));
  });
}

int scr_apply_pc(scr_handle h, const double* r, double* y) {
  if (h && h->k != 1) {
    set_last_error("this entry point takes one right-hand side (the handle has nrhs = %d)", h->k);
    return SCR_INVALID_ARG;
  }
  if (!h || !r || !y || !h->have_block) return SCR_INVALID_ARG;
  return guarded([&] {
    reset_solve_stats(h);
    apply_pc_any(h, r, y);
    collect_loops(h);
    SCR_CUDA(cudaStreamSynchronize(h->s));
  });
}

int scr_apply_schur(scr_handle h, const double* xp, double* yp) {
  if (h && h->k != 1) {
    set_last_error("this entry point takes one right-hand side (the handle has nrhs = %d)", h->k);
    return SCR_INVALID_ARG;
  }
  if (!h || !xp || !yp || !h->have_block) return SCR_INVALID_ARG;
  return guarded([&] {
    reset_solve_stats(h);
    if (h->o.precision == SCR_MIXED) {
      cast_d2f(xp, h->pr, h->np, h->s);
      PcView<float> v = view32(h);
      apply_S<float>(h, v, h->pr, h->py);
      cast_f2d(h->py, yp, h->np, h->s);
    } else {
      PcView<double> v = view64(h);
      apply_S<double>(h, v, xp, yp);
    }
    SCR_CUDA(cudaStreamSynchronize(h->s));
  });
}

static Hierarchy* pick_hier(scr_ctx* h, int which) {
  if (which == SCR_HIER_A && h->have_block) return &h->hA;
  if (which == SCR_HIER_SHAT && h->have_block) return &h->hS;
  if (which == SCR_HIER_MESH && h->have_mesh) return &h->hM;
  return nullptr;
}

int scr_amg_apply(scr_handle h, int which, const double* b, double* x) {
  if (!h || !b || !x) return SCR_INVALID_ARG;
  if (h->k != 1 && which != SCR_HIER_MESH) {
    set_last_error("scr_amg_apply: the block hierarchies of a handle with nrhs = %d act on %d interleaved vectors",
                   h->k, h->k);
    return SCR_INVALID_ARG;
  }
  Hierarchy* H = pick_hier(h, which);
  if (!H) {
    set_last_error("hierarchy not set up");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    const long long n = H->lv[0].n * H->nrhs;
    if (H->f32) {
      float* bf = H->lv[0].rf;  // level-0 scratch vectors double as staging here
      float* xf = H->lv[0].xf;
      cast_d2f(b, bf, n, h->s);
      float* bin = H->lv[0].bf;
      copy<float>(bf, bin, n, h->s);
      H->apply<float>(bin, xf, h->s);
      cast_f2d(xf, x, n, h->s);
    } else {
      H->apply<double>(b, x, h->s);
    }
    SCR_CUDA(cudaStreamSynchronize(h->s));
  });
}

int scr_amg_levels(scr_handle h, int which, int* n) {
  if (!h || !n) return SCR_INVALID_ARG;
  Hierarchy* H = pick_hier(h, which);
  *n = H ? H->n_levels() : 0;
  return SCR_OK;
}

int scr_export(scr_handle h, int which, int level, int kind, scr_bsr_out* out) {
  if (!h || !out) return SCR_INVALID_ARG;
  Hierarchy* H = pick_hier(h, which);
  if (!H || level < 0 || level >= H->n_levels()) {
    set_last_error("scr_export: no such hierarchy level");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    Level& L = H->lv[level];
    if (kind == SCR_EXPORT_AGGREGATES) {
      out->nb_rows = L.A.nbr;
      out->nb_cols = L.n_agg;
      out->br = out->bc = 1;
      out->nnzb = L.agg ? L.A.nbr : 0;
      if (out->col_idx && L.agg)
        SCR_CUDA(cudaMemcpyAsync(out->col_idx, L.agg, sizeof(int) * L.A.nbr, cudaMemcpyDeviceToHost, h->s));
      SCR_CUDA(cudaStreamSynchronize(h->s));
      return;
    }
    if (kind == SCR_EXPORT_ROOTS) {
      out->nb_rows = L.agg ? L.n_agg : 0;
      out->nb_cols = L.A.nbr;
      out->br = out->bc = 1;
      out->nnzb = L.agg ? L.n_agg : 0;
      if (out->col_idx && L.agg && L.n_agg)
        SCR_CUDA(cudaMemcpyAsync(out->col_idx, L.roots, sizeof(int) * L.n_agg, cudaMemcpyDeviceToHost, h->s));
      SCR_CUDA(cudaStreamSynchronize(h->s));
      return;
    }
    const DBsr<double>* M = nullptr;
    if (kind == SCR_EXPORT_OPERATOR) M = &L.A;
    else if (kind == SCR_EXPORT_PROLONGATOR) M = &L.P;
    else if (kind == SCR_EXPORT_BLOCK_B && level == 0 && h->have_block) M = &h->B;
    else if (kind == SCR_EXPORT_BLOCK_C && level == 0 && h->have_block) M = &h->C;
    else if (kind == SCR_EXPORT_BLOCK_D && level == 0 && h->have_block) M = &h->D;
    else throw std::invalid_argument("scr_export: unknown kind (B, C, D: level 0 of a set-up block system)");
    out->nb_rows = M->nbr;
    out->nb_cols = M->nbc;
    out->br = M->br;
    out->bc = M->bc;
    out->nnzb = (int)M->nnzb;
    if (!out->row_ptr || !out->col_idx || !out->val) return;
    if (M->nbr == 0) return;
    DeviceArena tmp(h->s);
    const size_t nv = (size_t)M->nnzb * M->br * M->bc;
    double* v = tmp.alloc<double>(nv + 1);
    from_slab(M->rp, M->val, v, M->nbr, M->br, M->bc, M->nnzb, h->s);
    SCR_CUDA(cudaMemcpyAsync(out->row_ptr, M->rp, sizeof(int) * (M->nbr + 1), cudaMemcpyDeviceToHost, h->s));
    SCR_CUDA(cudaMemcpyAsync(out->col_idx, M->col, sizeof(int) * M->nnzb, cudaMemcpyDeviceToHost, h->s));
    SCR_CUDA(cudaMemcpyAsync(out->val, v, sizeof(double) * nv, cudaMemcpyDeviceToHost, h->s));
    SCR_CUDA(cudaStreamSynchronize(h->s));
  });
}

int scr_assembly_setup(scr_handle h, const scr_mesh* m, const scr_physics* ph) {
  if (!h || !m || !ph || m->n_nodes < 0 || m->n_elem < 0 || m->n_p < 0 ||
      (m->n_elem > 0 && (!m->ien || !m->pien || !m->etype)) || (m->n_nodes > 0 && !m->xyz)) {
    set_last_error("scr_assembly_setup: NULL argument or negative size");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    if (!(ph->rho_s > 0.0) || !(ph->E_s > 0.0) || !(ph->dt > 0.0) || !(ph->rho_f > 0.0))
      throw std::invalid_argument("scr_assembly_setup: densities, modulus and time step must be positive");
    cudaStream_t s = h->s;
    h->have_residual = false;
    h->have_coupling = false;  // a mesh coupling belongs to the previous mesh
    h->ta.ready = false;
    h->rmats.reset(new DeviceArena(s));
    ResidualPhysics rp{ph->rho_f, ph->mu_f, ph->rho_s, ph->E_s / (2.0 * (1.0 + ph->nu_s)), ph->dt,
                       ph->c_m_solid, ph->c_c_solid};
    h->ra.setup(m->n_nodes, m->n_elem, m->n_p, m->xyz, m->ien, m->pien, m->etype, rp, *h->rmats, s);
    if (m->dir_v) h->dir_v.assign(m->dir_v, m->dir_v + m->n_nodes);
    else h->dir_v.clear();
    h->phys = *ph;
    const long long nv3 = 3LL * m->n_nodes;
    // staging for the host path: v, vhat, vdot, u (3 n_nodes each), p (n_p), R (3 n_nodes + n_p)
    h->r_in = h->rmats->alloc<double>(5 * nv3 + 2LL * m->n_p + 1);
    h->d_dir = nullptr;
    if (!h->dir_v.empty()) {
      h->d_dir = h->rmats->alloc<unsigned char>(h->dir_v.size());
      SCR_CUDA(cudaMemcpyAsync(h->d_dir, h->dir_v.data(), h->dir_v.size(), cudaMemcpyHostToDevice, s));
      SCR_CUDA(cudaStreamSynchronize(s));
    }
    h->have_residual = true;
  });
}

int scr_assemble_residual(scr_handle h, const double* v, const double* vhat, const double* p,
                          const double* vdot, const double* u, double* R, int dev) {
  if (!h || !v || !p || !R) return SCR_INVALID_ARG;
  if (!h->have_residual) {
    set_last_error("scr_assemble_residual before scr_assembly_setup");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    cudaStream_t s = h->s;
    const long long nv3 = 3LL * h->ra.nn, np = h->ra.np;
    if (dev) {
      h->ra.evaluate(v, vhat, p, vdot, u, R, s);
    } else {
      double* dv = h->r_in;
      double* dvh = dv + nv3;
      double* dvd = dvh + nv3;
      double* du = dvd + nv3;
      double* dp = du + nv3;
      double* dR = dp + np;  // 3 n_nodes + n_p
      auto in = [&](const double* src, double* dst, long long n) -> const double* {
        if (!src) return nullptr;
        SCR_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        return dst;
      };
      const double* a = in(v, dv, nv3);
      const double* b = in(vhat, dvh, nv3);
      const double* c = in(vdot, dvd, nv3);
      const double* d = in(u, du, nv3);
      const double* e = in(p, dp, np);
      h->ra.evaluate(a, b, e, c, d, dR, s);
      SCR_CUDA(cudaMemcpyAsync(R, dR, sizeof(double) * (nv3 + np), cudaMemcpyDeviceToHost, s));
    }
    SCR_CUDA(cudaStreamSynchronize(s));
  });
}

namespace {

// Tangent at the state (device pointers) into the captured patterns, then
// the set-up of the block solve on it (Shat, hierarchies, copies)
void assemble_tangent_dev(scr_ctx* h, const double* v, const double* vhat, const double* p, const double* vd) {
  cudaStream_t s = h->s;
  if (!h->ta.ready) {
    h->tmats.reset(new DeviceArena(s));
    const DBsr<double>* mats[4] = {&h->A, &h->B, &h->C, &h->D};
    h->ta.setup(h->ra, mats, *h->tmats, s);
  }
  const double rho = h->phys.rho_inf;
  const double am = 0.5 * (3.0 - rho) / (1.0 + rho), af = 1.0 / (1.0 + rho), ga = af;
  const double cf = af * ga * h->phys.dt, cu = cf * cf / am;
  h->ta.evaluate(h->ra, h->d_dir, v, vhat, p, vd, am, cf, cu, s);
  scr_bsr d[4];
  for (int m = 0; m < 4; ++m) {
    const TangentAssembler::Pattern& P = h->ta.pat[m];
    d[m] = scr_bsr{P.nbr, P.nbc, P.br, P.bc, (int)P.nnzb, P.rp, P.col, P.val};
  }
  h->tangent_setup = true;
  const int rc = h->o.tangent_resetup ? scr_update_values(h, &d[0], &d[1], &d[2], &d[3], 1)
                                      : scr_setup(h, &d[0], &d[1], &d[2], &d[3], 1);
  h->tangent_setup = false;
  if (rc != SCR_OK) throw std::runtime_error(std::string("set-up on the assembled tangent: ") + scr_last_error());
}

// mesh-motion arguments of scr_corrector_ale (null: the mesh stays fixed)
struct AleArgs {
  const double* uhat_n;
  const double* vhat_n;  // may be null (zero)
  double* uhat;
};

int corrector_run(scr_handle h, double* v, double* p, double* vdot, double* u, int n_iter, double* res_norms,
                  int dev, const AleArgs* ale) {
  if (!h->have_block || !h->have_residual || h->k != 1 || h->ra.nn != h->nv || h->ra.np != h->np) {
    set_last_error("scr_corrector: needs scr_setup (nrhs = 1) and scr_assembly_setup on the same mesh");
    return SCR_INVALID_ARG;
  }
  if (ale && (!h->have_coupling || !h->have_mesh || h->nm != h->cpl_nf || h->cpl_nn != h->ra.nn)) {
    set_last_error("scr_corrector_ale: needs scr_mesh_coupling and mm_setup on the same fluid nodes");
    return SCR_INVALID_ARG;
  }
  int status = SCR_OK;
  int mesh_fail_it = 0;
  double mesh_fail_rel = 0.0;
  int rc = guarded([&] {
    cudaStream_t s = h->s;
    const long long nv3 = 3LL * h->nv, np = h->np, n = nv3 + np;
    // generalized-alpha weights of the rate increments (Sec. 3.4)
    const double rho = h->phys.rho_inf;
    const double am = 0.5 * (3.0 - rho) / (1.0 + rho), af = 1.0 / (1.0 + rho), ga = af;
    const double cf = af * ga * h->phys.dt, cu = cf * cf / am;
    // state on the device
    double *dv = v, *dp = p, *dvd = vdot, *du = u;
    if (!dev) {
      dv = h->r_in;
      dvd = dv + nv3;
      du = dvd + nv3;
      dp = du + nv3;
      SCR_CUDA(cudaMemcpyAsync(dv, v, sizeof(double) * nv3, cudaMemcpyHostToDevice, s));
      SCR_CUDA(cudaMemcpyAsync(dvd, vdot, sizeof(double) * nv3, cudaMemcpyHostToDevice, s));
      SCR_CUDA(cudaMemcpyAsync(du, u, sizeof(double) * nv3, cudaMemcpyHostToDevice, s));
      SCR_CUDA(cudaMemcpyAsync(dp, p, sizeof(double) * np, cudaMemcpyHostToDevice, s));
    }
    const long long nf3 = 3LL * h->cpl_nf;
    if (ale) {
      // the state enters at the same-Y predictor: u is u_n
      copy<double>(du, h->d_un, nv3, s);
      const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
      SCR_CUDA(cudaMemcpyAsync(h->d_uhn, ale->uhat_n, sizeof(double) * nf3, k, s));
      if (ale->vhat_n) SCR_CUDA(cudaMemcpyAsync(h->d_vhn, ale->vhat_n, sizeof(double) * nf3, k, s));
      else fill<double>(h->d_vhn, 0.0, nf3, s);
    }
    double* R = h->r_in + 4 * nv3 + np;  // 3 n_nodes + n_p
    EpiArgs plain;
    for (int it = 0; it <= n_iter; ++it) {
      if (ale) {
        // steps 3-4: mesh displacement at t_{n+1} as the harmonic extension
        // of the interface displacement (CG + AMG on the eliminated
        // Laplacian, right-hand side lifted with the raw one), mesh
        // velocity at t_{n+alpha_f}
        mesh_interface_data(h->d_node_of_f, h->d_follow, du, h->d_un, af, h->d_g, h->cpl_nf, s);
        spmv<double, double>(h->Lraw, h->d_g, h->d_lift, 3, plain, s);
        mesh_lift(h->d_dir_m, h->d_g, h->d_lift, h->cpl_nf, s);
        int mit = 0;
        double mrel = 0.0;
        if (!mesh_cg(h, h->d_lift, h->d_uh, &mit, &mrel)) {
          status = SCR_NOT_CONVERGED;
          mesh_fail_it = mit;
          mesh_fail_rel = mrel;
        }
        h->stats.mm_iters = mit;
        mesh_velocity(h->d_node_of_f, h->d_uh, h->d_uhn, h->d_vhn, af, ga, h->phys.dt, h->d_vhat, h->cpl_nf, s);
      }
      // full Newton (options.newton): the tangent at this iteration's state
      // and the set-up of the solve on it, before its right-hand side
      if (h->o.newton && it < n_iter) assemble_tangent_dev(h, dv, ale ? h->d_vhat : nullptr, dp, dvd);
      ArnoldiState* st = h->gOuter.st;
      h->ra.evaluate(dv, ale ? h->d_vhat : nullptr, dp, dvd, du, R, s);
      // resistance outlets: the traction P_j a_j with P_j = m_j (a_j^T v)
      // (the term whose derivative is the rank-1 tangent c_j a_j a_j^T,
      // c_j = alpha_f gamma dt m_j)
      if (h->n_out) outlet_terms<double>(h, h->out_a, dv, R, 1.0 / cf);
      negate_masked(R, h->d_dir, h->bvec, nv3, n, s);
      norm2<double>(h->bvec, n, &st->nrm2, h->red, s);
      double r2 = 0.0;
      SCR_CUDA(cudaMemcpyAsync(&r2, &st->nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaStreamSynchronize(s));
      res_norms[it] = std::sqrt(r2);
      if (it == n_iter) break;
      const int st_solve = solve_impl(h, h->bvec, h->xvec, h->o.rtol);
      if (st_solve != SCR_OK) status = st_solve;
      // rates at t_{n+alpha_m} move by alpha_m, values at t_{n+alpha_f} by
      // alpha_f gamma dt, the solid displacement by (alpha_f gamma dt)^2 / alpha_m
      axpby(am, h->xvec, 1.0, dvd, nv3, s);
      axpby(cf, h->xvec, 1.0, dv, nv3, s);
      axpby(cu, h->xvec, 1.0, du, nv3, s);
      axpby(cf, h->xvec + nv3, 1.0, dp, np, s);
    }
    if (!dev) {
      SCR_CUDA(cudaMemcpyAsync(v, dv, sizeof(double) * nv3, cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaMemcpyAsync(vdot, dvd, sizeof(double) * nv3, cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaMemcpyAsync(u, du, sizeof(double) * nv3, cudaMemcpyDeviceToHost, s));
      SCR_CUDA(cudaMemcpyAsync(p, dp, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
    }
    if (ale)
      SCR_CUDA(cudaMemcpyAsync(ale->uhat, h->d_uh, sizeof(double) * nf3,
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
  });
  if (rc != SCR_OK) return rc;
  if (mesh_fail_it)
    set_last_error("scr_corrector_ale: mesh CG stopped at %d iterations, relative residual %.3e", mesh_fail_it,
                   mesh_fail_rel);
  return status;
}

}  // namespace

int scr_assemble_tangent(scr_handle h, const double* v, const double* vhat, const double* p, const double* vdot,
                         int dev) {
  if (!h || !v || !p) return SCR_INVALID_ARG;
  if (!h->have_block || !h->have_residual || h->nbatch || h->ra.nn != h->nv || h->ra.np != h->np) {
    set_last_error("scr_assemble_tangent: needs scr_setup (not batched) and scr_assembly_setup on the same mesh");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    cudaStream_t s = h->s;
    const long long nv3 = 3LL * h->nv, np = h->np;
    const double *dv = v, *dvh = vhat, *dp = p, *dvd = vdot;
    if (!dev) {
      double* b = h->r_in;
      SCR_CUDA(cudaMemcpyAsync(b, v, sizeof(double) * nv3, cudaMemcpyHostToDevice, s));
      dv = b;
      if (vhat) {
        SCR_CUDA(cudaMemcpyAsync(b + nv3, vhat, sizeof(double) * nv3, cudaMemcpyHostToDevice, s));
        dvh = b + nv3;
      }
      if (vdot) {
        SCR_CUDA(cudaMemcpyAsync(b + 2 * nv3, vdot, sizeof(double) * nv3, cudaMemcpyHostToDevice, s));
        dvd = b + 2 * nv3;
      }
      SCR_CUDA(cudaMemcpyAsync(b + 4 * nv3, p, sizeof(double) * np, cudaMemcpyHostToDevice, s));
      dp = b + 4 * nv3;
    }
    assemble_tangent_dev(h, dv, dvh, dp, dvd);
    SCR_CUDA(cudaStreamSynchronize(s));
  });
}

int scr_corrector(scr_handle h, double* v, double* p, double* vdot, double* u, int n_iter, double* res_norms,
                  int dev) {
  if (!h || !v || !p || !vdot || !u || n_iter < 0 || !res_norms) return SCR_INVALID_ARG;
  return corrector_run(h, v, p, vdot, u, n_iter, res_norms, dev, nullptr);
}

int scr_corrector_ale(scr_handle h, double* v, double* p, double* vdot, double* u, const double* uhat_n,
                      const double* vhat_n, double* uhat, int n_iter, double* res_norms, int dev) {
  if (!h || !v || !p || !vdot || !u || !uhat_n || !uhat || n_iter < 0 || !res_norms) return SCR_INVALID_ARG;
  const AleArgs ale{uhat_n, vhat_n, uhat};
  return corrector_run(h, v, p, vdot, u, n_iter, res_norms, dev, &ale);
}

int scr_mesh_coupling(scr_handle h, int n_fluid, const int* fluid_id, const unsigned char* dir_m,
                      const unsigned char* follow, const scr_bsr* L_raw) {
  if (!h || n_fluid <= 0 || !fluid_id || !dir_m || !follow || !L_raw) {
    set_last_error("scr_mesh_coupling: NULL argument or no fluid nodes");
    return SCR_INVALID_ARG;
  }
  if (!h->have_residual) {
    set_last_error("scr_mesh_coupling: needs scr_assembly_setup first (the node count)");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    check_bsr(L_raw, 1, 1, n_fluid, n_fluid, "L_raw");
    const int nn = h->ra.nn;
    std::vector<int> node_of_f(n_fluid, -1);
    for (int i = 0; i < nn; ++i) {
      const int f = fluid_id[i];
      if (f < -1 || f >= n_fluid) throw std::invalid_argument("scr_mesh_coupling: fluid_id out of range");
      if (f < 0) continue;
      if (node_of_f[f] >= 0) throw std::invalid_argument("scr_mesh_coupling: fluid ordinal used twice");
      node_of_f[f] = i;
    }
    for (int f = 0; f < n_fluid; ++f) {
      if (node_of_f[f] < 0) throw std::invalid_argument("scr_mesh_coupling: fluid ordinal without a node");
      if (follow[f] && !dir_m[f]) throw std::invalid_argument("scr_mesh_coupling: follow set on a free mesh node");
    }
    cudaStream_t s = h->s;
    SCR_CUDA(cudaStreamSynchronize(s));
    h->have_coupling = false;
    h->cmats.reset(new DeviceArena(s));
    DeviceArena& a = *h->cmats;
    h->Lraw = upload(L_raw, 0, a, s);
    scr_opts o = h->o;
    o.sell = 0;
    tune_product<double>(h->Lraw, 3, o, a, s);
    const long long nf3 = 3LL * n_fluid, nv3 = 3LL * nn;
    h->d_node_of_f = a.alloc<int>(n_fluid);
    h->d_dir_m = a.alloc<unsigned char>(n_fluid);
    h->d_follow = a.alloc<unsigned char>(n_fluid);
    h->d_g = a.alloc<double>(nf3);
    h->d_lift = a.alloc<double>(nf3);
    h->d_uh = a.alloc<double>(nf3);
    h->d_uhn = a.alloc<double>(nf3);
    h->d_vhn = a.alloc<double>(nf3);
    h->d_un = a.alloc<double>(nv3);
    h->d_vhat = a.alloc<double>(nv3);
    SCR_CUDA(cudaMemcpyAsync(h->d_node_of_f, node_of_f.data(), sizeof(int) * n_fluid, cudaMemcpyHostToDevice, s));
    SCR_CUDA(cudaMemcpyAsync(h->d_dir_m, dir_m, n_fluid, cudaMemcpyHostToDevice, s));
    SCR_CUDA(cudaMemcpyAsync(h->d_follow, follow, n_fluid, cudaMemcpyHostToDevice, s));
    // the mesh velocity is zero away from the fluid nodes
    fill<double>(h->d_vhat, 0.0, nv3, s);
    SCR_CUDA(cudaStreamSynchronize(s));
    h->cpl_nf = n_fluid;
    h->cpl_nn = nn;
    h->have_coupling = true;
  });
}

int scr_set_outlets(scr_handle h, int n_out, int len, const double* a, const double* c) {
  if (!h || n_out < 0 || (n_out > 0 && (!a || !c || len <= 0))) {
    set_last_error("scr_set_outlets: NULL argument or negative count");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    for (int j = 0; j < n_out; ++j)
      if (!std::isfinite(c[j])) throw std::invalid_argument("scr_set_outlets: coefficient not finite");
    h->pend_n = n_out;
    h->pend_len = n_out ? len : 0;
    h->pend_a.assign(a, a + (size_t)n_out * len);
    h->pend_c.assign(c, c + n_out);
  });
}

int scr_tune_save(const char* path) {
  if (!path) {
    set_last_error("scr_tune_save: NULL path");
    return SCR_INVALID_ARG;
  }
  return guarded([&] { tune_save(path); });
}

int scr_tune_load(const char* path) {
  if (!path) {
    set_last_error("scr_tune_load: NULL path");
    return SCR_INVALID_ARG;
  }
  return guarded([&] { tune_load(path); });
}

int scr_profile_begin(scr_handle h, int kclass, int capacity) {
  if (!h || capacity < 0 || (kclass != SCR_PROF_SPMV_A && kclass != SCR_PROF_BLOCK_OP)) return SCR_INVALID_ARG;
  if (!h->have_block) {
    set_last_error("scr_profile_begin before scr_setup");
    return SCR_INVALID_ARG;
  }
  return guarded([&] {
    KernelProfiler& p = profiler();
    while ((int)p.ev.size() < 2 * capacity) {
      cudaEvent_t e;
      SCR_CUDA(cudaEventCreate(&e));
      p.ev.push_back(e);
    }
    p.active = true;
    p.kclass = kclass;
    p.target = kclass == SCR_PROF_SPMV_A
                   ? (h->o.precision == SCR_MIXED ? (const void*)h->Af.val : (const void*)h->A.val)
                   : nullptr;
    p.cap = capacity;
    p.used = 0;
    p.launches = 0;
    p.bytes = p.flops = 0;
  });
}

int scr_profile_end(scr_handle h, scr_kprof* out) {
  if (!h || !out) return SCR_INVALID_ARG;
  return guarded([&] {
    KernelProfiler& p = profiler();
    SCR_CUDA(cudaStreamSynchronize(h->s));
    double ms = 0;
    for (int i = 0; i < p.used; ++i) {
      float t = 0;
      SCR_CUDA(cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]));
      ms += t;
    }
    out->launches = p.launches;
    out->timed = p.used;
    out->ms = ms;
    out->bytes = p.bytes;
    out->flops = p.flops;
    p.active = false;
  });
}

int scr_bsr_spmv(const scr_bsr* M, const double* x, double* y, void* stream) {
  if (!M || !x || !y) return SCR_INVALID_ARG;
  return guarded([&] {
    if (!((M->br == 1 || M->br == 3) && (M->bc == 1 || M->bc == 3)))
      throw std::invalid_argument("scr_bsr_spmv: block sizes must be 1 or 3");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceArena tmp(s);
    DBsr<double> D;
    D.nbr = M->nb_rows;
    D.nbc = M->nb_cols;
    D.br = M->br;
    D.bc = M->bc;
    D.nnzb = M->nnzb;
    D.rp = const_cast<int*>(M->row_ptr);
    D.col = const_cast<int*>(M->col_idx);
    const size_t nv = (size_t)M->nnzb * M->br * M->bc;
    if (D.nbr < 0 || D.nbc < 0 || D.nnzb < 0) throw std::invalid_argument("scr_bsr_spmv: negative size");
    int* bad = tmp.alloc<int>(1);
    SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (D.nbr > 0) {
      k_check_cols<<<ceil_div(D.nbr, 256), 256, 0, s>>>(D.nbr, D.nbc, D.rp, D.col, D.nnzb, bad);
      SCR_LAUNCH();
    }
    int hb = 0;
    SCR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    if (hb) throw std::invalid_argument("scr_bsr_spmv: row_ptr/col_idx invalid");
    D.val = tmp.alloc<double>(nv + 1);
    if (nv) to_slab<double>(D.rp, M->val, D.val, D.nbr, D.br, D.bc, D.nnzb, s);
    // a forced 16-byte kernel (spmv_group 301..316) gets its padded copy
    if (forced_group() >= 300) build_vec<double>(D, tmp, s);
    spmv<double, double>(D, x, y, 1, EpiArgs(), s);
    SCR_CUDA(cudaStreamSynchronize(s));
  });
}

}  // extern "C"

namespace scr {
void check_bsr_indices(int nbr, int nbc, const int* rp, const int* col, long long nnzb, int* bad, cudaStream_t s) {
  if (nbr <= 0) return;
  k_check_cols<<<ceil_div(nbr, 256), 256, 0, s>>>(nbr, nbc, rp, col, nnzb, bad);
  SCR_LAUNCH();
}
}  // namespace scr
