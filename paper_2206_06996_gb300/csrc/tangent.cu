// Tangent assembly of the unified-continuum VMS formulation on linear
// tetrahedra: the consistent tangent of the segregated multi-corrector step
// (Sec. 3.5), K = alpha_m dR/d(ydot) + alpha_f gamma dt dR/dy with the
// stabilisation parameters tau_M, tau_C evaluated at the state and held
// fixed, for the element residuals of residual.cu (Sec. 3.2 fluid element;
// Sec. 3.5 solid element linearised at the reference state).  With the
// velocity increments as unknowns, a velocity rate moves by alpha_m (cm), a
// velocity or pressure value by alpha_f gamma dt (cf) and the solid
// displacement by cf^2 / alpha_m (cu).
//
// Two deterministic passes, as for the residual:
//  1. one thread per (element, column) forms one of the 16 columns of the
//     element's 16 x 16 tangent at the 4-point Gauss rule (momentum rows
//     against velocity columns: A, against the pressure column: B; mass rows
//     against velocity columns: C, against the pressure column: D) and
//     writes it to a per-element scratch; four of an element's threads first
//     form the element's geometry and its Gauss-point quantities (one point
//     each) in shared memory for all sixteen;
//  2. one thread per stored block of A, B, C and D (the pattern the solver
//     was set up with) adds the contributions of the elements that couple
//     its row and column, in increasing element order.
// Dirichlet velocity nodes follow the input convention: their rows of A are
// identity rows, and the pattern holds no other block in a Dirichlet row or
// column of A, B or C.
#include <vector>

#include "kernels.h"

namespace scr {
namespace {

constexpr int kTanVals = 256;  // A 144, B 48, C 48, D 16 per element
__host__ __device__ constexpr int offA(int a, int b, int i, int k) { return (a * 4 + b) * 9 + i * 3 + k; }
__host__ __device__ constexpr int offB(int a, int b, int i) { return 144 + (a * 4 + b) * 3 + i; }
__host__ __device__ constexpr int offC(int a, int b, int k) { return 192 + (a * 4 + b) * 3 + k; }
__host__ __device__ constexpr int offD(int a, int b) { return 240 + a * 4 + b; }

struct TangentArgs {
  int n_elem;
  const double* xyz;
  const int* ien;
  const int* pien;
  const unsigned char* etype;
  const double *v, *vhat, *p, *vd;  // vhat, vd may be null (zero)
  double rho_f, mu_f, rho_s, mu_s, dt, c_m_solid, c_c_solid;
  double cm, cf, cu;
  double* E;  // n_elem x kTanVals
};

// shape-function gradients and volume of a linear tet; dxi[k][i] = d xi_k /
// d x_i (rows of the inverse Jacobian); false for a degenerate element
__device__ bool tet_geometry(const double (&x)[4][3], double (&dN)[4][3], double (&dxi)[3][3], double& V) {
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) e[k][i] = x[k + 1][i] - x[0][i];
  const double c[3][3] = {
      {e[1][1] * e[2][2] - e[1][2] * e[2][1], e[1][2] * e[2][0] - e[1][0] * e[2][2],
       e[1][0] * e[2][1] - e[1][1] * e[2][0]},
      {e[2][1] * e[0][2] - e[2][2] * e[0][1], e[2][2] * e[0][0] - e[2][0] * e[0][2],
       e[2][0] * e[0][1] - e[2][1] * e[0][0]},
      {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
       e[0][0] * e[1][1] - e[0][1] * e[1][0]}};
  const double det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
  if (det == 0.0) return false;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) dxi[k][i] = c[k][i] / det;
  for (int i = 0; i < 3; ++i) {
    dN[1][i] = dxi[0][i];
    dN[2][i] = dxi[1][i];
    dN[3][i] = dxi[2][i];
    dN[0][i] = -(dN[1][i] + dN[2][i] + dN[3][i]);
  }
  V = fabs(det) / 6.0;
  return true;
}

__device__ double circum_diameter(const double (&x)[4][3]) {
  double M[3][3], rhs[3];
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
      M[k][i] = 2.0 * (x[k + 1][i] - x[0][i]);
      s += x[k + 1][i] * x[k + 1][i] - x[0][i] * x[0][i];
    }
    rhs[k] = s;
  }
  auto det3 = [](const double (&a)[3][3]) {
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  };
  const double d = det3(M);
  double r2 = 0.0;
  for (int col = 0; col < 3; ++col) {
    double Mc[3][3];
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) Mc[r][q] = q == col ? rhs[r] : M[r][q];
    const double cc = det3(Mc) / d - x[0][col];
    r2 += cc * cc;
  }
  return 2.0 * sqrt(r2);
}

// Per-element quantities shared by the element's 16 column threads (one
// CTA holds kTanElems elements): geometry, the velocity gradient, and for
// each Gauss point q the stabilisation parameters, the fine-scale velocity
// and the two directional derivatives of the shape functions.
constexpr int kTanElems = 8;
struct TanGeom {
  double dN[4][3];
  double gv[3][3];
  double w;
  int kind;  // -1: degenerate or no element, 0: fluid, 1: solid
};
struct TanGauss {
  double tauM, tauC, vp[3], dNu[4], dNvp[4];
};

// column (b, c) of element e's tangent, c = 0..2 the velocity component k =
// c of vertex b, c = 3 its pressure: the 12 momentum rows and 4 mass rows
// (A and C entries, or B and D entries), accumulated over the Gauss points.
// Phase 1: the element's threads c16 = q < 4 form the element's geometry
// (each) and the quantities of Gauss point q; phase 2: every thread its
// column from those shared values.
__global__ void __launch_bounds__(16 * kTanElems) k_element_tangent(TangentArgs T) {
  __shared__ TanGeom sg[kTanElems];
  __shared__ TanGauss sq[kTanElems][4];
  const int el = threadIdx.x >> 4, c16 = threadIdx.x & 15;
  const int e = blockIdx.x * kTanElems + el;
  const int b = c16 >> 2, c = c16 & 3;
  const double ga = (5.0 + 3.0 * sqrt(5.0)) / 20.0, gb = (5.0 - sqrt(5.0)) / 20.0;
  const double cm = T.cm, cf = T.cf, cu = T.cu;
  if (c16 < 4) {
    const int q = c16;
    int kind = -1;
    if (e < T.n_elem) {
      double x[4][3], v[4][3], p[4], dN[4][3], dxi[3][3], V = 0.0;
      for (int a = 0; a < 4; ++a) {
        const int n = T.ien[4 * e + a];
        for (int i = 0; i < 3; ++i) {
          x[a][i] = T.xyz[3 * n + i];
          v[a][i] = T.v[3 * n + i];
        }
        p[a] = T.p[T.pien[4 * e + a]];
      }
      if (tet_geometry(x, dN, dxi, V)) {
        kind = T.etype[e] == 0 ? 0 : 1;
        double gv[3][3] = {};
        if (kind == 0) {
          // ---- fluid (Sec. 3.2): tau_M, tau_C and the fine scales at q ----
          const double rho = T.rho_f, mu = T.mu_f, nu = mu / rho;
          double G[3][3];
          const double cM = 0.5 * cbrt(2.0);
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              double s = 0.0;
              for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) s += dxi[k][i] * (k == l ? 2.0 * cM : cM) * dxi[l][j];
              G[i][j] = s;
            }
          double GG = 0.0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) GG += G[i][j] * G[i][j];
          const double trG = G[0][0] + G[1][1] + G[2][2];
          double gp[3];
          for (int i = 0; i < 3; ++i) {
            gp[i] = 0.0;
            for (int j = 0; j < 3; ++j) {
              double s = 0.0;
              for (int a = 0; a < 4; ++a) s += v[a][i] * dN[a][j];
              gv[i][j] = s;
            }
            for (int a = 0; a < 4; ++a) gp[i] += p[a] * dN[a][i];
          }
          double N[4];
          for (int a = 0; a < 4; ++a) N[a] = a == q ? ga : gb;
          double uq[3], vdq[3];
          for (int i = 0; i < 3; ++i) {
            uq[i] = vdq[i] = 0.0;
            for (int a = 0; a < 4; ++a) {
              const int n = T.ien[4 * e + a];
              uq[i] += N[a] * (v[a][i] - (T.vhat ? T.vhat[3 * n + i] : 0.0));
              vdq[i] += N[a] * (T.vd ? T.vd[3 * n + i] : 0.0);
            }
          }
          double uGu = 0.0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) uGu += uq[i] * G[i][j] * uq[j];
          TanGauss& g = sq[el][q];
          g.tauM = 1.0 / (rho * sqrt(4.0 / (T.dt * T.dt) + uGu + 36.0 * nu * nu * GG));
          g.tauC = 1.0 / (g.tauM * trG);
          for (int i = 0; i < 3; ++i)
            g.vp[i] = -g.tauM * (rho * (vdq[i] + gv[i][0] * uq[0] + gv[i][1] * uq[1] + gv[i][2] * uq[2]) + gp[i]);
          for (int a = 0; a < 4; ++a) {
            g.dNu[a] = dN[a][0] * uq[0] + dN[a][1] * uq[1] + dN[a][2] * uq[2];
            g.dNvp[a] = dN[a][0] * g.vp[0] + dN[a][1] * g.vp[1] + dN[a][2] * g.vp[2];
          }
        } else if (q == 0) {
          // ---- solid: its stabilisation from the circumsphere diameter ----
          const double rho = T.rho_s, mu = T.mu_s;
          const double cs = sqrt(mu / rho), dx = circum_diameter(x);
          sq[el][0].tauM = T.c_m_solid * dx / (cs * rho);
          sq[el][0].tauC = T.c_c_solid * cs * dx * rho;
        }
        if (q == 0) {
          for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 3; ++i) sg[el].dN[a][i] = dN[a][i];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) sg[el].gv[i][j] = gv[i][j];
          sg[el].w = V / 4.0;
        }
      }
    }
    if (q == 0) sg[el].kind = kind;
  }
  __syncthreads();
  const int kind = sg[el].kind;
  if (kind < 0) {
    if (e < T.n_elem) {  // degenerate element: zero column
      double* out = T.E + (long long)e * kTanVals;
      for (int a = 0; a < 4; ++a) {
        if (c < 3) {
          for (int i = 0; i < 3; ++i) out[offA(a, b, i, c)] = 0.0;
          out[offC(a, b, c)] = 0.0;
        } else {
          for (int i = 0; i < 3; ++i) out[offB(a, b, i)] = 0.0;
          out[offD(a, b)] = 0.0;
        }
      }
    }
    return;
  }
  double dN[4][3];
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i) dN[a][i] = sg[el].dN[a][i];
  const double w = sg[el].w;
  double Km[4][3] = {}, Kq[4] = {};  // momentum rows (a, i) and mass rows a of this column
  if (kind == 0) {
    const double rho = T.rho_f, mu = T.mu_f;
    double gv[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gv[i][j] = sg[el].gv[i][j];
    for (int q = 0; q < 4; ++q) {
      double N[4];
      for (int a = 0; a < 4; ++a) N[a] = a == q ? ga : gb;
      const TanGauss& g = sq[el][q];
      const double tauM = g.tauM, tauC = g.tauC;
      const double vp[3] = {g.vp[0], g.vp[1], g.vp[2]};
      double dNu[4], dNvp[4];
      for (int a = 0; a < 4; ++a) {
        dNu[a] = g.dNu[a];
        dNvp[a] = g.dNvp[a];
      }
      if (c < 3) {
        // velocity column (b, k): the strong residual rM moves by drM through
        // the rate (cm), the convective velocity and the velocity gradient
        // (cf); the fine-scale velocity by -tau_M drM
        const int k = c;
        const double dNbvp = dN[b][0] * vp[0] + dN[b][1] * vp[1] + dN[b][2] * vp[2];
        double drM[3], dvp[3], gvdvp[3];
        for (int i = 0; i < 3; ++i) {
          drM[i] = rho * ((i == k ? cm * N[b] + cf * dNu[b] : 0.0) + cf * gv[i][k] * N[b]);
          dvp[i] = -tauM * drM[i];
        }
        for (int i = 0; i < 3; ++i) gvdvp[i] = gv[i][0] * dvp[0] + gv[i][1] * dvp[1] + gv[i][2] * dvp[2];
        for (int a = 0; a < 4; ++a) {
          const double dNadvp = dN[a][0] * dvp[0] + dN[a][1] * dvp[1] + dN[a][2] * dvp[2];
          const double dNab = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2];
          for (int i = 0; i < 3; ++i) {
            double s = N[a] * drM[i];
            s += tauC * cf * dN[a][i] * dN[b][k];
            s += mu * cf * ((i == k ? dNab : 0.0) + dN[a][k] * dN[b][i]) - (2.0 * mu / 3.0) * cf * dN[a][i] * dN[b][k];
            s += -rho * (dvp[i] * dNu[a] + vp[i] * cf * N[b] * dN[a][k]);
            s += rho * N[a] * ((i == k ? cf * dNbvp : 0.0) + gvdvp[i]);
            s += -rho * (dvp[i] * dNvp[a] + vp[i] * dNadvp);
            Km[a][i] += w * s;
          }
          Kq[a] += w * (N[a] * cf * dN[b][k] - dNadvp);
        }
      } else {
        // pressure column b: the pressure gradient in rM moves by cf dN_b
        double dvpP[3], gvdvpP[3];
        for (int i = 0; i < 3; ++i) dvpP[i] = -tauM * cf * dN[b][i];
        for (int i = 0; i < 3; ++i) gvdvpP[i] = gv[i][0] * dvpP[0] + gv[i][1] * dvpP[1] + gv[i][2] * dvpP[2];
        for (int a = 0; a < 4; ++a) {
          const double dNadvp = dN[a][0] * dvpP[0] + dN[a][1] * dvpP[1] + dN[a][2] * dvpP[2];
          for (int i = 0; i < 3; ++i) {
            double s = -dN[a][i] * cf * N[b];
            s += -rho * dvpP[i] * dNu[a];
            s += rho * N[a] * gvdvpP[i];
            s += -rho * (dvpP[i] * dNvp[a] + vp[i] * dNadvp);
            Km[a][i] += w * s;
          }
          Kq[a] += w * (-dNadvp);
        }
      }
    }
  } else {
    // ---- solid (Sec. 3.5, small-strain deviatoric elasticity, incompressible) ----
    const double rho = T.rho_s, mu = T.mu_s;
    const double tauM = sq[el][0].tauM, tauC = sq[el][0].tauC;
    for (int q = 0; q < 4; ++q) {
      double N[4];
      for (int a = 0; a < 4; ++a) N[a] = a == q ? ga : gb;
      for (int a = 0; a < 4; ++a) {
        const double dd = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2];
        if (c < 3) {
          const int k = c;
          for (int i = 0; i < 3; ++i) {
            double s = i == k ? cm * rho * N[a] * N[b] : 0.0;
            s += cu * (mu * ((i == k ? dd : 0.0) + dN[a][k] * dN[b][i]) - (2.0 * mu / 3.0) * dN[a][i] * dN[b][k]);
            s += cf * tauC * dN[a][i] * dN[b][k];
            Km[a][i] += w * s;
          }
          Kq[a] += w * (cf * N[a] * dN[b][k] + cm * tauM * rho * dN[a][k] * N[b]);
        } else {
          for (int i = 0; i < 3; ++i) Km[a][i] += w * (-cf * dN[a][i] * N[b]);
          Kq[a] += w * (cf * tauM * dd);
        }
      }
    }
  }
  double* out = T.E + (long long)e * kTanVals;
  for (int a = 0; a < 4; ++a) {
    if (c < 3) {
      for (int i = 0; i < 3; ++i) out[offA(a, b, i, c)] = Km[a][i];
      out[offC(a, b, c)] = Kq[a];
    } else {
      for (int i = 0; i < 3; ++i) out[offB(a, b, i)] = Km[a][i];
      out[offD(a, b)] = Kq[a];
    }
  }
}

// block row of every stored block
__global__ void k_block_rows(int nbr, const int* __restrict__ rp, int* __restrict__ brow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int t = rp[i]; t < rp[i + 1]; ++t) brow[t] = i;
}

// kind 0: A (3x3; rows: velocity nodes, list of the row node; columns matched
// against ien), 1: B (3x1; columns against pien), 2: C (1x3; rows: pressure
// indices, list of the pressure index; columns against ien), 3: D (1x1)
template <int KIND>
__global__ void k_gather_tangent(long long nnzb, const int* __restrict__ brow, const int* __restrict__ col,
                                 const int* __restrict__ lptr, const int* __restrict__ lent,
                                 const int* __restrict__ ien, const int* __restrict__ pien,
                                 const unsigned char* __restrict__ dir, const double* __restrict__ E,
                                 double* __restrict__ val) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  constexpr int BS = KIND == 0 ? 9 : (KIND == 3 ? 1 : 3);
  const int r = brow[t], c = col[t];
  double acc[BS];
  for (int q = 0; q < BS; ++q) acc[q] = 0.0;
  if (KIND == 0 && dir && dir[r]) {
    // Dirichlet velocity node: identity row (the pattern keeps the diagonal block only)
    if (r == c) acc[0] = acc[4] = acc[8] = 1.0;
  } else if (KIND == 1 && dir && dir[r]) {
    // a Dirichlet row of B has no blocks; zero if the caller's pattern kept one
  } else {
    const int* cm = (KIND == 0 || KIND == 2) ? ien : pien;
    for (int s = lptr[r]; s < lptr[r + 1]; ++s) {
      const int ea = lent[s];
      const int e = ea >> 2, a = ea & 3;
      for (int b = 0; b < 4; ++b) {
        if (cm[4 * e + b] != c) continue;
        const double* o = E + (long long)e * kTanVals;
        if constexpr (KIND == 0) {
          for (int q = 0; q < 9; ++q) acc[q] += o[offA(a, b, q / 3, q % 3)];
        } else if constexpr (KIND == 1) {
          for (int q = 0; q < 3; ++q) acc[q] += o[offB(a, b, q)];
        } else if constexpr (KIND == 2) {
          for (int q = 0; q < 3; ++q) acc[q] += o[offC(a, b, q)];
        } else {
          acc[0] += o[offD(a, b)];
        }
      }
    }
  }
  for (int q = 0; q < BS; ++q) val[t * BS + q] = acc[q];
}

}  // namespace

void TangentAssembler::setup(const ResidualAssembler& ra, const DBsr<double>* const mats[4], DeviceArena& a,
                             cudaStream_t s) {
  E = a.alloc<double>((size_t)ra.ne * kTanVals + 1);
  for (int m = 0; m < 4; ++m) {
    const DBsr<double>& M = *mats[m];
    Pattern& P = pat[m];
    P.nbr = M.nbr;
    P.nbc = M.nbc;
    P.br = M.br;
    P.bc = M.bc;
    P.nnzb = M.nnzb;
    P.rp = a.alloc<int>(M.nbr + 1);
    P.col = a.alloc<int>(M.nnzb + 1);
    P.brow = a.alloc<int>(M.nnzb + 1);
    P.val = a.alloc<double>((size_t)M.nnzb * M.br * M.bc + 1);
    SCR_CUDA(cudaMemcpyAsync(P.rp, M.rp, sizeof(int) * (M.nbr + 1), cudaMemcpyDeviceToDevice, s));
    if (M.nnzb) SCR_CUDA(cudaMemcpyAsync(P.col, M.col, sizeof(int) * M.nnzb, cudaMemcpyDeviceToDevice, s));
    if (M.nbr) {
      k_block_rows<<<ceil_div(M.nbr, 256), 256, 0, s>>>(M.nbr, P.rp, P.brow);
      SCR_LAUNCH();
      counters().launches++;
    }
  }
  SCR_CUDA(cudaStreamSynchronize(s));
  ready = true;
}

void TangentAssembler::evaluate(const ResidualAssembler& ra, const unsigned char* d_dir, const double* v,
                                const double* vhat, const double* p, const double* vd, double cm, double cf,
                                double cu, cudaStream_t s) {
  const int ne = ra.ne;
  if (ne > 0) {
    TangentArgs T{ne,          ra.d_xyz,    ra.d_ien, ra.d_pien, ra.d_etype, v,    vhat, p, vd,
                  ra.ph.rho_f, ra.ph.mu_f,  ra.ph.rho_s, ra.ph.mu_s, ra.ph.dt, ra.ph.c_m_solid, ra.ph.c_c_solid,
                  cm,          cf,          cu,       E};
    k_element_tangent<<<ceil_div(ne, kTanElems), 16 * kTanElems, 0, s>>>(T);
    SCR_LAUNCH();
    counters().launches++;
  }
  const int kT = 256;
  // rows of A and B: the velocity node's (element, vertex) list; rows of C
  // and D: the pressure index's list
  if (pat[0].nnzb) {
    k_gather_tangent<0><<<ceil_div(pat[0].nnzb, kT), kT, 0, s>>>(pat[0].nnzb, pat[0].brow, pat[0].col, ra.d_vptr,
                                                             ra.d_vent, ra.d_ien, ra.d_pien, d_dir, E, pat[0].val);
    SCR_LAUNCH();
  }
  if (pat[1].nnzb) {
    k_gather_tangent<1><<<ceil_div(pat[1].nnzb, kT), kT, 0, s>>>(pat[1].nnzb, pat[1].brow, pat[1].col, ra.d_vptr,
                                                             ra.d_vent, ra.d_ien, ra.d_pien, d_dir, E, pat[1].val);
    SCR_LAUNCH();
  }
  if (pat[2].nnzb) {
    k_gather_tangent<2><<<ceil_div(pat[2].nnzb, kT), kT, 0, s>>>(pat[2].nnzb, pat[2].brow, pat[2].col, ra.d_pptr,
                                                             ra.d_pent, ra.d_ien, ra.d_pien, nullptr, E, pat[2].val);
    SCR_LAUNCH();
  }
  if (pat[3].nnzb) {
    k_gather_tangent<3><<<ceil_div(pat[3].nnzb, kT), kT, 0, s>>>(pat[3].nnzb, pat[3].brow, pat[3].col, ra.d_pptr,
                                                             ra.d_pent, ra.d_ien, ra.d_pien, nullptr, E, pat[3].val);
    SCR_LAUNCH();
  }
  counters().launches += 4;
}

}  // namespace scr
