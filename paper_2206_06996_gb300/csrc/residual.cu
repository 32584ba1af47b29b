// Residual assembly of the unified-continuum VMS formulation on linear
// tetrahedra (Sec. 3.2 fluid element with tau_M, tau_C and the metric G;
// Sec. 3.5 solid element linearised at the reference state, incompressible,
// with its own stabilisation), the element loop of the segregated
// multi-corrector step (Sec. 3.5) moved to the GPU.
//
// Two deterministic passes: one thread per element forms the element's
// momentum and mass residuals at the 4-point Gauss rule and writes them to
// a per-element scratch; one thread per velocity node (pressure index)
// then adds the contributions of its elements in increasing element order,
// so every run adds the same terms in the same order.
#include <algorithm>
#include <vector>

#include "kernels.h"

namespace scr {
namespace {

constexpr int kElemVals = 16;  // 4 x 3 momentum + 4 mass entries per element

struct ElemGeom {
  double V;          // volume
  double dN[4][3];   // shape-function gradients
  double dxi[3][3];  // d xi_k / d x_i
  bool ok;
};

__device__ ElemGeom elem_geom(const double (&x)[4][3]) {
  ElemGeom g;
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) e[k][i] = x[k + 1][i] - x[0][i];
  // the rows of the inverse Jacobian are the cofactor vectors / det
  const double c[3][3] = {
      {e[1][1] * e[2][2] - e[1][2] * e[2][1], e[1][2] * e[2][0] - e[1][0] * e[2][2],
       e[1][0] * e[2][1] - e[1][1] * e[2][0]},
      {e[2][1] * e[0][2] - e[2][2] * e[0][1], e[2][2] * e[0][0] - e[2][0] * e[0][2],
       e[2][0] * e[0][1] - e[2][1] * e[0][0]},
      {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
       e[0][0] * e[1][1] - e[0][1] * e[1][0]}};
  const double det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
  g.ok = det != 0.0;
  if (!g.ok) return g;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) g.dxi[k][i] = c[k][i] / det;
  for (int i = 0; i < 3; ++i) {
    g.dN[1][i] = g.dxi[0][i];
    g.dN[2][i] = g.dxi[1][i];
    g.dN[3][i] = g.dxi[2][i];
    g.dN[0][i] = -(g.dN[1][i] + g.dN[2][i] + g.dN[3][i]);
  }
  g.V = fabs(det) / 6.0;
  return g;
}

// diameter of the sphere through the four vertices (Cramer's rule on the
// bisector-plane system)
__device__ double circumsphere_diameter(const double (&x)[4][3]) {
  double M[3][3], b[3];
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
      M[k][i] = 2.0 * (x[k + 1][i] - x[0][i]);
      s += x[k + 1][i] * x[k + 1][i] - x[0][i] * x[0][i];
    }
    b[k] = s;
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
      for (int q = 0; q < 3; ++q) Mc[r][q] = q == col ? b[r] : M[r][q];
    const double cc = det3(Mc) / d - x[0][col];
    r2 += cc * cc;
  }
  return 2.0 * sqrt(r2);
}

struct ResidualArgs {
  int n_elem;
  const double* xyz;
  const int* ien;
  const int* pien;
  const unsigned char* etype;
  const double *v, *vhat, *p, *vd, *u;  // vhat, vd, u may be null (zero)
  double rho_f, mu_f, rho_s, mu_s, dt, c_m_solid, c_c_solid;
  double* E;  // n_elem x kElemVals
};

__global__ void __launch_bounds__(128) k_element_residual(ResidualArgs A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.n_elem) return;
  double x[4][3], v[4][3], vh[4][3], vd[4][3], u[4][3], p[4];
  for (int a = 0; a < 4; ++a) {
    const int n = A.ien[4 * e + a];
    for (int i = 0; i < 3; ++i) {
      x[a][i] = A.xyz[3 * n + i];
      v[a][i] = A.v[3 * n + i];
      vh[a][i] = A.vhat ? A.vhat[3 * n + i] : 0.0;
      vd[a][i] = A.vd ? A.vd[3 * n + i] : 0.0;
      u[a][i] = A.u ? A.u[3 * n + i] : 0.0;
    }
    p[a] = A.p[A.pien[4 * e + a]];
  }
  double Rm[4][3] = {}, Rp[4] = {};
  const ElemGeom g = elem_geom(x);
  // 4-point rule: barycentric (ga, gb, gb, gb) and permutations, weight V/4
  const double ga = (5.0 + 3.0 * sqrt(5.0)) / 20.0, gb = (5.0 - sqrt(5.0)) / 20.0;
  if (g.ok && A.etype[e] == 0) {
    // ---- fluid (Sec. 3.2) ----
    const double rho = A.rho_f, mu = A.mu_f, w = g.V / 4.0;
    double G[3][3];
    const double cM = 0.5 * cbrt(2.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) s += g.dxi[k][i] * (k == l ? 2.0 * cM : cM) * g.dxi[l][j];
        G[i][j] = s;
      }
    double GG = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) GG += G[i][j] * G[i][j];
    const double trG = G[0][0] + G[1][1] + G[2][2], nu = mu / rho;
    double gv[3][3], gp[3];
    for (int i = 0; i < 3; ++i) {
      gp[i] = 0.0;
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int a = 0; a < 4; ++a) s += v[a][i] * g.dN[a][j];
        gv[i][j] = s;
      }
      for (int a = 0; a < 4; ++a) gp[i] += p[a] * g.dN[a][i];
    }
    const double div = gv[0][0] + gv[1][1] + gv[2][2];
    for (int q = 0; q < 4; ++q) {
      double N[4];
      for (int a = 0; a < 4; ++a) N[a] = a == q ? ga : gb;
      double uq[3], vdq[3], pq = 0.0;
      for (int i = 0; i < 3; ++i) {
        uq[i] = vdq[i] = 0.0;
        for (int a = 0; a < 4; ++a) {
          uq[i] += N[a] * (v[a][i] - vh[a][i]);
          vdq[i] += N[a] * vd[a][i];
        }
      }
      for (int a = 0; a < 4; ++a) pq += N[a] * p[a];
      double uGu = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) uGu += uq[i] * G[i][j] * uq[j];
      const double tauM = 1.0 / (rho * sqrt(4.0 / (A.dt * A.dt) + uGu + 36.0 * nu * nu * GG));
      const double tauC = 1.0 / (tauM * trG);
      // strong momentum residual of the coarse scales and the fine scales
      double rM[3], vp[3];
      for (int i = 0; i < 3; ++i) {
        rM[i] = rho * (vdq[i] + gv[i][0] * uq[0] + gv[i][1] * uq[1] + gv[i][2] * uq[2]) + gp[i];
        vp[i] = -tauM * rM[i];
      }
      const double pp = -tauC * div;
      double gvvp[3];
      for (int i = 0; i < 3; ++i) gvvp[i] = gv[i][0] * vp[0] + gv[i][1] * vp[1] + gv[i][2] * vp[2];
      for (int a = 0; a < 4; ++a) {
        const double dNu = g.dN[a][0] * uq[0] + g.dN[a][1] * uq[1] + g.dN[a][2] * uq[2];
        const double dNvp = g.dN[a][0] * vp[0] + g.dN[a][1] * vp[1] + g.dN[a][2] * vp[2];
        for (int i = 0; i < 3; ++i) {
          // deviatoric viscous stress 2 mu dev(sym grad v), row i, against grad N_a
          double visc = 0.0;
          for (int j = 0; j < 3; ++j)
            visc += g.dN[a][j] * (mu * (gv[i][j] + gv[j][i]) - (i == j ? 2.0 * mu * div / 3.0 : 0.0));
          const double s = N[a] * (rM[i] - gp[i]) - g.dN[a][i] * (pq + pp) + visc - rho * vp[i] * dNu +
                           rho * N[a] * gvvp[i] - rho * vp[i] * dNvp;
          Rm[a][i] += w * s;
        }
        Rp[a] += w * (N[a] * div - dNvp);
      }
    }
  } else if (g.ok) {
    // ---- solid (Sec. 3.5, small strain at the reference state) ----
    const double rho = A.rho_s, mu = A.mu_s, w = g.V / 4.0;
    const double cs = sqrt(mu / rho), dx = circumsphere_diameter(x);
    const double tauM = A.c_m_solid * dx / (cs * rho), tauC = A.c_c_solid * cs * dx * rho;
    double gu[3][3], gv[3][3], gp[3];
    for (int i = 0; i < 3; ++i) {
      gp[i] = 0.0;
      for (int j = 0; j < 3; ++j) {
        double su = 0.0, sv = 0.0;
        for (int a = 0; a < 4; ++a) {
          su += u[a][i] * g.dN[a][j];
          sv += v[a][i] * g.dN[a][j];
        }
        gu[i][j] = su;
        gv[i][j] = sv;
      }
      for (int a = 0; a < 4; ++a) gp[i] += p[a] * g.dN[a][i];
    }
    const double divu = gu[0][0] + gu[1][1] + gu[2][2], divv = gv[0][0] + gv[1][1] + gv[2][2];
    for (int q = 0; q < 4; ++q) {
      double N[4];
      for (int a = 0; a < 4; ++a) N[a] = a == q ? ga : gb;
      double vdq[3], pq = 0.0;
      for (int i = 0; i < 3; ++i) {
        vdq[i] = 0.0;
        for (int a = 0; a < 4; ++a) vdq[i] += N[a] * vd[a][i];
      }
      for (int a = 0; a < 4; ++a) pq += N[a] * p[a];
      for (int a = 0; a < 4; ++a) {
        for (int i = 0; i < 3; ++i) {
          double elas = 0.0;
          for (int j = 0; j < 3; ++j)
            elas += g.dN[a][j] * (mu * (gu[i][j] + gu[j][i]) - (i == j ? 2.0 * mu * divu / 3.0 : 0.0));
          Rm[a][i] += w * (N[a] * rho * vdq[i] - g.dN[a][i] * pq + g.dN[a][i] * tauC * divv + elas);
        }
        double s = N[a] * divv;
        for (int j = 0; j < 3; ++j) s += g.dN[a][j] * tauM * (rho * vdq[j] + gp[j]);
        Rp[a] += w * s;
      }
    }
  }
  double* out = A.E + (long long)e * kElemVals;
  for (int a = 0; a < 4; ++a) {
    for (int i = 0; i < 3; ++i) out[3 * a + i] = Rm[a][i];
    out[12 + a] = Rp[a];
  }
}

// R[3 n + i] = sum over (e, a) in node n's list of E[e].Rm[a][i]; then the
// pressure rows from their own lists (entries e * 4 + a, increasing e)
__global__ void k_gather_velocity(int nn, const int* __restrict__ ptr, const int* __restrict__ ent,
                                  const double* __restrict__ E, double* __restrict__ R) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  double r0 = 0.0, r1 = 0.0, r2 = 0.0;
  for (int t = ptr[n]; t < ptr[n + 1]; ++t) {
    const int ea = ent[t];
    const double* o = E + (long long)(ea >> 2) * kElemVals + 3 * (ea & 3);
    r0 += o[0];
    r1 += o[1];
    r2 += o[2];
  }
  R[3LL * n] = r0;
  R[3LL * n + 1] = r1;
  R[3LL * n + 2] = r2;
}

__global__ void k_gather_pressure(int np, const int* __restrict__ ptr, const int* __restrict__ ent,
                                  const double* __restrict__ E, double* __restrict__ R) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  double r = 0.0;
  for (int t = ptr[q]; t < ptr[q + 1]; ++t) {
    const int ea = ent[t];
    r += E[(long long)(ea >> 2) * kElemVals + 12 + (ea & 3)];
  }
  R[q] = r;
}

// lists of (element, local vertex) per row, increasing element order
void build_lists(int nrows, int ne, const int* conn, std::vector<int>& ptr, std::vector<int>& ent) {
  ptr.assign(nrows + 1, 0);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 4; ++a) ptr[conn[4 * e + a] + 1]++;
  for (int r = 0; r < nrows; ++r) ptr[r + 1] += ptr[r];
  ent.assign(ptr[nrows], 0);
  std::vector<int> cur(ptr.begin(), ptr.end() - 1);
  for (int e = 0; e < ne; ++e)
    for (int a = 0; a < 4; ++a) ent[cur[conn[4 * e + a]]++] = e * 4 + a;
}

}  // namespace

void ResidualAssembler::setup(int nn_, int ne_, int np_, const double* xyz, const int* ien, const int* pien,
                              const unsigned char* etype, const ResidualPhysics& ph_, DeviceArena& a,
                              cudaStream_t s) {
  nn = nn_;
  ne = ne_;
  np = np_;
  ph = ph_;
  for (long long i = 0; i < 4LL * ne; ++i)
    if (ien[i] < 0 || ien[i] >= nn || pien[i] < 0 || pien[i] >= np)
      throw CudaError{cudaErrorInvalidValue, "residual mesh: connectivity index out of range"};
  std::vector<int> vp, ve, pp, pe;
  build_lists(nn, ne, ien, vp, ve);
  build_lists(np, ne, pien, pp, pe);
  auto up = [&](const void* src, size_t bytes) {
    void* d = a.alloc<unsigned char>(bytes);
    SCR_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    return d;
  };
  d_xyz = static_cast<double*>(up(xyz, sizeof(double) * 3 * nn));
  d_ien = static_cast<int*>(up(ien, sizeof(int) * 4 * ne));
  d_pien = static_cast<int*>(up(pien, sizeof(int) * 4 * ne));
  d_etype = static_cast<unsigned char*>(up(etype, ne));
  d_vptr = static_cast<int*>(up(vp.data(), sizeof(int) * vp.size()));
  d_vent = static_cast<int*>(up(ve.data(), sizeof(int) * std::max<size_t>(ve.size(), 1)));
  d_pptr = static_cast<int*>(up(pp.data(), sizeof(int) * pp.size()));
  d_pent = static_cast<int*>(up(pe.data(), sizeof(int) * std::max<size_t>(pe.size(), 1)));
  d_E = a.alloc<double>((size_t)ne * kElemVals + 1);
  SCR_CUDA(cudaStreamSynchronize(s));
}

void ResidualAssembler::evaluate(const double* v, const double* vhat, const double* p, const double* vd,
                                 const double* u, double* R, cudaStream_t s) {
  if (ne > 0) {
    ResidualArgs A{ne, d_xyz, d_ien, d_pien, d_etype, v, vhat, p, vd, u,
                   ph.rho_f, ph.mu_f, ph.rho_s, ph.mu_s, ph.dt, ph.c_m_solid, ph.c_c_solid, d_E};
    k_element_residual<<<ceil_div(ne, 128), 128, 0, s>>>(A);
    SCR_LAUNCH();
  }
  if (nn > 0) {
    k_gather_velocity<<<ceil_div(nn, 256), 256, 0, s>>>(nn, d_vptr, d_vent, d_E, R);
    SCR_LAUNCH();
  }
  if (np > 0) {
    k_gather_pressure<<<ceil_div(np, 256), 256, 0, s>>>(np, d_pptr, d_pent, d_E, R + 3LL * nn);
    SCR_LAUNCH();
  }
  counters().launches += 3;
}

}  // namespace scr
