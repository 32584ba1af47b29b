/*
 * Seeded synthetic inputs for the vascular FSI linear-solver path.
 *
 * This file produces the matrices that the solver consumes; it holds none of
 * the solver's arithmetic.  It builds
 *   - a structured tetrahedral mesh of a straight or stenosed elastic tube
 *     (lumen + wall, one node set, C0 velocity across the fluid-solid
 *     interface, a duplicated pressure index for every interface node as in
 *     Sec. 3.3 of the paper, where the solid elements' IEN is remapped);
 *   - the element loop of the unified-continuum VMS formulation on linear
 *     tets (fluid residual-based VMS, Sec. 3.2, Eqs. for B_m^f, B_p^f, v', p',
 *     tau_M, tau_C, G with the matrix M; solid VMS, Sec. 3.1 with
 *     tau_M^s = c_m dx/(c rho), tau_C^s = c_c c dx rho), 4-point Gauss rule;
 *   - the consistent tangent of the first-order generalized-alpha scheme
 *     (Sec. 3.5, K = alpha_m dR/d(ydot) + alpha_f gamma dt dR/dy, tau frozen)
 *     reduced to the 2x2 velocity-pressure blocks A, B, C, D of Sec. 3.5
 *     (fluid and solid definitions), and the residual right-hand side;
 *   - the harmonic-extension mesh-motion Laplacian (B_k^f, Sec. 3.2) on the
 *     fluid nodes with its Dirichlet data (Sec. 2.3: interface displacement,
 *     zero at inlet and outlet).
 *
 * All random draws come from splitmix64 (Steele, Lea, Flood 2014) keyed by
 * the seed and a counter.  Assembly is deterministic: element contributions
 * are added to each matrix row in element order, whatever the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* parameters                                                          */
/* ------------------------------------------------------------------ */
typedef struct {
  int kind;      /* 0 straight tube, 1 stenosed tube, 2 bifurcation        */
  int n_circ;    /* nodes around the circumference                         */
  int n_rad_f;   /* radial node rings in the lumen (the last is the wall)  */
  int n_rad_s;   /* radial node rings in the vessel wall                   */
  int n_ax;      /* axial element layers                                   */
  int fluid_only;/* 1: rigid wall, no solid elements, no-slip lumen wall   */
  double R, wall, L, sten_sigma, sten_frac;
  double rho_f, mu_f, rho_s, E_s, nu_s;
  double dt, rho_inf;
  double u_max, pert_amp, mesh_amp;
  double c_m_solid, c_c_solid;
  uint64_t seed;
  /* kind 2 (bifurcation): half-angle between each daughter's axis and the
     parent's (degrees), daughter length along its axis, element layers of
     the solid carina tip */
  double bif_angle_deg, bif_daughter_len;
  int bif_tip_layers;
  /* kind 2: the last bif_bl_layers lumen-ring intervals next to the wall
     shrink geometrically by bif_bl_ratio each (0: uniform rings) */
  int bif_bl_layers;
  double bif_bl_ratio;
} tg_params;

typedef struct {
  int n_sec, n_nodes, n_elem, n_iface, n_p, n_fluid;
  double *xyz;            /* n_nodes*3                                  */
  int *ring, *layer, *sec;/* per node                                   */
  int *ien;               /* n_elem*4 velocity (node) connectivity      */
  int *pien;              /* n_elem*4 pressure-index connectivity       */
  unsigned char *etype;   /* 0 fluid, 1 solid                           */
  int *iface_of;          /* node -> interface ordinal or -1            */
  int *fluid_id;          /* node -> fluid-node ordinal or -1           */
  unsigned char *dir_v;   /* velocity Dirichlet flag per node           */
  unsigned char *dir_m;   /* mesh Dirichlet flag per fluid node         */
} tg_mesh;

typedef struct {
  int nb_rows, nb_cols, br, bc, nnzb;
  int *row_ptr, *col;
  double *val;
} tg_bsr;

void tg_default_params(tg_params *p) {
  memset(p, 0, sizeof(*p));
  p->kind = 0;
  p->n_circ = 24; p->n_rad_f = 4; p->n_rad_s = 2; p->n_ax = 40;
  p->R = 0.3; p->wall = 0.06; p->L = 5.0;
  p->sten_sigma = 0.6; p->sten_frac = 1.0 - 1.0 / sqrt(2.0);
  p->rho_f = 1.06; p->mu_f = 0.04;
  p->rho_s = 1.0; p->E_s = 4.0e6; p->nu_s = 0.5;
  p->dt = 1.0e-4; p->rho_inf = 0.5;
  p->u_max = 30.0; p->pert_amp = 0.05; p->mesh_amp = 1.0e-3;
  p->c_m_solid = 1.0; p->c_c_solid = 0.0;
  p->seed = 2206;
  p->bif_angle_deg = 35.0; p->bif_daughter_len = 4.0; p->bif_tip_layers = 2;
  p->bif_bl_layers = 0; p->bif_bl_ratio = 0.6;
}

/* generalized-alpha constants of the first-order scheme (Sec. 3.4) */
void tg_genalpha(double rho_inf, double *alpha_m, double *alpha_f, double *gamma) {
  *alpha_m = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf);
  *alpha_f = 1.0 / (1.0 + rho_inf);
  *gamma = 1.0 / (1.0 + rho_inf);
}

/* splitmix64: x += golden gamma; mix */
static uint64_t splitmix64(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
/* uniform in [-1, 1) from the top 53 bits */
static double uniform_pm1(uint64_t *state) {
  return 2.0 * ((double)(splitmix64(state) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

/* lumen radius at axial position z (stenosis: Gaussian bump, sten_frac of R) */
static double lumen_radius(const tg_params *p, double z) {
  if (p->kind == 1) {
    double d = z - 0.5 * p->L;
    return p->R * (1.0 - p->sten_frac * exp(-d * d / (2.0 * p->sten_sigma * p->sten_sigma)));
  }
  return p->R;
}

/* ------------------------------------------------------------------ */
/* mesh                                                                */
/* ------------------------------------------------------------------ */
/* Prism (v0 v1 v2 bottom, v3 v4 v5 top, v_{i+3} above v_i) to 3 tets with
   the minimum-global-index rule of Dompierre et al. (1999): rotate so the
   smallest index sits at position 0, then split the quad face opposite it
   along the diagonal that holds the smaller of its two candidate vertices.
   Every quad face is cut through its smallest vertex, so neighbouring
   prisms agree on the shared face whatever the numbering. */
static const int PRISM_ROT[6][6] = {
    {0, 1, 2, 3, 4, 5}, {1, 2, 0, 4, 5, 3}, {2, 0, 1, 5, 3, 4},
    {3, 5, 4, 0, 2, 1}, {4, 3, 5, 1, 0, 2}, {5, 4, 3, 2, 1, 0}};

static void split_prism(const int v[6], int tets[3][4]) {
  int m = 0;
  for (int i = 1; i < 6; ++i)
    if (v[i] < v[m]) m = i;
  int w[6];
  for (int i = 0; i < 6; ++i) w[i] = v[PRISM_ROT[m][i]];
  int a = w[1] < w[5] ? w[1] : w[5];
  int b = w[2] < w[4] ? w[2] : w[4];
  if (a < b) { /* diagonal w1-w5 */
    int t[3][4] = {{w[0], w[1], w[2], w[5]}, {w[0], w[1], w[5], w[4]}, {w[0], w[4], w[5], w[3]}};
    memcpy(tets, t, sizeof(t));
  } else {     /* diagonal w2-w4 */
    int t[3][4] = {{w[0], w[1], w[2], w[4]}, {w[0], w[4], w[2], w[5]}, {w[0], w[4], w[5], w[3]}};
    memcpy(tets, t, sizeof(t));
  }
}

void tg_mesh_free(tg_mesh *m) {
  if (!m) return;
  free(m->xyz); free(m->ring); free(m->layer); free(m->sec);
  free(m->ien); free(m->pien); free(m->etype);
  free(m->iface_of); free(m->fluid_id); free(m->dir_v); free(m->dir_m);
  free(m);
}

/* ------------------------------------------------------------------ */
/* bifurcation (kind 2)                                                */
/* ------------------------------------------------------------------ */
/* One cross-section is extruded along z and its cells change class per
   element layer.  The section is an O-grid of the parent: a square core of
   NC x NC cells (half-width h = 0.6 R / sqrt 2) and rings along rays from
   the origin, NRF lumen rings from the square to the lumen circle R and NRS
   wall rings out to R + wall.  A septum band of core columns through the
   middle, [c0, c3), and the ring cells over it split the section into side
   A | wall A [c0, c1) | void [c1, c2) | wall B [c2, c3) | side B.
     parent layers  (k < k_tip):        the band is lumen (its wall-ring
                                         cells stay wall): a round tube;
     carina tip     (k_tip <= k < k_dau): the whole band is solid;
     daughters      (k >= k_dau):        void cells are removed, wall A / B
                                         become the daughters' inner walls.
   Each daughter keeps its half of the parent section (a half-disk lumen
   with its wall) and is sheared sideways, x -/+= (z - z_dau) tan(angle):
   a shear has determinant 1, so every tet keeps its volume and its
   orientation.  Nodes that only removed cells use are dropped. */
#define BIF_MAX_RINGS 256
typedef struct {
  int NC, NRF, NRS, NR, ncore, nsec;
  int c0, c1, c2, c3;
  int k_tip, k_dau;
  double h, dz, tan_a, z_dau;
  double frac[BIF_MAX_RINGS + 1]; /* lumen ring q sits at frac[q] of the way from the square to R */
} bif_geom;

static int bif_geom_init(const tg_params *p, bif_geom *g) {
  memset(g, 0, sizeof(*g));
  g->NC = p->n_circ; g->NRF = p->n_rad_f; g->NRS = p->n_rad_s; g->NR = g->NRF + g->NRS;
  if (g->NC < 8 || (g->NC & 1) || g->NRF < 1 || g->NRS < 1 || p->n_ax < 4 || p->fluid_only) return -1;
  if (g->NRF > BIF_MAX_RINGS || p->bif_bl_layers < 0 || p->bif_bl_layers > g->NRF) return -1;
  if (p->bif_bl_layers > 0 && !(p->bif_bl_ratio > 0.0 && p->bif_bl_ratio <= 1.0)) return -1;
  {
    /* interval widths: uniform w inside, then w r, w r^2, ..., w r^nbl next to the wall */
    const int nbl = p->bif_bl_layers;
    double width[BIF_MAX_RINGS], tot = 0.0, f = 1.0;
    for (int q = 0; q < g->NRF; ++q) {
      if (q >= g->NRF - nbl) f *= p->bif_bl_ratio;
      width[q] = f;
      tot += f;
    }
    g->frac[0] = 0.0;
    for (int q = 0; q < g->NRF; ++q)
      g->frac[q + 1] = nbl ? g->frac[q] + width[q] / tot : (double)(q + 1) / g->NRF;
    g->frac[g->NRF] = 1.0;
  }
  g->ncore = (g->NC + 1) * (g->NC + 1);
  g->nsec = g->ncore + g->NR * 4 * g->NC;
  g->h = 0.6 * p->R / sqrt(2.0);
  const double cw = 2.0 * g->h / g->NC;
  int ws = (int)lround(p->wall / cw);
  if (ws < 1) ws = 1;
  g->c1 = g->NC / 2 - 1; g->c2 = g->NC / 2 + 1;
  g->c0 = g->c1 - ws; g->c3 = g->c2 + ws;
  if (g->c0 < 2) return -1;
  const double a = p->bif_angle_deg * M_PI / 180.0;
  g->tan_a = tan(a);
  g->dz = (p->L + p->bif_daughter_len * cos(a)) / p->n_ax;
  g->k_dau = (int)lround(p->L / g->dz);
  g->k_tip = g->k_dau - (p->bif_tip_layers > 0 ? p->bif_tip_layers : 1);
  if (g->k_tip < 1 || g->k_dau >= p->n_ax) return -1;
  g->z_dau = g->k_dau * g->dz;
  return 0;
}

/* perimeter node pp of the core square (counter-clockwise from (0, 0)) */
static void bif_perimeter(const bif_geom *g, int pp, int *i, int *j) {
  const int NC = g->NC;
  pp %= 4 * NC;
  if (pp < NC) { *i = pp; *j = 0; }
  else if (pp < 2 * NC) { *i = NC; *j = pp - NC; }
  else if (pp < 3 * NC) { *i = 3 * NC - pp; *j = NC; }
  else { *i = 0; *j = 4 * NC - pp; }
}

/* section coordinates of section node s, its core column (the column of the
   core node it hangs from) and its ring (0: core) */
static void bif_section_xy(const bif_geom *g, const tg_params *p, int s, double *X, double *Y, int *col,
                           int *ring) {
  const int NC = g->NC;
  int i, j, q = 0;
  if (s < g->ncore) {
    i = s % (NC + 1); j = s / (NC + 1);
    *X = g->h * (2.0 * i / NC - 1.0); *Y = g->h * (2.0 * j / NC - 1.0);
  } else {
    const int r = s - g->ncore;
    q = 1 + r / (4 * NC);
    bif_perimeter(g, r % (4 * NC), &i, &j);
    const double Sx = g->h * (2.0 * i / NC - 1.0), Sy = g->h * (2.0 * j / NC - 1.0);
    const double th = atan2(Sy, Sx);
    if (q <= g->NRF) {
      const double f = g->frac[q];
      *X = Sx + f * (p->R * cos(th) - Sx); *Y = Sy + f * (p->R * sin(th) - Sy);
    } else {
      const double rad = p->R + p->wall * (double)(q - g->NRF) / g->NRS;
      *X = rad * cos(th); *Y = rad * sin(th);
    }
  }
  *col = i; *ring = q;
}

/* -1 side A, +1 side B, 0 the void columns, for a node in core column col */
static int bif_side(const bif_geom *g, int col) { return col <= g->c1 ? -1 : (col >= g->c2 ? 1 : 0); }

/* class of a section cell over core column col (-1: left/right ring cells)
   in element layer k: 0 fluid, 1 solid, 2 removed */
static int bif_class(const bif_geom *g, int k, int col, int base_solid) {
  const int band = col >= g->c0 && col < g->c3;
  if (!band || k < g->k_tip) return base_solid;
  if (k < g->k_dau) return 1;
  if (col >= g->c1 && col < g->c2) return 2;
  return 1;
}

static tg_mesh *bif_mesh_build(const tg_params *p) {
  bif_geom g;
  if (bif_geom_init(p, &g)) return NULL;
  const int NC = g.NC, P4 = 4 * NC, nl = p->n_ax + 1;
  /* section triangles with their column and base class */
  const int ntri = 2 * NC * NC + 2 * P4 * g.NR;
  int *tri = (int *)malloc(sizeof(int) * 3 * ntri);
  int *tcol = (int *)malloc(sizeof(int) * ntri);
  unsigned char *tbase = (unsigned char *)malloc(ntri);
  int t = 0;
  for (int j = 0; j < NC; ++j)
    for (int i = 0; i < NC; ++i) {
      const int a = j * (NC + 1) + i, b = a + 1, c = a + NC + 2, d = a + NC + 1;
      tri[3 * t] = a; tri[3 * t + 1] = b; tri[3 * t + 2] = c; tcol[t] = i; tbase[t++] = 0;
      tri[3 * t] = a; tri[3 * t + 1] = c; tri[3 * t + 2] = d; tcol[t] = i; tbase[t++] = 0;
    }
  for (int q = 0; q < g.NR; ++q)
    for (int pp = 0; pp < P4; ++pp) {
      int i0, j0, i1, j1;
      bif_perimeter(&g, pp, &i0, &j0);
      bif_perimeter(&g, pp + 1, &i1, &j1);
      const int a = q == 0 ? j0 * (NC + 1) + i0 : g.ncore + (q - 1) * P4 + pp;
      const int b = q == 0 ? j1 * (NC + 1) + i1 : g.ncore + (q - 1) * P4 + (pp + 1) % P4;
      const int c = g.ncore + q * P4 + (pp + 1) % P4, d = g.ncore + q * P4 + pp;
      const int col = (j0 == j1) ? (i0 < i1 ? i0 : i1) : -1; /* bottom/top edge cells lie over a column */
      const unsigned char base = (unsigned char)(q >= g.NRF);
      tri[3 * t] = a; tri[3 * t + 1] = b; tri[3 * t + 2] = c; tcol[t] = col; tbase[t++] = base;
      tri[3 * t] = a; tri[3 * t + 1] = c; tri[3 * t + 2] = d; tcol[t] = col; tbase[t++] = base;
    }
  /* elements over candidate node numbers (layer * nsec + section node) */
  long long ne = 0;
  for (int k = 0; k < p->n_ax; ++k)
    for (int q = 0; q < ntri; ++q) ne += bif_class(&g, k, tcol[q], tbase[q]) != 2;
  ne *= 3;
  const long long ncand = (long long)nl * g.nsec;
  int *ien = (int *)malloc(sizeof(int) * 4 * ne);
  unsigned char *et = (unsigned char *)malloc(ne);
  int *newid = (int *)malloc(sizeof(int) * ncand);
  for (long long c = 0; c < ncand; ++c) newid[c] = -1;
  long long e = 0;
  for (int k = 0; k < p->n_ax; ++k)
    for (int q = 0; q < ntri; ++q) {
      const int cls = bif_class(&g, k, tcol[q], tbase[q]);
      if (cls == 2) continue;
      int v[6], tets[3][4];
      for (int i = 0; i < 3; ++i) {
        v[i] = k * g.nsec + tri[3 * q + i];
        v[i + 3] = (k + 1) * g.nsec + tri[3 * q + i];
      }
      split_prism(v, tets);
      for (int i = 0; i < 3; ++i) {
        memcpy(&ien[4 * e], tets[i], sizeof(int) * 4);
        for (int a = 0; a < 4; ++a) newid[tets[i][a]] = 0;
        et[e++] = (unsigned char)cls;
      }
    }
  free(tri); free(tcol); free(tbase);
  /* keep the used candidates, in candidate order (the Dompierre splits
     depend only on the order of the indices, which compaction keeps) */
  int nn = 0;
  for (long long c = 0; c < ncand; ++c)
    if (newid[c] == 0) newid[c] = nn++;
  tg_mesh *m = (tg_mesh *)calloc(1, sizeof(tg_mesh));
  m->n_sec = g.nsec;
  m->n_nodes = nn;
  m->n_elem = (int)ne;
  m->xyz = (double *)malloc(sizeof(double) * 3 * nn);
  m->ring = (int *)malloc(sizeof(int) * nn);
  m->layer = (int *)malloc(sizeof(int) * nn);
  m->sec = (int *)malloc(sizeof(int) * nn);
  for (long long c = 0; c < ncand; ++c) {
    const int n = newid[c];
    if (n < 0) continue;
    const int kn = (int)(c / g.nsec), sidx = (int)(c % g.nsec);
    double X, Y;
    int col, q;
    bif_section_xy(&g, p, sidx, &X, &Y, &col, &q);
    const double z = kn * g.dz;
    const double shift = kn > g.k_dau ? bif_side(&g, col) * (z - g.z_dau) * g.tan_a : 0.0;
    m->xyz[3 * n] = X + shift; m->xyz[3 * n + 1] = Y; m->xyz[3 * n + 2] = z;
    m->ring[n] = q; m->layer[n] = kn; m->sec[n] = sidx;
  }
  m->ien = (int *)malloc(sizeof(int) * 4 * ne);
  m->pien = (int *)malloc(sizeof(int) * 4 * ne);
  m->etype = et;
  for (long long i = 0; i < 4 * ne; ++i) m->ien[i] = newid[ien[i]];
  free(ien); free(newid);
  /* interface: nodes of both fluid and solid elements; fluid nodes */
  unsigned char *hf = (unsigned char *)calloc(nn, 1), *hs = (unsigned char *)calloc(nn, 1);
  for (long long i = 0; i < ne; ++i)
    for (int a = 0; a < 4; ++a) (et[i] ? hs : hf)[m->ien[4 * i + a]] = 1;
  m->iface_of = (int *)malloc(sizeof(int) * nn);
  m->fluid_id = (int *)malloc(sizeof(int) * nn);
  int ni = 0, nf = 0;
  for (int n = 0; n < nn; ++n) {
    m->iface_of[n] = (hf[n] && hs[n]) ? ni++ : -1;
    m->fluid_id[n] = hf[n] ? nf++ : -1;
  }
  m->n_iface = ni; m->n_fluid = nf; m->n_p = nn + ni;
  for (long long i = 0; i < ne; ++i)
    for (int a = 0; a < 4; ++a) {
      const int n = m->ien[4 * i + a];
      m->pien[4 * i + a] = (et[i] == 1 && m->iface_of[n] >= 0) ? nn + m->iface_of[n] : n;
    }
  /* Dirichlet sets: the whole inlet section, the wall (solid nodes) at the
     daughters' outlets; mesh: inlet, outlets and the interface */
  m->dir_v = (unsigned char *)calloc(nn, 1);
  m->dir_m = (unsigned char *)calloc(nf > 0 ? nf : 1, 1);
  for (int n = 0; n < nn; ++n) {
    const int k = m->layer[n];
    m->dir_v[n] = (unsigned char)(k == 0 || (k == p->n_ax && hs[n]));
    if (hf[n]) m->dir_m[m->fluid_id[n]] = (unsigned char)(k == 0 || k == p->n_ax || m->iface_of[n] >= 0);
  }
  free(hf); free(hs);
  return m;
}

tg_mesh *tg_mesh_build(const tg_params *p) {
  if (p->kind == 2) return bif_mesh_build(p);
  tg_mesh *m = (tg_mesh *)calloc(1, sizeof(tg_mesh));
  const int nc = p->n_circ;
  const int nrad = p->fluid_only ? p->n_rad_f : p->n_rad_f + p->n_rad_s;
  const int n_sec = 1 + nc * nrad;
  const int nl = p->n_ax + 1;
  m->n_sec = n_sec;
  m->n_nodes = n_sec * nl;
  m->xyz = (double *)malloc(sizeof(double) * 3 * m->n_nodes);
  m->ring = (int *)malloc(sizeof(int) * m->n_nodes);
  m->layer = (int *)malloc(sizeof(int) * m->n_nodes);
  m->sec = (int *)malloc(sizeof(int) * m->n_nodes);
  for (int k = 0; k < nl; ++k) {
    double z = p->L * (double)k / (double)p->n_ax;
    double Rl = lumen_radius(p, z);
    for (int s = 0; s < n_sec; ++s) {
      int n = k * n_sec + s;
      int r = s == 0 ? 0 : 1 + (s - 1) / nc;
      int j = s == 0 ? 0 : (s - 1) % nc;
      double rad;
      if (r <= p->n_rad_f) rad = Rl * (double)r / (double)p->n_rad_f;
      else rad = Rl + p->wall * (double)(r - p->n_rad_f) / (double)p->n_rad_s;
      double th = 2.0 * M_PI * (double)j / (double)nc;
      m->xyz[3 * n + 0] = rad * cos(th);
      m->xyz[3 * n + 1] = rad * sin(th);
      m->xyz[3 * n + 2] = z;
      m->ring[n] = r; m->layer[n] = k; m->sec[n] = s;
    }
  }
  /* section triangles: centre fan, then two per quad between rings */
  const int ntri = nc + 2 * nc * (nrad - 1);
  int *tri = (int *)malloc(sizeof(int) * 3 * ntri);
  unsigned char *tri_solid = (unsigned char *)malloc(ntri);
  int t = 0;
  for (int j = 0; j < nc; ++j) {
    tri[3 * t] = 0; tri[3 * t + 1] = 1 + j; tri[3 * t + 2] = 1 + (j + 1) % nc;
    tri_solid[t++] = 0;
  }
  for (int r = 1; r < nrad; ++r) {
    for (int j = 0; j < nc; ++j) {
      int a = 1 + (r - 1) * nc + j, b = 1 + (r - 1) * nc + (j + 1) % nc;
      int c = 1 + r * nc + (j + 1) % nc, d = 1 + r * nc + j;
      unsigned char solid = (unsigned char)(r + 1 > p->n_rad_f);
      tri[3 * t] = a; tri[3 * t + 1] = b; tri[3 * t + 2] = c; tri_solid[t++] = solid;
      tri[3 * t] = a; tri[3 * t + 1] = c; tri[3 * t + 2] = d; tri_solid[t++] = solid;
    }
  }
  m->n_elem = 3 * ntri * p->n_ax;
  m->ien = (int *)malloc(sizeof(int) * 4 * m->n_elem);
  m->pien = (int *)malloc(sizeof(int) * 4 * m->n_elem);
  m->etype = (unsigned char *)malloc(m->n_elem);
  int e = 0;
  for (int k = 0; k < p->n_ax; ++k) {
    for (int q = 0; q < ntri; ++q) {
      int v[6];
      for (int i = 0; i < 3; ++i) {
        v[i] = k * n_sec + tri[3 * q + i];
        v[i + 3] = (k + 1) * n_sec + tri[3 * q + i];
      }
      int tets[3][4];
      split_prism(v, tets);
      for (int i = 0; i < 3; ++i) {
        memcpy(&m->ien[4 * e], tets[i], sizeof(int) * 4);
        m->etype[e] = tri_solid[q];
        ++e;
      }
    }
  }
  free(tri); free(tri_solid);
  /* interface ordinals, fluid ordinals, pressure IEN */
  m->iface_of = (int *)malloc(sizeof(int) * m->n_nodes);
  m->fluid_id = (int *)malloc(sizeof(int) * m->n_nodes);
  int ni = 0, nf = 0;
  for (int n = 0; n < m->n_nodes; ++n) {
    int r = m->ring[n];
    m->iface_of[n] = (!p->fluid_only && r == p->n_rad_f) ? ni++ : -1;
    m->fluid_id[n] = r <= p->n_rad_f ? nf++ : -1;
  }
  m->n_iface = ni;
  m->n_fluid = nf;
  m->n_p = m->n_nodes + ni;
  for (int e2 = 0; e2 < m->n_elem; ++e2)
    for (int a = 0; a < 4; ++a) {
      int n = m->ien[4 * e2 + a];
      m->pien[4 * e2 + a] = (m->etype[e2] == 1 && m->iface_of[n] >= 0) ? m->n_nodes + m->iface_of[n] : n;
    }
  /* Dirichlet sets: whole inlet section (fluid inflow profile + fixed wall
     annulus), the wall annulus at the outlet (interface ring included), and
     in the rigid-wall variant the lumen wall ring everywhere. */
  m->dir_v = (unsigned char *)calloc(m->n_nodes, 1);
  m->dir_m = (unsigned char *)calloc(nf > 0 ? nf : 1, 1);
  for (int n = 0; n < m->n_nodes; ++n) {
    int r = m->ring[n], k = m->layer[n];
    int d = 0;
    if (k == 0) d = 1;
    if (k == p->n_ax && r >= p->n_rad_f && !p->fluid_only) d = 1;
    if (p->fluid_only && r == p->n_rad_f) d = 1;
    m->dir_v[n] = (unsigned char)d;
    if (m->fluid_id[n] >= 0) {
      int dm = (k == 0 || k == p->n_ax || r == p->n_rad_f) ? 1 : 0;
      m->dir_m[m->fluid_id[n]] = (unsigned char)dm;
    }
  }
  return m;
}

/* ------------------------------------------------------------------ */
/* state                                                               */
/* ------------------------------------------------------------------ */
/* Poiseuille velocity (peak u_max scaled by the local area for the
   stenosis) plus a smooth seeded perturbation that vanishes at the wall
   and at the inlet/outlet sections; pressure linear in z with the
   Poiseuille gradient -4 mu u_max / R^2, zero at the outlet; the solid is
   at rest (u = v = p = 0); all time derivatives and the mesh velocity are
   zero (same-Y predictor from a state with zero rates). */
/* Bifurcation state: a Poiseuille-like profile along the local axis (the
   parent's z, each daughter's sheared axis), 1 - r^2 / R^2 in section
   coordinates, in the daughters also ramped to zero over 0.25 R towards the
   inner wall; the same seeded perturbation as the tube; pressure falling
   linearly along the arc length with the parent's Poiseuille gradient;
   interface and solid nodes at rest. */
static void bif_state_init(const tg_params *p, const tg_mesh *m, double *v, double *pr) {
  bif_geom g;
  if (bif_geom_init(p, &g)) return;
  uint64_t st = p->seed;
  double a[3];
  for (int i = 0; i < 3; ++i) a[i] = uniform_pm1(&st);
  const double G = 4.0 * p->mu_f * p->u_max / (p->R * p->R);
  const double ang = p->bif_angle_deg * M_PI / 180.0, ca = cos(ang), sa = sin(ang);
  const double Ltot = p->L + p->bif_daughter_len;
  const double xa = g.h * (2.0 * g.c0 / g.NC - 1.0), xb = g.h * (2.0 * g.c3 / g.NC - 1.0);
  for (int n = 0; n < m->n_nodes; ++n) {
    v[3 * n] = v[3 * n + 1] = v[3 * n + 2] = 0.0;
    pr[n] = 0.0;
    if (m->fluid_id[n] < 0) continue;
    double X, Y;
    int col, q;
    bif_section_xy(&g, p, m->sec[n], &X, &Y, &col, &q);
    const double z = m->xyz[3 * n + 2];
    const int side = m->layer[n] > g.k_dau ? bif_side(&g, col) : 0;
    const double s_arc = z <= g.z_dau ? z : g.z_dau + (z - g.z_dau) / ca;
    pr[n] = G * (Ltot - s_arc);
    if (m->iface_of[n] >= 0) continue;
    double phi = 1.0 - (X * X + Y * Y) / (p->R * p->R);
    if (phi < 0.0) phi = 0.0;
    if (side != 0) {
      double d = side < 0 ? xa - X : X - xb;
      d /= 0.25 * p->R;
      phi *= d < 0.0 ? 0.0 : (d > 1.0 ? 1.0 : d);
    }
    const double dir[3] = {side * sa, 0.0, side ? ca : 1.0};
    for (int k = 0; k < 3; ++k)
      v[3 * n + k] = p->u_max * phi * dir[k] +
                     p->pert_amp * p->u_max * a[k] * sin((double)(k + 1) * M_PI * s_arc / Ltot) * phi;
  }
  for (int i = m->n_nodes; i < m->n_p; ++i) pr[i] = 0.0;
}

void tg_state_init(const tg_params *p, const tg_mesh *m, double *v, double *pr) {
  if (p->kind == 2) {
    bif_state_init(p, m, v, pr);
    return;
  }
  uint64_t st = p->seed;
  double a[3];
  for (int i = 0; i < 3; ++i) a[i] = uniform_pm1(&st);
  const double G = 4.0 * p->mu_f * p->u_max / (p->R * p->R);
  for (int n = 0; n < m->n_nodes; ++n) {
    double x = m->xyz[3 * n], y = m->xyz[3 * n + 1], z = m->xyz[3 * n + 2];
    v[3 * n] = v[3 * n + 1] = v[3 * n + 2] = 0.0;
    pr[n] = 0.0;
    if (m->fluid_id[n] < 0) continue;
    double Rl = lumen_radius(p, z);
    double s = 1.0 - (x * x + y * y) / (Rl * Rl);
    if (s < 0.0) s = 0.0;
    double um = p->u_max * (p->R * p->R) / (Rl * Rl);
    v[3 * n + 2] = um * s;
    for (int k = 0; k < 3; ++k)
      v[3 * n + k] += p->pert_amp * p->u_max * a[k] * sin((double)(k + 1) * M_PI * z / p->L) * s;
    pr[n] = G * (p->L - z);
  }
  for (int i = m->n_nodes; i < m->n_p; ++i) pr[i] = 0.0;
}

/* ------------------------------------------------------------------ */
/* element kernels                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  double V;           /* volume                                */
  double dN[4][3];    /* shape-function gradients              */
  double dxi[3][3];   /* d xi_k / d x_i, rows k = 1..3         */
} tet_geom;

int tg_tet_geom(const double x[4][3], tet_geom *g) {
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) e[k][i] = x[k + 1][i] - x[0][i];
  double c0[3] = {e[1][1] * e[2][2] - e[1][2] * e[2][1], e[1][2] * e[2][0] - e[1][0] * e[2][2],
                  e[1][0] * e[2][1] - e[1][1] * e[2][0]};
  double c1[3] = {e[2][1] * e[0][2] - e[2][2] * e[0][1], e[2][2] * e[0][0] - e[2][0] * e[0][2],
                  e[2][0] * e[0][1] - e[2][1] * e[0][0]};
  double c2[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                  e[0][0] * e[1][1] - e[0][1] * e[1][0]};
  double det = e[0][0] * c0[0] + e[0][1] * c0[1] + e[0][2] * c0[2];
  if (det == 0.0) return -1;
  for (int i = 0; i < 3; ++i) {
    g->dxi[0][i] = c0[i] / det;
    g->dxi[1][i] = c1[i] / det;
    g->dxi[2][i] = c2[i] / det;
  }
  for (int i = 0; i < 3; ++i) {
    g->dN[1][i] = g->dxi[0][i];
    g->dN[2][i] = g->dxi[1][i];
    g->dN[3][i] = g->dxi[2][i];
    g->dN[0][i] = -(g->dN[1][i] + g->dN[2][i] + g->dN[3][i]);
  }
  g->V = fabs(det) / 6.0;
  return 0;
}

/* metric tensor G_ij = sum_kl dxi_k/dx_i M_kl dxi_l/dx_j with
   M = 2^(1/3)/2 [[2,1,1],[1,2,1],[1,1,2]] (Sec. 3.2) */
void tg_metric(const double dxi[3][3], double G[3][3]) {
  const double c = 0.5 * cbrt(2.0);
  const double M[3][3] = {{2 * c, c, c}, {c, 2 * c, c}, {c, c, 2 * c}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += dxi[k][i] * M[k][l] * dxi[l][j];
      G[i][j] = s;
    }
}

/* fluid stabilisation parameters (Sec. 3.2) */
void tg_tau_fluid(const double G[3][3], const double u[3], double rho, double mu, double dt,
                  double *tauM, double *tauC) {
  const double CT = 4.0, CI = 36.0;
  double uGu = 0.0, GG = 0.0, trG = G[0][0] + G[1][1] + G[2][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      uGu += u[i] * G[i][j] * u[j];
      GG += G[i][j] * G[i][j];
    }
  double nu = mu / rho;
  *tauM = 1.0 / (rho * sqrt(CT / (dt * dt) + uGu + CI * nu * nu * GG));
  *tauC = 1.0 / (*tauM * trG);
}

/* diameter of the circumscribed sphere */
double tg_circum_diameter(const double x[4][3]) {
  double Amat[3][3], b[3];
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
      Amat[k][i] = 2.0 * (x[k + 1][i] - x[0][i]);
      s += x[k + 1][i] * x[k + 1][i] - x[0][i] * x[0][i];
    }
    b[k] = s;
  }
  double det = Amat[0][0] * (Amat[1][1] * Amat[2][2] - Amat[1][2] * Amat[2][1]) -
               Amat[0][1] * (Amat[1][0] * Amat[2][2] - Amat[1][2] * Amat[2][0]) +
               Amat[0][2] * (Amat[1][0] * Amat[2][1] - Amat[1][1] * Amat[2][0]);
  double c[3];
  for (int col = 0; col < 3; ++col) {
    double Mc[3][3];
    memcpy(Mc, Amat, sizeof(Mc));
    for (int r = 0; r < 3; ++r) Mc[r][col] = b[r];
    c[col] = (Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
              Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
              Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0])) / det;
  }
  double r2 = 0.0;
  for (int i = 0; i < 3; ++i) r2 += (c[i] - x[0][i]) * (c[i] - x[0][i]);
  return 2.0 * sqrt(r2);
}

/* 4-point Gauss rule on the tet: barycentric (a,b,b,b) and permutations,
   a = (5+3 sqrt5)/20, b = (5-sqrt5)/20, each weight V/4 */
static void gauss_N(double N[4][4]) {
  const double ga = (5.0 + 3.0 * sqrt(5.0)) / 20.0, gb = (5.0 - sqrt(5.0)) / 20.0;
  for (int q = 0; q < 4; ++q)
    for (int a = 0; a < 4; ++a) N[q][a] = (a == q) ? ga : gb;
}
void tg_gauss_points(double N[4][4]) { gauss_N(N); }

typedef struct {
  double Ae[4][4][3][3]; /* [a][b][i][k]: momentum row (a,i), velocity col (b,k) */
  double Be[4][4][3];    /* [a][b][i]:    momentum row (a,i), pressure col b     */
  double Ce[4][4][3];    /* [a][b][k]:    mass row a, velocity col (b,k)         */
  double De[4][4];       /* [a][b]                                              */
  double Rm[4][3];
  double Rp[4];
} elem_out;

/* Fluid element.  Unknown increments are (vdot, pdot) at t_{n+1}; through
   the generalized-alpha chain rule vdot_{n+am} moves by cm and
   v_{n+af}, p_{n+af} by cf = alpha_f gamma dt.  tau is evaluated at the
   state (tau_mode 0), also written to tau[4][2] (mode 1), or read from
   tau[4][2] (mode 2: frozen, for finite-difference checks). */
void tg_fluid_element(const double x[4][3], const double v[4][3], const double vhat[4][3],
                      const double p[4], const double vd[4][3], double rho, double mu, double dt,
                      double cm, double cf, int tau_mode, double *tau, int want_mat,
                      elem_out *out) {
  tet_geom g;
  memset(out, 0, sizeof(*out));
  if (tg_tet_geom(x, &g)) return;
  double G[3][3];
  tg_metric(g.dxi, G);
  double Nq[4][4];
  gauss_N(Nq);
  const double w = g.V / 4.0;
  const double (*dN)[3] = g.dN;
  double gradv[3][3], gradp[3], div = 0.0;
  for (int i = 0; i < 3; ++i) {
    gradp[i] = 0.0;
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int a = 0; a < 4; ++a) s += v[a][i] * dN[a][j];
      gradv[i][j] = s;
    }
    for (int a = 0; a < 4; ++a) gradp[i] += p[a] * dN[a][i];
  }
  div = gradv[0][0] + gradv[1][1] + gradv[2][2];
  double sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) sig[i][j] = mu * (gradv[i][j] + gradv[j][i]) - (i == j ? 2.0 * mu * div / 3.0 : 0.0);
  double dNdN[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) dNdN[a][b] = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2];

  for (int q = 0; q < 4; ++q) {
    const double *N = Nq[q];
    double vq[3], uq[3], vdq[3], pq = 0.0;
    for (int i = 0; i < 3; ++i) {
      vq[i] = uq[i] = vdq[i] = 0.0;
      for (int a = 0; a < 4; ++a) {
        vq[i] += N[a] * v[a][i];
        uq[i] += N[a] * (v[a][i] - vhat[a][i]);
        vdq[i] += N[a] * vd[a][i];
      }
    }
    for (int a = 0; a < 4; ++a) pq += N[a] * p[a];
    double tauM, tauC;
    if (tau_mode == 2) {
      tauM = tau[2 * q]; tauC = tau[2 * q + 1];
    } else {
      tg_tau_fluid(G, uq, rho, mu, dt, &tauM, &tauC);
      if (tau_mode == 1) { tau[2 * q] = tauM; tau[2 * q + 1] = tauC; }
    }
    /* coarse-scale momentum residual (div sigma_dev vanishes for P1) */
    double rM[3], vp[3];
    for (int i = 0; i < 3; ++i) {
      double adv = 0.0;
      for (int j = 0; j < 3; ++j) adv += gradv[i][j] * uq[j];
      rM[i] = rho * (vdq[i] + adv) + gradp[i];
      vp[i] = -tauM * rM[i];
    }
    const double pp = -tauC * div;
    double dNu[4], dNvp[4];
    for (int a = 0; a < 4; ++a) {
      dNu[a] = dN[a][0] * uq[0] + dN[a][1] * uq[1] + dN[a][2] * uq[2];
      dNvp[a] = dN[a][0] * vp[0] + dN[a][1] * vp[1] + dN[a][2] * vp[2];
    }
    double gvvp[3];
    for (int i = 0; i < 3; ++i) gvvp[i] = gradv[i][0] * vp[0] + gradv[i][1] * vp[1] + gradv[i][2] * vp[2];
    /* residual */
    for (int a = 0; a < 4; ++a) {
      for (int i = 0; i < 3; ++i) {
        double s = N[a] * (rM[i] - gradp[i]) - dN[a][i] * (pq + pp);
        for (int j = 0; j < 3; ++j) s += dN[a][j] * sig[i][j];
        s += -rho * vp[i] * dNu[a] + rho * N[a] * gvvp[i] - rho * vp[i] * dNvp[a];
        out->Rm[a][i] += w * s;
      }
      out->Rp[a] += w * (N[a] * div - dNvp[a]);
    }
    if (!want_mat) continue;
    /* velocity columns (b,k) */
    for (int b = 0; b < 4; ++b) {
      for (int k = 0; k < 3; ++k) {
        double drM[3], dvp[3];
        for (int i = 0; i < 3; ++i) {
          drM[i] = rho * ((i == k ? cm * N[b] + cf * dNu[b] : 0.0) + cf * gradv[i][k] * N[b]);
          dvp[i] = -tauM * drM[i];
        }
        double gvdvp[3];
        for (int i = 0; i < 3; ++i) gvdvp[i] = gradv[i][0] * dvp[0] + gradv[i][1] * dvp[1] + gradv[i][2] * dvp[2];
        double dNbvp = dN[b][0] * vp[0] + dN[b][1] * vp[1] + dN[b][2] * vp[2];
        for (int a = 0; a < 4; ++a) {
          double dNadvp = dN[a][0] * dvp[0] + dN[a][1] * dvp[1] + dN[a][2] * dvp[2];
          for (int i = 0; i < 3; ++i) {
            double s = N[a] * drM[i];
            s += tauC * cf * dN[a][i] * dN[b][k];
            s += mu * cf * ((i == k ? dNdN[a][b] : 0.0) + dN[a][k] * dN[b][i]) -
                 (2.0 * mu / 3.0) * cf * dN[a][i] * dN[b][k];
            s += -rho * (dvp[i] * dNu[a] + vp[i] * cf * N[b] * dN[a][k]);
            s += rho * N[a] * ((i == k ? cf * dNbvp : 0.0) + gvdvp[i]);
            s += -rho * (dvp[i] * dNvp[a] + vp[i] * dNadvp);
            out->Ae[a][b][i][k] += w * s;
          }
          out->Ce[a][b][k] += w * (N[a] * cf * dN[b][k] - dNadvp);
        }
      }
      /* pressure column b */
      double dvpP[3];
      for (int i = 0; i < 3; ++i) dvpP[i] = -tauM * cf * dN[b][i];
      double gvdvpP[3];
      for (int i = 0; i < 3; ++i) gvdvpP[i] = gradv[i][0] * dvpP[0] + gradv[i][1] * dvpP[1] + gradv[i][2] * dvpP[2];
      for (int a = 0; a < 4; ++a) {
        double dNadvp = dN[a][0] * dvpP[0] + dN[a][1] * dvpP[1] + dN[a][2] * dvpP[2];
        for (int i = 0; i < 3; ++i) {
          double s = -dN[a][i] * cf * N[b];
          s += -rho * dvpP[i] * dNu[a];
          s += rho * N[a] * gvdvpP[i];
          s += -rho * (dvpP[i] * dNvp[a] + vp[i] * dNadvp);
          out->Be[a][b][i] += w * s;
        }
        out->De[a][b] += w * (-dNadvp);
      }
    }
  }
}

/* Solid element, small-strain deviatoric elasticity linearised at the
   reference state (2 mu_s dev eps), incompressible (beta = 0).  The solid
   2x2 blocks follow Sec. 3.5: A = K_{m,vdot} + (cf/am) K_{m,udot}, i.e. the
   displacement moves by cu = cf^2/am per unit velocity-rate increment. */
void tg_solid_element(const double x[4][3], const double u[4][3], const double v[4][3],
                      const double p[4], const double vd[4][3], double rho, double mu_s,
                      double tauM, double tauC, double cm, double cf, double cu, int want_mat,
                      elem_out *out) {
  tet_geom g;
  memset(out, 0, sizeof(*out));
  if (tg_tet_geom(x, &g)) return;
  double Nq[4][4];
  gauss_N(Nq);
  const double w = g.V / 4.0;
  const double (*dN)[3] = g.dN;
  double gradu[3][3], gradv[3][3], gradp[3];
  for (int i = 0; i < 3; ++i) {
    gradp[i] = 0.0;
    for (int j = 0; j < 3; ++j) {
      double su = 0.0, sv = 0.0;
      for (int a = 0; a < 4; ++a) {
        su += u[a][i] * dN[a][j];
        sv += v[a][i] * dN[a][j];
      }
      gradu[i][j] = su;
      gradv[i][j] = sv;
    }
    for (int a = 0; a < 4; ++a) gradp[i] += p[a] * dN[a][i];
  }
  double divu = gradu[0][0] + gradu[1][1] + gradu[2][2];
  double divv = gradv[0][0] + gradv[1][1] + gradv[2][2];
  double sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      sig[i][j] = mu_s * (gradu[i][j] + gradu[j][i]) - (i == j ? 2.0 * mu_s * divu / 3.0 : 0.0);
  for (int q = 0; q < 4; ++q) {
    const double *N = Nq[q];
    double vdq[3], pq = 0.0;
    for (int i = 0; i < 3; ++i) {
      vdq[i] = 0.0;
      for (int a = 0; a < 4; ++a) vdq[i] += N[a] * vd[a][i];
    }
    for (int a = 0; a < 4; ++a) pq += N[a] * p[a];
    for (int a = 0; a < 4; ++a) {
      for (int i = 0; i < 3; ++i) {
        double s = N[a] * rho * vdq[i] - dN[a][i] * pq + dN[a][i] * tauC * divv;
        for (int j = 0; j < 3; ++j) s += dN[a][j] * sig[i][j];
        out->Rm[a][i] += w * s;
      }
      double s = N[a] * divv;
      for (int j = 0; j < 3; ++j) s += dN[a][j] * tauM * (rho * vdq[j] + gradp[j]);
      out->Rp[a] += w * s;
    }
    if (!want_mat) continue;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double dd = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2];
        for (int i = 0; i < 3; ++i) {
          for (int k = 0; k < 3; ++k) {
            double s = (i == k ? cm * rho * N[a] * N[b] : 0.0);
            s += cu * (mu_s * ((i == k ? dd : 0.0) + dN[a][k] * dN[b][i]) - (2.0 * mu_s / 3.0) * dN[a][i] * dN[b][k]);
            s += cf * tauC * dN[a][i] * dN[b][k];
            out->Ae[a][b][i][k] += w * s;
          }
          out->Be[a][b][i] += w * (-cf * dN[a][i] * N[b]);
          out->Ce[a][b][i] += w * (cf * N[a] * dN[b][i] + cm * tauM * rho * dN[a][i] * N[b]);
        }
        out->De[a][b] += w * (cf * tauM * dd);
      }
  }
}

/* ------------------------------------------------------------------ */
/* sparsity patterns                                                   */
/* ------------------------------------------------------------------ */
static int cmp_int(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  return (x > y) - (x < y);
}

/* rows[e*4+a] -> cols[e*4+b] over elements with mask (NULL = all) */
static void build_pattern(int n_rows, int n_cols, int n_elem, const int *rows, const int *cols,
                          const unsigned char *mask, int *out_nnz, int **out_rp, int **out_col) {
  int *cnt = (int *)calloc(n_rows + 1, sizeof(int));
  for (int e = 0; e < n_elem; ++e) {
    if (mask && !mask[e]) continue;
    for (int a = 0; a < 4; ++a) cnt[rows[4 * e + a] + 1]++;
  }
  for (int r = 0; r < n_rows; ++r) cnt[r + 1] += cnt[r];
  int *inc = (int *)malloc(sizeof(int) * (cnt[n_rows] > 0 ? cnt[n_rows] : 1));
  int *fill = (int *)malloc(sizeof(int) * (n_rows > 0 ? n_rows : 1));
  memcpy(fill, cnt, sizeof(int) * n_rows);
  for (int e = 0; e < n_elem; ++e) {
    if (mask && !mask[e]) continue;
    for (int a = 0; a < 4; ++a) inc[fill[rows[4 * e + a]]++] = e;
  }
  int *rlen = (int *)calloc(n_rows + 1, sizeof(int));
  int maxinc = 0;
  for (int r = 0; r < n_rows; ++r)
    if (cnt[r + 1] - cnt[r] > maxinc) maxinc = cnt[r + 1] - cnt[r];
#pragma omp parallel
  {
    int *buf = (int *)malloc(sizeof(int) * (4 * maxinc + 1));
#pragma omp for schedule(static)
    for (int r = 0; r < n_rows; ++r) {
      int nb = 0;
      for (int t = cnt[r]; t < cnt[r + 1]; ++t)
        for (int b = 0; b < 4; ++b) buf[nb++] = cols[4 * inc[t] + b];
      qsort(buf, nb, sizeof(int), cmp_int);
      int u = 0;
      for (int t = 0; t < nb; ++t)
        if (t == 0 || buf[t] != buf[t - 1]) ++u;
      rlen[r + 1] = u;
    }
    free(buf);
  }
  for (int r = 0; r < n_rows; ++r) rlen[r + 1] += rlen[r];
  int nnz = rlen[n_rows];
  int *col = (int *)malloc(sizeof(int) * (nnz > 0 ? nnz : 1));
#pragma omp parallel
  {
    int *buf = (int *)malloc(sizeof(int) * (4 * maxinc + 1));
#pragma omp for schedule(static)
    for (int r = 0; r < n_rows; ++r) {
      int nb = 0;
      for (int t = cnt[r]; t < cnt[r + 1]; ++t)
        for (int b = 0; b < 4; ++b) buf[nb++] = cols[4 * inc[t] + b];
      qsort(buf, nb, sizeof(int), cmp_int);
      int u = rlen[r];
      for (int t = 0; t < nb; ++t)
        if (t == 0 || buf[t] != buf[t - 1]) col[u++] = buf[t];
    }
    free(buf);
  }
  (void)n_cols;
  free(cnt); free(inc); free(fill);
  *out_nnz = nnz;
  *out_rp = rlen;
  *out_col = col;
}

static int find_col(const int *col, int lo, int hi, int c) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

/* ------------------------------------------------------------------ */
/* assembly                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
  tg_bsr A, B, C, D, L;   /* raw (before boundary conditions) */
  double *Rm, *Rp;        /* n_nodes*3, n_p                    */
} tg_raw;

static void bsr_alloc(tg_bsr *M, int nbr, int nbc, int br, int bc, int nnzb, int *rp, int *col) {
  M->nb_rows = nbr; M->nb_cols = nbc; M->br = br; M->bc = bc; M->nnzb = nnzb;
  M->row_ptr = rp; M->col = col;
  M->val = (double *)calloc((size_t)nnzb * br * bc > 0 ? (size_t)nnzb * br * bc : 1, sizeof(double));
}

void tg_bsr_free(tg_bsr *M) {
  free(M->row_ptr); free(M->col); free(M->val);
  M->row_ptr = NULL; M->col = NULL; M->val = NULL;
}

void tg_raw_free(tg_raw *r) {
  if (!r) return;
  tg_bsr_free(&r->A); tg_bsr_free(&r->B); tg_bsr_free(&r->C); tg_bsr_free(&r->D); tg_bsr_free(&r->L);
  free(r->Rm); free(r->Rp);
  free(r);
}

static int nthreads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
static int thread_id(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

/* Evaluate residual and (optionally) the 2x2 tangent blocks at a state.
   State arrays: v, vhat, vd, u are n_nodes*3; p is n_p.  tau (optional)
   holds 2 values per element and Gauss point for fluid elements and 2 per
   element for solid elements (stride 8 doubles per element). */
tg_raw *tg_assemble(const tg_params *P, const tg_mesh *m, const double *v, const double *vhat,
                    const double *p, const double *vd, const double *u, double cm, double cf,
                    double cu, int tau_mode, double *tau, int want_mat) {
  tg_raw *R = (tg_raw *)calloc(1, sizeof(tg_raw));
  const int nn = m->n_nodes, np = m->n_p, ne = m->n_elem;
  int nnz, *rp, *col;
  if (want_mat) {
    build_pattern(nn, nn, ne, m->ien, m->ien, NULL, &nnz, &rp, &col);
    bsr_alloc(&R->A, nn, nn, 3, 3, nnz, rp, col);
    build_pattern(nn, np, ne, m->ien, m->pien, NULL, &nnz, &rp, &col);
    bsr_alloc(&R->B, nn, np, 3, 1, nnz, rp, col);
    build_pattern(np, nn, ne, m->pien, m->ien, NULL, &nnz, &rp, &col);
    bsr_alloc(&R->C, np, nn, 1, 3, nnz, rp, col);
    build_pattern(np, np, ne, m->pien, m->pien, NULL, &nnz, &rp, &col);
    bsr_alloc(&R->D, np, np, 1, 1, nnz, rp, col);
  }
  R->Rm = (double *)calloc((size_t)nn * 3, sizeof(double));
  R->Rp = (double *)calloc((size_t)np, sizeof(double));
  const double mu_s = P->E_s / (2.0 * (1.0 + P->nu_s));
  const double cs = sqrt(mu_s / P->rho_s); /* shear wave speed */
  const int CH = 32768;
  elem_out *buf = (elem_out *)malloc(sizeof(elem_out) * CH);
  const int T = nthreads();
  for (int e0 = 0; e0 < ne; e0 += CH) {
    int e1 = e0 + CH < ne ? e0 + CH : ne;
#pragma omp parallel for schedule(static)
    for (int e = e0; e < e1; ++e) {
      double x[4][3], ve[4][3], vh[4][3], pe[4], vde[4][3], ue[4][3];
      for (int a = 0; a < 4; ++a) {
        int n = m->ien[4 * e + a];
        for (int i = 0; i < 3; ++i) {
          x[a][i] = m->xyz[3 * n + i];
          ve[a][i] = v[3 * n + i];
          vh[a][i] = vhat ? vhat[3 * n + i] : 0.0;
          vde[a][i] = vd ? vd[3 * n + i] : 0.0;
          ue[a][i] = u ? u[3 * n + i] : 0.0;
        }
        pe[a] = p[m->pien[4 * e + a]];
      }
      double *te = tau ? tau + (size_t)8 * e : NULL;
      if (m->etype[e] == 0) {
        tg_fluid_element(x, ve, vh, pe, vde, P->rho_f, P->mu_f, P->dt, cm, cf, tau ? tau_mode : 0, te,
                         want_mat, &buf[e - e0]);
      } else {
        double dx = tg_circum_diameter(x);
        double tM = P->c_m_solid * dx / (cs * P->rho_s);
        double tC = P->c_c_solid * cs * dx * P->rho_s;
        if (te && tau_mode == 2) { tM = te[0]; tC = te[1]; }
        if (te && tau_mode == 1) { te[0] = tM; te[1] = tC; }
        tg_solid_element(x, ue, ve, pe, vde, P->rho_s, mu_s, tM, tC, cm, cf, cu, want_mat, &buf[e - e0]);
      }
    }
    /* deterministic scatter: each thread owns a contiguous range of rows
       and adds the chunk's contributions in element order */
#pragma omp parallel num_threads(T)
    {
      int t = thread_id(), Tn = nthreads();
#ifdef _OPENMP
      Tn = omp_get_num_threads();
#endif
      int v0 = (int)((long long)nn * t / Tn), v1 = (int)((long long)nn * (t + 1) / Tn);
      int p0 = (int)((long long)np * t / Tn), p1 = (int)((long long)np * (t + 1) / Tn);
      for (int e = e0; e < e1; ++e) {
        const elem_out *o = &buf[e - e0];
        const int *ien = &m->ien[4 * e], *pien = &m->pien[4 * e];
        for (int a = 0; a < 4; ++a) {
          int r = ien[a];
          if (r >= v0 && r < v1) {
            for (int i = 0; i < 3; ++i) R->Rm[3 * r + i] += o->Rm[a][i];
            if (want_mat) {
              for (int b = 0; b < 4; ++b) {
                int pa = find_col(R->A.col, R->A.row_ptr[r], R->A.row_ptr[r + 1], ien[b]);
                double *blk = R->A.val + (size_t)9 * pa;
                for (int i = 0; i < 3; ++i)
                  for (int k = 0; k < 3; ++k) blk[3 * i + k] += o->Ae[a][b][i][k];
                int pb = find_col(R->B.col, R->B.row_ptr[r], R->B.row_ptr[r + 1], pien[b]);
                for (int i = 0; i < 3; ++i) R->B.val[(size_t)3 * pb + i] += o->Be[a][b][i];
              }
            }
          }
          int rpq = pien[a];
          if (rpq >= p0 && rpq < p1) {
            R->Rp[rpq] += o->Rp[a];
            if (want_mat) {
              for (int b = 0; b < 4; ++b) {
                int pc = find_col(R->C.col, R->C.row_ptr[rpq], R->C.row_ptr[rpq + 1], ien[b]);
                for (int k = 0; k < 3; ++k) R->C.val[(size_t)3 * pc + k] += o->Ce[a][b][k];
                int pd = find_col(R->D.col, R->D.row_ptr[rpq], R->D.row_ptr[rpq + 1], pien[b]);
                R->D.val[pd] += o->De[a][b];
              }
            }
          }
        }
      }
    }
  }
  free(buf);
  return R;
}

/* mesh-motion Laplacian L_ab = int grad N_a . grad N_b over fluid elements
   in the reference configuration, rows/cols = fluid-node ordinals */
tg_bsr *tg_mesh_laplacian_raw(const tg_mesh *m) {
  const int ne = m->n_elem, nf = m->n_fluid;
  int *fien = (int *)malloc(sizeof(int) * 4 * (ne > 0 ? ne : 1));
  unsigned char *mask = (unsigned char *)malloc(ne > 0 ? ne : 1);
  for (int e = 0; e < ne; ++e) {
    mask[e] = m->etype[e] == 0;
    for (int a = 0; a < 4; ++a) {
      int f = m->fluid_id[m->ien[4 * e + a]];
      fien[4 * e + a] = f < 0 ? 0 : f;
    }
  }
  int nnz, *rp, *col;
  build_pattern(nf, nf, ne, fien, fien, mask, &nnz, &rp, &col);
  tg_bsr *L = (tg_bsr *)calloc(1, sizeof(tg_bsr));
  bsr_alloc(L, nf, nf, 1, 1, nnz, rp, col);
  /* row-owned deterministic accumulation */
#pragma omp parallel
  {
    int t = thread_id(), Tn = 1;
#ifdef _OPENMP
    Tn = omp_get_num_threads();
#endif
    int r0 = (int)((long long)nf * t / Tn), r1 = (int)((long long)nf * (t + 1) / Tn);
    for (int e = 0; e < ne; ++e) {
      if (!mask[e]) continue;
      int own = 0;
      for (int a = 0; a < 4; ++a)
        if (fien[4 * e + a] >= r0 && fien[4 * e + a] < r1) own = 1;
      if (!own) continue;
      double x[4][3];
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) x[a][i] = m->xyz[3 * m->ien[4 * e + a] + i];
      tet_geom g;
      if (tg_tet_geom(x, &g)) continue;
      for (int a = 0; a < 4; ++a) {
        int r = fien[4 * e + a];
        if (r < r0 || r >= r1) continue;
        for (int b = 0; b < 4; ++b) {
          int pos = find_col(L->col, L->row_ptr[r], L->row_ptr[r + 1], fien[4 * e + b]);
          L->val[pos] += g.V * (g.dN[a][0] * g.dN[b][0] + g.dN[a][1] * g.dN[b][1] + g.dN[a][2] * g.dN[b][2]);
        }
      }
    }
  }
  free(fien); free(mask);
  return L;
}

/* ------------------------------------------------------------------ */
/* boundary conditions                                                 */
/* ------------------------------------------------------------------ */
/* Copy M dropping every block in a row or column flagged by the row/col
   masks (NULL = none) and putting an identity block on flagged diagonal
   rows when set_identity is nonzero. */
static void bsr_dirichlet(const tg_bsr *M, const unsigned char *rmask, const unsigned char *cmask,
                          int set_identity, tg_bsr *out) {
  const int bs = M->br * M->bc;
  int *rp = (int *)malloc(sizeof(int) * (M->nb_rows + 1));
  rp[0] = 0;
  for (int r = 0; r < M->nb_rows; ++r) {
    int c = 0;
    int rd = rmask && rmask[r];
    for (int t = M->row_ptr[r]; t < M->row_ptr[r + 1]; ++t) {
      int cc = M->col[t];
      if (rd) { if (set_identity && cc == r) ++c; continue; }
      if (cmask && cmask[cc]) continue;
      ++c;
    }
    rp[r + 1] = rp[r] + c;
  }
  int nnz = rp[M->nb_rows];
  int *col = (int *)malloc(sizeof(int) * (nnz > 0 ? nnz : 1));
  double *val = (double *)calloc((size_t)(nnz > 0 ? nnz : 1) * bs, sizeof(double));
  for (int r = 0; r < M->nb_rows; ++r) {
    int o = rp[r];
    int rd = rmask && rmask[r];
    for (int t = M->row_ptr[r]; t < M->row_ptr[r + 1]; ++t) {
      int cc = M->col[t];
      if (rd) {
        if (set_identity && cc == r) {
          col[o] = cc;
          for (int i = 0; i < M->br; ++i) val[(size_t)o * bs + i * M->bc + i] = 1.0;
          ++o;
        }
        continue;
      }
      if (cmask && cmask[cc]) continue;
      col[o] = cc;
      memcpy(val + (size_t)o * bs, M->val + (size_t)t * bs, sizeof(double) * bs);
      ++o;
    }
  }
  out->nb_rows = M->nb_rows; out->nb_cols = M->nb_cols; out->br = M->br; out->bc = M->bc;
  out->nnzb = nnz; out->row_ptr = rp; out->col = col; out->val = val;
}

typedef struct {
  tg_bsr A, B, C, D;       /* block Jacobian with boundary conditions   */
  double *b;               /* rhs = -[Rm; Rp], Dirichlet rows zero       */
  tg_bsr L;                /* mesh Laplacian with Dirichlet rows = I     */
  double *mesh_b;          /* n_fluid*3 interleaved                      */
  double *mesh_g;          /* Dirichlet displacement values, n_fluid*3   */
} tg_system;

void tg_system_free(tg_system *s) {
  if (!s) return;
  tg_bsr_free(&s->A); tg_bsr_free(&s->B); tg_bsr_free(&s->C); tg_bsr_free(&s->D); tg_bsr_free(&s->L);
  free(s->b); free(s->mesh_b); free(s->mesh_g);
  free(s);
}

/* Apply boundary conditions to the raw blocks: Dirichlet velocity nodes
   become identity rows of A with zero rows in B and zero columns in A and
   C (increments vanish there); rhs = -R with zeros on Dirichlet rows. */
tg_system *tg_finalize(const tg_mesh *m, const tg_raw *R, const tg_bsr *Lraw, const tg_params *P) {
  tg_system *S = (tg_system *)calloc(1, sizeof(tg_system));
  const int nn = m->n_nodes, np = m->n_p, nf = m->n_fluid;
  bsr_dirichlet(&R->A, m->dir_v, m->dir_v, 1, &S->A);
  bsr_dirichlet(&R->B, m->dir_v, NULL, 0, &S->B);
  bsr_dirichlet(&R->C, NULL, m->dir_v, 0, &S->C);
  bsr_dirichlet(&R->D, NULL, NULL, 0, &S->D);
  S->b = (double *)malloc(sizeof(double) * ((size_t)3 * nn + np));
  for (int n = 0; n < nn; ++n)
    for (int i = 0; i < 3; ++i) S->b[3 * n + i] = m->dir_v[n] ? 0.0 : -R->Rm[3 * n + i];
  for (int q = 0; q < np; ++q) S->b[3 * nn + q] = -R->Rp[q];
  /* mesh motion: Dirichlet data = smooth radial interface displacement
     mesh_amp * sin(pi z / L), zero on inlet/outlet sections */
  if (Lraw && nf > 0) {
    S->mesh_g = (double *)calloc((size_t)3 * nf, sizeof(double));
    bif_geom g;
    const int bif = P->kind == 2 && bif_geom_init(P, &g) == 0;
    for (int n = 0; n < nn; ++n) {
      int f = m->fluid_id[n];
      if (f < 0 || !m->dir_m[f]) continue;
      int k = m->layer[n];
      if (k == 0 || k == P->n_ax) continue;
      double x = m->xyz[3 * n], y = m->xyz[3 * n + 1], z = m->xyz[3 * n + 2];
      double zl = P->L;
      if (bif) {
        /* the lateral wall (the lumen circle's ring, in section coordinates:
           the daughters unsheared); the carina and septum faces stay put */
        if (m->iface_of[n] < 0) continue;
        int col, q;
        bif_section_xy(&g, P, m->sec[n], &x, &y, &col, &q);
        if (q != g.NRF) continue;
        zl = P->n_ax * g.dz;
      } else if (m->ring[n] != P->n_rad_f) {
        continue;
      }
      double r = sqrt(x * x + y * y);
      double a = P->mesh_amp * sin(M_PI * z / zl);
      S->mesh_g[3 * f] = a * x / r;
      S->mesh_g[3 * f + 1] = a * y / r;
    }
    bsr_dirichlet(Lraw, m->dir_m, m->dir_m, 1, &S->L);
    S->mesh_b = (double *)calloc((size_t)3 * nf, sizeof(double));
    for (int r = 0; r < nf; ++r) {
      if (m->dir_m[r]) {
        for (int c = 0; c < 3; ++c) S->mesh_b[3 * r + c] = S->mesh_g[3 * r + c];
        continue;
      }
      for (int t = Lraw->row_ptr[r]; t < Lraw->row_ptr[r + 1]; ++t) {
        int cc = Lraw->col[t];
        if (!m->dir_m[cc]) continue;
        for (int c = 0; c < 3; ++c) S->mesh_b[3 * r + c] -= Lraw->val[t] * S->mesh_g[3 * cc + c];
      }
    }
  }
  return S;
}

/* One call for a whole system at the configured state. */
tg_system *tg_build_system(const tg_params *P, tg_mesh **mesh_out) {
  tg_mesh *m = tg_mesh_build(P);
  double am, af, ga;
  tg_genalpha(P->rho_inf, &am, &af, &ga);
  const double cf = af * ga * P->dt;
  const double cu = cf * cf / am;
  double *v = (double *)malloc(sizeof(double) * 3 * m->n_nodes);
  double *p = (double *)malloc(sizeof(double) * m->n_p);
  tg_state_init(P, m, v, p);
  tg_raw *R = tg_assemble(P, m, v, NULL, p, NULL, NULL, am, cf, cu, 0, NULL, 1);
  tg_bsr *L = P->fluid_only ? NULL : tg_mesh_laplacian_raw(m);
  tg_system *S = tg_finalize(m, R, L, P);
  tg_raw_free(R);
  if (L) { tg_bsr_free(L); free(L); }
  free(v); free(p);
  if (mesh_out) *mesh_out = m;
  else tg_mesh_free(m);
  return S;
}

void tg_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
