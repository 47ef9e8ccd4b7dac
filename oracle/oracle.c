/*
 * Plain FP64 CPU oracle of the fully adaptive MR-LBM time step of
 * Bellotti, Gouarin, Graille, Massot (arXiv 2103.02903).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  Independent of the
 * CUDA library (no shared code, header or table).
 *
 * Everything is dense and literal: each level is a full array, the tree is a
 * set of cells, the reconstruction is computed on every cell of every level,
 * and the transport sums the reconstructed finest values over the sets E and
 * A of Eq. AdaptiveAdvectionPhase cell by cell.  Compiled with
 * -ffp-contract=off so that the encode arithmetic is evaluated exactly as
 * written.
 *
 * Readings of the paper that the code takes (where the paper is silent or
 * inconsistent) are marked "reading:" next to the code they affect.
 *
 * Parity unpinned: none of the functions below is unpinned; see the tests
 * under tests/ (prediction: Table 1, Appendix 2, polynomial exactness,
 * consistency Eq. ConsistencyPrediction; details: Eq. DetailRedundancy;
 * step: epsilon = 0 reduces to Eq. StreamFinest; conservation; Eq.
 * PredictionWithMatrix; brute-force minimal grading; the group norms of
 * the details and the T / H / G decisions in 2D and 3D against a numpy
 * restatement of the set definitions, and the obstacle penalisation
 * against integer lattice counts and the rest equilibrium, in
 * tests/test_oracle_obstacle_and_decisions.py; the exact collision:
 * linear equilibria, finest leaves, mass, closed-form D1Q2 composition in
 * tests/test_oracle_exact_collision.py; the prediction of half-width s = 2,
 * 3 and the grading it widens: Appendix 2 coefficients, exactness to degree
 * 2s and not beyond, consistency, the 2^-(2s+1) decay of details,
 * brute-force minimal grading with the radius-2 stencil, in
 * tests/test_oracle_prediction_s.py).
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define MAXL 24
#define MAXQ 16

struct or_state {
  or_config cfg;
  int d, q, m, Q, ncons;
  int eta[9][3];
  int opp[9];
  double M[9][9], Minv[9][9];
  double srel[4][9];
  int cons_lat[4], cons_mom[4];
  int Jmin, J;
  int s_pred; /* prediction stencil half-width s */
  int n[MAXL][3];
  long long nc[MAXL];
  unsigned char* leaf[MAXL];
  double* val[MAXL];
  double* G[MAXL];
  double last_margin;
};

/* ------------------------------------------------------------------------ */
/* indexing                                                                  */
/* ------------------------------------------------------------------------ */

static long long cidx(const or_state* S, int l, int x, int y, int z) {
  return ((long long)z * S->n[l][1] + y) * S->n[l][0] + x;
}

static int periodic(const or_state* S, int axis) { return S->cfg.bc[2 * axis] == OR_BC_PERIODIC; }

/* Stencil index for the prediction operator.  Reading: outside a non-periodic
 * domain the value of a cell is that of the nearest cell of the same level
 * (constant extension; for s = 1 this is the mirror image). */
static int stencil_coord(const or_state* S, int l, int axis, int v) {
  int N = S->n[l][axis];
  if (axis >= S->d) return 0;
  if (periodic(S, axis)) return ((v % N) + N) % N;
  if (v < 0) return 0;
  if (v >= N) return N - 1;
  return v;
}

/* Neighbour in the mesh-building rules: wrap on periodic axes, -1 outside. */
static int mesh_coord(const or_state* S, int l, int axis, int v) {
  int N = S->n[l][axis];
  if (axis >= S->d) return v == 0 ? 0 : -1;
  if (periodic(S, axis)) return ((v % N) + N) % N;
  if (v < 0 || v >= N) return -1;
  return v;
}

static void cell_coords(const or_state* S, int l, long long c, int* x, int* y, int* z) {
  long long nx = S->n[l][0], ny = S->n[l][1];
  *x = (int)(c % nx);
  *y = (int)((c / nx) % ny);
  *z = (int)(c / (nx * ny));
}

/* ------------------------------------------------------------------------ */
/* schemes (Sec. 7 and the D1 schemes read as in the design notes)           */
/* ------------------------------------------------------------------------ */

static int invert(int n, double A[9][9], double Ainv[9][9]) {
  double a[9][18];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) a[i][j] = j < n ? A[i][j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (fabs(a[piv][col]) < 1e-300) return -1;
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        double t = a[col][j];
        a[col][j] = a[piv][j];
        a[piv][j] = t;
      }
    double inv = 1.0 / a[col][col];
    for (int j = 0; j < 2 * n; ++j) a[col][j] *= inv;
    for (int r = 0; r < n; ++r)
      if (r != col) {
        double f = a[r][col];
        for (int j = 0; j < 2 * n; ++j) a[r][j] -= f * a[col][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i][j] = a[i][j + n];
  return 0;
}

static int setup_scheme(or_state* S) {
  const double L = S->cfg.lambda;
  memset(S->eta, 0, sizeof(S->eta));
  memset(S->M, 0, sizeof(S->M));
  memset(S->srel, 0, sizeof(S->srel));
  switch (S->cfg.scheme) {
    case OR_D1Q2_ADVECTION:
    case OR_D1Q2_BURGERS:
      /* reading: eta = (+1, -1), M = [[1,1],[l,-l]], S = diag(0, s) */
      S->d = 1; S->q = 2; S->m = 1;
      S->eta[0][0] = 1; S->eta[1][0] = -1;
      S->opp[0] = 1; S->opp[1] = 0;
      S->M[0][0] = 1; S->M[0][1] = 1;
      S->M[1][0] = L; S->M[1][1] = -L;
      S->srel[0][1] = S->cfg.s[0];
      S->ncons = 1; S->cons_lat[0] = 0; S->cons_mom[0] = 0;
      break;
    case OR_D1Q3_SHALLOW_WATER:
      /* reading: eta = (0, +1, -1), M = [[1,1,1],[0,l,-l],[0,l^2,l^2]] */
      S->d = 1; S->q = 3; S->m = 1;
      S->eta[1][0] = 1; S->eta[2][0] = -1;
      S->opp[0] = 0; S->opp[1] = 2; S->opp[2] = 1;
      S->M[0][0] = 1; S->M[0][1] = 1; S->M[0][2] = 1;
      S->M[1][1] = L; S->M[1][2] = -L;
      S->M[2][1] = L * L; S->M[2][2] = L * L;
      S->srel[0][2] = S->cfg.s[0];
      S->ncons = 2;
      S->cons_lat[0] = 0; S->cons_mom[0] = 0;
      S->cons_lat[1] = 0; S->cons_mom[1] = 1;
      break;
    case OR_D2Q4x4_EULER: {
      /* Sec. 7.1.2: xi^h = lambda (cos(pi h/2), sin(pi h/2)), M and S_i as printed */
      S->d = 2; S->q = 4; S->m = 4;
      int ex[4] = {1, 0, -1, 0}, ey[4] = {0, 1, 0, -1};
      for (int h = 0; h < 4; ++h) { S->eta[h][0] = ex[h]; S->eta[h][1] = ey[h]; }
      S->opp[0] = 2; S->opp[1] = 3; S->opp[2] = 0; S->opp[3] = 1;
      double row[4][4] = {{1, 1, 1, 1}, {L, 0, -L, 0}, {0, L, 0, -L}, {L * L, -L * L, L * L, -L * L}};
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) S->M[i][j] = row[i][j];
      for (int i = 0; i < 4; ++i) {
        S->srel[i][1] = S->cfg.s[i];
        S->srel[i][2] = S->cfg.s[i];
        S->srel[i][3] = S->cfg.s[4 + i];
      }
      S->ncons = 4;
      for (int i = 0; i < 4; ++i) { S->cons_lat[i] = i; S->cons_mom[i] = 0; }
      break;
    }
    case OR_D2Q9_NS: {
      /* Sec. 7.2.2, Lallemand-Luo.  Reading: diagonal logical velocities are
       * (+-1, +-1) (the printed magnitude lambda is a misprint). */
      S->d = 2; S->q = 9; S->m = 1;
      int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
      for (int h = 0; h < 9; ++h) { S->eta[h][0] = ex[h]; S->eta[h][1] = ey[h]; }
      int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
      for (int h = 0; h < 9; ++h) S->opp[h] = op[h];
      double L2 = L * L, L3 = L2 * L, L4 = L2 * L2;
      double row[9][9] = {
          {1, 1, 1, 1, 1, 1, 1, 1, 1},
          {0, L, 0, -L, 0, L, -L, -L, L},
          {0, 0, L, 0, -L, L, L, -L, -L},
          {-4 * L2, -L2, -L2, -L2, -L2, 2 * L2, 2 * L2, 2 * L2, 2 * L2},
          {0, -2 * L3, 0, 2 * L3, 0, L3, -L3, -L3, L3},
          {0, 0, -2 * L3, 0, 2 * L3, L3, L3, -L3, -L3},
          {4 * L4, -2 * L4, -2 * L4, -2 * L4, -2 * L4, L4, L4, L4, L4},
          {0, L2, -L2, L2, -L2, 0, 0, 0, 0},
          {0, 0, 0, 0, 0, L2, -L2, L2, -L2}};
      for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) S->M[i][j] = row[i][j];
      for (int r = 3; r <= 6; ++r) S->srel[0][r] = S->cfg.s[0];
      S->srel[0][7] = S->cfg.s[1];
      S->srel[0][8] = S->cfg.s[1];
      S->ncons = 3;
      for (int i = 0; i < 3; ++i) { S->cons_lat[i] = 0; S->cons_mom[i] = i; }
      break;
    }
    case OR_D3Q6_ADVECTION: {
      /* Sec. 7.3: xi^h = lambda (+-e_x, +-e_y, +-e_z), M as printed,
       * S = diag(0, s1, s1, s1, s2, s2) with s1 = s[0], s2 = s[1] */
      S->d = 3; S->q = 6; S->m = 1;
      for (int h = 0; h < 6; ++h) S->eta[h][h / 2] = (h & 1) ? -1 : 1;
      int op[6] = {1, 0, 3, 2, 5, 4};
      for (int h = 0; h < 6; ++h) S->opp[h] = op[h];
      double L2 = L * L;
      double row[6][6] = {{1, 1, 1, 1, 1, 1},     {L, -L, 0, 0, 0, 0},       {0, 0, L, -L, 0, 0},
                          {0, 0, 0, 0, L, -L},     {L2, L2, -L2, -L2, 0, 0},  {L2, L2, 0, 0, -L2, -L2}};
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) S->M[i][j] = row[i][j];
      for (int r = 1; r <= 3; ++r) S->srel[0][r] = S->cfg.s[0];
      S->srel[0][4] = S->cfg.s[1];
      S->srel[0][5] = S->cfg.s[1];
      S->ncons = 1;
      S->cons_lat[0] = 0; S->cons_mom[0] = 0;
      break;
    }
    default:
      return -1;
  }
  S->Q = S->q * S->m;
  return invert(S->q, S->M, S->Minv);
}

/* Equilibrium moments m^eq(conserved), per lattice [m][q]. */
static void equilibrium(const or_state* S, const double* u, double meq[4][9]) {
  memset(meq, 0, sizeof(double) * 4 * 9);
  const double* ph = S->cfg.phys;
  switch (S->cfg.scheme) {
    case OR_D1Q2_ADVECTION:
      meq[0][0] = u[0];
      meq[0][1] = ph[0] * u[0];
      break;
    case OR_D1Q2_BURGERS:
      meq[0][0] = u[0];
      meq[0][1] = 0.5 * u[0] * u[0];
      break;
    case OR_D1Q3_SHALLOW_WATER: {
      double h = u[0], qq = u[1], g = ph[0];
      meq[0][0] = h;
      meq[0][1] = qq;
      meq[0][2] = qq * qq / h + 0.5 * g * h * h;
      break;
    }
    case OR_D2Q4x4_EULER: {
      /* Sec. 7.1.1 fluxes with E = p/(gamma-1) + rho |v|^2 / 2 */
      double rho = u[0], mx = u[1], my = u[2], E = u[3], gam = ph[0];
      double vx = mx / rho, vy = my / rho;
      double p = (gam - 1.0) * (E - 0.5 * (mx * vx + my * vy));
      double fx[4] = {mx, mx * vx + p, my * vx, vx * (E + p)};
      double fy[4] = {my, mx * vy, my * vy + p, vy * (E + p)};
      for (int i = 0; i < 4; ++i) {
        meq[i][0] = u[i];
        meq[i][1] = fx[i];
        meq[i][2] = fy[i];
        meq[i][3] = 0.0;
      }
      break;
    }
    case OR_D3Q6_ADVECTION:
      /* Sec. 7.3: m^eq = (u, V_x u, V_y u, V_z u, 0, 0), V = phys[0..2] */
      meq[0][0] = u[0];
      meq[0][1] = ph[0] * u[0];
      meq[0][2] = ph[1] * u[0];
      meq[0][3] = ph[2] * u[0];
      break;
    case OR_D2Q9_NS: {
      /* Sec. 7.2.2.  Reading: the printed |q|/rho terms are |q|^2/rho and the
       * c_s^4 term carries rho (Lallemand-Luo at lambda = 1). */
      double rho = u[0], qx = u[1], qy = u[2];
      double cs2 = S->cfg.lambda * S->cfg.lambda / 3.0;
      double q2 = qx * qx + qy * qy;
      meq[0][0] = rho;
      meq[0][1] = qx;
      meq[0][2] = qy;
      meq[0][3] = 3.0 * (-2.0 * cs2 * rho + q2 / rho);
      meq[0][4] = -3.0 * cs2 * qx;
      meq[0][5] = -3.0 * cs2 * qy;
      meq[0][6] = 9.0 * (cs2 * cs2 * rho - cs2 * q2 / rho);
      meq[0][7] = (qx * qx - qy * qy) / rho;
      meq[0][8] = qx * qy / rho;
      break;
    }
  }
}

static void moments(const or_state* S, const double* f, double mo[4][9]) {
  for (int i = 0; i < S->m; ++i)
    for (int r = 0; r < S->q; ++r) {
      double acc = 0.0;
      for (int h = 0; h < S->q; ++h) acc += S->M[r][h] * f[i * S->q + h];
      mo[i][r] = acc;
    }
}

static void from_moments(const or_state* S, double mo[4][9], double* f) {
  for (int i = 0; i < S->m; ++i)
    for (int h = 0; h < S->q; ++h) {
      double acc = 0.0;
      for (int r = 0; r < S->q; ++r) acc += S->Minv[h][r] * mo[i][r];
      f[i * S->q + h] = acc;
    }
}

static void conserved_of(const or_state* S, double mo[4][9], double* u) {
  for (int k = 0; k < S->ncons; ++k) u[k] = mo[S->cons_lat[k]][S->cons_mom[k]];
}

/* Eq. CollisionOnFinest / Eq. AdaptiveCollision applied to one cell. */
static void collide_cell(const or_state* S, double* f) {
  double mo[4][9], meq[4][9], u[4];
  moments(S, f, mo);
  conserved_of(S, mo, u);
  equilibrium(S, u, meq);
  for (int i = 0; i < S->m; ++i)
    for (int r = 0; r < S->q; ++r) {
      double s = S->srel[i][r];
      mo[i][r] = (1.0 - s) * mo[i][r] + s * meq[i][r];
    }
  from_moments(S, mo, f);
}

static void equilibrium_populations(const or_state* S, const double* u, double* f) {
  double meq[4][9];
  equilibrium(S, u, meq);
  from_moments(S, meq, f);
}

/* ------------------------------------------------------------------------ */
/* multiresolution operators (Sec. 4)                                        */
/* ------------------------------------------------------------------------ */

/* Table 1: c_1 .. c_s of the centred prediction of stencil half-width s. */
static const double CTAB[4][3] = {
    {0.0, 0.0, 0.0},
    {-1.0 / 8.0, 0.0, 0.0},
    {-22.0 / 128.0, 3.0 / 128.0, 0.0},
    {-201.0 / 1024.0, 11.0 / 256.0, -5.0 / 1024.0},
};
static const double C1 = -0.125; /* s = 1 */

double or_prediction_coefficient(void) { return C1; }

int or_prediction_coefficients(int s, double* out) {
  if (s < 1 || s > 3) return -1;
  for (int i = 0; i < s; ++i) out[i] = CTAB[s][i];
  return 0;
}

/* Prediction operator of Sec. 4.1 on a (2s+1)^d stencil v (x fastest) for
 * the child delta: the one-dimensional sums along each axis, the products
 * c_a c_b over the diagonals of each pair of axes and, in 3D, c_a c_b c_t
 * over the cube's diagonals (the tensor-product construction of Bihari and
 * Harten that Sec. 4.1 states for general s).  Every sum starts from its
 * (1, 1, 1) term, so that s = 1 evaluates exactly the expressions of the
 * 3^d formulas.  Reading: the diagonal (pair) term enters with the sign of
 * the tensor product of the one-dimensional operator, cross_sign = +1 (the
 * construction of Appendix 2 and the exactness on polynomials of degree 2s);
 * cross_sign = -1 reproduces the sign printed in the formula and Fig. 2. */
static double predict_stencil_s(int d, int cross_sign, int s, const double* v, int dx, int dy, int dz) {
  const double* c = CTAB[s];
  const int w = 2 * s + 1;
  double sx = dx ? -1.0 : 1.0, sy = dy ? -1.0 : 1.0, sz = dz ? -1.0 : 1.0;
  double cs = (double)cross_sign;
  if (d == 1) {
#define V1(a) v[(a) + s]
    double qx = c[0] * (V1(1) - V1(-1));
    for (int a = 2; a <= s; ++a) qx = qx + c[a - 1] * (V1(a) - V1(-a));
    return V1(0) + sx * qx;
#undef V1
  }
  if (d == 2) {
#define V2(a, b) v[((b) + s) * w + ((a) + s)]
    double qx = c[0] * (V2(1, 0) - V2(-1, 0));
    double qy = c[0] * (V2(0, 1) - V2(0, -1));
    for (int a = 2; a <= s; ++a) {
      qx = qx + c[a - 1] * (V2(a, 0) - V2(-a, 0));
      qy = qy + c[a - 1] * (V2(0, a) - V2(0, -a));
    }
    double q2 = 0.0;
    for (int b = 1; b <= s; ++b)
      for (int a = 1; a <= s; ++a) {
        double t = (c[a - 1] * c[b - 1]) * (((V2(a, b) - V2(-a, b)) - V2(a, -b)) + V2(-a, -b));
        q2 = (a == 1 && b == 1) ? t : q2 + t;
      }
    double t = V2(0, 0);
    t = t + sx * qx;
    t = t + sy * qy;
    t = t + (cs * sx * sy) * q2;
    return t;
#undef V2
  }
  {
#define V3(a, b, e) v[(((e) + s) * w + ((b) + s)) * w + ((a) + s)]
    double qx = c[0] * (V3(1, 0, 0) - V3(-1, 0, 0));
    double qy = c[0] * (V3(0, 1, 0) - V3(0, -1, 0));
    double qz = c[0] * (V3(0, 0, 1) - V3(0, 0, -1));
    for (int a = 2; a <= s; ++a) {
      qx = qx + c[a - 1] * (V3(a, 0, 0) - V3(-a, 0, 0));
      qy = qy + c[a - 1] * (V3(0, a, 0) - V3(0, -a, 0));
      qz = qz + c[a - 1] * (V3(0, 0, a) - V3(0, 0, -a));
    }
    double qxy = 0.0, qxz = 0.0, qyz = 0.0, q3 = 0.0;
    for (int b = 1; b <= s; ++b)
      for (int a = 1; a <= s; ++a) {
        const double cc = c[a - 1] * c[b - 1];
        const int first = a == 1 && b == 1;
        double t;
        t = cc * (((V3(a, b, 0) - V3(-a, b, 0)) - V3(a, -b, 0)) + V3(-a, -b, 0));
        qxy = first ? t : qxy + t;
        t = cc * (((V3(a, 0, b) - V3(-a, 0, b)) - V3(a, 0, -b)) + V3(-a, 0, -b));
        qxz = first ? t : qxz + t;
        t = cc * (((V3(0, a, b) - V3(0, -a, b)) - V3(0, a, -b)) + V3(0, -a, -b));
        qyz = first ? t : qyz + t;
      }
    for (int e = 1; e <= s; ++e)
      for (int b = 1; b <= s; ++b)
        for (int a = 1; a <= s; ++a) {
          double t = (c[a - 1] * c[b - 1] * c[e - 1]) *
                     (((((((V3(a, b, e) - V3(-a, b, e)) - V3(a, -b, e)) - V3(a, b, -e)) + V3(-a, -b, e)) +
                        V3(-a, b, -e)) +
                       V3(a, -b, -e)) -
                      V3(-a, -b, -e));
          q3 = (a == 1 && b == 1 && e == 1) ? t : q3 + t;
        }
    double t = V3(0, 0, 0);
    t = t + sx * qx;
    t = t + sy * qy;
    t = t + sz * qz;
    t = t + (cs * sx * sy) * qxy;
    t = t + (cs * sx * sz) * qxz;
    t = t + (cs * sy * sz) * qyz;
    t = t + (sx * sy * sz) * q3;
    return t;
#undef V3
  }
}

int or_predict_children(int d, int cross_sign, const double* stencil, double* out) {
  int nch = 1 << d;
  for (int ci = 0; ci < nch; ++ci)
    out[ci] = predict_stencil_s(d, cross_sign, 1, stencil, ci & 1, (ci >> 1) & 1, (ci >> 2) & 1);
  return 0;
}

int or_predict_children_s(int d, int cross_sign, int s, const double* stencil, double* out) {
  if (s < 1 || s > 3 || d < 1 || d > 3) return -1;
  int nch = 1 << d;
  for (int ci = 0; ci < nch; ++ci)
    out[ci] = predict_stencil_s(d, cross_sign, s, stencil, ci & 1, (ci >> 1) & 1, (ci >> 2) & 1);
  return 0;
}

/* Predicted value of population p on child cell (l, x, y, z) from level l-1. */
static double predict(const or_state* S, double* const* F, int l, int x, int y, int z, int p) {
  int L = l - 1, px = x >> 1, py = y >> 1, pz = z >> 1;
  double v[343]; /* (2s+1)^d <= 7^3 */
  int d = S->d, s = S->s_pred, w = 2 * s + 1;
  int nz = d >= 3 ? w : 1, ny = d >= 2 ? w : 1;
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < w; ++a) {
        int sx = stencil_coord(S, L, 0, px + a - s);
        int sy = d >= 2 ? stencil_coord(S, L, 1, py + b - s) : 0;
        int sz = d >= 3 ? stencil_coord(S, L, 2, pz + c - s) : 0;
        v[(c * ny + b) * w + a] = F[L][cidx(S, L, sx, sy, sz) * S->Q + p];
      }
  return predict_stencil_s(d, S->cfg.cross_sign, s, v, x & 1, y & 1, z & 1);
}

/* Membership of R(Lambda): leaves and all their ancestors. */
static void tree_of_leaves(const or_state* S, unsigned char* const* leaf, unsigned char** inR) {
  for (int l = S->J; l >= S->Jmin; --l) {
    for (long long c = 0; c < S->nc[l]; ++c) {
      unsigned char v = leaf[l][c];
      if (!v && l < S->J) {
        int x, y, z;
        cell_coords(S, l, c, &x, &y, &z);
        for (int ci = 0; ci < (1 << S->d) && !v; ++ci)
          v = inR[l + 1][cidx(S, l + 1, 2 * x + (ci & 1), S->d >= 2 ? 2 * y + ((ci >> 1) & 1) : 0,
                                  S->d >= 3 ? 2 * z + ((ci >> 2) & 1) : 0)];
      }
      inR[l][c] = v;
    }
  }
}

/* Full reconstruction of the leaf data on every cell of every level: cells of
 * R(Lambda) take the projection of Def. Projection (children summed in the
 * order ci = dx + 2 dy + 4 dz, then scaled by 2^-d), cells inside a leaf take
 * the recursive prediction (the reconstruction operator of Sec. 4.4). */
static void reconstruct_all(const or_state* S, unsigned char* const* leaf, double* const* val,
                            double** F, unsigned char** inR) {
  const int Q = S->Q, d = S->d, nch = 1 << d;
  const double scale = ldexp(1.0, -d);
  tree_of_leaves(S, leaf, inR);
  for (int l = S->J; l >= S->Jmin; --l)
    for (long long c = 0; c < S->nc[l]; ++c) {
      if (leaf[l][c]) {
        memcpy(&F[l][c * Q], &val[l][c * Q], sizeof(double) * Q);
      } else if (inR[l][c]) {
        int x, y, z;
        cell_coords(S, l, c, &x, &y, &z);
        for (int p = 0; p < Q; ++p) {
          double acc = 0.0;
          for (int ci = 0; ci < nch; ++ci)
            acc = acc + F[l + 1][cidx(S, l + 1, 2 * x + (ci & 1), d >= 2 ? 2 * y + ((ci >> 1) & 1) : 0,
                                      d >= 3 ? 2 * z + ((ci >> 2) & 1) : 0) * Q + p];
          F[l][c * Q + p] = acc * scale;
        }
      }
    }
  for (int l = S->Jmin + 1; l <= S->J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c)
      if (!inR[l][c]) {
        int x, y, z;
        cell_coords(S, l, c, &x, &y, &z);
        for (int p = 0; p < Q; ++p) F[l][c * Q + p] = predict(S, F, l, x, y, z, p);
      }
}

/* ------------------------------------------------------------------------ */
/* allocation helpers                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  double* F[MAXL];
  unsigned char* u8[MAXL];
} levels_t;

static int alloc_F(const or_state* S, double** F) {
  for (int l = 0; l < MAXL; ++l) F[l] = NULL;
  for (int l = S->Jmin; l <= S->J; ++l) {
    F[l] = (double*)calloc((size_t)S->nc[l] * S->Q, sizeof(double));
    if (!F[l]) return -1;
  }
  return 0;
}
static int alloc_u8(const or_state* S, unsigned char** A) {
  for (int l = 0; l < MAXL; ++l) A[l] = NULL;
  for (int l = S->Jmin; l <= S->J; ++l) {
    A[l] = (unsigned char*)calloc((size_t)S->nc[l], 1);
    if (!A[l]) return -1;
  }
  return 0;
}
static void free_F(const or_state* S, double** F) {
  for (int l = S->Jmin; l <= S->J; ++l) { free(F[l]); F[l] = NULL; }
}
static void free_u8(const or_state* S, unsigned char** A) {
  for (int l = S->Jmin; l <= S->J; ++l) { free(A[l]); A[l] = NULL; }
}

/* ------------------------------------------------------------------------ */
/* state                                                                     */
/* ------------------------------------------------------------------------ */

or_state* or_create(const or_config* cfg) {
  or_state* S = (or_state*)calloc(1, sizeof(or_state));
  if (!S) return NULL;
  S->cfg = *cfg;
  if (S->cfg.cross_sign == 0) S->cfg.cross_sign = 1;
  if (setup_scheme(S) != 0) { free(S); return NULL; }
  S->Jmin = cfg->min_level;
  S->J = cfg->max_level;
  if (S->Jmin < 0 || S->J >= MAXL || S->Jmin > S->J) { free(S); return NULL; }
  S->s_pred = cfg->pred_s == 0 ? 1 : cfg->pred_s;
  if (S->s_pred < 1 || S->s_pred > 3) { free(S); return NULL; }
  /* Sec. 5.1: the regularity guess mu_bar of the refinement rule lies in
   * [0, 2s + 1], the order of the prediction operator */
  if (cfg->mu_bar < 0 || cfg->mu_bar > 2 * S->s_pred + 1) { free(S); return NULL; }
  for (int l = S->Jmin; l <= S->J; ++l) {
    long long tot = 1;
    for (int a = 0; a < 3; ++a) {
      int r = a < S->d ? (cfg->roots[a] > 0 ? cfg->roots[a] : 1) : 1;
      S->n[l][a] = a < S->d ? r << l : 1;
      tot *= S->n[l][a];
    }
    S->nc[l] = tot;
  }
  if (alloc_u8(S, S->leaf) || alloc_F(S, S->val)) { or_destroy(S); return NULL; }
  for (int l = 0; l < MAXL; ++l) S->G[l] = NULL;
  S->last_margin = INFINITY;
  return S;
}

void or_destroy(or_state* S) {
  if (!S) return;
  free_u8(S, S->leaf);
  free_F(S, S->val);
  for (int l = 0; l < MAXL; ++l) free(S->G[l]);
  free(S);
}

int or_scheme_info(const or_state* S, int* d, int* q, int* m, int* Q, int* ncons) {
  *d = S->d; *q = S->q; *m = S->m; *Q = S->Q; *ncons = S->ncons;
  return 0;
}

/* Algorithm 1: full finest mesh, f = M^-1 m^eq. */
int or_init(or_state* S, const double* cons) {
  for (int l = S->Jmin; l <= S->J; ++l) {
    memset(S->leaf[l], 0, (size_t)S->nc[l]);
    memset(S->val[l], 0, sizeof(double) * S->nc[l] * S->Q);
  }
  const long long N = S->nc[S->J];
  for (long long c = 0; c < N; ++c) {
    double u[4];
    for (int k = 0; k < S->ncons; ++k) u[k] = cons[k * N + c];
    equilibrium_populations(S, u, &S->val[S->J][c * S->Q]);
    S->leaf[S->J][c] = 1;
  }
  return 0;
}

long long or_num_leaves(const or_state* S) {
  long long n = 0;
  for (int l = S->Jmin; l <= S->J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c) n += S->leaf[l][c];
  return n;
}

int or_get_leaves(const or_state* S, int* level, int* ix, int* iy, int* iz, double* f) {
  long long n = or_num_leaves(S), k = 0;
  for (int l = S->Jmin; l <= S->J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c)
      if (S->leaf[l][c]) {
        int x, y, z;
        cell_coords(S, l, c, &x, &y, &z);
        if (level) level[k] = l;
        if (ix) ix[k] = x;
        if (iy) iy[k] = y;
        if (iz) iz[k] = z;
        if (f)
          for (int p = 0; p < S->Q; ++p) f[(long long)p * n + k] = S->val[l][c * S->Q + p];
        ++k;
      }
  return 0;
}

int or_set_leaves(or_state* S, long long n, const int* level, const int* ix, const int* iy,
                  const int* iz, const double* f) {
  for (int l = S->Jmin; l <= S->J; ++l) {
    memset(S->leaf[l], 0, (size_t)S->nc[l]);
    memset(S->val[l], 0, sizeof(double) * S->nc[l] * S->Q);
  }
  unsigned char* cover = (unsigned char*)calloc((size_t)S->nc[S->J], 1);
  if (!cover) return -1;
  int rc = 0;
  for (long long k = 0; k < n && rc == 0; ++k) {
    int l = level[k], x = ix[k], y = iy ? iy[k] : 0, z = iz ? iz[k] : 0;
    if (l < S->Jmin || l > S->J || x < 0 || x >= S->n[l][0] || y < 0 || y >= S->n[l][1] || z < 0 ||
        z >= S->n[l][2]) { rc = -2; break; }
    long long c = cidx(S, l, x, y, z);
    S->leaf[l][c] = 1;
    for (int p = 0; p < S->Q; ++p) S->val[l][c * S->Q + p] = f[(long long)p * n + k];
    int g = S->J - l, w = 1 << g;
    for (int cz = 0; cz < (S->d >= 3 ? w : 1); ++cz)
      for (int cy = 0; cy < (S->d >= 2 ? w : 1); ++cy)
        for (int cx = 0; cx < w; ++cx) {
          long long fc = cidx(S, S->J, x * w + cx, S->d >= 2 ? y * w + cy : 0, S->d >= 3 ? z * w + cz : 0);
          if (cover[fc]) rc = -3;
          cover[fc] = 1;
        }
  }
  for (long long c = 0; c < S->nc[S->J] && rc == 0; ++c)
    if (!cover[c]) rc = -4;
  free(cover);
  return rc;
}

double or_last_margin(const or_state* S) { return S->last_margin; }

int or_group_norms(const or_state* S, int level, double* out) {
  if (level < S->Jmin || level >= S->J || !S->G[level]) return -1;
  memcpy(out, S->G[level], sizeof(double) * S->nc[level]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* tree operations (Sec. 4.3, 4.4, 5.1) on sets of cells                     */
/* ------------------------------------------------------------------------ */

/* Add cell (l, x, y, z) with its siblings and all its ancestors (with their
 * siblings) to the tree `T`, which is kept closed under these operations. */
static void add_cell(const or_state* S, unsigned char** T, int l, int x, int y, int z) {
  while (l > S->Jmin) {
    if (T[l][cidx(S, l, x, y, z)]) return; /* closed: siblings and ancestors already in */
    int px = x >> 1, py = y >> 1, pz = z >> 1;
    for (int ci = 0; ci < (1 << S->d); ++ci)
      T[l][cidx(S, l, 2 * px + (ci & 1), S->d >= 2 ? 2 * py + ((ci >> 1) & 1) : 0,
                S->d >= 3 ? 2 * pz + ((ci >> 2) & 1) : 0)] = 1;
    x = px; y = py; z = pz; --l;
  }
  T[S->Jmin][cidx(S, S->Jmin, x, y, z)] = 1;
}

static double eps_level(const or_state* S, int l) { return ldexp(S->cfg.eps, S->d * (l - S->J)); }

/* Mesh adaptation Lambda(t+dt) = G o H o T (Lambda(t)) with details of the
 * stored field, then the data transfer of Sec. 5.1 (projection where cells
 * merge, prediction where cells are created): both are values of the full
 * reconstruction F of the old data. */
static int adapt_impl(or_state* S) {
  const int Q = S->Q, d = S->d, Jmin = S->Jmin, J = S->J;
  double* F[MAXL];
  unsigned char *inR[MAXL], *T[MAXL], *snap[MAXL];
  if (alloc_F(S, F) || alloc_u8(S, inR) || alloc_u8(S, T) || alloc_u8(S, snap)) return -1;
  reconstruct_all(S, S->leaf, S->val, F, inR);

  /* details (Def. Details) and the sibling-group norm max over populations */
  for (int l = Jmin; l < J; ++l) {
    free(S->G[l]);
    S->G[l] = (double*)malloc(sizeof(double) * S->nc[l]);
    for (long long c = 0; c < S->nc[l]; ++c) S->G[l][c] = (inR[l][c] && !S->leaf[l][c]) ? 0.0 : -1.0;
  }
  for (int l = Jmin + 1; l <= J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c) {
      if (!inR[l][c]) continue;
      int x, y, z;
      cell_coords(S, l, c, &x, &y, &z);
      long long pc = cidx(S, l - 1, x >> 1, y >> 1, z >> 1);
      double g = S->G[l - 1][pc];
      for (int p = 0; p < Q; ++p) {
        double det = F[l][c * Q + p] - predict(S, F, l, x, y, z, p);
        double a = fabs(det);
        if (a > g) g = a;
      }
      S->G[l - 1][pc] = g;
    }

  /* decision margin */
  double margin = INFINITY;
  for (int l = Jmin; l < J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c) {
      double g = S->G[l][c];
      if (g < 0) continue;
      double t1 = eps_level(S, l + 1);
      if (t1 > 0) { double r = fabs(g - t1) / t1; if (r < margin) margin = r; }
      if (l + 1 > Jmin && l + 1 < J) {
        double t2 = ldexp(t1, S->cfg.mu_bar + d);
        if (t2 > 0) { double r = fabs(g - t2) / t2; if (r < margin) margin = r; }
      }
    }
  S->last_margin = margin;

  /* T_eps (Eq. Thresholding).  Reading: the kept set is closed into a tree
   * (siblings and ancestors of kept cells are kept). */
  for (long long c = 0; c < S->nc[Jmin]; ++c) T[Jmin][c] = 1;
  for (int l = Jmin + 1; l <= J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c) {
      if (!inR[l][c]) continue;
      int x, y, z;
      cell_coords(S, l, c, &x, &y, &z);
      if (S->G[l - 1][cidx(S, l - 1, x >> 1, y >> 1, z >> 1)] >= eps_level(S, l)) add_cell(S, T, l, x, y, z);
    }

  /* H_eps: neighbours k - eta^h (Eq. AdditionNeigh) and children of cells
   * with large details, both applied to the cells of R(T_eps(Lambda)). */
  for (int l = Jmin; l <= J; ++l) memcpy(snap[l], T[l], (size_t)S->nc[l]);
  for (int l = Jmin; l <= J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c) {
      if (!snap[l][c]) continue;
      int x, y, z;
      cell_coords(S, l, c, &x, &y, &z);
      for (int h = 0; h < S->q; ++h) {
        int nx = mesh_coord(S, l, 0, x - S->eta[h][0]);
        int ny = mesh_coord(S, l, 1, y - S->eta[h][1]);
        int nz = mesh_coord(S, l, 2, z - S->eta[h][2]);
        if (nx < 0 || ny < 0 || nz < 0) continue;
        add_cell(S, T, l, nx, ny, nz);
      }
      if (l > Jmin && l < J) {
        double g = S->G[l - 1][cidx(S, l - 1, x >> 1, y >> 1, z >> 1)];
        if (g >= ldexp(eps_level(S, l), S->cfg.mu_bar + d))
          for (int ci = 0; ci < (1 << d); ++ci)
            add_cell(S, T, l + 1, 2 * x + (ci & 1), d >= 2 ? 2 * y + ((ci >> 1) & 1) : 0,
                     d >= 3 ? 2 * z + ((ci >> 2) & 1) : 0);
      }
    }

  /* G: minimal graded tree, iterated to a fixed point (Def. Grading): every
   * cell above J_min has the (2s+1)^d stencil around its parent in the tree. */
  const int sp = S->s_pred;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int l = Jmin + 1; l <= J; ++l)
      for (long long c = 0; c < S->nc[l]; ++c) {
        if (!T[l][c]) continue;
        int x, y, z;
        cell_coords(S, l, c, &x, &y, &z);
        int px = x >> 1, py = y >> 1, pz = z >> 1;
        for (int oc = (d >= 3 ? -sp : 0); oc <= (d >= 3 ? sp : 0); ++oc)
          for (int ob = (d >= 2 ? -sp : 0); ob <= (d >= 2 ? sp : 0); ++ob)
            for (int oa = -sp; oa <= sp; ++oa) {
              int nx = mesh_coord(S, l - 1, 0, px + oa);
              int ny = mesh_coord(S, l - 1, 1, py + ob);
              int nz = mesh_coord(S, l - 1, 2, pz + oc);
              if (nx < 0 || ny < 0 || nz < 0) continue;
              if (!T[l - 1][cidx(S, l - 1, nx, ny, nz)]) {
                add_cell(S, T, l - 1, nx, ny, nz);
                changed = 1;
              }
            }
      }
  }

  /* new leaves and their data (Sec. 5.1, last paragraph) */
  for (int l = Jmin; l <= J; ++l)
    for (long long c = 0; c < S->nc[l]; ++c) {
      int isleaf = 0;
      if (T[l][c]) {
        if (l == J) {
          isleaf = 1;
        } else {
          int x, y, z;
          cell_coords(S, l, c, &x, &y, &z);
          isleaf = !T[l + 1][cidx(S, l + 1, 2 * x, d >= 2 ? 2 * y : 0, d >= 3 ? 2 * z : 0)];
        }
      }
      S->leaf[l][c] = (unsigned char)isleaf;
      if (isleaf)
        memcpy(&S->val[l][c * Q], &F[l][c * Q], sizeof(double) * Q);
      else
        memset(&S->val[l][c * Q], 0, sizeof(double) * Q);
    }
  free_F(S, F);
  free_u8(S, inR);
  free_u8(S, T);
  free_u8(S, snap);
  return 0;
}

int or_adapt(or_state* S) { return adapt_impl(S); }

/* Value entering through a boundary face, Eq. refBoundaryConditions with the
 * direct evaluation of Sec. 5.3: the leaf's own post-collision values.
 * Reading for the bounce back with a given velocity: the bounced value plus
 * f^{h,eq} - f^{h dagger,eq} at (rho0, u0). */
static double boundary_value(const or_state* S, int face, const double* fleaf, int p) {
  int lat = p / S->q, h = p % S->q;
  int pd = lat * S->q + S->opp[h];
  switch (S->cfg.bc[face]) {
    case OR_BC_COPY: return fleaf[p];
    case OR_BC_BOUNCE_BACK: return fleaf[pd];
    case OR_BC_ANTI_BOUNCE_BACK: return -fleaf[pd];
    case OR_BC_BOUNCE_BACK_VELOCITY: {
      double u[4] = {S->cfg.phys[0], S->cfg.phys[0] * S->cfg.phys[1], S->cfg.phys[0] * S->cfg.phys[2], 0};
      double feq[MAXQ];
      equilibrium_populations(S, u, feq);
      return fleaf[pd] + (feq[p] - feq[pd]);
    }
    default: return 0.0;
  }
}

/* The "original adaptive" collision (Sec. 5.3, the right-hand side of
 * Eq. sourceoferror): instead of colliding the leaf's own averages
 * (Eq. AdaptiveCollision), reconstruct the post-transport data on every
 * finest cell (the reconstruction operator of Sec. 4.4), collide each finest
 * cell of B_{j,k} (Eq. CellSplitting) and give the leaf the average,
 * 2^{-d(J-j)} times the sum over B_{j,k} taken x fastest, then y, then z. */
static int exact_collision_impl(or_state* S) {
  const int Q = S->Q, d = S->d, J = S->J;
  double* F[MAXL];
  unsigned char* inR[MAXL];
  if (alloc_F(S, F) || alloc_u8(S, inR)) return -1;
  reconstruct_all(S, S->leaf, S->val, F, inR);
  double* g = (double*)malloc(sizeof(double) * Q);
  double* acc = (double*)malloc(sizeof(double) * Q);
  for (int j = S->Jmin; j <= J; ++j)
    for (long long c = 0; c < S->nc[j]; ++c) {
      if (!S->leaf[j][c]) continue;
      int kx, ky, kz;
      cell_coords(S, j, c, &kx, &ky, &kz);
      const int w = 1 << (J - j);
      const int wy = d >= 2 ? w : 1, wz = d >= 3 ? w : 1;
      for (int p = 0; p < Q; ++p) acc[p] = 0.0;
      for (int cz = 0; cz < wz; ++cz)
        for (int cy = 0; cy < wy; ++cy)
          for (int cx = 0; cx < w; ++cx) {
            const long long k = cidx(S, J, kx * w + cx, d >= 2 ? ky * wy + cy : 0, d >= 3 ? kz * wz + cz : 0);
            memcpy(g, &F[J][k * Q], sizeof(double) * Q);
            collide_cell(S, g);
            for (int p = 0; p < Q; ++p) acc[p] += g[p];
          }
      for (int p = 0; p < Q; ++p) S->val[j][c * Q + p] = acc[p] * ldexp(1.0, -d * (J - j));
    }
  free(g);
  free(acc);
  free_F(S, F);
  free_u8(S, inR);
  return 0;
}

/* Eq. AdaptiveAdvectionPhase with Eq. AdvectionOnBoundary, literally: the sums
 * run over the finest cells of E = (B - eta) \ B and A = B \ (B - eta). */
static int stream_impl(or_state* S, int do_collide) {
  const int Q = S->Q, d = S->d, J = S->J;
  double* F[MAXL];
  unsigned char* inR[MAXL];
  if (alloc_F(S, F) || alloc_u8(S, inR)) return -1;
  reconstruct_all(S, S->leaf, S->val, F, inR);
  const double* FJ = F[J];
  double* out = (double*)malloc(sizeof(double) * Q);
  for (int j = S->Jmin; j <= J; ++j)
    for (long long c = 0; c < S->nc[j]; ++c) {
      if (!S->leaf[j][c]) continue;
      int kx, ky, kz;
      cell_coords(S, j, c, &kx, &ky, &kz);
      const int w = 1 << (J - j);
      const int wy = d >= 2 ? w : 1, wz = d >= 3 ? w : 1;
      const int b0[3] = {kx * w, ky * wy, kz * wz}, bw[3] = {w, wy, wz};
      const double* fl = &S->val[j][c * Q];
      for (int p = 0; p < Q; ++p) {
        const int* e = S->eta[p % S->q];
        double sumE = 0.0, sumA = 0.0, sumB = 0.0;
        for (int cz = 0; cz < wz; ++cz)
          for (int cy = 0; cy < wy; ++cy)
            for (int cx = 0; cx < w; ++cx) {
              int xb[3] = {b0[0] + cx, b0[1] + cy, b0[2] + cz};
              /* y = x - eta in E iff not in B */
              int yy[3], inB = 1;
              for (int a = 0; a < 3; ++a) {
                yy[a] = xb[a] - (a < d ? e[a] : 0);
                if (yy[a] < b0[a] || yy[a] >= b0[a] + bw[a]) inB = 0;
              }
              if (!inB) {
                int face = -1;
                for (int a = 0; a < d && face < 0; ++a) {
                  int N = S->n[J][a];
                  if (yy[a] < 0 || yy[a] >= N) {
                    if (periodic(S, a)) yy[a] = ((yy[a] % N) + N) % N;
                    else face = 2 * a + (yy[a] >= N ? 1 : 0);
                  }
                }
                if (face < 0) {
                  for (int a = 0; a < d; ++a) {
                    int N = S->n[J][a];
                    yy[a] = ((yy[a] % N) + N) % N;
                  }
                  sumE += FJ[cidx(S, J, yy[0], yy[1], yy[2]) * Q + p];
                } else {
                  sumB += boundary_value(S, face, fl, p);
                }
              }
              /* x in A iff x + eta not in B */
              int inB2 = 1;
              for (int a = 0; a < d; ++a) {
                int z2 = xb[a] + e[a];
                if (z2 < b0[a] || z2 >= b0[a] + bw[a]) inB2 = 0;
              }
              if (!inB2) sumA += FJ[cidx(S, J, xb[0], xb[1], xb[2]) * Q + p];
            }
        out[p] = fl[p] + ldexp(1.0, d * (j - J)) * ((sumE - sumA) + sumB);
      }
      if (do_collide && !S->cfg.exact_collision) collide_cell(S, out);
      memcpy(&S->val[j][c * Q], out, sizeof(double) * Q);
    }
  free(out);
  free_F(S, F);
  free_u8(S, inR);
  if (do_collide && S->cfg.exact_collision && exact_collision_impl(S)) return -1;
  if (do_collide && S->cfg.obstacle) {
    /* Sec. 7.2.2 penalisation.  Reading: the volume fraction is the share of
     * finest-cell centres of B inside the disc. */
    const double rho0 = S->cfg.phys[0], cx = S->cfg.phys[3], cy = S->cfg.phys[4], r = S->cfg.phys[5];
    const double dx = (S->cfg.xmax[0] - S->cfg.xmin[0]) / S->n[J][0];
    double u[4] = {rho0, 0, 0, 0}, feq[MAXQ];
    equilibrium_populations(S, u, feq);
    for (int j = S->Jmin; j <= J; ++j)
      for (long long c = 0; c < S->nc[j]; ++c) {
        if (!S->leaf[j][c]) continue;
        int kx, ky, kz;
        cell_coords(S, j, c, &kx, &ky, &kz);
        int w = 1 << (J - j);
        long long inside = 0;
        for (int by = 0; by < w; ++by)
          for (int bx = 0; bx < w; ++bx) {
            double xc = S->cfg.xmin[0] + (kx * w + bx + 0.5) * dx;
            double yc = S->cfg.xmin[1] + (ky * w + by + 0.5) * dx;
            if ((xc - cx) * (xc - cx) + (yc - cy) * (yc - cy) <= r * r) ++inside;
          }
        if (!inside) continue;
        double phi = (double)inside / ((double)w * w);
        double* f = &S->val[j][c * Q];
        for (int p = 0; p < Q; ++p) f[p] = phi * feq[p] + (1.0 - phi) * f[p];
      }
  }
  return 0;
}

int or_stream_collide(or_state* S, int do_collide) { return stream_impl(S, do_collide); }

/* Algorithm 1, with the phases in the order adapt, remesh, stream, collide. */
int or_step(or_state* S, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    if (adapt_impl(S)) return -1;
    if (stream_impl(S, 1)) return -1;
  }
  return 0;
}

static int reconstruct_level(or_state* S, int level, double* out, int conserved) {
  if (level < S->Jmin || level > S->J) return -1;
  double* F[MAXL];
  unsigned char* inR[MAXL];
  if (alloc_F(S, F) || alloc_u8(S, inR)) return -1;
  reconstruct_all(S, S->leaf, S->val, F, inR);
  long long N = S->nc[level];
  for (long long c = 0; c < N; ++c) {
    const double* f = &F[level][c * S->Q];
    if (conserved) {
      double mo[4][9], u[4];
      moments(S, f, mo);
      conserved_of(S, mo, u);
      for (int k = 0; k < S->ncons; ++k) out[k * N + c] = u[k];
    } else {
      for (int p = 0; p < S->Q; ++p) out[p * N + c] = f[p];
    }
  }
  free_F(S, F);
  free_u8(S, inR);
  return 0;
}

int or_project(or_state* S, int level, double* out) { return reconstruct_level(S, level, out, 1); }
int or_reconstruct(or_state* S, int level, double* out) { return reconstruct_level(S, level, out, 0); }

int or_check_graded(const or_state* S) {
  unsigned char* inR[MAXL];
  if (alloc_u8(S, inR)) return -1;
  tree_of_leaves(S, S->leaf, inR);
  int ok = 1;
  for (long long c = 0; c < S->nc[S->Jmin]; ++c)
    if (!inR[S->Jmin][c]) ok = 0;
  for (int l = S->Jmin + 1; l <= S->J && ok; ++l)
    for (long long c = 0; c < S->nc[l] && ok; ++c) {
      if (!inR[l][c]) continue;
      int x, y, z;
      cell_coords(S, l, c, &x, &y, &z);
      int px = x >> 1, py = y >> 1, pz = z >> 1;
      const int sp = S->s_pred;
      for (int oc = (S->d >= 3 ? -sp : 0); oc <= (S->d >= 3 ? sp : 0); ++oc)
        for (int ob = (S->d >= 2 ? -sp : 0); ob <= (S->d >= 2 ? sp : 0); ++ob)
          for (int oa = -sp; oa <= sp; ++oa) {
            int nx = mesh_coord(S, l - 1, 0, px + oa);
            int ny = mesh_coord(S, l - 1, 1, py + ob);
            int nz = mesh_coord(S, l - 1, 2, pz + oc);
            if (nx < 0 || ny < 0 || nz < 0) continue;
            if (!inR[l - 1][cidx(S, l - 1, nx, ny, nz)]) ok = 0;
          }
    }
  free_u8(S, inR);
  return ok;
}
