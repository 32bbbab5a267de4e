/*
 * iilbm3d_oracle.c -- plain, slow FP64 CPU oracle of one three-dimensional immersed
 * interface-lattice Boltzmann (II-LBM) time step on the D3Q19 lattice (Qin, Kolahdouz &
 * Griffith, arXiv 2003.12186: sections 2.1 and 2.2.1 give the D3Q19 velocity set, its
 * weights and its MRT rates; section 3.1 derives the jump conditions in three
 * dimensions; the conclusion notes that the method carries over to 3-D).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark may load this file.  It shares no code, header, table or
 * constant with the CUDA library (nor with the two-dimensional oracle); it is compiled
 * on its own with gcc (-ffp-contract=off, no fused multiply-adds).
 *
 * Every routine is a direct transcription of a definition (section / equation beside
 * it) in FP64 with plain loops.  The immersed interface is a closed triangulated
 * surface: vertices X_k (the Lagrangian markers) and triangles (A, B, C) ordered
 * counter-clockwise seen from outside, so (B - A) x (C - A) points outward.
 *
 * Populations are shifted, df_i = f_i - w_i rho0 (exact change of variables).
 * Layout: df[i*nz*ny*nx + (z*ny + y)*nx + x].  The box is periodic on every axis.
 *
 * The same source also builds with -fopenmp (the all-core CPU baseline): the "omp
 * parallel for" lines mark per-node loops whose iterations touch disjoint nodes, so the
 * parallel build computes every value exactly as the serial one does.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- D3Q19 velocity set (section 2.1) and weights (section 2.2.1) ----------------
 * 0 rest; 1..6 the axes (+x, -x, +y, -y, +z, -z); 7..18 the twelve edge diagonals,
 * in opposite pairs.  Weights 1/3, 1/18, 1/36. */
static const int EX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double WT[19] = {1.0 / 3,
                              1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
/* 1/c_s^2 = 3 exactly (c_s = 1/sqrt(3)): applied as a multiplication. */
#define INV_CS2 3.0

int o3_opp(int i) { return i == 0 ? 0 : (i % 2 ? i + 1 : i - 1); }

/* The velocity set and weights, for the tests' isotropy pins. */
void o3_lattice(int *ex, int *ey, int *ez, double *w) {
  for (int i = 0; i < 19; i++) { ex[i] = EX[i]; ey[i] = EY[i]; ez[i] = EZ[i]; w[i] = WT[i]; }
}

/* ---------------------------------------------------------------- config --- */
enum { O3_SRT = 0, O3_MRT = 1 };
enum { O3_FORCE_GUO = 0, O3_FORCE_SIMPLE = 1 };
enum { O3_PRESCRIBED = 0, O3_TENSION = 1 };

typedef struct {
  int nx, ny, nz;
  int collision;    /* O3_SRT or O3_MRT */
  double tau;       /* relaxation time lambda */
  double s[19];     /* MRT rates in the d'Humieres moment order (below) */
  double rho0;
  double body[3];   /* uniform body force density added to g */
  int jump;         /* 1: II-LBM (normal force through the jump), 0: IB-LBM */
  int force;        /* O3_FORCE_GUO (Eqs. 21-22) or O3_FORCE_SIMPLE (Eq. 16) */
} o3_cfg;

typedef struct {
  int n, m;          /* vertices, triangles */
  double *X;         /* [n][3] */
  int *tri;          /* [m][3] */
  double *Aref;      /* [n] reference vertex area (the surface element dr ds of Eq. 17) */
  int model;         /* O3_PRESCRIBED or O3_TENSION */
  int moves;         /* 1: X += U (Eq. 20) */
  double gamma;      /* O3_TENSION: surface tension */
  double *Gp;        /* [n][3] O3_PRESCRIBED: the force density G */
} o3_iface;

typedef struct {
  o3_cfg c;
  double M[19 * 19], Minv[19 * 19];
  double *df, *f, *tmp;          /* [19][N] */
  double *gx, *gy, *gz;          /* [N] Eulerian force density */
  double *rho, *ux, *uy, *uz;    /* [N] density deviation and velocity of the collision */
  int has_iface;
  o3_iface I;
  double *G, *Fn, *Gpar, *U;     /* [n][3] / [n] / [n][3] / [n][3] */
  double *nrm, *area;            /* [n][3] vertex normals, [n] current vertex areas */
  int ncut;
  long step;
} o3_state;

/* ------------------------------------------------------------ MRT matrix ---
 * d'Humieres et al. (2002) D3Q19 moment basis, the one section 2.2.1 cites: rows are
 * the polynomials, evaluated on the nineteen velocities,
 *   0 rho = 1                       1 e = 19|e|^2 - 30       2 eps = (21|e|^4 - 53|e|^2 + 24)/2
 *   3 j_x = e_x                     4 q_x = (5|e|^2 - 9) e_x
 *   5 j_y = e_y                     6 q_y = (5|e|^2 - 9) e_y
 *   7 j_z = e_z                     8 q_z = (5|e|^2 - 9) e_z
 *   9 3p_xx = 3e_x^2 - |e|^2        10 3pi_xx = (3|e|^2 - 5)(3e_x^2 - |e|^2)
 *  11 p_ww = e_y^2 - e_z^2          12 pi_ww = (3|e|^2 - 5)(e_y^2 - e_z^2)
 *  13 p_xy = e_x e_y   14 p_yz = e_y e_z   15 p_xz = e_x e_z
 *  16 m_x = (e_y^2 - e_z^2) e_x   17 m_y = (e_z^2 - e_x^2) e_y   18 m_z = (e_x^2 - e_y^2) e_z
 * The rates s_0..s_18 of section 2.2.1 index these rows in this order (s_0 = s_3 = s_5 =
 * s_7 = 0 are the conserved density and momentum). */
void o3_mrt_matrix(double *M) {
  for (int i = 0; i < 19; i++) {
    double ex = EX[i], ey = EY[i], ez = EZ[i];
    double e2 = ex * ex + ey * ey + ez * ez;
    double *c = M + i;
    c[0 * 19] = 1.0;
    c[1 * 19] = 19.0 * e2 - 30.0;
    c[2 * 19] = (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0;
    c[3 * 19] = ex;
    c[4 * 19] = (5.0 * e2 - 9.0) * ex;
    c[5 * 19] = ey;
    c[6 * 19] = (5.0 * e2 - 9.0) * ey;
    c[7 * 19] = ez;
    c[8 * 19] = (5.0 * e2 - 9.0) * ez;
    c[9 * 19] = 3.0 * ex * ex - e2;
    c[10 * 19] = (3.0 * e2 - 5.0) * (3.0 * ex * ex - e2);
    c[11 * 19] = ey * ey - ez * ez;
    c[12 * 19] = (3.0 * e2 - 5.0) * (ey * ey - ez * ez);
    c[13 * 19] = ex * ey;
    c[14 * 19] = ey * ez;
    c[15 * 19] = ex * ez;
    c[16 * 19] = (ey * ey - ez * ez) * ex;
    c[17 * 19] = (ez * ez - ex * ex) * ey;
    c[18 * 19] = (ex * ex - ey * ey) * ez;
  }
}

/* M^-1 of the orthogonal-row basis: M^T diag(1 / |row_r|^2) (squared row norms are sums
 * of squared integers, exact). */
void o3_mrt_inverse(const double *M, double *Minv) {
  for (int r = 0; r < 19; r++) {
    double nrm = 0;
    for (int i = 0; i < 19; i++) nrm += M[r * 19 + i] * M[r * 19 + i];
    for (int i = 0; i < 19; i++) Minv[i * 19 + r] = M[r * 19 + i] / nrm;
  }
}

/* ------------------------------------------------------ equilibrium, force --
 * Equilibrium (Eq. 23 with the D3Q19 weights): f_eq_i = w_i rho [1 + e.u/c_s^2 +
 * (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)], returned shifted by w_i rho0 from drho. */
void o3_feq_shifted(double drho, double rho0, double ux, double uy, double uz, double *dfeq) {
  double u2 = ux * ux + uy * uy + uz * uz, rho = rho0 + drho;
  for (int i = 0; i < 19; i++) {
    double eu = EX[i] * ux + EY[i] * uy + EZ[i] * uz;
    double poly = eu * INV_CS2 + eu * eu * (INV_CS2 * INV_CS2 / 2.0) - u2 * (INV_CS2 / 2.0);
    dfeq[i] = WT[i] * (drho + rho * poly);
  }
}

/* Guo's source without its relaxation prefactor (Eqs. 21-22):
 * Gt_i = w_i [ (e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4 ] . g */
void o3_guo_source(double ux, double uy, double uz, double gx, double gy, double gz,
                   double *Gt) {
  for (int i = 0; i < 19; i++) {
    double eu = EX[i] * ux + EY[i] * uy + EZ[i] * uz;
    double t1 = ((EX[i] - ux) * gx + (EY[i] - uy) * gy + (EZ[i] - uz) * gz) * INV_CS2;
    double t2 = eu * (EX[i] * gx + EY[i] * gy + EZ[i] * gz) * (INV_CS2 * INV_CS2);
    Gt[i] = WT[i] * (t1 + t2);
  }
}

/* drho = sum df (Eq. 11 less rho0); rho u = sum e_i f_i + h (Eq. 24 with h = g/2 under
 * Guo's forcing, h = 0 for the simple force term). */
void o3_cell_macros(const double *dfc, double rho0, double hx, double hy, double hz,
                    double *drho, double *ux, double *uy, double *uz) {
  double s = 0, jx = 0, jy = 0, jz = 0;
  for (int i = 0; i < 19; i++) {
    s += dfc[i];
    jx += EX[i] * dfc[i];
    jy += EY[i] * dfc[i];
    jz += EZ[i] * dfc[i];
  }
  *drho = s;
  *ux = (jx + hx) / (rho0 + s);
  *uy = (jy + hy) / (rho0 + s);
  *uz = (jz + hz) / (rho0 + s);
}

/* Collision of one node, shifted populations in and out.
 *  Guo:    SRT f* = f - (f - f_eq)/lambda + (1 - 1/(2 lambda)) Gt            (Eqs. 14, 21)
 *          MRT f* = f - M^-1 S (M f - M f_eq) + M^-1 (I - S/2) M Gt          (Eqs. 15, 22)
 *          with u = (sum e f + g/2) / rho.
 *  simple: the relaxation with u = sum e f / rho, then (1/c_s^2) w_i e_i . g added (Eq. 16). */
void o3_collide_cell(const o3_cfg *c, const double *M, const double *Minv, const double *dfc,
                     double gx, double gy, double gz, double *out) {
  const int simple = c->force == O3_FORCE_SIMPLE;
  double drho, ux, uy, uz, dfeq[19], Gt[19];
  o3_cell_macros(dfc, c->rho0, simple ? 0.0 : 0.5 * gx, simple ? 0.0 : 0.5 * gy,
                 simple ? 0.0 : 0.5 * gz, &drho, &ux, &uy, &uz);
  o3_feq_shifted(drho, c->rho0, ux, uy, uz, dfeq);
  if (simple) {
    for (int i = 0; i < 19; i++) Gt[i] = 0.0;
  } else {
    o3_guo_source(ux, uy, uz, gx, gy, gz, Gt);
  }
  if (c->collision == O3_SRT) {
    double lam = c->tau;
    for (int i = 0; i < 19; i++)
      out[i] = dfc[i] - (dfc[i] - dfeq[i]) / lam + (1.0 - 1.0 / (2.0 * lam)) * Gt[i];
  } else {
    double m[19], meq[19], mG[19], ms[19];
    for (int r = 0; r < 19; r++) {
      m[r] = meq[r] = mG[r] = 0;
      for (int i = 0; i < 19; i++) {
        m[r] += M[r * 19 + i] * dfc[i];
        meq[r] += M[r * 19 + i] * dfeq[i];
        mG[r] += M[r * 19 + i] * Gt[i];
      }
    }
    for (int r = 0; r < 19; r++)
      ms[r] = m[r] - c->s[r] * (m[r] - meq[r]) + (1.0 - 0.5 * c->s[r]) * mG[r];
    for (int i = 0; i < 19; i++) {
      out[i] = 0;
      for (int r = 0; r < 19; r++) out[i] += Minv[i * 19 + r] * ms[r];
    }
  }
  if (simple)
    for (int i = 0; i < 19; i++)
      out[i] += WT[i] * INV_CS2 * (EX[i] * gx + EY[i] * gy + EZ[i] * gz);
}

/* --------------------------------------------------- Peskin delta kernel ---
 * delta_h(x) = phi(x) phi(y) phi(z) with Peskin's four-point phi (the kernel the paper
 * names after Eq. 6, in three dimensions):
 *   phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2)) / 8,   |r| <= 1
 *          = (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2)) / 8,  1 <= |r| <= 2,  0 beyond. */
double o3_phi(double r) {
  double a = fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}

static int wrapn(int v, int n) { v %= n; return v < 0 ? v + n : v; }
static long node(const o3_cfg *c, int x, int y, int z) {
  return ((long)wrapn(z, c->nz) * c->ny + wrapn(y, c->ny)) * c->nx + wrapn(x, c->nx);
}

/* Spreading (Eq. 17 in three dimensions): g(x) += P_k delta_h(x - X_k) over the 4 x 4 x 4
 * nodes of each marker's support, P_k = G_k dA_k the force the marker carries. */
void o3_spread(const o3_cfg *c, const double *X, int n, const double *P, double *gx,
               double *gy, double *gz) {
  for (int k = 0; k < n; k++) {
    int bx = (int)floor(X[3 * k]) - 1, by = (int)floor(X[3 * k + 1]) - 1;
    int bz = (int)floor(X[3 * k + 2]) - 1;
    for (int dz = 0; dz < 4; dz++)
      for (int dy = 0; dy < 4; dy++)
        for (int dx = 0; dx < 4; dx++) {
          int x = bx + dx, y = by + dy, z = bz + dz;
          double w = o3_phi(x - X[3 * k]) * o3_phi(y - X[3 * k + 1]) * o3_phi(z - X[3 * k + 2]);
          long p = node(c, x, y, z);
          gx[p] += P[3 * k] * w;
          gy[p] += P[3 * k + 1] * w;
          gz[p] += P[3 * k + 2] * w;
        }
  }
}

/* Interpolation (Eq. 20): U_k = sum_x u(x) delta_h(x - X_k). */
void o3_interp(const o3_cfg *c, const double *X, int n, const double *ux, const double *uy,
               const double *uz, double *U) {
  for (int k = 0; k < n; k++) {
    int bx = (int)floor(X[3 * k]) - 1, by = (int)floor(X[3 * k + 1]) - 1;
    int bz = (int)floor(X[3 * k + 2]) - 1;
    double s[3] = {0, 0, 0};
    for (int dz = 0; dz < 4; dz++)
      for (int dy = 0; dy < 4; dy++)
        for (int dx = 0; dx < 4; dx++) {
          int x = bx + dx, y = by + dy, z = bz + dz;
          double w = o3_phi(x - X[3 * k]) * o3_phi(y - X[3 * k + 1]) * o3_phi(z - X[3 * k + 2]);
          long p = node(c, x, y, z);
          s[0] += ux[p] * w;
          s[1] += uy[p] * w;
          s[2] += uz[p] * w;
        }
    U[3 * k] = s[0];
    U[3 * k + 1] = s[1];
    U[3 * k + 2] = s[2];
  }
}

/* ----------------------------------------------------- surface geometry ---
 * For the triangulated surface X (triangles counter-clockwise seen from outside):
 *   N_t = (B - A) x (C - A), the outward normal of triangle t times twice its area;
 *   area_k = sum over the triangles t at vertex k of |N_t| / 6 (a third of each);
 *   n_k = sum_t N_t / |sum_t N_t| (the area-weighted vertex normal, section 3.1's n).
 * The surface Jacobian |X_r x X_s| of section 3.1 at vertex k is area_k / Aref_k: the
 * current area of the vertex's surface element over its reference area. */
void o3_surface_geometry(const double *X, int n, const int *tri, int m, double *nrm,
                         double *area) {
  for (int k = 0; k < n; k++) {
    nrm[3 * k] = nrm[3 * k + 1] = nrm[3 * k + 2] = 0;
    area[k] = 0;
  }
  for (int t = 0; t < m; t++) {
    const double *A = X + 3 * tri[3 * t], *B = X + 3 * tri[3 * t + 1], *C = X + 3 * tri[3 * t + 2];
    double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double N[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double a = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]) / 6.0;
    for (int j = 0; j < 3; j++) {
      int k = tri[3 * t + j];
      area[k] += a;
      nrm[3 * k] += N[0];
      nrm[3 * k + 1] += N[1];
      nrm[3 * k + 2] += N[2];
    }
  }
  for (int k = 0; k < n; k++) {
    double l = sqrt(nrm[3 * k] * nrm[3 * k] + nrm[3 * k + 1] * nrm[3 * k + 1] +
                    nrm[3 * k + 2] * nrm[3 * k + 2]);
    if (l > 0) {
      nrm[3 * k] /= l;
      nrm[3 * k + 1] /= l;
      nrm[3 * k + 2] /= l;
    }
  }
}

/* Surface tension (the three-dimensional counterpart of the membrane force of Eq. 19):
 * the surface's energy is gamma times its area, and the force on the fluid at vertex k,
 * per unit reference area, is G_k = -gamma (d Area / d X_k) / Aref_k, with
 *   d area_t / d X_k = (1/2) N_t/|N_t| x (X_q - X_p)
 * for triangle t = (k, p, q) in counter-clockwise order. */
void o3_tension_forces(const double *X, int n, const int *tri, int m, const double *Aref,
                       double gamma, double *G) {
  for (int k = 0; k < 3 * n; k++) G[k] = 0;
  for (int t = 0; t < m; t++) {
    int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    const double *A = X + 3 * v[0], *B = X + 3 * v[1], *C = X + 3 * v[2];
    double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double N[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double l = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    double h[3] = {N[0] / l, N[1] / l, N[2] / l};
    for (int j = 0; j < 3; j++) {
      int k = v[j], p = v[(j + 1) % 3], q = v[(j + 2) % 3];
      double e[3] = {X[3 * q] - X[3 * p], X[3 * q + 1] - X[3 * p + 1], X[3 * q + 2] - X[3 * p + 2]};
      double dA[3] = {0.5 * (h[1] * e[2] - h[2] * e[1]), 0.5 * (h[2] * e[0] - h[0] * e[2]),
                      0.5 * (h[0] * e[1] - h[1] * e[0])};
      for (int d = 0; d < 3; d++) G[3 * k + d] -= gamma * dA[d];
    }
  }
  for (int k = 0; k < n; k++)
    for (int d = 0; d < 3; d++) G[3 * k + d] /= Aref[k];
}

/* Normal split (section 3.1, Eqs. 32 and 46 in three dimensions): with the vertex normal
 * n_k and Jacobian J_k = area_k / Aref_k,
 *   Fn_k = G_k . n_k / J_k          (the jump strength; the pressure jump [[p]])
 *   Gpar_k = G_k - (G_k . n_k) n_k  (spread like the IB-LBM force). */
void o3_normal_split(const double *G, int n, const double *nrm, const double *area,
                     const double *Aref, double *Fn, double *Gpar) {
  for (int k = 0; k < n; k++) {
    double gn = G[3 * k] * nrm[3 * k] + G[3 * k + 1] * nrm[3 * k + 1] + G[3 * k + 2] * nrm[3 * k + 2];
    Fn[k] = gn / (area[k] / Aref[k]);
    for (int d = 0; d < 3; d++) Gpar[3 * k + d] = G[3 * k + d] - gn * nrm[3 * k + d];
  }
}

/* ------------------------------------------------------------- cut links ---
 * Crossing predicate.  Coordinates are snapped to multiples of 2^-20
 * (q = llrint(v 2^20)); lattice node x is the integer point x 2^20.  A link runs from
 * P = x - e_i to Q = x.  Every lattice node is displaced by the same symbolic vector
 * delta = (eps, eps^2, eps^3), eps -> 0+, which settles every tie (a node on a
 * triangle's plane, a link through an edge or a vertex) consistently:
 *  - plane side of node X:  N.(X + delta - A) = N.(X - A) + eps N_x + eps^2 N_y + eps^3 N_z,
 *    N = (B - A) x (C - A); its sign is that of the first non-zero of
 *    (N.(X - A), N_x, N_y, N_z);
 *  - side of the displaced link line (direction d = e_i) about the edge U -> V:
 *    det[d, U - P - delta, V - P - delta] = det[d, U - P, V - P] - delta.((V - U) x d),
 *    sign of the first non-zero of (det, -w_x, -w_y, -w_z), w = (V - U) x d.
 * The link crosses the triangle iff P and Q lie on opposite sides of its plane and the
 * line is on the same side of all three edges (the side test is then never zero: a
 * line parallel to an edge is parallel to the plane, and P, Q lie on one side of it).
 * The crossing's sign s is the plane side of Q: +1 from inside to outside.  Snapped
 * coordinates within 2^12 of the origin and triangle edges below 8 lattice units keep
 * every determinant exact: edge tests in 64-bit, the plane product in 128-bit. */
#define O3_QBITS 20
#define O3_QSCALE 1048576.0

int64_t o3_quantize(double v) { return (int64_t)llrint(v * O3_QSCALE); }

static int sgn128(__int128 v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }
static int sgn64(int64_t v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

/* Plane side of the (displaced) point X of the triangle A, B, C (snapped). */
int o3_plane_side(const int64_t *A, const int64_t *B, const int64_t *C, const int64_t *X) {
  int64_t u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
  int64_t v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
  int64_t N[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  __int128 r = (__int128)N[0] * (X[0] - A[0]) + (__int128)N[1] * (X[1] - A[1]) +
               (__int128)N[2] * (X[2] - A[2]);
  if (r != 0) return sgn128(r);
  for (int d = 0; d < 3; d++)
    if (N[d] != 0) return sgn64(N[d]);
  return 0;
}

/* Side of the (displaced) line P + t d about the edge U -> V; *det receives the
 * undisplaced determinant det[d, U - P, V - P]. */
int o3_edge_side(const int64_t *P, const int *d, const int64_t *U, const int64_t *V,
                 int64_t *det) {
  int64_t a[3] = {U[0] - P[0], U[1] - P[1], U[2] - P[2]};
  int64_t b[3] = {V[0] - P[0], V[1] - P[1], V[2] - P[2]};
  int64_t axb[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  int64_t o = d[0] * axb[0] + d[1] * axb[1] + d[2] * axb[2];
  *det = o;
  if (o != 0) return sgn64(o);
  int64_t e[3] = {V[0] - U[0], V[1] - U[1], V[2] - U[2]};
  int64_t w[3] = {e[1] * d[2] - e[2] * d[1], e[2] * d[0] - e[0] * d[2], e[0] * d[1] - e[1] * d[0]};
  for (int k = 0; k < 3; k++)
    if (w[k] != 0) return -sgn64(w[k]);
  return 0;
}

/* Does the link of direction i into node (px, py, pz) (unwrapped integers) cross the
 * snapped triangle A, B, C?  Returns the crossing's sign (+1 / -1) or 0, and the
 * barycentric coordinates of the crossing in lam[3] (for A, B, C). */
int o3_link_crosses(const int64_t *A, const int64_t *B, const int64_t *C, int px, int py,
                    int pz, int i, double *lam) {
  const int64_t S = (int64_t)1 << O3_QBITS;
  int d[3] = {EX[i], EY[i], EZ[i]};
  int64_t Q[3] = {(int64_t)px * S, (int64_t)py * S, (int64_t)pz * S};
  int64_t P[3] = {Q[0] - d[0] * S, Q[1] - d[1] * S, Q[2] - d[2] * S};
  int sP = o3_plane_side(A, B, C, P), sQ = o3_plane_side(A, B, C, Q);
  if (sP == sQ || sP == 0 || sQ == 0) return 0;
  int64_t vAB, vBC, vCA;
  int e1 = o3_edge_side(P, d, A, B, &vAB), e2 = o3_edge_side(P, d, B, C, &vBC);
  int e3 = o3_edge_side(P, d, C, A, &vCA);
  if (e1 == 0 || e1 != e2 || e2 != e3) return 0;
  /* barycentric coordinates of the crossing: the signed volumes opposite each vertex */
  double s = (double)vAB + (double)vBC + (double)vCA;
  lam[0] = (double)vBC / s;
  lam[1] = (double)vCA / s;
  lam[2] = (double)vAB / s;
  return sQ;
}

/* Cut links of the surface (Eq. 47 with Eq. 32 in three dimensions): for every triangle
 * and every link x - e_i -> x that crosses it, the record (destination node, i, coef),
 * coef = s w_i / c_s^2 Fn(crossing), Fn interpolated linearly over the triangle from its
 * vertices' Fn.  Candidate destinations: the displaced link spans at most
 * [x - 1 + eps, x + 1 + eps] on each axis, which meets the triangle's bounding box
 * [min, max] only for ceil(min) - 1 <= x <= ceil(max).  Returns the number of records,
 * or -1 past cap. */
int o3_cut_links(const o3_cfg *c, const double *X, const int *tri, int m, const double *Fn,
                 long *cell, int *dir, double *coef, int cap) {
  int r = 0;
  for (int t = 0; t < m; t++) {
    int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
    int64_t q[3][3];
    for (int j = 0; j < 3; j++)
      for (int a = 0; a < 3; a++) q[j][a] = o3_quantize(X[3 * v[j] + a]);
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
      int64_t mn = q[0][a], mx = q[0][a];
      for (int j = 1; j < 3; j++) {
        if (q[j][a] < mn) mn = q[j][a];
        if (q[j][a] > mx) mx = q[j][a];
      }
      lo[a] = (int)-((-mn) >> O3_QBITS) - 1;  /* ceil(min) - 1 */
      hi[a] = (int)-((-mx) >> O3_QBITS);      /* ceil(max) */
    }
    for (int z = lo[2]; z <= hi[2]; z++)
      for (int y = lo[1]; y <= hi[1]; y++)
        for (int x = lo[0]; x <= hi[0]; x++)
          for (int i = 1; i < 19; i++) {
            double lam[3];
            int s = o3_link_crosses(q[0], q[1], q[2], x, y, z, i, lam);
            if (!s) continue;
            if (r >= cap) return -1;
            double fc = lam[0] * Fn[v[0]] + lam[1] * Fn[v[1]] + lam[2] * Fn[v[2]];
            cell[r] = node(c, x, y, z);
            dir[r] = i;
            coef[r] = s * WT[i] * INV_CS2 * fc;
            r++;
          }
  }
  return r;
}

/* Inside indicator of node (x, y, z) (unwrapped): the signed crossings of the chain of
 * +x links from a node left of every vertex up to it (inside = 1).  Used by the tests'
 * path-independence pin and the exact initial states. */
int o3_inside(const double *X, int n, const int *tri, int m, int x, int y, int z) {
  double xmin = X[0];
  for (int k = 1; k < n; k++)
    if (X[3 * k] < xmin) xmin = X[3 * k];
  int x0 = (int)floor(xmin) - 2;
  int w = 0;
  for (int t = 0; t < m; t++) {
    int64_t q[3][3];
    for (int j = 0; j < 3; j++)
      for (int a = 0; a < 3; a++) q[j][a] = o3_quantize(X[3 * tri[3 * t + j] + a]);
    for (int px = x0 + 1; px <= x; px++) {
      double lam[3];
      w -= o3_link_crosses(q[0], q[1], q[2], px, y, z, 1, lam);  /* +1 leaves the inside */
    }
  }
  return w;
}

/* ----------------------------------------------------------------- state --- */
o3_state *o3_create(const o3_cfg *cfg) {
  o3_state *S = (o3_state *)calloc(1, sizeof(o3_state));
  S->c = *cfg;
  long N = (long)cfg->nx * cfg->ny * cfg->nz;
  S->df = (double *)calloc(19 * N, sizeof(double));
  S->f = (double *)calloc(19 * N, sizeof(double));
  S->tmp = (double *)calloc(19 * N, sizeof(double));
  S->gx = (double *)calloc(N, sizeof(double));
  S->gy = (double *)calloc(N, sizeof(double));
  S->gz = (double *)calloc(N, sizeof(double));
  S->rho = (double *)calloc(N, sizeof(double));
  S->ux = (double *)calloc(N, sizeof(double));
  S->uy = (double *)calloc(N, sizeof(double));
  S->uz = (double *)calloc(N, sizeof(double));
  o3_mrt_matrix(S->M);
  o3_mrt_inverse(S->M, S->Minv);
  return S;
}

static void free_iface(o3_state *S) {
  if (!S->has_iface) return;
  free(S->I.X); free(S->I.tri); free(S->I.Aref); free(S->I.Gp);
  free(S->G); free(S->Fn); free(S->Gpar); free(S->U); free(S->nrm); free(S->area);
  S->has_iface = 0;
}

void o3_destroy(o3_state *S) {
  free_iface(S);
  free(S->df); free(S->f); free(S->tmp); free(S->gx); free(S->gy); free(S->gz);
  free(S->rho); free(S->ux); free(S->uy); free(S->uz);
  free(S);
}

static long nnodes(const o3_cfg *c) { return (long)c->nx * c->ny * c->nz; }
void o3_set_df(o3_state *S, const double *df) { memcpy(S->df, df, 19 * nnodes(&S->c) * sizeof(double)); }
void o3_get_df(const o3_state *S, double *df) { memcpy(df, S->df, 19 * nnodes(&S->c) * sizeof(double)); }

/* The equilibrium of rho(x) = rho0 + drho(x), u(x) (NULL: 0). */
void o3_init_equilibrium(o3_state *S, const double *drho, const double *ux, const double *uy,
                         const double *uz) {
  long N = nnodes(&S->c);
  #pragma omp parallel for schedule(static)
  for (long p = 0; p < N; p++) {
    double e[19];
    o3_feq_shifted(drho ? drho[p] : 0, S->c.rho0, ux ? ux[p] : 0, uy ? uy[p] : 0,
                   uz ? uz[p] : 0, e);
    for (int i = 0; i < 19; i++) S->df[i * N + p] = e[i];
  }
}

/* Install the surface: n vertices X[n][3], m triangles tri[m][3] (counter-clockwise from
 * outside).  The reference vertex areas are the initial mesh's (o3_surface_geometry).
 * Returns -1 for a degenerate triangle or an edge of 8 lattice units or more. */
int o3_set_surface(o3_state *S, const double *X, int n, const int *tri, int m, int model,
                   int moves, double gamma, const double *Gp) {
  free_iface(S);
  if (n <= 0) return 0;
  for (int t = 0; t < m; t++) {
    const double *A = X + 3 * tri[3 * t], *B = X + 3 * tri[3 * t + 1], *C = X + 3 * tri[3 * t + 2];
    const double *E[3][2] = {{A, B}, {B, C}, {C, A}};
    for (int j = 0; j < 3; j++) {
      double l2 = 0;
      for (int a = 0; a < 3; a++) l2 += (E[j][1][a] - E[j][0][a]) * (E[j][1][a] - E[j][0][a]);
      if (!(l2 < 64.0) || l2 == 0.0) return -1;
    }
  }
  o3_iface *I = &S->I;
  I->n = n; I->m = m; I->model = model; I->moves = moves; I->gamma = gamma;
  I->X = (double *)malloc(3 * n * sizeof(double));
  I->tri = (int *)malloc(3 * m * sizeof(int));
  I->Aref = (double *)malloc(n * sizeof(double));
  I->Gp = (double *)calloc(3 * n, sizeof(double));
  memcpy(I->X, X, 3 * n * sizeof(double));
  memcpy(I->tri, tri, 3 * m * sizeof(int));
  if (Gp) memcpy(I->Gp, Gp, 3 * n * sizeof(double));
  S->G = (double *)calloc(3 * n, sizeof(double));
  S->Fn = (double *)calloc(n, sizeof(double));
  S->Gpar = (double *)calloc(3 * n, sizeof(double));
  S->U = (double *)calloc(3 * n, sizeof(double));
  S->nrm = (double *)calloc(3 * n, sizeof(double));
  S->area = (double *)calloc(n, sizeof(double));
  o3_surface_geometry(I->X, n, I->tri, m, S->nrm, I->Aref);
  S->has_iface = 1;
  return 0;
}

/* Streaming on the periodic box: out_i(x) = in_i(x - e_i). */
static void stream(const o3_cfg *c, const double *in, double *out) {
  long N = nnodes(c);
  for (int i = 0; i < 19; i++)
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < c->nz; z++)
      for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++)
          out[i * N + node(c, x, y, z)] = in[i * N + node(c, x - EX[i], y - EY[i], z - EZ[i])];
}

/* One time step, t -> t+1 (section 3.2 / Eq. 47, in three dimensions):
 *  1. surface geometry of X^t; Lagrangian force G (prescribed, or surface tension);
 *  2. split: Fn_k (jump strength), Gpar_k;
 *  3. II-LBM: f = df + [[f]] on every cut link (Eq. 47), g = spread(Gpar dA) + body;
 *     IB-LBM: f = df, g = spread(G dA) + body;
 *  4. rho, u from f and g (Eq. 24; the simple force term: u = sum e f / rho), U_k =
 *     interp(u) (Eq. 20);
 *  5. collide every node, stream;
 *  6. X^{t+1} = X^t + U (moving surface). */
int o3_prepare(o3_state *S) {
  const o3_cfg *c = &S->c;
  long N = nnodes(c);
  memcpy(S->f, S->df, 19 * N * sizeof(double));
  for (long p = 0; p < N; p++) { S->gx[p] = c->body[0]; S->gy[p] = c->body[1]; S->gz[p] = c->body[2]; }
  S->ncut = 0;
  if (S->has_iface) {
    o3_iface *I = &S->I;
    int n = I->n;
    o3_surface_geometry(I->X, n, I->tri, I->m, S->nrm, S->area);
    if (I->model == O3_TENSION) o3_tension_forces(I->X, n, I->tri, I->m, I->Aref, I->gamma, S->G);
    else memcpy(S->G, I->Gp, 3 * n * sizeof(double));
    o3_normal_split(S->G, n, S->nrm, S->area, I->Aref, S->Fn, S->Gpar);
    double *P = (double *)malloc(3 * n * sizeof(double));
    if (c->jump) {
      int cap = 256 * I->m + 64;
      long *cell = (long *)malloc(cap * sizeof(long));
      int *dir = (int *)malloc(cap * sizeof(int));
      double *coef = (double *)malloc(cap * sizeof(double));
      int r = o3_cut_links(c, I->X, I->tri, I->m, S->Fn, cell, dir, coef, cap);
      if (r < 0) { free(cell); free(dir); free(coef); free(P); return -1; }
      for (int q = 0; q < r; q++) S->f[dir[q] * N + cell[q]] += coef[q];
      S->ncut = r;
      free(cell); free(dir); free(coef);
      for (int k = 0; k < n; k++)
        for (int d = 0; d < 3; d++) P[3 * k + d] = S->Gpar[3 * k + d] * I->Aref[k];
    } else {
      for (int k = 0; k < n; k++)
        for (int d = 0; d < 3; d++) P[3 * k + d] = S->G[3 * k + d] * I->Aref[k];
    }
    o3_spread(c, I->X, n, P, S->gx, S->gy, S->gz);
    free(P);
  }
  const int simple = c->force == O3_FORCE_SIMPLE;
  #pragma omp parallel for schedule(static)
  for (long p = 0; p < N; p++) {
    double dfc[19];
    for (int i = 0; i < 19; i++) dfc[i] = S->f[i * N + p];
    o3_cell_macros(dfc, c->rho0, simple ? 0 : 0.5 * S->gx[p], simple ? 0 : 0.5 * S->gy[p],
                   simple ? 0 : 0.5 * S->gz[p], &S->rho[p], &S->ux[p], &S->uy[p], &S->uz[p]);
  }
  if (S->has_iface) o3_interp(c, S->I.X, S->I.n, S->ux, S->uy, S->uz, S->U);
  return 0;
}

void o3_advance(o3_state *S) {
  const o3_cfg *c = &S->c;
  long N = nnodes(c);
  #pragma omp parallel for schedule(static)
  for (long p = 0; p < N; p++) {
    double dfc[19], out[19];
    for (int i = 0; i < 19; i++) dfc[i] = S->f[i * N + p];
    o3_collide_cell(c, S->M, S->Minv, dfc, S->gx[p], S->gy[p], S->gz[p], out);
    for (int i = 0; i < 19; i++) S->tmp[i * N + p] = out[i];
  }
  stream(c, S->tmp, S->df);
  if (S->has_iface && S->I.moves)
    for (int k = 0; k < 3 * S->I.n; k++) S->I.X[k] += S->U[k];
  S->step++;
}

int o3_step(o3_state *S, int nsteps) {
  for (int s = 0; s < nsteps; s++) {
    if (o3_prepare(S)) return -1;
    o3_advance(S);
  }
  return 0;
}

/* The macroscopic fields the next collision uses (runs the preparation of the current
 * state): drho, u of Eq. 24. */
int o3_current_macros(o3_state *S, double *drho, double *ux, double *uy, double *uz) {
  if (o3_prepare(S)) return -1;
  long N = nnodes(&S->c);
  memcpy(drho, S->rho, N * sizeof(double));
  memcpy(ux, S->ux, N * sizeof(double));
  memcpy(uy, S->uy, N * sizeof(double));
  memcpy(uz, S->uz, N * sizeof(double));
  return 0;
}

/* Markers of the most recent preparation: X (current), G, U, Fn. */
void o3_get_markers(const o3_state *S, double *X, double *G, double *U, double *Fn) {
  int n = S->I.n;
  if (X) memcpy(X, S->I.X, 3 * n * sizeof(double));
  if (G) memcpy(G, S->G, 3 * n * sizeof(double));
  if (U) memcpy(U, S->U, 3 * n * sizeof(double));
  if (Fn) memcpy(Fn, S->Fn, n * sizeof(double));
}
int o3_cut_link_count(const o3_state *S) { return S->ncut; }
void o3_get_ref_area(const o3_state *S, double *A) { memcpy(A, S->I.Aref, S->I.n * sizeof(double)); }

/* Enclosed volume of the surface: (1/6) sum over triangles of A . (B x C). */
double o3_volume(const double *X, const int *tri, int m) {
  double v = 0;
  for (int t = 0; t < m; t++) {
    const double *A = X + 3 * tri[3 * t], *B = X + 3 * tri[3 * t + 1], *C = X + 3 * tri[3 * t + 2];
    v += A[0] * (B[1] * C[2] - B[2] * C[1]) + A[1] * (B[2] * C[0] - B[0] * C[2]) +
         A[2] * (B[0] * C[1] - B[1] * C[0]);
  }
  return v / 6.0;
}

/* The jump field of the current state's surface, J[i-1][N] (i = 1..18), for the tests. */
int o3_jump_field(o3_state *S, double *J) {
  long N = nnodes(&S->c);
  memset(J, 0, 18 * N * sizeof(double));
  if (!S->has_iface || !S->c.jump) return 0;
  if (o3_prepare(S)) return -1;
  int cap = 256 * S->I.m + 64;
  long *cell = (long *)malloc(cap * sizeof(long));
  int *dir = (int *)malloc(cap * sizeof(int));
  double *coef = (double *)malloc(cap * sizeof(double));
  int r = o3_cut_links(&S->c, S->I.X, S->I.tri, S->I.m, S->Fn, cell, dir, coef, cap);
  for (int q = 0; q < r; q++) J[(dir[q] - 1) * N + cell[q]] += coef[q];
  free(cell); free(dir); free(coef);
  return r;
}
