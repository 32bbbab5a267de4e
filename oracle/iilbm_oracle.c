/*
 * iilbm_oracle.c -- plain, slow FP64 CPU oracle of one immersed interface–lattice
 * Boltzmann (II-LBM) time step (Qin, Kolahdouz & Griffith, arXiv 2003.12186).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or constant with the CUDA library; it is compiled on its own with gcc
 * (-ffp-contract=off so the host never fuses multiply-adds).
 *
 * Every routine below is a direct transcription of a definition in the paper
 * (section / equation given beside it) in FP64, with plain loops and no blocking,
 * fusion or reordering beyond what the definition states.  Where the paper is
 * silent or garbled the reading taken is stated in the routine's comment.
 *
 * Notation follows the paper: D2Q9 velocities e_i, weights w_i (Eq. 9),
 * c_s^2 = 1/3, relaxation time lambda (here "tau"), Lagrangian markers X_k,
 * Lagrangian force density G_k, Eulerian force density g, delta kernel delta_h.
 *
 * Populations are held as shifted deviations df_i = f_i - w_i*rho0.  This is an
 * exact change of variables (sum_i w_i = 1, sum_i w_i e_i = 0); it keeps the
 * FP64 rounding of the O(1) rest state out of the O(u) flow quantities.
 *
 * Layout: df[i*ny*nx + y*nx + x]  (structure of arrays, natural "pull" order).
 *
 * The same source also builds with -fopenmp (the all-core CPU baseline): the
 * "omp parallel for" lines mark the per-node loops whose iterations touch disjoint
 * nodes, so the parallel build computes every value exactly as the serial one does.
 * Spreading, which accumulates, and the marker loops stay serial.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- D2Q9 lattice, section 2.2.1 (velocity set), Eq. 9 (weights) ----------
 * Ordering: 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.  This is the
 * ordering the schematic of the paper implies (point P1 of its first figure
 * receives the jump on f3 and f7, point P2 on f1, f5, f8). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* c_s = 1/sqrt(3) (section 2.2.1), so 1/c_s^2 = 3 exactly: every 1/c_s^2 and 1/c_s^4
 * of the paper is applied as a multiplication by 3 or 9, never as a division by a
 * rounded 1/3 (which would bias every equilibrium by the same one-ulp error). */
#define INV_CS2 3.0

/* ---------------------------------------------------------------- config --- */
enum { ORC_SRT = 0, ORC_MRT = 1 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_WALLS_Y = 1, ORC_BC_CHANNEL = 2, ORC_BC_BOX_OUTFLOW = 3,
       ORC_BC_BOX_WALL = 4 };
enum { ORC_FORCE_GUO = 0, ORC_FORCE_SIMPLE = 1 };
enum { ORC_SPRING = 0, ORC_SPRING_REST = 1, ORC_PRESCRIBED = 2, ORC_DIRECT = 3 };

typedef struct {
  int nx, ny;
  int collision;   /* ORC_SRT or ORC_MRT */
  double tau;      /* relaxation time lambda (Eq. 7) */
  double s[9];     /* MRT rates, moment order (rho, e, eps, jx, qx, jy, qy, pxx, pxy) */
  double rho0;     /* reference density of the shifted storage */
  int bc;          /* ORC_BC_* */
  double u_max;    /* channel: centre-line inflow speed */
  double body_x, body_y; /* uniform body force density added to g */
  int jump;        /* 1: II-LBM (normal force through the jump, tangential spread);
                      0: IB-LBM with Guo forcing (whole G spread) */
  int force;       /* ORC_FORCE_GUO (Eqs. 21-24) or ORC_FORCE_SIMPLE (the simple
                      external force term of Eq. 16, u = sum e f / rho) */
} orc_cfg;

typedef struct {
  int n;           /* number of markers (closed polygon, counter-clockwise) */
  int model;       /* ORC_SPRING / ORC_SPRING_REST / ORC_PRESCRIBED / ORC_DIRECT */
  int moves;       /* 1: markers advected (membrane); 0: fixed (rigid, at rest) */
  double kappa;    /* spring stiffness */
  double dX;       /* Lagrangian parameter spacing Delta X */
  double l0;       /* rest length (ORC_SPRING_REST) */
  double eta;      /* direct-forcing gain (ORC_DIRECT) */
  int mdf_iters;   /* direct forcing: maximum iterations */
  double mdf_tol;  /* direct forcing: stop when max_k |U^D - U_k| < tol (0: run all) */
  int curve;       /* interface for the jump: 0 the marker polygon; m >= 1 the cubic
                      spline through the markers (normals, |X_s|, Fn along it), its
                      crossings taken on m chords per segment */
  double *X;       /* [n][2] */
  double *Gp;      /* prescribed G [n][2] (ORC_PRESCRIBED) / warm-start G (ORC_DIRECT) */
  double *UD;      /* desired velocity [n][2] (ORC_DIRECT) */
} orc_iface;

typedef struct {
  orc_cfg c;
  double *df;      /* [9][ny][nx] state: streamed populations, jump not yet added */
  double *tmp;     /* [9][ny][nx] scratch */
  double *f;       /* [9][ny][nx] populations of the current step (state + jump) */
  double *gx, *gy; /* Eulerian force density of the current step */
  double *rho, *ux, *uy; /* current step's drho = rho - rho0 and u (Eqs. 11, 24) */
  double M[81], Minv[81];
  int has_iface;
  orc_iface I;
  double *G;       /* [n][2] Lagrangian force of the current step */
  double *Fn;      /* [n] normal traction G.n/|X_s| */
  double *Gpar;    /* [n][2] tangential force G - (G.n)n */
  double *U;       /* [n][2] interpolated marker velocity */
  int mdf_last_iters;
  double mdf_last_res;
  double *Ustar;   /* [n][2] U* = interp(u*): marker velocity without the body's force */
  int ws_previous; /* direct forcing starts from the force of the previous call, */
  double *Gprev;   /* kept here, instead of from Gp */
  int ncut;        /* cut-link crossings of the most recent prepare */
  long step;
  /* rigid body (section 2.3) carrying a directly forced interface */
  int has_body;
  int body_mode;     /* ORC_BODY_PRESCRIBED_X or ORC_BODY_FREE */
  int body_dof;      /* FREE: free degrees of freedom, bits 1 x, 2 y, 4 rotation */
  double body_A, body_umax;              /* PRESCRIBED_X: amplitude, peak velocity */
  double body_m, body_I, body_Vs;        /* mass, moment of inertia, area */
  double body_k[3], body_c[3];           /* spring and damper per degree of freedom */
  double Xc0[2], Xc[2], Uc[2], Ucp[2], ac[2], th, Wb, Wbp, wb;  /* state */
  double Fext[3];                        /* the last F_ext (x, y) and T_ext (Eqs. 25-26) */
  double *X0;                            /* marker offsets from Xc0 at theta = 0 */
} orc_state;

enum { ORC_BODY_PRESCRIBED_X = 1, ORC_BODY_FREE = 2 };

/* ------------------------------------------------------------ MRT matrix ---
 * Lallemand & Luo D2Q9 moment basis (cited in section 2.1.1 / 2.2.1): rows are
 * the polynomials 1, -4+3|e|^2, 4-21/2|e|^2+9/2|e|^4, e_x, (-5+3|e|^2)e_x, e_y,
 * (-5+3|e|^2)e_y, e_x^2-e_y^2, e_x e_y evaluated on the nine velocities.
 * The rates s_0..s_8 of section 2.2.1 index these rows in this order. */
void orc_mrt_matrix(double *M) {
  for (int i = 0; i < 9; i++) {
    double ex = EX[i], ey = EY[i], e2 = ex * ex + ey * ey;
    M[0 * 9 + i] = 1.0;
    M[1 * 9 + i] = -4.0 + 3.0 * e2;
    M[2 * 9 + i] = 4.0 - 10.5 * e2 + 4.5 * e2 * e2;
    M[3 * 9 + i] = ex;
    M[4 * 9 + i] = (-5.0 + 3.0 * e2) * ex;
    M[5 * 9 + i] = ey;
    M[6 * 9 + i] = (-5.0 + 3.0 * e2) * ey;
    M[7 * 9 + i] = ex * ex - ey * ey;
    M[8 * 9 + i] = ex * ey;
  }
}

/* M^-1 of an orthogonal-row basis: M^-1 = M^T diag(1/|row_r|^2).  The squared row
 * norms are sums of squared small integers (exact), so each entry is the correctly
 * rounded M_ri / |row_r|^2. */
void orc_mrt_inverse(const double *M, double *Minv) {
  for (int r = 0; r < 9; r++) {
    double nrm = 0;
    for (int i = 0; i < 9; i++) nrm += M[r * 9 + i] * M[r * 9 + i];
    for (int i = 0; i < 9; i++) Minv[i * 9 + r] = M[r * 9 + i] / nrm;
  }
}

/* Gauss–Jordan inverse with partial pivoting (library-style primitive; used by the
 * tests to check the orthogonal-basis inverse). */
int orc_invert9(const double *A, double *Ainv) {
  double a[9][18];
  for (int r = 0; r < 9; r++)
    for (int c = 0; c < 18; c++)
      a[r][c] = c < 9 ? A[r * 9 + c] : (c - 9 == r ? 1.0 : 0.0);
  for (int col = 0; col < 9; col++) {
    int piv = col;
    for (int r = col + 1; r < 9; r++)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (fabs(a[piv][col]) < 1e-300) return -1;
    if (piv != col)
      for (int c = 0; c < 18; c++) { double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t; }
    double p = a[col][col];
    for (int c = 0; c < 18; c++) a[col][c] /= p;
    for (int r = 0; r < 9; r++) {
      if (r == col) continue;
      double m = a[r][col];
      if (m != 0.0)
        for (int c = 0; c < 18; c++) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < 9; r++)
    for (int c = 0; c < 9; c++) Ainv[r * 9 + c] = a[r][c + 9];
  return 0;
}

/* ------------------------------------------------------ equilibrium, force --
 * Guo-form equilibrium, Eq. 23: f_eq_i = w_i (p/c_s^2)[1 + e.u/c_s^2 +
 * (e.u)^2/(2c_s^4) - u^2/(2c_s^2)], with p/c_s^2 = rho = sum_i f_i (Eq. 11; the
 * sum runs over every i including the rest population -- the printed lower limit
 * 1 is read as a typo).  Returned shifted by w_i*rho0, from the density deviation
 * drho = rho - rho0 = sum_i df_i (carried as such, never formed as a difference). */
void orc_feq_shifted(double drho, double rho0, double ux, double uy, double *dfeq) {
  double u2 = ux * ux + uy * uy;
  double rho = rho0 + drho;
  for (int i = 0; i < 9; i++) {
    double eu = EX[i] * ux + EY[i] * uy;
    double poly = eu * INV_CS2 + eu * eu * (INV_CS2 * INV_CS2 / 2.0) - u2 * (INV_CS2 / 2.0);
    dfeq[i] = WT[i] * (drho + rho * poly);
  }
}

/* Guo source without its relaxation prefactor, Eqs. 21-22:
 * Gt_i = w_i [ (e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4 ] . g */
void orc_guo_source(double ux, double uy, double gx, double gy, double *Gt) {
  for (int i = 0; i < 9; i++) {
    double eu = EX[i] * ux + EY[i] * uy;
    double t1 = ((EX[i] - ux) * gx + (EY[i] - uy) * gy) * INV_CS2;
    double t2 = eu * (EX[i] * gx + EY[i] * gy) * (INV_CS2 * INV_CS2);
    Gt[i] = WT[i] * (t1 + t2);
  }
}

/* Macroscopic density deviation and velocity of one cell: drho = sum df
 * (Eq. 11 less rho0), rho u = sum_i e_i f_i + g/2 (Eq. 24), rho = rho0 + drho. */
void orc_cell_macros(const double *dfc, double rho0, double gx, double gy,
                     double *drho, double *ux, double *uy) {
  double s = 0, jx = 0, jy = 0;
  for (int i = 0; i < 9; i++) {
    s += dfc[i];
    jx += EX[i] * dfc[i];
    jy += EY[i] * dfc[i];
  }
  *drho = s;
  *ux = (jx + 0.5 * gx) / (rho0 + s);
  *uy = (jy + 0.5 * gy) / (rho0 + s);
}

/* Collision of one cell (shifted populations in and out).
 *  SRT, Eq. 14 with Guo's term Eq. 21:
 *    f* = f - (f - f_eq)/lambda + (1 - 1/(2 lambda)) Gt
 *  MRT, Eq. 15 with Guo's term Eq. 22:
 *    f* = f - M^-1 S (M f - M f_eq) + M^-1 (I - S/2) M Gt
 * The shift w_i rho0 cancels in f - f_eq and passes through M^-1 M unchanged. */
void orc_collide_cell(const orc_cfg *c, const double *M, const double *Minv,
                      const double *dfc, double gx, double gy, double *out) {
  double drho, ux, uy, dfeq[9], Gt[9];
  if (c->force == ORC_FORCE_SIMPLE) {
    /* Eq. 16 with Eq. 14 / 15: u = sum e f / rho, the relaxation, then the simple
     * external force term (1/c_s^2) w_i e_i . g added to every population */
    orc_cell_macros(dfc, c->rho0, 0.0, 0.0, &drho, &ux, &uy);
    orc_feq_shifted(drho, c->rho0, ux, uy, dfeq);
    if (c->collision == ORC_SRT) {
      for (int i = 0; i < 9; i++) out[i] = dfc[i] - (dfc[i] - dfeq[i]) / c->tau;
    } else {
      double m[9], meq[9], ms[9];
      for (int r = 0; r < 9; r++) {
        m[r] = meq[r] = 0;
        for (int i = 0; i < 9; i++) {
          m[r] += M[r * 9 + i] * dfc[i];
          meq[r] += M[r * 9 + i] * dfeq[i];
        }
      }
      for (int r = 0; r < 9; r++) ms[r] = m[r] - c->s[r] * (m[r] - meq[r]);
      for (int i = 0; i < 9; i++) {
        out[i] = 0;
        for (int r = 0; r < 9; r++) out[i] += Minv[i * 9 + r] * ms[r];
      }
    }
    for (int i = 0; i < 9; i++) out[i] += WT[i] * INV_CS2 * (EX[i] * gx + EY[i] * gy);
    return;
  }
  orc_cell_macros(dfc, c->rho0, gx, gy, &drho, &ux, &uy);
  orc_feq_shifted(drho, c->rho0, ux, uy, dfeq);
  orc_guo_source(ux, uy, gx, gy, Gt);
  if (c->collision == ORC_SRT) {
    double lam = c->tau;
    for (int i = 0; i < 9; i++)
      out[i] = dfc[i] - (dfc[i] - dfeq[i]) / lam + (1.0 - 1.0 / (2.0 * lam)) * Gt[i];
  } else {
    double m[9], meq[9], mG[9], ms[9];
    for (int r = 0; r < 9; r++) {
      m[r] = meq[r] = mG[r] = 0;
      for (int i = 0; i < 9; i++) {
        m[r] += M[r * 9 + i] * dfc[i];
        meq[r] += M[r * 9 + i] * dfeq[i];
        mG[r] += M[r * 9 + i] * Gt[i];
      }
    }
    for (int r = 0; r < 9; r++)
      ms[r] = m[r] - c->s[r] * (m[r] - meq[r]) + (1.0 - 0.5 * c->s[r]) * mG[r];
    for (int i = 0; i < 9; i++) {
      out[i] = 0;
      for (int r = 0; r < 9; r++) out[i] += Minv[i * 9 + r] * ms[r];
    }
  }
}

/* --------------------------------------------------- Peskin delta kernel ---
 * Four-point regularised delta of Peskin (Acta Numerica 2002), the kernel the
 * paper names after Eq. 6: delta_h(x) = phi(x) phi(y) with
 *   phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2)) / 8,   |r| <= 1
 *          = (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2)) / 8,  1 <= |r| <= 2
 *          = 0 otherwise. */
double orc_phi(double r) {
  double a = fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}

/* Map a lattice coordinate to a cell index along one axis; -1 if outside a
 * non-periodic axis. */
static int wrap_axis(int v, int n, int periodic) {
  if (periodic) { v %= n; if (v < 0) v += n; return v; }
  return (v >= 0 && v < n) ? v : -1;
}
static int periodic_x(const orc_cfg *c) { return c->bc == ORC_BC_PERIODIC || c->bc == ORC_BC_WALLS_Y; }
static int periodic_y(const orc_cfg *c) { return c->bc == ORC_BC_PERIODIC; }
static int is_box(const orc_cfg *c) { return c->bc == ORC_BC_BOX_OUTFLOW || c->bc == ORC_BC_BOX_WALL; }

/* Force spreading, Eq. 17 / Eq. 46: g(x) += sum_k P_k delta_h(x - X_k), where
 * P_k = G_k Delta X is the point force of marker k (lattice units, Delta x = 1). */
void orc_spread(const orc_cfg *c, const double *X, int n, const double *P,
                double *gx, double *gy) {
  for (int k = 0; k < n; k++) {
    int x0 = (int)floor(X[2 * k]) - 1, y0 = (int)floor(X[2 * k + 1]) - 1;
    for (int b = 0; b < 4; b++)
      for (int a = 0; a < 4; a++) {
        int xi = wrap_axis(x0 + a, c->nx, periodic_x(c));
        int yi = wrap_axis(y0 + b, c->ny, periodic_y(c));
        if (xi < 0 || yi < 0) continue;
        double d = orc_phi(x0 + a - X[2 * k]) * orc_phi(y0 + b - X[2 * k + 1]);
        gx[yi * c->nx + xi] += P[2 * k] * d;
        gy[yi * c->nx + xi] += P[2 * k + 1] * d;
      }
  }
}

/* Velocity interpolation, Eq. 20 (and U* of Eq. 18): U_k = sum_x u(x) delta_h(x - X_k). */
void orc_interp(const orc_cfg *c, const double *X, int n, const double *ux,
                const double *uy, double *U) {
  for (int k = 0; k < n; k++) {
    int x0 = (int)floor(X[2 * k]) - 1, y0 = (int)floor(X[2 * k + 1]) - 1;
    double sx = 0, sy = 0;
    for (int b = 0; b < 4; b++)
      for (int a = 0; a < 4; a++) {
        int xi = wrap_axis(x0 + a, c->nx, periodic_x(c));
        int yi = wrap_axis(y0 + b, c->ny, periodic_y(c));
        if (xi < 0 || yi < 0) continue;
        double d = orc_phi(x0 + a - X[2 * k]) * orc_phi(y0 + b - X[2 * k + 1]);
        sx += ux[yi * c->nx + xi] * d;
        sy += uy[yi * c->nx + xi] * d;
      }
    U[2 * k] = sx;
    U[2 * k + 1] = sy;
  }
}

/* --------------------------------------------------- Lagrangian forces -----
 * Membrane spring force, Eq. 19: G_k = kappa (X_{k+1} - 2 X_k + X_{k-1}) / dX^2.
 * Rest-length spring (a linear spring of rest length l0 on every segment, a
 * variant the paper's Eq. 19 reduces to at l0 = 0): segment tension
 * T = kappa (l/l0 - 1) along the segment, point force on marker k
 * P_k = T_k t_k - T_{k-1} t_{k-1}, G_k = P_k / dX. */
void orc_spring_forces(const orc_iface *I, double *G) {
  int n = I->n;
  for (int k = 0; k < n; k++) {
    int kp = (k + 1) % n, km = (k + n - 1) % n;
    const double *Xk = I->X + 2 * k, *Xp = I->X + 2 * kp, *Xm = I->X + 2 * km;
    if (I->model == ORC_SPRING) {
      G[2 * k] = I->kappa * (Xp[0] - 2.0 * Xk[0] + Xm[0]) / (I->dX * I->dX);
      G[2 * k + 1] = I->kappa * (Xp[1] - 2.0 * Xk[1] + Xm[1]) / (I->dX * I->dX);
    } else {
      double ax = Xp[0] - Xk[0], ay = Xp[1] - Xk[1];
      double bx = Xk[0] - Xm[0], by = Xk[1] - Xm[1];
      double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
      double Ta = I->kappa * (la / I->l0 - 1.0), Tb = I->kappa * (lb / I->l0 - 1.0);
      G[2 * k] = (Ta * ax / la - Tb * bx / lb) / I->dX;
      G[2 * k + 1] = (Ta * ay / la - Tb * by / lb) / I->dX;
    }
  }
}

/* -------------------------------------------------- cubic spline interface ---
 * For flexible boundaries the paper represents the interface by a cubic spline (after
 * Lee & LeVeque, end of section 3.2).  Reading: the periodic interpolating cubic spline
 * through the markers, parametrised by the marker index (s = k at marker k, the
 * markers being about equally spaced), in uniform B-spline form
 *   v(k + t) = c_{k-1} (1-t)^3/6 + c_k (3t^3 - 6t^2 + 4)/6
 *            + c_{k+1} (-3t^3 + 3t^2 + 3t + 1)/6 + c_{k+2} t^3/6,   0 <= t < 1,
 * whose interpolation conditions v(k) = (c_{k-1} + 4 c_k + c_{k+1})/6 = v_k form a
 * cyclic tridiagonal system for the coefficients c. */

/* Coefficients c[k*stride] of the periodic spline through v[k*stride], k < n (n >= 3):
 * the cyclic system (c_{k-1} + 4 c_k + c_{k+1}) = 6 v_k solved by the Sherman-Morrison
 * formula around a tridiagonal (Thomas) solve. */
void orc_spline_coeffs(const double *v, int n, int stride, double *c) {
  /* A = T + u w^T, u = (g, 0, .., 0, 1), w = (1, 0, .., 0, 1/g), g = -4: T is the
   * tridiagonal part with its first and last diagonal entries changed so that u w^T
   * restores the two corner entries (each 1). */
  const double g = -4.0;
  double *diag = (double *)malloc(n * sizeof(double));
  double *y = (double *)malloc(n * sizeof(double)), *z = (double *)malloc(n * sizeof(double));
  double *rhs = (double *)malloc(n * sizeof(double)), *u = (double *)malloc(n * sizeof(double));
  double *cp = (double *)malloc(n * sizeof(double)), *dp = (double *)malloc(n * sizeof(double));
  for (int k = 0; k < n; k++) { diag[k] = 4.0; rhs[k] = 6.0 * v[k * stride]; u[k] = 0.0; }
  diag[0] -= g;
  diag[n - 1] -= 1.0 / g;
  u[0] = g;
  u[n - 1] = 1.0;
  /* Thomas solves of T y = rhs and T z = u (sub- and super-diagonal entries 1) */
  for (int pass = 0; pass < 2; pass++) {
    const double *b = pass == 0 ? rhs : u;
    double *x = pass == 0 ? y : z;
    cp[0] = 1.0 / diag[0];
    dp[0] = b[0] / diag[0];
    for (int k = 1; k < n; k++) {
      double m = diag[k] - cp[k - 1];
      cp[k] = 1.0 / m;
      dp[k] = (b[k] - dp[k - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int k = n - 2; k >= 0; k--) x[k] = dp[k] - cp[k] * x[k + 1];
  }
  double wy = y[0] + y[n - 1] / g, wz = z[0] + z[n - 1] / g;
  double f = wy / (1.0 + wz);
  for (int k = 0; k < n; k++) c[k * stride] = y[k] - f * z[k];
  free(diag); free(y); free(z); free(rhs); free(u); free(cp); free(dp);
}

/* The spline (deriv = 0) or its derivative d/ds (deriv = 1) at s (any real, periodic
 * with period n) from coefficients c[k*stride]. */
double orc_spline_eval(const double *c, int n, int stride, double s, int deriv) {
  double fl = floor(s);
  double t = s - fl;
  int k = (int)fl;
  double b[4];
  if (!deriv) {
    b[0] = (1 - t) * (1 - t) * (1 - t) / 6.0;
    b[1] = (3 * t * t * t - 6 * t * t + 4) / 6.0;
    b[2] = (-3 * t * t * t + 3 * t * t + 3 * t + 1) / 6.0;
    b[3] = t * t * t / 6.0;
  } else {
    b[0] = -(1 - t) * (1 - t) / 2.0;
    b[1] = 1.5 * t * t - 2 * t;
    b[2] = -1.5 * t * t + t + 0.5;
    b[3] = t * t / 2.0;
  }
  double r = 0;
  for (int j = 0; j < 4; j++) {
    int q = ((k - 1 + j) % n + n) % n;
    r += c[q * stride] * b[j];
  }
  return r;
}

/* Normal / tangential split, Eqs. 31-32 and Eq. 46.
 * n_k: outward unit normal of the counter-clockwise polygon at marker k, the
 * central tangent X_{k+1} - X_{k-1} turned by -90 degrees (Eq. 31 in 2D).
 * |X_s|_k = |X_{k+1} - X_{k-1}| / (2 dX) (Eq. 31's |X_r x X_s| for a curve);
 * for a rigid body it is 1 as the paper states after Eq. 31.
 * Fn_k = G_k.n_k / |X_s|_k  (the jump strength of Eq. 32),
 * Gpar_k = G_k - (G_k.n_k) n_k  (the printed "G - G.n" after Eq. 46 read as
 * the vector tangential part). */
void orc_normal_split(const orc_iface *I, const double *G, double *Fn, double *Gpar,
                      double *nrm) {
  int n = I->n;
  double *cx = NULL;
  if (I->curve > 0) {  /* spline interface: tangents X'(k) of the spline */
    cx = (double *)malloc(2 * n * sizeof(double));
    orc_spline_coeffs(I->X, n, 2, cx);
    orc_spline_coeffs(I->X + 1, n, 2, cx + 1);
  }
  for (int k = 0; k < n; k++) {
    int kp = (k + 1) % n, km = (k + n - 1) % n;
    double tx, ty, Xs;
    if (cx) {  /* X'(k) = (c_{k+1} - c_{k-1}) / 2; |X_s| = |X'(k)| / dX */
      tx = orc_spline_eval(cx, n, 2, k, 1);
      ty = orc_spline_eval(cx + 1, n, 2, k, 1);
    } else {   /* central difference of the polygon: |X_s| = |X_{k+1} - X_{k-1}| / (2 dX) */
      tx = I->X[2 * kp] - I->X[2 * km];
      ty = I->X[2 * kp + 1] - I->X[2 * km + 1];
    }
    double tl = sqrt(tx * tx + ty * ty);
    double nx = ty / tl, ny = -tx / tl;
    if (cx) Xs = I->moves ? tl / I->dX : 1.0;
    else Xs = I->moves ? tl / (2.0 * I->dX) : 1.0;
    double Gn = G[2 * k] * nx + G[2 * k + 1] * ny;
    Fn[k] = Gn / Xs;
    Gpar[2 * k] = G[2 * k] - Gn * nx;
    Gpar[2 * k + 1] = G[2 * k + 1] - Gn * ny;
    if (nrm) { nrm[2 * k] = nx; nrm[2 * k + 1] = ny; }
  }
  free(cx);
}

/* ------------------------------------------------------------ cut links ----
 * Which streamed populations carry the jump (section 3.2, Eq. 47 and the P1/P2
 * example): f_i arriving at node x gets [[f_i]] when the streaming path
 * x - e_i -> x crosses the interface.  The interface is the marker polygon and
 * the jump strength Fn is linear in the segment parameter.
 *
 * Sign (Eq. 30: [[psi]] = psi(+) - psi(-), + = exterior): a population that
 * passes from the interior (-) to the exterior (+) gains +[[f_i]], one passing
 * the other way gains -[[f_i]].  Value (Eq. 32): [[f_i]] = w_i/c_s^2 Fn.
 *
 * Predicate (reading; the paper uses a spline and gives no crossing rule):
 * marker coordinates are snapped to multiples of 2^-24 lattice units, so every
 * orientation test is exact 64-bit integer arithmetic, and degenerate contacts
 * are resolved by symbolically displacing every lattice node by (eps, eps^2),
 * eps -> 0+.  With this rule the signed number of crossings on a link equals
 * winding(x - e_i) - winding(x) of the polygon, exactly. */
#define ORC_QSCALE 16777216.0 /* 2^24 */

static int sgn64(int64_t v) { return v > 0 ? 1 : (v < 0 ? -1 : 0); }

/* orient(A, B, P + (eps, eps^2)) = cross(B - A, P - A) + dx eps^2 - dy eps */
int orc_orient_seg_node(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py) {
  int64_t dx = bx - ax, dy = by - ay;
  int64_t o = dx * (py - ay) - dy * (px - ax);
  if (o != 0) return sgn64(o);
  if (dy != 0) return -sgn64(dy);
  return sgn64(dx);
}
/* orient(P + d, P + e + d, A) with d = (eps, eps^2) = cross(e, A - P) + ey eps - ex eps^2 */
int orc_orient_link_pt(int64_t px, int64_t py, int ex, int ey, int64_t ax, int64_t ay) {
  int64_t o = (int64_t)ex * (ay - py) - (int64_t)ey * (ax - px);
  if (o != 0) return sgn64(o);
  if (ey != 0) return ey > 0 ? 1 : -1;
  return ex > 0 ? -1 : 1;
}

int64_t orc_quantize(double v) { return (int64_t)llrint(v * ORC_QSCALE); }

/* Test one lattice link (source node p, direction i) against one segment A->B
 * (quantised).  Returns 0 if it does not cross, else the sign s and the crossing
 * parameter t along A->B. */
int orc_link_crosses(int64_t ax, int64_t ay, int64_t bx, int64_t by, int px, int py,
                     int i, int *s, double *t) {
  int64_t Px = (int64_t)px * (int64_t)ORC_QSCALE, Py = (int64_t)py * (int64_t)ORC_QSCALE;
  int64_t Qx = (int64_t)(px + EX[i]) * (int64_t)ORC_QSCALE, Qy = (int64_t)(py + EY[i]) * (int64_t)ORC_QSCALE;
  int s1 = orc_orient_seg_node(ax, ay, bx, by, Px, Py);
  int s2 = orc_orient_seg_node(ax, ay, bx, by, Qx, Qy);
  if (s1 == s2) return 0;
  int s3 = orc_orient_link_pt(Px, Py, EX[i], EY[i], ax, ay);
  int s4 = orc_orient_link_pt(Px, Py, EX[i], EY[i], bx, by);
  if (s3 == s4) return 0;
  int64_t o3 = (int64_t)EX[i] * (ay - Py) - (int64_t)EY[i] * (ax - Px);
  int64_t o4 = (int64_t)EX[i] * (by - Py) - (int64_t)EY[i] * (bx - Px);
  *t = (double)o3 / ((double)o3 - (double)o4);
  if (*t < 0.0) *t = 0.0;
  if (*t > 1.0) *t = 1.0;
  *s = s1; /* source left of A->B = interior of a CCW polygon: - to +, sign +1 */
  return 1;
}

/* Enumerate every crossing of every segment.  Output records: destination cell
 * (row-major y*nx+x), direction i, coefficient s * w_i / c_s^2 * Fn(t).
 * Candidates per segment: destination nodes within one node of the segment's
 * bounding box (a crossing lies in both the segment's box and the link's unit
 * box).  Returns the number of records, or -1 if cap is exceeded. */
int orc_cut_links(const orc_cfg *c, const double *X, int n, const double *Fn,
                  int *cell, int *dir, double *coef, int cap) {
  int cnt = 0;
  for (int k = 0; k < n; k++) {
    int kp = (k + 1) % n;
    int64_t ax = orc_quantize(X[2 * k]), ay = orc_quantize(X[2 * k + 1]);
    int64_t bx = orc_quantize(X[2 * kp]), by = orc_quantize(X[2 * kp + 1]);
    double minx = fmin(X[2 * k], X[2 * kp]), maxx = fmax(X[2 * k], X[2 * kp]);
    double miny = fmin(X[2 * k + 1], X[2 * kp + 1]), maxy = fmax(X[2 * k + 1], X[2 * kp + 1]);
    int x0 = (int)floor(minx) - 1, x1 = (int)ceil(maxx) + 1;
    int y0 = (int)floor(miny) - 1, y1 = (int)ceil(maxy) + 1;
    for (int qy = y0; qy <= y1; qy++)
      for (int qx = x0; qx <= x1; qx++)
        for (int i = 1; i < 9; i++) {
          int s; double t;
          if (!orc_link_crosses(ax, ay, bx, by, qx - EX[i], qy - EY[i], i, &s, &t)) continue;
          int xd = wrap_axis(qx, c->nx, periodic_x(c)), yd = wrap_axis(qy, c->ny, periodic_y(c));
          int xs = wrap_axis(qx - EX[i], c->nx, periodic_x(c)), ys = wrap_axis(qy - EY[i], c->ny, periodic_y(c));
          if (xd < 0 || yd < 0 || xs < 0 || ys < 0) continue;
          if (cnt >= cap) return -1;
          double F = (1.0 - t) * Fn[k] + t * Fn[kp];
          cell[cnt] = yd * c->nx + xd;
          dir[cnt] = i;
          coef[cnt] = (double)s * WT[i] * INV_CS2 * F;
          cnt++;
        }
  }
  return cnt;
}

/* Cut links of the spline interface (curve = m chords per segment): the spline
 * through the markers is replaced by the polygon of its points X(k + j/m), j < m, and
 * every crossing of a chord (k, j) at chord parameter t, found as orc_cut_links finds
 * them, lies at spline parameter s = k + (j + t)/m, where Fn(s) is the periodic spline
 * through the markers' Fn_k.  Same records and return as orc_cut_links. */
int orc_cut_links_spline(const orc_cfg *c, const double *X, int n, const double *Fn, int m,
                         int *cell, int *dir, double *coef, int cap) {
  int N = n * m, cnt = 0;
  double *cx = (double *)malloc(2 * n * sizeof(double)), *cf = (double *)malloc(n * sizeof(double));
  double *P = (double *)malloc(2 * N * sizeof(double));
  orc_spline_coeffs(X, n, 2, cx);
  orc_spline_coeffs(X + 1, n, 2, cx + 1);
  orc_spline_coeffs(Fn, n, 1, cf);
  for (int k = 0; k < n; k++)
    for (int j = 0; j < m; j++) {
      double sp = k + (double)j / m;
      P[2 * (k * m + j)] = orc_spline_eval(cx, n, 2, sp, 0);
      P[2 * (k * m + j) + 1] = orc_spline_eval(cx + 1, n, 2, sp, 0);
    }
  for (int q = 0; q < N && cnt >= 0; q++) {
    int qp = (q + 1) % N;
    int64_t ax = orc_quantize(P[2 * q]), ay = orc_quantize(P[2 * q + 1]);
    int64_t bx = orc_quantize(P[2 * qp]), by = orc_quantize(P[2 * qp + 1]);
    double minx = fmin(P[2 * q], P[2 * qp]), maxx = fmax(P[2 * q], P[2 * qp]);
    double miny = fmin(P[2 * q + 1], P[2 * qp + 1]), maxy = fmax(P[2 * q + 1], P[2 * qp + 1]);
    int x0 = (int)floor(minx) - 1, x1 = (int)ceil(maxx) + 1;
    int y0 = (int)floor(miny) - 1, y1 = (int)ceil(maxy) + 1;
    for (int qy = y0; qy <= y1 && cnt >= 0; qy++)
      for (int qx = x0; qx <= x1 && cnt >= 0; qx++)
        for (int i = 1; i < 9; i++) {
          int sg; double t;
          if (!orc_link_crosses(ax, ay, bx, by, qx - EX[i], qy - EY[i], i, &sg, &t)) continue;
          int xd = wrap_axis(qx, c->nx, periodic_x(c)), yd = wrap_axis(qy, c->ny, periodic_y(c));
          int xs = wrap_axis(qx - EX[i], c->nx, periodic_x(c)), ys = wrap_axis(qy - EY[i], c->ny, periodic_y(c));
          if (xd < 0 || yd < 0 || xs < 0 || ys < 0) continue;
          if (cnt >= cap) { cnt = -1; break; }
          double F = orc_spline_eval(cf, n, 1, (q + t) / m, 0);
          cell[cnt] = yd * c->nx + xd;
          dir[cnt] = i;
          coef[cnt] = (double)sg * WT[i] * INV_CS2 * F;
          cnt++;
        }
  }
  free(cx); free(cf); free(P);
  return cnt;
}

/* Winding number of the closed polygon around node (px, py) displaced by
 * (eps, eps^2), by the crossing-parity rule on the horizontal ray to +x
 * (used only by tests as an independent check of the cut-link signs). */
int orc_winding(const double *X, int n, int px, int py) {
  int64_t Px = (int64_t)px * (int64_t)ORC_QSCALE, Py = (int64_t)py * (int64_t)ORC_QSCALE;
  int w = 0;
  for (int k = 0; k < n; k++) {
    int kp = (k + 1) % n;
    int64_t ax = orc_quantize(X[2 * k]), ay = orc_quantize(X[2 * k + 1]);
    int64_t bx = orc_quantize(X[2 * kp]), by = orc_quantize(X[2 * kp + 1]);
    /* node y + eps^2 against the vertex heights: a vertex is "above" iff ay > Py
     * (equal heights count as below, since the node sits eps^2 higher) */
    int aup = ay > Py, bup = by > Py;
    if (aup == bup) continue;
    int o = orc_orient_seg_node(ax, ay, bx, by, Px, Py);
    if (bup && o > 0) w += 1;  /* upward edge with the node on its left */
    if (!bup && o < 0) w -= 1; /* downward edge with the node on its right */
  }
  return w;
}

/* ------------------------------------------------------------- streaming ---
 * Collide-then-stream form of Eqs. 14-15 and Eq. 47: f_i(x, t+1) = f*_i(x - e_i).
 * Eq. 47 places RHS at the destination; the standard collide-at-source form is
 * taken (section 2.2.1 discretisation read as the usual lattice update).
 * Walls (ORC_BC_WALLS_Y, ORC_BC_CHANNEL): halfway bounce-back at y = -1/2 and
 * y = ny - 1/2: a population whose source lies beyond a wall is the reflected
 * post-collision population of the destination node, f_i(x) = f*_{opp(i)}(x).
 * Channel: populations whose source lies beyond x = 0 or x = nx - 1 are left as
 * the post-collision value of the node itself and are overwritten by
 * orc_channel_bc. */
static void stream(const orc_cfg *c, const double *fs, double *out) {
  int nx = c->nx, ny = c->ny, N = nx * ny;
  #pragma omp parallel for collapse(2) schedule(static)
  for (int i = 0; i < 9; i++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        int sx = x - EX[i], sy = y - EY[i];
        /* a box streams as if periodic: what reaches its boundary nodes from the far
         * side is replaced by box_bc */
        int wy = (sy < 0 || sy >= ny) && !periodic_y(c) && !is_box(c);
        int wx = (sx < 0 || sx >= nx) && !periodic_x(c) && !is_box(c);
        double v;
        if (wy) {
          v = fs[OPP[i] * N + y * nx + x];
        } else if (wx) {
          v = fs[i * N + y * nx + x];
        } else {
          sx = ((sx % nx) + nx) % nx;
          sy = ((sy % ny) + ny) % ny;
          v = fs[i * N + sy * nx + sx];
        }
        out[i * N + y * nx + x] = v;
      }
}

/* Channel inflow / outflow on the streamed state.
 * Inflow column x = 0: non-equilibrium extrapolation of Guo, Zheng & Shi (the
 * paper's boundary method for open and wall boundaries in section 4):
 *   f_i(0,y) = f_eq_i(rho(1,y), u_in(y)) + [f_i(1,y) - f_eq_i(rho(1,y), u(1,y))]
 * with the parabolic profile u_in(y) = 4 u_max (y+1/2)(ny-y-1/2)/ny^2, v = 0.
 * Outflow column x = nx-1: zero gradient on the unknown populations (e_x < 0),
 * f_i(nx-1,y) = f_i(nx-2,y). */
static void channel_bc(const orc_cfg *c, double *df) {
  int nx = c->nx, ny = c->ny, N = nx * ny;
  for (int y = 0; y < ny; y++) {
    double dfc[9], r, ux, uy, a[9], b[9];
    for (int i = 0; i < 9; i++) dfc[i] = df[i * N + y * nx + 1];
    orc_cell_macros(dfc, c->rho0, 0.0, 0.0, &r, &ux, &uy);
    double yy = y + 0.5;
    double uin = 4.0 * c->u_max * yy * (ny - yy) / ((double)ny * ny);
    orc_feq_shifted(r, c->rho0, uin, 0.0, a);  /* r is the deviation drho(1,y) */
    orc_feq_shifted(r, c->rho0, ux, uy, b);
    for (int i = 0; i < 9; i++) df[i * N + y * nx + 0] = a[i] + (dfc[i] - b[i]);
    for (int i = 0; i < 9; i++)
      if (EX[i] < 0) df[i * N + y * nx + nx - 1] = df[i * N + y * nx + nx - 2];
  }
}

/* Box boundaries of the paper's section 4 setups, non-equilibrium extrapolation
 * (Guo, Zheng & Shi): every node b on the box's edge takes
 *   f_i(b) = f_eq_i(rho_b, u_b) + [f_i(n) - f_eq_i(rho(n), u(n))]
 * from its inward neighbour n (b plus the inward normal; diagonal at a corner), with
 * ORC_BC_BOX_OUTFLOW: rho_b = rho0, u_b = u(n) (an open boundary at the reference
 * pressure, section 4.1); ORC_BC_BOX_WALL: u_b = 0, rho_b = rho(n) (no-slip walls,
 * section 4.2).  Applied to the streamed state; rho(n), u(n) from the streamed
 * populations of n (no force acts near the box's edge). */
static void box_bc(const orc_cfg *c, double *df) {
  int nx = c->nx, ny = c->ny, N = nx * ny;
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      if (x != 0 && x != nx - 1 && y != 0 && y != ny - 1) continue;
      int px = x + (x == 0) - (x == nx - 1), py = y + (y == 0) - (y == ny - 1);
      double fn[9], r, ux, uy, eb[9], en[9];
      for (int i = 0; i < 9; i++) fn[i] = df[i * N + py * nx + px];
      orc_cell_macros(fn, c->rho0, 0.0, 0.0, &r, &ux, &uy);
      orc_feq_shifted(r, c->rho0, ux, uy, en);
      if (c->bc == ORC_BC_BOX_OUTFLOW) orc_feq_shifted(0.0, c->rho0, ux, uy, eb);
      else orc_feq_shifted(r, c->rho0, 0.0, 0.0, eb);
      for (int i = 0; i < 9; i++) df[i * N + y * nx + x] = eb[i] + (fn[i] - en[i]);
    }
}

/* --------------------------------------------------------------- state ---- */
orc_state *orc_create(const orc_cfg *cfg) {
  orc_state *S = (orc_state *)calloc(1, sizeof(orc_state));
  S->c = *cfg;
  size_t N = (size_t)cfg->nx * cfg->ny;
  S->df = (double *)calloc(9 * N, sizeof(double));
  S->tmp = (double *)calloc(9 * N, sizeof(double));
  S->f = (double *)calloc(9 * N, sizeof(double));
  S->gx = (double *)calloc(N, sizeof(double));
  S->gy = (double *)calloc(N, sizeof(double));
  S->rho = (double *)calloc(N, sizeof(double));
  S->ux = (double *)calloc(N, sizeof(double));
  S->uy = (double *)calloc(N, sizeof(double));
  orc_mrt_matrix(S->M);
  orc_mrt_inverse(S->M, S->Minv);
  return S;
}

static void free_iface(orc_state *S) {
  free(S->X0);
  S->X0 = NULL;
  S->has_body = 0;
  if (!S->has_iface) return;
  free(S->I.X); free(S->I.Gp); free(S->I.UD);
  free(S->G); free(S->Fn); free(S->Gpar); free(S->U); free(S->Ustar); free(S->Gprev);
  S->has_iface = 0;
}

void orc_destroy(orc_state *S) {
  if (!S) return;
  free_iface(S);
  free(S->df); free(S->tmp); free(S->f); free(S->gx); free(S->gy);
  free(S->rho); free(S->ux); free(S->uy);
  free(S);
}

void orc_set_df(orc_state *S, const double *df) {
  memcpy(S->df, df, 9 * (size_t)S->c.nx * S->c.ny * sizeof(double));
}
void orc_get_df(const orc_state *S, double *df) {
  memcpy(df, S->df, 9 * (size_t)S->c.nx * S->c.ny * sizeof(double));
}

/* Equilibrium initial state at density rho(x), velocity u(x) (arrays may be NULL
 * for rho0 / zero). */
void orc_init_equilibrium(orc_state *S, const double *rho, const double *ux, const double *uy) {
  int N = S->c.nx * S->c.ny;
  #pragma omp parallel for schedule(static)
  for (int p = 0; p < N; p++) {
    double e[9];
    orc_feq_shifted(rho ? rho[p] - S->c.rho0 : 0.0, S->c.rho0, ux ? ux[p] : 0.0, uy ? uy[p] : 0.0, e);
    for (int i = 0; i < 9; i++) S->df[i * N + p] = e[i];
  }
}

int orc_set_interface(orc_state *S, const double *X, int n, int model, int moves,
                      double kappa, double dX, double l0, double eta, int mdf_iters,
                      double mdf_tol, const double *Gp, const double *UD) {
  free_iface(S);
  if (n <= 0) return 0;
  orc_iface *I = &S->I;
  I->n = n; I->model = model; I->moves = moves; I->kappa = kappa; I->dX = dX; I->l0 = l0;
  I->eta = eta; I->mdf_iters = mdf_iters; I->mdf_tol = mdf_tol;
  I->X = (double *)malloc(2 * n * sizeof(double));
  I->Gp = (double *)calloc(2 * n, sizeof(double));
  I->UD = (double *)calloc(2 * n, sizeof(double));
  memcpy(I->X, X, 2 * n * sizeof(double));
  if (Gp) memcpy(I->Gp, Gp, 2 * n * sizeof(double));
  if (UD) memcpy(I->UD, UD, 2 * n * sizeof(double));
  S->G = (double *)calloc(2 * n, sizeof(double));
  S->Fn = (double *)calloc(n, sizeof(double));
  S->Gpar = (double *)calloc(2 * n, sizeof(double));
  S->U = (double *)calloc(2 * n, sizeof(double));
  S->Ustar = (double *)calloc(2 * n, sizeof(double));
  S->Gprev = (double *)calloc(2 * n, sizeof(double));
  S->has_iface = 1;
  return 0;
}

/* The forcing of the step for a Lagrangian force G on the markers X (section 3.2):
 * f = dfs plus, in II-LBM, the jump of the normal part on every cut link of the polygon
 * (Eq. 47 with Eq. 32), and g = body + the spread of the tangential part (Eq. 46); in
 * IB-LBM f = dfs and g = body + the spread of the whole G (Eq. 17).  Fn and Gpar
 * receive the split of Eqs. 31-32 / 46.  Returns the number of cut-link crossings, or
 * -1 if the record capacity is exceeded. */
static int apply_forcing(const orc_cfg *c, const orc_iface *I, const double *G,
                         const double *dfs, double *f, double *gx, double *gy, double *Fn,
                         double *Gpar) {
  int N = c->nx * c->ny, n = I->n, m = 0;
  memcpy(f, dfs, 9 * (size_t)N * sizeof(double));
  for (int p = 0; p < N; p++) { gx[p] = c->body_x; gy[p] = c->body_y; }
  orc_normal_split(I, G, Fn, Gpar, NULL);
  double *P = (double *)malloc(2 * n * sizeof(double));
  if (c->jump) {
    int cap = 64 * n * (I->curve > 0 ? I->curve : 1) + 64;
    int *cell = (int *)malloc(cap * sizeof(int)), *dir = (int *)malloc(cap * sizeof(int));
    double *coef = (double *)malloc(cap * sizeof(double));
    m = I->curve > 0 ? orc_cut_links_spline(c, I->X, n, Fn, I->curve, cell, dir, coef, cap)
                     : orc_cut_links(c, I->X, n, Fn, cell, dir, coef, cap);
    for (int r = 0; r < m; r++) f[dir[r] * N + cell[r]] += coef[r];
    free(cell); free(dir); free(coef);
    for (int k = 0; k < 2 * n; k++) P[k] = Gpar[k] * I->dX;
  } else {
    for (int k = 0; k < 2 * n; k++) P[k] = G[k] * I->dX;
  }
  if (m >= 0) orc_spread(c, I->X, n, P, gx, gy);
  free(P);
  return m;
}

/* Direct forcing with repeated correction, Eq. 18 (reading: multi-direct forcing,
 * Guo half-force velocity).  u* = (sum e df + body/2)/rho is the velocity without the
 * body's forcing, and U* = interp(u*) is kept.  A pass applies the step's forcing of
 * the current G (apply_forcing: in II-LBM the normal part through the jump, the
 * tangential part spread), interpolates the velocity the collision will then use
 * (Eq. 24 from f and g, Eq. 20), and adds eta (U^D - U) to G; the iteration stops
 * after mdf_iters passes or when max_k |U^D - U_k| < mdf_tol.  The passes thus see G
 * through the operator the step applies it with.  (Spreading the whole G in the passes
 * and then moving its normal part into the jump applies the normal part through an
 * operator the iteration never saw: the jump moves the velocity at the markers about
 * twice as much as the half-force spread, and the channel at Re 100 diverges.)  The
 * pass count and final residual are kept.  The iteration starts from Gp, or with
 * ws_previous from the force the previous call ended with. */
static int direct_forcing(orc_state *S, const double *dfs) {
  const orc_cfg *c = &S->c;
  orc_iface *I = &S->I;
  int N = c->nx * c->ny, n = I->n;
  double *us_x = (double *)calloc(N, sizeof(double)), *us_y = (double *)calloc(N, sizeof(double));
  double *r = (double *)calloc(N, sizeof(double)); /* drho */
  double *f = (double *)malloc(9 * (size_t)N * sizeof(double));
  double *gx = (double *)calloc(N, sizeof(double)), *gy = (double *)calloc(N, sizeof(double));
  double *vx = (double *)calloc(N, sizeof(double)), *vy = (double *)calloc(N, sizeof(double));
  double *Fn = (double *)calloc(n, sizeof(double)), *Gpar = (double *)calloc(2 * n, sizeof(double));
  #pragma omp parallel for schedule(static)
  for (int p = 0; p < N; p++) {
    double dfc[9];
    for (int i = 0; i < 9; i++) dfc[i] = dfs[i * N + p];
    orc_cell_macros(dfc, c->rho0, c->body_x, c->body_y, &r[p], &us_x[p], &us_y[p]);
  }
  orc_interp(c, I->X, n, us_x, us_y, S->Ustar);
  const double *G0 = S->ws_previous ? S->Gprev : I->Gp;
  for (int k = 0; k < 2 * n; k++) S->G[k] = G0[k]; /* warm start (0 = plain) */
  int it = 0, rc = 0;
  double res = 0;
  for (it = 0; it < I->mdf_iters; it++) {
    if (apply_forcing(c, I, S->G, dfs, f, gx, gy, Fn, Gpar) < 0) { rc = -1; break; }
    #pragma omp parallel for schedule(static)
    for (int p = 0; p < N; p++) {
      double dfc[9], d;
      for (int i = 0; i < 9; i++) dfc[i] = f[i * N + p];
      orc_cell_macros(dfc, c->rho0, gx[p], gy[p], &d, &vx[p], &vy[p]);
    }
    orc_interp(c, I->X, n, vx, vy, S->U);
    res = 0;
    for (int k = 0; k < 2 * n; k++) res = fmax(res, fabs(I->UD[k] - S->U[k]));
    if (I->mdf_tol > 0 && res < I->mdf_tol) break;
    for (int k = 0; k < 2 * n; k++) S->G[k] += I->eta * (I->UD[k] - S->U[k]);
  }
  S->mdf_last_iters = it;
  S->mdf_last_res = res;
  memcpy(S->Gprev, S->G, 2 * n * sizeof(double));
  free(us_x); free(us_y); free(r); free(f); free(gx); free(gy); free(vx); free(vy);
  free(Fn); free(Gpar);
  return rc;
}

/* One II-LBM time step, t -> t+1 (section 3.2, Eq. 47, with Eqs. 17-24).
 * orc_prepare does items 1-4 (a pure function of the state and the markers),
 * orc_advance items 5-6.
 *  1. Lagrangian force G_k from X^t (Eq. 19, its rest-length variant, a
 *     prescribed force, or direct forcing Eq. 18).
 *  2. Split: Fn_k (jump strength, Eq. 32), Gpar_k (Eq. 46).
 *  3. II-LBM: f = df + [[f]] on every cut link of the polygon X^t (Eq. 47 adds
 *     the jump at the new time level, evaluated on the interface of that level);
 *     g = spread(Gpar dX) + body (Eq. 46).  IB-LBM: f = df, g = spread(G dX) + body.
 *  4. rho, u from f and g (Eqs. 11, 24); U_k = interp(u) (Eq. 20).
 *  5. Collide every cell (Eqs. 14/15 with 21/22), stream (Eq. 47), boundaries.
 *  6. X^{t+1} = X^t + U_k for a membrane (Eq. 20). */
int orc_prepare(orc_state *S) {
  const orc_cfg *c = &S->c;
  int N = c->nx * c->ny;
  S->ncut = 0;
  if (S->has_iface) {
    orc_iface *I = &S->I;
    int n = I->n;
    if (I->model == ORC_SPRING || I->model == ORC_SPRING_REST) orc_spring_forces(I, S->G);
    else if (I->model == ORC_PRESCRIBED) memcpy(S->G, I->Gp, 2 * n * sizeof(double));
    else if (direct_forcing(S, S->df)) return -1;
    int m = apply_forcing(c, I, S->G, S->df, S->f, S->gx, S->gy, S->Fn, S->Gpar);
    if (m < 0) return -1;
    S->ncut = m;
  } else {
    memcpy(S->f, S->df, 9 * (size_t)N * sizeof(double));
    for (int p = 0; p < N; p++) { S->gx[p] = c->body_x; S->gy[p] = c->body_y; }
  }
  #pragma omp parallel for schedule(static)
  for (int p = 0; p < N; p++) {
    double dfc[9];
    for (int i = 0; i < 9; i++) dfc[i] = S->f[i * N + p];
    /* the velocity the collision uses: (sum e f + g/2) / rho (Guo), sum e f / rho (simple) */
    double hx = c->force == ORC_FORCE_SIMPLE ? 0.0 : S->gx[p];
    double hy = c->force == ORC_FORCE_SIMPLE ? 0.0 : S->gy[p];
    orc_cell_macros(dfc, c->rho0, hx, hy, &S->rho[p], &S->ux[p], &S->uy[p]);
  }
  if (S->has_iface) orc_interp(c, S->I.X, S->I.n, S->ux, S->uy, S->U);
  return 0;
}

void orc_advance(orc_state *S) {
  const orc_cfg *c = &S->c;
  int N = c->nx * c->ny;
  #pragma omp parallel for schedule(static)
  for (int p = 0; p < N; p++) {
    double dfc[9], out[9];
    for (int i = 0; i < 9; i++) dfc[i] = S->f[i * N + p];
    orc_collide_cell(c, S->M, S->Minv, dfc, S->gx[p], S->gy[p], out);
    for (int i = 0; i < 9; i++) S->tmp[i * N + p] = out[i];
  }
  stream(c, S->tmp, S->df);
  if (c->bc == ORC_BC_CHANNEL) channel_bc(c, S->df);
  if (is_box(c)) box_bc(c, S->df);
  if (S->has_iface && S->I.moves)
    for (int k = 0; k < 2 * S->I.n; k++) S->I.X[k] += S->U[k];
  S->step++;
}

/* ---------------------------------------------------------- rigid body -------
 * A rigid body carrying a directly forced interface (section 2.3).  Its markers are
 * the body's reference polygon X0 (offsets from the centre Xc0, at angle 0) placed at
 * the centre Xc and angle theta; the desired velocity of marker k is the body's,
 * U^D_k = U_c + W x (X_k - X_c).  After a step whose force iteration gave G:
 *   F_ext = -sum_k G_k dX + rho_f V_s (U_c(t) - U_c(t-1))                 (Eq. 25)
 *   T_ext = -sum_k (X_k - X_c) x G_k dX + (rho_f/rho_s) I_s (W(t) - W(t-1))  (Eq. 26)
 * and, for a free body, on each free degree of freedom with its spring k and damper c
 * (the paper's 1-DOF oscillator of section 4.5, Eq. 54, in dimensional form):
 *   m a(t+1) = F_ext - k (X_c - X_c0) - c U_c,  I_s w(t+1) = T_ext - k theta - c W
 *                                                                         (Eq. 27)
 *   U_c(t+1) = U_c(t) + a(t+1),  W(t+1) = W(t) + w(t+1)                   (Eq. 28)
 *   X_c(t+1) = X_c(t) + U_c(t) + (a(t) + a(t+1))/2, the same for theta     (Eq. 29)
 * A prescribed body follows section 4.4's harmonic translation in x:
 *   X_c(t) = X_c0 - A sin(U_max t / A),  U_c(t) = -U_max cos(U_max t / A). */
int orc_set_body(orc_state *S, int mode, int dof, double A, double umax, double m, double I,
                 double Vs, const double *k, const double *c) {
  if (!S->has_iface || S->I.model != ORC_DIRECT) return -1;
  int n = S->I.n;
  free(S->X0);
  S->X0 = (double *)malloc(2 * n * sizeof(double));
  double cx = 0, cy = 0;
  for (int q = 0; q < n; q++) { cx += S->I.X[2 * q]; cy += S->I.X[2 * q + 1]; }
  cx /= n; cy /= n;
  for (int q = 0; q < n; q++) {
    S->X0[2 * q] = S->I.X[2 * q] - cx;
    S->X0[2 * q + 1] = S->I.X[2 * q + 1] - cy;
  }
  S->has_body = 1;
  S->body_mode = mode; S->body_dof = dof; S->body_A = A; S->body_umax = umax;
  S->body_m = m; S->body_I = I; S->body_Vs = Vs;
  for (int d = 0; d < 3; d++) { S->body_k[d] = k ? k[d] : 0; S->body_c[d] = c ? c[d] : 0; }
  S->Xc0[0] = S->Xc[0] = cx; S->Xc0[1] = S->Xc[1] = cy;
  S->Uc[0] = S->Uc[1] = S->Ucp[0] = S->Ucp[1] = S->ac[0] = S->ac[1] = 0;
  S->th = S->Wb = S->Wbp = S->wb = 0;
  S->Fext[0] = S->Fext[1] = S->Fext[2] = 0;
  if (mode == ORC_BODY_PRESCRIBED_X) S->Uc[0] = S->Ucp[0] = -umax;  /* U_c(0) */
  /* the markers and their desired velocity at t = 0 */
  for (int q = 0; q < n; q++) {
    double rx = S->I.X[2 * q] - S->Xc[0], ry = S->I.X[2 * q + 1] - S->Xc[1];
    S->I.UD[2 * q] = S->Uc[0] - S->Wb * ry;
    S->I.UD[2 * q + 1] = S->Uc[1] + S->Wb * rx;
  }
  return 0;
}

/* The body's update after a step (the force G of that step's iteration), then its
 * markers and desired velocities at the new time level. */
static void body_update(orc_state *S) {
  orc_iface *I = &S->I;
  int n = I->n;
  double Fx = 0, Fy = 0, T = 0;
  for (int q = 0; q < n; q++) {
    double rx = I->X[2 * q] - S->Xc[0], ry = I->X[2 * q + 1] - S->Xc[1];
    Fx -= S->G[2 * q] * I->dX;
    Fy -= S->G[2 * q + 1] * I->dX;
    T -= (rx * S->G[2 * q + 1] - ry * S->G[2 * q]) * I->dX;
  }
  double rho_f = S->c.rho0;
  Fx += rho_f * S->body_Vs * (S->Uc[0] - S->Ucp[0]);
  Fy += rho_f * S->body_Vs * (S->Uc[1] - S->Ucp[1]);
  T += rho_f * S->body_Vs / S->body_m * S->body_I * (S->Wb - S->Wbp);  /* rho_f/rho_s = rho_f V_s / m */
  S->Fext[0] = Fx; S->Fext[1] = Fy; S->Fext[2] = T;
  double t1 = (double)(S->step);  /* the new time level */
  S->Ucp[0] = S->Uc[0]; S->Ucp[1] = S->Uc[1]; S->Wbp = S->Wb;
  if (S->body_mode == ORC_BODY_PRESCRIBED_X) {
    double A = S->body_A, um = S->body_umax;
    S->Xc[0] = S->Xc0[0] - A * sin(um * t1 / A);
    S->Uc[0] = -um * cos(um * t1 / A);
  } else {
    double F[3] = {Fx, Fy, T};
    double inert[3] = {S->body_m, S->body_m, S->body_I};
    double *pos[3] = {&S->Xc[0], &S->Xc[1], &S->th};
    double *vel[3] = {&S->Uc[0], &S->Uc[1], &S->Wb};
    double *acc[3] = {&S->ac[0], &S->ac[1], &S->wb};
    double org[3] = {S->Xc0[0], S->Xc0[1], 0.0};
    for (int d = 0; d < 3; d++) {
      if (!(S->body_dof & (1 << d))) continue;
      double a1 = (F[d] - S->body_k[d] * (*pos[d] - org[d]) - S->body_c[d] * (*vel[d])) / inert[d];
      double v0 = *vel[d], a0 = *acc[d];
      *vel[d] = v0 + a1;
      *pos[d] = *pos[d] + v0 + 0.5 * (a0 + a1);
      *acc[d] = a1;
    }
  }
  double cth = cos(S->th), sth = sin(S->th);
  for (int q = 0; q < n; q++) {
    double ox = S->X0[2 * q], oy = S->X0[2 * q + 1];
    I->X[2 * q] = S->Xc[0] + cth * ox - sth * oy;
    I->X[2 * q + 1] = S->Xc[1] + sth * ox + cth * oy;
    double rx = I->X[2 * q] - S->Xc[0], ry = I->X[2 * q + 1] - S->Xc[1];
    I->UD[2 * q] = S->Uc[0] - S->Wb * ry;
    I->UD[2 * q + 1] = S->Uc[1] + S->Wb * rx;
  }
}

/* Body state: X_c, Y_c, theta, U_x, U_y, W, F_x, F_y, T (the last F_ext, T_ext). */
void orc_get_body(const orc_state *S, double *out) {
  double v[9] = {S->Xc[0], S->Xc[1], S->th, S->Uc[0], S->Uc[1], S->Wb,
                 S->Fext[0], S->Fext[1], S->Fext[2]};
  memcpy(out, v, sizeof v);
}

int orc_step(orc_state *S) {
  if (orc_prepare(S)) return -1;
  orc_advance(S);
  if (S->has_body) body_update(S);
  return 0;
}

int orc_cut_link_count(const orc_state *S) { return S->ncut; }

int orc_run(orc_state *S, int nsteps) {
  for (int s = 0; s < nsteps; s++)
    if (orc_step(S)) return -1;
  return 0;
}

/* Macroscopic fields of the most recent step's collision (drho = rho - rho0 and
 * u of Eq. 24 at time t, the velocity the markers moved with). */
void orc_get_step_macros(const orc_state *S, double *rho, double *ux, double *uy) {
  size_t N = (size_t)S->c.nx * S->c.ny;
  if (rho) memcpy(rho, S->rho, N * sizeof(double));
  if (ux) memcpy(ux, S->ux, N * sizeof(double));
  if (uy) memcpy(uy, S->uy, N * sizeof(double));
}

void orc_get_markers(const orc_state *S, double *X, double *G, double *U, double *Fn) {
  if (!S->has_iface) return;
  int n = S->I.n;
  if (X) memcpy(X, S->I.X, 2 * n * sizeof(double));
  if (G) memcpy(G, S->G, 2 * n * sizeof(double));
  if (U) memcpy(U, S->U, 2 * n * sizeof(double));
  if (Fn) memcpy(Fn, S->Fn, n * sizeof(double));
}

/* Interface representation for the jump (orc_iface.curve) of the current interface. */
void orc_set_curve(orc_state *S, int curve) {
  if (S->has_iface) S->I.curve = curve;
}

int orc_mdf_iters(const orc_state *S) { return S->mdf_last_iters; }
void orc_set_ws_previous(orc_state *S, int on) { S->ws_previous = on; }
void orc_get_ustar(const orc_state *S, double *out) {
  if (S->has_iface) memcpy(out, S->Ustar, 2 * S->I.n * sizeof(double));
}
double orc_mdf_residual(const orc_state *S) { return S->mdf_last_res; }

/* Enclosed area of the marker polygon (shoelace formula); the area-loss metrics
 * of Eqs. 49-50 are differences of this quantity. */
double orc_polygon_area(const double *X, int n) {
  double a = 0;
  for (int k = 0; k < n; k++) {
    int kp = (k + 1) % n;
    a += X[2 * k] * X[2 * kp + 1] - X[2 * kp] * X[2 * k + 1];
  }
  return 0.5 * a;
}

/* Array-argument entry points of the two force routines (for tests). */
void orc_spring_forces_arr(const double *X, int n, int model, double kappa, double dX,
                           double l0, double *G) {
  orc_iface I;
  memset(&I, 0, sizeof I);
  I.n = n; I.model = model; I.kappa = kappa; I.dX = dX; I.l0 = l0; I.X = (double *)X;
  orc_spring_forces(&I, G);
}
void orc_normal_split_arr(const double *X, int n, int moves, double dX, const double *G,
                          double *Fn, double *Gpar, double *nrm, int curve) {
  orc_iface I;
  memset(&I, 0, sizeof I);
  I.n = n; I.moves = moves; I.dX = dX; I.X = (double *)X; I.curve = curve;
  orc_normal_split(&I, G, Fn, Gpar, nrm);
}
