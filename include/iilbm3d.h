/*
 * iilbm3d.h -- C ABI of the three-dimensional immersed interface-lattice Boltzmann
 * method (II-LBM) on the D3Q19 lattice (Qin, Kolahdouz & Griffith, arXiv 2003.12186:
 * the D3Q19 velocity set and weights of sections 2.1 and 2.2.1, its MRT rates of section
 * 2.2.1, and the jump conditions of section 3.1, derived there in three dimensions).
 *
 * Same conventions as iilbm.h: plain pointers and sizes, status codes IILBM_*, and
 * FP64 arrays that may be host or device memory (the library detects which; copies are
 * taken, the caller keeps ownership).  Every call runs on the lattice's CUDA stream and
 * fails loudly (IILBM_ERR_NO_DEVICE) without a GPU.  The box is periodic on every axis.
 *
 * The immersed interface is a closed triangulated surface: n vertices X[n][3] (the
 * Lagrangian markers) and m triangles tri[m][3] of vertex indices, each counter-clockwise
 * seen from outside so that (B - A) x (C - A) points outward.
 *
 * Layout of populations exchanged through the ABI: df[19][nz][ny][nx] FP64, the shifted
 * deviations f_i - w_i rho0, in the velocity order 0 rest; 1..6 = +x, -x, +y, -y, +z, -z;
 * 7..18 = (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
 * (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1) (opposite directions pair as (1,2), (3,4), ...).
 */
#ifndef IILBM3D_H
#define IILBM3D_H

#include <stdint.h>

#include "iilbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct iilbm3d_lattice *iilbm3d_t;

typedef struct {
  int32_t nx, ny, nz;   /* lattice nodes, each 4 <= n <= 2048; nx * ny * nz < 2^31 */
  int32_t collision;    /* IILBM_SRT or IILBM_MRT (d'Humieres D3Q19 basis, section 2.2.1) */
  int32_t storage;      /* IILBM_F64 / F32 / F16 / BF16: the populations' storage; the
                           arithmetic is FP64 for F64 and FP32 for the others */
  int32_t jump;         /* 1: II-LBM (the normal force through the jump of Eq. 32 on
                           every cut link, the tangential part spread); 0: IB-LBM */
  int32_t force;        /* IILBM_FORCE_GUO (Eqs. 21-22) or IILBM_FORCE_SIMPLE (Eq. 16) */
  int32_t storage_scale_log2; /* F16 / BF16: stored value = df * 2^k (exact), |k| <= 24;
                           0 for F32 / F64 */
  double tau;           /* relaxation time lambda, nu = (lambda - 1/2) / 3; > 0.5 */
  double s[19];         /* MRT rates in the d'Humieres moment order (rho, e, eps, j_x, q_x,
                           j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz,
                           m_x, m_y, m_z); the rates of the conserved moments are not used */
  double rho0;          /* reference density of the shifted storage */
  double body[3];       /* uniform body force density added to g */
  void *stream;         /* cudaStream_t to run on; NULL: the library creates one */
} iilbm3d_config;

/* Lagrangian force models of a surface:
 *   IILBM3D_PRESCRIBED  G [n][3] given per vertex (force per unit reference area);
 *   IILBM3D_TENSION     surface tension gamma: G_k = -gamma (d Area / d X_k) / Aref_k,
 *                       the three-dimensional counterpart of the membrane force of Eq. 19.
 * Aref_k, the reference area of vertex k (a third of its triangles' areas), is taken
 * from the surface as installed. */
enum { IILBM3D_PRESCRIBED = 0, IILBM3D_TENSION = 1 };

typedef struct {
  int32_t model;        /* IILBM3D_PRESCRIBED or IILBM3D_TENSION */
  int32_t moves;        /* 1: the vertices move with the fluid, X += U (Eq. 20) */
  double gamma;         /* IILBM3D_TENSION: surface tension */
} iilbm3d_surface_params;

/* Create a D3Q19 lattice at rest (df = 0); allocates all device memory of the lattice.
 * Errors: INVALID_ARG, OOM, CUDA, NO_DEVICE. */
int iilbm3d_create(iilbm3d_t *out, const iilbm3d_config *cfg);

/* Release the handle and its device memory (synchronises its stream). */
int iilbm3d_destroy(iilbm3d_t h);

/* Install (replace) the surface: X[n][3] vertices, tri[m][3] triangles (int32), G[n][3]
 * the prescribed force (PRESCRIBED; else may be NULL).  Every triangle must be
 * non-degenerate with edges shorter than 8 lattice units, every vertex within
 * |coordinate| < 4096.  n = 0 removes the surface.  Section 3.1 (Eq. 32 in three
 * dimensions, n and |X_r x X_s| from the triangulation).
 * Errors: INVALID_ARG, INTERFACE, OOM, CUDA. */
int iilbm3d_set_surface(iilbm3d_t h, const double *X, int32_t n, const int32_t *tri, int32_t m,
                        const iilbm3d_surface_params *p, const double *G);

/* Equilibrium (Eq. 23 with the D3Q19 weights) of rho0 + drho(x) and u(x), each
 * [nz][ny][nx] FP64 (NULL: 0). */
int iilbm3d_init_equilibrium(iilbm3d_t h, const double *drho, const double *ux, const double *uy,
                             const double *uz);

/* Set / read the stored state: df[19][nz][ny][nx] FP64, the streamed populations without
 * the jump of the current surface (converted to / from the storage precision). */
int iilbm3d_set_populations(iilbm3d_t h, const double *df);
int iilbm3d_get_populations(iilbm3d_t h, double *df);

/* Advance n >= 0 steps of section 3.2 in three dimensions: surface geometry and force,
 * normal split, the jump on every cut link of the triangulation (Eq. 47), tangential
 * spreading, the fused stream-collide, interpolation (Eq. 20) and the vertex update.
 * Asynchronous; replayed from CUDA graphs of two steps.  Inside each step the forced
 * tiles and the interpolation run on a second stream the library owns, forked from the
 * lattice's stream and joined back to it, so work queued on the lattice's stream after
 * the call sees the finished step. */
int iilbm3d_step(iilbm3d_t h, int32_t n);

/* drho and u (Eq. 24) the next collision will use, from the populations plus the current
 * surface's jump and force; each [nz][ny][nx] FP64, host or device, any may be NULL.
 * Synchronises. */
int iilbm3d_get_macros(iilbm3d_t h, double *drho, double *ux, double *uy, double *uz);

/* Vertices: X, the Lagrangian force G and velocity U ([n][3] each) and Fn ([n]) of the
 * most recent step.  Synchronises. */
int iilbm3d_get_markers(iilbm3d_t h, double *X, double *G, double *U, double *Fn);

/* The jump of the current state's surface: J[i-1][nz][ny][nx] (i = 1..18) FP64, the sum
 * of s w_i / c_s^2 Fn(crossing) over the crossings of the link x - e_i -> x. Synchronises. */
int iilbm3d_get_jump(iilbm3d_t h, double *J);

/* Cut-link crossings of the most recent step's surface. */
int iilbm3d_get_cut_link_count(iilbm3d_t h, int32_t *count);

/* Kernel timing (diagnostic): enable = 1 records a CUDA event pair around every
 * stream-collide launch and counts the library's kernels; get_timing synchronises and
 * returns the summed stream-collide time (ms), its launches and the kernels launched. */
int iilbm3d_set_timing(iilbm3d_t h, int32_t enable);
int iilbm3d_get_timing(iilbm3d_t h, double *stream_collide_ms, int32_t *launches,
                       int64_t *kernels);

/* Wait for the lattice's work; returns the latched device status (NONFINITE, INTERFACE). */
int iilbm3d_synchronize(iilbm3d_t h);

#ifdef __cplusplus
}
#endif

#endif
