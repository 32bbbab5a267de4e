// interface.cu -- the Lagrangian side of the II-LBM step on sm_103a (FP64 geometry):
//   * marker forces (Eq. 19 spring, a rest-length spring, a prescribed force) and
//     the normal / tangential split (Eqs. 31-32, 46);
//   * the cut-link kernel: one warp per polygon segment enumerates the lattice links
//     x - e_i -> x that cross it (exact 64-bit integer orientation tests on marker
//     coordinates snapped to 2^-24) and adds the jump [[f_i]] = +-w_i/c_s^2 Fn of
//     Eq. 32 to the jump field of the destination node (Eq. 47);
//   * spreading of the tangential force with Peskin's four-point kernel (Eq. 46),
//     16 threads per marker, into the force field.
// Both fields are dense [.][ny][pitch] arrays that only flagged tiles touch; the
// flagged tiles are listed for the forced stream-collide, which consumes and
// re-zeroes them.
#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

__device__ inline int tile_of(const Geom &g, int x, int y) {
  return (y / TILE_Y) * g.ntx + x / TILE_X;
}

__device__ inline double phi4i(double r) {
  const double a = fabs(r);
  if (a < 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
  if (a < 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
  return 0.0;
}

// ------------------------------------------------------------ marker forces
// One thread per marker.  Writes G_k, Fn_k = G_k.n_k/|X_s|_k, the point force to
// spread P_k = dX * (Gpar_k in II-LBM, G_k in IB-LBM), and the normal.
__global__ void k_marker_forces(const double *__restrict__ X, const double *__restrict__ aux,
                                int n, iilbm_interface_params ip, int jump, Geom geo,
                                double *G, double *Fn, double *P, double *nrm, int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int kp = k + 1 == n ? 0 : k + 1, km = k == 0 ? n - 1 : k - 1;
  const double x = X[2 * k], y = X[2 * k + 1];
  const double xp = X[2 * kp], yp = X[2 * kp + 1], xm = X[2 * km], ym = X[2 * km + 1];
  // validity: finite, inside the representable / valid region, short segments
  bool bad = !(isfinite(x) && isfinite(y)) || fabs(x) > MAX_COORD || fabs(y) > MAX_COORD;
  const double sgx = xp - x, sgy = yp - y;
  bad = bad || !(sgx * sgx + sgy * sgy < MAX_SEGMENT * MAX_SEGMENT);
  if (geo.bc != IILBM_BC_PERIODIC) bad = bad || y < 3.0 || y > geo.ny - 4.0;
  if (geo.bc == IILBM_BC_CHANNEL) bad = bad || x < 3.0 || x > geo.nx - 4.0;
  if (bad) atomicOr(status, ST_INTERFACE);
  double gx, gy;
  if (ip.model == IILBM_SPRING) {
    const double c = ip.stiffness / (ip.dX * ip.dX);
    gx = c * ((xp - x) - (x - xm));
    gy = c * ((yp - y) - (y - ym));
  } else if (ip.model == IILBM_SPRING_REST) {
    const double ax = xp - x, ay = yp - y, bx = x - xm, by = y - ym;
    const double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
    const double Ta = ip.stiffness * (la / ip.rest_length - 1.0);
    const double Tb = ip.stiffness * (lb / ip.rest_length - 1.0);
    gx = (Ta * (ax / la) - Tb * (bx / lb)) / ip.dX;
    gy = (Ta * (ay / la) - Tb * (by / lb)) / ip.dX;
  } else {  // prescribed
    gx = aux[2 * k];
    gy = aux[2 * k + 1];
  }
  const double tx = xp - xm, ty = yp - ym;
  const double tl = sqrt(tx * tx + ty * ty);
  const double nx = ty / tl, ny = -tx / tl;  // outward for a CCW polygon
  const double xs = ip.moves ? tl / (2.0 * ip.dX) : 1.0;
  const double gn = gx * nx + gy * ny;
  G[2 * k] = gx;
  G[2 * k + 1] = gy;
  Fn[k] = gn / xs;
  nrm[2 * k] = nx;
  nrm[2 * k + 1] = ny;
  if (jump) {
    P[2 * k] = (gx - gn * nx) * ip.dX;
    P[2 * k + 1] = (gy - gn * ny) * ip.dX;
  } else {
    P[2 * k] = gx * ip.dX;
    P[2 * k + 1] = gy * ip.dX;
  }
}

// --------------------------------------------------------------- cut links
// Orientation of (A, B, node) with the node displaced by (eps, eps^2), eps -> 0+.
__device__ inline int orient_seg_node(long long ax, long long ay, long long bx, long long by,
                                      long long px, long long py) {
  const long long dx = bx - ax, dy = by - ay;
  const long long o = dx * (py - ay) - dy * (px - ax);
  if (o != 0) return o > 0 ? 1 : -1;
  if (dy != 0) return dy > 0 ? -1 : 1;
  return dx > 0 ? 1 : -1;
}
// Orientation of (node, node + e, A) with both nodes displaced by (eps, eps^2).
__device__ inline int orient_link_pt(long long px, long long py, int ex, int ey, long long ax,
                                     long long ay, long long &raw) {
  raw = (long long)ex * (ay - py) - (long long)ey * (ax - px);
  if (raw != 0) return raw > 0 ? 1 : -1;
  if (ey != 0) return ey > 0 ? 1 : -1;
  return ex > 0 ? -1 : 1;
}

template <typename T>
__global__ void k_cut_links(const double *__restrict__ X, const double *__restrict__ Fn, int n,
                            Geom geo, T *Jf, uint8_t *flags, int *ncut) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int k = warp, kp = k + 1 == n ? 0 : k + 1;
  const double Ax = X[2 * k], Ay = X[2 * k + 1], Bx = X[2 * kp], By = X[2 * kp + 1];
  if (!(fabs(Ax) <= MAX_COORD && fabs(Ay) <= MAX_COORD && fabs(Bx) <= MAX_COORD &&
        fabs(By) <= MAX_COORD))
    return;
  if (!(fabs(Bx - Ax) < MAX_SEGMENT && fabs(By - Ay) < MAX_SEGMENT)) return;
  const long long ax = __double2ll_rn(Ax * QSCALE), ay = __double2ll_rn(Ay * QSCALE);
  const long long bx = __double2ll_rn(Bx * QSCALE), by = __double2ll_rn(By * QSCALE);
  const int x0 = (int)floor(fmin(Ax, Bx)) - 1, x1 = (int)ceil(fmax(Ax, Bx)) + 1;
  const int y0 = (int)floor(fmin(Ay, By)) - 1, y1 = (int)ceil(fmax(Ay, By)) + 1;
  const int W = x1 - x0 + 1, H = y1 - y0 + 1;
  const int ncand = W * H * 8;
  const double FnA = Fn[k], FnB = Fn[kp];
  const long long Q = (long long)QSCALE;
  int found = 0;
  for (int c = lane; c < ncand; c += 32) {
    const int i = 1 + c % 8;
    const int cell = c / 8;
    const int qx = x0 + cell % W, qy = y0 + cell / W;  // destination node
    const int ex = cx(i), ey = cy(i);
    const long long Px = (long long)(qx - ex) * Q, Py = (long long)(qy - ey) * Q;
    const int s1 = orient_seg_node(ax, ay, bx, by, Px, Py);
    const int s2 = orient_seg_node(ax, ay, bx, by, (long long)qx * Q, (long long)qy * Q);
    if (s1 == s2) continue;
    long long o3, o4;
    const int s3 = orient_link_pt(Px, Py, ex, ey, ax, ay, o3);
    const int s4 = orient_link_pt(Px, Py, ex, ey, bx, by, o4);
    if (s3 == s4) continue;
    double t = (double)o3 / ((double)o3 - (double)o4);
    t = fmin(fmax(t, 0.0), 1.0);
    // destination and source inside the lattice (periodic axes wrap)
    int xd = qx, yd = qy, xs = qx - ex, ys = qy - ey;
    if (geo.bc == IILBM_BC_CHANNEL) {
      if (xd < 0 || xd >= geo.nx || xs < 0 || xs >= geo.nx) continue;
    } else {
      xd = wrap(xd, geo.nx);
    }
    if (geo.bc == IILBM_BC_PERIODIC) {
      yd = wrap(yd, geo.ny);
    } else if (yd < 0 || yd >= geo.ny || ys < 0 || ys >= geo.ny) {
      continue;
    }
    const double F = (1.0 - t) * FnA + t * FnB;
    const double coef = (double)s1 * 3.0 * wt<double>(i) * F;  // w_i / c_s^2 Fn
    atomicAdd(&Jf[(long long)(i - 1) * geo.plane + (long long)yd * geo.pitch + xd], (T)coef);
    flags[tile_of(geo, xd, yd)] = 1;
    found++;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
  if (lane == 0 && found) atomicAdd(ncut, found);
}

// ------------------------------------------------------------------- spread
// g(x) += P_k delta_h(x - X_k) (Eq. 46 / Eq. 17), 16 threads per marker.
template <typename T>
__global__ void k_spread(const double *__restrict__ X, const double *__restrict__ P, int n,
                         Geom geo, T *gf, uint8_t *flags) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = tid >> 4, l = tid & 15;
  if (k >= n) return;
  const double Xk = X[2 * k], Yk = X[2 * k + 1];
  if (!(fabs(Xk) <= MAX_COORD && fabs(Yk) <= MAX_COORD)) return;
  const int xa = (int)floor(Xk) - 1 + (l & 3), yb = (int)floor(Yk) - 1 + (l >> 2);
  int xi = xa, yi = yb;
  if (geo.bc == IILBM_BC_CHANNEL) {
    if (xi < 0 || xi >= geo.nx) return;
  } else {
    xi = wrap(xi, geo.nx);
  }
  if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
  else if (yi < 0 || yi >= geo.ny) return;
  const double w = phi4i((double)xa - Xk) * phi4i((double)yb - Yk);
  if (w == 0.0) return;
  const long long here = (long long)yi * geo.pitch + xi;
  atomicAdd(&gf[here], (T)(P[2 * k] * w));
  atomicAdd(&gf[geo.plane + here], (T)(P[2 * k + 1] * w));
  flags[tile_of(geo, xi, yi)] = 1;
}

// ------------------------------------------------------------- tile list
// Compact the flagged tiles into a list for the forced stream-collide.
__global__ void k_tile_list(const uint8_t *__restrict__ flags, int ntiles, int *list, int *count,
                            unsigned long long *total) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool f = t < ntiles && flags[t] != 0;
  const unsigned m = __ballot_sync(0xffffffffu, f);
  int base = 0;
  if ((threadIdx.x & 31) == 0 && m) {
    base = atomicAdd(count, __popc(m));
    atomicAdd(total, (unsigned long long)__popc(m));
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (f) list[base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = t;
}

// ---------------------------------------------------------- interface phase
// Items 1-3 of the step for the current state: marker forces and split, the jump on
// every cut link, spreading.  Leaves J, g, flags ready for interpolation and for the
// stream-collide that consumes them.
int launch_interface_phase(iilbm_lattice *h, int buf, cudaStream_t s) {
  if (h->nm == 0) return IILBM_OK;
  const int n = h->nm;
  if (h->ip.model == IILBM_DIRECT) return IILBM_ERR_INVALID_ARG;
  uint8_t *flags = h->flagsb[buf];
  if (cudaMemsetAsync(flags, 0, (size_t)h->ntiles, s) != cudaSuccess ||
      cudaMemsetAsync(h->d_ncut, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(h->tile_count[buf], 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  k_marker_forces<<<(n + 127) / 128, 128, 0, s>>>(h->X, h->aux, n, h->ip, h->cfg.jump, h->geom,
                                                  h->G, h->Fn, h->P, h->nrm, h->d_status);
  const bool dbl = h->cfg.storage == IILBM_F64;
  if (h->cfg.jump) {
    const int threads = 32 * n;
    if (dbl)
      k_cut_links<double><<<(threads + 255) / 256, 256, 0, s>>>(
          h->X, h->Fn, n, h->geom, (double *)h->Jb[buf], flags, h->d_ncut);
    else
      k_cut_links<float><<<(threads + 255) / 256, 256, 0, s>>>(
          h->X, h->Fn, n, h->geom, (float *)h->Jb[buf], flags, h->d_ncut);
  }
  const int threads = 16 * n;
  if (dbl)
    k_spread<double><<<(threads + 255) / 256, 256, 0, s>>>(h->X, h->P, n, h->geom,
                                                          (double *)h->gb[buf], flags);
  else
    k_spread<float><<<(threads + 255) / 256, 256, 0, s>>>(h->X, h->P, n, h->geom,
                                                         (float *)h->gb[buf], flags);
  k_tile_list<<<(h->ntiles + 255) / 256, 256, 0, s>>>(flags, h->ntiles, h->tile_list[buf],
                                                      h->tile_count[buf], h->d_tiles_total);
  return cudaGetLastError() == cudaSuccess ? IILBM_OK : IILBM_ERR_CUDA;
}

}  // namespace iilbm
