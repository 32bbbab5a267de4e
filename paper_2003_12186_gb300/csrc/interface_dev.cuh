// interface_dev.cuh -- device building blocks of the interface phase, shared by the
// single-lattice and the batched kernels (see interface.cu for the method).
#pragma once

#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

__device__ inline int tile_of(const Geom &g, int x, int y) {
  return (y / TILE_Y) * g.ntx + x / TILE_X;
}

struct TileBuf {
  unsigned *flags;            // a tile is flagged iff its entry equals *tag
  const unsigned *tag;
  int *list;
  int *ctr;                   // [0] flagged tiles, [1] cut-link crossings
  unsigned long long *total;  // flagged tiles summed over phases (diagnostic)
};

// Flag a tile for this time level; the first thread to do so appends it to the list.
__device__ inline void flag_tile(const TileBuf &tb, int tile, unsigned tag) {
  if (tb.flags[tile] != tag && atomicExch(&tb.flags[tile], tag) != tag) {
    tb.list[atomicAdd(tb.ctr, 1)] = tile;
    atomicAdd(tb.total, 1ull);
  }
}

// Tile indices (along one axis of n nodes, tiles of width w) covered by the node range
// [a, b], wrapped on a periodic axis, clipped otherwise.  Returns their number (at most
// MAX_TILE_SPAN; ranges here span at most 23 nodes).
constexpr int MAX_TILE_SPAN = 8;
__device__ inline int tile_span(int a, int b, int n, bool periodic, int w, int *out) {
  if (!periodic) {
    a = max(a, 0);
    b = min(b, n - 1);
  }
  int cnt = 0, last = -1;
  for (int v = a; v <= b && cnt < MAX_TILE_SPAN;) {
    const int u = periodic ? wrap(v, n) : v;
    const int t = u / w;
    if (t != last) out[cnt++] = t;
    last = t;
    v += min(w - u % w, n - u);  // to the next tile boundary (or the end of the axis)
  }
  return cnt;
}

// Peskin's four-point kernel phi(r) in the arithmetic type T.
template <typename T>
__device__ inline T phi4t(T r) {
  const T a = fabs(r);
  if (a < T(1)) return T(0.125) * (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a));
  if (a < T(2)) return T(0.125) * (T(5) - T(2) * a - sqrt(T(-7) + T(12) * a - T(4) * a * a));
  return T(0);
}

// Force of marker j and its split: G_j, n_j, Fn_j = G_j.n_j/|X_s|_j, and the point
// force to spread P_j = dX * (tangential part in II-LBM, whole G in IB-LBM).  Marker
// positions and their differences (including the spring's second difference, a small
// difference of O(1) numbers) are FP64; the rest runs in the arithmetic type T.
template <typename T>
struct MarkerForce {
  T gx, gy, nx, ny, fn, px, py;
  bool bad;
};

template <typename T>
__device__ inline MarkerForce<T> marker_force(const double *__restrict__ X,
                                              const double *__restrict__ aux, int n, int j,
                                              const iilbm_interface_params &ip, int jump,
                                              const Geom &geo) {
  MarkerForce<T> m;
  const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
  const double x = X[2 * j], y = X[2 * j + 1];
  const double xp = X[2 * jp], yp = X[2 * jp + 1], xm = X[2 * jm], ym = X[2 * jm + 1];
  const double dax = xp - x, day = yp - y, dbx = x - xm, dby = y - ym;  // segments k, k-1
  // validity: finite, inside the representable / valid region, short segments
  bool bad = !(isfinite(x) && isfinite(y)) || fabs(x) > MAX_COORD || fabs(y) > MAX_COORD;
  bad = bad || !(dax * dax + day * day < MAX_SEGMENT * MAX_SEGMENT);
  if (geo.bc != IILBM_BC_PERIODIC) bad = bad || y < 3.0 || y > geo.ny - 4.0;
  if (geo.bc == IILBM_BC_CHANNEL) bad = bad || x < 3.0 || x > geo.nx - 4.0;
  m.bad = bad;
  T gx, gy;
  if (ip.model == IILBM_SPRING) {
    const T c = T(ip.stiffness / (ip.dX * ip.dX));
    gx = c * T(dax - dbx);
    gy = c * T(day - dby);
  } else if (ip.model == IILBM_SPRING_REST) {
    const T ax = T(dax), ay = T(day), bx = T(dbx), by = T(dby);
    const T la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
    const T Ta = T(ip.stiffness) * (la / T(ip.rest_length) - T(1));
    const T Tb = T(ip.stiffness) * (lb / T(ip.rest_length) - T(1));
    gx = (Ta * (ax / la) - Tb * (bx / lb)) / T(ip.dX);
    gy = (Ta * (ay / la) - Tb * (by / lb)) / T(ip.dX);
  } else {  // prescribed, or the converged direct-forcing force
    gx = T(aux[2 * j]);
    gy = T(aux[2 * j + 1]);
  }
  const T tx = T(xp - xm), ty = T(yp - ym);
  const T tl = sqrt(tx * tx + ty * ty);
  m.nx = ty / tl;  // outward for a counter-clockwise polygon
  m.ny = -tx / tl;
  const T xs = ip.moves ? tl / T(2.0 * ip.dX) : T(1);
  const T gn = gx * m.nx + gy * m.ny;
  m.gx = gx;
  m.gy = gy;
  m.fn = gn / xs;
  const T dX = T(ip.dX);
  if (jump) {
    m.px = (gx - gn * m.nx) * dX;
    m.py = (gy - gn * m.ny) * dX;
  } else {
    m.px = gx * dX;
    m.py = gy * dX;
  }
  return m;
}

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

// Crossings found by a lane are buffered (candidate index, sign, raw orientations) and
// their FP64 coefficients computed together, so the FP64 division runs about once per
// warp rather than once per candidate sweep.
constexpr int CROSS_BUF = 4;

// All interface work of marker k (and segment k -> k+1) for one warp (lane 0..31).
template <typename T>
__device__ __forceinline__ void interface_warp(const double *__restrict__ X,
                                               const double *__restrict__ aux, int n, int k,
                                               int lane, const iilbm_interface_params &ip,
                                               int jump, const Geom &geo, T *Jf, T *gf,
                                               const TileBuf &tb, double *G, double *Fn,
                                               double *nrm, int *status) {
  const int kp = k + 1 == n ? 0 : k + 1;
  // forces of k (lane 0) and k + 1 (lane 1)
  MarkerForce<T> m{};
  if (lane < 2) m = marker_force<T>(X, aux, n, lane == 0 ? k : kp, ip, jump, geo);
  const double FnA = (double)__shfl_sync(0xffffffffu, m.fn, 0);
  const double FnB = (double)__shfl_sync(0xffffffffu, m.fn, 1);
  const T Pkx = __shfl_sync(0xffffffffu, m.px, 0);  // point force of marker k
  const T Pky = __shfl_sync(0xffffffffu, m.py, 0);
  if (lane == 0) {
    if (m.bad) atomicOr(status, ST_INTERFACE);
    G[2 * k] = (double)m.gx;
    G[2 * k + 1] = (double)m.gy;
    Fn[k] = (double)m.fn;
    nrm[2 * k] = (double)m.nx;
    nrm[2 * k + 1] = (double)m.ny;
  }
  const double Ax = X[2 * k], Ay = X[2 * k + 1], Bx = X[2 * kp], By = X[2 * kp + 1];
  // Everything geometric below runs on the coordinates snapped to 2^-24 (exact, as the
  // crossing predicate needs) in 64-bit integers: GB300 executes FP64 -- compares,
  // conversions and rounding included -- at a small fraction of its integer rate.
  const bool inside = fabs(Ax) <= MAX_COORD && fabs(Ay) <= MAX_COORD && fabs(Bx) <= MAX_COORD &&
                      fabs(By) <= MAX_COORD;
  const long long ax = inside ? __double2ll_rn(Ax * QSCALE) : 0;
  const long long ay = inside ? __double2ll_rn(Ay * QSCALE) : 0;
  const long long bx = inside ? __double2ll_rn(Bx * QSCALE) : 0;
  const long long by = inside ? __double2ll_rn(By * QSCALE) : 0;
  const long long Q = (long long)QSCALE;
  const long long QMAX = (long long)(MAX_SEGMENT * QSCALE);
  // floor / ceil of a snapped coordinate in lattice units
  auto qfloor = [](long long v) { return (int)(v >> 24); };
  auto qceil = [](long long v) { return (int)-((-v) >> 24); };
  // ---- cut links of segment k -> k+1
  int found = 0;
  if (jump && inside && llabs(bx - ax) < QMAX && llabs(by - ay) < QMAX) {
    const int x0 = qfloor(min(ax, bx)) - 1, x1 = qceil(max(ax, bx)) + 1;
    const int y0 = qfloor(min(ay, by)) - 1, y1 = qceil(max(ay, by)) + 1;
    const int W = x1 - x0 + 1, H = y1 - y0 + 1;
    const int ncand = W * H * 8;
    int bc_idx[CROSS_BUF], bc_s[CROSS_BUF];
    long long bc_o3[CROSS_BUF], bc_o4[CROSS_BUF];
    int nb = 0;
    // apply the buffered crossings: coefficient s w_i/c_s^2 Fn(t), t = o3 / (o3 - o4)
    // along A -> B (an FP32 quotient refined by one FP64 Newton step, ~1e-14)
    auto flush = [&]() {
#pragma unroll
      for (int q = 0; q < CROSS_BUF; q++) {
        if (q >= nb) break;
        const int c = bc_idx[q];
        const int i = 1 + c % 8, cell = c / 8;
        int xd = x0 + cell % W, yd = y0 + cell / W;
        xd = geo.bc == IILBM_BC_CHANNEL ? xd : wrap(xd, geo.nx);
        yd = geo.bc == IILBM_BC_PERIODIC ? wrap(yd, geo.ny) : yd;
        const long long den = bc_o3[q] - bc_o4[q];  // nonzero: the link crosses A -> B
        const double num = (double)bc_o3[q], dd = (double)den;
        const float rf = 1.0f / (float)dd;
        double t = (double)((float)num * rf);
        t = fma(num - t * dd, (double)rf, t);  // one Newton correction with the FP32 reciprocal
        t = fmin(fmax(t, 0.0), 1.0);
        const double F = (1.0 - t) * FnA + t * FnB;
        const double coef = (double)bc_s[q] * 3.0 * wt<double>(i) * F;  // w_i / c_s^2 Fn
        atomicAdd(&Jf[(long long)(i - 1) * geo.plane + (long long)yd * geo.pitch + xd],
                  (T)coef);
      }
      found += nb;
      nb = 0;
    };
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
      // destination and source inside the lattice (periodic axes wrap)
      const int xs = qx - ex, ys = qy - ey;
      if (geo.bc == IILBM_BC_CHANNEL && (qx < 0 || qx >= geo.nx || xs < 0 || xs >= geo.nx))
        continue;
      if (geo.bc != IILBM_BC_PERIODIC && (qy < 0 || qy >= geo.ny || ys < 0 || ys >= geo.ny))
        continue;
      if (nb == CROSS_BUF) flush();
      bc_idx[nb] = c;
      bc_s[nb] = s1;
      bc_o3[nb] = o3;
      bc_o4[nb] = o4;
      nb++;
    }
    flush();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
  if (lane == 0 && found) atomicAdd(&tb.ctr[1], found);
  // ---- spread P_k (Eq. 46 / Eq. 17), lanes 0..15 one stencil node each
  if (lane < 16 && inside) {
    // the stencil is chosen from the FP64 coordinate, as the interpolation does
    const int xa = (int)floor(Ax) - 1 + (lane & 3), yb = (int)floor(Ay) - 1 + (lane >> 2);
    int xi = xa, yi = yb;
    bool ok = true;
    if (geo.bc == IILBM_BC_CHANNEL) ok = xi >= 0 && xi < geo.nx;
    else xi = wrap(xi, geo.nx);
    if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
    else ok = ok && yi >= 0 && yi < geo.ny;
    // node offsets: exact in FP64 for FP64 storage; from the snapped integers otherwise
    T rx, ry;
    if (sizeof(T) == 8) {
      rx = T((double)xa - Ax);
      ry = T((double)yb - Ay);
    } else {
      rx = T((int)((long long)xa * Q - ax)) * T(1.0 / QSCALE);
      ry = T((int)((long long)yb * Q - ay)) * T(1.0 / QSCALE);
    }
    const T w = ok ? phi4t<T>(rx) * phi4t<T>(ry) : T(0);
    if (w != T(0)) {
      const long long here = (long long)yi * geo.pitch + xi;
      atomicAdd(&gf[here], Pkx * w);
      atomicAdd(&gf[geo.plane + here], Pky * w);
    }
  }
  // ---- flag the tiles of the warp's footprint once: every node written above lies in
  // [floor(min x) - 2, ceil(max x) + 2] x [floor(min y) - 2, ceil(max y) + 2]
  if (inside) {
    int cols[MAX_TILE_SPAN], rows[MAX_TILE_SPAN];
    const int nc = tile_span(qfloor(min(ax, bx)) - 2, qceil(max(ax, bx)) + 2, geo.nx,
                             geo.bc != IILBM_BC_CHANNEL, TILE_X, cols);
    const int nr = tile_span(qfloor(min(ay, by)) - 2, qceil(max(ay, by)) + 2, geo.ny,
                             geo.bc == IILBM_BC_PERIODIC, TILE_Y, rows);
    const unsigned tag = *tb.tag;
    for (int t = lane; t < nc * nr; t += 32)
      flag_tile(tb, rows[t / nc] * geo.ntx + cols[t % nc], tag);
  }
}


}  // namespace iilbm
