// interface_dev.cuh -- device building blocks of the interface phase, shared by the
// single-lattice and the batched kernels (see interface.cu for the method).
#pragma once

#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

struct TileBuf {
  unsigned *flags;            // a tile is flagged iff its entry equals *tag
  const unsigned *tag;
  int *list;
  int *ctr;                   // [0] flagged tiles, [1] cut-link crossings
  unsigned long long *total;  // flagged tiles summed over phases (diagnostic)
};

// Flag a tile for this time level; the first thread to do so appends it to the list.
// One exchange, without reading the flag first: a read would put one more memory round
// trip on the interface phase's critical path, which runs beside the bandwidth-bound
// stream-collide (repeated exchanges on a flagged tile cost atomic throughput only).
__device__ inline void flag_tile(const TileBuf &tb, int tile, unsigned tag) {
  if (atomicExch(&tb.flags[tile], tag) != tag) {
    tb.list[atomicAdd(tb.ctr, 1)] = tile;
    atomicAdd(tb.total, 1ull);
  }
}

// Tiles (along one axis of n nodes, tiles of width w) covered by the node range
// [a, b]: the cyclic range of cnt tiles from t0 on a periodic axis (all of them once
// the range spans the axis), the clipped range otherwise.  Tile k of the range is
// (t0 + k) mod (number of tiles on the axis).
__device__ inline void tile_range(int a, int b, int n, bool periodic, int w, int &t0,
                                  int &cnt) {
  const int nt = (n + w - 1) / w;
  if (periodic) {
    if (b - a + 1 >= n) {
      t0 = 0;
      cnt = nt;
      return;
    }
    t0 = wrap(a, n) / w;
    const int t1 = wrap(b, n) / w;
    cnt = t1 >= t0 ? t1 - t0 + 1 : t1 + nt - t0 + 1;
    return;
  }
  a = max(a, 0);
  b = min(b, n - 1);
  t0 = a / w;
  cnt = a <= b ? b / w - t0 + 1 : 0;
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

// (x, y): marker j; (xp, yp), (xm, ym): its successor and predecessor on the polygon;
// (tgx, tgy) the tangent the normal is taken from and |X_s| = |tangent| / tg_len (the
// polygon's central difference X_{j+1} - X_{j-1} with tg_len = 2 dX, or the spline's
// derivative X'(j) with tg_len = dX).
template <typename T, typename GG>
__device__ inline MarkerForce<T> marker_force_tangent(double x, double y, double xp, double yp,
                                                      double xm, double ym, double tgx,
                                                      double tgy, double tg_len,
                                                      const double *__restrict__ aux, int j,
                                                      const iilbm_interface_params &ip,
                                                      int jump, const GG &geo) {
  MarkerForce<T> m;
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
  const T tx = T(tgx), ty = T(tgy);
  const T tl = sqrt(tx * tx + ty * ty);
  m.nx = ty / tl;  // outward for a counter-clockwise polygon
  m.ny = -tx / tl;
  const T xs = ip.moves ? tl / T(tg_len) : T(1);
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

// The polygon's marker force: normal from the central difference X_{j+1} - X_{j-1}.
template <typename T, typename GG>
__device__ inline MarkerForce<T> marker_force_at(double x, double y, double xp, double yp,
                                                 double xm, double ym,
                                                 const double *__restrict__ aux, int j,
                                                 const iilbm_interface_params &ip, int jump,
                                                 const GG &geo) {
  return marker_force_tangent<T>(x, y, xp, yp, xm, ym, xp - xm, yp - ym, 2.0 * ip.dX, aux, j,
                                 ip, jump, geo);
}

template <typename T, typename GG>
__device__ inline MarkerForce<T> marker_force(const double *__restrict__ X,
                                              const double *__restrict__ aux, int n, int j,
                                              const iilbm_interface_params &ip, int jump,
                                              const GG &geo) {
  const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
  return marker_force_at<T>(X[2 * j], X[2 * j + 1], X[2 * jp], X[2 * jp + 1], X[2 * jm],
                            X[2 * jm + 1], aux, j, ip, jump, geo);
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

// ----------------------------------------------------------- Peskin stencil
// The marker pass (interface_block) runs one thread per marker: its force and normal
// split, its coordinates snapped to 2^-24 for the segment pass.  Running this per
// thread rather than once per warp keeps GB300's FP64 pipe (a small fraction of its
// FP32 rate) off the critical path: the FP64 work of a marker is done once, by one lane.
// Its point force P_j is spread over the 4 x 4 stencil (Eq. 46 in II-LBM, Eq. 17 in
// IB-LBM) by 16 lanes of the warp of its segment (by the marker's own thread in the
// batched marker pass).
//
// Stencil: nodes floor(X) - 1 .. floor(X) + 2 on each axis.  For FP64 storage the
// floor and the node offsets are taken from the FP64 coordinate; otherwise from the
// snapped one (the choices differ only within 2^-25 below a lattice line, where the
// dropped node's weight is O(2^-50)), so the 32-bit path needs no FP64 here.
template <typename T>
__device__ inline void stencil_weights(double x, long long q, int &base, T w[4]) {
  if (sizeof(T) == 8) {
    base = (int)floor(x) - 1;
#pragma unroll
    for (int a = 0; a < 4; a++) w[a] = phi4<T>(T((double)(base + a) - x));
  } else {
    base = (int)(q >> 24) - 1;
#pragma unroll
    for (int a = 0; a < 4; a++)
      w[a] = phi4<T>(T((int)((long long)(base + a) * (long long)QSCALE - q)) * T(1.0 / QSCALE));
  }
}

// The weight of stencil node base + k alone (the same value stencil_weights gives it).
template <typename T>
__device__ inline T stencil_weight(double x, long long q, int k, int &base) {
  if (sizeof(T) == 8) {
    base = (int)floor(x) - 1;
    return phi4<T>(T((double)(base + k) - x));
  }
  base = (int)(q >> 24) - 1;
  return phi4<T>(T((int)((long long)(base + k) * (long long)QSCALE - q)) * T(1.0 / QSCALE));
}

__device__ inline bool in_region(double x, double y) {
  return fabs(x) <= MAX_COORD && fabs(y) <= MAX_COORD;
}

// The marker pass of the batched executor, one thread per marker j of its flattened
// list: force, split, snapped coordinates, and the spread of P_j over the stencil.
// cs: the spline coefficients of the marker coordinates (the spline interface: the
// normal from the spline's tangent X'(j) = (c_{j+1} - c_{j-1}) / 2, |X_s| = |X'(j)| / dX),
// or null (the polygon).
template <typename T, typename GG>
__device__ __forceinline__ void interface_marker(const double *__restrict__ X,
                                                 const double *__restrict__ aux, int n, int j,
                                                 const iilbm_interface_params &ip, int jump,
                                                 const GG &geo, T *gf, double *G, double *Fn,
                                                 double *nrm, long long *Xq, int *status,
                                                 const double *__restrict__ cs = nullptr) {
  MarkerForce<T> m;
  if (cs) {
    const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
    m = marker_force_tangent<T>(X[2 * j], X[2 * j + 1], X[2 * jp], X[2 * jp + 1], X[2 * jm],
                                X[2 * jm + 1], 0.5 * (cs[2 * jp] - cs[2 * jm]),
                                0.5 * (cs[2 * jp + 1] - cs[2 * jm + 1]), ip.dX, aux, j, ip, jump,
                                geo);
  } else {
    m = marker_force<T>(X, aux, n, j, ip, jump, geo);
  }
  if (m.bad) atomicOr(status, ST_INTERFACE);
  G[2 * j] = (double)m.gx;
  G[2 * j + 1] = (double)m.gy;
  Fn[j] = (double)m.fn;
  nrm[2 * j] = (double)m.nx;
  nrm[2 * j + 1] = (double)m.ny;
  const int jp = j + 1 == n ? 0 : j + 1;
  const double x = X[2 * j], y = X[2 * j + 1];
  const bool inside = in_region(x, y);
  const long long qx = inside ? __double2ll_rn(x * QSCALE) : XQ_OUT;
  const long long qy = inside ? __double2ll_rn(y * QSCALE) : XQ_OUT;
  Xq[2 * j] = qx;
  Xq[2 * j + 1] = qy;
  // the spread goes into the tiles that the segment j -> j+1 flags, so it needs both ends
  if (!inside || !in_region(X[2 * jp], X[2 * jp + 1])) return;
  int bx, by;
  T wx[4], wy[4];
  stencil_weights<T>(x, qx, bx, wx);
  stencil_weights<T>(y, qy, by, wy);
#pragma unroll
  for (int b = 0; b < 4; b++) {
    int yi = by + b;
    bool oky = true;
    if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
    else oky = yi >= 0 && yi < geo.ny;
#pragma unroll
    for (int a = 0; a < 4; a++) {
      int xi = bx + a;
      bool ok = oky;
      if (geo.bc == IILBM_BC_CHANNEL) ok = ok && xi >= 0 && xi < geo.nx;
      else xi = wrap(xi, geo.nx);
      const T w = wx[a] * wy[b];
      if (ok && w != T(0)) {
        const long long here = (long long)yi * geo.pitch + xi;
        atomicAdd(&gf[here], m.px * w);
        atomicAdd(&gf[geo.plane + here], m.py * w);
      }
    }
  }
}

// ------------------------------------------------------------ segment pass
// One warp per segment k -> k+1: every lattice link x - e_i -> x that crosses it, and
// the tiles of its footprint.  Integer geometry on the snapped coordinates written by
// the marker pass.  The orientation of a lattice node against the segment's line is
// shared by the 8 links that end there and the 8 that start there, so for a short
// segment each node's sign is computed once and published to the warp as one bit of a
// 64-bit ballot; a candidate link then costs two bit lookups, and only links whose ends
// straddle the line take the two link-side tests.

// Every lattice link x - e_i -> x that crosses segment A -> B (snapped coordinates),
// enumerated by the 32 lanes of a warp; each crossing calls emit(i, dx, dy, s, t) with
// the destination node (dx, dy) wrapped onto the lattice, the sign s (+1 when the link
// leaves the interior, the left of A -> B) and the crossing parameter t along A -> B in
// the arithmetic type T (FP64 for FP64 storage: an FP32 quotient refined by one Newton
// step; FP32 otherwise: |o3|, |o3 - o4| < 2^31 fit the int casts, and converting each to
// FP32 rounds it with a relative error of at most 2^-24, so t carries a few FP32 ulps).
// Links whose source or destination lies outside a non-periodic lattice are skipped.
// Returns this lane's number of crossings.  Every lane of the warp must call this.
template <typename T, typename GG, typename Emit>
__device__ __forceinline__ int segment_crossings(long long ax, long long ay, long long bx,
                                                 long long by, int lane, const GG &geo,
                                                 Emit &&emit) {
  const long long Q = (long long)QSCALE;
  auto qceil = [](long long v) { return (int)-((-v) >> 24); };
  int found = 0;
  // destinations x of links that can reach the segment: with the node displaced by
  // (eps, eps^2) the link x - e_i -> x spans [x - 1 + eps, x + 1 + eps] at most on
  // each axis, which meets [min, max] only for ceil(min) - 1 <= x <= ceil(max)
  const int x0 = qceil(min(ax, bx)) - 1, x1 = qceil(max(ax, bx));
  const int y0 = qceil(min(ay, by)) - 1, y1 = qceil(max(ay, by));
  const int W = x1 - x0 + 1, H = y1 - y0 + 1;
  const int ncand = W * H * 8;
  // node signs on the grid [x0-1, x1+1] x [y0-1, y1+1] (GW x GH nodes)
  const int GW = W + 2, GH = H + 2;
  const bool fast = GW * GH <= 64;
  unsigned lo = 0u, hi = 0u;
  if (fast) {
    bool p0 = false, p1 = false;
    if (lane < GW * GH)
      p0 = orient_seg_node(ax, ay, bx, by, (long long)(x0 - 1 + lane % GW) * Q,
                           (long long)(y0 - 1 + lane / GW) * Q) > 0;
    if (lane + 32 < GW * GH)
      p1 = orient_seg_node(ax, ay, bx, by, (long long)(x0 - 1 + (lane + 32) % GW) * Q,
                           (long long)(y0 - 1 + (lane + 32) / GW) * Q) > 0;
    lo = __ballot_sync(0xffffffffu, p0);
    hi = __ballot_sync(0xffffffffu, p1);
  }
  auto node_sign = [&](int qx, int qy) {
    if (fast) {
      const int idx = (qy - y0 + 1) * GW + (qx - x0 + 1);
      const unsigned bit = idx < 32 ? (lo >> idx) & 1u : (hi >> (idx - 32)) & 1u;
      return bit ? 1 : -1;
    }
    return orient_seg_node(ax, ay, bx, by, (long long)qx * Q, (long long)qy * Q);
  };
  // cell -> (column, row) of the W-wide box by an FP32 quotient: (cell + 1/2) / W is
  // at least 1/(2W) away from an integer, far above its rounding error (W <= 19)
  const float invW = 1.0f / (float)W;
  for (int c = lane; c < ncand; c += 32) {
    const int i = 1 + (c & 7);
    const int cell = c >> 3;
    const int gy = (int)(((float)cell + 0.5f) * invW), gx = cell - gy * W;
    const int qx = x0 + gx, qy = y0 + gy;  // destination node
    const int ex = cx(i), ey = cy(i);
    const int s1 = node_sign(qx - ex, qy - ey);
    const int s2 = node_sign(qx, qy);
    if (s1 == s2) continue;
    const long long Px = (long long)(qx - ex) * Q, Py = (long long)(qy - ey) * Q;
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
    T t;
    if (sizeof(T) == 8) {
      const double num = (double)o3, dd = (double)(o3 - o4);
      const float rf = 1.0f / (float)dd;
      double td = (double)((float)num * rf);
      td = fma(num - td * dd, (double)rf, td);
      t = T(fmin(fmax(td, 0.0), 1.0));
    } else {
      const float num = (float)(int)o3, dd = (float)(int)(o3 - o4);
      t = T(fminf(fmaxf(num / dd, 0.0f), 1.0f));
    }
    const int dx = geo.bc == IILBM_BC_CHANNEL ? qx : wrap(qx, geo.nx);
    const int dy = geo.bc == IILBM_BC_PERIODIC ? wrap(qy, geo.ny) : qy;
    emit(i, dx, dy, s1, t);
    found++;
  }
  return found;
}

// The jump of Eq. 32 on every link crossing segment A -> B: coef(i, s, t) (the jump
// s w_i/c_s^2 Fn at crossing parameter t) added to the jump field of the link's
// destination (Eq. 47), the crossings counted, and the flags of the tiles of the
// segment's footprint set.
template <typename T, typename GG, typename Coef>
__device__ __forceinline__ void segment_jump(long long ax, long long ay, long long bx,
                                             long long by, int lane, int jump, const GG &geo,
                                             T *Jf, const TileBuf &tb, unsigned tag,
                                             Coef &&coef) {
  const bool inside = ax != XQ_OUT && bx != XQ_OUT;
  const long long QMAX = (long long)(MAX_SEGMENT * QSCALE);
  // floor / ceil of a snapped coordinate in lattice units
  auto qfloor = [](long long v) { return (int)(v >> 24); };
  auto qceil = [](long long v) { return (int)-((-v) >> 24); };
  int found = 0;
  if (jump && inside && llabs(bx - ax) < QMAX && llabs(by - ay) < QMAX) {
    found = segment_crossings<T>(ax, ay, bx, by, lane, geo, [&](int i, int dx, int dy, int s1,
                                                                T t) {
      atomicAdd(&Jf[(long long)(i - 1) * geo.plane + (long long)dy * geo.pitch + dx],
                coef(i, s1, t));
    });
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
  if (lane == 0 && found) atomicAdd(&tb.ctr[1], found);
  // ---- flag the tiles of the footprint once: every node written for this segment
  // (its cut links, and the spread of marker k) lies in
  // [floor(min x) - 2, ceil(max x) + 2] x [floor(min y) - 2, ceil(max y) + 2]
  if (inside) {
    int c0, nc, r0, nr;
    tile_range(qfloor(min(ax, bx)) - 2, qceil(max(ax, bx)) + 2, geo.nx,
               geo.bc != IILBM_BC_CHANNEL, TILE_X, c0, nc);
    tile_range(qfloor(min(ay, by)) - 2, qceil(max(ay, by)) + 2, geo.ny,
               geo.bc == IILBM_BC_PERIODIC, TILE_Y, r0, nr);
    const int nty = (geo.ny + TILE_Y - 1) / TILE_Y;
    for (int t = lane; t < nc * nr; t += 32) {
      int col = c0 + t % nc, row = r0 + t / nc;
      if (col >= geo.ntx) col -= geo.ntx;
      if (row >= nty) row -= nty;
      flag_tile(tb, row * geo.ntx + col, tag);
    }
  }
}

// The polygon's segment pass: Fn linear along the segment, s w_i/c_s^2 Fn(t).
template <typename T, typename GG>
__device__ __forceinline__ void segment_links(long long ax, long long ay, long long bx,
                                              long long by, double FnA, double FnB, int lane,
                                              int jump, const GG &geo, T *Jf,
                                              const TileBuf &tb, unsigned tag) {
  const float fA = (float)FnA, fB = (float)FnB;  // FP32 path: converted once per warp
  segment_jump<T>(ax, ay, bx, by, lane, jump, geo, Jf, tb, tag, [&](int i, int s1, T t) -> T {
    if (sizeof(T) == 8)
      return T((double)s1 * 3.0 * wt<double>(i) * ((1.0 - (double)t) * FnA + (double)t * FnB));
    return T((float)s1 * 3.0f * wt<float>(i) * ((1.0f - (float)t) * fA + (float)t * fB));
  });
}

// The segment pass of segment k -> k+1 from the marker pass's outputs in global memory.
template <typename T, typename GG>
__device__ __forceinline__ void interface_segment(const long long *__restrict__ Xq,
                                                  const double *__restrict__ Fn, int n, int k,
                                                  int lane, int jump, const GG &geo, T *Jf,
                                                  const TileBuf &tb) {
  const unsigned tag = *tb.tag;
  const int kp = k + 1 == n ? 0 : k + 1;
  segment_links<T>(Xq[2 * k], Xq[2 * k + 1], Xq[2 * kp], Xq[2 * kp + 1], Fn[k], Fn[kp], lane,
                   jump, geo, Jf, tb, tag);
}

// ------------------------------------------------------------- interpolation
// U_k = sum_x u(x) delta_h(x - X_k) (Eq. 20) from the collision velocity the forced
// stream-collide left in uf, one thread per marker, on the stencil the marker pass
// spread to (same floor and weights); the marker moves X += U when it moves.  FP64
// storage: FP64 throughout.  Otherwise each stencil row is summed in FP32 and the four
// row sums are accumulated in FP64.
template <typename T, typename GG>
__device__ __forceinline__ void interp_at(const T *__restrict__ uf, const GG &geo, double x,
                                          long long qx, double y, long long qy, double &sx,
                                          double &sy) {
  sx = 0.0;
  sy = 0.0;
  if (qx == XQ_OUT) return;
  int bx, by;
  T wx[4], wy[4];
  stencil_weights<T>(x, qx, bx, wx);
  stencil_weights<T>(y, qy, by, wy);
#pragma unroll
  for (int b = 0; b < 4; b++) {
    int yi = by + b;
    bool oky = true;
    if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
    else oky = yi >= 0 && yi < geo.ny;
    T rx = T(0), ry = T(0);
#pragma unroll
    for (int a = 0; a < 4; a++) {
      int xi = bx + a;
      bool ok = oky;
      if (geo.bc == IILBM_BC_CHANNEL) ok = ok && xi >= 0 && xi < geo.nx;
      else xi = wrap(xi, geo.nx);
      if (ok) {
        const long long here = (long long)yi * geo.pitch + xi;
        if (sizeof(T) == 8) {  // FP64: every weight wx * wy formed, as the definition reads
          sx += (double)uf[here] * (double)(wx[a] * wy[b]);
          sy += (double)uf[geo.plane + here] * (double)(wx[a] * wy[b]);
        } else {
          rx += uf[here] * wx[a];
          ry += uf[geo.plane + here] * wx[a];
        }
      }
    }
    if (sizeof(T) != 8) {
      sx += (double)rx * (double)wy[b];
      sy += (double)ry * (double)wy[b];
    }
  }
}

template <typename T, typename GG>
__device__ __forceinline__ void interp_marker(const T *__restrict__ uf, const GG &geo,
                                              double *X, const long long *__restrict__ Xq,
                                              int k, double *U, int moves) {
  const double x = X[2 * k], y = X[2 * k + 1];
  double sx, sy;
  interp_at<T>(uf, geo, x, Xq[2 * k], y, Xq[2 * k + 1], sx, sy);
  U[2 * k] = sx;
  U[2 * k + 1] = sy;
  if (moves) {
    X[2 * k] = x + sx;
    X[2 * k + 1] = y + sy;
  }
}

// ------------------------------------------------------ snapshot for the fused phase
// Work the forced stream-collide of level n does on the side for what follows it:
// advance the tag of the next level's buffer and reset its counters (the readers of
// that buffer's previous level, the lean and forced kernels of level n - 1, are done),
// and, when the interpolation and the next interface phase run fused, copy the marker
// positions and snapped coordinates of level n to Xp, Xqp (the fused kernel reads its
// neighbours' markers there while their owners overwrite X, Xq).
struct MarkerPrep {
  const double *X;
  double *Xp;
  const long long *Xq;
  long long *Xqp;
  int n2;  // entries to copy (2 per marker), 0 for none
  unsigned *next_tag;
  int *next_ctr;
};

__device__ __forceinline__ void marker_prep(const MarkerPrep &mp) {
  const int nt = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && tid == 0) {
    *mp.next_tag += 1u;
    mp.next_ctr[0] = 0;
    mp.next_ctr[1] = 0;
  }
  for (int i = blockIdx.x * nt + tid; i < mp.n2; i += gridDim.x * nt) {
    mp.Xp[i] = mp.X[i];
    mp.Xqp[i] = mp.Xq[i];
  }
}

// ------------------------------------------------------- interface phase block
constexpr int SEGS_PER_BLOCK = 8;
// Warps per block: each takes segments w, w + WARPS, ...  A single lattice's interface
// kernel (one wave of blocks) waits on memory most of its time beside the register-
// heavy lean stream-collide, and 4 warps per 8 segments hold fewer of the registers
// that stream-collide blocks could use.  (The batched executor, with many waves of
// blocks, is limited by throughput instead: there separate marker and segment passes
// with every thread busy beat this block, whose other warps wait while one warp
// interpolates and forms the forces.)
constexpr int IFACE_WARPS = 4;

// Inputs of the fused interpolation (INTERP = true): the collision velocity of the
// streamed level and that level's marker snapshot; U and the new X go to the markers.
template <typename T>
struct InterpIn {
  const T *uf;
  const double *Xp;
  const long long *Xqp;
  double *U;
  int moves;
};

// The interface work of segments a .. a + 7 (and their end markers) of one lattice,
// for a block of 32 WARPS threads; with INTERP, preceded by the interpolation of the
// level just streamed (see interface.cu).
template <typename T, bool INTERP, int WARPS, typename GG>
__device__ __forceinline__ void interface_block(const int a, double *X,
                                                const double *__restrict__ aux, int n,
                                                const iilbm_interface_params &ip, int jump,
                                                const GG &geo, T *gf, T *Jf, const TileBuf &tb,
                                                double *G, double *Fn, double *nrm, long long *Xq,
                                                int *status, const InterpIn<T> &in) {
  __shared__ double sx[SEGS_PER_BLOCK + 3][2];  // markers a - 1 .. a + nseg + 1
  __shared__ long long sq[SEGS_PER_BLOCK + 1][2];
  __shared__ double sfn[SEGS_PER_BLOCK + 1];
  __shared__ T spx[SEGS_PER_BLOCK], spy[SEGS_PER_BLOCK];
  __shared__ int sspread[SEGS_PER_BLOCK];
  const int nseg = min(SEGS_PER_BLOCK, n - a);
  const int t = threadIdx.x;
  const unsigned tag = *tb.tag;  // issued early: the tile flags need it last
  // ---- positions of markers a - 1 .. a + nseg + 1 (n >= 3: one wrap at most)
  if (t < nseg + 3) {
    int j = a - 1 + t;
    if (j < 0) j += n;
    else if (j >= n) j -= n;
    if (INTERP) {
      const double x = in.Xp[2 * j], y = in.Xp[2 * j + 1];
      double ux, uy;
      interp_at<T>(in.uf, geo, x, in.Xqp[2 * j], y, in.Xqp[2 * j + 1], ux, uy);
      const double xn = in.moves ? x + ux : x, yn = in.moves ? y + uy : y;
      sx[t][0] = xn;
      sx[t][1] = yn;
      if (t >= 1 && t <= nseg) {  // owned by this block
        in.U[2 * j] = ux;
        in.U[2 * j + 1] = uy;
        if (in.moves) {
          X[2 * j] = xn;
          X[2 * j + 1] = yn;
        }
      }
    } else {
      sx[t][0] = X[2 * j];
      sx[t][1] = X[2 * j + 1];
    }
  }
  __syncthreads();
  // ---- markers a .. a + nseg (the last is the next block's first, or marker 0)
  if (t <= nseg) {
    const int j = a + t == n ? 0 : a + t;
    const double x = sx[t + 1][0], y = sx[t + 1][1];
    const MarkerForce<T> m = marker_force_at<T>(x, y, sx[t + 2][0], sx[t + 2][1], sx[t][0],
                                                sx[t][1], aux, j, ip, jump, geo);
    const bool inside = in_region(x, y);
    const long long qx = inside ? __double2ll_rn(x * QSCALE) : XQ_OUT;
    const long long qy = inside ? __double2ll_rn(y * QSCALE) : XQ_OUT;
    sq[t][0] = qx;
    sq[t][1] = qy;
    sfn[t] = (double)m.fn;
    if (t < nseg) {  // owned by this block
      if (m.bad) atomicOr(status, ST_INTERFACE);
      G[2 * j] = (double)m.gx;
      G[2 * j + 1] = (double)m.gy;
      Fn[j] = (double)m.fn;
      nrm[2 * j] = (double)m.nx;
      nrm[2 * j + 1] = (double)m.ny;
      Xq[2 * j] = qx;
      Xq[2 * j + 1] = qy;
      // the spread goes into the tiles that segment j -> j+1 flags: it needs both ends
      sspread[t] = inside && in_region(sx[t + 2][0], sx[t + 2][1]);
      spx[t] = m.px;
      spy[t] = m.py;
    }
  }
  __syncthreads();
  const int w = t >> 5, lane = t & 31;
  // ---- cut links and tile flags of segments a + w, a + w + WARPS, ...
  for (int k = w; k < nseg; k += WARPS)
    segment_links<T>(sq[k][0], sq[k][1], sq[k + 1][0], sq[k + 1][1], sfn[k], sfn[k + 1], lane,
                     jump, geo, Jf, tb, tag);
  // ---- spread of the segments' first markers, 16 lanes (one stencil node each) per
  // marker (Eq. 46 / 17)
  for (int k0 = w; k0 < nseg; k0 += 2 * WARPS) {
    const int k = k0 + (lane < 16 ? 0 : WARPS), l = lane & 15;
    if (k >= nseg || !sspread[k]) continue;
    int bx, by;
    const T wxl = stencil_weight<T>(sx[k + 1][0], sq[k][0], l & 3, bx);
    const T wyl = stencil_weight<T>(sx[k + 1][1], sq[k][1], l >> 2, by);
    int xi = bx + (l & 3), yi = by + (l >> 2);
    bool ok = true;
    if (geo.bc == IILBM_BC_PERIODIC) yi = wrap(yi, geo.ny);
    else ok = yi >= 0 && yi < geo.ny;
    if (geo.bc == IILBM_BC_CHANNEL) ok = ok && xi >= 0 && xi < geo.nx;
    else xi = wrap(xi, geo.nx);
    const T wgt = wxl * wyl;
    if (ok && wgt != T(0)) {
      const long long here = (long long)yi * geo.pitch + xi;
      atomicAdd(&gf[here], spx[k] * wgt);
      atomicAdd(&gf[geo.plane + here], spy[k] * wgt);
    }
  }
}

}  // namespace iilbm
