// lattice_dev.cuh -- device building blocks of the stream-collide, shared by the
// single-lattice and the batched kernels: collision parameters, the SRT / MRT
// collision with Guo forcing, vector storage access, and the per-(sub-)tile bodies of
// the lean and forced AA-pattern stream-collide.
#pragma once

#include <type_traits>

#include "iilbm_internal.cuh"

#include <cmath>

namespace iilbm {

template <typename T>
struct CollP {
  T omega;          // 1/tau (SRT)
  T s1, s2, s4, s6, s7, s8;  // MRT rates of the non-conserved moments
  T rho0;
  T scale, inv_scale;        // storage scale 2^k and 2^-k
  T bodyx, bodyy;
  int he;                    // the simple force term (Eq. 16) instead of Guo's (Eqs. 21-24)
};

template <typename T>
CollP<T> make_collp(const iilbm_config &c) {
  CollP<T> p;
  p.he = c.force == IILBM_FORCE_SIMPLE;
  p.omega = T(1.0 / c.tau);
  p.s1 = T(c.s[1]); p.s2 = T(c.s[2]); p.s4 = T(c.s[4]); p.s6 = T(c.s[6]);
  p.s7 = T(c.s[7]); p.s8 = T(c.s[8]);
  p.rho0 = T(c.rho0);
  p.scale = T(std::ldexp(1.0, c.storage_scale_log2));
  p.inv_scale = T(std::ldexp(1.0, -c.storage_scale_log2));
  p.bodyx = T(c.body[0]);
  p.bodyy = T(c.body[1]);
  return p;
}

// ------------------------------------------------------------------ collision
// Shifted populations in, post-collision shifted populations out.
//   rho = rho0 + drho,  rho u = j + g/2  (Eqs. 11, 24)
//   feq_i - w_i rho0 = w_i [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u^2)]  (Eq. 23)
//   Guo source  Gt_i = w_i [3 (e_i - u).g + 9 (e_i.u)(e_i.g)]  (Eqs. 21-22)
// The populations and the force come in the storage's units, multiplied by its scale
// 2^k (f' = 2^k f, g' = 2^k g), and the populations go out in them: every moment is
// linear in f and g, and the velocity is j' / (2^k rho), so the collision runs on the
// scaled values directly.  Multiplying by a power of two is exact, so each operation
// rounds as it would on the unscaled values: the results are the unscaled collision's
// times 2^k, bit for bit, with no conversion multiply per population.  Returns the
// unscaled drho; ux_out, uy_out are the unscaled velocity.
// BODY = false: the force is zero (lean tiles without a body force) and Guo's source
// terms are left out.  With p.he (the simple external force term of Eq. 16) the
// velocity is j / rho, the relaxation has no source, and (1/c_s^2) w_i e_i . g is added
// to every population afterwards.
// PP is CollP<T>, or a volatile view of one in shared memory (the batched kernels:
// every rate is then re-read where it is used instead of held in a register).
template <typename T, int COLL, typename PP = CollP<T>, bool BODY = true>
__device__ __forceinline__ T collide(T f[9], T gx, T gy, const PP &p, T &ux_out,
                                     T &uy_out) {
  const T drs = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const T jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const T jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  const T drho = drs * p.inv_scale;
  const T rho = p.rho0 + drho;
  const T irs = (T(1) / rho) * p.inv_scale;                   // 1 / (2^k rho)
  const bool guo = BODY && !p.he;
  const T jxh = guo ? jx + T(0.5) * gx : jx, jyh = guo ? jy + T(0.5) * gy : jy;  // rho u
  const T ux = jxh * irs, uy = jyh * irs;
  ux_out = ux;
  uy_out = uy;
  if (COLL == IILBM_SRT) {
    const T u2 = ux * ux + uy * uy;
    const T ug = ux * gx + uy * gy;
    const T om = p.omega, fo = T(1) - T(0.5) * p.omega;
    const T rhos = rho * p.scale;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      const T eu = T(cx(i)) * ux + T(cy(i)) * uy;
      const T feq = wt<T>(i) * (drs + rhos * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * u2));
      f[i] = f[i] - om * (f[i] - feq);
      if (BODY) {
        const T eg = T(cx(i)) * gx + T(cy(i)) * gy;
        if (guo) f[i] += fo * (wt<T>(i) * (T(3) * (eg - ug) + T(9) * eu * eg));
        else f[i] += wt<T>(i) * (T(3) * eg);
      }
    }
  } else {
    // Lallemand-Luo moments of df: e, eps, qx, qy, pxx, pxy (rho, jx, jy above).
    const T sa = (f[1] + f[2]) + (f[3] + f[4]);
    const T sd = (f[5] + f[6]) + (f[7] + f[8]);
    const T m1 = T(-4) * f[0] - sa + T(2) * sd;
    const T m2 = T(4) * f[0] - T(2) * sa + sd;
    const T m4 = T(-2) * (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    const T m6 = T(-2) * (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
    const T m7 = (f[1] + f[3]) - (f[2] + f[4]);
    const T m8 = (f[5] + f[7]) - (f[6] + f[8]);
    // equilibrium moments of the shifted equilibrium
    const T ru2 = jxh * ux + jyh * uy;  // rho u^2
    const T e1 = T(-2) * drs + T(3) * ru2;
    const T e2 = drs - T(3) * ru2;
    const T e4 = -jxh, e6 = -jyh;
    const T e7 = jxh * ux - jyh * uy;
    const T e8 = jxh * uy;
    T d1 = -p.s1 * (m1 - e1), d2 = -p.s2 * (m2 - e2), d4 = -p.s4 * (m4 - e4);
    T d6 = -p.s6 * (m6 - e6), d7 = -p.s7 * (m7 - e7), d8 = -p.s8 * (m8 - e8);
    T a3 = T(0), a5 = T(0);
    if (guo) {
      // moments of Guo's source
      const T ug = ux * gx + uy * gy;
      const T F1 = T(6) * ug, F2 = T(-6) * ug, F4 = -gx, F6 = -gy;
      const T F7 = T(2) * (ux * gx - uy * gy), F8 = ux * gy + uy * gx;
      d1 += (T(1) - T(0.5) * p.s1) * F1;
      d2 += (T(1) - T(0.5) * p.s2) * F2;
      d4 += (T(1) - T(0.5) * p.s4) * F4;
      d6 += (T(1) - T(0.5) * p.s6) * F6;
      d7 += (T(1) - T(0.5) * p.s7) * F7;
      d8 += (T(1) - T(0.5) * p.s8) * F8;
      // conserved moments: rho unchanged, j gains exactly g (any s3, s5)
      a3 = gx * T(1.0 / 6);
      a5 = gy * T(1.0 / 6);
    }
    const T a1 = d1 * T(1.0 / 36), a2 = d2 * T(1.0 / 36);
    const T a4 = d4 * T(1.0 / 12), a6 = d6 * T(1.0 / 12);
    const T a7 = d7 * T(0.25), a8 = d8 * T(0.25);
    const T b = -a1 - T(2) * a2;        // common to the axis velocities
    const T c = T(2) * a1 + a2;         // common to the diagonals
    f[0] += T(-4) * a1 + T(4) * a2;
    if (BODY) {
      f[1] += b + a3 - T(2) * a4 + a7;
      f[2] += b + a5 - T(2) * a6 - a7;
      f[3] += b - a3 + T(2) * a4 + a7;
      f[4] += b - a5 + T(2) * a6 - a7;
      f[5] += c + (a3 + a4) + (a5 + a6) + a8;
      f[6] += c - (a3 + a4) + (a5 + a6) - a8;
      f[7] += c - (a3 + a4) - (a5 + a6) + a8;
      f[8] += c + (a3 + a4) - (a5 + a6) - a8;
      if (!guo) {  // the simple force term, (1/c_s^2) w_i e_i . g
        const T ax = gx * T(1.0 / 3), ay = gy * T(1.0 / 3);
        const T dx = gx * T(1.0 / 12), dy = gy * T(1.0 / 12);
        f[1] += ax;
        f[2] += ay;
        f[3] -= ax;
        f[4] -= ay;
        f[5] += dx + dy;
        f[6] += dy - dx;
        f[7] -= dx + dy;
        f[8] += dx - dy;
      }
    } else {
      f[1] += b - T(2) * a4 + a7;
      f[2] += b - T(2) * a6 - a7;
      f[3] += b + T(2) * a4 + a7;
      f[4] += b + T(2) * a6 - a7;
      f[5] += c + a4 + a6 + a8;
      f[6] += c - a4 + a6 - a8;
      f[7] += c - a4 - a6 + a8;
      f[8] += c + a4 - a6 - a8;
    }
  }
  return drho;
}

// -------------------------------------------------------------- stream-collide
// The stream-collide is split by tile.  Tiles (TILE_X x TILE_Y nodes) that carry no
// jump and no spread force -- all but O(interface length) of them -- go through a
// lean kernel with no jump / force code at all, which keeps its register count and
// so its memory parallelism high.  The flagged tiles are listed by the interface phase
// and processed by a "forced" kernel that adds the jump of Eq. 47 and the spread
// force of Eq. 46.  Under the AA pattern every population
// slot is read and written by one and the same node, so the two kernels touch
// disjoint slots and may run in either order or concurrently.

// Each thread owns V consecutive nodes of one row (V = 4 for FP32 / FP16 / BF16
// storage, 2 for FP64) and moves every population plane with one 16-byte (8-byte
// for 16-bit storage) vector access per plane.  A warp covers 32 V consecutive nodes
// of one row, a block of 8 warps 8 rows.  In the odd step the planes with e_x = +-1
// are shifted by one node: the aligned vector is loaded (stored) and the one element
// that crosses into the neighbouring lane travels by warp shuffle; lanes 0 and 31
// (and the last active lane of a row) fetch / write that element with a scalar
// access instead, wrapping around the periodic row.  Requires nx % V == 0.
template <typename S> struct Vec { static constexpr int V = sizeof(S) == 8 ? 2 : 4; };

// V consecutive stored values moved with one aligned access (V * sizeof(S) bytes) and
// converted to / from the arithmetic type with the storage scale.  The batched
// kernels also run V = 2: half the registers per thread, and a 64-node row fills a
// warp.
template <typename S, int V>
struct alignas(sizeof(S) * V) Pack {
  S v[V];
};

// 16-bit storage converts two values per instruction where it can (the same rounding,
// to nearest even, as one at a time).
template <typename S, int V>
__device__ inline void vld(const S *p, typename Store<S>::T *o) {
  const Pack<S, V> t = *reinterpret_cast<const Pack<S, V> *>(p);
  if constexpr (std::is_same<S, __half>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V; j += 2) {
      const float2 f = __half22float2(__halves2half2(t.v[j], t.v[j + 1]));
      o[j] = f.x;
      o[j + 1] = f.y;
    }
  } else if constexpr (std::is_same<S, __nv_bfloat16>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V; j += 2) {
      const float2 f = __bfloat1622float2(__halves2bfloat162(t.v[j], t.v[j + 1]));
      o[j] = f.x;
      o[j + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; j++) o[j] = Store<S>::ld(t.v[j]);
  }
}

template <typename S, int V>
__device__ inline void vst(S *p, const typename Store<S>::T *v) {
  Pack<S, V> t;
  if constexpr (std::is_same<S, __half>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V; j += 2) {
      const __half2 h = __floats2half2_rn(v[j], v[j + 1]);
      t.v[j] = __low2half(h);
      t.v[j + 1] = __high2half(h);
    }
  } else if constexpr (std::is_same<S, __nv_bfloat16>::value && V % 2 == 0) {
#pragma unroll
    for (int j = 0; j < V; j += 2) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[j], v[j + 1]);
      t.v[j] = __low2bfloat16(h);
      t.v[j + 1] = __high2bfloat16(h);
    }
  } else {
#pragma unroll
    for (int j = 0; j < V; j++) t.v[j] = Store<S>::st(v[j]);
  }
  *reinterpret_cast<Pack<S, V> *>(p) = t;
}

// V consecutive arithmetic values (jump / force fields), one aligned access.
template <typename T, int V>
__device__ inline void stT(T *p, const T *v) {
  Pack<T, V> t;
#pragma unroll
  for (int j = 0; j < V; j++) t.v[j] = v[j];
  *reinterpret_cast<Pack<T, V> *>(p) = t;
}
template <typename T, int V>
__device__ inline void ldT(const T *p, T *o) {
  const Pack<T, V> t = *reinterpret_cast<const Pack<T, V> *>(p);
#pragma unroll
  for (int j = 0; j < V; j++) o[j] = t.v[j];
}


// One node per thread on a 32 x TILE_Y sub-block whose first node is (xb, yb).  BC is
// IILBM_BC_PERIODIC, IILBM_BC_WALLS_Y (periodic x, halfway bounce-back in y) or
// IILBM_BC_CHANNEL (walls in y, ghost columns in x filled by the channel boundary).
template <typename S, int COLL, bool ODD, int BC, bool FORCED, bool YWALL = true,
          typename GG = Geom, typename PP = CollP<typename Store<S>::T>>
__device__ __forceinline__ void sc_scalar_block(S *__restrict__ A,
                                                typename Store<S>::T *__restrict__ Jf,
                                                typename Store<S>::T *__restrict__ gf,
                                                typename Store<S>::T *__restrict__ uf,
                                                const GG &geo, const PP &p, int *status,
                                                int xb, int yb) {
  using T = typename Store<S>::T;
  const int x = xb + threadIdx.x, y = yb + threadIdx.y;
  if (x >= geo.nx || y >= geo.ny) return;
  const long long P = geo.plane;
  const long long here = (long long)y * geo.pitch + x;
  const int xm = x == 0 ? (BC == IILBM_BC_CHANNEL ? geo.pitch - 1 : geo.nx - 1) : x - 1;
  const int xp = x == geo.nx - 1 ? (BC == IILBM_BC_CHANNEL ? geo.nx : 0) : x + 1;
  int ym = y - 1, yp = y + 1;
  bool wall_m = false, wall_p = false;
  if (BC == IILBM_BC_PERIODIC) {
    ym = y == 0 ? geo.ny - 1 : ym;
    yp = y == geo.ny - 1 ? 0 : yp;
  } else if (YWALL) {  // otherwise the caller guarantees 1 <= y <= ny - 2
    wall_m = y == 0;
    wall_p = y == geo.ny - 1;
  }
  const long long col[3] = {xm, x, xp};
  const long long row[3] = {(long long)ym * geo.pitch, (long long)y * geo.pitch,
                            (long long)yp * geo.pitch};
  T f[9];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    long long src = i * P + here;
    if (ODD) {
      const bool from_wall = (cy(i) > 0 && wall_m) || (cy(i) < 0 && wall_p);
      if (!from_wall) src = opp(i) * P + row[1 - cy(i)] + col[1 - cx(i)];
    }
    f[i] = Store<S>::ld(A[src]);  // in storage units (collide)
  }
  T gx = p.bodyx, gy = p.bodyy;
  if (FORCED) {
#pragma unroll
    for (int i = 1; i < 9; i++) f[i] += Jf[(i - 1) * P + here] * p.scale;
    gx += gf[here];
    gy += gf[P + here];
  }
  T ux, uy;
  const T drho = collide<T, COLL>(f, gx * p.scale, gy * p.scale, p, ux, uy);
  if (!isfinite(drho)) atomicOr(status, ST_NONFINITE);
  if (FORCED) {  // the velocity the markers are interpolated from (Eq. 20)
    uf[here] = ux;
    uf[P + here] = uy;
    // consumed: leave the buffer clean for the interface phase two steps on
#pragma unroll
    for (int i = 1; i < 9; i++) Jf[(i - 1) * P + here] = T(0);
    gf[here] = T(0);
    gf[P + here] = T(0);
  }
#pragma unroll
  for (int i = 0; i < 9; i++) {
    long long dst = opp(i) * P + here;
    if (ODD) {
      const bool to_wall = (cy(i) > 0 && wall_p) || (cy(i) < 0 && wall_m);
      if (!to_wall) dst = i * P + row[1 + cy(i)] + col[1 + cx(i)];
    }
    A[dst] = Store<S>::st(f[i]);
  }
}

// Vectorised: each thread owns V consecutive nodes of one row (V = 4 for FP32 /
// FP16 / BF16 storage, 2 for FP64) and moves every population plane with one 16-byte
// (8-byte for 16-bit storage) access.  A warp covers 32 V nodes of row yb + warp, the
// first at xb.  In the odd step the planes with e_x = +-1 are shifted by one node: the
// aligned vector is loaded (stored) and the single element that crosses into the
// neighbouring lane travels by warp shuffle; lane 0, lane 31 and the last active lane
// of a row fetch / write that element with a scalar access instead, wrapping around
// the periodic row.  Requires nx % V == 0.  Every lane of the warp must call this.
template <typename S, int COLL, bool ODD, int BC, bool FORCED, int V = Vec<S>::V,
          bool YWALL = true, bool BODY = true, typename GG = Geom,
          typename PP = CollP<typename Store<S>::T>>
__device__ __forceinline__ void sc_vec_block(S *__restrict__ A,
                                             typename Store<S>::T *__restrict__ Jf,
                                             typename Store<S>::T *__restrict__ gf,
                                             typename Store<S>::T *__restrict__ uf,
                                             const GG &geo, const PP &p, int *status,
                                             int xb, int yb) {
  using T = typename Store<S>::T;
  const int lane = threadIdx.x & 31;
  const int y = yb + (threadIdx.x >> 5);
  if (y >= geo.ny) return;  // uniform per warp
  const int x0 = xb + lane * V;
  const bool active = x0 < geo.nx;
  const bool edge_r = active && (lane == 31 || x0 + V >= geo.nx);
  const long long P = geo.plane;
  int ym = y - 1, yp = y + 1;
  bool wall_m = false, wall_p = false;
  if (BC == IILBM_BC_PERIODIC) {
    ym = y == 0 ? geo.ny - 1 : ym;
    yp = y == geo.ny - 1 ? 0 : yp;
  } else if (YWALL) {  // otherwise the caller guarantees 1 <= y <= ny - 2
    wall_m = y == 0;
    wall_p = y == geo.ny - 1;
  }
  const long long row[3] = {(long long)ym * geo.pitch, (long long)y * geo.pitch,
                            (long long)yp * geo.pitch};
  const long long here = row[1] + x0;
  // left / right neighbour column of the chunk (wrapped, or a channel's ghost column)
  const int xl = x0 == 0 ? (BC == IILBM_BC_CHANNEL ? geo.pitch - 1 : geo.nx - 1) : x0 - 1;
  const int xr = x0 + V >= geo.nx ? (BC == IILBM_BC_CHANNEL ? geo.nx : 0) : x0 + V;

  T f[9][V];
#pragma unroll
  for (int i = 0; i < 9; i++) {
#pragma unroll
    for (int j = 0; j < V; j++) f[i][j] = T(0);
    const bool from_wall = ODD && ((cy(i) > 0 && wall_m) || (cy(i) < 0 && wall_p));
    if (!ODD || from_wall) {
      if (active) vld<S, V>(A + i * P + here, f[i]);
    } else {
      const long long base = opp(i) * P + row[1 - cy(i)];
      T c[V];
#pragma unroll
      for (int j = 0; j < V; j++) c[j] = T(0);
      if (active) vld<S, V>(A + base + x0, c);
      if (cx(i) == 0) {
#pragma unroll
        for (int j = 0; j < V; j++) f[i][j] = c[j];
      } else if (cx(i) > 0) {  // source x - 1
        T left = __shfl_up_sync(0xffffffffu, c[V - 1], 1);
        if (active && lane == 0) left = Store<S>::ld(A[base + xl]);
        f[i][0] = left;
#pragma unroll
        for (int j = 1; j < V; j++) f[i][j] = c[j - 1];
      } else {  // source x + 1
        T right = __shfl_down_sync(0xffffffffu, c[0], 1);
        if (edge_r) right = Store<S>::ld(A[base + xr]);
#pragma unroll
        for (int j = 0; j < V - 1; j++) f[i][j] = c[j + 1];
        f[i][V - 1] = right;
      }
    }
  }
  T gx[V], gy[V];
#pragma unroll
  for (int j = 0; j < V; j++) { gx[j] = p.bodyx; gy[j] = p.bodyy; }
  if (FORCED && active) {
#pragma unroll
    for (int i = 1; i < 9; i++) {
      T jv[V];
      ldT<T, V>(Jf + (i - 1) * P + here, jv);
#pragma unroll
      for (int j = 0; j < V; j++) f[i][j] += jv[j] * p.scale;
    }
    T a[V], b[V];
    ldT<T, V>(gf + here, a);
    ldT<T, V>(gf + P + here, b);
#pragma unroll
    for (int j = 0; j < V; j++) { gx[j] += a[j]; gy[j] += b[j]; }
  }
  if (BODY) {
#pragma unroll
    for (int j = 0; j < V; j++) { gx[j] *= p.scale; gy[j] *= p.scale; }  // storage units
  }
  bool finite = true;
  T uxv[V], uyv[V];
#pragma unroll
  for (int j = 0; j < V; j++) {
    T fc[9];
#pragma unroll
    for (int i = 0; i < 9; i++) fc[i] = f[i][j];
    const T drho = collide<T, COLL, PP, BODY>(fc, gx[j], gy[j], p, uxv[j], uyv[j]);
    finite = finite && isfinite(drho);
#pragma unroll
    for (int i = 0; i < 9; i++) f[i][j] = fc[i];
  }
  if (active && !finite) atomicOr(status, ST_NONFINITE);
  if (FORCED && active) {  // the velocity the markers are interpolated from (Eq. 20)
    stT<T, V>(uf + here, uxv);
    stT<T, V>(uf + P + here, uyv);
    // consumed: leave the buffer clean for the interface phase two steps on
    T z[V];
#pragma unroll
    for (int j = 0; j < V; j++) z[j] = T(0);
#pragma unroll
    for (int i = 1; i < 9; i++) stT<T, V>(Jf + (i - 1) * P + here, z);
    stT<T, V>(gf + here, z);
    stT<T, V>(gf + P + here, z);
  }

#pragma unroll
  for (int i = 0; i < 9; i++) {
    const bool to_wall = ODD && ((cy(i) > 0 && wall_p) || (cy(i) < 0 && wall_m));
    if (!ODD || to_wall) {
      if (active) vst<S, V>(A + opp(i) * P + here, f[i]);
    } else {
      const long long base = i * P + row[1 + cy(i)];
      if (cx(i) == 0) {
        if (active) vst<S, V>(A + base + x0, f[i]);
      } else if (cx(i) > 0) {  // destination x + 1
        const T in = __shfl_up_sync(0xffffffffu, f[i][V - 1], 1);
        if (active) {
          if (lane != 0) {
            T v[V];
            v[0] = in;
#pragma unroll
            for (int j = 1; j < V; j++) v[j] = f[i][j - 1];
            vst<S, V>(A + base + x0, v);
          } else {
#pragma unroll
            for (int j = 0; j < V - 1; j++) A[base + x0 + 1 + j] = Store<S>::st(f[i][j]);
          }
          if (edge_r) A[base + xr] = Store<S>::st(f[i][V - 1]);
        }
      } else {  // destination x - 1
        const T in = __shfl_down_sync(0xffffffffu, f[i][0], 1);
        if (active) {
          if (!edge_r) {
            T v[V];
#pragma unroll
            for (int j = 0; j < V - 1; j++) v[j] = f[i][j + 1];
            v[V - 1] = in;
            vst<S, V>(A + base + x0, v);
          } else {
#pragma unroll
            for (int j = 1; j < V; j++) A[base + x0 + j - 1] = Store<S>::st(f[i][j]);
          }
          if (lane == 0) A[base + xl] = Store<S>::st(f[i][0]);
        }
      }
    }
  }
}

constexpr int VEC_ROWS = TILE_Y;  // warps (rows) per block of the vectorised kernels

// A tile row that holds no wall row (neither y = 0 nor y = ny - 1) runs the stream-
// collide compiled without the wall cases (YWALL = false): with walls in y, the general
// code tests every population plane of every row for a wall, which the odd step pays
// for in instructions and registers although only two rows are walls.  yb is the tile
// row's first row; the test is uniform per block.
template <typename S, int COLL, bool ODD, int BC, bool FORCED, int V = Vec<S>::V,
          bool BODY = true, typename GG = Geom, typename PP = CollP<typename Store<S>::T>>
__device__ __forceinline__ void sc_vec_rows(S *__restrict__ A, typename Store<S>::T *__restrict__ Jf,
                                            typename Store<S>::T *__restrict__ gf,
                                            typename Store<S>::T *__restrict__ uf, const GG &geo,
                                            const PP &p, int *status, int xb, int yb) {
  if (BC != IILBM_BC_PERIODIC && (yb == 0 || yb + VEC_ROWS >= geo.ny))
    sc_vec_block<S, COLL, ODD, BC, FORCED, V, true, BODY>(A, Jf, gf, uf, geo, p, status, xb, yb);
  else
    sc_vec_block<S, COLL, ODD, BC, FORCED, V, false, BODY>(A, Jf, gf, uf, geo, p, status, xb, yb);
}

template <typename S, int COLL, bool ODD, int BC, bool FORCED, typename GG = Geom,
          typename PP = CollP<typename Store<S>::T>>
__device__ __forceinline__ void sc_scalar_rows(S *__restrict__ A,
                                               typename Store<S>::T *__restrict__ Jf,
                                               typename Store<S>::T *__restrict__ gf,
                                               typename Store<S>::T *__restrict__ uf,
                                               const GG &geo, const PP &p, int *status, int xb,
                                               int yb) {
  if (BC != IILBM_BC_PERIODIC && (yb == 0 || yb + TILE_Y >= geo.ny))
    sc_scalar_block<S, COLL, ODD, BC, FORCED, true>(A, Jf, gf, uf, geo, p, status, xb, yb);
  else
    sc_scalar_block<S, COLL, ODD, BC, FORCED, false>(A, Jf, gf, uf, geo, p, status, xb, yb);
}

// Inflow / outflow of one channel row on the streamed state (see lattice.cu).
template <typename S>
__device__ __forceinline__ void channel_bc_row(S *A, const Geom &geo,
                                               const CollP<typename Store<S>::T> &p, bool odd,
                                               double u_max, int y) {
  using T = typename Store<S>::T;
  T f[9];
#pragma unroll
  for (int i = 0; i < 9; i++) f[i] = Store<S>::ld(A[aa_loc(geo, odd, i, 1, y)]) * p.inv_scale;
  const T d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const T rho = p.rho0 + d;
  const T ux = ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7])) / rho;
  const T uy = ((f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8])) / rho;
  const double yy = y + 0.5;
  const T uin = T(4.0 * u_max * yy * (geo.ny - yy) / ((double)geo.ny * geo.ny));
  const T u2 = ux * ux + uy * uy, uin2 = uin * uin;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const T eu = T(cx(i)) * ux + T(cy(i)) * uy, ei = T(cx(i)) * uin;
    const T feq_in = wt<T>(i) * (d + rho * (T(3) * ei + T(4.5) * ei * ei - T(1.5) * uin2));
    const T feq_1 = wt<T>(i) * (d + rho * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * u2));
    A[aa_loc(geo, odd, i, 0, y)] = Store<S>::st((feq_in + (f[i] - feq_1)) * p.scale);
  }
  constexpr int out[3] = {3, 6, 7};
#pragma unroll
  for (int q = 0; q < 3; q++)
    A[aa_loc(geo, odd, out[q], geo.nx - 1, y)] = A[aa_loc(geo, odd, out[q], geo.nx - 2, y)];
}

// Box boundary node (x, y) on the streamed state, non-equilibrium extrapolation from its
// inward neighbour n (the diagonal one at a corner):
//   f_i = f_eq_i(rho_b, u_b) + [f_i(n) - f_eq_i(rho(n), u(n))],
// outflow: rho_b = rho0, u_b = u(n); wall: u_b = 0, rho_b = rho(n).  The box streams
// periodically (geo.bc periodic), so what the edge received from the far side is
// replaced here.
template <typename S>
__device__ __forceinline__ void box_bc_node(S *A, const Geom &geo,
                                            const CollP<typename Store<S>::T> &p, bool odd,
                                            bool outflow, int x, int y) {
  using T = typename Store<S>::T;
  const int px = x + (x == 0) - (x == geo.nx - 1), py = y + (y == 0) - (y == geo.ny - 1);
  T f[9];
#pragma unroll
  for (int i = 0; i < 9; i++) f[i] = Store<S>::ld(A[aa_loc(geo, odd, i, px, py)]) * p.inv_scale;
  const T d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const T rho = p.rho0 + d;
  const T ux = ((f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7])) / rho;
  const T uy = ((f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8])) / rho;
  const T u2 = ux * ux + uy * uy;
  const T db = outflow ? T(0) : d, rb = p.rho0 + db;
  const T ubx = outflow ? ux : T(0), uby = outflow ? uy : T(0);
  const T ub2 = ubx * ubx + uby * uby;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const T eu = T(cx(i)) * ux + T(cy(i)) * uy, eb = T(cx(i)) * ubx + T(cy(i)) * uby;
    const T feq_n = wt<T>(i) * (d + rho * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * u2));
    const T feq_b = wt<T>(i) * (db + rb * (T(3) * eb + T(4.5) * eb * eb - T(1.5) * ub2));
    A[aa_loc(geo, odd, i, x, y)] = Store<S>::st((feq_b + (f[i] - feq_n)) * p.scale);
  }
}

}  // namespace iilbm
