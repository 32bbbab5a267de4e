// forcing_dev.cuh -- device body of the direct-forcing iteration (see forcing.cu),
// shared by the single-lattice and the batched launch.
#pragma once

#include "iilbm_internal.cuh"
#include "interface_dev.cuh"
#include "mlp_dev.cuh"

#include <cmath>

namespace iilbm {

// Where the force iteration starts (G^(0)).
enum { WS_GIVEN = 0, WS_PREVIOUS = 1, WS_MLP = 2 };

// A cut link of a fixed body's polygon: the link x - e_i -> x crosses segment
// k -> k+1 at parameter t (in the arithmetic type's precision, as the interface phase
// computes it) with sign s; its destination x is band node b.  The body does not move,
// so the records are found once, when the interface is set.
struct DfLink {
  double t;
  int b, k;
  int i, s;
};

struct DfArgs {
  const double *X, *UD, *G0;
  double *G, *U;
  double *Ustar;  // out: U*_k, the interpolated velocity without immersed-boundary force
  int *iters;
  double *res;
  int n;
  double eta, dX, tol;
  int max_iters;
  // the band: every node a marker stencil or a cut link touches, as sorted keys
  // y * nx + x; st[16 k + l] is the band index of stencil node l of marker k (-1 off
  // the lattice); links[nl] the cut links (nl = 0 in IB-LBM)
  const int *band;
  int nb;
  const int *st;
  const DfLink *links;
  int nl;
  // a moving (rigid) body: the band and the cut links are rebuilt in the CTA from the
  // current markers every call, into shared memory of these capacities (words of the
  // bitmap of the body's window, band nodes, cut links); ig is the interface's geometry
  int moving;
  int words_max, nb_max, nl_max;
  Geom ig;
  int *status;
  int jump;               // II-LBM: the normal part acts through the jump
  double bodyx, bodyy, rho0;
  int ws_mode;            // WS_GIVEN: G0; WS_PREVIOUS: the G of the last iteration (in G);
                          // WS_MLP: the network's proposal from the step's features
  const float *mlp_P;     // WS_MLP: packed parameters (W1..W3 transposed), normalisation,
                          // Re feature
  const float *mlp_norm;
  float re;
};

constexpr int DF_THREADS = 1024;

// Shared memory of the force iteration on a band of nb nodes with n markers: per band
// node rho*, j* (3 values) and three correction sets (density, momentum: 3 values
// each), the stencil of every marker (16 n weights and band indices), and the marker
// arrays G, U, U^D, G of the pass start, U*, normals (2 n values each) and Fn (n).
// With the network's proposal (mlp), the per-marker feature blocks, two activation
// buffers and the transposed hidden-layer weights follow.
template <typename T>
__host__ __device__ inline size_t df_smem_bytes(int nb, int n, bool mlp = false) {
  size_t b = 12 * (size_t)nb * sizeof(T);
  b += 16 * (size_t)n * (sizeof(T) + sizeof(int));
  b = (b + 15) & ~(size_t)15;
  b += 13 * (size_t)n * sizeof(T);
  b = (b + 15) & ~(size_t)15;
  if (mlp) b += ((size_t)n * (MLP_BLOCK + 2 * MLP_H) + (MLP_IN + 2 * MLP_H) * MLP_H) * sizeof(float);
  return b + 16;
}

// What a moving body adds: the window's bitmap and its word prefix sums, each band
// node's window position, and the cut-link records (after the rest, 16-byte aligned).
__host__ __device__ inline size_t df_move_bytes(int words, int nb, int nl) {
  size_t b = (2 * (size_t)words + (size_t)nb) * sizeof(int);
  b = (b + 15) & ~(size_t)15;
  return b + (size_t)nl * sizeof(DfLink) + 16;
}

// Bit pattern of a non-negative value of T; such patterns order as the values do, so
// the residual's maximum is taken with integer maxima.
template <typename T> struct BitsOf;
template <> struct BitsOf<float> {
  using U = unsigned;
  __device__ static U of(float v) { return __float_as_uint(v); }
  __device__ static float val(U b) { return __uint_as_float(b); }
};
template <> struct BitsOf<double> {
  using U = unsigned long long;
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
  __device__ static double val(U b) { return __longlong_as_double((long long)b); }
};

// The jump of one cut link for the jump strengths FnA, FnB at the segment's ends (the
// interface phase's arithmetic, segment_links).
template <typename T>
__device__ __forceinline__ T df_link_coef(const DfLink &L, T FnA, T FnB) {
  if (sizeof(T) == 8)
    return T((double)L.s * 3.0 * wt<double>(L.i) * ((1.0 - L.t) * (double)FnA + L.t * (double)FnB));
  const float t = (float)L.t;
  return T((float)L.s * 3.0f * wt<float>(L.i) * ((1.0f - t) * (float)FnA + t * (float)FnB));
}

// Is node (x, y) (unwrapped) on the lattice, as the interface sees it?
__device__ inline bool df_on_lattice(const DfArgs &a, int x, int y) {
  const bool px = a.ig.bc != IILBM_BC_CHANNEL, py = a.ig.bc == IILBM_BC_PERIODIC;
  return (px || (x >= 0 && x < a.ig.nx)) && (py || (y >= 0 && y < a.ig.ny));
}

// Band index of node (x, y) of a moving body's window (-1 off the lattice, outside the
// window or unmarked), from the bitmap and its word prefix sums.
__device__ inline int df_window_index(const DfArgs &a, const unsigned *bits, const int *wpre,
                                      const int *mv, int x, int y) {
  const int lx = x - mv[0], ly = y - mv[1];
  if (!df_on_lattice(a, x, y) || lx < 0 || ly < 0 || lx >= mv[2] || ly >= mv[3]) return -1;
  const int p = ly * mv[2] + lx, w = p >> 5, b = p & 31;
  const unsigned word = bits[w];
  if (!(word >> b & 1u)) return -1;
  return wpre[w] + __popc(word & ((1u << b) - 1u));
}

// A moving body's band, built by the whole CTA from the current markers: the window
// [floor(min X) - 3, floor(max X) + 4] on each axis; a bitmap of the window's nodes that a
// marker stencil or a cut link of the current polygon can touch; the band index of each
// as the number of marked nodes before it (word popcounts, prefix-summed); each band
// node's window position; and the cut links found by the interface phase's crossing
// enumeration, one warp per segment.  Returns false (uniformly) if a capacity is
// exceeded.  mv: window x0, y0, width, height, band nodes, cut links, failed flag.
template <typename T>
__device__ bool df_build_band(const DfArgs &a, unsigned *bits, int *wpre, int *bpos,
                              DfLink *slinks, int *mv) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n = a.n;
  __shared__ double ext[4][DF_THREADS / 32];
  double lx = 1e300, hx = -1e300, ly = 1e300, hy = -1e300;
  int bad = 0;  // a marker that is not finite, is outside the coordinate range, or whose
                // segment is too long: no band (the status reports it)
  for (int k = tid; k < n; k += DF_THREADS) {
    const int kp = k + 1 == n ? 0 : k + 1;
    const double x = a.X[2 * k], y = a.X[2 * k + 1];
    const double ex = a.X[2 * kp] - x, ey = a.X[2 * kp + 1] - y;
    bad |= !(fabs(x) <= MAX_COORD && fabs(y) <= MAX_COORD &&
             ex * ex + ey * ey < MAX_SEGMENT * MAX_SEGMENT);
    lx = fmin(lx, x);
    hx = fmax(hx, x);
    ly = fmin(ly, y);
    hy = fmax(hy, y);
  }
  if (__syncthreads_or(bad)) return false;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lx = fmin(lx, __shfl_xor_sync(0xffffffffu, lx, o));
    hx = fmax(hx, __shfl_xor_sync(0xffffffffu, hx, o));
    ly = fmin(ly, __shfl_xor_sync(0xffffffffu, ly, o));
    hy = fmax(hy, __shfl_xor_sync(0xffffffffu, hy, o));
  }
  if (lane == 0) {
    ext[0][warp] = lx;
    ext[1][warp] = hx;
    ext[2][warp] = ly;
    ext[3][warp] = hy;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < DF_THREADS / 32; w++) {
      lx = fmin(lx, ext[0][w]);
      hx = fmax(hx, ext[1][w]);
      ly = fmin(ly, ext[2][w]);
      hy = fmax(hy, ext[3][w]);
    }
    mv[0] = (int)floor(lx) - 3;
    mv[1] = (int)floor(ly) - 3;
    mv[2] = (int)floor(hx) + 4 - mv[0] + 1;
    mv[3] = (int)floor(hy) + 4 - mv[1] + 1;
    mv[5] = 0;
    // the window must fit its bitmap, and on a periodic axis be narrower than the lattice
    // (two window positions would be one node)
    const bool px = a.ig.bc != IILBM_BC_CHANNEL, py = a.ig.bc == IILBM_BC_PERIODIC;
    mv[6] = (mv[2] * mv[3] + 31) / 32 > a.words_max || (px && mv[2] > a.ig.nx) ||
            (py && mv[3] > a.ig.ny);
  }
  __syncthreads();
  if (mv[6]) return false;
  const int words = (mv[2] * mv[3] + 31) / 32;
  for (int w = tid; w < words; w += DF_THREADS) bits[w] = 0u;
  __syncthreads();
  auto mark = [&](int x, int y) {
    if (!df_on_lattice(a, x, y)) return;
    const int wx = x - mv[0], wy = y - mv[1];
    if (wx < 0 || wy < 0 || wx >= mv[2] || wy >= mv[3]) {  // cannot happen: the window
      mv[6] = 1;                                            // covers every marked node
      return;
    }
    const int p = wy * mv[2] + wx;
    atomicOr(&bits[p >> 5], 1u << (p & 31));
  };
  for (int k = tid; k < n; k += DF_THREADS) {  // stencils
    const int bx = (int)floor(a.X[2 * k]) - 1, by = (int)floor(a.X[2 * k + 1]) - 1;
    for (int l = 0; l < 16; l++) mark(bx + (l & 3), by + (l >> 2));
  }
  if (a.jump)
    for (int k = tid; k < n; k += DF_THREADS) {  // the destinations a cut link can reach
      const int kp = k + 1 == n ? 0 : k + 1;
      const long long ax = __double2ll_rn(a.X[2 * k] * QSCALE), ay = __double2ll_rn(a.X[2 * k + 1] * QSCALE);
      const long long bx = __double2ll_rn(a.X[2 * kp] * QSCALE), by = __double2ll_rn(a.X[2 * kp + 1] * QSCALE);
      auto qceil = [](long long v) { return (int)-((-v) >> 24); };
      const int x0 = qceil(min(ax, bx)) - 1, x1 = qceil(max(ax, bx));
      const int y0 = qceil(min(ay, by)) - 1, y1 = qceil(max(ay, by));
      for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) mark(x, y);
    }
  __syncthreads();
  if (mv[6]) return false;
  if (warp == 0) {  // word prefix sums of the bitmap
    int base = 0;
    for (int w0 = 0; w0 < words; w0 += 32) {
      const int w = w0 + lane;
      const int c = w < words ? __popc(bits[w]) : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (w < words) wpre[w] = base + incl - c;
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      mv[4] = base;
      mv[6] = base > a.nb_max;
    }
  }
  __syncthreads();
  if (mv[6]) return false;
  for (int w = tid; w < words; w += DF_THREADS) {
    unsigned word = bits[w];
    int p = wpre[w];
    while (word) {
      const int b = __ffs(word) - 1;
      bpos[p++] = w * 32 + b;
      word &= word - 1u;
    }
  }
  if (a.jump)
    for (int k = warp; k < n; k += DF_THREADS / 32) {  // cut links, a warp per segment
      const int kp = k + 1 == n ? 0 : k + 1;
      const long long ax = __double2ll_rn(a.X[2 * k] * QSCALE), ay = __double2ll_rn(a.X[2 * k + 1] * QSCALE);
      const long long bx = __double2ll_rn(a.X[2 * kp] * QSCALE), by = __double2ll_rn(a.X[2 * kp + 1] * QSCALE);
      segment_crossings<T>(ax, ay, bx, by, lane, a.ig, [&](int i, int dx, int dy, int s1, T t) {
        // back to the window's (unwrapped) coordinates
        int x = dx, y = dy;
        if (a.ig.bc != IILBM_BC_CHANNEL) {
          if (x - mv[0] >= a.ig.nx) x -= a.ig.nx;
          if (x < mv[0]) x += a.ig.nx;
        }
        if (a.ig.bc == IILBM_BC_PERIODIC) {
          if (y - mv[1] >= a.ig.ny) y -= a.ig.ny;
          if (y < mv[1]) y += a.ig.ny;
        }
        const int b = df_window_index(a, bits, wpre, mv, x, y);
        const int slot = atomicAdd(&mv[5], 1);
        if (b < 0 || slot >= a.nl_max) {
          mv[6] = 1;
          return;
        }
        DfLink L;
        L.t = (double)t;
        L.b = b;
        L.k = k;
        L.i = i;
        L.s = s1;
        slinks[slot] = L;
      });
    }
  __syncthreads();
  return !mv[6];
}

// The whole force iteration of one body by one CTA of DF_THREADS threads; smem_raw is
// the CTA's dynamic shared memory (df_smem_bytes<T>(nb, n)).
//
// The iteration (Eq. 18 repeated) sees G through the operator the step applies it
// with: a pass forms the step's forcing of the current G -- in II-LBM the jump of its
// normal part Fn_k = G_k . n_k on the cut links (Eq. 47 with Eq. 32), which changes the
// density and momentum of the links' destinations, and the spread of its tangential
// part (Eq. 46); in IB-LBM the spread of the whole G (Eq. 17) -- and interpolates the
// velocity the collision will then use, u = (j* + dj + g/2) / (rho* + drho) (Eqs. 24,
// 20), with j* = sum_i e_i f~_i + body/2 and rho* from the streamed state f~.  Then
// G += eta (U^D - U).
//
// The markers do not move, so each marker's 4 x 4 stencil (band indices and weights
// phi(x - X) phi(y - Y), from the FP64 position) is formed once per call.  Everything
// runs in the arithmetic type T (FP64 for FP64 storage; FP32 otherwise, where GB300's
// FP64 pipe would cost a whole warp's time even for the few lanes that hold a marker).
// A pass: the 16 lanes of a marker interpolate from the current correction set; after
// the xor butterfly each holds the same U_k, so they update G_k and spread its new
// (tangential) part into the next set at once, and the marker's first lane records U_k,
// the residual |U^D - U_k| and the new Fn_k; the set after next is cleared meanwhile.
// Barrier; a pass whose residual (taken before its update) is below the tolerance puts
// the G it started from back and ends the iteration (the result of checking before
// updating); otherwise the cut links add the new jump to the next set, and a second
// barrier (none without cut links) completes it.  U* (the interpolation with G = 0)
// is recorded for the learned warm start.
template <typename S>
__device__ __forceinline__ void direct_forcing_cta(const S *__restrict__ A, const Geom &geo,
                                                   bool odd, const DfArgs &a, double inv_scale,
                                                   unsigned char *smem_raw) {
  using T = typename Store<S>::T;
  using B = typename BitsOf<T>::U;
  const int NB = a.moving ? a.nb_max : a.nb;  // stride of the band's arrays
  const int n = a.n;
  T *rs = reinterpret_cast<T *>(smem_raw);  // rho* = rho0 + drho*
  T *jsx = rs + NB;                         // j* (with body / 2)
  T *jsy = jsx + NB;
  T *cset = jsy + NB;  // three correction sets of 3 NB values: drho, djx + gx/2, djy + gy/2
  T *pw = cset + 9 * NB;                            // stencil weights [16 n]
  int *pc = reinterpret_cast<int *>(pw + 16 * n);   // stencil band indices [16 n]
  size_t off = (size_t)(reinterpret_cast<unsigned char *>(pc + 16 * n) - smem_raw);
  off = (off + 15) & ~(size_t)15;
  T *Gk = reinterpret_cast<T *>(smem_raw + off);    // [2 n] each
  T *Uk = Gk + 2 * n;
  T *UDk = Uk + 2 * n;
  T *Gp = UDk + 2 * n;                              // G at the start of the pass
  T *Us = Gp + 2 * n;                               // U*
  T *nrm = Us + 2 * n;                              // outward unit normals
  T *Fnk = nrm + 2 * n;                             // [n] jump strengths of the new G
  size_t off2 = (size_t)(reinterpret_cast<unsigned char *>(Fnk + n) - smem_raw);
  off2 = (off2 + 15) & ~(size_t)15;
  // WS_MLP scratch: the transposed weights first (16-byte aligned for 16-byte loads),
  // then the per-marker feature blocks and two activation buffers
  float *wt1 = reinterpret_cast<float *>(smem_raw + off2);
  float *wt2 = wt1 + MLP_IN * MLP_H;
  float *wt3 = wt2 + MLP_H * MLP_H;
  float *blk = wt3 + MLP_H * MLP_H;
  float *act0 = blk + MLP_BLOCK * n;
  float *act1 = act0 + MLP_H * n;
  // a moving body's band, built below (after the network's scratch when it is used)
  size_t off3 = off2;
  if (a.ws_mode == WS_MLP)
    off3 += ((size_t)n * (MLP_BLOCK + 2 * MLP_H) + (MLP_IN + 2 * MLP_H) * MLP_H) * sizeof(float);
  off3 = (off3 + 15) & ~(size_t)15;
  unsigned *bits = reinterpret_cast<unsigned *>(smem_raw + off3);  // window bitmap
  int *wpre = reinterpret_cast<int *>(bits + a.words_max);           // band nodes before word
  int *bpos = wpre + a.words_max;                                    // window position
  size_t off4 = (size_t)(reinterpret_cast<unsigned char *>(bpos + a.nb_max) - smem_raw);
  off4 = (off4 + 15) & ~(size_t)15;
  DfLink *slinks = reinterpret_cast<DfLink *>(smem_raw + off4);
  __shared__ int mv[8];  // window x0, y0, width, height; band nodes; cut links; failed
  __shared__ B red[2][DF_THREADS / 32];
  __shared__ T cst[6];  // 2^-k, rho0, body force, eta, dX: converted once, by one thread
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    cst[0] = T(inv_scale);
    cst[1] = T(a.rho0);
    cst[2] = T(a.bodyx);
    cst[3] = T(a.bodyy);
    cst[4] = T(a.eta);
    cst[5] = T(a.dX);
  }
  __syncthreads();
  const T is = cst[0], rho0 = cst[1], bodyx = cst[2], bodyy = cst[3], eta = cst[4], dX = cst[5];

  if (a.moving && !df_build_band<T>(a, bits, wpre, bpos, slinks, mv)) {
    if (tid == 0) atomicOr(a.status, ST_CAPACITY);
    return;  // uniform: the band or its cut links exceed the capacities
  }
  const int nb = a.moving ? mv[4] : a.nb;
  const int nl = a.moving ? mv[5] : a.nl;
  const DfLink *links = a.moving ? slinks : a.links;
  // lattice node of band node c
  auto band_node = [&](int c, int &x, int &y) {
    if (a.moving) {
      const int pos = bpos[c], ly = pos / mv[2];
      x = mv[0] + pos - ly * mv[2];
      y = mv[1] + ly;
      if (a.ig.bc != IILBM_BC_CHANNEL) x = wrap(x, geo.nx);
      if (a.ig.bc == IILBM_BC_PERIODIC) y = wrap(y, geo.ny);
    } else {
      const int key = a.band[c];
      y = key / geo.nx;
      x = key - y * geo.nx;
    }
  };

  // rho*, j* on the band (every band node lies on the lattice); corrections cleared
  for (int c = tid; c < nb; c += DF_THREADS) {
    int x, y;
    band_node(c, x, y);
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = Store<S>::ld(A[aa_loc(geo, odd, i, x, y)]) * is;
    const T d = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    rs[c] = rho0 + d;
    jsx[c] = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]) + T(0.5) * bodyx;
    jsy[c] = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]) + T(0.5) * bodyy;
#pragma unroll
    for (int q = 0; q < 9; q++) cset[q * NB + c] = T(0);
  }
  // stencils, one thread per marker (an entry off the lattice gets weight 0)
  for (int k = tid; k < n; k += DF_THREADS) {
    const double Xk = a.X[2 * k], Yk = a.X[2 * k + 1];
    const int bx = (int)floor(Xk) - 1, by = (int)floor(Yk) - 1;
    T wx[4], wy[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      wx[q] = phi4<T>(T((double)(bx + q) - Xk));
      wy[q] = phi4<T>(T((double)(by + q) - Yk));
    }
#pragma unroll
    for (int l = 0; l < 16; l++) {
      const int b = a.moving ? df_window_index(a, bits, wpre, mv, bx + (l & 3), by + (l >> 2))
                             : a.st[16 * k + l];
      pw[16 * k + l] = b < 0 ? T(0) : wx[l & 3] * wy[l >> 2];
      pc[16 * k + l] = b < 0 ? 0 : b;
    }
    // outward normal of the counter-clockwise polygon (as the marker pass forms it)
    const int kp = k + 1 == n ? 0 : k + 1, km = k == 0 ? n - 1 : k - 1;
    const T tx = T(a.X[2 * kp] - a.X[2 * km]), ty = T(a.X[2 * kp + 1] - a.X[2 * km + 1]);
    const T tl = sqrt(tx * tx + ty * ty);
    nrm[2 * k] = ty / tl;
    nrm[2 * k + 1] = -tx / tl;
  }
  // marker arrays, one thread per component: the start of the iteration, U^D
  const double *g0 = a.ws_mode == WS_PREVIOUS ? a.G : a.G0;
  for (int k = tid; k < 2 * n; k += DF_THREADS) {
    Gk[k] = T(g0[k]);
    UDk[k] = T(a.UD[k]);
  }
  __syncthreads();

  T *cur = cset, *nxt = cset + 3 * NB, *clr = cset + 6 * NB;
  const int npairs = 16 * n;
  // u at band node c from correction set F
  auto vel = [&](const T *F, int c, T &ux, T &uy) {
    const T ir = T(1) / (rs[c] + F[c]);
    ux = (jsx[c] + F[NB + c]) * ir;
    uy = (jsy[c] + F[2 * NB + c]) * ir;
  };
  // the point force of marker k for force G (the tangential part in II-LBM), times dX/2
  auto half_point_force = [&](int k, T gx, T gy, T &px, T &py, T &fn) {
    fn = gx * nrm[2 * k] + gy * nrm[2 * k + 1];  // |X_s| = 1 for a rigid body
    if (a.jump) {
      px = (gx - fn * nrm[2 * k]) * dX * T(0.5);
      py = (gy - fn * nrm[2 * k + 1]) * dX * T(0.5);
    } else {
      px = gx * dX * T(0.5);
      py = gy * dX * T(0.5);
    }
  };
  // cut links of the current jump strengths into set F
  auto add_links = [&](T *F) {
    for (int l = tid; l < nl; l += DF_THREADS) {
      const DfLink L = links[l];
      const int kp = L.k + 1 == n ? 0 : L.k + 1;
      const T c = df_link_coef<T>(L, Fnk[L.k], Fnk[kp]);
      atomicAdd(&F[L.b], c);
      if (cx(L.i)) atomicAdd(&F[NB + L.b], T(cx(L.i)) * c);
      if (cy(L.i)) atomicAdd(&F[2 * NB + L.b], T(cy(L.i)) * c);
    }
  };

  // U* = interp(u*), 16 consecutive threads per marker
  for (int base = 0; base < npairs; base += DF_THREADS) {
    const int q = base + tid;
    T sx = T(0), sy = T(0);
    if (q < npairs) {
      T ux, uy;
      vel(cur, pc[q], ux, uy);
      sx = ux * pw[q];
      sy = uy * pw[q];
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o, 16);
      sy += __shfl_xor_sync(0xffffffffu, sy, o, 16);
    }
    if (q < npairs && (q & 15) == 0) {
      Us[2 * (q >> 4)] = sx;
      Us[2 * (q >> 4) + 1] = sy;
      Uk[2 * (q >> 4)] = sx;  // the last interpolated velocity, should no pass run
      Uk[2 * (q >> 4) + 1] = sy;
    }
  }

  if (a.ws_mode == WS_MLP) {
    // G^(0) proposed by the network from each marker's features (U* from above)
    __syncthreads();
    for (int j = tid; j < n; j += DF_THREADS)
      marker_feature_block(a.X, n, j, a.dX, (float)(UDk[2 * j] - Us[2 * j]),
                           (float)(UDk[2 * j + 1] - Us[2 * j + 1]), a.re, blk + MLP_BLOCK * j);
    __syncthreads();
    for (int k = tid; k < n; k += DF_THREADS) mlp_gather_input(blk, n, k, a.mlp_norm, act1 + MLP_IN * k);
    // mlp_P holds W1, W2, W3 already transposed to [in][64]
    mlp_copy4(a.mlp_P + OFF_W1, wt1, MLP_IN * MLP_H, tid, DF_THREADS);
    mlp_copy4(a.mlp_P + OFF_W2, wt2, MLP_H * MLP_H, tid, DF_THREADS);
    mlp_copy4(a.mlp_P + OFF_W3, wt3, MLP_H * MLP_H, tid, DF_THREADS);
    __syncthreads();
    mlp_hidden_layer_t(wt1, a.mlp_P + OFF_B1, act1, MLP_IN, act0, n, tid, DF_THREADS);
    __syncthreads();
    mlp_hidden_layer_t(wt2, a.mlp_P + OFF_B2, act0, MLP_H, act1, n, tid, DF_THREADS);
    __syncthreads();
    mlp_hidden_layer_t(wt3, a.mlp_P + OFF_B3, act1, MLP_H, act0, n, tid, DF_THREADS);
    __syncthreads();
    mlp_output_layer(a.mlp_P, act0, act1, n, tid, DF_THREADS);
    __syncthreads();
    for (int k = tid; k < 2 * n; k += DF_THREADS) {
      const int o = k & 1;
      Gk[k] = T(act1[k] * a.mlp_norm[NORM_OUT_SCALE + o] + a.mlp_norm[NORM_OUT_MEAN + o]);
    }
  }
  __syncthreads();

  // the forcing of the start G^(0) into the current set: spread, then the cut links
  for (int q = tid; q < npairs; q += DF_THREADS) {
    const int k = q >> 4;
    T px, py, fn;
    half_point_force(k, Gk[2 * k], Gk[2 * k + 1], px, py, fn);
    if ((q & 15) == 0) Fnk[k] = fn;
    const T w = pw[q];
    if (w != T(0)) {
      atomicAdd(&cur[NB + pc[q]], px * w);
      atomicAdd(&cur[2 * NB + pc[q]], py * w);
    }
  }
  __syncthreads();
  if (nl) {
    add_links(cur);
    __syncthreads();
  }

  int it = 0;
  B rm = 0;
  // stop once the residual's bit pattern is below the tolerance's (both non-negative)
  const bool stop_on_tol = a.tol > 0.0;
  const B tol_bits = BitsOf<T>::of(T(a.tol));
  for (it = 0; it < a.max_iters; it++) {
    B r = 0;
    for (int base = 0; base < npairs; base += DF_THREADS) {
      const int q = base + tid, k = q >> 4;
      T sx = T(0), sy = T(0);
      if (q < npairs) {
        T ux, uy;
        vel(cur, pc[q], ux, uy);
        sx = ux * pw[q];
        sy = uy * pw[q];
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o, 16);
        sy += __shfl_xor_sync(0xffffffffu, sy, o, 16);
      }
      T gxo = T(0), gyo = T(0), nx = T(0), ny = T(0);
      if (q < npairs) {
        gxo = Gk[2 * k];
        gyo = Gk[2 * k + 1];
        nx = gxo + eta * (UDk[2 * k] - sx);
        ny = gyo + eta * (UDk[2 * k + 1] - sy);
      }
      __syncwarp();  // every lane of the marker has read the old G
      if (q < npairs) {
        T px, py, fn;
        half_point_force(k, nx, ny, px, py, fn);
        if ((q & 15) == 0) {
          Uk[2 * k] = sx;
          Uk[2 * k + 1] = sy;
          r = max(r, max(BitsOf<T>::of(fabs(UDk[2 * k] - sx)),
                         BitsOf<T>::of(fabs(UDk[2 * k + 1] - sy))));
          Gp[2 * k] = gxo;
          Gp[2 * k + 1] = gyo;
          Gk[2 * k] = nx;
          Gk[2 * k + 1] = ny;
          Fnk[k] = fn;
        }
        const T w = pw[q];
        if (w != T(0)) {
          atomicAdd(&nxt[NB + pc[q]], px * w);
          atomicAdd(&nxt[2 * NB + pc[q]], py * w);
        }
      }
    }
    for (int c = tid; c < 3 * NB; c += DF_THREADS) clr[c] = T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = max(r, (B)__shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) red[it & 1][tid >> 5] = r;  // two sets: a warp may run a pass ahead
    __syncthreads();
    rm = lane < DF_THREADS / 32 ? red[it & 1][lane] : B(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rm = max(rm, (B)__shfl_xor_sync(0xffffffffu, rm, o));
    if (stop_on_tol && rm < tol_bits) {  // uniform
      for (int k = tid; k < 2 * n; k += DF_THREADS) Gk[k] = Gp[k];
      __syncthreads();
      break;
    }
    if (nl) {
      add_links(nxt);
      __syncthreads();
    }
    T *t0 = cur;  // rotate: next -> current, cleared -> next, current -> to clear
    cur = nxt;
    nxt = clr;
    clr = t0;
  }
  for (int k = tid; k < 2 * n; k += DF_THREADS) {
    a.G[k] = (double)Gk[k];
    a.U[k] = (double)Uk[k];
    a.Ustar[k] = (double)Us[k];
  }
  if (tid == 0) {
    *a.iters = it;
    *a.res = (double)BitsOf<T>::val(rm);
  }
}

// Cut-link records of segment k of a fixed body (one warp): every crossing's band
// index (binary search of the sorted band keys), direction, sign and parameter,
// appended to links[] (capacity cap; *count may exceed it, which the host reports).
template <typename T, typename GG>
__device__ __forceinline__ void df_segment_links(const double *__restrict__ X, int n, int k,
                                                 int lane, const GG &geo,
                                                 const int *__restrict__ band, int nb,
                                                 DfLink *links, int *count, int cap,
                                                 int *missing) {
  const int kp = k + 1 == n ? 0 : k + 1;
  const long long ax = __double2ll_rn(X[2 * k] * QSCALE), ay = __double2ll_rn(X[2 * k + 1] * QSCALE);
  const long long bx = __double2ll_rn(X[2 * kp] * QSCALE), by = __double2ll_rn(X[2 * kp + 1] * QSCALE);
  segment_crossings<T>(ax, ay, bx, by, lane, geo, [&](int i, int dx, int dy, int s1, T t) {
    const int key = dy * geo.nx + dx;
    int lo = 0, hi = nb - 1, b = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int v = band[mid];
      if (v == key) {
        b = mid;
        break;
      }
      if (v < key) lo = mid + 1;
      else hi = mid - 1;
    }
    if (b < 0) {
      atomicAdd(missing, 1);
      return;
    }
    const int slot = atomicAdd(count, 1);
    if (slot < cap) {
      DfLink L;
      L.t = (double)t;
      L.b = b;
      L.k = k;
      L.i = i;
      L.s = s1;
      links[slot] = L;
    }
  });
}

// Raw (unnormalised) features [n][30] of every marker from the U* of the most recent
// force iteration: one CTA, blocks in shared memory (n * 6 floats).
__device__ inline void df_features_cta(const double *__restrict__ X, const double *__restrict__ UD,
                                       const double *__restrict__ Ustar, int n, double dX,
                                       float re, float *F, float *blk) {
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    marker_feature_block(X, n, j, dX, (float)(UD[2 * j] - Ustar[2 * j]),
                         (float)(UD[2 * j + 1] - Ustar[2 * j + 1]), re, blk + MLP_BLOCK * j);
  __syncthreads();
  for (int e = threadIdx.x; e < n * MLP_IN; e += blockDim.x) {
    const int k = e / MLP_IN, i = e % MLP_IN, q = i / MLP_BLOCK, r = i % MLP_BLOCK;
    int j = k + q - 2;
    j = j < 0 ? j + n : (j >= n ? j - n : j);
    F[e] = blk[MLP_BLOCK * j + r];
  }
}

}  // namespace iilbm
