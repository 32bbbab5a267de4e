// lattice3d.cu -- the three-dimensional II-LBM on the D3Q19 lattice (arXiv 2003.12186:
// the D3Q19 velocity set and weights of sections 2.1 and 2.2.1, its MRT rates of section
// 2.2.1, and the jump conditions of section 3.1, which the paper derives in three
// dimensions).  C ABI in include/iilbm3d.h.
//
// One step (the vertex pass, the cut links and the lean kernel on the lattice's stream; the
// forced kernel and the interpolation on a second stream beside the lean kernel):
//   k3_vertex        one thread per vertex: surface normal and area from the incident
//                    triangles, the Lagrangian force (prescribed or surface tension), the
//                    normal split Fn = G.n / J, the spread of the tangential part (the
//                    whole G in IB-LBM) into g, and the flags of the tiles the vertex's
//                    4 x 4 x 4 support touches (marked with the level's tag 1 + (n & 1));
//   k3_cut           one warp per triangle: every link x - e_i -> x that crosses it (exact
//                    integer predicate with symbolic tie-breaks) adds s w_i/c_s^2 Fn to the
//                    streamed population f_i(x) in place (Eq. 47);
//   k3_sc_lean       one thread per node, blocks of 32 x 4 nodes (a tile): AA-pattern
//                    in-place streaming, SRT or MRT collision, on every tile not flagged;
//   k3_sc_forced     the flagged tiles, from the list the vertex pass built: the same with
//                    g (Guo's term or the simple force term), which it clears, and the
//                    collision's velocity recorded for the interpolation; it also clears
//                    the previous level's marks;
//   k3_interp        one thread per vertex: U = interp(u) (Eq. 20), X += U for a moving
//                    surface.
// Between steps the stored populations carry no jump: the jump of the next step's
// surface is added at the start of that step.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/iilbm3d.h"

// Blocks per SM of the forced stream-collide, which runs beside the lean one: each
// forced block holds an SM's registers that lean blocks would otherwise use.
#ifndef K3_FORCED_BLOCKS_PER_SM
#define K3_FORCED_BLOCKS_PER_SM 16
#endif
// Resident blocks per SM the FP32 forced kernel is compiled for (its register budget).
#ifndef K3_FORCED_MIN_BLOCKS
#define K3_FORCED_MIN_BLOCKS 4
#endif

namespace iilbm3d {

// ---------------------------------------------------------------- D3Q19 lattice
// 0 rest; 1..6 = +x, -x, +y, -y, +z, -z; 7..18 the edge diagonals in opposite pairs.
__host__ __device__ constexpr int ex(int i) {
  return i == 1 || i == 7 || i == 9 || i == 11 || i == 13
             ? 1
             : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
  return i == 3 || i == 7 || i == 10 || i == 15 || i == 17
             ? 1
             : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18 ? -1 : 0);
}
__host__ __device__ constexpr int ez(int i) {
  return i == 5 || i == 11 || i == 14 || i == 15 || i == 18
             ? 1
             : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i & 1 ? i + 1 : i - 1); }
template <typename T>
__host__ __device__ constexpr T wt(int i) {
  return i == 0 ? T(1) / T(3) : (i <= 6 ? T(1) / T(18) : T(1) / T(36));
}
static_assert(ex(opp(7)) == -ex(7) && ey(opp(9)) == -ey(9) && ez(opp(13)) == -ez(13), "pairs");
static_assert(ex(17) == 0 && ey(17) == 1 && ez(17) == -1, "velocity 17");

// d'Humieres' D3Q19 moment basis (section 2.2.1 cites it): row r evaluated on velocity i.
__host__ __device__ constexpr int mrow(int r, int i) {
  const int x = ex(i), y = ey(i), z = ez(i), e2 = x * x + y * y + z * z;
  return r == 0    ? 1
         : r == 1  ? 19 * e2 - 30
         : r == 2  ? (21 * e2 * e2 - 53 * e2 + 24) / 2
         : r == 3  ? x
         : r == 4  ? (5 * e2 - 9) * x
         : r == 5  ? y
         : r == 6  ? (5 * e2 - 9) * y
         : r == 7  ? z
         : r == 8  ? (5 * e2 - 9) * z
         : r == 9  ? 3 * x * x - e2
         : r == 10 ? (3 * e2 - 5) * (3 * x * x - e2)
         : r == 11 ? y * y - z * z
         : r == 12 ? (3 * e2 - 5) * (y * y - z * z)
         : r == 13 ? x * y
         : r == 14 ? y * z
         : r == 15 ? x * z
         : r == 16 ? (y * y - z * z) * x
         : r == 17 ? (z * z - x * x) * y
                   : (x * x - y * y) * z;
}
__host__ __device__ constexpr int mnorm(int r) {
  int s = 0;
  for (int i = 0; i < 19; i++) s += mrow(r, i) * mrow(r, i);
  return s;
}
__host__ __device__ constexpr bool conserved(int r) { return r == 0 || r == 3 || r == 5 || r == 7; }
// Parity of a basis row under e -> -e: even rows take equal values on opposite directions,
// odd rows opposite values (every row of the basis is one or the other).
__host__ __device__ constexpr bool row_even(int r) {
  for (int i = 1; i < 19; i++)
    if (mrow(r, opp(i)) != mrow(r, i)) return false;
  return true;
}
__host__ __device__ constexpr bool row_odd(int r) {
  for (int i = 0; i < 19; i++)
    if (mrow(r, opp(i)) != -mrow(r, i)) return false;
  return true;
}
__host__ __device__ constexpr bool rows_have_parity() {
  for (int r = 0; r < 19; r++)
    if (row_even(r) == row_odd(r)) return false;
  return true;
}
static_assert(rows_have_parity(), "every basis row is even or odd");
static_assert(mnorm(0) == 19 && mnorm(1) == 2394 && mnorm(2) == 252 && mnorm(3) == 10, "norms");

// Compile-time loop: f(std::integral_constant<int, k>) for k = B .. E-1, so every basis
// entry, weight and velocity component inside is a constant expression (a constexpr
// function called with a loop counter is not guaranteed to be folded).
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// The velocity components as 2-bit fields (e + 1) of one word per axis, for directions
// that are only known at run time.
__host__ __device__ constexpr unsigned long long pack_e(int axis) {
  unsigned long long v = 0;
  for (int i = 0; i < 19; i++) {
    const int e = axis == 0 ? ex(i) : (axis == 1 ? ey(i) : ez(i));
    v |= (unsigned long long)(e + 1) << (2 * i);
  }
  return v;
}
constexpr unsigned long long EXP = pack_e(0), EYP = pack_e(1), EZP = pack_e(2);
__host__ __device__ inline int exr(int i) { return (int)((EXP >> (2 * i)) & 3ull) - 1; }
__host__ __device__ inline int eyr(int i) { return (int)((EYP >> (2 * i)) & 3ull) - 1; }
__host__ __device__ inline int ezr(int i) { return (int)((EZP >> (2 * i)) & 3ull) - 1; }

// A tile is TX x TY nodes of one z-plane: one 128-thread block of the stream-collide, one
// warp per row of 32 consecutive x (each warp access a full 128-byte line in FP32).
constexpr int TX = 32, TY = 4, TB = TX * TY;
constexpr double QS = 1048576.0;     // crossing predicate: coordinates snapped to 2^-20
constexpr int QBITS = 20;
constexpr double MAX_EDGE = 8.0;
// The candidate destinations of a triangle span ceil(max) - ceil(min) + 2 <= 10 nodes per
// axis (edges below 8 per axis); widened by one node on each side: at most 12.
constexpr int CUT_BOX = 12;
constexpr double MAX_COORD = 4096.0;
constexpr int ST_NONFINITE = 1, ST_INTERFACE = 2;
constexpr long long XQ_OUT = 1LL << 62;  // snapped coordinate of a vertex out of range

struct Geom3 {
  int nx, ny, nz, ntx, nty;  // nodes; tiles along x and y
  long long plane;  // nodes
};

__host__ __device__ inline int wrapn(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__host__ __device__ inline long long nodeix(const Geom3 &g, int x, int y, int z) {
  return ((long long)z * g.ny + y) * g.nx + x;
}
// Where the streamed population f_i of node (x, y, z) lives at the current parity of the
// AA pattern: even levels in place, odd levels in the opposite slot of the upstream node.
__device__ __forceinline__ long long aa_read(const Geom3 &g, bool odd, int i, int x, int y, int z) {
  if (!odd) return i * g.plane + nodeix(g, x, y, z);
  return opp(i) * g.plane +
         nodeix(g, wrapn(x - exr(i), g.nx), wrapn(y - eyr(i), g.ny), wrapn(z - ezr(i), g.nz));
}
// The same for a compile-time direction I (the stream-collide's unrolled loops).
template <int I>
__device__ __forceinline__ long long aa_read_c(const Geom3 &g, bool odd, int x, int y, int z) {
  constexpr int X = ex(I), Y = ey(I), Z = ez(I), O = opp(I);
  if (!odd) return I * g.plane + nodeix(g, x, y, z);
  return O * g.plane + nodeix(g, X ? wrapn(x - X, g.nx) : x, Y ? wrapn(y - Y, g.ny) : y,
                              Z ? wrapn(z - Z, g.nz) : z);
}

// The spread force g and the collision velocity u of the flagged nodes: FP32 as one float4
// per node (x, y, z, unused: one vector atomic per spread contribution, one 16-byte access
// per node), FP64 as three planes of the node count.
template <typename T>
struct Vec3;
template <>
struct Vec3<float> {
  __device__ static void add(float *b, long long, long long c, float x, float y, float z) {
    atomicAdd(reinterpret_cast<float4 *>(b) + c, make_float4(x, y, z, 0.f));
  }
  __device__ static void take(float *b, long long, long long c, float &x, float &y, float &z) {
    float4 *q = reinterpret_cast<float4 *>(b) + c;
    const float4 v = *q;
    *q = make_float4(0.f, 0.f, 0.f, 0.f);
    x = v.x;
    y = v.y;
    z = v.z;
  }
  __device__ static void put(float *b, long long, long long c, float x, float y, float z) {
    reinterpret_cast<float4 *>(b)[c] = make_float4(x, y, z, 0.f);
  }
  __device__ static void get(const float *b, long long, long long c, float &x, float &y, float &z) {
    const float4 v = reinterpret_cast<const float4 *>(b)[c];
    x = v.x;
    y = v.y;
    z = v.z;
  }
};
template <>
struct Vec3<double> {
  __device__ static void add(double *b, long long pl, long long c, double x, double y, double z) {
    atomicAdd(b + c, x);
    atomicAdd(b + pl + c, y);
    atomicAdd(b + 2 * pl + c, z);
  }
  __device__ static void take(double *b, long long pl, long long c, double &x, double &y, double &z) {
    x = b[c];
    y = b[pl + c];
    z = b[2 * pl + c];
    b[c] = b[pl + c] = b[2 * pl + c] = 0.0;
  }
  __device__ static void put(double *b, long long pl, long long c, double x, double y, double z) {
    b[c] = x;
    b[pl + c] = y;
    b[2 * pl + c] = z;
  }
  __device__ static void get(const double *b, long long pl, long long c, double &x, double &y,
                             double &z) {
    x = b[c];
    y = b[pl + c];
    z = b[2 * pl + c];
  }
};

// Storage of the populations: FP64 and FP32 as the arithmetic type, FP16 and BF16 with FP32
// arithmetic.  FP16 values are kept times 2^k (the lattice's scale; exact), so the small
// shifted deviations sit in its normal range; ld / st convert, add adds in storage units.
template <typename S>
struct St3;
template <>
struct St3<double> {
  using T = double;
  static constexpr bool SCALED = false;
  __device__ static double ld(double v) { return v; }
  __device__ static double st(double v) { return v; }
  __device__ static void add(double *a, double v) { atomicAdd(a, v); }
};
template <>
struct St3<float> {
  using T = float;
  static constexpr bool SCALED = false;
  __device__ static float ld(float v) { return v; }
  __device__ static float st(float v) { return v; }
  __device__ static void add(float *a, float v) { atomicAdd(a, v); }
};
template <>
struct St3<__half> {
  using T = float;
  static constexpr bool SCALED = true;
  __device__ static float ld(__half v) { return __half2float(v); }
  __device__ static __half st(float v) { return __float2half_rn(v); }
  __device__ static void add(__half *a, float v) { atomicAdd(a, __float2half_rn(v)); }
};
template <>
struct St3<__nv_bfloat16> {
  using T = float;
  static constexpr bool SCALED = true;
  __device__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
  __device__ static void add(__nv_bfloat16 *a, float v) { atomicAdd(a, __float2bfloat16_rn(v)); }
};

template <typename T>
struct Coll3 {
  T scale, inv_scale;  // stored value = population x scale (2^k; 1 unless 16-bit storage)
  T omega;     // SRT: 1 / lambda
  T s[19];     // MRT rates (conserved moments' unused)
  T rho0;
  T body[3];
};

// ------------------------------------------------------------------- collision
// One node's collision, shifted populations in place (the oracle's definitions):
//   rho = rho0 + sum f, j = sum e f; u = (j + g/2) / rho (Guo, Eq. 24) or j / rho (simple);
//   f_eq_i = w_i (drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2));
//   SRT: f -= omega (f - f_eq) - (1 - omega/2) Gt   (Eqs. 14, 21)
//   MRT: f -= M^-1 [S M (f - f_eq) - (I - S/2) M Gt] (Eqs. 15, 22), M^-1 = M^T / |row|^2,
//        the transforms unrolled over the constant integer basis;
//   simple force term: no Gt, then 3 w_i e_i.g added (Eq. 16).
// FORCED = false: g = 0 and the force terms are left out.
// Opposite directions pair as (2k - 1, 2k), k = 1..9.  The collision works on the pair sums
// and differences of f - f_eq (and of Guo's source): even basis rows see only the sums,
// odd rows only the differences, so the transform to moments and back takes about half
// the operations of the plain 19 x 19 products.
template <typename T, bool MRT, bool FORCED, bool SIMPLE>
__device__ __forceinline__ T collide3(T f[19], T gx, T gy, T gz, const Coll3<T> &p, T &ux,
                                      T &uy, T &uz) {
  T ps[10], pd[10];
  T drho = f[0], jx = T(0), jy = T(0), jz = T(0);
  static_for<1, 10>([&](auto kc) {
    constexpr int k = decltype(kc)::value, i = 2 * k - 1;
    ps[k] = f[i] + f[i + 1];
    pd[k] = f[i] - f[i + 1];
    drho += ps[k];
    if constexpr (ex(i) > 0) jx += pd[k];
    if constexpr (ex(i) < 0) jx -= pd[k];
    if constexpr (ey(i) > 0) jy += pd[k];
    if constexpr (ey(i) < 0) jy -= pd[k];
    if constexpr (ez(i) > 0) jz += pd[k];
    if constexpr (ez(i) < 0) jz -= pd[k];
  });
  const T rho = p.rho0 + drho, inv = T(1) / rho;
  constexpr bool GUO = FORCED && !SIMPLE;
  ux = (GUO ? jx + T(0.5) * gx : jx) * inv;
  uy = (GUO ? jy + T(0.5) * gy : jy) * inv;
  uz = (GUO ? jz + T(0.5) * gz : jz) * inv;
  const T u2 = ux * ux + uy * uy + uz * uz;
  // f_eq_i = w_i (base + rho (3 e.u + 4.5 (e.u)^2)), base = drho - 1.5 rho u^2
  const T base = drho - T(1.5) * rho * u2;
  T ds[10], da[10];  // pair sums / differences of f - f_eq; ds[0] = the rest population's
  ds[0] = f[0] - wt<T>(0) * base;
  da[0] = T(0);
  static_for<1, 10>([&](auto kc) {
    constexpr int k = decltype(kc)::value, i = 2 * k - 1;
    constexpr T w = wt<T>(i);
    const T eu = T(ex(i)) * ux + T(ey(i)) * uy + T(ez(i)) * uz;
    ds[k] = ps[k] - T(2) * w * (base + T(4.5) * rho * eu * eu);
    da[k] = pd[k] - T(6) * w * rho * eu;
  });
  T gs[10], ga[10];  // the same for Guo's source Gt_i = w_i (3 (e_i - u).g + 9 (e_i.u)(e_i.g))
  if constexpr (GUO) {
    const T ug = ux * gx + uy * gy + uz * gz;
    gs[0] = wt<T>(0) * T(-3) * ug;
    ga[0] = T(0);
    static_for<1, 10>([&](auto kc) {
      constexpr int k = decltype(kc)::value, i = 2 * k - 1;
      constexpr T w = wt<T>(i);
      const T eu = T(ex(i)) * ux + T(ey(i)) * uy + T(ez(i)) * uz;
      const T eg = T(ex(i)) * gx + T(ey(i)) * gy + T(ez(i)) * gz;
      gs[k] = w * (T(18) * eu * eg - T(6) * ug);
      ga[k] = T(6) * w * eg;
    });
  }
  if constexpr (!MRT) {
    const T om = p.omega, fo = T(1) - T(0.5) * p.omega;
    f[0] -= om * ds[0];
    if constexpr (GUO) f[0] += fo * gs[0];
    static_for<1, 10>([&](auto kc) {
      constexpr int k = decltype(kc)::value, i = 2 * k - 1;
      T e = om * ds[k], o = om * da[k];
      if constexpr (GUO) {
        e -= fo * gs[k];
        o -= fo * ga[k];
      }
      f[i] -= T(0.5) * (e + o);
      f[i + 1] -= T(0.5) * (e - o);
    });
  } else {
    T E[10], O[10];  // back-transform accumulators of the even and odd rows per pair
    static_for<0, 10>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      E[k] = T(0);
      O[k] = T(0);
    });
    static_for<0, 19>([&](auto rc) {
      constexpr int r = decltype(rc)::value;
      constexpr bool EVEN = row_even(r);
      constexpr T inv_norm = T(1) / T(mnorm(r));
      T c = T(0);
      if constexpr (!conserved(r)) {
        T a = T(0);
        static_for<0, 10>([&](auto kc) {
          constexpr int k = decltype(kc)::value, i = k == 0 ? 0 : 2 * k - 1;
          constexpr int m = mrow(r, i);
          const T v = EVEN ? ds[k] : da[k];
          if constexpr (m == 1) a += v;
          else if constexpr (m == -1) a -= v;
          else if constexpr (m != 0) a += T(m) * v;
        });
        c = p.s[r] * a;
      }
      if constexpr (GUO) {
        T b = T(0);
        static_for<0, 10>([&](auto kc) {
          constexpr int k = decltype(kc)::value, i = k == 0 ? 0 : 2 * k - 1;
          constexpr int m = mrow(r, i);
          const T v = EVEN ? gs[k] : ga[k];
          if constexpr (m == 1) b += v;
          else if constexpr (m == -1) b -= v;
          else if constexpr (m != 0) b += T(m) * v;
        });
        c -= (conserved(r) ? T(1) : T(1) - T(0.5) * p.s[r]) * b;
      }
      if constexpr (!conserved(r) || GUO) {
        c *= inv_norm;
        static_for<0, 10>([&](auto kc) {
          constexpr int k = decltype(kc)::value, i = k == 0 ? 0 : 2 * k - 1;
          constexpr int m = mrow(r, i);
          T &acc = EVEN ? E[k] : O[k];
          if constexpr (m == 1) acc += c;
          else if constexpr (m == -1) acc -= c;
          else if constexpr (m != 0) acc += T(m) * c;
        });
      }
    });
    // pair sums and differences: a pair's sum carries the even rows twice over,
    // (E + O) to its first direction and (E - O) to its second
    f[0] -= E[0];
    static_for<1, 10>([&](auto kc) {
      constexpr int k = decltype(kc)::value, i = 2 * k - 1;
      f[i] -= E[k] + O[k];
      f[i + 1] -= E[k] - O[k];
    });
  }
  if constexpr (FORCED && SIMPLE) {
    static_for<1, 10>([&](auto kc) {
      constexpr int k = decltype(kc)::value, i = 2 * k - 1;
      constexpr T w3 = T(3) * wt<T>(i);
      const T t = w3 * (T(ex(i)) * gx + T(ey(i)) * gy + T(ez(i)) * gz);
      f[i] += t;
      f[i + 1] -= t;
    });
  }
  return drho;
}

}  // namespace iilbm3d

// ---------------------------------------------------------------------- handle
struct iilbm3d_lattice {
  iilbm3d_config cfg;
  iilbm3d::Geom3 geo;
  int device;
  cudaStream_t stream;
  bool own_stream;
  bool f64;           // arithmetic FP64 (FP64 storage), else FP32
  int storage;        // IILBM_F64 / F32 / F16 / BF16
  double scale;       // stored population = df x scale (16-bit storage: 2^k; else 1)
  void *A;            // [19][plane] populations in the storage type
  void *gf;           // spread force (arithmetic type; Vec3 layout), zero outside flagged tiles
  void *uf;           // collision velocity on flagged tiles (Vec3 layout)
  unsigned *flags;    // [ntiles] tile flagged at level n iff it holds tag(n) = 1 + (n & 1)
  int *tile_list;     // [2][ntiles] the flagged tiles of the levels of each parity, in
                      // flagging order
  int *tile_count;    // [2] their numbers
  long long ntiles;
  int sms;            // the device's multiprocessors
  cudaStream_t side;  // forced stream-collide and interpolation, beside the lean kernel
  cudaEvent_t ev_fork, ev_forced, ev_join;
  int *d_status;
  int *d_count;       // cut-link crossings of the most recent surface pass
  long long step;     // time level; AA parity = step & 1
  bool prepared;      // the current level's vertex pass already ran (g, flags, Fn)
  // surface
  int n, m;
  iilbm3d_surface_params sp;
  double *X, *Gp, *G, *U, *Fn, *Aref;
  void *Fnt;          // Fn in the arithmetic type (FP32 lattices: a copy; FP64: Fn itself)
  long long *Xq;      // [n][3] vertex coordinates snapped to 2^-20 (the vertex pass)
  int *tri, *vt_start, *vt_list;  // triangles; each vertex's triangles (CSR, ascending)
  // graphs: two steps from an even level
  cudaGraphExec_t gexec;
  // timing
  bool timing;
  std::vector<cudaEvent_t> ev;
  int nev;
  double sc_ms;
  int sc_launches;
  long long kernels;
};

namespace iilbm3d {

// --------------------------------------------------------------- stream-collide
// One node: AA-pattern load of its streamed populations, collision, in-place store.
// FORCED: the spread force of the node (cleared for the next step) plus the body force;
// RECORD: the collision's velocity is kept for the interpolation.
// The AA-pattern locations of one node (ODD: the level's parity, a compile-time constant
// of the kernel): at even levels the node's own index plus i planes; at odd levels the
// opposite slot at node (x - ex, y - ey, z - ez), from the three wrapped coordinates per
// axis kept once per thread.  Node indices are below 2^31 (the lattice's limit) and are
// formed in 32 bits.
struct NodeLoc {
  int c;                    // even levels: the node's index
  int xs[3], ys[3], zs[3];  // odd levels: x - d, y - d, z - d wrapped, index d + 1
};
template <bool ODD>
__device__ __forceinline__ void node_loc(const Geom3 &g, int x, int y, int z, NodeLoc &L) {
  if constexpr (!ODD) {
    L.c = (z * g.ny + y) * g.nx + x;
  } else {
    L.xs[0] = wrapn(x + 1, g.nx), L.xs[1] = x, L.xs[2] = wrapn(x - 1, g.nx);
    L.ys[0] = wrapn(y + 1, g.ny), L.ys[1] = y, L.ys[2] = wrapn(y - 1, g.ny);
    L.zs[0] = wrapn(z + 1, g.nz), L.zs[1] = z, L.zs[2] = wrapn(z - 1, g.nz);
  }
}
// Location of the streamed f_I of the node (compile-time direction I).
template <int I, bool ODD>
__device__ __forceinline__ long long loc_of(const Geom3 &g, const NodeLoc &L) {
  if constexpr (!ODD) {
    return I * g.plane + L.c;
  } else {
    constexpr int X = ex(I), Y = ey(I), Z = ez(I);
    const int node = (L.zs[Z + 1] * g.ny + L.ys[Y + 1]) * g.nx + L.xs[X + 1];
    return opp(I) * g.plane + node;
  }
}

template <typename S, bool ODD, typename T = typename St3<S>::T>
__device__ __forceinline__ void sc_load(const S *__restrict__ A, const Geom3 &g,
                                        const NodeLoc &L, T f[19], T inv_scale) {
  static_for<0, 19>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    f[i] = St3<S>::ld(A[loc_of<i, ODD>(g, L)]);
    if constexpr (St3<S>::SCALED) f[i] *= inv_scale;
  });
}

// Collision and in-place store of one node whose streamed populations are in f.
template <typename S, bool ODD, bool MRT, bool SIMPLE, bool FORCED, bool RECORD,
          typename T = typename St3<S>::T>
__device__ __forceinline__ void sc_finish(S *__restrict__ A, const Geom3 &g, const Coll3<T> &p,
                                          const NodeLoc &L, long long c, T f[19],
                                          T *__restrict__ gf, T *__restrict__ uf,
                                          int *__restrict__ status) {
  T ux, uy, uz, drho;
  if constexpr (FORCED) {
    T gx = p.body[0], gy = p.body[1], gz = p.body[2];
    if constexpr (RECORD) {
      T sx, sy, sz;
      Vec3<T>::take(gf, g.plane, c, sx, sy, sz);
      gx += sx;
      gy += sy;
      gz += sz;
    }
    drho = collide3<T, MRT, true, SIMPLE>(f, gx, gy, gz, p, ux, uy, uz);
    if constexpr (RECORD) Vec3<T>::put(uf, g.plane, c, ux, uy, uz);
  } else {
    drho = collide3<T, MRT, false, SIMPLE>(f, T(0), T(0), T(0), p, ux, uy, uz);
  }
  if (!(fabs(drho) < T(1e30))) atomicOr(status, ST_NONFINITE);  // also NaN
  // post-collision f_i goes where the streamed f_opp(i) was read (in place)
  static_for<0, 19>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    A[loc_of<opp(i), ODD>(g, L)] = St3<S>::st(St3<S>::SCALED ? f[i] * p.scale : f[i]);
  });
}

template <typename S, bool ODD, bool MRT, bool SIMPLE, bool FORCED, bool RECORD,
          typename T = typename St3<S>::T>
__device__ __forceinline__ void sc_node(S *__restrict__ A, const Geom3 &g, const Coll3<T> &p,
                                        int x, int y, int z, T *__restrict__ gf,
                                        T *__restrict__ uf, int *__restrict__ status) {
  T f[19];
  {
    NodeLoc L;
    node_loc<ODD>(g, x, y, z, L);
    sc_load<S, ODD>(A, g, L, f, p.inv_scale);
  }
  // the stores' locations are formed again from coordinates the compiler cannot see
  // through, so it does not keep nineteen addresses live across the collision
  int xo = x, yo = y, zo = z;
  if constexpr (!RECORD) asm volatile("" : "+r"(xo), "+r"(yo), "+r"(zo));  // the lean kernel
  NodeLoc L;
  node_loc<ODD>(g, xo, yo, zo, L);
  sc_finish<S, ODD, MRT, SIMPLE, FORCED, RECORD>(A, g, p, L, nodeix(g, xo, yo, zo), f, gf, uf,
                                                 status);
}

// Tile (blockIdx.x, blockIdx.y, z) = nodes [32 blockIdx.x, +32) x [4 blockIdx.y, +4) of
// plane z.  The lean kernel updates every tile the vertex pass did not flag (with the body force alone when
// there is one); the forced kernel takes the flagged tiles from the vertex pass's list.
// AA-pattern locations belong to one node each per step, so the two kernels' node sets
// touch disjoint memory.
template <typename S, bool ODD, bool MRT, bool SIMPLE, bool BODY,
          typename T = typename St3<S>::T>
__global__ void __launch_bounds__(TB, sizeof(T) == 4 ? 8 : 4)
    k3_sc_lean(S *__restrict__ A, const Geom3 g, const Coll3<T> p,
               const unsigned *__restrict__ flags, unsigned tag, int *__restrict__ status) {
  const int x = blockIdx.x * TX + (threadIdx.x & (TX - 1));
  const int y = blockIdx.y * TY + (threadIdx.x / TX), z = blockIdx.z;
  if (flags[((long long)z * g.nty + blockIdx.y) * g.ntx + blockIdx.x] == tag) return;  // whole block
  if (x >= g.nx || y >= g.ny) return;
  sc_node<S, ODD, MRT, SIMPLE, BODY, false, T>(A, g, p, x, y, z, nullptr, nullptr, status);
}

template <typename S, bool ODD, bool MRT, bool SIMPLE, typename T = typename St3<S>::T>
__global__ void __launch_bounds__(TB, sizeof(T) == 4 ? K3_FORCED_MIN_BLOCKS : 2)
    k3_sc_forced(S *__restrict__ A, const Geom3 g, const Coll3<T> p,
                 unsigned *__restrict__ flags, const int *__restrict__ tile_list,
                 const int *__restrict__ tile_count, const int *__restrict__ prev_list,
                 const int *__restrict__ prev_count, unsigned prev_tag, T *__restrict__ gf,
                 T *__restrict__ uf, int *__restrict__ status) {
  // the previous level's marks go back to 0 (a tile flagged again holds this level's
  // tag and keeps it): the next level's vertex pass then finds only 0 or this tag
  const int pc = *prev_count;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pc; k += gridDim.x * blockDim.x)
    atomicCAS(&flags[prev_list[k]], prev_tag, 0u);
  const int cnt = *tile_count;
  for (int k = blockIdx.x; k < cnt; k += gridDim.x) {
    const int tile = tile_list[k];
    const int tx = tile % g.ntx, rest = tile / g.ntx;
    const int ty = rest % g.nty, z = rest / g.nty;
    const int x = tx * TX + (threadIdx.x & (TX - 1)), y = ty * TY + (threadIdx.x / TX);
    if (x < g.nx && y < g.ny)
      sc_node<S, ODD, MRT, SIMPLE, true, true>(A, g, p, x, y, z, gf, uf, status);
  }
}

}  // namespace iilbm3d

namespace iilbm3d {

// Peskin's four-point kernel (the delta function the paper names after Eq. 6).
template <typename T>
__device__ __forceinline__ T phi4t(T r) {
  const T a = fabs(r);
  if (a <= T(1)) return (T(3) - T(2) * a + sqrt(T(1) + T(4) * a - T(4) * a * a)) * T(0.125);
  if (a <= T(2)) return (T(5) - T(2) * a - sqrt(T(-7) + T(12) * a - T(4) * a * a)) * T(0.125);
  return T(0);
}

__device__ __forceinline__ int wrapfull(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// ------------------------------------------------------------------ vertex pass
// Vertex k: from its triangles (ascending), N_t = (B - A) x (C - A), the current area
// a_k = sum |N_t| / 6 and normal n_k = sum N_t / |sum N_t|; the force G_k (prescribed, or
// surface tension -gamma sum_t (1/2) N_t/|N_t| x (X_q - X_p) / Aref_k for t = (k, p, q));
// Fn_k = G_k.n_k / (a_k / Aref_k); the spread of P_k = (G_k - (G_k.n_k) n_k) Aref_k (II-LBM)
// or G_k Aref_k (IB-LBM) over its 4 x 4 x 4 support, and the flags of the tiles there.
template <typename T>
__global__ void __launch_bounds__(128)
    k3_vertex(const double *__restrict__ X, int n, const int *__restrict__ tri,
              const int *__restrict__ vt_start, const int *__restrict__ vt_list,
              const double *__restrict__ Aref, int model, double gamma,
              const double *__restrict__ Gp, int jump, const Geom3 g, double *__restrict__ G,
              double *__restrict__ Fn, T *__restrict__ gf, unsigned *__restrict__ flags,
              unsigned tag, int *__restrict__ tile_list, int *__restrict__ tile_count,
              T *__restrict__ Fnt,
              long long *__restrict__ Xq, int *__restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double xk = X[3 * k], yk = X[3 * k + 1], zk = X[3 * k + 2];
  if (!(fabs(xk) < MAX_COORD && fabs(yk) < MAX_COORD && fabs(zk) < MAX_COORD)) {
    atomicOr(status, ST_INTERFACE);
    Xq[3 * k] = Xq[3 * k + 1] = Xq[3 * k + 2] = XQ_OUT;  // its triangles get no cut links
    return;
  }
  // the snapped coordinates of the crossing predicate, once per vertex
  Xq[3 * k] = __double2ll_rn(xk * QS);
  Xq[3 * k + 1] = __double2ll_rn(yk * QS);
  Xq[3 * k + 2] = __double2ll_rn(zk * QS);
  // geometry in the arithmetic type from FP64 coordinate differences
  T ns[3] = {T(0), T(0), T(0)}, area = T(0), Gk[3] = {T(0), T(0), T(0)};
  const T gam = T(gamma);
  for (int q = vt_start[k]; q < vt_start[k + 1]; q++) {
    const int t = vt_list[q];
    const int v0 = tri[3 * t], v1 = tri[3 * t + 1], v2 = tri[3 * t + 2];
    const double *A = X + 3 * v0, *B = X + 3 * v1, *C = X + 3 * v2;
    const T u[3] = {T(B[0] - A[0]), T(B[1] - A[1]), T(B[2] - A[2])};
    const T v[3] = {T(C[0] - A[0]), T(C[1] - A[1]), T(C[2] - A[2])};
    const T N[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    const T l = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    area += l / T(6);
    ns[0] += N[0];
    ns[1] += N[1];
    ns[2] += N[2];
    if (model == IILBM3D_TENSION) {
      const int p = v0 == k ? v1 : (v1 == k ? v2 : v0);
      const int r = v0 == k ? v2 : (v1 == k ? v0 : v1);
      const T h[3] = {N[0] / l, N[1] / l, N[2] / l};
      const T e[3] = {T(X[3 * r] - X[3 * p]), T(X[3 * r + 1] - X[3 * p + 1]),
                      T(X[3 * r + 2] - X[3 * p + 2])};
      const T dA[3] = {T(0.5) * (h[1] * e[2] - h[2] * e[1]), T(0.5) * (h[2] * e[0] - h[0] * e[2]),
                       T(0.5) * (h[0] * e[1] - h[1] * e[0])};
      Gk[0] -= gam * dA[0];
      Gk[1] -= gam * dA[1];
      Gk[2] -= gam * dA[2];
    }
  }
  const T ln = sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
  const T nk[3] = {ns[0] / ln, ns[1] / ln, ns[2] / ln};
  const T ar = T(Aref[k]);
  if (model == IILBM3D_TENSION) {
    Gk[0] /= ar;
    Gk[1] /= ar;
    Gk[2] /= ar;
  } else {
    Gk[0] = T(Gp[3 * k]);
    Gk[1] = T(Gp[3 * k + 1]);
    Gk[2] = T(Gp[3 * k + 2]);
  }
  G[3 * k] = (double)Gk[0];
  G[3 * k + 1] = (double)Gk[1];
  G[3 * k + 2] = (double)Gk[2];
  const T gn = Gk[0] * nk[0] + Gk[1] * nk[1] + Gk[2] * nk[2];
  const T fnk = gn / (area / ar);
  Fn[k] = (double)fnk;
  Fnt[k] = fnk;
  T Pt[3];
#pragma unroll
  for (int d = 0; d < 3; d++) Pt[d] = (jump ? Gk[d] - gn * nk[d] : Gk[d]) * ar;
  const int bx = (int)floor(xk) - 1, by = (int)floor(yk) - 1, bz = (int)floor(zk) - 1;
  // kernel weights in the arithmetic type (the offsets taken in FP64 from the position)
  T wx[4], wy[4], wz[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    wx[q] = phi4t<T>(T((double)(bx + q) - xk));
    wy[q] = phi4t<T>(T((double)(by + q) - yk));
    wz[q] = phi4t<T>(T((double)(bz + q) - zk));
  }
#pragma unroll
  for (int dz = 0; dz < 4; dz++) {
    const int z = wrapfull(bz + dz, g.nz);
#pragma unroll
    for (int dy = 0; dy < 4; dy++) {
      const int y = wrapfull(by + dy, g.ny);
      int last = -1;
#pragma unroll
      for (int dx = 0; dx < 4; dx++) {
        const int x = wrapfull(bx + dx, g.nx);
        const T w = wx[dx] * wy[dy] * wz[dz];
        Vec3<T>::add(gf, g.plane, nodeix(g, x, y, z), Pt[0] * w, Pt[1] * w, Pt[2] * w);
        const int tx = x / TX;
        if (tx != last) {
          const int tile = (int)(((long long)z * g.nty + y / TY) * g.ntx + tx);
          if (atomicExch(&flags[tile], tag) != tag) tile_list[atomicAdd(tile_count, 1)] = tile;
          last = tx;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ cut links
// The exact crossing predicate (coordinates snapped to 2^-20, every lattice node displaced
// by (eps, eps^2, eps^3), eps -> 0+):
//  - plane side of node X: the sign of the first non-zero of (N.(X - A), N_x, N_y, N_z),
//    N = (B - A) x (C - A);
//  - side of the displaced link line P + t d about the edge U -> V: the sign of the first
//    non-zero of (det[d, U - P, V - P], d x (V - U)).
// The link crosses the triangle iff its ends lie on opposite sides of the plane and the
// line on the same side of all three edges; its sign s is the plane side of the
// destination.  In coordinates relative to a corner O of the triangle's candidate box,
// (U - P) x (V - P) = U' x V' + (V - U) x P', so with P' = 2^20 p (p a small integer
// vector) det = d.(U' x V') + 2^20 p.(d x (V - U)): per edge one cross product per
// triangle and a few small multiply-adds per link.
struct CutEdge {
  long long K[3];  // U' x V' (below 2^51)
  int D[3];        // V - U (below 2^23 per axis)
};

// Side of the link (direction d, source offset p from O) about edge e; det receives the
// undisplaced determinant (for the barycentric coordinates).
__device__ __forceinline__ int cut_edge_side(const CutEdge &e, int dx, int dy, int dz, int px,
                                             int py, int pz, long long &det) {
  const int c0 = dy * e.D[2] - dz * e.D[1];  // d x (V - U), below 2^24
  const int c1 = dz * e.D[0] - dx * e.D[2];
  const int c2 = dx * e.D[1] - dy * e.D[0];
  // p (below 12 per axis) . (d x (V - U)): below 2^30
  const long long o = (dx * e.K[0] + dy * e.K[1] + dz * e.K[2]) +
                      ((long long)(px * c0 + py * c1 + pz * c2) << QBITS);
  det = o;
  if (o != 0) return o > 0 ? 1 : -1;
  if (c0 != 0) return c0 > 0 ? 1 : -1;
  if (c1 != 0) return c1 > 0 ? 1 : -1;
  if (c2 != 0) return c2 > 0 ? 1 : -1;
  return 0;
}

// One warp per triangle.  The candidate destinations x span [ceil(min) - 1, ceil(max)] per
// axis (the displaced link spans at most [x - 1 + eps, x + 1 + eps]); the warp tabulates
// the plane side of every node of that box widened by one node (every source lies there,
// N.(X - A) affine in the node's offset), then, a pass of 32 destinations at a time,
// marks the directions whose link ends straddle the plane, gathers those (node,
// direction) candidates into a list, and tests them with all 32 lanes.  A crossing adds
// coef = s w_i / c_s^2 Fn(crossing), Fn the barycentric mean of the vertices' Fn, to the
// streamed population in place (INPLACE; times the storage scale) or to the field
// J[i-1][node] (read-outs).  S is the storage type, T the arithmetic type.
constexpr int CUT_LIST = 32 * 18;  // candidates of one pass at most
template <bool INPLACE, typename S, typename T = typename St3<S>::T>
__global__ void __launch_bounds__(128, 5)
    k3_cut(const long long *__restrict__ Xq, const int *__restrict__ tri, int m,
           const T *__restrict__ Fn, const Geom3 g, int odd, S *__restrict__ A, T scale,
           double *__restrict__ J, int *__restrict__ count, int *__restrict__ status) {
  // per warp: the plane sides of the widened box (the per-axis edge bound below keeps it
  // within CUT_BOX^3 nodes) and the pass's candidate list
  __shared__ signed char cut_sides[4][CUT_BOX * CUT_BOX * CUT_BOX];
  __shared__ unsigned cut_list[4][CUT_LIST];
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int wslot = threadIdx.x >> 5;
  if (t >= m) return;
  const int vi[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  long long q[3][3];
  bool ok = true;
  const long long qmax = (long long)(MAX_COORD * QS);
#pragma unroll
  for (int j = 0; j < 3; j++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      q[j][a] = Xq[3 * vi[j] + a];
      ok = ok && q[j][a] < qmax && -q[j][a] < qmax;
    }
  const long long lim = (long long)(MAX_EDGE * QS);
#pragma unroll
  for (int j = 0; j < 3; j++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const long long d = q[(j + 1) % 3][a] - q[j][a];
      ok = ok && d < lim && -d < lim;
    }
  if (!ok) {
    if (lane == 0) atomicOr(status, ST_INTERFACE);
    return;
  }
  int lo[3], ext[3], bmn[3], bmx[3];
  const long long Sx = 1LL << QBITS;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const long long mn = min(q[0][a], min(q[1][a], q[2][a]));
    const long long mx = max(q[0][a], max(q[1][a], q[2][a]));
    lo[a] = (int)(-((-mn) >> QBITS)) - 1;
    ext[a] = (int)(-((-mx) >> QBITS)) - lo[a] + 1;
    // the triangle's bounding box relative to O = (lo - 1) 2^20 (below 2^24)
    bmn[a] = (int)(mn - (long long)(lo[a] - 1) * Sx);
    bmx[a] = (int)(mx - (long long)(lo[a] - 1) * Sx);
  }
  // vertices relative to the widened box's corner O = (lo - 1) 2^20
  long long r[3][3];
#pragma unroll
  for (int j = 0; j < 3; j++)
#pragma unroll
    for (int a = 0; a < 3; a++) r[j][a] = q[j][a] - (long long)(lo[a] - 1) * Sx;
  const long long u[3] = {r[1][0] - r[0][0], r[1][1] - r[0][1], r[1][2] - r[0][2]};
  const long long v[3] = {r[2][0] - r[0][0], r[2][1] - r[0][1], r[2][2] - r[0][2]};
  const long long N[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                          u[0] * v[1] - u[1] * v[0]};
  CutEdge E[3];
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const long long *U = r[j], *V = r[(j + 1) % 3];
    E[j].K[0] = U[1] * V[2] - U[2] * V[1];
    E[j].K[1] = U[2] * V[0] - U[0] * V[2];
    E[j].K[2] = U[0] * V[1] - U[1] * V[0];
    E[j].D[0] = (int)(V[0] - U[0]);
    E[j].D[1] = (int)(V[1] - U[1]);
    E[j].D[2] = (int)(V[2] - U[2]);
  }
  // plane sides: N.(X - A) at X = O + 2^20 (a, b, c) is r0 + 2^20 (a N_x + b N_y + c N_z)
  const int tie = N[0] ? (N[0] > 0 ? 1 : -1) : (N[1] ? (N[1] > 0 ? 1 : -1) : (N[2] > 0 ? 1 : -1));
  const int E0 = ext[0] + 2, E1 = ext[1] + 2, E2 = ext[2] + 2;
  signed char *side = cut_sides[wslot];
  unsigned *list = cut_list[wslot];
  // r0 = 2^20 q + m with q = floor(r0 / 2^20), 0 <= m < 2^20 (|r0| < 2^73, |q| < 2^53), so
  // r0 + 2^20 L = 2^20 (q + L) + m has the sign of q + L, or of m where q + L = 0: one
  // 128-bit product per triangle, 64-bit sums per node (|L| < 2^53)
  const __int128 r0 = -((__int128)N[0] * r[0][0] + (__int128)N[1] * r[0][1] + (__int128)N[2] * r[0][2]);
  const long long q0 = (long long)(r0 >> QBITS);
  const bool m_pos = ((unsigned long long)r0 & ((1ull << QBITS) - 1ull)) != 0ull;
  // box index -> (a, b, c) by FP32 quotients: (k + 1/2) / E is at least 1/(2E) from an
  // integer (E <= 12, k < 1728), far beyond the quotient's rounding error
  const float iE0 = 1.0f / (float)E0, iE01 = 1.0f / (float)(E0 * E1);
  for (int c = lane; c < E0 * E1 * E2; c += 32) {
    const int cz = (int)(((float)c + 0.5f) * iE01), rem = c - cz * E0 * E1;
    const int b = (int)(((float)rem + 0.5f) * iE0), a = rem - b * E0;
    const long long t = q0 + (a * N[0] + b * N[1] + cz * N[2]);
    side[c] = (signed char)(t > 0 ? 1 : (t < 0 ? -1 : (m_pos ? 1 : tie)));
  }
  __syncwarp();
  int found = 0;
  const int nn = ext[0] * ext[1] * ext[2];
  const float iX = 1.0f / (float)ext[0], iXY = 1.0f / (float)(ext[0] * ext[1]);
  for (int base0 = 0; base0 < nn; base0 += 32) {
    // the destinations of this pass: one per lane, its straddling directions as a mask
    const int cidx = base0 + lane;
    unsigned mask = 0u;
    int a = 0, b = 0, cz = 0;
    if (cidx < nn) {
      cz = (int)(((float)cidx + 0.5f) * iXY);
      const int rem = cidx - cz * ext[0] * ext[1];
      b = (int)(((float)rem + 0.5f) * iX);
      a = rem - b * ext[0];
      a++, b++, cz++;  // offsets in the widened box
      const int base = a + E0 * (b + E1 * cz);
      const int sQ = side[base];
      // A link that crosses the triangle meets its bounding box.  The displaced link
      // from s to d spans [min + eps, max + eps] per axis, which meets [mn, mx] iff
      // 2^20 min < mx and 2^20 max >= mn; okX[e + 1]: that test for the component e.
      const int o[3] = {a, b, cz};
      bool ok[3][3];
#pragma unroll
      for (int ax = 0; ax < 3; ax++) {
        const int P = o[ax] << QBITS;
        const bool lt = P < bmx[ax], ge = P >= bmn[ax];
        ok[ax][0] = lt && (P + (1 << QBITS)) >= bmn[ax];  // e = -1: source at d + 1
        ok[ax][1] = lt && ge;                              // e = 0
        ok[ax][2] = (P - (1 << QBITS)) < bmx[ax] && ge;    // e = +1: source at d - 1
      }
      static_for<1, 19>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const int off = ex(i) + E0 * (ey(i) + E1 * ez(i));
        if (ok[0][ex(i) + 1] && ok[1][ey(i) + 1] && ok[2][ez(i) + 1] && side[base - off] != sQ)
          mask |= 1u << i;
      });
    }
    // gather: (a, b, c, i) packed, each lane's candidates at its prefix position
    const int cnt = __popc(mask);
    int pre = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int vv = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += vv;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    int slot = pre - cnt;
    while (mask) {
      const int i = __ffs(mask) - 1;
      mask &= mask - 1u;
      list[slot++] = (unsigned)i | ((unsigned)a << 5) | ((unsigned)b << 9) | ((unsigned)cz << 13);
    }
    __syncwarp();
    for (int j = lane; j < total; j += 32) {
      const unsigned e = list[j];
      const int i = (int)(e & 31u), qa = (int)((e >> 5) & 15u), qb = (int)((e >> 9) & 15u);
      const int qc = (int)((e >> 13) & 15u);
      const int dx = exr(i), dy = eyr(i), dz = ezr(i);
      const int px = qa - dx, py = qb - dy, pz = qc - dz;  // the link's source, from O
      long long vAB, vBC, vCA;
      const int e1 = cut_edge_side(E[0], dx, dy, dz, px, py, pz, vAB);
      const int e2 = cut_edge_side(E[1], dx, dy, dz, px, py, pz, vBC);
      const int e3 = cut_edge_side(E[2], dx, dy, dz, px, py, pz, vCA);
      if (e1 == 0 || e1 != e2 || e2 != e3) continue;
      const int sQ = side[qa + E0 * (qb + E1 * qc)];
      // Fn at the crossing: the barycentric mean of the vertices' Fn (one division), in the
      // arithmetic type (GB300's FP64 pipe would make this the kernel's cost in FP32 runs)
      const T sum = T(vAB) + T(vBC) + T(vCA);
      const T fc = (T(vBC) * Fn[vi[0]] + T(vCA) * Fn[vi[1]] + T(vAB) * Fn[vi[2]]) / sum;
      const T coef = T(sQ) * (T(3) * wt<T>(i)) * fc;
      const int x = lo[0] - 1 + qa, y = lo[1] - 1 + qb, z = lo[2] - 1 + qc;
      const int xw = (unsigned)x < (unsigned)g.nx ? x : wrapfull(x, g.nx);
      const int yw = (unsigned)y < (unsigned)g.ny ? y : wrapfull(y, g.ny);
      const int zw = (unsigned)z < (unsigned)g.nz ? z : wrapfull(z, g.nz);
      if constexpr (INPLACE)
        St3<S>::add(&A[aa_read(g, odd != 0, i, xw, yw, zw)], St3<S>::SCALED ? coef * scale : coef);
      else
        atomicAdd(&J[(long long)(i - 1) * g.plane + nodeix(g, xw, yw, zw)], (double)coef);
      found++;
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
  if (lane == 0 && found) atomicAdd(count, found);
}

// ------------------------------------------------------------------ interpolation
// U_k = sum over the 4 x 4 x 4 support of u(x) phi phi phi (Eq. 20), u the collision's
// velocity recorded by the flagged tiles; X_k += U_k for a moving surface.
template <typename T>
__global__ void __launch_bounds__(128)
    k3_interp(const T *__restrict__ uf, const Geom3 g, double *__restrict__ X, int n,
              double *__restrict__ U, int moves) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double xk = X[3 * k], yk = X[3 * k + 1], zk = X[3 * k + 2];
  if (!(fabs(xk) < MAX_COORD && fabs(yk) < MAX_COORD && fabs(zk) < MAX_COORD)) return;
  const int bx = (int)floor(xk) - 1, by = (int)floor(yk) - 1, bz = (int)floor(zk) - 1;
  T wx[4], wy[4], wz[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    wx[q] = phi4t<T>(T((double)(bx + q) - xk));
    wy[q] = phi4t<T>(T((double)(by + q) - yk));
    wz[q] = phi4t<T>(T((double)(bz + q) - zk));
  }
  T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
  for (int dz = 0; dz < 4; dz++) {
    const int z = wrapfull(bz + dz, g.nz);
#pragma unroll
    for (int dy = 0; dy < 4; dy++) {
      const int y = wrapfull(by + dy, g.ny);
#pragma unroll
      for (int dx = 0; dx < 4; dx++) {
        T u0, u1, u2;
        Vec3<T>::get(uf, g.plane, nodeix(g, wrapfull(bx + dx, g.nx), y, z), u0, u1, u2);
        const T w = wx[dx] * wy[dy] * wz[dz];
        s0 += u0 * w;
        s1 += u1 * w;
        s2 += u2 * w;
      }
    }
  }
  U[3 * k] = (double)s0;
  U[3 * k + 1] = (double)s1;
  U[3 * k + 2] = (double)s2;
  if (moves) {
    X[3 * k] = xk + (double)s0;
    X[3 * k + 1] = yk + (double)s1;
    X[3 * k + 2] = zk + (double)s2;
  }
}

// ------------------------------------------------------------- conversions, read-out
// FP64 natural layout df[i][node] <-> the stored populations at the current AA parity
// (stored = df x scale, rounded once to the storage type).
template <typename S>
__device__ __forceinline__ S to_store(double v, double scale) {
  return St3<S>::st((typename St3<S>::T)(v * scale));
}
template <typename S>
__device__ __forceinline__ double from_store(S v, double inv_scale) {
  return (double)St3<S>::ld(v) * inv_scale;
}
template <typename S>
__global__ void k3_store(S *__restrict__ A, const double *__restrict__ df, const Geom3 g, int odd,
                         double scale) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.plane) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  for (int i = 0; i < 19; i++)
    A[aa_read(g, odd != 0, i, x, y, z)] = to_store<S>(df[i * g.plane + c], scale);
}
template <typename S>
__global__ void k3_load(const S *__restrict__ A, double *__restrict__ df, const Geom3 g, int odd,
                        double inv_scale) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.plane) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  for (int i = 0; i < 19; i++)
    df[i * g.plane + c] = from_store<S>(A[aa_read(g, odd != 0, i, x, y, z)], inv_scale);
}
// drho and u (Eq. 24) from the stored populations plus the jump field J (may be null) and
// the spread force plus the body force; h = 1/2 (Guo) or 0 (simple force term).
template <typename S, typename T = typename St3<S>::T>
__global__ void k3_macros(const S *__restrict__ A, double inv_scale, const double *__restrict__ J,
                          const T *__restrict__ gf, const Geom3 g, int odd, double rho0,
                          double bx, double by, double bz, double h, double *__restrict__ out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.plane) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  double s = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < 19; i++) {
    double f = from_store<S>(A[aa_read(g, odd != 0, i, x, y, z)], inv_scale);
    if (J && i > 0) f += J[(long long)(i - 1) * g.plane + c];
    s += f;
    jx += ex(i) * f;
    jy += ey(i) * f;
    jz += ez(i) * f;
  }
  T sx, sy, sz;
  Vec3<T>::get(gf, g.plane, c, sx, sy, sz);
  const double gx = bx + (double)sx, gy = by + (double)sy, gz = bz + (double)sz;
  out[c] = s;
  out[g.plane + c] = (jx + h * gx) / (rho0 + s);
  out[2 * g.plane + c] = (jy + h * gy) / (rho0 + s);
  out[3 * g.plane + c] = (jz + h * gz) / (rho0 + s);
}

}  // namespace iilbm3d

namespace iilbm3d {

template <typename S>
__global__ void k3_equilibrium(S *__restrict__ A, const Geom3 g, int odd, double rho0, double scale,
                               const double *__restrict__ drho, const double *__restrict__ ux,
                               const double *__restrict__ uy, const double *__restrict__ uz) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.plane) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  const double d = drho ? drho[c] : 0.0, u0 = ux ? ux[c] : 0.0, u1 = uy ? uy[c] : 0.0,
               u2 = uz ? uz[c] : 0.0;
  const double rho = rho0 + d, uu = u0 * u0 + u1 * u1 + u2 * u2;
  for (int i = 0; i < 19; i++) {
    const double eu = ex(i) * u0 + ey(i) * u1 + ez(i) * u2;
    const double poly = eu * 3.0 + eu * eu * 4.5 - uu * 1.5;
    A[aa_read(g, odd != 0, i, x, y, z)] = to_store<S>(wt<double>(i) * (d + rho * poly), scale);
  }
}

}  // namespace iilbm3d

// ------------------------------------------------------------------------ host
namespace {
using namespace iilbm3d;
using H = iilbm3d_lattice;

#define CK3(call)                        \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) {             \
      cudaGetLastError();                \
      return IILBM_ERR_CUDA;             \
    }                                    \
  } while (0)
#define RC3(expr)          \
  do {                     \
    int r_ = (expr);       \
    if (r_) return r_;     \
  } while (0)

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
Coll3<T> coll_params(const H *h) {
  Coll3<T> p;
  p.scale = T(h->scale);
  p.inv_scale = T(1.0 / h->scale);
  p.omega = T(1.0 / h->cfg.tau);
  for (int r = 0; r < 19; r++) p.s[r] = T(h->cfg.s[r]);
  p.rho0 = T(h->cfg.rho0);
  for (int d = 0; d < 3; d++) p.body[d] = T(h->cfg.body[d]);
  return p;
}

// f(S{}) with S the lattice's storage type.
template <typename F>
void with_storage(const H *h, F &&f) {
  switch (h->storage) {
    case IILBM_F64: f(double{}); break;
    case IILBM_F32: f(float{}); break;
    case IILBM_F16: f(__half{}); break;
    default: f(__nv_bfloat16{}); break;
  }
}

bool has_body(const H *h) { return h->cfg.body[0] != 0.0 || h->cfg.body[1] != 0.0 || h->cfg.body[2] != 0.0; }

// Tag of the flagged tiles of level n (flags hold 0, or the tag of the level that marked
// them, cleared one level later).
unsigned level_tag(long long n) { return 1u + (unsigned)(n & 1); }

// The lean stream-collide on stream s (every tile without this level's tag); forced: the
// flagged tiles instead, on its own stream, with the previous level's marks cleared.
template <typename S, bool ODD, bool MRT, bool SIMPLE>
void launch_sc_p(H *h, cudaStream_t s, bool forced) {
  using T = typename St3<S>::T;
  const Geom3 &g = h->geo;
  const Coll3<T> p = coll_params<T>(h);
  const int b = (int)(h->step & 1);
  if (!forced) {
    const dim3 grid(g.ntx, g.nty, g.nz);
    const unsigned tag = level_tag(h->step);
    if (has_body(h))
      k3_sc_lean<S, ODD, MRT, SIMPLE, true><<<grid, TB, 0, s>>>((S *)h->A, g, p, h->flags, tag,
                                                                h->d_status);
    else
      k3_sc_lean<S, ODD, MRT, SIMPLE, false><<<grid, TB, 0, s>>>((S *)h->A, g, p, h->flags, tag,
                                                                 h->d_status);
  } else {
    const unsigned blocks =
        (unsigned)std::min<long long>(h->ntiles, (long long)h->sms * K3_FORCED_BLOCKS_PER_SM);
    k3_sc_forced<S, ODD, MRT, SIMPLE><<<blocks, TB, 0, s>>>(
        (S *)h->A, g, p, h->flags, h->tile_list + b * h->ntiles, h->tile_count + b,
        h->tile_list + (b ^ 1) * h->ntiles, h->tile_count + (b ^ 1), level_tag(h->step + 1),
        (T *)h->gf, (T *)h->uf, h->d_status);
  }
}

template <typename S, bool MRT, bool SIMPLE>
void launch_sc_t(H *h, cudaStream_t s, bool forced) {
  if (h->step & 1) launch_sc_p<S, true, MRT, SIMPLE>(h, s, forced);
  else launch_sc_p<S, false, MRT, SIMPLE>(h, s, forced);
}

template <typename S>
void launch_sc_s(H *h, cudaStream_t s, bool forced) {
  const bool mrt = h->cfg.collision == IILBM_MRT, simple = h->cfg.force == IILBM_FORCE_SIMPLE;
  if (mrt && simple) launch_sc_t<S, true, true>(h, s, forced);
  else if (mrt) launch_sc_t<S, true, false>(h, s, forced);
  else if (simple) launch_sc_t<S, false, true>(h, s, forced);
  else launch_sc_t<S, false, false>(h, s, forced);
}

void launch_sc(H *h, cudaStream_t s, bool forced) {
  with_storage(h, [&](auto tag) { launch_sc_s<decltype(tag)>(h, s, forced); });
}

void launch_vertex(H *h) {
  const Geom3 &g = h->geo;
  const unsigned b = blocks_for(h->n, 128);
  const int par = (int)(h->step & 1);
  int *list = h->tile_list + par * h->ntiles, *count = h->tile_count + par;
  const unsigned tag = level_tag(h->step);
  cudaMemsetAsync(count, 0, sizeof(int), h->stream);
  if (h->f64)
    k3_vertex<double><<<b, 128, 0, h->stream>>>(h->X, h->n, h->tri, h->vt_start, h->vt_list, h->Aref,
                                                h->sp.model, h->sp.gamma, h->Gp, h->cfg.jump, g,
                                                h->G, h->Fn, (double *)h->gf, h->flags, tag,
                                                list, count, h->Fn, h->Xq, h->d_status);
  else
    k3_vertex<float><<<b, 128, 0, h->stream>>>(h->X, h->n, h->tri, h->vt_start, h->vt_list, h->Aref,
                                               h->sp.model, h->sp.gamma, h->Gp, h->cfg.jump, g,
                                               h->G, h->Fn, (float *)h->gf, h->flags, tag,
                                               list, count, (float *)h->Fnt, h->Xq, h->d_status);
}

// the jump of the current level: in place into the populations (J null) or into J
void launch_cut(H *h, double *J) {
  const unsigned b = blocks_for((long long)h->m * 32, 128);
  const int odd = (int)(h->step & 1);
  if (J) {
    // read-out: the field only (the populations are not touched)
    if (h->f64)
      k3_cut<false, double><<<b, 128, 0, h->stream>>>(h->Xq, h->tri, h->m, (double *)h->Fnt, h->geo,
                                                      odd, nullptr, 1.0, J, h->d_count, h->d_status);
    else
      k3_cut<false, float><<<b, 128, 0, h->stream>>>(h->Xq, h->tri, h->m, (float *)h->Fnt, h->geo,
                                                     odd, nullptr, 1.0f, J, h->d_count, h->d_status);
    return;
  }
  with_storage(h, [&](auto tag) {
    using S = decltype(tag);
    using T = typename St3<S>::T;
    k3_cut<true, S><<<b, 128, 0, h->stream>>>(h->Xq, h->tri, h->m, (const T *)h->Fnt, h->geo, odd,
                                             (S *)h->A, T(h->scale), nullptr, h->d_count,
                                             h->d_status);
  });
}

void launch_interp(H *h, cudaStream_t s) {
  const unsigned b = blocks_for(h->n, 128);
  if (h->f64)
    k3_interp<double><<<b, 128, 0, s>>>((const double *)h->uf, h->geo, h->X, h->n, h->U,
                                        h->sp.moves);
  else
    k3_interp<float><<<b, 128, 0, s>>>((const float *)h->uf, h->geo, h->X, h->n, h->U,
                                       h->sp.moves);
}

// One time step (see the file's head).  Main stream: vertex pass, cut links, then the lean
// stream-collide; the side stream (highest priority), forked after the cut links: the
// forced stream-collide of the flagged tiles, then the interpolation and vertex update.
// The two touch disjoint tiles (a node's AA reads and writes are its own), and the main
// stream joins the side stream at the end of the step.  With timing on, an event pair
// brackets both stream-collide kernels (eager steps only).
int one_step(H *h) {
  const bool surf = h->n > 0;
  if (surf) {
    if (!h->prepared) launch_vertex(h);
    CK3(cudaMemsetAsync(h->d_count, 0, sizeof(int), h->stream));
    if (h->cfg.jump) launch_cut(h, nullptr);
  }
  if (h->timing) {
    if (2 * h->nev + 2 > (int)h->ev.size()) {
      for (int q = 0; q < 64; q++) {
        cudaEvent_t e;
        CK3(cudaEventCreate(&e));
        h->ev.push_back(e);
      }
    }
    CK3(cudaEventRecord(h->ev[2 * h->nev], h->stream));
  }
  if (surf) {
    CK3(cudaEventRecord(h->ev_fork, h->stream));
    CK3(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    launch_sc(h, h->side, true);
    if (h->timing) CK3(cudaEventRecord(h->ev_forced, h->side));
    launch_interp(h, h->side);
    CK3(cudaEventRecord(h->ev_join, h->side));
  }
  launch_sc(h, h->stream, false);
  if (h->timing) {
    if (surf) CK3(cudaStreamWaitEvent(h->stream, h->ev_forced, 0));
    CK3(cudaEventRecord(h->ev[2 * h->nev + 1], h->stream));
    h->nev++;
    h->kernels += surf ? (h->cfg.jump ? 5 : 4) - (h->prepared ? 1 : 0) : 1;
  }
  if (surf) CK3(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  CK3(cudaGetLastError());
  h->step++;
  h->prepared = false;
  return IILBM_OK;
}

void drop_graph(H *h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
}

// Two steps from an even level, captured once and replayed.
int capture_pair(H *h) {
  cudaGraph_t graph = nullptr;
  CK3(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = one_step(h);
  if (!rc) rc = one_step(h);
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  h->step -= 2;  // capture only recorded the launches
  if (rc || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : IILBM_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&h->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->gexec = nullptr;
    cudaGetLastError();
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

int read_status3(H *h) {
  int st = 0;
  CK3(cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaStreamSynchronize(h->stream));
  if (st & ST_NONFINITE) return IILBM_ERR_NONFINITE;
  if (st & ST_INTERFACE) return IILBM_ERR_INTERFACE;
  return IILBM_OK;
}

void free_surface(H *h) {
  if (h->Fnt && h->Fnt != (void *)h->Fn) cudaFree(h->Fnt);
  h->Fnt = nullptr;
  if (h->Xq) cudaFree(h->Xq);
  h->Xq = nullptr;
  void *p[] = {h->X, h->Gp, h->G, h->U, h->Fn, h->Aref, h->tri, h->vt_start, h->vt_list};
  for (void *q : p)
    if (q) cudaFree(q);
  h->X = h->Gp = h->G = h->U = h->Fn = h->Aref = nullptr;
  h->tri = h->vt_start = h->vt_list = nullptr;
  h->n = h->m = 0;
}

// FP64 [count] from host or device memory into a fresh device buffer (caller frees).
int to_device(const double *src, size_t count, cudaStream_t s, double **out) {
  *out = nullptr;
  if (!src) return IILBM_OK;
  if (cudaMalloc(out, count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return IILBM_ERR_OOM;
  }
  if (cudaMemcpyAsync(*out, src, count * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(*out);
    *out = nullptr;
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

}  // namespace

extern "C" {

int iilbm3d_create(iilbm3d_t *out, const iilbm3d_config *cfg) {
  if (!out || !cfg) return IILBM_ERR_INVALID_ARG;
  *out = nullptr;
  const iilbm3d_config &c = *cfg;
  const int lim[3] = {c.nx, c.ny, c.nz};
  for (int a = 0; a < 3; a++)
    if (lim[a] < 4 || lim[a] > 2048) return IILBM_ERR_INVALID_ARG;
  if ((long long)c.nx * c.ny * c.nz >= (1LL << 31)) return IILBM_ERR_INVALID_ARG;
  if (c.collision != IILBM_SRT && c.collision != IILBM_MRT) return IILBM_ERR_INVALID_ARG;
  if (c.storage < IILBM_F64 || c.storage > IILBM_BF16) return IILBM_ERR_INVALID_ARG;
  const bool half = c.storage == IILBM_F16 || c.storage == IILBM_BF16;
  if (half ? (c.storage_scale_log2 < -24 || c.storage_scale_log2 > 24) : c.storage_scale_log2 != 0)
    return IILBM_ERR_INVALID_ARG;
  if ((c.jump != 0 && c.jump != 1) || (c.force != IILBM_FORCE_GUO && c.force != IILBM_FORCE_SIMPLE))
    return IILBM_ERR_INVALID_ARG;
  if (!(c.tau > 0.5 && c.tau < 1e6) || !(c.rho0 > 0.0 && std::isfinite(c.rho0)))
    return IILBM_ERR_INVALID_ARG;
  for (int d = 0; d < 3; d++)
    if (!std::isfinite(c.body[d])) return IILBM_ERR_INVALID_ARG;
  if (c.collision == IILBM_MRT)
    for (int r = 0; r < 19; r++)
      if (!conserved(r) && !(c.s[r] > 0.0 && c.s[r] < 2.0)) return IILBM_ERR_INVALID_ARG;
  int ndev = 0, dev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return IILBM_ERR_NO_DEVICE;
  }
  CK3(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK3(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3) return IILBM_ERR_NO_DEVICE;
  H *h = new (std::nothrow) H();
  if (!h) return IILBM_ERR_OOM;
  h->cfg = c;
  h->device = dev;
  h->sms = prop.multiProcessorCount;
  h->f64 = c.storage == IILBM_F64;
  h->storage = c.storage;
  h->scale = std::ldexp(1.0, c.storage_scale_log2);
  Geom3 &g = h->geo;
  g.nx = c.nx;
  g.ny = c.ny;
  g.nz = c.nz;
  g.ntx = (c.nx + TX - 1) / TX;
  g.nty = (c.ny + TY - 1) / TY;
  g.plane = (long long)c.nx * c.ny * c.nz;
  const size_t sb = h->f64 ? 8 : 4;                      // arithmetic type
  const size_t sa = c.storage == IILBM_F64 ? 8 : (half ? 2 : 4);  // storage type
  const size_t ntiles = (size_t)g.ntx * g.nty * c.nz;
  h->ntiles = (long long)ntiles;
  bool ok = true;
  // the side stream at the highest priority, so the forced tiles' few blocks are
  // dispatched ahead of the lean stream-collide's backlog
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  ok = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
       cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&h->ev_forced, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess;
  if (ok && c.stream) {
    h->stream = (cudaStream_t)c.stream;
  } else if (ok) {
    ok = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) == cudaSuccess;
    h->own_stream = ok;
  }
  ok = ok && cudaMalloc(&h->A, 19 * g.plane * sa) == cudaSuccess &&
       cudaMalloc(&h->gf, 4 * g.plane * sb) == cudaSuccess &&
       cudaMalloc(&h->uf, 4 * g.plane * sb) == cudaSuccess &&
       cudaMalloc(&h->flags, ntiles * sizeof(unsigned)) == cudaSuccess &&
       cudaMalloc(&h->tile_list, 2 * ntiles * sizeof(int)) == cudaSuccess &&
       cudaMalloc(&h->tile_count, 2 * sizeof(int)) == cudaSuccess &&
       cudaMalloc(&h->d_status, sizeof(int)) == cudaSuccess &&
       cudaMalloc(&h->d_count, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMemsetAsync(h->A, 0, 19 * g.plane * sa, h->stream) == cudaSuccess &&
       cudaMemsetAsync(h->gf, 0, 4 * g.plane * sb, h->stream) == cudaSuccess &&
       cudaMemsetAsync(h->uf, 0, 4 * g.plane * sb, h->stream) == cudaSuccess &&
       cudaMemsetAsync(h->flags, 0, ntiles * sizeof(unsigned), h->stream) == cudaSuccess &&
       cudaMemsetAsync(h->tile_count, 0, 2 * sizeof(int), h->stream) == cudaSuccess &&
       cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream) == cudaSuccess &&
       cudaMemsetAsync(h->d_count, 0, sizeof(int), h->stream) == cudaSuccess &&
       cudaStreamSynchronize(h->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    iilbm3d_destroy(h);
    return IILBM_ERR_OOM;
  }
  *out = h;
  return IILBM_OK;
}

int iilbm3d_destroy(iilbm3d_t h) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  drop_graph(h);
  free_surface(h);
  void *p[] = {h->A, h->gf, h->uf, h->flags, h->tile_list, h->tile_count, h->d_status, h->d_count};
  for (void *q : p)
    if (q) cudaFree(q);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  cudaEvent_t own[] = {h->ev_fork, h->ev_forced, h->ev_join};
  for (cudaEvent_t e : own)
    if (e) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete h;
  return IILBM_OK;
}

int iilbm3d_set_surface(iilbm3d_t h, const double *X, int32_t n, const int32_t *tri, int32_t m,
                        const iilbm3d_surface_params *p, const double *G) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  if (n > 0 && (!X || !tri || !p || m < 4 || n < 4 || n > (1 << 24) || m > (1 << 25)))
    return IILBM_ERR_INVALID_ARG;
  if (n > 0 && (p->model != IILBM3D_PRESCRIBED && p->model != IILBM3D_TENSION))
    return IILBM_ERR_INVALID_ARG;
  if (n > 0 && ((p->model == IILBM3D_PRESCRIBED && !G) || (p->moves != 0 && p->moves != 1) ||
                !std::isfinite(p->gamma)))
    return IILBM_ERR_INVALID_ARG;
  CK3(cudaStreamSynchronize(h->stream));
  drop_graph(h);
  free_surface(h);
  // clear what a prepared level left behind
  const size_t sb = h->f64 ? 8 : 4;
  const size_t ntiles = (size_t)h->geo.ntx * h->geo.nty * h->geo.nz;
  CK3(cudaMemsetAsync(h->gf, 0, 4 * h->geo.plane * sb, h->stream));
  CK3(cudaMemsetAsync(h->flags, 0, ntiles * sizeof(unsigned), h->stream));
  CK3(cudaMemsetAsync(h->tile_count, 0, 2 * sizeof(int), h->stream));
  h->prepared = false;
  if (n == 0) return IILBM_OK;
  std::vector<double> hx(3 * (size_t)n), hg;
  std::vector<int> ht(3 * (size_t)m);
  CK3(cudaMemcpy(hx.data(), X, hx.size() * sizeof(double), cudaMemcpyDefault));
  CK3(cudaMemcpy(ht.data(), tri, ht.size() * sizeof(int), cudaMemcpyDefault));
  if (p->model == IILBM3D_PRESCRIBED) {
    hg.resize(3 * (size_t)n);
    CK3(cudaMemcpy(hg.data(), G, hg.size() * sizeof(double), cudaMemcpyDefault));
  }
  for (double v : hx)
    if (!(std::fabs(v) < MAX_COORD)) return IILBM_ERR_INTERFACE;
  // reference vertex areas (a third of each triangle's), triangles per vertex (ascending)
  std::vector<double> aref(n, 0.0);
  std::vector<int> cnt(n + 1, 0);
  for (int t = 0; t < m; t++) {
    const int v[3] = {ht[3 * t], ht[3 * t + 1], ht[3 * t + 2]};
    for (int j = 0; j < 3; j++)
      if (v[j] < 0 || v[j] >= n) return IILBM_ERR_INVALID_ARG;
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return IILBM_ERR_INTERFACE;
    const double *A = &hx[3 * v[0]], *B = &hx[3 * v[1]], *C = &hx[3 * v[2]];
    const double *E[3][2] = {{A, B}, {B, C}, {C, A}};
    for (int j = 0; j < 3; j++) {
      double l2 = 0;
      for (int a = 0; a < 3; a++) l2 += (E[j][1][a] - E[j][0][a]) * (E[j][1][a] - E[j][0][a]);
      if (!(l2 < MAX_EDGE * MAX_EDGE) || l2 == 0.0) return IILBM_ERR_INTERFACE;
    }
    const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    const double N[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    const double a = std::sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]) / 6.0;
    if (!(a > 0.0)) return IILBM_ERR_INTERFACE;
    for (int j = 0; j < 3; j++) {
      aref[v[j]] += a;
      cnt[v[j] + 1]++;
    }
  }
  for (int k = 0; k < n; k++) {
    if (cnt[k + 1] == 0) return IILBM_ERR_INTERFACE;  // a vertex on no triangle
    cnt[k + 1] += cnt[k];
  }
  std::vector<int> fill(cnt.begin(), cnt.end() - 1), list(3 * (size_t)m);
  for (int t = 0; t < m; t++)
    for (int j = 0; j < 3; j++) list[fill[ht[3 * t + j]]++] = t;
  const size_t b3 = 3 * (size_t)n * sizeof(double);
  bool ok = cudaMalloc(&h->X, b3) == cudaSuccess && cudaMalloc(&h->Gp, b3) == cudaSuccess &&
            cudaMalloc(&h->G, b3) == cudaSuccess && cudaMalloc(&h->U, b3) == cudaSuccess &&
            cudaMalloc(&h->Fn, n * sizeof(double)) == cudaSuccess &&
            (h->f64 || cudaMalloc(&h->Fnt, n * sizeof(float)) == cudaSuccess) &&
            cudaMalloc(&h->Xq, 3 * (size_t)n * sizeof(long long)) == cudaSuccess &&
            cudaMalloc(&h->Aref, n * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&h->tri, 3 * (size_t)m * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->vt_start, (n + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&h->vt_list, 3 * (size_t)m * sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_surface(h);
    return IILBM_ERR_OOM;
  }
  if (h->f64) h->Fnt = h->Fn;
  h->n = n;
  h->m = m;
  h->sp = *p;
  ok = cudaMemcpy(h->X, hx.data(), b3, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(h->Gp, 0, b3) == cudaSuccess && cudaMemset(h->G, 0, b3) == cudaSuccess &&
       cudaMemset(h->U, 0, b3) == cudaSuccess &&
       cudaMemset(h->Fn, 0, n * sizeof(double)) == cudaSuccess &&
       cudaMemcpy(h->Aref, aref.data(), n * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->tri, ht.data(), ht.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->vt_start, cnt.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(h->vt_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  if (ok && !hg.empty()) ok = cudaMemcpy(h->Gp, hg.data(), b3, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_surface(h);
    return IILBM_ERR_CUDA;
  }
  return IILBM_OK;
}

int iilbm3d_init_equilibrium(iilbm3d_t h, const double *drho, const double *ux, const double *uy,
                             const double *uz) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  const long long N = h->geo.plane;
  double *d[4] = {nullptr, nullptr, nullptr, nullptr};
  const double *src[4] = {drho, ux, uy, uz};
  int rc = IILBM_OK;
  for (int q = 0; q < 4 && !rc; q++) rc = to_device(src[q], (size_t)N, h->stream, &d[q]);
  if (!rc) {
    const unsigned b = blocks_for(N, 256);
    with_storage(h, [&](auto tag) {
      using S = decltype(tag);
      k3_equilibrium<S><<<b, 256, 0, h->stream>>>((S *)h->A, h->geo, (int)(h->step & 1), h->cfg.rho0,
                                                   h->scale, d[0], d[1], d[2], d[3]);
    });
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IILBM_ERR_CUDA;
  }
  for (double *q : d)
    if (q) cudaFree(q);
  // the vertex pass of the level (g, flags, G, Fn) depends on the surface only: a pass
  // that already ran stays valid (running it again would spread g twice)
  return rc;
}

int iilbm3d_set_populations(iilbm3d_t h, const double *df) {
  if (!h || !df) return IILBM_ERR_INVALID_ARG;
  double *d = nullptr;
  int rc = to_device(df, 19 * (size_t)h->geo.plane, h->stream, &d);
  if (rc) return rc;
  const unsigned b = blocks_for(h->geo.plane, 256);
  with_storage(h, [&](auto tag) {
    using S = decltype(tag);
    k3_store<S><<<b, 256, 0, h->stream>>>((S *)h->A, d, h->geo, (int)(h->step & 1), h->scale);
  });
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IILBM_ERR_CUDA;
  cudaFree(d);
  return rc;
}

int iilbm3d_get_populations(iilbm3d_t h, double *df) {
  if (!h || !df) return IILBM_ERR_INVALID_ARG;
  double *d = nullptr;
  const size_t cnt = 19 * (size_t)h->geo.plane;
  if (cudaMalloc(&d, cnt * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_OOM;
  }
  const unsigned b = blocks_for(h->geo.plane, 256);
  with_storage(h, [&](auto tag) {
    using S = decltype(tag);
    k3_load<S><<<b, 256, 0, h->stream>>>((const S *)h->A, d, h->geo, (int)(h->step & 1),
                                         1.0 / h->scale);
  });
  int rc = IILBM_OK;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(df, d, cnt * sizeof(double), cudaMemcpyDefault, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    rc = IILBM_ERR_CUDA;
  }
  cudaFree(d);
  return rc ? rc : read_status3(h);
}

int iilbm3d_step(iilbm3d_t h, int32_t n) {
  if (!h || n < 0) return IILBM_ERR_INVALID_ARG;
  while (n > 0) {
    const bool graph_ok = !h->timing && !h->prepared && (h->step & 1) == 0 && n >= 2;
    if (graph_ok) {
      if (!h->gexec) RC3(capture_pair(h));
      CK3(cudaGraphLaunch(h->gexec, h->stream));
      h->step += 2;
      n -= 2;
    } else {
      RC3(one_step(h));
      n -= 1;
    }
  }
  return IILBM_OK;
}

// The vertex pass of the current level, once (its g and flags then await the step).
static int prepare_level(H *h) {
  if (h->n > 0 && !h->prepared) {
    launch_vertex(h);
    CK3(cudaGetLastError());
    h->prepared = true;
  }
  return IILBM_OK;
}

// The jump field of the current level into the device buffer J (zeroed here).
static int jump_field(H *h, double *J) {
  CK3(cudaMemsetAsync(J, 0, 18 * (size_t)h->geo.plane * sizeof(double), h->stream));
  if (h->n > 0 && h->cfg.jump) {
    RC3(prepare_level(h));
    CK3(cudaMemsetAsync(h->d_count, 0, sizeof(int), h->stream));
    launch_cut(h, J);
    CK3(cudaGetLastError());
  }
  return IILBM_OK;
}

int iilbm3d_get_macros(iilbm3d_t h, double *drho, double *ux, double *uy, double *uz) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  const size_t N = (size_t)h->geo.plane;
  double *J = nullptr, *out = nullptr;
  const bool want_j = h->n > 0 && h->cfg.jump;
  if ((want_j && cudaMalloc(&J, 18 * N * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&out, 4 * N * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (J) cudaFree(J);
    return IILBM_ERR_OOM;
  }
  int rc = want_j ? jump_field(h, J) : prepare_level(h);
  if (!rc) {
    const double hh = h->cfg.force == IILBM_FORCE_SIMPLE ? 0.0 : 0.5;
    const unsigned b = blocks_for((long long)N, 256);
    with_storage(h, [&](auto tag) {
      using S = decltype(tag);
      using T = typename St3<S>::T;
      k3_macros<S><<<b, 256, 0, h->stream>>>((const S *)h->A, 1.0 / h->scale, J, (const T *)h->gf,
                                             h->geo, (int)(h->step & 1), h->cfg.rho0, h->cfg.body[0],
                                             h->cfg.body[1], h->cfg.body[2], hh, out);
    });
    double *dst[4] = {drho, ux, uy, uz};
    if (cudaGetLastError() != cudaSuccess) rc = IILBM_ERR_CUDA;
    for (int q = 0; q < 4 && !rc; q++)
      if (dst[q] &&
          cudaMemcpyAsync(dst[q], out + q * N, N * sizeof(double), cudaMemcpyDefault, h->stream) != cudaSuccess)
        rc = IILBM_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = IILBM_ERR_CUDA;
  }
  cudaGetLastError();
  if (J) cudaFree(J);
  cudaFree(out);
  return rc ? rc : read_status3(h);
}

int iilbm3d_get_markers(iilbm3d_t h, double *X, double *G, double *U, double *Fn) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  const size_t b3 = 3 * (size_t)h->n * sizeof(double);
  if (h->n > 0) {
    if (X) CK3(cudaMemcpyAsync(X, h->X, b3, cudaMemcpyDefault, h->stream));
    if (G) CK3(cudaMemcpyAsync(G, h->G, b3, cudaMemcpyDefault, h->stream));
    if (U) CK3(cudaMemcpyAsync(U, h->U, b3, cudaMemcpyDefault, h->stream));
    if (Fn) CK3(cudaMemcpyAsync(Fn, h->Fn, h->n * sizeof(double), cudaMemcpyDefault, h->stream));
  }
  return read_status3(h);
}

int iilbm3d_get_jump(iilbm3d_t h, double *J) {
  if (!h || !J) return IILBM_ERR_INVALID_ARG;
  const size_t cnt = 18 * (size_t)h->geo.plane;
  double *d = nullptr;
  if (cudaMalloc(&d, cnt * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return IILBM_ERR_OOM;
  }
  int rc = jump_field(h, d);
  if (!rc && (cudaMemcpyAsync(J, d, cnt * sizeof(double), cudaMemcpyDefault, h->stream) != cudaSuccess ||
              cudaStreamSynchronize(h->stream) != cudaSuccess))
    rc = IILBM_ERR_CUDA;
  cudaGetLastError();
  cudaFree(d);
  return rc ? rc : read_status3(h);
}

int iilbm3d_get_cut_link_count(iilbm3d_t h, int32_t *count) {
  if (!h || !count) return IILBM_ERR_INVALID_ARG;
  int c = 0;
  CK3(cudaMemcpyAsync(&c, h->d_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK3(cudaStreamSynchronize(h->stream));
  *count = c;
  return IILBM_OK;
}

int iilbm3d_set_timing(iilbm3d_t h, int32_t enable) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  CK3(cudaStreamSynchronize(h->stream));
  h->timing = enable != 0;
  h->nev = 0;
  h->sc_ms = 0.0;
  h->sc_launches = 0;
  h->kernels = 0;
  return IILBM_OK;
}

int iilbm3d_get_timing(iilbm3d_t h, double *stream_collide_ms, int32_t *launches, int64_t *kernels) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  CK3(cudaStreamSynchronize(h->stream));
  for (int e = 0; e < h->nev; e++) {
    float ms = 0.f;
    CK3(cudaEventElapsedTime(&ms, h->ev[2 * e], h->ev[2 * e + 1]));
    h->sc_ms += ms;
  }
  h->sc_launches += h->nev;
  h->nev = 0;
  if (stream_collide_ms) *stream_collide_ms = h->sc_ms;
  if (launches) *launches = h->sc_launches;
  if (kernels) *kernels = h->kernels;
  return IILBM_OK;
}

int iilbm3d_synchronize(iilbm3d_t h) {
  if (!h) return IILBM_ERR_INVALID_ARG;
  return read_status3(h);
}

}  // extern "C"
