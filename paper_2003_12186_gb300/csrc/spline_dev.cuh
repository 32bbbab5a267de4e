// spline_dev.cuh -- the cubic-spline interface of a flexible boundary (the paper
// represents such an interface by a cubic spline for its jump conditions, end of
// section 3.2, after Lee & LeVeque).
//
// The curve is the periodic interpolating cubic spline through the markers,
// parametrised by the marker index (s = k at marker k), in uniform B-spline form
//   v(k + t) = c_{k-1} B0(t) + c_k B1(t) + c_{k+1} B2(t) + c_{k+2} B3(t),  0 <= t <= 1,
// with the interpolation conditions (c_{k-1} + 4 c_k + c_{k+1}) / 6 = v_k.  The inverse
// of that cyclic system is a two-sided geometric filter: with z = sqrt(3) - 2,
//   c_k = sum_j h_j v_{k+j},  h_j = sqrt(3) (z^|j| + z^(n-|j|)) / (1 - z^n)  (periodic),
// whose weights fall below 2^-53 beyond |j| = 28, so every coefficient is a short
// independent sum -- one thread per marker, no sequential tridiagonal solve.  The sum
// runs over differences v_{k+j} - v_k (the weights sum to 1), which keeps a coordinate
// of size 10^3 from swamping the curve's O(1) detail.
//
// The jump uses the spline's tangent for the normal and |X_s| = |X'(k)| / dX, the
// spline of the markers' Fn for the jump strength at a crossing, and the crossings of
// the curve taken on m chords per segment: the polygon of the points X(k + j/m).
#pragma once

#include "iilbm_internal.cuh"

namespace iilbm {

constexpr int SPLINE_HALF = 28;  // |j| beyond which the filter's weights are below 2^-53

// Spline coefficient c_k of the periodic sequence v[stride * k], k < n (FP64).
__device__ inline double spline_coeff(const double *__restrict__ v, int n, int stride, int k) {
  const double z = 1.7320508075688772 - 2.0;  // sqrt(3) - 2
  const double r3 = 1.7320508075688772;
  const double vk = v[stride * k];
  double acc = 0.0;
  if (n > 2 * SPLINE_HALF + 1) {
    double zj = 1.0;
    for (int j = 1; j <= SPLINE_HALF; j++) {
      zj *= z;
      const int kp = k + j >= n ? k + j - n : k + j, km = k - j < 0 ? k - j + n : k - j;
      acc += zj * ((v[stride * kp] - vk) + (v[stride * km] - vk));
    }
    return vk + r3 * acc;
  }
  // short polygons: the exact periodic weights over every offset
  double zn = 1.0;
  for (int j = 0; j < n; j++) zn *= z;
  double zj = 1.0;
  for (int j = 1; j < n; j++) {
    zj *= z;
    double znj = 1.0;  // z^(n - j)
    for (int q = 0; q < n - j; q++) znj *= z;
    const int kp = k + j >= n ? k + j - n : k + j;
    acc += (zj + znj) * (v[stride * kp] - vk);
  }
  return vk + r3 * acc / (1.0 - zn);
}

// The uniform cubic B-spline weights of v(k + t) (deriv = false) or of dv/ds.
template <typename T>
__device__ inline void bspline_weights(T t, T b[4], bool deriv = false) {
  const T u = T(1) - t;
  if (!deriv) {
    b[0] = u * u * u * T(1.0 / 6);
    b[1] = (T(3) * t * t * t - T(6) * t * t + T(4)) * T(1.0 / 6);
    b[2] = (T(-3) * t * t * t + T(3) * t * t + T(3) * t + T(1)) * T(1.0 / 6);
    b[3] = t * t * t * T(1.0 / 6);
  } else {
    b[0] = T(-0.5) * u * u;
    b[1] = T(1.5) * t * t - T(2) * t;
    b[2] = T(-1.5) * t * t + t + T(0.5);
    b[3] = T(0.5) * t * t;
  }
}

// v(k + t) (or its derivative) from coefficients c[stride * q], periodic in n.
template <typename T>
__device__ inline T spline_at(const T *__restrict__ c, int n, int stride, int k, T t,
                              bool deriv = false) {
  T b[4];
  bspline_weights<T>(t, b, deriv);
  T r = T(0);
#pragma unroll
  for (int j = 0; j < 4; j++) {
    int q = k - 1 + j;
    q = q < 0 ? q + n : (q >= n ? q - n : q);
    r += c[stride * q] * b[j];
  }
  return r;
}

}  // namespace iilbm
