// ipm_model.cuh -- the cart with a double pendulum (textbook Lagrangian
// mechanics: point masses m1, m2 on massless links l1, l2, cart mass m0, no
// friction; angles from the upright) and its RK4 step, written once for
// plain numbers and for the forward-mode derivative numbers that give the
// Jacobians and the Hessian of the Lagrangian of the nonlinear IPM (Section
// "Applying the regularized IPM to optimal control").
//
//   M(th) qdd = tau(th, dth, u),  q = (p, th1, th2)
//   M = [[m0+m1+m2, a1 cos th1, a2 cos th2],
//        [a1 cos th1, b1,        b12 cos(th1-th2)],
//        [a2 cos th2, b12 cos(th1-th2), b2]]
//   tau = (u + a1 sin th1 dth1^2 + a2 sin th2 dth2^2,
//          a1 g sin th1 - b12 sin(th1-th2) dth2^2,
//          m2 g l2 sin th2 + b12 sin(th1-th2) dth1^2)
//   a1 = (m1+m2) l1, a2 = m2 l2, b1 = (m1+m2) l1^2, b12 = m2 l1 l2, b2 = m2 l2^2
// M^{-1} tau by the cofactors of the symmetric M.  Included by ipm.cu only.
#pragma once

#include <cuda_runtime.h>

#include "../../include/rlqr_ipm.h"

namespace rlqr {
namespace ipm {

// ---- number types
// D1: value and one directional derivative.  HD: value, derivatives along
// two directions e1, e2 and the mixed second derivative (hyper-dual).
template <class T>
struct D1 {
  T v, d;
};
template <class T>
struct HD {
  T v, a, b, ab;
};

__device__ __forceinline__ void sin_cos(double x, double &s, double &c) { sincos(x, &s, &c); }
__device__ __forceinline__ void sin_cos(float x, float &s, float &c) { sincosf(x, &s, &c); }

template <class T>
__device__ __forceinline__ D1<T> operator+(D1<T> x, D1<T> y) { return {x.v + y.v, x.d + y.d}; }
template <class T>
__device__ __forceinline__ D1<T> operator-(D1<T> x, D1<T> y) { return {x.v - y.v, x.d - y.d}; }
template <class T>
__device__ __forceinline__ D1<T> operator*(D1<T> x, D1<T> y) {
  return {x.v * y.v, x.v * y.d + x.d * y.v};
}
template <class T>
__device__ __forceinline__ D1<T> operator*(D1<T> x, T c) { return {x.v * c, x.d * c}; }
template <class T>
__device__ __forceinline__ D1<T> operator+(D1<T> x, T c) { return {x.v + c, x.d}; }
template <class T>
__device__ __forceinline__ D1<T> operator-(T c, D1<T> x) { return {c - x.v, -x.d}; }
template <class T>
__device__ __forceinline__ D1<T> reciprocal(D1<T> x) {
  const T iv = T(1) / x.v;
  return {iv, -x.d * iv * iv};
}
template <class T>
__device__ __forceinline__ void sin_cos(D1<T> x, D1<T> &s, D1<T> &c) {
  T sv, cv;
  sin_cos(x.v, sv, cv);
  s = {sv, cv * x.d};
  c = {cv, -sv * x.d};
}

template <class T>
__device__ __forceinline__ HD<T> operator+(HD<T> x, HD<T> y) {
  return {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab};
}
template <class T>
__device__ __forceinline__ HD<T> operator-(HD<T> x, HD<T> y) {
  return {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab};
}
template <class T>
__device__ __forceinline__ HD<T> operator*(HD<T> x, HD<T> y) {
  return {x.v * y.v, x.v * y.a + x.a * y.v, x.v * y.b + x.b * y.v,
          x.v * y.ab + x.a * y.b + x.b * y.a + x.ab * y.v};
}
template <class T>
__device__ __forceinline__ HD<T> operator*(HD<T> x, T c) {
  return {x.v * c, x.a * c, x.b * c, x.ab * c};
}
template <class T>
__device__ __forceinline__ HD<T> operator+(HD<T> x, T c) { return {x.v + c, x.a, x.b, x.ab}; }
template <class T>
__device__ __forceinline__ HD<T> operator-(T c, HD<T> x) { return {c - x.v, -x.a, -x.b, -x.ab}; }
template <class T>
__device__ __forceinline__ HD<T> reciprocal(HD<T> x) {
  const T iv = T(1) / x.v, iv2 = iv * iv;
  return {iv, -x.a * iv2, -x.b * iv2, (T(2) * x.a * x.b * iv - x.ab) * iv2};
}
template <class T>
__device__ __forceinline__ void sin_cos(HD<T> x, HD<T> &s, HD<T> &c) {
  T sv, cv;
  sin_cos(x.v, sv, cv);
  const T ab = x.a * x.b;
  s = {sv, cv * x.a, cv * x.b, cv * x.ab - sv * ab};
  c = {cv, -sv * x.a, -sv * x.b, -sv * x.ab - cv * ab};
}

__device__ __forceinline__ double reciprocal(double x) { return 1.0 / x; }
__device__ __forceinline__ float reciprocal(float x) { return 1.0f / x; }

// ---- model constants (derived once on the host, in the evaluation type)
template <class T>
struct CdpConst {
  T a1, a2, b1, b2, b12, mt, a1g, m2gl2, b1b2, mtb2, mtb1;
  T h, h2, h6;  // dt, dt/2, dt/6
};

template <class T>
inline CdpConst<T> cdp_const(const rlqr_cdp_model &md) {
  const double a1 = (md.m1 + md.m2) * md.l1, a2 = md.m2 * md.l2;
  const double b1 = (md.m1 + md.m2) * md.l1 * md.l1, b2 = md.m2 * md.l2 * md.l2;
  const double b12 = md.m2 * md.l1 * md.l2, mt = md.m0 + md.m1 + md.m2;
  CdpConst<T> k;
  k.a1 = T(a1);
  k.a2 = T(a2);
  k.b1 = T(b1);
  k.b2 = T(b2);
  k.b12 = T(b12);
  k.mt = T(mt);
  k.a1g = T(a1 * md.grav);
  k.m2gl2 = T(md.m2 * md.grav * md.l2);
  k.b1b2 = T(b1 * b2);
  k.mtb2 = T(mt * b2);
  k.mtb1 = T(mt * b1);
  k.h = T(md.dt);
  k.h2 = T(0.5 * md.dt);
  k.h6 = T(md.dt / 6.0);
  return k;
}

// The sines and cosines of one right-hand side (of th1, th2, th1 - th2):
// computed (TrigCompute), computed and recorded as plain doubles
// (TrigRecord), or replayed from a record with the derivative parts formed
// from the caller's numbers (TrigReplay) -- the value path of every forward
// direction of a stage is the same RK4, so its transcendental evaluations are
// done once per stage.
// Plain FP64: sin and cos of th1 - th2 from those of th1 and th2 (angle
// difference identities; absolute error of a few ulps, which the model only
// multiplies by O(1) terms), saving a third of the FP64 transcendentals.
__device__ __forceinline__ void sin_cos3(const double &a, const double &b, double *sc) {
  sin_cos(a, sc[0], sc[1]);
  sin_cos(b, sc[2], sc[3]);
  sc[4] = sc[0] * sc[3] - sc[1] * sc[2];
  sc[5] = sc[1] * sc[3] + sc[0] * sc[2];
}

struct TrigCompute {
  template <class Num>
  __device__ __forceinline__ void operator()(const Num &a, const Num &b, const Num &d, Num *sc) {
    sin_cos(a, sc[0], sc[1]);
    sin_cos(b, sc[2], sc[3]);
    sin_cos(d, sc[4], sc[5]);
  }
  __device__ __forceinline__ void operator()(const double &a, const double &b, const double &,
                                             double *sc) {
    sin_cos3(a, b, sc);
  }
};

struct TrigRecord {
  double *rec;  // 6 values per right-hand side, appended
  __device__ __forceinline__ void operator()(const double &a, const double &b, const double &,
                                             double *sc) {
    sin_cos3(a, b, sc);
#pragma unroll
    for (int j = 0; j < 6; ++j) rec[j] = sc[j];
    rec += 6;
  }
};

struct TrigReplay {
  const double *rec;
  __device__ __forceinline__ void one(const D1<double> &x, double s, double c, D1<double> &S,
                                      D1<double> &C) {
    S = {s, c * x.d};
    C = {c, -s * x.d};
  }
  __device__ __forceinline__ void operator()(const D1<double> &a, const D1<double> &b,
                                             const D1<double> &d, D1<double> *sc) {
    one(a, rec[0], rec[1], sc[0], sc[1]);
    one(b, rec[2], rec[3], sc[2], sc[3]);
    one(d, rec[4], rec[5], sc[4], sc[5]);
    rec += 6;
  }
};

// xdot = f(x, u) for any number type Num over the scalar type T.
template <class Num, class T, class Trig = TrigCompute>
__device__ __forceinline__ void cdp_rhs(const CdpConst<T> &k, const Num x[6], const Num &u,
                                        Num f[6], Trig &&trig = Trig{}) {
  Num sc[6];
  trig(x[1], x[2], x[1] - x[2], sc);
  const Num &s1 = sc[0], &c1 = sc[1], &s2 = sc[2], &c2 = sc[3], &s12 = sc[4], &c12 = sc[5];
  const Num w1s = x[4] * x[4], w2s = x[5] * x[5];
  const Num M12 = c1 * k.a1, M13 = c2 * k.a2, M23 = c12 * k.b12;
  const Num t1 = u + (s1 * w1s * k.a1 + s2 * w2s * k.a2);
  const Num t2 = s1 * k.a1g - s12 * w2s * k.b12;
  const Num t3 = s2 * k.m2gl2 + s12 * w1s * k.b12;
  const Num C11 = k.b1b2 - M23 * M23;
  const Num C12 = M13 * M23 - M12 * k.b2;
  const Num C13 = M12 * M23 - M13 * k.b1;
  const Num C22 = k.mtb2 - M13 * M13;
  const Num C23 = M12 * M13 - M23 * k.mt;
  const Num C33 = k.mtb1 - M12 * M12;
  const Num idet = reciprocal(C11 * k.mt + M12 * C12 + M13 * C13);
  f[0] = x[3];
  f[1] = x[4];
  f[2] = x[5];
  f[3] = (C11 * t1 + C12 * t2 + C13 * t3) * idet;
  f[4] = (C12 * t1 + C22 * t2 + C23 * t3) * idet;
  f[5] = (C13 * t1 + C23 * t2 + C33 * t3) * idet;
}

// One classical RK4 step of length dt with the control held.
template <class Num, class T, class Trig = TrigCompute>
__device__ __forceinline__ void cdp_rk4(const CdpConst<T> &k, const Num x[6], const Num &u,
                                        Num out[6], Trig &&trig = Trig{}) {
  Num kk[6], acc[6], z[6];
  cdp_rhs(k, x, u, kk, trig);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    acc[j] = kk[j];
    z[j] = x[j] + kk[j] * k.h2;
  }
  cdp_rhs(k, z, u, kk, trig);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    acc[j] = acc[j] + kk[j] * T(2);
    z[j] = x[j] + kk[j] * k.h2;
  }
  cdp_rhs(k, z, u, kk, trig);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    acc[j] = acc[j] + kk[j] * T(2);
    z[j] = x[j] + kk[j] * k.h;
  }
  cdp_rhs(k, z, u, kk, trig);
#pragma unroll
  for (int j = 0; j < 6; ++j) out[j] = x[j] + (acc[j] + kk[j]) * k.h6;
}

}  // namespace ipm
}  // namespace rlqr
