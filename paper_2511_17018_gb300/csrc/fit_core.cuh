// Device code of the batched TPC track fit.  Included by exactly one kernel
// module per mode; the module's compile flags select the arithmetic:
//   fit_fast.cu : FMA contraction, approximate division / square root, FTZ;
//   fit_det.cu  : -fmad=false -prec-div=true -prec-sqrt=true -ftz=false, i.e.
//                 the deterministic-mode rules of Sec. 2 (no FMA, IEEE
//                 operations, fixed order, functions without a deterministic
//                 FP32 result evaluated in FP64 by a fixed routine).
// The module defines TPCFIT_DET (0/1) and TPCFIT_NS before including this.
//
// The fit (per track): extended Kalman filter in the local frame of a TPC
// sector, state p = (y, z, sin phi, tan lambda, q/pt), covariance kept as a
// square-root factor C = L L^T (Potter form).  Outward pass from the seed with
// C0 = 100 I, updating at the first cluster first; inward refit from the
// outward result with C reset to C0 and chi2 reset; the output is the inward
// state at the first cluster, ndf = 2 n_used - 5.  Each step: rotation into the
// next cluster's sector frame if needed, analytic helix propagation to that pad
// row with its Jacobian, L <- J L, two scalar Potter updates (y then z).
//
// Work mapping: a persistent grid; each warp takes 32-track work items from a
// global counter and fits one track per lane.  While a lane computes the steps
// of the current chunk, the warp's asynchronous copies (cp.async) bring the
// next `RPS` clusters of all 32 tracks into the other half of a shared-memory
// double buffer.  The alignment table and the geometry live in shared memory.
// Tracks are taken in an order that puts tracks of equal length into the same
// warp (length_order.cu) so that a warp's lanes finish together.
//
// Compiled ahead of time by the two kernel modules, and at run time by NVRTC
// (TPCFIT_RTC = 1, Sec. 5): the run-time source first defines c_geo with the
// time frame's scalars as compile-time constants and its tables as
// initialised constant memory, so the compiler folds them into the code.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#else
#include "kernel_abi.h"
#endif
#include "device_util.cuh"

#ifndef TPCFIT_DET
#error "define TPCFIT_DET before including fit_core.cuh"
#endif
#ifndef TPCFIT_RTC
#define TPCFIT_RTC 0
#endif

namespace tpcfit {
namespace TPCFIT_NS {

// Per-time-frame constants.  Ahead of time they travel with every launch as
// part of its argument block (kernel parameters live in constant bank 0, read
// as free operands like __constant__ data), so each launch -- and each node of
// a captured CUDA graph -- carries its own time frame's constants and no
// launch can see another handle's.  At run time (NVRTC) the source defines
// c_geo with the scalars as compile-time constants instead.
#if TPCFIT_RTC
using GeoRef = GeoFold;
#define TPCFIT_GEO(args) c_geo
#else
using GeoRef = GeoConst;
#define TPCFIT_GEO(args) (args).geo
#endif

// Maclaurin coefficients of arcsin, a_n = a_{n-1} (2n-1)^2 / ((2n)(2n+1)),
// a_0 = 1 (Abramowitz & Stegun 4.4.40), evaluated in FP64 at compile time; the
// same for every time frame, so they are a fixed table of the module.
struct AsinCoef {
  double a[30];
};
__host__ __device__ constexpr AsinCoef asin_coefficients() {
  AsinCoef c{};
  c.a[0] = 1.0;
  for (int n = 1; n < 30; ++n)
    c.a[n] = c.a[n - 1] * ((double)(2 * n - 1) * (double)(2 * n - 1)) / ((double)(2 * n) * (double)(2 * n + 1));
  return c;
}
__constant__ AsinCoef c_asin = asin_coefficients();

struct Jac {
  bool rot;
  float yy, ys, yq, zy, zs, zt, zq, sy, ss, sq;
};

// ---------------------------------------------------------------- arcsin pieces
// FP64 arcsin: Maclaurin series for |u| <= 1/2, asin u = pi/2 - 2 asin(sqrt((1-u)/2))
// above (Abramowitz & Stegun 4.4.40-4.4.41).
__device__ __forceinline__ double asin_series_f64(double u) {
  const double q = u * u;
  double acc = c_asin.a[29];
#pragma unroll 1
  for (int n = 28; n >= 0; --n) acc = acc * q + c_asin.a[n];
  return acc * u;
}

__device__ __noinline__ double asin_f64(double u) {
  const double au = u < 0.0 ? -u : u;
  double r;
  if (au <= 0.5) {
    r = asin_series_f64(au);
  } else {
    const double h = sqrt((1.0 - au) * 0.5);
    r = 1.5707963267948966 - 2.0 * asin_series_f64(h);
  }
  return u < 0.0 ? -r : r;
}

// asin(u)/u: Horner in u^2 over the Maclaurin coefficients (c0..c6) for
// |u| <= 1/4, else the FP64 island (deterministic) or asinf (fast).
__device__ __forceinline__ float asinc_f(float u) {
  const float au = u < 0.0f ? -u : u;
#if !TPCFIT_DET
  if (au < 0.05f) {  // fast: three terms reach FP32 accuracy here (next term < 3e-11)
    const float q = u * u;
    return 1.0f + q * (static_cast<float>(1.0 / 6.0) + q * (static_cast<float>(3.0 / 40.0) +
                                                           q * static_cast<float>(5.0 / 112.0)));
  }
#endif
  if (au <= 0.25f) {
    const float c0 = 1.0f;
    const float c1 = static_cast<float>(1.0 / 6.0);
    const float c2 = static_cast<float>(3.0 / 40.0);
    const float c3 = static_cast<float>(5.0 / 112.0);
    const float c4 = static_cast<float>(35.0 / 1152.0);
    const float c5 = static_cast<float>(63.0 / 2816.0);
    const float c6 = static_cast<float>(231.0 / 13312.0);
    const float q = u * u;
    float acc = c6;
    acc = acc * q + c5;
    acc = acc * q + c4;
    acc = acc * q + c3;
    acc = acc * q + c2;
    acc = acc * q + c1;
    acc = acc * q + c0;
    return acc;
  }
#if TPCFIT_DET
  const double ud = (double)u;
  return (float)(asin_f64(ud) / ud);
#else
  return asinf(u) / u;
#endif
}

// c = sqrt(u) and 1/c.  Deterministic: IEEE square root and division, in the
// canonical order; fast: one reciprocal square root.
__device__ __forceinline__ void sqrt_and_inv(float u, float& c, float& ic) {
#if TPCFIT_DET
  c = sqrtf(u);
  ic = 1.0f / c;
#else
  ic = rsqrtf(u);
  c = u * ic;
#endif
}

// Potter coefficients for innovation variance s2 and cluster variance v:
// alpha = 1/s2, beta = sqrt(alpha v), gamma = 1/(1 + beta).  Fast mode derives
// alpha and beta from one reciprocal square root (beta = sqrt(v) rsqrt(s2)).
__device__ __forceinline__ void potter_coeffs(float s2, float v, float sqrt_v, float& alpha, float& beta,
                                              float& gamma) {
#if TPCFIT_DET
  (void)sqrt_v;
  alpha = 1.0f / s2;
  beta = sqrtf(alpha * v);
  gamma = 1.0f / (1.0f + beta);
#else
  (void)v;
  const float r = rsqrtf(s2);
  alpha = r * r;
  beta = sqrt_v * r;
  gamma = __fdividef(1.0f, 1.0f + beta);
#endif
}

// ---------------------------------------------------------------- geometry in smem
struct SmemTables {
  float row_x[kMaxRows];
  float rot_c[kNSide * kNSide];
  float rot_s[kNSide * kNSide];
};

__device__ __forceinline__ void load_tables(const GeoRef& G, SmemTables& t) {
  for (int i = threadIdx.x; i < kMaxRows; i += blockDim.x) t.row_x[i] = G.row_x[i];
  for (int i = threadIdx.x; i < kNSide * kNSide; i += blockDim.x) {
    t.rot_c[i] = G.rot_c[i];
    t.rot_s[i] = G.rot_s[i];
  }
}

// ---------------------------------------------------------------- one prediction step
// Intermediates of one prediction, kept for its adjoint.  The fit ignores
// them (the compiler drops the dead stores).
struct PredTape {
  float x, y, s;                // state before the step (pre-rotation)
  float c, cr, ca, sa;          // rotation pieces
  float x1, s1, dx, k, kdx, s2;
  float c1, ic1, c2, ic2, Tm, den, w, sig, A, dl, tt;
  float Jys0, Jzs0, Lk;
  float kap, xm, ym, zm;        // curvature per unit q/pt used; the field map's midpoint
  bool series;
};

// From state (p, x) in sector-frame a (mod 18) to pad row X in frame b: optional
// rotation at the current point, then helix propagation at fixed Bz.  Returns
// false, leaving nothing changed, if the step is impossible.
//
// Field map (G.field): the step's curvature uses Bz at its midpoint,
// estimated by a straight half step from the start point (after the rotation),
// kappa_step = kappa (1 + f_r (x_m^2 + y_m^2) + f_z z_m^2); the Jacobian
// treats kappa_step as a constant.  (yo, zo) turn pin's y, z into absolute
// positions (residual form).  FIELD: 0 uniform (no map code), 1 the map,
// 2 decided at run time by G.field.
template <int FIELD = 2>
__device__ __forceinline__ bool predict_t(const GeoRef& G, const SmemTables& T, const float pin[5], float xin, int a, int b, float X,
                                          float pout[5], Jac& J, PredTape& tp, float yo = 0.0f, float zo = 0.0f) {
  float kappa = G.kappa;
  const float maxsnp = G.max_snp;
  float x1 = xin, y1 = pin[0], s1 = pin[2];
  const float t = pin[3];
  const float q = pin[4];
  J.rot = (a != b);
  float cprev = 0.0f, crot = 0.0f, ca = 1.0f, sa = 0.0f;
  tp.x = xin;
  tp.y = pin[0];
  tp.s = pin[2];
  if (J.rot) {
    ca = T.rot_c[a * kNSide + b];
    sa = T.rot_s[a * kNSide + b];
    const float s = pin[2];
    const float c = sqrtf((1.0f - s) * (1.0f + s));
    const float xr = xin * ca + pin[0] * sa;
    const float yr = pin[0] * ca - xin * sa;
    const float sr = s * ca - c * sa;
    const float cr = c * ca + s * sa;
    if (!(cr > 0.0f)) return false;
    if (!(fabsf(sr) < maxsnp)) return false;
    x1 = xr;
    y1 = yr;
    s1 = sr;
    cprev = c;
    crot = cr;
  }
  tp.c = cprev;
  tp.cr = crot;
  tp.ca = ca;
  tp.sa = sa;
  const float dx = X - x1;
  if (FIELD == 1 || (FIELD == 2 && G.field)) {
    const float c1f = sqrtf((1.0f - s1) * (1.0f + s1));
    const float hdx = dx * 0.5f;
    const float ym = (yo + y1) + hdx * (s1 / c1f);
    const float zm = (zo + pin[1]) + hdx * (t / c1f);
    const float xm = x1 + hdx;
    kappa = kappa * ((1.0f + G.f_r * (xm * xm + ym * ym)) + G.f_z * (zm * zm));
    tp.xm = xm;
    tp.ym = ym;
    tp.zm = zm;
  }
  tp.kap = kappa;
  const float k = q * kappa;
  const float kdx = k * dx;
  const float s2 = s1 + kdx;
  if (!(fabsf(s2) < maxsnp)) return false;
  float c1, ic1, c2, ic2;
  sqrt_and_inv((1.0f - s1) * (1.0f + s1), c1, ic1);
  sqrt_and_inv((1.0f - s2) * (1.0f + s2), c2, ic2);
  const float den = c1 + c2;
#if TPCFIT_DET
  const float Tm = (s1 + s2) / den;
#else
  const float Tm = __fdividef(s1 + s2, den);
#endif
  const float w = c1 + s1 * Tm;
  const float sig = kdx * w;
  const float A = asinc_f(sig);
  const float dl = (dx * w) * A;
  pout[0] = y1 + dx * Tm;
  pout[1] = pin[1] + t * dl;
  pout[2] = s2;
  pout[3] = t;
  pout[4] = q;
  const float tt = 1.0f + Tm * Tm;
  J.ys = (dx * tt) * ((ic1 + ic2) * 0.5f);
  J.yq = ((dx * kappa) * dx) * (tt * (ic2 * 0.5f));
  J.zs = (t * dx) * (Tm * (ic1 * ic2));
  J.zt = dl;
  float Lk;  // d(path)/dk
  const bool series = fabsf(kdx) < 0.01f;
  if (series) {
    const float i2 = ic1 * ic1;
    const float i3 = i2 * ic1;
    const float i5 = i3 * i2;
    const float i7 = i5 * i2;
    const float s1s = s1 * s1;
    const float a1 = (s1 * i3) * 0.5f;
    const float a2 = ((1.0f + 2.0f * s1s) * i5) * static_cast<float>(1.0 / 3.0);
#if TPCFIT_DET
    const float a3 = ((s1 * (3.0f + 2.0f * s1s)) * i7) * 0.125f;
    Lk = (dx * dx) * (a1 + kdx * (a2 + kdx * a3));
#else
    (void)i7;
    Lk = (dx * dx) * (a1 + kdx * a2);
#endif
  } else {
#if TPCFIT_DET
    Lk = (dx * ic2 - dl) / k;
#else
    Lk = __fdividef(dx * ic2 - dl, k);
#endif
  }
  J.zq = (t * kappa) * Lk;
  J.sq = dx * kappa;
  tp.x1 = x1; tp.s1 = s1; tp.dx = dx; tp.k = k; tp.kdx = kdx; tp.s2 = s2;
  tp.c1 = c1; tp.ic1 = ic1; tp.c2 = c2; tp.ic2 = ic2; tp.Tm = Tm; tp.den = den; tp.w = w; tp.sig = sig;
  tp.A = A; tp.dl = dl; tp.tt = tt; tp.Jys0 = J.ys; tp.Jzs0 = J.zs; tp.Lk = Lk; tp.series = series;
  if (J.rot) {
    const float rr = crot / cprev;
    J.yy = ca - sa * (s2 * ic2);
    J.zy = -(sa * (t * ic2));
    J.sy = -(sa * k);
    J.ss = rr;
    J.ys = J.ys * rr;
    J.zs = J.zs * rr;
  } else {
    J.yy = 1.0f;
    J.zy = 0.0f;
    J.sy = 0.0f;
    J.ss = 1.0f;
  }
  return true;
}

__device__ __forceinline__ bool predict(const GeoRef& G, const SmemTables& T, const float pin[5], float xin, int a, int b, float X,
                                        float pout[5], Jac& J) {
  PredTape tp;
  return predict_t<2>(G, T, pin, xin, a, b, X, pout, J, tp);
}

// Prediction in residual coordinates: p[0..1] are residuals from (my, mz), the
// output is relative to the next cluster's measurement (m0, m1).  Without a
// rotation the exact difference of the two measurements is added; across a
// rotation the absolute position is formed, rotated, propagated and
// re-referenced.
template <int FIELD = 2>
__device__ __forceinline__ bool predict_residual(const GeoRef& G, const SmemTables& T, const float p[5], float x, int sec, float my,
                                                 float mz, int sec_to, float X, float m0, float m1, float pout[5],
                                                 Jac& J, PredTape& tp) {
  float pin[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) pin[c] = p[c];
  const bool rot = sec != sec_to;
  if (rot) {
    pin[0] = my + p[0];
    pin[1] = mz + p[1];
  }
  if (!predict_t<FIELD>(G, T, pin, x, sec, sec_to, X, pout, J, tp, rot ? 0.0f : my, rot ? 0.0f : mz)) return false;
  if (rot) {
    pout[0] = pout[0] - m0;
    pout[1] = pout[1] - m1;
  } else {
    pout[0] = pout[0] + (my - m0);
    pout[1] = pout[1] + (mz - m1);
  }
  return true;
}

// L <- J L (rows t, q of J are identity).
__device__ __forceinline__ void transport(float L[5][5], const Jac& J) {
  if (!J.rot) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const float ny = (L[0][c] + J.ys * L[2][c]) + J.yq * L[4][c];
      const float nz = ((L[1][c] + J.zs * L[2][c]) + J.zt * L[3][c]) + J.zq * L[4][c];
      const float ns = L[2][c] + J.sq * L[4][c];
      L[0][c] = ny;
      L[1][c] = nz;
      L[2][c] = ns;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const float ny = (J.yy * L[0][c] + J.ys * L[2][c]) + J.yq * L[4][c];
      const float nz = (((J.zy * L[0][c] + L[1][c]) + J.zs * L[2][c]) + J.zt * L[3][c]) + J.zq * L[4][c];
      const float ns = (J.sy * L[0][c] + J.ss * L[2][c]) + J.sq * L[4][c];
      L[0][c] = ny;
      L[1][c] = nz;
      L[2][c] = ns;
    }
  }
}

// Potter scalar update of component H (0 = y, 1 = z) with measured value mv.
template <int H>
__device__ __forceinline__ void scalar_update(const GeoRef& G, float p[5], float L[5][5], float& chi2, float mv) {
  const float v = G.v_meas;
  float a[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) a[c] = L[H][c];
  float s2 = v + a[0] * a[0];
#pragma unroll
  for (int c = 1; c < 5; ++c) s2 = s2 + a[c] * a[c];
  float alpha, beta, gamma;
  potter_coeffs(s2, v, G.sqrt_v, alpha, beta, gamma);
  const float r = mv - p[H];
#if TPCFIT_DET
  // canonical sequence: K = alpha L a, p += K r, gain factors gamma K
  float K[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float la = L[i][0] * a[0];
#pragma unroll
    for (int c = 1; c < 5; ++c) la = la + L[i][c] * a[c];
    K[i] = la * alpha;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + K[i] * r;
  chi2 = chi2 + (r * r) * alpha;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) continue;
    const float gk = gamma * K[i];
#pragma unroll
    for (int c = 0; c < 5; ++c) L[i][c] = L[i][c] - gk * a[c];
  }
#else
  // fast: the same algebra with alpha folded into the fused multiply-adds;
  // row H of L a is a . a = s2 - v
  const float ar = alpha * r;
  const float ga = gamma * alpha;
  float la[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) {
      la[i] = s2 - v;
      continue;
    }
    float acc = L[i][0] * a[0];
#pragma unroll
    for (int c = 1; c < 5; ++c) acc = acc + L[i][c] * a[c];
    la[i] = acc;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + la[i] * ar;
  chi2 = chi2 + r * ar;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) continue;
    const float gk = la[i] * ga;
#pragma unroll
    for (int c = 0; c < 5; ++c) L[i][c] = L[i][c] - gk * a[c];
  }
#endif
#pragma unroll
  for (int c = 0; c < 5; ++c) L[H][c] = a[c] * beta;
}

}  // namespace TPCFIT_NS
}  // namespace tpcfit

#include "ud_filter.cuh"

namespace tpcfit {
namespace TPCFIT_NS {

// ---------------------------------------------------------------- material
// A thin material layer at every pad row (G.mat): the state at a row is
// the one the track leaves it with; the outward pass crosses a row's layer on
// arriving (dir = +1), the inward pass undoes it before leaving the row
// against the flight (dir = -1).  Path through the layer
// l = d sqrt(1 + t^2) / c; energy loss dE/dx_mip l / beta^2 (pion); multiple
// scattering with the Highland angle (no logarithmic term) as the process
// noise Q = B B^T; the q row of the factor scaled by p / p'.  Returns false if
// the particle would stop.  The operation sequence is the canonical one of the
// strict-FP32 reference (the deterministic mode matches it bit for bit).
struct MatNoise {
  float qq, b_s, b_t, b_q;
};

__device__ __forceinline__ bool material_step(const GeoRef& G, float p[5], int dir, MatNoise& N) {
  const float s = p[2];
  const float t = p[3];
  const float q = p[4];
  const float q2 = q * q;
  if (!(q2 > 0.0f)) {
    N.qq = 1.0f;
    N.b_s = N.b_t = N.b_q = 0.0f;
    return true;
  }
  const float tt1 = 1.0f + t * t;
  const float c = sqrtf((1.0f - s) * (1.0f + s));
  const float st1 = sqrtf(tt1);
  const float ell = (G.d_row * st1) / c;
  const float p2 = tt1 / q2;
  const float e2 = p2 + G.mass2;
  const float th2 = ((static_cast<float>(0.0136 * 0.0136) * ell) * G.x0_inv) * (e2 / (p2 * p2));
  const float de = (G.dedx * ell) * (e2 / p2);
  const float e = sqrtf(e2);
  const float en = dir > 0 ? e - de : e + de;
  const float pn2 = en * en - G.mass2;
  if (!(pn2 > 0.0f)) return false;
  const float ratio = sqrtf(p2 / pn2);
  p[4] = q * ratio;
  const float th = sqrtf(th2);
  N.qq = ratio;
  N.b_s = (th * c) * st1;
  N.b_t = th * tt1;
  N.b_q = (th * p[4]) * t;
  return true;
}

// L <- D L (D = diag(1, 1, 1, 1, qq)), then B folded in: the Householder QR of
// X = [L^T; B^T] (7x5) gives L L^T + B B^T = R^T R, and L <- R^T.  Column k:
// |x|^2 of rows k..6, alpha = -sign(x_k) |x|, v = x - alpha e_k,
// g = 1 / (alpha v_k); later columns j: t = (v_k X_kj + sum_r X_rk X_rj) g,
// X_kj += t v_k, X_rj += t X_rk; X_kk = alpha.
__device__ __forceinline__ void material_factor(float L[5][5], const MatNoise& N) {
#pragma unroll
  for (int c = 0; c < 5; ++c) L[4][c] = L[4][c] * N.qq;
  float X[7][5];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int i = 0; i < 5; ++i) X[r][i] = L[i][r];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    X[5][i] = 0.0f;
    X[6][i] = 0.0f;
  }
  X[5][2] = N.b_s;
  X[6][3] = N.b_t;
  X[6][4] = N.b_q;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float nrm2 = X[k][k] * X[k][k];
#pragma unroll
    for (int r = k + 1; r < 7; ++r) nrm2 = nrm2 + X[r][k] * X[r][k];
    const float nrm = sqrtf(nrm2);
    const float alpha = X[k][k] > 0.0f ? 0.0f - nrm : nrm;
    const float v0 = X[k][k] - alpha;
    const float gk = 1.0f / (alpha * v0);
#pragma unroll
    for (int j = k + 1; j < 5; ++j) {
      float t = v0 * X[k][j];
#pragma unroll
      for (int r = k + 1; r < 7; ++r) t = t + X[r][k] * X[r][j];
      t = t * gk;
      X[k][j] = X[k][j] + t * v0;
#pragma unroll
      for (int r = k + 1; r < 7; ++r) X[r][j] = X[r][j] + t * X[r][k];
    }
    X[k][k] = alpha;
  }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) L[i][j] = j <= i ? X[j][i] : 0.0f;
}

__device__ __forceinline__ void reset_factor(const GeoRef& G, float L[5][5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) L[i][c] = (i == c) ? G.l0 : 0.0f;
}

// Sector mod 18 (its azimuth) of a validated sector number (< 36).
__device__ __forceinline__ int side_sector(int sec) { return sec >= kNSide ? sec - kNSide : sec; }

__device__ __forceinline__ void record_error(unsigned long long* err, unsigned long long code, int64_t track) {
  const unsigned long long v = (code << 56) | ((unsigned long long)track & 0x00FFFFFFFFFFFFFFull);
  atomicCAS(err, 0ull, v);
}

// ---------------------------------------------------------------- the fit kernel
// Lane state across the two passes.
// y and z are carried as residuals from the measurement (my, mz) of the
// current cluster: p[0] = y - my, p[1] = z - mz.
struct TrackState {
  float p[5];
  float L[5][5];   // square-root factor (C = L L^T), or
  float u[10];     // the U-D factor (C = U D U^T), by the kernel's FORM
  float d[5];
  float x;
  float chi2;
  float my, mz;
  int sec;      // sector (mod 18) of the current frame
  int used;
};

// Asynchronous 4-byte global -> shared copies (no register staging).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Double-buffered staging of RPS clusters for each of a warp's 32 tracks.  Row
// pitch RPS + 1 keeps the consumer's reads (lane t reads row t) conflict-free.
// rowsec travels as the aligned 32-bit word that contains it.
template <int RPS>
struct WarpStage {
  float y[2][kWarp][RPS + 1];
  float z[2][kWarp][RPS + 1];
  uint32_t rs[2][kWarp][RPS + 1];
};

// Issue the copies of local steps [c0, c0 + RPS) of every lane's pass into
// buffer b: lane t's step i is hit first_t + dir * i (valid for i < count_t).
// Each group of RPS lanes copies RPS consecutive clusters of one track.
template <int RPS>
__device__ __forceinline__ void stage_issue(WarpStage<RPS>& st, int b, const FitArgs& a, int my_first,
                                            int my_count, int dir, int c0, int lane) {
  const uintptr_t rs_begin = (uintptr_t)a.rowsec;
  const uintptr_t rs_end = (uintptr_t)(a.rowsec + a.n_hits);
#pragma unroll
  for (int it = 0; it < RPS; ++it) {
    const int e = it * kWarp + lane;
    const int t = e / RPS;
    const int k = e % RPS;
    const int first_t = __shfl_sync(0xffffffffu, my_first, t);
    const int count_t = __shfl_sync(0xffffffffu, my_count, t);
    const int i = c0 + k;
    if (i < count_t) {
      const int h = first_t + dir * i;
      cp_async4(&st.y[b][t][k], a.y + h);
      cp_async4(&st.z[b][t][k], a.z + h);
      const uint16_t* rp = a.rowsec + h;
      const uintptr_t wa = (uintptr_t)rp & ~(uintptr_t)3;
      if (wa >= rs_begin && wa + 4 <= rs_end) {
        cp_async4(&st.rs[b][t][k], (const void*)wa);
      } else {  // a cluster whose 32-bit word reaches outside the array
        st.rs[b][t][k] = (uint32_t)__ldg(rp) << (16u * (unsigned)(((uintptr_t)rp >> 1) & 1u));
      }
    }
  }
  cp_async_commit();
}

struct BlockSmem {
  SmemTables T;
  float align[kAlignFloats];
};
static_assert(sizeof(BlockSmem) == kFitBlockSmemBytes, "kernel_abi.h block shared-memory size");
static_assert(sizeof(WarpStage<4>) == fit_warp_stage_bytes(4) && sizeof(WarpStage<8>) == fit_warp_stage_bytes(8) &&
                  sizeof(WarpStage<16>) == fit_warp_stage_bytes(16),
              "kernel_abi.h staging size");

template <int FIELD>
__device__ __forceinline__ bool step_predict(const GeoRef& G, const SmemTables& T, const TrackState& S, int sec_to, float X, float m0,
                                             float m1, float pout[5], Jac& J) {
  PredTape tp;
  return predict_residual<FIELD>(G, T, S.p, S.x, S.sec, S.my, S.mz, sec_to, X, m0, m1, pout, J, tp);
}

// Checkpoint: the state and its covariance factor (32 floats: p, the factor,
// x, sector).  The square-root form writes L row by row in floats 5..29; the
// U-D form writes u (10) in floats 5..14, d (5) in 15..19 and zeros after.
template <int FORM>
__device__ __forceinline__ void write_ckpt(const FitArgs& a, int pass, int begin, int trk, int seg,
                                           const TrackState& S) {
  float4* dst = reinterpret_cast<float4*>(a.ck + ((int64_t)pass * a.ck_slots + (begin >> kCkptShift) + trk + seg) * kCkptFloats);
  float v[kCkptFloats];
#pragma unroll
  for (int c = 0; c < 5; ++c) v[c] = S.p[c];
  if (FORM == 1) {
#pragma unroll
    for (int e = 0; e < 10; ++e) v[5 + e] = S.u[e];
#pragma unroll
    for (int c = 0; c < 5; ++c) v[15 + c] = S.d[c];
#pragma unroll
    for (int e = 20; e < 30; ++e) v[e] = 0.0f;
  } else {
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int c = 0; c < 5; ++c) v[5 + 5 * i + c] = S.L[i][c];
  }
  v[30] = S.x;
  v[31] = __int_as_float(S.sec);
#pragma unroll
  for (int j = 0; j < kCkptFloats / 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// PHYS: bit 0 the material layers, bit 1 the field map (compile-time variants,
// so that the plain fit carries neither).  FORM: the covariance's factor, 0
// the square-root factor with Potter's updates (the canonical sequence of the
// deterministic mode), 1 U-D with Bierman's (fast mode, no material layers).
template <int RPS, int WARPS, int MINB, bool RECORD, bool FRAMES, int PHYS, int FORM = 0>
__global__ void __launch_bounds__(WARPS * 32, MINB) fit_kernel(const __grid_constant__ FitArgs a) {
  const GeoRef& G = TPCFIT_GEO(a);
  constexpr bool MAT = (PHYS & 1) != 0;
  constexpr int FIELD = (PHYS & 2) ? 1 : 0;
  static_assert(FORM == 0 || (!MAT && !TPCFIT_DET), "the U-D fit: fast mode without material layers");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSmem& B = *reinterpret_cast<BlockSmem*>(smem_raw);
  WarpStage<RPS>* stages = reinterpret_cast<WarpStage<RPS>*>(smem_raw + sizeof(BlockSmem));
  load_tables(G, B.T);
  for (int i = threadIdx.x; i < kAlignFloats; i += blockDim.x) B.align[i] = __ldg(a.align + i);
  __syncthreads();
  const SmemTables& T = B.T;
  const int lane = threadIdx.x & 31;
  WarpStage<RPS>& st = stages[threadIdx.x >> 5];
  const unsigned rs_par0 = (unsigned)(((uintptr_t)a.rowsec >> 1) & 1u);
  const int64_t n_chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;

#pragma unroll 1
  for (;;) {
    // ---- take the next 32-track work item
    int64_t chunk = 0;
    if (lane == 0) chunk = (int64_t)atomicAdd(a.work, 1u);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= n_chunks) break;
    const int64_t slot = chunk * kWarp + lane;
    const bool have = slot < a.n_tracks;
    const int32_t trk = have ? (a.perm ? a.perm[slot] : (int32_t)slot) : 0;

    // ---- per-track input checks
    // hit indices fit in int32: the host rejects n_hits > INT32_MAX
    int status = have ? 0 : 1;  // 0 fitting, 1 idle, 2 numerical failure, 3 invalid input, 4 timeout
    int begin = 0;
    int n = 0;
    const float* lane_align = B.align;
    if (FRAMES && have) {
      // the track's time frame: its alignment table and, when streaming, its ready flag
      const int f = frame_of(a.frame_base, a.n_frames, trk);
      if (f < 0) {
        status = 3;
        record_error(a.err, kErrOffsets, trk);
      } else {
        if (a.frame_ready && !wait_flag(a.frame_ready + f, a.wait_ns)) {
          status = 4;
          record_error(a.err, kErrTimeout, trk);
        }
        if (a.frame_align) lane_align = a.frame_align + (int64_t)f * kAlignFloats;
      }
    }
    if (FRAMES) __syncwarp();  // every lane's frame is in place before the warp stages clusters
    if (have && status == 0) {
      const int b = a.off[trk];
      const int e = a.off[trk + 1];
      if (b < 0 || e < b || (int64_t)e > a.n_hits) {
        status = 3;
        record_error(a.err, kErrOffsets, trk);
      } else {
        begin = b;
        n = e - b;
        if (n < 1) status = 2;
      }
    }
    TrackState S;
    S.x = 0.0f;
    S.sec = 0;
    int last = 0;
    if (status == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) S.p[c] = __ldg(a.seeds + (int64_t)c * a.n_tracks + trk);
      if (!(fabsf(S.p[2]) < G.max_snp)) status = 2;
    }

    // ---- two passes: outward (dir +1 from hit 0) and inward (dir -1 from `last`)
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int dir = pass == 0 ? 1 : -1;
      const int my_first = begin + (pass == 0 ? 0 : last);
      const int my_count = (status == 0) ? (pass == 0 ? n : last + 1) : 0;
      bool go = status == 0;
      if (go) {
        if (FORM == 1) {
#pragma unroll
          for (int e = 0; e < 10; ++e) S.u[e] = 0.0f;
#pragma unroll
          for (int c = 0; c < 5; ++c) S.d[c] = G.l0 * G.l0;
        } else {
          reset_factor(G, S.L);
        }
        S.chi2 = 0.0f;
        S.used = 0;
      }
      int count_max = my_count;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) count_max = max(count_max, __shfl_xor_sync(0xffffffffu, count_max, o));
      if (count_max == 0) continue;
      __syncwarp();
      stage_issue<RPS>(st, 0, a, my_first, my_count, dir, 0, lane);
      int buf = 0;
#pragma unroll 1
      for (int c0 = 0; c0 < count_max; c0 += RPS) {
        const bool more = c0 + RPS < count_max;
        if (more) {
          stage_issue<RPS>(st, buf ^ 1, a, my_first, my_count, dir, c0 + RPS, lane);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncwarp();
#pragma unroll 1
        for (int k = 0; k < RPS; ++k) {
          const int i = c0 + k;
          if (!go || i >= my_count) continue;
          const int h = my_first + dir * i;
          const unsigned shift = 16u * ((rs_par0 + (unsigned)h) & 1u);
          const int rsv = (int)((st.rs[buf][lane][k] >> shift) & 0xffffu);
          const int row = rsv >> 6;
          const int sec = rsv & 63;
          if (row >= G.n_rows || sec >= kNSectors) {
            status = 3;
            go = false;
            record_error(a.err, kErrRowSector, trk);
            continue;
          }
          const float2 d = FRAMES ? reinterpret_cast<const float2*>(lane_align)[sec * kMaxRows + row]
                                  : reinterpret_cast<const float2*>(B.align)[sec * kMaxRows + row];
          const float m0 = st.y[buf][lane][k] - d.x;
          const float m1 = st.z[buf][lane][k] - d.y;
          const int sec18 = side_sector(sec);
          if (RECORD && (i & (kCkptEvery - 1)) == 0) write_ckpt<FORM>(a, pass, begin, trk, i >> kCkptShift, S);
          if (i == 0) {
            // first cluster of the pass: the state sits on its row already; the
            // outward pass turns the seed's (y, z) into residuals
            S.x = T.row_x[row];
            S.sec = sec18;
            if (pass == 0) {
              S.my = m0;
              S.mz = m1;
              S.p[0] = S.p[0] - m0;
              S.p[1] = S.p[1] - m1;
            }
          } else {
            float pn[5];
            Jac J;
            if (MAT && pass == 1) {  // the layer of the row left, undone against the flight
              MatNoise N;
              if (!material_step(G, S.p, -1, N)) {
                go = false;
                status = 2;
                continue;
              }
              material_factor(S.L, N);
            }
            if (!step_predict<FIELD>(G, T, S, sec18, T.row_x[row], m0, m1, pn, J)) {
              go = false;
              if (pass == 1) status = 2;  // the inward pass must reach the first cluster
              continue;
            }
            MatNoise N;
            // the layer of the row arrived at (a particle that stops there ends
            // the outward pass with the state before the step)
            if (MAT && pass == 0 && !material_step(G, pn, 1, N)) {
              go = false;
              continue;
            }
#pragma unroll
            for (int c = 0; c < 5; ++c) S.p[c] = pn[c];
            S.x = T.row_x[row];
            S.sec = sec18;
            S.my = m0;
            S.mz = m1;
            if (FORM == 1) {
              if (J.rot)
                rotate_ud(S.u, S.d, J);
              else
                transport_ud(S.u, J);
            } else {
              transport(S.L, J);
            }
            if (MAT && pass == 0) material_factor(S.L, N);
          }
          if (FORM == 1) {
            bierman_update<0>(S.p, S.u, S.d, S.chi2, G.v_meas);
            bierman_update<1>(S.p, S.u, S.d, S.chi2, G.v_meas);
          } else {
            scalar_update<0>(G, S.p, S.L, S.chi2, 0.0f);
            scalar_update<1>(G, S.p, S.L, S.chi2, 0.0f);
          }
          S.used += 1;
          if (pass == 0) last = i;
        }
        __syncwarp();
        buf ^= 1;
      }
    }

    // ---- outputs at the track's own index
    if (!have) continue;
    if (RECORD) a.ck_last[trk] = last;
    const int64_t N = a.n_tracks;
    if (status == 0 && S.used >= 3) {
      a.params[trk] = S.my + S.p[0];
      a.params[N + trk] = S.mz + S.p[1];
#pragma unroll
      for (int c = 2; c < 5; ++c) a.params[(int64_t)c * N + trk] = S.p[c];
      int e = 0;
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          float acc;
          if (FORM == 1) {  // C_ij = sum over k >= i of u_ik d_k u_jk (j <= i, u_kk = 1)
            acc = (j == i ? 1.0f : S.u[ui(j, i)]) * S.d[i];
#pragma unroll
            for (int k = i + 1; k < 5; ++k) acc = acc + (S.u[ui(i, k)] * S.d[k]) * S.u[ui(j, k)];
          } else {
            acc = S.L[i][0] * S.L[j][0];
#pragma unroll
            for (int c = 1; c < 5; ++c) acc = acc + S.L[i][c] * S.L[j][c];
          }
          a.cov[(int64_t)e * N + trk] = acc;
          ++e;
        }
      a.chi2[trk] = S.chi2;
      a.ndf[trk] = 2 * S.used - 5;
    } else {
      const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
      for (int c = 0; c < 5; ++c) a.params[(int64_t)c * N + trk] = qnan;
#pragma unroll
      for (int e = 0; e < 15; ++e) a.cov[(int64_t)e * N + trk] = qnan;
      a.chi2[trk] = qnan;
      a.ndf[trk] = (status == 3) ? -2 : (status == 4 ? -3 : -1);
    }
  }
}

#ifndef __CUDACC_RTC__
template <int RPS, int WARPS, int MINB, bool RECORD, bool FRAMES, int PHYS, int FORM>
cudaError_t launch_cfg(const FitArgs& a, cudaStream_t s) {
  constexpr int kThreads = WARPS * 32;
  const size_t smem = sizeof(BlockSmem) + WARPS * sizeof(WarpStage<RPS>);
  auto kernel = fit_kernel<RPS, WARPS, MINB, RECORD, FRAMES, PHYS, FORM>;
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = sms * per_sm;
  }
  const int64_t chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t need = (chunks + WARPS - 1) / WARPS;
  const int blocks = (int)(need < grid ? need : grid);
  cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  kernel<<<blocks, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Supported (rows per stage, warps per block) shapes; the shared-memory budget
// (alignment table + double buffer) decides how many blocks fit on an SM.
// With material or a field map the fit runs at (4, 24).
template <bool RECORD, bool FRAMES, int FORM>
inline cudaError_t launch_rec(const FitArgs& a, int rps, int warps, cudaStream_t s) {
  const int phys = (a.mat ? 1 : 0) | (a.field ? 2 : 0);
  if (FORM == 0) {
    if (phys == 1) return launch_cfg<4, 24, fit_min_blocks(4, 24), RECORD, FRAMES, 1, 0>(a, s);
    if (phys == 3) return launch_cfg<4, 24, fit_min_blocks(4, 24), RECORD, FRAMES, 3, 0>(a, s);
  } else if (phys & 1) {
    return cudaErrorInvalidValue;
  }
  if (phys == 2) return launch_cfg<4, 24, fit_min_blocks(4, 24), RECORD, FRAMES, 2, FORM>(a, s);
  if (rps == 4 && warps == 8) return launch_cfg<4, 8, fit_min_blocks(4, 8), RECORD, FRAMES, 0, FORM>(a, s);
  if (rps == 4 && warps == 12) return launch_cfg<4, 12, fit_min_blocks(4, 12), RECORD, FRAMES, 0, FORM>(a, s);
  if (rps == 4 && warps == 24) return launch_cfg<4, 24, fit_min_blocks(4, 24), RECORD, FRAMES, 0, FORM>(a, s);
  if (rps == 8 && warps == 8) return launch_cfg<8, 8, fit_min_blocks(8, 8), RECORD, FRAMES, 0, FORM>(a, s);
  if (rps == 8 && warps == 16) return launch_cfg<8, 16, fit_min_blocks(8, 16), RECORD, FRAMES, 0, FORM>(a, s);
  if (rps == 16 && warps == 8) return launch_cfg<16, 8, fit_min_blocks(16, 8), RECORD, FRAMES, 0, FORM>(a, s);
  return cudaErrorInvalidValue;
}

template <int FORM>
inline cudaError_t launch_form(const FitArgs& a, int rps, int warps, cudaStream_t s) {
  if (a.frame_base)
    return a.ck ? launch_rec<true, true, FORM>(a, rps, warps, s) : launch_rec<false, true, FORM>(a, rps, warps, s);
  return a.ck ? launch_rec<true, false, FORM>(a, rps, warps, s) : launch_rec<false, false, FORM>(a, rps, warps, s);
}

// One lane per track.  FORM 1 (U-D) in fast mode without material layers,
// otherwise the square-root factor.
inline cudaError_t launch(const FitArgs& a, int lanes_per_track, int rps, int warps, cudaStream_t s) {
  if (a.n_tracks <= 0) return cudaSuccess;
  if (lanes_per_track != 1) return cudaErrorInvalidValue;
#if !TPCFIT_DET
  if (a.form == 1 && !a.mat) return launch_form<1>(a, rps, warps, s);
#endif
  return launch_form<0>(a, rps, warps, s);
}

#endif  // !__CUDACC_RTC__

}  // namespace TPCFIT_NS
}  // namespace tpcfit
