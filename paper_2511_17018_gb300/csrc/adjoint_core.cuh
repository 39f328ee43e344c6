// Adjoint (reverse mode) of the batched track fit.  Included after
// fit_core.cuh by the same kernel module, so that the forward recomputation
// uses the module's own arithmetic bit for bit.
//
// Objective: L = sum_i g_i chi2_i, chi2_i the inward-refit chi2 of track i.
// Gradients: dL/dm_h for every cluster measurement m_h = (y - dy, z - dz)
// (hence dL/d(dy, dz)[sector][row] = -sum over the clusters with that key),
// and dL/dseed_i.  The outward pass feeds the inward one through its final
// state (the covariance is reset, the outward chi2 is not part of L).
//
// Checkpoints: the forward writes the filter state (p, L, x, sector)
// before every kCkptEvery-th step of each pass.  The backward walks the
// segments of a track in reverse: it recomputes a segment's steps from its
// checkpoint into a per-warp segment store, then reverses the steps one by one
// (recomputing each step's intermediates from the state before it).  States carry y and z
// as residuals from the current cluster's measurement, like the fit.
#pragma once

namespace tpcfit {
namespace TPCFIT_NS {


struct JacBar {
  float yy, ys, yq, zy, zs, zt, zq, sy, ss, sq;
};

// d/du of asinc_f(u), consistent with the branch asinc_f takes.
__device__ __forceinline__ float asinc_deriv(float u) {
  const float au = u < 0.0f ? -u : u;
#if !TPCFIT_DET
  if (au < 0.05f) {  // derivative of the three-term fast-mode polynomial
    const float q = u * u;
    return (2.0f * u) * (static_cast<float>(1.0 / 6.0) +
                         q * (2.0f * static_cast<float>(3.0 / 40.0) + q * (3.0f * static_cast<float>(5.0 / 112.0))));
  }
#endif
  if (au <= 0.25f) {
    const float c1 = static_cast<float>(1.0 / 6.0);
    const float c2 = static_cast<float>(3.0 / 40.0);
    const float c3 = static_cast<float>(5.0 / 112.0);
    const float c4 = static_cast<float>(35.0 / 1152.0);
    const float c5 = static_cast<float>(63.0 / 2816.0);
    const float c6 = static_cast<float>(231.0 / 13312.0);
    const float q = u * u;
    float acc = 6.0f * c6;
    acc = acc * q + 5.0f * c5;
    acc = acc * q + 4.0f * c4;
    acc = acc * q + 3.0f * c3;
    acc = acc * q + 2.0f * c2;
    acc = acc * q + c1;
    return (2.0f * u) * acc;
  }
#if TPCFIT_DET
  const double ud = (double)u;
  const double sq = sqrt((1.0 - ud) * (1.0 + ud));
  return (float)((ud / sq - asin_f64(ud)) / (ud * ud));
#else
  return (u * rsqrtf((1.0f - u) * (1.0f + u)) - asinf(u)) / (u * u);
#endif
}

// Reverse of scalar_update<H>.  p, L: state before the update; b_p, b_L: in =
// adjoint after the update, out = adjoint before; b_chi: adjoint of chi2 (the
// same before and after).  b_m receives the adjoint of the measured value.
template <int H>
__device__ __forceinline__ void scalar_update_rev(const GeoRef& G, const float p[5], const float L[5][5], float mv, float b_p[5],
                                                  float b_L[5][5], float b_chi, float& b_m) {
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
  float la[5], K[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float acc = L[i][0] * a[0];
#pragma unroll
    for (int c = 1; c < 5; ++c) acc = acc + L[i][c] * a[c];
    la[i] = acc;
    K[i] = acc * alpha;
  }
  // p' = p + K r ; chi2' = chi2 + r^2 alpha
  float b_K[5], b_a[5];
  float b_r = 0.0f, b_alpha = 0.0f, b_gamma = 0.0f, b_beta = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    b_K[i] = r * b_p[i];
    b_r += K[i] * b_p[i];
  }
  b_r += 2.0f * r * alpha * b_chi;
  b_alpha += r * r * b_chi;
#pragma unroll
  for (int c = 0; c < 5; ++c) b_a[c] = 0.0f;
  // L'_i = L_i - (gamma K_i) a (i != H)
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) continue;
    const float gk = gamma * K[i];
    float b_gk = 0.0f;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      b_gk -= b_L[i][c] * a[c];
      b_a[c] -= gk * b_L[i][c];
    }
    b_gamma += K[i] * b_gk;
    b_K[i] += gamma * b_gk;
  }
  // L'_H = beta a
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    b_a[c] += beta * b_L[H][c];
    b_beta += a[c] * b_L[H][c];
  }
  // gamma = 1/(1 + beta)
  b_beta -= gamma * gamma * b_gamma;
  // K_i = la_i alpha
  float b_la[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    b_la[i] = alpha * b_K[i];
    b_alpha += la[i] * b_K[i];
  }
  // r = m - p_H
  b_m = b_r;
  b_p[H] -= b_r;
  // alpha = 1/s2, beta = sqrt(v/s2)
  const float b_s2 = -(alpha * alpha) * b_alpha - 0.5f * (beta * alpha) * b_beta;
  // la_i = L_i . a (i != H); la_H = a . a
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) continue;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      b_L[i][c] += a[c] * b_la[i];
      b_a[c] += L[i][c] * b_la[i];
    }
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) b_a[c] += 2.0f * a[c] * (b_la[H] + b_s2);
  // a = L_H: row H enters only through a
#pragma unroll
  for (int c = 0; c < 5; ++c) b_L[H][c] = b_a[c];
}

// Reverse of transport (L' = J L): b_L in = adjoint of L', out = adjoint of L;
// bJ = adjoint of the Jacobian entries.  L: the factor before the transport.
__device__ __forceinline__ void transport_rev(const float L[5][5], const Jac& J, float b_L[5][5], JacBar& bJ) {
  bJ.yy = bJ.ys = bJ.yq = bJ.zy = bJ.zs = bJ.zt = bJ.zq = bJ.sy = bJ.ss = bJ.sq = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const float b0 = b_L[0][c], b1 = b_L[1][c], b2 = b_L[2][c];
    bJ.ys += b0 * L[2][c];
    bJ.yq += b0 * L[4][c];
    bJ.zs += b1 * L[2][c];
    bJ.zt += b1 * L[3][c];
    bJ.zq += b1 * L[4][c];
    bJ.sq += b2 * L[4][c];
    b_L[3][c] += J.zt * b1;
    b_L[4][c] += J.yq * b0 + J.zq * b1 + J.sq * b2;
    if (!J.rot) {
      b_L[2][c] = b2 + J.ys * b0 + J.zs * b1;
    } else {
      bJ.yy += b0 * L[0][c];
      bJ.zy += b1 * L[0][c];
      bJ.sy += b2 * L[0][c];
      bJ.ss += b2 * L[2][c];
      b_L[0][c] = J.yy * b0 + J.zy * b1 + J.sy * b2;
      b_L[2][c] = J.ys * b0 + J.zs * b1 + J.ss * b2;
    }
  }
}

// Reverse of predict_t<FIELD> (FIELD 0: uniform field, 1: the map): b_po =
// adjoint of the predicted state, bJ = adjoint of the Jacobian entries; b_pi
// receives the adjoint of the state before the step (t, q: its tan(lambda) and
// q/pt).  With the map the curvature depends on the step's midpoint, hence on
// y, z, s, t and on the offsets (yo, zo) of residual coordinates, whose
// adjoints go to b_yo, b_zo (zero without the map).
template <int FIELD = 0>
__device__ __forceinline__ void predict_rev(const GeoRef& G, const PredTape& tp, const Jac& J, float t, float q, const float b_po[5],
                                            const JacBar& bJ, float b_pi[5], float& b_yo, float& b_zo) {
  const float kappa = FIELD == 1 ? tp.kap : G.kappa;
  float b_kap = 0.0f;  // adjoint of the curvature per unit q/pt (map only)
  const float dx = tp.dx, s1 = tp.s1, s2 = tp.s2, ic1 = tp.ic1, ic2 = tp.ic2, Tm = tp.Tm, tt = tp.tt;
  float b_t = b_po[3], b_q = b_po[4], b_s2 = b_po[2];
  float b_s1 = 0.0f, b_dx = 0.0f, b_k = 0.0f, b_kdx = 0.0f, b_ic1 = 0.0f, b_ic2 = 0.0f, b_c1 = 0.0f, b_c2 = 0.0f;
  float b_Tm = 0.0f, b_tt = 0.0f, b_dl = 0.0f, b_w = 0.0f, b_rr = 0.0f;
  float bJys0 = bJ.ys, bJzs0 = bJ.zs;
  if (J.rot) {
    const float rr = J.ss;
    b_rr = bJ.ss + bJ.ys * tp.Jys0 + bJ.zs * tp.Jzs0;
    bJys0 = bJ.ys * rr;
    bJzs0 = bJ.zs * rr;
    b_k -= tp.sa * bJ.sy;
    b_t -= tp.sa * ic2 * bJ.zy;
    b_ic2 -= tp.sa * t * bJ.zy;
    b_s2 -= tp.sa * ic2 * bJ.yy;
    b_ic2 -= tp.sa * s2 * bJ.yy;
  }
  // Jsq = dx kappa ; Jzq = (t kappa) Lk
  b_dx += kappa * bJ.sq;
  b_t += kappa * tp.Lk * bJ.zq;
  const float b_Lk = t * kappa * bJ.zq;
  if (FIELD == 1) b_kap += tp.dx * bJ.sq + (t * tp.Lk) * bJ.zq;
  if (tp.series) {
    const float i2 = ic1 * ic1, i3 = i2 * ic1, i5 = i3 * i2, i7 = i5 * i2, s1s = s1 * s1;
    const float a1 = (s1 * i3) * 0.5f;
    const float a2 = ((1.0f + 2.0f * s1s) * i5) * static_cast<float>(1.0 / 3.0);
#if TPCFIT_DET
    const float a3 = ((s1 * (3.0f + 2.0f * s1s)) * i7) * 0.125f;
#else
    const float a3 = 0.0f;  // the fast forward keeps two terms of the series
#endif
    const float kdx = tp.kdx, Q = a2 + kdx * a3, P = a1 + kdx * Q;
    b_dx += 2.0f * dx * P * b_Lk;
    const float b_P = dx * dx * b_Lk;
    const float b_a1 = b_P;
    b_kdx += Q * b_P;
    const float b_Q = kdx * b_P;
    const float b_a2 = b_Q;
    b_kdx += a3 * b_Q;
    const float b_a3 = kdx * b_Q;
    float b_s1s = 0.0f, b_i2 = 0.0f, b_i3 = 0.0f, b_i5 = 0.0f, b_i7 = 0.0f;
    b_s1 += 0.5f * i3 * b_a1;
    b_i3 += 0.5f * s1 * b_a1;
    b_s1s += static_cast<float>(2.0 / 3.0) * i5 * b_a2;
    b_i5 += (1.0f + 2.0f * s1s) * static_cast<float>(1.0 / 3.0) * b_a2;
    b_s1 += 0.125f * (3.0f + 2.0f * s1s) * i7 * b_a3;
    b_s1s += 0.25f * s1 * i7 * b_a3;
    b_i7 += 0.125f * s1 * (3.0f + 2.0f * s1s) * b_a3;
    b_s1 += 2.0f * s1 * b_s1s;
    b_i5 += i2 * b_i7;
    b_i2 += i5 * b_i7;
    b_i3 += i2 * b_i5;
    b_i2 += i3 * b_i5;
    b_i2 += ic1 * b_i3;
    b_ic1 += i2 * b_i3;
    b_ic1 += 2.0f * ic1 * b_i2;
  } else {
    const float k = tp.k;
    const float b_D = b_Lk / k;
    b_k -= tp.Lk / k * b_Lk;
    b_dx += ic2 * b_D;
    b_ic2 += dx * b_D;
    b_dl -= b_D;
  }
  b_dl += bJ.zt;  // Jzt = dl
  {  // Jzs0 = (t dx) (Tm (ic1 ic2))
    const float E = ic1 * ic2, F = Tm * E, G = t * dx;
    const float b_G = F * bJzs0, b_F = G * bJzs0, b_E = Tm * b_F;
    b_Tm += E * b_F;
    b_ic1 += ic2 * b_E;
    b_ic2 += ic1 * b_E;
    b_t += dx * b_G;
    b_dx += t * b_G;
  }
  {  // Jyq = ((dx kappa) dx) (tt (ic2 / 2))
    const float M = (dx * kappa) * dx;
    b_dx += 2.0f * kappa * dx * (tt * (ic2 * 0.5f)) * bJ.yq;
    b_tt += ic2 * 0.5f * M * bJ.yq;
    b_ic2 += tt * 0.5f * M * bJ.yq;
    if (FIELD == 1) b_kap += (dx * dx) * (tt * (ic2 * 0.5f)) * bJ.yq;
  }
  {  // Jys0 = (dx tt) ((ic1 + ic2) / 2)
    const float Hh = (ic1 + ic2) * 0.5f;
    b_dx += tt * Hh * bJys0;
    b_tt += dx * Hh * bJys0;
    b_ic1 += 0.5f * dx * tt * bJys0;
    b_ic2 += 0.5f * dx * tt * bJys0;
  }
  b_Tm += 2.0f * Tm * b_tt;  // tt = 1 + Tm^2
  // z2 = z1 + t dl ; y2 = y1 + dx Tm
  b_t += tp.dl * b_po[1];
  b_dl += t * b_po[1];
  b_dx += Tm * b_po[0];
  b_Tm += dx * b_po[0];
  // dl = (dx w) A ; A = asinc(sig) ; sig = kdx w
  const float b_A = dx * tp.w * b_dl;
  b_dx += tp.w * tp.A * b_dl;
  b_w += dx * tp.A * b_dl;
  const float b_sig = asinc_deriv(tp.sig) * b_A;
  b_kdx += tp.w * b_sig;
  b_w += tp.kdx * b_sig;
  // w = c1 + s1 Tm
  b_c1 += b_w;
  b_s1 += Tm * b_w;
  b_Tm += s1 * b_w;
  // Tm = (s1 + s2) / den, den = c1 + c2
  const float b_num = b_Tm / tp.den;
  const float b_den = -Tm * b_Tm / tp.den;
  b_s1 += b_num;
  b_s2 += b_num;
  b_c1 += b_den;
  b_c2 += b_den;
  // (c, 1/c) = sqrt_and_inv(u), u = (1 - s)(1 + s)
  const float b_u2 = 0.5f * ic2 * (b_c2 - ic2 * ic2 * b_ic2);
  const float b_u1 = 0.5f * ic1 * (b_c1 - ic1 * ic1 * b_ic1);
  b_s2 -= 2.0f * s2 * b_u2;
  b_s1 -= 2.0f * s1 * b_u1;
  // s2 = s1 + kdx ; kdx = k dx ; k = q kappa
  b_s1 += b_s2;
  b_kdx += b_s2;
  b_k += dx * b_kdx;
  b_dx += tp.k * b_kdx;
  b_q += kappa * b_k;
  // the map: kappa = kappa0 (1 + f_r (xm^2 + ym^2) + f_z zm^2) at the midpoint of
  // a straight half step, xm = x1 + dx/2, ym = (yo + y1) + (dx/2) s1/c1,
  // zm = (zo + z1) + (dx/2) t/c1
  float b_y1 = b_po[0], b_z1 = b_po[1], b_xm = 0.0f;
  b_yo = 0.0f;
  b_zo = 0.0f;
  if (FIELD == 1) {
    b_kap += q * b_k;
    const float k0 = 2.0f * G.kappa;
    b_xm = (k0 * G.f_r) * tp.xm * b_kap;
    const float b_ym = (k0 * G.f_r) * tp.ym * b_kap;
    const float b_zm = (k0 * G.f_z) * tp.zm * b_kap;
    const float hdx = 0.5f * dx, ic1c = ic1 * ic1 * ic1;
    b_yo = b_ym;
    b_zo = b_zm;
    b_y1 += b_ym;
    b_z1 += b_zm;
    b_t += (hdx * ic1) * b_zm;
    b_s1 += hdx * ic1c * (b_ym + (t * s1) * b_zm);  // d(s/c)/ds = 1/c^3, d(1/c)/ds = s/c^3
    b_dx += 0.5f * (b_xm + (s1 * ic1) * b_ym + (t * ic1) * b_zm);
  }
  // dx = X - x1
  const float b_x1 = b_xm - b_dx;
  if (J.rot) {
    // x1 = x ca + y sa ; y1 = y ca - x sa ; s1 = s ca - c sa ; cr = c ca + s sa ;
    // rr = cr / c ; c = sqrt((1 - s)(1 + s))
    const float rr = J.ss;
    const float b_cr = b_rr / tp.c;
    float b_c = -rr * b_rr / tp.c;
    b_pi[0] = tp.sa * b_x1 + tp.ca * b_y1;
    float b_s = tp.ca * b_s1;
    b_c -= tp.sa * b_s1;
    b_c += tp.ca * b_cr;
    b_s += tp.sa * b_cr;
    b_s -= (tp.s / tp.c) * b_c;
    b_pi[2] = b_s;
  } else {
    b_pi[0] = b_y1;
    b_pi[2] = b_s1;
  }
  b_pi[1] = b_z1;
  b_pi[3] = b_t;
  b_pi[4] = b_q;
}

// ---------------------------------------------------------------- backward kernel
struct StepState {
  float p[5];
  float L[5][5];
  float x;
  int sec;
};

__device__ __forceinline__ void load_ckpt(const float* src, StepState& S) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float v[32];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float4 f = __ldg(s4 + j);
    v[4 * j] = f.x;
    v[4 * j + 1] = f.y;
    v[4 * j + 2] = f.z;
    v[4 * j + 3] = f.w;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) S.p[c] = v[c];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) S.L[i][c] = v[5 + 5 * i + c];
  S.x = v[30];
  S.sec = __float_as_int(v[31]);
}

// A checkpoint of the U-D fit, loaded as if it held L (u in rows 0-1, d in
// row 2): turned into the square-root factor L = U sqrt(D), upper triangular.
__device__ __forceinline__ void sqrt_from_ud_ckpt(StepState& S) {
  float u[10], sd[5];
#pragma unroll
  for (int e = 0; e < 10; ++e) u[e] = S.L[e / 5][e % 5];
#pragma unroll
  for (int c = 0; c < 5; ++c) sd[c] = sqrtf(S.L[2][c]);
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) S.L[i][c] = c < i ? 0.0f : (c == i ? sd[c] : u[4 * i - (i * (i - 1)) / 2 + (c - i - 1)] * sd[c]);
}

// One cluster as stored (y, z, packed row/sector), loaded ahead of its use.
struct HitRaw {
  float y, z;
  int rs;
};

__device__ __forceinline__ HitRaw load_hit(const float* y, const float* z, const uint16_t* rowsec, int h) {
  HitRaw r;
  r.y = __ldg(y + h);
  r.z = __ldg(z + h);
  r.rs = (int)__ldg(rowsec + h);
  return r;
}
__device__ __forceinline__ HitRaw load_hit(const BwdArgs& a, int h) { return load_hit(a.y, a.z, a.rowsec, h); }

// Measurement (alignment subtracted), row and sector of a loaded cluster.  Row
// and sector are clamped into the table: the recorded fit has validated them,
// the clamp only keeps a mismatched call inside shared memory.
__device__ __forceinline__ void decode_hit(const float* align, const HitRaw& r, float& m0, float& m1, int& row,
                                           int& sec) {
  row = min(r.rs >> 6, kMaxRows - 1);
  sec = min(r.rs & 63, kNSectors - 1);
  const float2 d = reinterpret_cast<const float2*>(align)[sec * kMaxRows + row];
  m0 = r.y - d.x;
  m1 = r.z - d.y;
}

// States between checkpoints: 8 float4 (p 5, L 25, x, sector bits), stored
// lane-interleaved ([float4 j][lane]) so that a warp's stores and copies coalesce.
constexpr int kStateF4 = 8;

__device__ __forceinline__ void pack_state(const StepState& S, float v[32]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) v[c] = S.p[c];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) v[5 + 5 * i + c] = S.L[i][c];
  v[30] = S.x;
  v[31] = __int_as_float(S.sec);
}

__device__ __forceinline__ void unpack_state(const float v[32], StepState& S) {
#pragma unroll
  for (int c = 0; c < 5; ++c) S.p[c] = v[c];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) S.L[i][c] = v[5 + 5 * i + c];
  S.x = v[30];
  S.sec = __float_as_int(v[31]);
}

// dst[j * kWarp] = float4 j of the state (dst already offset by the lane).
__device__ __forceinline__ void store_state(float4* dst, const StepState& S) {
  float v[32];
  pack_state(S, v);
#pragma unroll
  for (int j = 0; j < kStateF4; ++j) dst[j * kWarp] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// The same read, but never merged with an earlier one: the state is read again
// from shared memory where it is needed instead of being kept in registers.
__device__ __forceinline__ float4 lds_volatile(const float4* p) {
  float4 r;
  asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return r;
}

__device__ __forceinline__ void reread_state(const float4* src, StepState& S) {
  float v[32];
#pragma unroll
  for (int j = 0; j < kStateF4; ++j) {
    const float4 f = lds_volatile(src + j * kWarp);
    v[4 * j] = f.x;
    v[4 * j + 1] = f.y;
    v[4 * j + 2] = f.z;
    v[4 * j + 3] = f.w;
  }
  unpack_state(v, S);
}

__device__ __forceinline__ void read_state(const float4* src, StepState& S) {
  float v[32];
#pragma unroll
  for (int j = 0; j < kStateF4; ++j) {
    const float4 f = src[j * kWarp];
    v[4 * j] = f.x;
    v[4 * j + 1] = f.y;
    v[4 * j + 2] = f.z;
    v[4 * j + 3] = f.w;
  }
  unpack_state(v, S);
}

// Asynchronous 16-byte global -> shared copies (L2 only, no L1 allocation).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

// One lane's state: F4 float4 from a lane-interleaved global slot into its
// lane-interleaved shared slot, as one commit group.
template <int F4 = kStateF4>
__device__ __forceinline__ void fetch_state(float4* sdst, const float4* gsrc) {
#pragma unroll
  for (int j = 0; j < F4; ++j) cp_async16(sdst + j * kWarp, gsrc + j * kWarp);
  cp_async_commit();
}

// A checkpoint (32 contiguous floats, 16-byte aligned: the
// state) into a lane-interleaved shared slot, as one commit group.
__device__ __forceinline__ void fetch_ckpt(float4* sdst, const float* ck) {
  const float4* g = reinterpret_cast<const float4*>(ck);
#pragma unroll
  for (int j = 0; j < kStateF4; ++j) cp_async16(sdst + j * kWarp, g + j);
  cp_async_commit();
}

// Forward of one step on a StepState (the same operations as the fit, in
// residual coordinates).  my, mz: measurement of the previous cluster on
// entry, of this cluster on exit.  conv: the first step of the outward pass,
// whose state is the seed in absolute coordinates.
// MAT: the material layers of the rows; FIELD as for predict_t (the smoother
// follows both; the adjoint runs without either).
template <bool MAT = false, int FIELD = 0>
__device__ __forceinline__ void step_fwd(const GeoRef& G, const SmemTables& T, StepState& S, float& my, float& mz, bool first, bool conv,
                                         int row, int sec18, float m0, float m1) {
  float chi2 = 0.0f;
  if (first) {
    S.x = T.row_x[row];
    S.sec = sec18;
    if (conv) {
      S.p[0] = S.p[0] - m0;
      S.p[1] = S.p[1] - m1;
    }
  } else {
    float pn[5];
    Jac J;
    PredTape tp;
    MatNoise N;
    if (MAT && !conv) {  // inward: the layer of the row left
      material_step(G, S.p, -1, N);
      material_factor(S.L, N);
    }
    predict_residual<FIELD>(G, T, S.p, S.x, S.sec, my, mz, sec18, T.row_x[row], m0, m1, pn, J, tp);
    if (MAT && conv) material_step(G, pn, 1, N);
#pragma unroll
    for (int c = 0; c < 5; ++c) S.p[c] = pn[c];
    S.x = T.row_x[row];
    S.sec = sec18;
    transport(S.L, J);
    if (MAT && conv) material_factor(S.L, N);
  }
  my = m0;
  mz = m1;
  scalar_update<0>(G, S.p, S.L, chi2, 0.0f);
  scalar_update<1>(G, S.p, S.L, chi2, 0.0f);
}

// Reverse of one step from the state before it, which sits in shared memory
// at src ([float4 j][lane]; read twice so that it need not stay in registers
// through the update reverses).  my_prev, mz_prev: measurement of the previous
// cluster.  b_p, b_L: in = adjoint after the step, out = adjoint before it.
// The measurements enter only through the residual shifts: b_mc = adjoint of
// this cluster's (y, z), b_mp = of the previous one's.
template <int FIELD = 0>
__device__ __forceinline__ void step_rev(const GeoRef& G, const SmemTables& T, const float4* src, float my_prev, float mz_prev,
                                         bool first, bool conv, int row, int sec18, float m0, float m1, float b_p[5],
                                         float b_L[5][5], float b_chi, float b_mc[2], float b_mp[2]) {
  StepState S0;
  read_state(src, S0);
  float p1[5];
  Jac J;
  float L[5][5];
  PredTape tp;
  if (first) {
#pragma unroll
    for (int c = 0; c < 5; ++c) p1[c] = S0.p[c];
    if (conv) {
      p1[0] = S0.p[0] - m0;
      p1[1] = S0.p[1] - m1;
    }
  } else {
    predict_residual<FIELD>(G, T, S0.p, S0.x, S0.sec, my_prev, mz_prev, sec18, T.row_x[row], m0, m1, p1, J, tp);
  }
  // the factor before the y update (kept) and before the z update
  float p2[5];
  float chi_dummy = 0.0f, b_dummy = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) p2[c] = p1[c];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) L[i][c] = S0.L[i][c];
  if (!first) transport(L, J);
  float L2[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) L2[i][c] = L[i][c];
  scalar_update<0>(G, p2, L2, chi_dummy, 0.0f);
  scalar_update_rev<1>(G, p2, L2, 0.0f, b_p, b_L, b_chi, b_dummy);
  scalar_update_rev<0>(G, p1, L, 0.0f, b_p, b_L, b_chi, b_dummy);
  // b_p is now the adjoint of the predicted (shifted) state p1
  b_mc[0] = -b_p[0];
  b_mc[1] = -b_p[1];
  b_mp[0] = 0.0f;
  b_mp[1] = 0.0f;
  if (first) {
    if (!conv) b_mc[0] = b_mc[1] = 0.0f;  // the inward pass starts from residuals already
    return;
  }
  reread_state(src, S0);
  JacBar bJ;
  transport_rev(S0.L, J, b_L, bJ);
  const bool rot = S0.sec != sec18;
  if (!rot) {
    b_mp[0] = b_p[0];
    b_mp[1] = b_p[1];
  }
  // the prediction's intermediates (tp, J) are those of the forward above
  float b_pi[5], b_yo, b_zo;
  predict_rev<FIELD>(G, tp, J, S0.p[3], S0.p[4], b_p, bJ, b_pi, b_yo, b_zo);
  if (rot) {
    b_mp[0] = b_pi[0];
    b_mp[1] = b_pi[1];
  } else if (FIELD == 1) {  // the map's midpoint sits at the previous cluster plus the residual
    b_mp[0] += b_yo;
    b_mp[1] += b_zo;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) b_p[c] = b_pi[c];
}

// Reverse of material_step for a step that was taken.  p: the state before it;
// b_p in: adjoint of the state after, out: of the state before; bN: adjoints of
// the terms it handed on (qq, b_s, b_t, b_q).  Only s, t and q enter.
__device__ __forceinline__ void material_step_rev(const GeoRef& G, const float p[5], int dir, const MatNoise& bN, float b_p[5]) {
  const float s = p[2], t = p[3], q = p[4];
  const float q2 = q * q;
  if (!(q2 > 0.0f)) return;  // no material effect: nothing depends on the state
  const float tt1 = 1.0f + t * t;
  const float c = sqrtf((1.0f - s) * (1.0f + s));
  const float st1 = sqrtf(tt1);
  const float ell = (G.d_row * st1) / c;
  const float p2 = tt1 / q2;
  const float e2 = p2 + G.mass2;
  const float kx = static_cast<float>(0.0136 * 0.0136) * G.x0_inv;
  const float ip2 = 1.0f / p2;
  const float th2 = (kx * ell) * (e2 * (ip2 * ip2));
  const float e = sqrtf(e2);
  const float de = (G.dedx * ell) * (e2 * ip2);
  const float en = dir > 0 ? e - de : e + de;
  const float pn2 = en * en - G.mass2;
  const float ratio = sqrtf(p2 / pn2);
  const float qo = q * ratio;
  const float th = sqrtf(th2);
  // b_s = th c st1, b_t = th tt1, b_q = th qo t, qq = ratio, q' = q ratio
  const float b_qo = b_p[4] + (bN.b_q * th) * t;
  float b_t = b_p[3] + (bN.b_q * th) * qo;
  const float b_th = (bN.b_s * c) * st1 + bN.b_t * tt1 + (bN.b_q * qo) * t;
  float b_c = (bN.b_s * th) * st1;
  float b_st1 = (bN.b_s * th) * c;
  float b_tt1 = bN.b_t * th;
  const float b_ratio = bN.qq + b_qo * q;
  float b_q = b_qo * ratio;
  const float b_th2 = th > 0.0f ? 0.5f * b_th / th : 0.0f;
  // ratio = sqrt(u), u = p2 / pn2; pn2 = en^2 - m^2; en = e -+ de; e = sqrt(e2)
  const float b_u = 0.5f * b_ratio / ratio;
  const float ipn2 = 1.0f / pn2;
  float b_p2 = b_u * ipn2;
  const float b_pn2 = -(b_u * (p2 * ipn2)) * ipn2;
  const float b_en = 2.0f * en * b_pn2;
  float b_e2 = 0.5f * b_en / e;
  const float b_de = dir > 0 ? -b_en : b_en;
  // de = (dedx ell) (e2 / p2); th2 = (kx ell) (e2 / p2^2); e2 = p2 + m^2
  float b_ell = (G.dedx * (e2 * ip2)) * b_de + (kx * (e2 * (ip2 * ip2))) * b_th2;
  b_e2 += ((G.dedx * ell) * ip2) * b_de + ((kx * ell) * (ip2 * ip2)) * b_th2;
  b_p2 -= ((G.dedx * ell) * (e2 * (ip2 * ip2))) * b_de + 2.0f * ((kx * ell) * (e2 * (ip2 * ip2 * ip2))) * b_th2;
  b_p2 += b_e2;
  // p2 = tt1 / q^2; ell = d st1 / c; st1 = sqrt(tt1); c = sqrt((1 - s)(1 + s)); tt1 = 1 + t^2
  b_tt1 += b_p2 / q2;
  b_q += 2.0f * q * (-(b_p2 * p2) / q2);
  b_st1 += (G.d_row / c) * b_ell;
  b_c -= (ell / c) * b_ell;
  b_tt1 += 0.5f * b_st1 / st1;
  b_t += 2.0f * t * b_tt1;
  b_p[2] = b_p[2] - (s / c) * b_c;
  b_p[3] = b_t;
  b_p[4] = b_q;
}

// Reverse of material_factor.  Lin: the factor it was given (row q not yet
// scaled by qq); F: the factor it returned, lower triangular with
// F F^T = M = G G^T + B B^T, G = diag(1, 1, 1, 1, qq) Lin, B the noise columns
// (b_s in row s; b_t, b_q in rows t, q).  bL in: adjoint of F (its lower
// triangle; the rest of F is structurally zero), out: adjoint of Lin; bN
// receives the adjoints of qq, b_s, b_t, b_q.  From dM = dF F^T + F dF^T with
// F^-1 dF lower triangular: F^-1 dF = Phi(F^-1 dM F^-T), Phi keeping the lower
// triangle with the diagonal halved, hence b_M = F^-T Phi(F^T b_F) F^-1, and
// b_G = (b_M + b_M^T) G, b_B = (b_M + b_M^T) B.  (The Householder arithmetic
// of the forward is not reversed step by step: this is the derivative of the
// map it computes.)
__device__ __forceinline__ void material_factor_rev(const float Lin[5][5], const MatNoise& N, const float F[5][5],
                                                    float bL[5][5], MatNoise& bN) {
  float Fi[5][5];  // F^-1, lower triangular
#pragma unroll
  for (int i = 0; i < 5; ++i) Fi[i][i] = 1.0f / F[i][i];
#pragma unroll
  for (int i = 1; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      float acc = F[i][j] * Fi[j][j];
#pragma unroll
      for (int k = j + 1; k < i; ++k) acc = acc + F[i][k] * Fi[k][j];
      Fi[i][j] = -(acc * Fi[i][i]);
    }
  // P = Phi(F^T b_F): P_ij = sum_{k >= i} F_ki bF_kj (i >= j), diagonal halved
  float P[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float acc = F[i][i] * bL[i][j];
#pragma unroll
      for (int k = i + 1; k < 5; ++k) acc = acc + F[k][i] * bL[k][j];
      P[i][j] = i == j ? 0.5f * acc : acc;
    }
  // T = P F^-1 (lower), then b_M = F^-T T
  float Tm[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float acc = P[i][j] * Fi[j][j];
#pragma unroll
      for (int k = j + 1; k <= i; ++k) acc = acc + P[i][k] * Fi[k][j];
      Tm[i][j] = acc;
    }
  float Sm[5][5];  // b_M + b_M^T
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int k0 = i > j ? i : j;
      float acc = Fi[k0][i] * Tm[k0][j];
#pragma unroll
      for (int k = k0 + 1; k < 5; ++k) acc = acc + Fi[k][i] * Tm[k][j];
      Sm[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const float v = Sm[i][j] + Sm[j][i];
      Sm[i][j] = v;
      Sm[j][i] = v;
    }
#pragma unroll
  for (int i = 0; i < 5; ++i) Sm[i][i] = 2.0f * Sm[i][i];
  // b_G = Sm G, G = D Lin
  float qsum = 0.0f;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      float acc = Sm[i][0] * Lin[0][c];
#pragma unroll
      for (int j = 1; j < 4; ++j) acc = acc + Sm[i][j] * Lin[j][c];
      acc = acc + Sm[i][4] * (N.qq * Lin[4][c]);
      if (i == 4) {
        qsum = qsum + Lin[4][c] * acc;
        bL[i][c] = N.qq * acc;
      } else {
        bL[i][c] = acc;
      }
    }
  bN.qq = qsum;
  bN.b_s = Sm[2][2] * N.b_s;
  bN.b_t = Sm[3][3] * N.b_t + Sm[3][4] * N.b_q;
  bN.b_q = Sm[4][3] * N.b_t + Sm[4][4] * N.b_q;
}

// step_rev with the material layers of the rows.  Outward (conv): prediction,
// layer crossed on arrival (material_step on the predicted state), transport,
// noise folded (material_factor), updates.  Inward: the layer of the row left
// undone first (on the state before the step), then prediction, transport and
// updates.  Arguments as for step_rev.
template <int FIELD = 0>
__device__ __forceinline__ void step_rev_mat(const GeoRef& G, const SmemTables& T, const float4* src, float my_prev, float mz_prev,
                                             bool first, bool conv, int row, int sec18, float m0, float m1,
                                             float b_p[5], float b_L[5][5], float b_chi, float b_mc[2],
                                             float b_mp[2]) {
  StepState S0;
  read_state(src, S0);
  float p1[5];   // the state the updates start from
  float pb[5];   // outward: predicted state before the layer; inward: S0.p after undoing it
  float Lb[5][5];  // outward: transported factor before the noise; inward: S0.L after the layer
  Jac J;
  float L[5][5];
  PredTape tp;
  MatNoise N;
  if (first) {
#pragma unroll
    for (int c = 0; c < 5; ++c) p1[c] = S0.p[c];
    if (conv) {
      p1[0] = S0.p[0] - m0;
      p1[1] = S0.p[1] - m1;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int c = 0; c < 5; ++c) L[i][c] = S0.L[i][c];
  } else if (conv) {
    predict_residual<FIELD>(G, T, S0.p, S0.x, S0.sec, my_prev, mz_prev, sec18, T.row_x[row], m0, m1, p1, J, tp);
#pragma unroll
    for (int c = 0; c < 5; ++c) pb[c] = p1[c];
    material_step(G, p1, 1, N);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int c = 0; c < 5; ++c) L[i][c] = S0.L[i][c];
    transport(L, J);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int c = 0; c < 5; ++c) Lb[i][c] = L[i][c];
    material_factor(L, N);
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) pb[c] = S0.p[c];
    material_step(G, pb, -1, N);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int c = 0; c < 5; ++c) Lb[i][c] = S0.L[i][c];
    material_factor(Lb, N);
    predict_residual<FIELD>(G, T, pb, S0.x, S0.sec, my_prev, mz_prev, sec18, T.row_x[row], m0, m1, p1, J, tp);
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int c = 0; c < 5; ++c) L[i][c] = Lb[i][c];
    transport(L, J);
  }
  float p2[5];
  float chi_dummy = 0.0f, b_dummy = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) p2[c] = p1[c];
  float L2[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) L2[i][c] = L[i][c];
  scalar_update<0>(G, p2, L2, chi_dummy, 0.0f);
  scalar_update_rev<1>(G, p2, L2, 0.0f, b_p, b_L, b_chi, b_dummy);
  scalar_update_rev<0>(G, p1, L, 0.0f, b_p, b_L, b_chi, b_dummy);
  // b_p: adjoint of the (shifted) state the updates started from; the layers
  // change only q, so its y, z entries are those of the prediction
  b_mc[0] = -b_p[0];
  b_mc[1] = -b_p[1];
  b_mp[0] = 0.0f;
  b_mp[1] = 0.0f;
  if (first) {
    if (!conv) b_mc[0] = b_mc[1] = 0.0f;
    return;
  }
  reread_state(src, S0);
  const bool rot = S0.sec != sec18;
  JacBar bJ;
  MatNoise bN;
  float b_pi[5], b_yo, b_zo;
  if (conv) {
    material_factor_rev(Lb, N, L, b_L, bN);
    material_step_rev(G, pb, 1, bN, b_p);
    if (!rot) {
      b_mp[0] = b_p[0];
      b_mp[1] = b_p[1];
    }
    transport_rev(S0.L, J, b_L, bJ);
    predict_rev<FIELD>(G, tp, J, S0.p[3], S0.p[4], b_p, bJ, b_pi, b_yo, b_zo);
  } else {
    if (!rot) {
      b_mp[0] = b_p[0];
      b_mp[1] = b_p[1];
    }
    transport_rev(Lb, J, b_L, bJ);
    predict_rev<FIELD>(G, tp, J, pb[3], pb[4], b_p, bJ, b_pi, b_yo, b_zo);
    material_factor_rev(S0.L, N, Lb, b_L, bN);
    material_step_rev(G, S0.p, -1, bN, b_pi);
  }
  if (rot) {
    b_mp[0] = b_pi[0];
    b_mp[1] = b_pi[1];
  } else if (FIELD == 1) {
    b_mp[0] += b_yo;
    b_mp[1] += b_zo;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) b_p[c] = b_pi[c];
}

}  // namespace TPCFIT_NS
}  // namespace tpcfit

#include "ud_core.cuh"

namespace tpcfit {
namespace TPCFIT_NS {

// Fire-and-forget global float add (no value returned, nothing to wait for).
// No kernel reads the sums back, so the add carries no ordering constraint
// (no memory clobber): the compiler may schedule other accesses around it.
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;\n" ::"l"(__cvta_generic_to_global(p)), "f"(v));
}
// The same for two adjacent floats at an 8-byte-aligned address (each element
// added atomically): half the atomic operations at the alignment table, whose
// keys several lanes hit at once.
__device__ __forceinline__ void red_add2(float* p, float v0, float v1) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};\n" ::"l"(__cvta_generic_to_global(p)), "f"(v0), "f"(v1));
}

// prev: what the inward pass left at cluster h (read ahead by the caller; only
// the outward pass, pass 0, adds to it).
__device__ __forceinline__ void accumulate_meas_grad(const BwdArgs& a, int pass, int h, int row, int sec, float g0,
                                                     float g1, float2 prev) {
  if (a.grad_meas) {
    float2* gm = reinterpret_cast<float2*>(a.grad_meas) + h;
    if (pass == 1) {
      *gm = make_float2(g0, g1);
    } else {
      *gm = make_float2(prev.x + g0, prev.y + g1);
    }
  }
  if (a.grad_align_atomic) {
    float* dst = a.grad_align_atomic + (sec * kMaxRows + row) * 2;
    if ((reinterpret_cast<uintptr_t>(dst) & 7u) == 0) {
      red_add2(dst, -g0, -g1);  // one atomic for the key's (dy, dz) pair
    } else {
      red_add(dst, -g0);
      red_add(dst + 1, -g1);
    }
  }
}

// Shared memory of a backward block: geometry tables, the alignment table
// and, per warp, a double buffer for the state before the step being reversed
// and a buffer for the next segment's checkpoint (all [float4 j][lane]).
struct BwdSmem {
  SmemTables T;
  float align[kAlignFloats];
};
// F4: float4 per stored state (kStateF4 for the square-root form, kUDStateF4
// for U-D); the checkpoint buffer always holds kStateF4.
template <int F4 = kStateF4>
struct BwdWarpBufsT {
  float4 st[2][F4][kWarp];
  float4 ck[kStateF4][kWarp];
};
using BwdWarpBufs = BwdWarpBufsT<>;

template <int WARPS, int FORM = 0>
constexpr size_t backward_smem_bytes() {
  return sizeof(BwdSmem) + WARPS * sizeof(BwdWarpBufsT<FORM ? kUDStateF4 : kStateF4>);
}

// Per track, per pass (inward reversed first), segment by segment from the
// last: recompute the segment from its checkpoint, storing the state before
// each step in the warp's global segment store; then reverse the steps, last
// first, each state copied into shared memory asynchronously one step ahead.
// Clusters are loaded one step ahead as well; the next segment's checkpoint
// is copied while the current segment is reversed.
// PHYS: bit 1 the material layers, bit 2 the field map.  FORM: the factor the
// segments are recomputed in, 0 the fit's square-root factor L, 1 U-D (no
// material layers; the checkpoint's L is converted where a segment starts).
template <int WARPS, int PHYS, int FORM = 0>
__global__ void __launch_bounds__(WARPS * 32, 1) backward_kernel(const __grid_constant__ BwdArgs a) {
  const GeoRef& G = a.geo;
  constexpr bool MAT = (PHYS & 1) != 0;
  constexpr int FIELD = (PHYS & 2) ? 1 : 0;
  static_assert(FORM == 0 || !MAT, "the U-D backward runs without material layers");
  constexpr int F4 = FORM ? kUDStateF4 : kStateF4;
  using State = typename std::conditional<FORM == 1, UDState, StepState>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& B = *reinterpret_cast<BwdSmem*>(smem_raw);
  load_tables(G, B.T);
  for (int i = threadIdx.x; i < kAlignFloats; i += blockDim.x) B.align[i] = __ldg(a.align + i);
  __syncthreads();
  const SmemTables& T = B.T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  BwdWarpBufsT<F4>& W = reinterpret_cast<BwdWarpBufsT<F4>*>(smem_raw + sizeof(BwdSmem))[warp];
  // this warp's segment store: [step kk][float4 j][lane]
  float4* const gs = a.seg + ((int64_t)blockIdx.x * WARPS + warp) * (kCkptEvery * F4 * kWarp) + lane;
  const int64_t n_chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t N = a.n_tracks;
#pragma unroll 1
  for (;;) {
    int64_t chunk = 0;
    if (lane == 0) chunk = (int64_t)atomicAdd(a.work, 1u);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= n_chunks) break;
    const int64_t slot = chunk * kWarp + lane;
    if (slot >= N) continue;
    const int32_t trk = a.perm ? a.perm[slot] : (int32_t)slot;
    const float g = __ldg(a.grad_chi2 + trk);
    const bool fitted = a.ndf[trk] > 0;
    float b_p[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (fitted) {
      const int begin = a.off[trk];
      const int last = a.ck_last[trk];
      float b_L[5][5];         // FORM 0: adjoint of the square-root factor
      float b_u[10], b_d[5];   // FORM 1: adjoint of the U-D factor
#pragma unroll 1
      for (int pass = 1; pass >= 0; --pass) {
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
          for (int c = 0; c < 5; ++c) b_L[i][c] = 0.0f;
#pragma unroll
        for (int e = 0; e < 10; ++e) b_u[e] = 0.0f;
#pragma unroll
        for (int c = 0; c < 5; ++c) b_d[c] = 0.0f;
        const float b_chi = pass == 1 ? g : 0.0f;
        const int steps = last + 1;
        const int nseg = (steps + kCkptEvery - 1) / kCkptEvery;
        // hit index of step i of this pass
        const int h0 = pass == 0 ? begin : begin + last;
        const int hd = pass == 0 ? 1 : -1;
        const float* ckp = a.ck + ((int64_t)pass * a.ck_slots + (begin >> kCkptShift) + trk) * kCkptFloats;
        float pend0 = 0.0f, pend1 = 0.0f;  // gradient owed to the measurement of the step before
        // the outward pass adds to the inward pass's gradient of each cluster:
        // that value is read one reversed step ahead
        const float2* const gmr = reinterpret_cast<const float2*>(a.grad_meas);
        const bool addg = pass == 0 && gmr != nullptr;
        float2 gnx = addg ? gmr[h0 + hd * (steps - 1)] : make_float2(0.0f, 0.0f);
        fetch_ckpt(&W.ck[0][lane], ckp + (int64_t)(nseg - 1) * kCkptFloats);
        // a segment's first cluster and the one before it, loaded a segment
        // ahead; pv: the reverse's previous cluster, carried across segments
        HitRaw seg_first = load_hit(a, h0 + hd * ((nseg - 1) * kCkptEvery));
        HitRaw seg_prev{};
        if (nseg > 1) seg_prev = load_hit(a, h0 + hd * ((nseg - 1) * kCkptEvery - 1));
        HitRaw pv{};
#pragma unroll 1
        for (int s = nseg - 1; s >= 0; --s) {
          const int i0 = s * kCkptEvery;
          const int cnt = min(kCkptEvery, steps - i0);
          State S;
          float my = 0.0f, mz = 0.0f;
          HitRaw nx = seg_first;
          if (i0 > 0) {
            int row, sec;
            decode_hit(B.align, seg_prev, my, mz, row, sec);
          }
          cp_async_wait<0>();
          if constexpr (FORM == 1) {
            StepState C;
            read_state(&W.ck[0][lane], C);
            ud_state_from(C, a.ck_form == 1, S);
          } else {
            read_state(&W.ck[0][lane], S);
          }
          // level 1: the segment, storing the state before each step
          float m0 = 0.0f, m1 = 0.0f;
          int row = 0, sec = 0;
#pragma unroll 1
          for (int kk = 0; kk < cnt; ++kk) {
            const int i = i0 + kk;
            const HitRaw cur = nx;
            if (kk + 1 < cnt) nx = load_hit(a, h0 + hd * (i + 1));
            decode_hit(B.align, cur, m0, m1, row, sec);
            store_state(gs + kk * (F4 * kWarp), S);
            if constexpr (FORM == 1)
              step_fwd_ud<FIELD>(G, T, S, my, mz, i == 0, pass == 0, row, side_sector(sec), m0, m1);
            else
              step_fwd<MAT, FIELD>(G, T, S, my, mz, i == 0, pass == 0, row, side_sector(sec), m0, m1);
          }
          // the states just stored are read back by this thread's copies below
          __threadfence_block();
          // the next segment's checkpoint travels while this one is reversed.
          // Copy groups complete in order, so it is committed after the
          // loop's first state copy: the first reverse step then waits only
          // for its own state (a one-step segment commits it here)
          const bool ck_next = s > 0;
          if (ck_next && cnt == 1) fetch_ckpt(&W.ck[0][lane], ckp + (int64_t)(s - 1) * kCkptFloats);
          // reverse; (m0, m1, row, sec) hold the segment's last cluster, which is
          // the current cluster of its last step; each step's previous cluster
          // becomes the current one of the step before it
          fetch_state<F4>(&W.st[(cnt - 1) & 1][0][lane], gs + (cnt - 1) * (F4 * kWarp));
          // (in later segments the reverse of the segment after this one left
          // this cluster in pv)
          if (s == nseg - 1 && i0 + cnt - 1 > 0) pv = load_hit(a, h0 + hd * (i0 + cnt - 2));
          if (s > 0) {
            seg_first = load_hit(a, h0 + hd * (i0 - kCkptEvery));
            if (i0 - kCkptEvery > 0) seg_prev = load_hit(a, h0 + hd * (i0 - kCkptEvery - 1));
          }
#pragma unroll 1
          for (int kk = cnt - 1; kk >= 0; --kk) {
            const int i = i0 + kk;
            const int h = h0 + hd * i;
            if (kk > 0) {
              fetch_state<F4>(&W.st[(kk - 1) & 1][0][lane], gs + (kk - 1) * (F4 * kWarp));
              if (ck_next && kk == cnt - 1) {
                fetch_ckpt(&W.ck[0][lane], ckp + (int64_t)(s - 1) * kCkptFloats);
                cp_async_wait<2>();
              } else {
                cp_async_wait<1>();
              }
            } else {
              cp_async_wait<0>();
            }
            float mpy = 0.0f, mpz = 0.0f;
            int prow = 0, psec = 0;
            if (i > 0) {
              const HitRaw pc = pv;
              if (i > 1) pv = load_hit(a, h - 2 * hd);
              decode_hit(B.align, pc, mpy, mpz, prow, psec);
            }
            const float2 gcur = gnx;
            if (addg && i > 0) gnx = gmr[h - hd];
            float b_mc[2], b_mp[2];
            if constexpr (FORM == 1) {
              step_rev_ud<FIELD>(G, T, &W.st[kk & 1][0][lane], mpy, mpz, T.row_x[prow], side_sector(psec), i == 0,
                                 pass == 0, row, side_sector(sec), m0, m1, b_p, b_u, b_d, b_chi,
                                 [&](float g0, float g1) {
                                   accumulate_meas_grad(a, pass, h, row, sec, g0 + pend0, g1 + pend1, gcur);
                                 },
                                 b_mp);
            } else {
              if (MAT)
                step_rev_mat<FIELD>(G, T, &W.st[kk & 1][0][lane], mpy, mpz, i == 0, pass == 0, row, side_sector(sec), m0,
                                    m1, b_p, b_L, b_chi, b_mc, b_mp);
              else
                step_rev<FIELD>(G, T, &W.st[kk & 1][0][lane], mpy, mpz, i == 0, pass == 0, row, side_sector(sec), m0, m1,
                                b_p, b_L, b_chi, b_mc, b_mp);
              accumulate_meas_grad(a, pass, h, row, sec, b_mc[0] + pend0, b_mc[1] + pend1, gcur);
            }
            pend0 = b_mp[0];
            pend1 = b_mp[1];
            m0 = mpy;
            m1 = mpz;
            row = prow;
            sec = psec;
          }
        }
        // the inward pass starts from the outward result with the factor reset:
        // b_p carries over, b_L does not
      }
    } else if (a.grad_meas) {
      const int begin = a.off[trk];
      const int end = a.off[trk + 1];
      for (int h = begin; h < end; ++h) reinterpret_cast<float2*>(a.grad_meas)[h] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) a.grad_seeds[(int64_t)c * N + trk] = b_p[c];
  }
}

// ---------------------------------------------------------------- the tape
// The backward in two kernels.  recompute_kernel replays every 16-step
// segment of both passes from its checkpoint (the fit's own arithmetic, at the
// fit's occupancy) and writes the state before each step to a tape in device
// memory.  tape_reverse_kernel then reverses the steps of each pass from the
// last, copying each state from the tape into shared memory one step ahead;
// it holds the reverse step's registers but does no forward work.
// Tape layout: [pass][32-track work item][step][float4 j][lane], kTapeSteps
// steps per work item, so that a warp's store or copy of float4 j of one step
// moves 512 contiguous bytes.  Both kernels map processing slot k to work
// item k / 32 and lane k % 32.  A track of more than kTapeSteps clusters (no
// valid track has more than one per pad row) gets no gradient.
constexpr int kTapeSteps = kMaxRows;

__host__ __device__ constexpr int64_t tape_float4s(int64_t n_tracks) {
  return 2 * ((n_tracks + kWarp - 1) / kWarp) * (int64_t)kTapeSteps * kStateF4 * kWarp;
}

// Float4 0 of step 0 of (pass, work item), offset by the lane.
__device__ __forceinline__ int64_t tape_base(int pass, int64_t chunk, int64_t n_chunks, int lane) {
  return (((int64_t)pass * n_chunks + chunk) * kTapeSteps) * (kStateF4 * kWarp) + lane;
}

constexpr int kRecomputeWarps = 24;

template <int PHYS>
__global__ void __launch_bounds__(kRecomputeWarps * 32, 1) recompute_kernel(const __grid_constant__ BwdArgs a) {
  const GeoRef& G = a.geo;
  constexpr bool MAT = (PHYS & 1) != 0;
  constexpr int FIELD = (PHYS & 2) ? 1 : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& B = *reinterpret_cast<BwdSmem*>(smem_raw);
  load_tables(G, B.T);
  for (int i = threadIdx.x; i < kAlignFloats; i += blockDim.x) B.align[i] = __ldg(a.align + i);
  __syncthreads();
  const SmemTables& T = B.T;
  const int lane = threadIdx.x & 31;
  const int64_t n_chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
#pragma unroll 1
  for (;;) {
    int64_t chunk = 0;
    if (lane == 0) chunk = (int64_t)atomicAdd(a.work, 1u);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= n_chunks) break;
    const int64_t slot = chunk * kWarp + lane;
    if (slot >= a.n_tracks) continue;
    const int32_t trk = a.perm ? a.perm[slot] : (int32_t)slot;
    if (a.ndf[trk] <= 0) continue;
    const int begin = a.off[trk];
    const int last = a.ck_last[trk];
    const int steps = last + 1;
    if (steps > kTapeSteps) continue;
    const int nseg = (steps + kCkptEvery - 1) / kCkptEvery;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int h0 = pass == 0 ? begin : begin + last;
      const int hd = pass == 0 ? 1 : -1;
      const float* ckp = a.ck + ((int64_t)pass * a.ck_slots + (begin >> kCkptShift) + trk) * kCkptFloats;
      float4* const tp = a.tape + tape_base(pass, chunk, n_chunks, lane);
#pragma unroll 1
      for (int s = 0; s < nseg; ++s) {
        const int i0 = s * kCkptEvery;
        const int cnt = min(kCkptEvery, steps - i0);
        StepState S;
        load_ckpt(ckp + (int64_t)s * kCkptFloats, S);
        if (a.ck_form == 1) sqrt_from_ud_ckpt(S);
        float my = 0.0f, mz = 0.0f;
        if (i0 > 0) {
          int row, sec;
          decode_hit(B.align, load_hit(a, h0 + hd * (i0 - 1)), my, mz, row, sec);
        }
        HitRaw nx = load_hit(a, h0 + hd * i0);
#pragma unroll 1
        for (int kk = 0; kk < cnt; ++kk) {
          const int i = i0 + kk;
          const HitRaw cur = nx;
          if (kk + 1 < cnt) nx = load_hit(a, h0 + hd * (i + 1));
          float m0, m1;
          int row, sec;
          decode_hit(B.align, cur, m0, m1, row, sec);
          store_state(tp + (int64_t)i * (kStateF4 * kWarp), S);
          step_fwd<MAT, FIELD>(G, T, S, my, mz, i == 0, pass == 0, row, side_sector(sec), m0, m1);
        }
      }
    }
  }
}

// The reverse of both passes from the tape (inward pass first); the same
// reverse steps, cluster loads and gradient accumulation as backward_kernel.
template <int WARPS, int PHYS>
__global__ void __launch_bounds__(WARPS * 32, 1) tape_reverse_kernel(const __grid_constant__ BwdArgs a) {
  const GeoRef& G = a.geo;
  constexpr bool MAT = (PHYS & 1) != 0;
  constexpr int FIELD = (PHYS & 2) ? 1 : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& B = *reinterpret_cast<BwdSmem*>(smem_raw);
  load_tables(G, B.T);
  for (int i = threadIdx.x; i < kAlignFloats; i += blockDim.x) B.align[i] = __ldg(a.align + i);
  __syncthreads();
  const SmemTables& T = B.T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  float4 (*const st)[kStateF4][kWarp] =
      reinterpret_cast<float4 (*)[kStateF4][kWarp]>(smem_raw + sizeof(BwdSmem)) + 2 * warp;
  const int64_t n_chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t N = a.n_tracks;
#pragma unroll 1
  for (;;) {
    int64_t chunk = 0;
    if (lane == 0) chunk = (int64_t)atomicAdd(a.work, 1u);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= n_chunks) break;
    const int64_t slot = chunk * kWarp + lane;
    if (slot >= N) continue;
    const int32_t trk = a.perm ? a.perm[slot] : (int32_t)slot;
    const float g = __ldg(a.grad_chi2 + trk);
    const bool fitted = a.ndf[trk] > 0;
    float b_p[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    const int begin = fitted ? a.off[trk] : 0;
    const int last = fitted ? a.ck_last[trk] : 0;
    if (fitted && last + 1 <= kTapeSteps) {
      float b_L[5][5];         // FORM 0: adjoint of the square-root factor
      float b_u[10], b_d[5];   // FORM 1: adjoint of the U-D factor
#pragma unroll 1
      for (int pass = 1; pass >= 0; --pass) {
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
          for (int c = 0; c < 5; ++c) b_L[i][c] = 0.0f;
#pragma unroll
        for (int e = 0; e < 10; ++e) b_u[e] = 0.0f;
#pragma unroll
        for (int c = 0; c < 5; ++c) b_d[c] = 0.0f;
        const float b_chi = pass == 1 ? g : 0.0f;
        const int steps = last + 1;
        const int h0 = pass == 0 ? begin : begin + last;
        const int hd = pass == 0 ? 1 : -1;
        const float4* const tp = a.tape + tape_base(pass, chunk, n_chunks, lane);
        float pend0 = 0.0f, pend1 = 0.0f;  // gradient owed to the measurement of the step before
        const float2* const gmr = reinterpret_cast<const float2*>(a.grad_meas);
        const bool addg = pass == 0 && gmr != nullptr;
        float2 gnx = addg ? gmr[h0 + hd * (steps - 1)] : make_float2(0.0f, 0.0f);
        fetch_state(&st[(steps - 1) & 1][0][lane], tp + (int64_t)(steps - 1) * (kStateF4 * kWarp));
        float m0, m1;
        int row, sec;
        decode_hit(B.align, load_hit(a, h0 + hd * (steps - 1)), m0, m1, row, sec);
        HitRaw pv{};
        if (steps > 1) pv = load_hit(a, h0 + hd * (steps - 2));
#pragma unroll 1
        for (int i = steps - 1; i >= 0; --i) {
          const int h = h0 + hd * i;
          if (i > 0) {
            fetch_state(&st[(i - 1) & 1][0][lane], tp + (int64_t)(i - 1) * (kStateF4 * kWarp));
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
          float mpy = 0.0f, mpz = 0.0f;
          int prow = 0, psec = 0;
          if (i > 0) {
            const HitRaw pc = pv;
            if (i > 1) pv = load_hit(a, h - 2 * hd);
            decode_hit(B.align, pc, mpy, mpz, prow, psec);
          }
          const float2 gcur = gnx;
          if (addg && i > 0) gnx = gmr[h - hd];
          float b_mc[2], b_mp[2];
          if (MAT)
            step_rev_mat<FIELD>(G, T, &st[i & 1][0][lane], mpy, mpz, i == 0, pass == 0, row, side_sector(sec), m0,
                                m1, b_p, b_L, b_chi, b_mc, b_mp);
          else
            step_rev<FIELD>(G, T, &st[i & 1][0][lane], mpy, mpz, i == 0, pass == 0, row, side_sector(sec), m0, m1,
                            b_p, b_L, b_chi, b_mc, b_mp);
          accumulate_meas_grad(a, pass, h, row, sec, b_mc[0] + pend0, b_mc[1] + pend1, gcur);
          pend0 = b_mp[0];
          pend1 = b_mp[1];
          m0 = mpy;
          m1 = mpz;
          row = prow;
          sec = psec;
        }
        // the inward pass starts from the outward result with the factor reset:
        // b_p carries over, b_L does not
      }
    } else if (a.grad_meas) {
      const int b = a.off[trk];
      const int end = a.off[trk + 1];
      for (int h = b; h < end; ++h) reinterpret_cast<float2*>(a.grad_meas)[h] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) a.grad_seeds[(int64_t)c * N + trk] = b_p[c];
  }
}

template <int WARPS>
constexpr size_t tape_reverse_smem_bytes() {
  return sizeof(BwdSmem) + (size_t)WARPS * 2 * kStateF4 * kWarp * sizeof(float4);
}

// Persistent launch of a kernel with `warps` warps per block and `smem` bytes
// of shared memory (the grid cached per kernel).
template <class K>
cudaError_t launch_persistent(K kernel, int& cached, int warps, size_t smem, const BwdArgs& a, cudaStream_t s) {
  if (cached == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cached = sms * per_sm;
  }
  const int64_t chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t need = (chunks + warps - 1) / warps;
  const int blocks = (int)(need < cached ? need : cached);
  cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  kernel<<<blocks, warps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int WARPS, int PHYS>
cudaError_t launch_tape_backward_cfg(const BwdArgs& a, cudaStream_t s) {
  static int g_rec = 0, g_rev = 0;
  cudaError_t e = launch_persistent(recompute_kernel<PHYS>, g_rec, kRecomputeWarps, sizeof(BwdSmem), a, s);
  if (e != cudaSuccess) return e;
  return launch_persistent(tape_reverse_kernel<WARPS, PHYS>, g_rev, WARPS, tape_reverse_smem_bytes<WARPS>(), a, s);
}

// Persistent grid of the backward (blocks resident at once over all SMs).
template <int WARPS, int PHYS, int FORM>
cudaError_t backward_grid(int& grid) {
  static int cached = 0;
  if (cached == 0) {
    constexpr int kThreads = WARPS * 32;
    const size_t smem = backward_smem_bytes<WARPS, FORM>();
    cudaError_t e = cudaFuncSetAttribute(backward_kernel<WARPS, PHYS, FORM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_kernel<WARPS, PHYS, FORM>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cached = sms * per_sm;
  }
  grid = cached;
  return cudaSuccess;
}

template <int WARPS, int PHYS, int FORM>
cudaError_t backward_store_cfg(int64_t& float4s) {
  int grid = 0;
  cudaError_t e = backward_grid<WARPS, PHYS, FORM>(grid);
  float4s = (int64_t)grid * WARPS * kCkptEvery * (FORM ? kUDStateF4 : kStateF4) * kWarp;
  return e;
}

template <int WARPS, int PHYS, int FORM>
cudaError_t launch_backward_cfg(const BwdArgs& a, cudaStream_t s) {
  int grid = 0;
  cudaError_t e = backward_grid<WARPS, PHYS, FORM>(grid);
  if (e != cudaSuccess) return e;
  const int64_t chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t need = (chunks + WARPS - 1) / WARPS;
  const int blocks = (int)(need < grid ? need : grid);
  e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  backward_kernel<WARPS, PHYS, FORM><<<blocks, WARPS * 32, backward_smem_bytes<WARPS, FORM>(), s>>>(a);
  return cudaGetLastError();
}

// Warps per block of a backward launch: the configured shape in a uniform
// field without material; the other physics run in the 8-warp shape only.
inline int backward_warps(int warps, int phys) { return phys ? 8 : warps; }

// One-kernel fast backward (no material layers): FORM 0 or 1 in every
// compiled block shape, uniform field (PHYS 0) or the field map (PHYS 2, 8
// warps).
template <int FORM>
cudaError_t backward_store_form(int warps, int phys, int64_t& float4s) {
  switch (phys) {
    case 0: break;
    case 2: return backward_store_cfg<8, 2, FORM>(float4s);
    default: return cudaErrorInvalidValue;
  }
  switch (warps) {
    case 4: return backward_store_cfg<4, 0, FORM>(float4s);
    case 8: return backward_store_cfg<8, 0, FORM>(float4s);
    case 10: return backward_store_cfg<10, 0, FORM>(float4s);
    case 12: return backward_store_cfg<12, 0, FORM>(float4s);
    default: return cudaErrorInvalidValue;
  }
}

template <int FORM>
cudaError_t launch_backward_form(const BwdArgs& a, int warps, cudaStream_t s) {
  switch (a.phys) {
    case 0: break;
    case 2: return launch_backward_cfg<8, 2, FORM>(a, s);
    default: return cudaErrorInvalidValue;
  }
  switch (warps) {
    case 4: return launch_backward_cfg<4, 0, FORM>(a, s);
    case 8: return launch_backward_cfg<8, 0, FORM>(a, s);
    case 10: return launch_backward_cfg<10, 0, FORM>(a, s);
    case 12: return launch_backward_cfg<12, 0, FORM>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

// Segment store (float4 count) the backward needs for `warps` warps per block,
// the physics bits phys (1: material layers, 2: the field map) and the factor
// form (0: square root, 1: U-D).
inline cudaError_t backward_store(int warps, int phys, int form, int64_t& float4s) {
  if (form == 1) return backward_store_form<1>(warps, phys, float4s);
  if (form == 0) return backward_store_form<0>(warps, phys, float4s);
  return cudaErrorInvalidValue;
}

// The deterministic backward always, and the fast one with material layers,
// replay the segments onto the tape (recompute_kernel + tape_reverse_kernel);
// the fast backward without material recomputes into the segment store
// (backward_kernel).
inline cudaError_t launch_tape_backward(const BwdArgs& a, int warps, cudaStream_t s) {
  switch (a.phys) {
    case 0: break;
    case 1: return launch_tape_backward_cfg<8, 1>(a, s);
#if TPCFIT_DET
    case 2: return launch_tape_backward_cfg<8, 2>(a, s);
#endif
    case 3: return launch_tape_backward_cfg<8, 3>(a, s);
    default: return cudaErrorInvalidValue;
  }
#if TPCFIT_DET
  switch (warps) {
    case 4: return launch_tape_backward_cfg<4, 0>(a, s);
    case 8: return launch_tape_backward_cfg<8, 0>(a, s);
    case 10: return launch_tape_backward_cfg<10, 0>(a, s);
    case 12: return launch_tape_backward_cfg<12, 0>(a, s);
    default: return cudaErrorInvalidValue;
  }
#else
  (void)warps;
  return cudaErrorInvalidValue;
#endif
}

inline cudaError_t launch_backward(const BwdArgs& a, int warps, cudaStream_t s) {
  if (a.n_tracks <= 0) return cudaSuccess;
  if (a.tape) return launch_tape_backward(a, warps, s);
#if TPCFIT_DET
  return cudaErrorInvalidValue;
#else
  if (a.form == 1) return launch_backward_form<1>(a, warps, s);
  if (a.form == 0) return launch_backward_form<0>(a, warps, s);
  return cudaErrorInvalidValue;
#endif
}

}  // namespace TPCFIT_NS
}  // namespace tpcfit
