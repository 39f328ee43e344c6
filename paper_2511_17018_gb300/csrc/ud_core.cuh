// The backward's recomputation and reverse in U-D form (the forward pieces are
// in ud_filter.cuh).  Included by adjoint_core.cuh ahead of the backward
// kernels (both modules compile it; only the fast one launches it).
//
// The backward may recompute a segment in any factorisation of the same
// covariance: the adjoint of the objective depends on the covariance, not on
// its factor.  A segment starts from the fit's checkpoint: the U-D fit's
// (p, U, D) as they are, or the square-root fit's (p, L), whose rows,
// orthogonalised with unit weights, give U and D.  That conversion needs no
// reverse: the U-D factorisation of a covariance is unique, so the
// adjoint that reaches a segment's first state is the adjoint of the state
// the segment before it ends with, and the factor's adjoint is dropped where
// a pass starts from a fixed prior.
#pragma once

#include <type_traits>

namespace tpcfit {
namespace TPCFIT_NS {

struct UDState {
  float p[5];
  float u[10];
  float d[5];
  float x;
  int sec;
};

// States between checkpoints in U-D form: 5 float4 (p 5, u 10, d 5),
// lane-interleaved like the square-root states.  x and the sector of a stored
// state are those of the cluster before the step, which the reverse decodes
// anyway, so they are not stored.
constexpr int kUDStateF4 = 5;

// (U, D) of C = L L^T: the rows of L orthogonalised last first with unit
// weights, d_k = |w_k|^2, u_ik = (w_i . w_k) / d_k, w_i -= u_ik w_k.
__device__ __forceinline__ void ud_from_sqrt(const float L[5][5], float u[10], float d[5]) {
  float w[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) w[i][c] = L[i][c];
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    float s = w[k][0] * w[k][0];
#pragma unroll
    for (int c = 1; c < 5; ++c) s = s + w[k][c] * w[k][c];
    d[k] = s;
    const float is = ud_rcp(s);
#pragma unroll
    for (int i = 0; i < k; ++i) {
      float t = w[i][0] * w[k][0];
#pragma unroll
      for (int c = 1; c < 5; ++c) t = t + w[i][c] * w[k][c];
      t = t * is;
      u[ui(i, k)] = t;
#pragma unroll
      for (int c = 0; c < 5; ++c) w[i][c] = w[i][c] - t * w[k][c];
    }
  }
}

// Reverse of transport_ud: u = the factor before it; b_u in = adjoint after,
// out = before; bJ accumulates the Jacobian's adjoint.
__device__ __forceinline__ void transport_ud_rev(const float u[10], const Jac& J, float b_u[10], JacBar& bJ) {
  const float b04 = b_u[ui(0, 4)], b03 = b_u[ui(0, 3)], b02 = b_u[ui(0, 2)];
  const float b14 = b_u[ui(1, 4)], b13 = b_u[ui(1, 3)], b12 = b_u[ui(1, 2)], b24 = b_u[ui(2, 4)];
  bJ.ys += (b02 + u[ui(2, 3)] * b03) + u[ui(2, 4)] * b04;
  bJ.yq += b04;
  bJ.zs += (b12 + u[ui(2, 3)] * b13) + u[ui(2, 4)] * b14;
  bJ.zt += b13 + u[ui(3, 4)] * b14;
  bJ.zq += b14;
  bJ.sq += b24;
  b_u[ui(2, 3)] += J.ys * b03 + J.zs * b13;
  b_u[ui(2, 4)] += J.ys * b04 + J.zs * b14;
  b_u[ui(3, 4)] += J.zt * b14;
}

// Reverse of rotate_ud: u, d = the factor before it; b_u, b_d in = adjoint
// after, out = before; bJ accumulates.
__device__ __forceinline__ void rotate_ud_rev(const float u[10], const float d[5], const Jac& J, float b_u[10],
                                              float b_d[5], JacBar& bJ) {
  const RotW W = rot_w(u, J);
  const float e2 = wdot3(d, W.w[2], W.w[2]);
  const float i2 = ud_rcp(e2);
  const float n02 = wdot3(d, W.w[0], W.w[2]);
  const float n12 = wdot3(d, W.w[1], W.w[2]);
  const float a02 = n02 * i2, a12 = n12 * i2;
  float x0[3], x1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x0[c] = W.w[0][c] - a02 * W.w[2][c];
    x1[c] = W.w[1][c] - a12 * W.w[2][c];
  }
  const float e1 = wdot3(d, x1, x1);
  const float i1 = ud_rcp(e1);
  const float n01 = wdot3(d, x0, x1);
  const float a01 = n01 * i1;
  float y0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) y0[c] = x0[c] - a01 * x1[c];
  // adjoints of the leading block's outputs
  const float bE0 = b_d[0], bE1 = b_d[1], bE2 = b_d[2];
  float bd[3], by0[3], bx0[3], bx1[3], bw0[3], bw1[3], bw2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    by0[c] = 2.0f * (d[c] * y0[c]) * bE0;
    bd[c] = (y0[c] * y0[c]) * bE0;
  }
  float ba01 = b_u[ui(0, 1)];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bx0[c] = by0[c];
    ba01 -= by0[c] * x1[c];
    bx1[c] = -a01 * by0[c];
  }
  const float bn01 = i1 * ba01;
  const float bi1 = n01 * ba01;
  const float be1 = bE1 - (i1 * i1) * bi1;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bx0[c] += (d[c] * x1[c]) * bn01;
    bx1[c] += (d[c] * x0[c]) * bn01 + 2.0f * (d[c] * x1[c]) * be1;
    bd[c] += (x0[c] * x1[c]) * bn01 + (x1[c] * x1[c]) * be1;
  }
  float ba12 = b_u[ui(1, 2)], ba02 = b_u[ui(0, 2)];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bw1[c] = bx1[c];
    bw0[c] = bx0[c];
    ba12 -= bx1[c] * W.w[2][c];
    ba02 -= bx0[c] * W.w[2][c];
    bw2[c] = -a12 * bx1[c] - a02 * bx0[c];
  }
  const float bn12 = i2 * ba12, bn02 = i2 * ba02;
  const float bi2 = n12 * ba12 + n02 * ba02;
  const float be2 = bE2 - (i2 * i2) * bi2;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bw1[c] += (d[c] * W.w[2][c]) * bn12;
    bw0[c] += (d[c] * W.w[2][c]) * bn02;
    bw2[c] += (d[c] * W.w[1][c]) * bn12 + (d[c] * W.w[0][c]) * bn02 + 2.0f * (d[c] * W.w[2][c]) * be2;
    bd[c] += (W.w[1][c] * W.w[2][c]) * bn12 + (W.w[0][c] * W.w[2][c]) * bn02 + (W.w[2][c] * W.w[2][c]) * be2;
  }
  // W = J U, leading block
  const float u01 = u[ui(0, 1)], u02 = u[ui(0, 2)];
  bJ.yy += (bw0[0] + u01 * bw0[1]) + u02 * bw0[2];
  bJ.ys += bw0[2];
  bJ.zy += (bw1[0] + u01 * bw1[1]) + u02 * bw1[2];
  bJ.zs += bw1[2];
  bJ.sy += (bw2[0] + u01 * bw2[1]) + u02 * bw2[2];
  bJ.ss += bw2[2];
  const float c03 = b_u[ui(0, 3)], c04 = b_u[ui(0, 4)], c13 = b_u[ui(1, 3)], c14 = b_u[ui(1, 4)];
  const float c23 = b_u[ui(2, 3)], c24 = b_u[ui(2, 4)], c34 = b_u[ui(3, 4)];
  const float u03 = u[ui(0, 3)], u04 = u[ui(0, 4)], u23 = u[ui(2, 3)], u24 = u[ui(2, 4)], u34 = u[ui(3, 4)];
  b_u[ui(0, 1)] = (J.yy * bw0[1] + J.zy * bw1[1]) + J.sy * bw2[1];
  b_u[ui(0, 2)] = (J.yy * bw0[2] + J.zy * bw1[2]) + J.sy * bw2[2];
  b_u[ui(1, 2)] = bw1[2];
  // columns 3 and 4
  bJ.yy += u03 * c03 + u04 * c04;
  bJ.ys += u23 * c03 + u24 * c04;
  bJ.yq += c04;
  bJ.zy += u03 * c13 + u04 * c14;
  bJ.zs += u23 * c13 + u24 * c14;
  bJ.zt += c13 + u34 * c14;
  bJ.zq += c14;
  bJ.sy += u03 * c23 + u04 * c24;
  bJ.ss += u23 * c23 + u24 * c24;
  bJ.sq += c24;
  b_u[ui(0, 3)] = (J.yy * c03 + J.zy * c13) + J.sy * c23;
  b_u[ui(0, 4)] = (J.yy * c04 + J.zy * c14) + J.sy * c24;
  b_u[ui(1, 3)] = c13;
  b_u[ui(1, 4)] = c14;
  b_u[ui(2, 3)] = (J.ys * c03 + J.zs * c13) + J.ss * c23;
  b_u[ui(2, 4)] = (J.ys * c04 + J.zs * c14) + J.ss * c24;
  b_u[ui(3, 4)] = c34 + J.zt * c14;
#pragma unroll
  for (int c = 0; c < 3; ++c) b_d[c] = bd[c];
}

// Reverse of bierman_update<H>.  p, u, d: the state before the update; b_p,
// b_u, b_d: in = adjoint after, out = before; b_chi: adjoint of chi2.
template <int H>
__device__ __forceinline__ void bierman_update_rev(const float p[5], const float u[10], const float d[5], float v,
                                                   float b_p[5], float b_u[10], float b_d[5], float b_chi) {
  float al[5], ial[5], gv[5];
  float ap = v;
#pragma unroll
  for (int j = 0; j < 5; ++j) gv[j] = j < H ? 0.0f : (j == H ? d[j] : d[j] * u[ui(H, j)]);
#pragma unroll
  for (int j = H; j < 5; ++j) {
    const float f = j == H ? 1.0f : u[ui(H, j)];
    al[j] = j == H ? ap + gv[j] : ap + f * gv[j];
    ial[j] = ud_rcp(al[j]);
    ap = al[j];
  }
  // K_i before column j: g_i + sum over H <= k < j, k > i of u_ik g_k, summed
  // in the forward's order.  (Taking it back from the final K by subtraction
  // cancels where the partial sum is small against its terms, and the
  // seeds' gradient, which the diffuse prior makes ~1e-5 of the clusters',
  // loses its digits there.)
  auto k_before = [&](int i, int j) {
    float acc = gv[i];
#pragma unroll
    for (int k = (i + 1 > H ? i + 1 : H); k < j; ++k) acc = acc + u[ui(i, k)] * gv[k];
    return acc;
  };
  float K[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) K[i] = k_before(i, 5);
  const float r = -p[H];
  const float q = r * ial[4];
  float bK[5];
  float bqo = r * b_chi;  // the adjoint of q without the K_H b_p[H] term
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    bK[i] = q * b_p[i];
    if (i != H) bqo = bqo + K[i] * b_p[i];
  }
  const float bq = bqo + K[H] * b_p[H];
  float ba = -(ial[4] * ial[4]) * (r * bq);  // adjoint of alpha_j, j = 4 first
  // b_p[H] - (q b_chi + bq / alpha_4), with 1 - K_H / alpha_4 = v / alpha_4
  // (K_H = alpha_4 - v) taken exactly: near a diffuse prior the difference
  // would cancel to ~v / C_HH
  b_p[H] = (v * ial[4]) * b_p[H] - (q * b_chi + ial[4] * bqo);
#pragma unroll
  for (int j = 4; j >= H; --j) {
    const float f = j == H ? 1.0f : u[ui(H, j)];
    const float g = gv[j];
    const float apj = j > H ? al[j - 1] : v;
    float bg = bK[j];
    bK[j] = 0.0f;
    float bf = 0.0f, bap = 0.0f;
    if (j > H) {
      const float iapj = ial[j - 1];
      const float lam = -(f * iapj);
      float blam = 0.0f;
#pragma unroll
      for (int i = j - 1; i >= 0; --i) {
        const float uo = u[ui(i, j)];
        const float kb = k_before(i, j);
        const float bu = b_u[ui(i, j)];
        bg = bg + uo * bK[i];
        blam = blam + kb * bu;
        b_u[ui(i, j)] = bu + g * bK[i];
        bK[i] = bK[i] + lam * bu;
      }
      bf = -(blam * iapj);
      bap = -(lam * blam) * iapj;
    } else {
#pragma unroll
      for (int i = j - 1; i >= 0; --i) {
        const float uo = u[ui(i, j)];
        bg = bg + uo * bK[i];
        b_u[ui(i, j)] += g * bK[i];
      }
    }
    // d_j' = d_j alpha_{j-1} / alpha_j
    const float rho = apj * ial[j];
    const float bdn = b_d[j];
    bap = bap + (d[j] * bdn) * ial[j];
    ba = ba - ((d[j] * rho) * bdn) * ial[j];
    float bdj = bdn * rho;
    // alpha_j = alpha_{j-1} + f_j g_j
    bap = bap + ba;
    bf = bf + g * ba;
    bg = bg + f * ba;
    // g_j = d_j f_j; f_j = u_Hj (j > H) or 1
    bdj = bdj + f * bg;
    bf = bf + d[j] * bg;
    b_d[j] = bdj;
    if (j > H) b_u[ui(H, j)] += bf;
    ba = bap;
  }
}

// ---------------------------------------------------------------- one step in U-D form
__device__ __forceinline__ void store_state(float4* dst, const UDState& S) {
  float v[20];
#pragma unroll
  for (int c = 0; c < 5; ++c) v[c] = S.p[c];
#pragma unroll
  for (int e = 0; e < 10; ++e) v[5 + e] = S.u[e];
#pragma unroll
  for (int c = 0; c < 5; ++c) v[15 + c] = S.d[c];
#pragma unroll
  for (int j = 0; j < kUDStateF4; ++j) dst[j * kWarp] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

template <bool VOLATILE>
__device__ __forceinline__ void read_state_ud(const float4* src, UDState& S) {
  float v[20];
#pragma unroll
  for (int j = 0; j < kUDStateF4; ++j) {
    const float4 f = VOLATILE ? lds_volatile(src + j * kWarp) : src[j * kWarp];
    v[4 * j] = f.x;
    v[4 * j + 1] = f.y;
    v[4 * j + 2] = f.z;
    v[4 * j + 3] = f.w;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) S.p[c] = v[c];
#pragma unroll
  for (int e = 0; e < 10; ++e) S.u[e] = v[5 + e];
#pragma unroll
  for (int c = 0; c < 5; ++c) S.d[c] = v[15 + c];
}

// A segment's first state from the fit's checkpoint, loaded as a StepState:
// (u, d) as written by the U-D fit (ud_ck; u in rows 0-1 of C.L, d in row 2),
// else converted from the square-root factor.
__device__ __forceinline__ void ud_state_from(const StepState& C, bool ud_ck, UDState& S) {
#pragma unroll
  for (int c = 0; c < 5; ++c) S.p[c] = C.p[c];
  if (ud_ck) {
#pragma unroll
    for (int e = 0; e < 10; ++e) S.u[e] = C.L[e / 5][e % 5];
#pragma unroll
    for (int c = 0; c < 5; ++c) S.d[c] = C.L[2][c];
  } else {
    ud_from_sqrt(C.L, S.u, S.d);
  }
  S.x = C.x;
  S.sec = C.sec;
}

// Forward of one step in U-D form (the operations of step_fwd with the
// factor's arithmetic replaced).  A prediction that the recorded fit took but
// that fails here on a rounding difference leaves the state unpropagated.
template <int FIELD = 0>
__device__ __forceinline__ void step_fwd_ud(const GeoRef& G, const SmemTables& T, UDState& S, float& my, float& mz,
                                            bool first, bool conv, int row, int sec18, float m0, float m1) {
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
    if (predict_residual<FIELD>(G, T, S.p, S.x, S.sec, my, mz, sec18, T.row_x[row], m0, m1, pn, J, tp)) {
#pragma unroll
      for (int c = 0; c < 5; ++c) S.p[c] = pn[c];
      if (J.rot)
        rotate_ud(S.u, S.d, J);
      else
        transport_ud(S.u, J);
    }
    S.x = T.row_x[row];
    S.sec = sec18;
  }
  my = m0;
  mz = m1;
  bierman_update<0>(S.p, S.u, S.d, chi2, G.v_meas);
  bierman_update<1>(S.p, S.u, S.d, chi2, G.v_meas);
}

// Reverse of one step in U-D form; the arguments as for step_rev, with the
// factor's adjoint (b_u, b_d) in place of b_L, and x_prev, sec_prev (the
// previous cluster's row position and sector mod 18: the state's frame).
// The gradient of the current cluster's measurement is handed to acc(g0, g1)
// as soon as the update reverses have produced it, so that it is not held
// through the reverses of the transport and the prediction.
template <int FIELD = 0, class Acc>
__device__ __forceinline__ void step_rev_ud(const GeoRef& G, const SmemTables& T, const float4* src, float my_prev,
                                            float mz_prev, float x_prev, int sec_prev, bool first, bool conv, int row,
                                            int sec18, float m0, float m1, float b_p[5], float b_u[10], float b_d[5],
                                            float b_chi, Acc&& acc, float b_mp[2]) {
  UDState S0;
  read_state_ud<false>(src, S0);
  S0.x = x_prev;
  S0.sec = sec_prev;
  float p1[5];
  Jac J;
  PredTape tp;
  float u1[10], d1[5];
  bool moved = false;
  if (first) {
#pragma unroll
    for (int c = 0; c < 5; ++c) p1[c] = S0.p[c];
    if (conv) {
      p1[0] = S0.p[0] - m0;
      p1[1] = S0.p[1] - m1;
    }
  } else {
    moved = predict_residual<FIELD>(G, T, S0.p, S0.x, S0.sec, my_prev, mz_prev, sec18, T.row_x[row], m0, m1, p1, J, tp);
    if (!moved) {
#pragma unroll
      for (int c = 0; c < 5; ++c) p1[c] = S0.p[c];
    }
  }
#pragma unroll
  for (int e = 0; e < 10; ++e) u1[e] = S0.u[e];
#pragma unroll
  for (int c = 0; c < 5; ++c) d1[c] = S0.d[c];
  if (moved) {
    if (J.rot)
      rotate_ud(u1, d1, J);
    else
      transport_ud(u1, J);
  }
  // the state before the z update
  float p2[5], u2[10], d2[5];
  float chi_dummy = 0.0f;
#pragma unroll
  for (int c = 0; c < 5; ++c) p2[c] = p1[c];
#pragma unroll
  for (int e = 0; e < 10; ++e) u2[e] = u1[e];
#pragma unroll
  for (int c = 0; c < 5; ++c) d2[c] = d1[c];
  bierman_update<0>(p2, u2, d2, chi_dummy, G.v_meas);
  bierman_update_rev<1>(p2, u2, d2, G.v_meas, b_p, b_u, b_d, b_chi);
  bierman_update_rev<0>(p1, u1, d1, G.v_meas, b_p, b_u, b_d, b_chi);
  // b_p is now the adjoint of the predicted (shifted) state p1; the current
  // measurement enters it as -m, except where the inward pass starts from
  // residuals already and where the step did not move the state
  const bool none = first ? !conv : !moved;
  acc(none ? 0.0f : -b_p[0], none ? 0.0f : -b_p[1]);
  b_mp[0] = 0.0f;
  b_mp[1] = 0.0f;
  if (first || !moved) return;
  read_state_ud<true>(src, S0);
  JacBar bJ;
  bJ.yy = bJ.ys = bJ.yq = bJ.zy = bJ.zs = bJ.zt = bJ.zq = bJ.sy = bJ.ss = bJ.sq = 0.0f;
  if (J.rot)
    rotate_ud_rev(S0.u, S0.d, J, b_u, b_d, bJ);
  else
    transport_ud_rev(S0.u, J, b_u, bJ);
  const bool rot = S0.sec != sec18;
  if (!rot) {
    b_mp[0] = b_p[0];
    b_mp[1] = b_p[1];
  }
  float b_pi[5], b_yo, b_zo;
  predict_rev<FIELD>(G, tp, J, S0.p[3], S0.p[4], b_p, bJ, b_pi, b_yo, b_zo);
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
