// Forward pieces of the filter in U-D form, C = U D U^T (U unit upper
// triangular, D diagonal): transport, sector rotation and Bierman's
// measurement update.  Included by fit_core.cuh (the fast fit can run in this
// form) and, through it, by the backward's U-D recomputation.
//
// In the state order (y, z, sin phi, tan lambda, q/pt) the step Jacobian
// without a sector rotation is unit upper triangular, so the transport keeps
// U unit upper triangular and D unchanged (11 operations in place of the
// square-root factor's 30).  The measurement updates are Bierman's (Bierman
// 1977, "Factorization Methods for Discrete Sequential Estimation", Sec. V):
// no square root, 15 factor entries in place of 25.  A rotation turns the
// Jacobian's first column full; there the rows of J U are re-orthogonalised
// with the weights D (modified weighted Gram-Schmidt, Thornton & Bierman
// 1978), which touches only the leading 3x3 block.
#pragma once

namespace tpcfit {
namespace TPCFIT_NS {

// Strictly upper entries of U, row by row: (0,1) (0,2) (0,3) (0,4) (1,2) (1,3)
// (1,4) (2,3) (2,4) (3,4).
__host__ __device__ constexpr int ui(int i, int j) { return 4 * i - (i * (i - 1)) / 2 + (j - i - 1); }

__device__ __forceinline__ float ud_rcp(float x) { return __fdividef(1.0f, x); }

// U <- J U for a step without rotation (J unit upper triangular; D unchanged).
__device__ __forceinline__ void transport_ud(float u[10], const Jac& J) {
  u[ui(0, 4)] = (u[ui(0, 4)] + J.ys * u[ui(2, 4)]) + J.yq;
  u[ui(0, 3)] = u[ui(0, 3)] + J.ys * u[ui(2, 3)];
  u[ui(0, 2)] = u[ui(0, 2)] + J.ys;
  u[ui(1, 4)] = ((u[ui(1, 4)] + J.zs * u[ui(2, 4)]) + J.zt * u[ui(3, 4)]) + J.zq;
  u[ui(1, 3)] = (u[ui(1, 3)] + J.zs * u[ui(2, 3)]) + J.zt;
  u[ui(1, 2)] = u[ui(1, 2)] + J.zs;
  u[ui(2, 4)] = u[ui(2, 4)] + J.sq;
}

// Leading 3x3 block of W = J U at a rotation (rows y, z, s; columns 0..2).
struct RotW {
  float w[3][3];
};

__device__ __forceinline__ RotW rot_w(const float u[10], const Jac& J) {
  RotW r;
  const float u01 = u[ui(0, 1)], u02 = u[ui(0, 2)];
  r.w[0][0] = J.yy;
  r.w[0][1] = J.yy * u01;
  r.w[0][2] = J.yy * u02 + J.ys;
  r.w[1][0] = J.zy;
  r.w[1][1] = J.zy * u01 + 1.0f;
  r.w[1][2] = (J.zy * u02 + u[ui(1, 2)]) + J.zs;
  r.w[2][0] = J.sy;
  r.w[2][1] = J.sy * u01;
  r.w[2][2] = J.sy * u02 + J.ss;
  return r;
}

__device__ __forceinline__ float wdot3(const float d[5], const float a[3], const float b[3]) {
  return ((d[0] * a[0]) * b[0] + (d[1] * a[1]) * b[1]) + (d[2] * a[2]) * b[2];
}

// U D U^T <- J U D U^T J^T at a sector rotation.  Columns 3 and 4 of the new
// U are those of J U (rows 3 and 4 of J are identity rows); the leading block
// follows from the weighted Gram-Schmidt of rows s, z, y of W with the
// weights d0..d2: d'_2 = |w_2|^2_D, u'_02 and u'_12 the projections on w_2,
// then d'_1 and u'_01 on the reduced w_1, and d'_0 on the reduced w_0.
__device__ __forceinline__ void rotate_ud(float u[10], float d[5], const Jac& J) {
  const RotW W = rot_w(u, J);
  const float u03 = u[ui(0, 3)], u04 = u[ui(0, 4)], u13 = u[ui(1, 3)], u14 = u[ui(1, 4)];
  const float u23 = u[ui(2, 3)], u24 = u[ui(2, 4)], u34 = u[ui(3, 4)];
  u[ui(0, 3)] = J.yy * u03 + J.ys * u23;
  u[ui(0, 4)] = (J.yy * u04 + J.ys * u24) + J.yq;
  u[ui(1, 3)] = ((J.zy * u03 + u13) + J.zs * u23) + J.zt;
  u[ui(1, 4)] = (((J.zy * u04 + u14) + J.zs * u24) + J.zt * u34) + J.zq;
  u[ui(2, 3)] = J.sy * u03 + J.ss * u23;
  u[ui(2, 4)] = (J.sy * u04 + J.ss * u24) + J.sq;
  const float e2 = wdot3(d, W.w[2], W.w[2]);
  const float i2 = ud_rcp(e2);
  const float a02 = wdot3(d, W.w[0], W.w[2]) * i2;
  const float a12 = wdot3(d, W.w[1], W.w[2]) * i2;
  float x0[3], x1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x0[c] = W.w[0][c] - a02 * W.w[2][c];
    x1[c] = W.w[1][c] - a12 * W.w[2][c];
  }
  const float e1 = wdot3(d, x1, x1);
  const float a01 = wdot3(d, x0, x1) * ud_rcp(e1);
  float y0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) y0[c] = x0[c] - a01 * x1[c];
  const float e0 = wdot3(d, y0, y0);
  u[ui(0, 1)] = a01;
  u[ui(0, 2)] = a02;
  u[ui(1, 2)] = a12;
  d[0] = e0;
  d[1] = e1;
  d[2] = e2;
}

// Bierman's scalar update of component H (0 = y, 1 = z) in residual
// coordinates (measured value 0), cluster variance v.  f = row H of U,
// g = D f; alpha_j = alpha_{j-1} + f_j g_j from alpha = v; d_j <- d_j
// alpha_{j-1} / alpha_j; for j > H, lambda = -f_j / alpha_{j-1} and, for
// i < j, u_ij <- u_ij + lambda K_i, K_i += g_j u_ij (old); K_j = g_j.  The
// gain is K / alpha_4 and alpha_4 the innovation variance.
template <int H>
__device__ __forceinline__ void bierman_update(float p[5], float u[10], float d[5], float& chi2, float v) {
  float K[5];
  float ap = v, iap = 0.0f;
#pragma unroll
  for (int j = H; j < 5; ++j) {
    const float f = j == H ? 1.0f : u[ui(H, j)];
    const float g = j == H ? d[j] : d[j] * f;
    const float a = j == H ? ap + g : ap + f * g;
    const float ia = ud_rcp(a);
    if (j > H) {
      const float lam = -(f * iap);
#pragma unroll
      for (int i = 0; i < j; ++i) {
        const float uo = u[ui(i, j)];
        u[ui(i, j)] = uo + lam * K[i];
        K[i] = K[i] + g * uo;
      }
    } else {
#pragma unroll
      for (int i = 0; i < j; ++i) K[i] = g * u[ui(i, j)];
    }
    d[j] = d[j] * (ap * ia);
    K[j] = g;
    ap = a;
    iap = ia;
  }
  const float r = -p[H];
  const float q = r * iap;
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + K[i] * q;
  chi2 = chi2 + r * q;
}

}  // namespace TPCFIT_NS
}  // namespace tpcfit
