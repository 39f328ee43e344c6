// Two-filter smoother of a recorded fit (Fraser & Potter): for every cluster,
// the residual against the estimate from all the other clusters.  Included
// after fit_core.cuh and adjoint_core.cuh by each kernel module, so that the
// recomputed filter steps are the module's own arithmetic.
//
// Per cluster c of a fitted track: the outward prediction at c (seed and
// clusters 0..c-1) and the inward prediction at c (the inward pass's prior and
// clusters last..c+1) are independent estimates of the state at c.  Their
// combination x_u has
//   H x_u     = H x_out + H C_out S^-1 (x_in - x_out),
//   H C_u H^T = H C_out S^-1 C_in H^T,        S = C_out + C_in,
// (C_u = C_out S^-1 C_in, without a subtraction), evaluated in square-root
// form (smooth_combine).  Outputs: the residual m_c - H x_u,
// R = V + H C_u H^T and chi2 = r^T R^-1 r (2 degrees of freedom).
//
// Work mapping: the outward filter runs forward from the seed, cluster by
// cluster.  The inward predictions are needed in the same order, which is the
// reverse of the inward pass; they come from the inward checkpoints segment by
// segment (last segment first): a segment is recomputed into the warp's
// segment store and consumed in reverse, one state copied ahead into shared
// memory, as in the adjoint.
#pragma once

namespace tpcfit {
namespace TPCFIT_NS {

// Residual, its covariance and chi2 of one cluster from the outward (1) and
// inward (2) predictions (p, square-root factor L, C = L L^T), both in
// residual coordinates of that cluster.
//
// Square-root form: with A1 = L1^T, A2 = L2^T and the QR factorisation
// [A1; A2] = Q R (Householder, Q 10x5 with orthonormal columns, Q = [Q1; Q2]),
// S = C1 + C2 = R^T R and C1 S^-1 C2 = A1^T Q1 Q2^T A2, so that
//   H x_u - H x1 = W1 u,  H C_u H^T = W1 W2^T,  u = R^-T (x2 - x1),
//   W1 = [H L1, 0] Q,  W2 = [0, H L2] Q,
// computed by applying the reflectors to the two 2x10 row blocks.  Forming S
// (or C H^T) in FP32 instead squares the condition number of the factors and
// loses the residual next to a diffuse end of the track (the second and the
// second-last cluster).
__device__ __forceinline__ void smooth_combine(const GeoRef& G, const float p1[5], const float L1[5][5], const float p2[5],
                                               const float L2[5][5], float r[2], float R[3], float& chi2) {
  float M[10][5];   // [A1; A2]
  float E[4][10];   // rows 0-1: [H L1, 0]; rows 2-3: [0, H L2]
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      M[q][i] = L1[i][q];
      M[5 + q][i] = L2[i][q];
    }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      E[h][q] = L1[h][q];
      E[h][5 + q] = 0.0f;
      E[2 + h][q] = 0.0f;
      E[2 + h][5 + q] = L2[h][q];
    }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    // reflector of column k, rows k..9: v = x - alpha e_k, alpha = -sign(x_k) |x|
    float nrm2 = M[k][k] * M[k][k];
#pragma unroll
    for (int q = k + 1; q < 10; ++q) nrm2 = nrm2 + M[q][k] * M[q][k];
    float nrm, inrm;
    sqrt_and_inv(nrm2, nrm, inrm);
    const float alpha = M[k][k] > 0.0f ? -nrm : nrm;
    const float v0 = M[k][k] - alpha;
    // y <- y + (v^T y) / (alpha v0) v  (the reflection I - 2 v v^T / v^T v)
    const float g = 1.0f / (alpha * v0);
#pragma unroll
    for (int j = k + 1; j < 5; ++j) {
      float t = v0 * M[k][j];
#pragma unroll
      for (int q = k + 1; q < 10; ++q) t = t + M[q][k] * M[q][j];
      t = t * g;
      M[k][j] = M[k][j] + t * v0;
#pragma unroll
      for (int q = k + 1; q < 10; ++q) M[q][j] = M[q][j] + t * M[q][k];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float t = E[e][k] * v0;
#pragma unroll
      for (int q = k + 1; q < 10; ++q) t = t + E[e][q] * M[q][k];
      t = t * g;
      E[e][k] = E[e][k] + t * v0;
#pragma unroll
      for (int q = k + 1; q < 10; ++q) E[e][q] = E[e][q] + t * M[q][k];
    }
    M[k][k] = alpha;
  }
  // u = R^-T (p2 - p1), R = upper 5x5 of M
  float u[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float e = p2[i] - p1[i];
#pragma unroll
    for (int q = 0; q < i; ++q) e = e - M[q][i] * u[q];
    u[i] = e / M[i][i];
  }
  float c0 = E[0][0] * u[0], c1 = E[1][0] * u[0];
  float h00 = E[0][0] * E[2][0], h01 = E[0][0] * E[3][0], h10 = E[1][0] * E[2][0], h11 = E[1][0] * E[3][0];
#pragma unroll
  for (int q = 1; q < 5; ++q) {
    c0 = c0 + E[0][q] * u[q];
    c1 = c1 + E[1][q] * u[q];
    h00 = h00 + E[0][q] * E[2][q];
    h01 = h01 + E[0][q] * E[3][q];
    h10 = h10 + E[1][q] * E[2][q];
    h11 = h11 + E[1][q] * E[3][q];
  }
  // the state is relative to the measurement: r = m - H x_u = -(p1 + correction)
  r[0] = -(p1[0] + c0);
  r[1] = -(p1[1] + c1);
  const float v = G.v_meas;
  R[0] = v + h00;
  R[1] = 0.5f * (h01 + h10);
  R[2] = v + h11;
  const float det = R[0] * R[2] - R[1] * R[1];
  chi2 = (R[2] * r[0] * r[0] - 2.0f * R[1] * r[0] * r[1] + R[0] * r[1] * r[1]) / det;
}

// Smoothed state from all clusters at one cluster: the same square-root
// combination, of the outward pass's filtered state there (p1, L1) with the
// inward prediction (p2, L2), but with the five rows of [L1, 0] and of
// [0, L2] carried through the reflectors: W1 = [L1, 0] Q, W2 = [0, L2] Q,
//   x_s = p1 + W1 u,  C_s = W1 W2^T (symmetrised),  u = R^-T (p2 - p1).
__device__ __forceinline__ void smooth_state(const float p1[5], const float L1[5][5], const float p2[5],
                                             const float L2[5][5], float xs[5], float Cs[15]) {
  float M[10][5];   // [A1; A2]
  float E[10][10];  // rows 0-4: [L1, 0]; rows 5-9: [0, L2]
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      M[q][i] = L1[i][q];
      M[5 + q][i] = L2[i][q];
    }
#pragma unroll
  for (int h = 0; h < 5; ++h)
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      E[h][q] = L1[h][q];
      E[h][5 + q] = 0.0f;
      E[5 + h][q] = 0.0f;
      E[5 + h][5 + q] = L2[h][q];
    }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float nrm2 = M[k][k] * M[k][k];
#pragma unroll
    for (int q = k + 1; q < 10; ++q) nrm2 = nrm2 + M[q][k] * M[q][k];
    float nrm, inrm;
    sqrt_and_inv(nrm2, nrm, inrm);
    const float alpha = M[k][k] > 0.0f ? -nrm : nrm;
    const float v0 = M[k][k] - alpha;
    const float g = 1.0f / (alpha * v0);
#pragma unroll
    for (int j = k + 1; j < 5; ++j) {
      float t = v0 * M[k][j];
#pragma unroll
      for (int q = k + 1; q < 10; ++q) t = t + M[q][k] * M[q][j];
      t = t * g;
      M[k][j] = M[k][j] + t * v0;
#pragma unroll
      for (int q = k + 1; q < 10; ++q) M[q][j] = M[q][j] + t * M[q][k];
    }
#pragma unroll
    for (int e = 0; e < 10; ++e) {
      float t = E[e][k] * v0;
#pragma unroll
      for (int q = k + 1; q < 10; ++q) t = t + E[e][q] * M[q][k];
      t = t * g;
      E[e][k] = E[e][k] + t * v0;
#pragma unroll
      for (int q = k + 1; q < 10; ++q) E[e][q] = E[e][q] + t * M[q][k];
    }
    M[k][k] = alpha;
  }
  float u[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float e = p2[i] - p1[i];
#pragma unroll
    for (int q = 0; q < i; ++q) e = e - M[q][i] * u[q];
    u[i] = e / M[i][i];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float acc = E[i][0] * u[0];
#pragma unroll
    for (int q = 1; q < 5; ++q) acc = acc + E[i][q] * u[q];
    xs[i] = p1[i] + acc;
  }
  int e = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      float a12 = E[i][0] * E[5 + j][0];
      float a21 = E[j][0] * E[5 + i][0];
#pragma unroll
      for (int q = 1; q < 5; ++q) {
        a12 = a12 + E[i][q] * E[5 + j][q];
        a21 = a21 + E[j][q] * E[5 + i][q];
      }
      Cs[e++] = 0.5f * (a12 + a21);
    }
}

__device__ __forceinline__ void write_nan_clusters(const SmoothArgs& a, int h0, int h1) {
  const float qnan = __int_as_float(0x7fc00000);
  for (int h = h0; h < h1; ++h) {
    if (a.resid) {
      reinterpret_cast<float2*>(a.resid)[h] = make_float2(qnan, qnan);
      a.rcov[(int64_t)h * 3] = qnan;
      a.rcov[(int64_t)h * 3 + 1] = qnan;
      a.rcov[(int64_t)h * 3 + 2] = qnan;
      a.chi2[h] = qnan;
    }
    if (a.state) {
      for (int q = 0; q < 5; ++q) a.state[(int64_t)h * 5 + q] = qnan;
      for (int q = 0; q < 15; ++q) a.state_cov[(int64_t)h * 15 + q] = qnan;
    }
  }
}

// Shared memory of a smoother block: the tables, the alignment table and,
// per warp, a double buffer for the inward states and a checkpoint buffer.
template <int WARPS>
constexpr size_t smooth_smem_bytes() {
  return sizeof(BwdSmem) + WARPS * sizeof(BwdWarpBufs);
}

// STATES: the smoothed state and its covariance at every cluster as well
// (a.state, a.state_cov); without it the kernel carries none of that code.
template <int WARPS, bool MAT, bool STATES>
__global__ void __launch_bounds__(WARPS * 32, 1) smooth_kernel(const __grid_constant__ SmoothArgs a) {
  const GeoRef& G = a.geo;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& B = *reinterpret_cast<BwdSmem*>(smem_raw);
  load_tables(G, B.T);
  for (int i = threadIdx.x; i < kAlignFloats; i += blockDim.x) B.align[i] = __ldg(a.align + i);
  __syncthreads();
  const SmemTables& T = B.T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  BwdWarpBufs& W = reinterpret_cast<BwdWarpBufs*>(smem_raw + sizeof(BwdSmem))[warp];
  float4* const gs = a.seg + ((int64_t)blockIdx.x * WARPS + warp) * (kCkptEvery * kStateF4 * kWarp) + lane;
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
    const int begin = a.off[trk];
    const int end = a.off[trk + 1];
    if (a.ndf[trk] <= 0) {
      write_nan_clusters(a, begin, end);
      continue;
    }
    const int last = a.ck_last[trk];
    write_nan_clusters(a, begin + last + 1, end);  // clusters the outward pass did not reach
    const int64_t slot0 = (begin >> kCkptShift) + trk;
    // outward filter: from its first checkpoint (the seed, factor L0)
    StepState O;
    load_ckpt(a.ck + slot0 * kCkptFloats, O);
    if (a.ck_form == 1) sqrt_from_ud_ckpt(O);
    float omy = 0.0f, omz = 0.0f;  // measurement O's residuals refer to (none for the seed)
    // inward segments, last first: inward step j is cluster last - j
    const int steps = last + 1;
    const int nseg = (steps + kCkptEvery - 1) / kCkptEvery;
    const float* ckp = a.ck + ((int64_t)a.ck_slots + slot0) * kCkptFloats;
    const int h_last = begin + last;
    fetch_ckpt(&W.ck[0][lane], ckp + (int64_t)(nseg - 1) * kCkptFloats);
#pragma unroll 1
    for (int s = nseg - 1; s >= 0; --s) {
      const int j0 = s * kCkptEvery;
      const int cnt = min(kCkptEvery, steps - j0);
      StepState S;
      float my = 0.0f, mz = 0.0f;
      HitRaw nx = load_hit(a.y, a.z, a.rowsec, h_last - j0);
      if (j0 > 0) {
        int row, sec;
        decode_hit(B.align, load_hit(a.y, a.z, a.rowsec, h_last - (j0 - 1)), my, mz, row, sec);
      }
      cp_async_wait<0>();
      read_state(&W.ck[0][lane], S);
      if (a.ck_form == 1) sqrt_from_ud_ckpt(S);
      // level 1: the inward segment, storing the state before each step
#pragma unroll 1
      for (int kk = 0; kk < cnt; ++kk) {
        const int j = j0 + kk;
        const HitRaw cur = nx;
        if (kk + 1 < cnt) nx = load_hit(a.y, a.z, a.rowsec, h_last - (j + 1));
        float m0, m1;
        int row, sec;
        decode_hit(B.align, cur, m0, m1, row, sec);
        store_state(gs + kk * (kStateF4 * kWarp), S);
        step_fwd<MAT, 2>(G, T, S, my, mz, j == 0, false, row, side_sector(sec), m0, m1);
      }
      __threadfence_block();  // the states just stored are read back by this thread's copies below
      if (s > 0) fetch_ckpt(&W.ck[0][lane], ckp + (int64_t)(s - 1) * kCkptFloats);
      fetch_state(&W.st[(cnt - 1) & 1][0][lane], gs + (cnt - 1) * (kStateF4 * kWarp));
      // consume in reverse: cluster c = last - j ascending
#pragma unroll 1
      for (int kk = cnt - 1; kk >= 0; --kk) {
        const int j = j0 + kk;
        const int c = last - j;
        const int h = begin + c;
        if (kk > 0) {
          fetch_state(&W.st[(kk - 1) & 1][0][lane], gs + (kk - 1) * (kStateF4 * kWarp));
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        float m0, m1;
        int row, sec;
        decode_hit(B.align, load_hit(a.y, a.z, a.rowsec, h), m0, m1, row, sec);
        const int sec18 = side_sector(sec);
        const float X = T.row_x[row];
        // inward prediction at c
        StepState SI;
        read_state(&W.st[kk & 1][0][lane], SI);
        float pi[5];
        if (j == 0) {  // the inward pass starts on this cluster
#pragma unroll
          for (int q = 0; q < 5; ++q) pi[q] = SI.p[q];
        } else {
          float mpy, mpz;
          int prow, psec;
          decode_hit(B.align, load_hit(a.y, a.z, a.rowsec, h + 1), mpy, mpz, prow, psec);
          Jac J;
          PredTape tp;
          if (MAT) {  // the layer of row c + 1, undone against the flight
            MatNoise N;
            material_step(G, SI.p, -1, N);
            material_factor(SI.L, N);
          }
          predict_residual<2>(G, T, SI.p, SI.x, SI.sec, mpy, mpz, sec18, X, m0, m1, pi, J, tp);
          transport(SI.L, J);
        }
        // outward prediction at c
        float po[5];
        if (c == 0) {  // the seed, made relative to the first cluster
#pragma unroll
          for (int q = 0; q < 5; ++q) po[q] = O.p[q];
          po[0] = O.p[0] - m0;
          po[1] = O.p[1] - m1;
        } else {
          Jac J;
          PredTape tp;
          predict_residual<2>(G, T, O.p, O.x, O.sec, omy, omz, sec18, X, m0, m1, po, J, tp);
          MatNoise N;
          if (MAT) material_step(G, po, 1, N);  // the layer of row c
          transport(O.L, J);
          if (MAT) material_factor(O.L, N);
        }
        if (a.resid) {
          float r[2], R[3], c2;
          smooth_combine(G, po, O.L, pi, SI.L, r, R, c2);
          reinterpret_cast<float2*>(a.resid)[h] = make_float2(r[0], r[1]);
          a.rcov[(int64_t)h * 3] = R[0];
          a.rcov[(int64_t)h * 3 + 1] = R[1];
          a.rcov[(int64_t)h * 3 + 2] = R[2];
          a.chi2[h] = c2;
        }
        // the outward filter takes cluster c
#pragma unroll
        for (int q = 0; q < 5; ++q) O.p[q] = po[q];
        O.x = X;
        O.sec = sec18;
        omy = m0;
        omz = m1;
        float chi_unused = 0.0f;
        scalar_update<0>(G, O.p, O.L, chi_unused, 0.0f);
        scalar_update<1>(G, O.p, O.L, chi_unused, 0.0f);
        if (STATES) {  // the outward filtered state at c with the inward prediction
          float xs[5], Cs[15];
          smooth_state(O.p, O.L, pi, SI.L, xs, Cs);
          xs[0] = xs[0] + m0;  // residual coordinates back to positions
          xs[1] = xs[1] + m1;
#pragma unroll
          for (int q = 0; q < 5; ++q) a.state[(int64_t)h * 5 + q] = xs[q];
#pragma unroll
          for (int q = 0; q < 15; ++q) a.state_cov[(int64_t)h * 15 + q] = Cs[q];
        }
      }
    }
  }
}

#ifndef __CUDACC_RTC__
template <int WARPS, bool MAT, bool STATES>
cudaError_t smooth_grid(int& grid) {
  static int cached = 0;
  if (cached == 0) {
    const size_t smem = smooth_smem_bytes<WARPS>();
    cudaError_t e =
        cudaFuncSetAttribute(smooth_kernel<WARPS, MAT, STATES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smooth_kernel<WARPS, MAT, STATES>, WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cached = sms * per_sm;
  }
  grid = cached;
  return cudaSuccess;
}

constexpr int kSmoothWarps = 8;

// Segment store (float4 count) the smoother needs (the larger of its variants).
inline cudaError_t smooth_store(int64_t& float4s) {
  int g[4] = {0, 0, 0, 0};
  cudaError_t e = smooth_grid<kSmoothWarps, false, false>(g[0]);
  if (e == cudaSuccess) e = smooth_grid<kSmoothWarps, true, false>(g[1]);
  if (e == cudaSuccess) e = smooth_grid<kSmoothWarps, false, true>(g[2]);
  if (e == cudaSuccess) e = smooth_grid<kSmoothWarps, true, true>(g[3]);
  int gm = 0;
  for (int i = 0; i < 4; ++i) gm = g[i] > gm ? g[i] : gm;
  float4s = (int64_t)gm * kSmoothWarps * kCkptEvery * kStateF4 * kWarp;
  return e;
}

template <bool MAT, bool STATES>
cudaError_t launch_smooth_cfg(const SmoothArgs& a, cudaStream_t s) {
  int grid = 0;
  cudaError_t e = smooth_grid<kSmoothWarps, MAT, STATES>(grid);
  if (e != cudaSuccess) return e;
  const int64_t chunks = ((int64_t)a.n_tracks + kWarp - 1) / kWarp;
  const int64_t need = (chunks + kSmoothWarps - 1) / kSmoothWarps;
  const int blocks = (int)(need < grid ? need : grid);
  e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  smooth_kernel<kSmoothWarps, MAT, STATES><<<blocks, kSmoothWarps * 32, smooth_smem_bytes<kSmoothWarps>(), s>>>(a);
  return cudaGetLastError();
}

inline cudaError_t launch_smooth(const SmoothArgs& a, cudaStream_t s) {
  if (a.n_tracks <= 0) return cudaSuccess;
  if (a.state) return a.mat ? launch_smooth_cfg<true, true>(a, s) : launch_smooth_cfg<false, true>(a, s);
  return a.mat ? launch_smooth_cfg<true, false>(a, s) : launch_smooth_cfg<false, false>(a, s);
}
#endif

}  // namespace TPCFIT_NS
}  // namespace tpcfit
