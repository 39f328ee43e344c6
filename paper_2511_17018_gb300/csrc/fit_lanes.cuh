// The fit with P lanes per track (32 / P tracks per warp), P = 2, 4, 8, 16 or 32.
// Included after fit_core.cuh by the two kernel modules (not compiled at run
// time), for the uniform field without material layers.
//
// Lane g of a track's group of P lanes owns the factor columns
// c = g, g + P, g + 2P, ... (< 5); with P > 5 the lanes g >= 5 own none.  The
// state p, the prediction (with its Jacobian) and the scalars of each Potter
// update are computed on every lane of the group alike.  A sum over the
// columns (a . a, a row of L a, an element of L L^T) gathers the owners'
// terms with shuffles and adds them in column order, so every value goes
// through the operation sequence of the one-lane fit: in the deterministic
// mode the results are bit-identical to it (and to the strict-FP32 reference),
// whatever P.  The transport and the rank-one corrections of the factor touch
// a lane's own columns only.
//
// What P buys is latency per track: a step's factor algebra is split over P
// lanes, while the prediction is repeated on each of them and every column
// sum costs five shuffles.
#pragma once

namespace tpcfit {
namespace TPCFIT_NS {

template <int P>
struct Lanes {
  static constexpr int kTracks = kWarp / P;          // tracks per warp
  static constexpr int kCols = (5 + P - 1) / P;      // factor columns a lane owns, at most
};

// The term of column c, from the lane of the group that owns it (v: this
// lane's terms, one per owned column; base: the group's first lane).
template <int P>
__device__ __forceinline__ float col_term(const float* v, int base, int c) {
  return __shfl_sync(0xffffffffu, v[c / P], base + (c % P));
}

// sum_c v_c in column order, starting from `init` (init + v_0 + v_1 + ...).
template <int P>
__device__ __forceinline__ float col_sum(const float* v, int base, float init) {
  float acc = init + col_term<P>(v, base, 0);
#pragma unroll
  for (int c = 1; c < 5; ++c) acc = acc + col_term<P>(v, base, c);
  return acc;
}
// sum_c v_c in column order (v_0 + v_1 + ...).
template <int P>
__device__ __forceinline__ float col_sum(const float* v, int base) {
  float acc = col_term<P>(v, base, 0);
#pragma unroll
  for (int c = 1; c < 5; ++c) acc = acc + col_term<P>(v, base, c);
  return acc;
}

// Factor columns of one lane: Lc[i][j] = L[i][g + j P].
template <int P>
struct LaneFactor {
  float Lc[5][Lanes<P>::kCols];
};

template <int P>
__device__ __forceinline__ bool owns(int g, int j) {
  return g + j * P < 5;
}

template <int P>
__device__ __forceinline__ void reset_factor_lanes(const GeoRef& G, LaneFactor<P>& F, int g) {
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < Lanes<P>::kCols; ++j) F.Lc[i][j] = (i == g + j * P) ? G.l0 : 0.0f;
}

// L <- J L on the lane's columns (rows t, q of J are identity).
template <int P>
__device__ __forceinline__ void transport_lanes(LaneFactor<P>& F, const Jac& J) {
#pragma unroll
  for (int j = 0; j < Lanes<P>::kCols; ++j) {
    const float L0 = F.Lc[0][j], L1 = F.Lc[1][j], L2 = F.Lc[2][j], L3 = F.Lc[3][j], L4 = F.Lc[4][j];
    if (!J.rot) {
      F.Lc[0][j] = (L0 + J.ys * L2) + J.yq * L4;
      F.Lc[1][j] = ((L1 + J.zs * L2) + J.zt * L3) + J.zq * L4;
      F.Lc[2][j] = L2 + J.sq * L4;
    } else {
      F.Lc[0][j] = (J.yy * L0 + J.ys * L2) + J.yq * L4;
      F.Lc[1][j] = (((J.zy * L0 + L1) + J.zs * L2) + J.zt * L3) + J.zq * L4;
      F.Lc[2][j] = (J.sy * L0 + J.ss * L2) + J.sq * L4;
    }
  }
}

// Potter scalar update of component H (measured value 0 in residual
// coordinates), the columns split over the group: the operation sequence of
// scalar_update in each mode.
template <int P, int H>
__device__ __forceinline__ void scalar_update_lanes(const GeoRef& G, float p[5], LaneFactor<P>& F, float& chi2,
                                                    int base) {
  constexpr int NC = Lanes<P>::kCols;
  const float v = G.v_meas;
  float a[NC], t[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    a[j] = F.Lc[H][j];
    t[j] = a[j] * a[j];
  }
  const float s2 = col_sum<P>(t, base, v);
  float alpha, beta, gamma;
  potter_coeffs(s2, v, G.sqrt_v, alpha, beta, gamma);
  const float r = 0.0f - p[H];
  float la[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#if !TPCFIT_DET
    if (i == H) {
      la[i] = s2 - v;
      continue;
    }
#endif
#pragma unroll
    for (int j = 0; j < NC; ++j) t[j] = F.Lc[i][j] * a[j];
    la[i] = col_sum<P>(t, base);
  }
#if TPCFIT_DET
  float K[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) K[i] = la[i] * alpha;
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + K[i] * r;
  chi2 = chi2 + (r * r) * alpha;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) continue;
    const float gk = gamma * K[i];
#pragma unroll
    for (int j = 0; j < NC; ++j) F.Lc[i][j] = F.Lc[i][j] - gk * a[j];
  }
#else
  const float ar = alpha * r;
  const float ga = gamma * alpha;
#pragma unroll
  for (int i = 0; i < 5; ++i) p[i] = p[i] + la[i] * ar;
  chi2 = chi2 + r * ar;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    if (i == H) continue;
    const float gk = la[i] * ga;
#pragma unroll
    for (int j = 0; j < NC; ++j) F.Lc[i][j] = F.Lc[i][j] - gk * a[j];
  }
#endif
#pragma unroll
  for (int j = 0; j < NC; ++j) F.Lc[H][j] = a[j] * beta;
}

// Staging of RPS clusters for each of the warp's kTracks tracks (track slot t
// is held by lanes t P .. t P + P - 1).
template <int P, int RPS>
struct WarpStageLanes {
  float y[2][Lanes<P>::kTracks][RPS + 1];
  float z[2][Lanes<P>::kTracks][RPS + 1];
  uint32_t rs[2][Lanes<P>::kTracks][RPS + 1];
};

template <int P, int RPS>
__device__ __forceinline__ void stage_issue_lanes(WarpStageLanes<P, RPS>& st, int b, const FitArgs& a, int my_first,
                                                  int my_count, int dir, int c0, int lane) {
  constexpr int T = Lanes<P>::kTracks;
  constexpr int ITERS = (T * RPS + kWarp - 1) / kWarp;
  const uintptr_t rs_begin = (uintptr_t)a.rowsec;
  const uintptr_t rs_end = (uintptr_t)(a.rowsec + a.n_hits);
#pragma unroll
  for (int it = 0; it < ITERS; ++it) {
    const int e = it * kWarp + lane;
    const int t = e / RPS;
    const int k = e % RPS;
    const int src = (t < T ? t : 0) * P;
    const int first_t = __shfl_sync(0xffffffffu, my_first, src);
    const int count_t = __shfl_sync(0xffffffffu, my_count, src);
    const int i = c0 + k;
    if (t < T && i < count_t) {
      const int h = first_t + dir * i;
      cp_async4(&st.y[b][t][k], a.y + h);
      cp_async4(&st.z[b][t][k], a.z + h);
      const uint16_t* rp = a.rowsec + h;
      const uintptr_t wa = (uintptr_t)rp & ~(uintptr_t)3;
      if (wa >= rs_begin && wa + 4 <= rs_end) {
        cp_async4(&st.rs[b][t][k], (const void*)wa);
      } else {
        st.rs[b][t][k] = (uint32_t)__ldg(rp) << (16u * (unsigned)(((uintptr_t)rp >> 1) & 1u));
      }
    }
  }
  cp_async_commit();
}

template <int P, int RPS, int WARPS, bool RECORD, bool FRAMES>
__global__ void __launch_bounds__(WARPS * 32, 1) fit_kernel_lanes(const __grid_constant__ FitArgs a) {
  const GeoRef& G = TPCFIT_GEO(a);
  constexpr int T = Lanes<P>::kTracks;
  constexpr int NC = Lanes<P>::kCols;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSmem& B = *reinterpret_cast<BlockSmem*>(smem_raw);
  WarpStageLanes<P, RPS>* stages = reinterpret_cast<WarpStageLanes<P, RPS>*>(smem_raw + sizeof(BlockSmem));
  load_tables(G, B.T);
  for (int i = threadIdx.x; i < kAlignFloats; i += blockDim.x) B.align[i] = __ldg(a.align + i);
  __syncthreads();
  const SmemTables& Tb = B.T;
  const int lane = threadIdx.x & 31;
  const int slot_in_warp = lane / P;  // the track slot of this lane
  const int g = lane % P;             // its place in the track's group
  const int base = lane - g;          // the group's first lane
  WarpStageLanes<P, RPS>& st = stages[threadIdx.x >> 5];
  const unsigned rs_par0 = (unsigned)(((uintptr_t)a.rowsec >> 1) & 1u);
  const int64_t n_chunks = ((int64_t)a.n_tracks + T - 1) / T;

#pragma unroll 1
  for (;;) {
    int64_t chunk = 0;
    if (lane == 0) chunk = (int64_t)atomicAdd(a.work, 1u);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    if (chunk >= n_chunks) break;
    const int64_t slot = chunk * T + slot_in_warp;
    const bool have = slot < a.n_tracks;
    const int32_t trk = have ? (a.perm ? a.perm[slot] : (int32_t)slot) : 0;

    int status = have ? 0 : 1;  // 0 fitting, 1 idle, 2 numerical failure, 3 invalid input, 4 timeout
    int begin = 0;
    int n = 0;
    const float* lane_align = B.align;
    if (FRAMES && have) {
      const int f = frame_of(a.frame_base, a.n_frames, trk);
      if (f < 0) {
        status = 3;
        if (g == 0) record_error(a.err, kErrOffsets, trk);
      } else {
        if (a.frame_ready && !wait_flag(a.frame_ready + f, a.wait_ns)) {
          status = 4;
          if (g == 0) record_error(a.err, kErrTimeout, trk);
        }
        if (a.frame_align) lane_align = a.frame_align + (int64_t)f * kAlignFloats;
      }
    }
    if (FRAMES) {
      // a wait may run out on one lane of a group and not on another: the
      // group takes the first lane's verdict, so that its lanes stay in step
      status = __shfl_sync(0xffffffffu, status, base);
      __syncwarp();
    }
    if (have && status == 0) {
      const int b = a.off[trk];
      const int e = a.off[trk + 1];
      if (b < 0 || e < b || (int64_t)e > a.n_hits) {
        status = 3;
        if (g == 0) record_error(a.err, kErrOffsets, trk);
      } else {
        begin = b;
        n = e - b;
        if (n < 1) status = 2;
      }
    }
    float p[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    LaneFactor<P> F;
    reset_factor_lanes<P>(G, F, g);
    float x = 0.0f, chi2 = 0.0f, my = 0.0f, mz = 0.0f;
    int sec_cur = 0, used = 0;
    int last = 0;
    if (status == 0) {
#pragma unroll
      for (int c = 0; c < 5; ++c) p[c] = __ldg(a.seeds + (int64_t)c * a.n_tracks + trk);
      if (!(fabsf(p[2]) < G.max_snp)) status = 2;
    }

#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int dir = pass == 0 ? 1 : -1;
      const int my_first = begin + (pass == 0 ? 0 : last);
      const int my_count = (status == 0) ? (pass == 0 ? n : last + 1) : 0;
      bool go = status == 0;
      if (go) {
        reset_factor_lanes<P>(G, F, g);
        chi2 = 0.0f;
        used = 0;
      }
      int count_max = my_count;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) count_max = max(count_max, __shfl_xor_sync(0xffffffffu, count_max, o));
      if (count_max == 0) continue;
      __syncwarp();
      stage_issue_lanes<P, RPS>(st, 0, a, my_first, my_count, dir, 0, lane);
      int buf = 0;
#pragma unroll 1
      for (int c0 = 0; c0 < count_max; c0 += RPS) {
        const bool more = c0 + RPS < count_max;
        if (more) {
          stage_issue_lanes<P, RPS>(st, buf ^ 1, a, my_first, my_count, dir, c0 + RPS, lane);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncwarp();
#pragma unroll 1
        for (int k = 0; k < RPS; ++k) {
          const int i = c0 + k;
          // every lane takes part in the column sums, whatever its group does
          const bool active = go && i < my_count;
          int row = 0, sec = 0;
          float m0 = 0.0f, m1 = 0.0f;
          bool valid = false;
          if (active) {
            const int h = my_first + dir * i;
            const unsigned shift = 16u * ((rs_par0 + (unsigned)h) & 1u);
            const int rsv = (int)((st.rs[buf][slot_in_warp][k] >> shift) & 0xffffu);
            row = rsv >> 6;
            sec = rsv & 63;
            valid = row < G.n_rows && sec < kNSectors;
            if (!valid) {
              status = 3;
              go = false;
              if (g == 0) record_error(a.err, kErrRowSector, trk);
            } else {
              const float2 d = reinterpret_cast<const float2*>(FRAMES ? lane_align : B.align)[sec * kMaxRows + row];
              m0 = st.y[buf][slot_in_warp][k] - d.x;
              m1 = st.z[buf][slot_in_warp][k] - d.y;
            }
          }
          const bool step = active && valid;
          const int sec18 = side_sector(sec);
          if (RECORD && step && (i & (kCkptEvery - 1)) == 0) {
            float* dst = a.ck + ((int64_t)pass * a.ck_slots + (begin >> kCkptShift) + trk + (i >> kCkptShift)) *
                                    kCkptFloats;
#pragma unroll
            for (int ii = 0; ii < 5; ++ii)
#pragma unroll
              for (int j = 0; j < NC; ++j)
                if (owns<P>(g, j)) dst[5 + 5 * ii + g + j * P] = F.Lc[ii][j];
            if (g == 0) {
#pragma unroll
              for (int c = 0; c < 5; ++c) dst[c] = p[c];
              dst[30] = x;
              dst[31] = __int_as_float(sec_cur);
            }
          }
          bool ok = step;
          Jac J;
          J.rot = false;
          J.yy = J.ss = 1.0f;
          J.ys = J.yq = J.zy = J.zs = J.zt = J.zq = J.sy = J.sq = 0.0f;
          float pn[5];
          if (step && i == 0) {
            x = Tb.row_x[row];
            sec_cur = sec18;
            if (pass == 0) {
              my = m0;
              mz = m1;
              p[0] = p[0] - m0;
              p[1] = p[1] - m1;
            }
          } else if (step) {
            PredTape tp;
            if (!predict_residual<0>(G, Tb, p, x, sec_cur, my, mz, sec18, Tb.row_x[row], m0, m1, pn, J, tp)) {
              go = false;
              ok = false;
              if (pass == 1) status = 2;  // the inward pass must reach the first cluster
            } else {
#pragma unroll
              for (int c = 0; c < 5; ++c) p[c] = pn[c];
              x = Tb.row_x[row];
              sec_cur = sec18;
              my = m0;
              mz = m1;
              transport_lanes<P>(F, J);
            }
          }
          // the updates' column sums need every lane of the warp: lanes whose
          // group takes no step here join with their (unchanged) state and
          // throw the result away
          float pk[5];
#pragma unroll
          for (int c = 0; c < 5; ++c) pk[c] = p[c];
          LaneFactor<P> Fk = F;
          float ck = chi2;
          scalar_update_lanes<P, 0>(G, pk, Fk, ck, base);
          scalar_update_lanes<P, 1>(G, pk, Fk, ck, base);
          if (ok) {
#pragma unroll
            for (int c = 0; c < 5; ++c) p[c] = pk[c];
            F = Fk;
            chi2 = ck;
            used += 1;
            if (pass == 0) last = i;
          }
        }
        __syncwarp();
        buf ^= 1;
      }
    }

    // ---- outputs at the track's own index (all lanes take part in the sums)
    if (RECORD && have && g == 0) a.ck_last[trk] = last;
    const int64_t N = a.n_tracks;
    const bool good = have && status == 0 && used >= 3;
    float cov[15];
    {
      int e = 0;
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
          float t[NC];
#pragma unroll
          for (int jj = 0; jj < NC; ++jj) t[jj] = F.Lc[i][jj] * F.Lc[j][jj];
          cov[e++] = col_sum<P>(t, base);
        }
    }
    if (!have || g != 0) continue;
    if (good) {
      a.params[trk] = my + p[0];
      a.params[N + trk] = mz + p[1];
#pragma unroll
      for (int c = 2; c < 5; ++c) a.params[(int64_t)c * N + trk] = p[c];
#pragma unroll
      for (int e = 0; e < 15; ++e) a.cov[(int64_t)e * N + trk] = cov[e];
      a.chi2[trk] = chi2;
      a.ndf[trk] = 2 * used - 5;
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

template <int P, int RPS, int WARPS, bool RECORD, bool FRAMES>
cudaError_t launch_lanes_cfg(const FitArgs& a, cudaStream_t s) {
  constexpr int kThreads = WARPS * 32;
  const size_t smem = sizeof(BlockSmem) + WARPS * sizeof(WarpStageLanes<P, RPS>);
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(fit_kernel_lanes<P, RPS, WARPS, RECORD, FRAMES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fit_kernel_lanes<P, RPS, WARPS, RECORD, FRAMES>,
                                                        kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = sms * per_sm;
  }
  constexpr int T = Lanes<P>::kTracks;
  const int64_t chunks = ((int64_t)a.n_tracks + T - 1) / T;
  const int64_t need = (chunks + WARPS - 1) / WARPS;
  const int blocks = (int)(need < grid ? need : grid);
  cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  fit_kernel_lanes<P, RPS, WARPS, RECORD, FRAMES><<<blocks, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Shapes with P lanes per track: 4 rows per stage, 24 warps per block.
template <bool RECORD, bool FRAMES>
inline cudaError_t launch_lanes_rec(const FitArgs& a, int lanes, cudaStream_t s) {
  switch (lanes) {
    case 2: return launch_lanes_cfg<2, 4, 24, RECORD, FRAMES>(a, s);
    case 4: return launch_lanes_cfg<4, 4, 24, RECORD, FRAMES>(a, s);
    case 8: return launch_lanes_cfg<8, 4, 24, RECORD, FRAMES>(a, s);
    case 16: return launch_lanes_cfg<16, 4, 24, RECORD, FRAMES>(a, s);
    case 32: return launch_lanes_cfg<32, 4, 24, RECORD, FRAMES>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

inline cudaError_t launch_lanes(const FitArgs& a, int lanes, cudaStream_t s) {
  if (a.frame_base) return a.ck ? launch_lanes_rec<true, true>(a, lanes, s) : launch_lanes_rec<false, true>(a, lanes, s);
  return a.ck ? launch_lanes_rec<true, false>(a, lanes, s) : launch_lanes_rec<false, false>(a, lanes, s);
}

}  // namespace TPCFIT_NS
}  // namespace tpcfit
