// CPU oracle for the batched TPC Kalman track fit -- TEST INFRASTRUCTURE ONLY.
//
// Only tests, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
// this library.  It shares no code, header, table or constant generator with
// the CUDA library: it is an independent, plain restatement of the fit.
//
// What it computes.  The paper (Sec. 4) names track propagation through the
// magnetic field as the shared component of TPC tracking and (Sec. 1) the time
// frame as the processing unit; it prints no fit formulas.  The fit below is
// the textbook extended Kalman filter (Fruehwirth, NIM A262 (1987) 444) for a
// helix in a uniform Bz field, in the local frame of a TPC sector, in the
// reading fixed for this project:
//   state p = (y, z, s = sin phi, t = tan lambda, q = q/pt) at local x,
//   covariance C packed lower-triangular (00,10,11,20,21,22,30,...,44),
//   outward pass from the seed (C0 = 100 * I, update at the first hit first),
//   inward refit from the outward result with C reset to C0 and chi2 reset,
//   output = inward state at the first hit, ndf = 2 * n_used - 5.
//
// Precision.  One template, three instantiations:
//   double       -- the FP64 accuracy reference;
//   float        -- the strict-FP32 build (compiled with -ffp-contract=off):
//                   the deterministic GPU mode must match it bit for bit.
//                   It follows the deterministic-mode rules of Sec. 2
//                   (no FMA, IEEE +,-,*,/,sqrt, fixed operation order,
//                   non-elementary functions evaluated by a fixed routine);
//   Dual         -- FP64 forward-mode derivatives, the gradient reference.
// The FP64 and Dual instantiations use the covariance form of the filter, the
// float one the square-root form (see Filter below).
//
// Every formula is written with explicit evaluation order; the float
// instantiation therefore defines the canonical FP32 operation sequence,
// including the residual coordinates for y and z (see fit_track).

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <vector>
#include <type_traits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kNSectorsPerSide = 18;
constexpr int kMaxRows = 256;
constexpr int kMaxD = 2 * 152 + 5;  // forward-mode directions: 2 per hit + 5 seed

std::atomic<long long> g_guard_hits{0};

// ------------------------------------------------------------------ dual numbers
// Forward-mode derivatives: a value of type VT and g_nd FP64 directional
// derivatives.  VT = double is the FP64 gradient reference.  VT = float
// evaluates the strict-FP32 operation sequence itself (the values are bit for
// bit those of the float instantiation) and carries the exact derivative of
// that sequence, every rounding treated as the identity, in FP64: the
// reference for a reverse-mode FP32 adjoint of the same sequence, free of the
// rounding of the derivatives themselves.
thread_local int g_nd = 0;

template <class VT> struct DualT;
template <class VT> DualT<VT> dual_add(const DualT<VT>& a, const DualT<VT>& b);
template <class VT> DualT<VT> dual_sub(const DualT<VT>& a, const DualT<VT>& b);
template <class VT> DualT<VT> dual_neg(const DualT<VT>& a);
template <class VT> DualT<VT> dual_mul(const DualT<VT>& a, const DualT<VT>& b);
template <class VT> DualT<VT> dual_div(const DualT<VT>& a, const DualT<VT>& b);

template <class VT> struct DualT {
  VT v;
  double d[kMaxD];
  DualT() : v(0) { std::memset(d, 0, sizeof(double) * (size_t)g_nd); }
  DualT(VT x) : v(x) { std::memset(d, 0, sizeof(double) * (size_t)g_nd); }  // NOLINT: constants enter implicitly
  // hidden friends, so that a constant operand converts implicitly
  friend DualT operator+(const DualT& a, const DualT& b) { return dual_add(a, b); }
  friend DualT operator-(const DualT& a, const DualT& b) { return dual_sub(a, b); }
  friend DualT operator-(const DualT& a) { return dual_neg(a); }
  friend DualT operator*(const DualT& a, const DualT& b) { return dual_mul(a, b); }
  friend DualT operator/(const DualT& a, const DualT& b) { return dual_div(a, b); }
};
template <class VT> DualT<VT> dual_add(const DualT<VT>& a, const DualT<VT>& b) {
  DualT<VT> r(a.v + b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class VT> DualT<VT> dual_sub(const DualT<VT>& a, const DualT<VT>& b) {
  DualT<VT> r(a.v - b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class VT> DualT<VT> dual_neg(const DualT<VT>& a) {
  DualT<VT> r(-a.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class VT> DualT<VT> dual_mul(const DualT<VT>& a, const DualT<VT>& b) {
  DualT<VT> r(a.v * b.v);
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * (double)b.v + (double)a.v * b.d[i];
  return r;
}
template <class VT> DualT<VT> dual_div(const DualT<VT>& a, const DualT<VT>& b) {
  DualT<VT> r(a.v / b.v);
  const double ib = 1.0 / (double)b.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <class VT> DualT<VT> dsqrt(const DualT<VT>& a) {
  DualT<VT> r(std::sqrt(a.v));
  const double h = 0.5 / (double)r.v;
  for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * h;
  return r;
}
using Dual = DualT<double>;
using DualF = DualT<float>;

// ------------------------------------------------------------------ scalar traits
template <class T> struct Traits;
template <> struct Traits<double> {
  using S = double;  // type of constants / tables
  static double val(double x) { return x; }
  static double sqrt_(double x) { return std::sqrt(x); }
  static constexpr double kLkSeries = 1e-5;  // |k dx| below which dl/dk uses its series
};
template <> struct Traits<float> {
  using S = float;
  static double val(float x) { return (double)x; }
  static float sqrt_(float x) { return std::sqrt(x); }  // IEEE, correctly rounded
  static constexpr double kLkSeries = 1e-2;
};
template <> struct Traits<Dual> {
  using S = double;
  static double val(const Dual& x) { return x.v; }
  static Dual sqrt_(const Dual& x) { return dsqrt(x); }
  static constexpr double kLkSeries = 1e-5;
};
template <> struct Traits<DualF> {
  using S = float;
  static double val(const DualF& x) { return (double)x.v; }
  static DualF sqrt_(const DualF& x) { return dsqrt(x); }
  static constexpr double kLkSeries = 1e-2;
};

// ------------------------------------------------------------------ arcsin routines
// FP64 arcsin from the Maclaurin series (Abramowitz & Stegun 4.4.40) for
// |u| <= 1/2 and asin u = pi/2 - 2 asin(sqrt((1-u)/2)) above; coefficients by the
// recurrence a_n = a_{n-1} (2n-1)^2 / ((2n)(2n+1)), a_0 = 1.
struct AsinTable {
  double a[30];
  AsinTable() {
    a[0] = 1.0;
    for (int n = 1; n < 30; ++n) {
      const double num = (double)(2 * n - 1) * (double)(2 * n - 1);
      const double den = (double)(2 * n) * (double)(2 * n + 1);
      a[n] = a[n - 1] * num / den;
    }
  }
};
const AsinTable g_asin;

double asin_series(double u) {  // |u| <= 0.5
  const double q = u * u;
  double acc = g_asin.a[29];
  for (int n = 28; n >= 0; --n) acc = acc * q + g_asin.a[n];
  return acc * u;
}
double asin_f64(double u) {
  const double au = u < 0.0 ? -u : u;
  double r;
  if (au <= 0.5) {
    r = asin_series(au);
  } else {
    const double h = std::sqrt((1.0 - au) * 0.5);
    r = 1.5707963267948966 - 2.0 * asin_series(h);
  }
  return u < 0.0 ? -r : r;
}

// asinc(u) = asin(u)/u.
// float: |u| <= 1/4 -> Horner in u^2 with the Maclaurin coefficients of asin(u)/u
//        rounded to float (c0..c6; truncation < 1e-10 there), else the FP64
//        routine above rounded to float (an FP64 island, as Sec. 2 does for
//        functions without a deterministic single-precision result).
inline float asinc_(float u) {
  const float au = u < 0.0f ? -u : u;
  if (au <= 0.25f) {
    const float c0 = 1.0f;
    const float c1 = (float)(1.0 / 6.0);
    const float c2 = (float)(3.0 / 40.0);
    const float c3 = (float)(5.0 / 112.0);
    const float c4 = (float)(35.0 / 1152.0);
    const float c5 = (float)(63.0 / 2816.0);
    const float c6 = (float)(231.0 / 13312.0);
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
  const double ud = (double)u;
  return (float)(asin_f64(ud) / ud);
}
inline double asinc_(double u) { return u == 0.0 ? 1.0 : std::asin(u) / u; }
inline Dual asinc_(const Dual& u) {
  const double x = u.v;
  double f, fp;
  if (std::fabs(x) < 1e-2) {
    const double q = x * x;
    f = 1.0 + q * (1.0 / 6.0 + q * (3.0 / 40.0 + q * (5.0 / 112.0 + q * (35.0 / 1152.0))));
    fp = x * (1.0 / 3.0 + q * (3.0 / 10.0 + q * (15.0 / 56.0 + q * (35.0 / 144.0))));
  } else {
    f = std::asin(x) / x;
    fp = (x / std::sqrt(1.0 - x * x) - std::asin(x)) / (x * x);
  }
  Dual r(f);
  for (int i = 0; i < g_nd; ++i) r.d[i] = u.d[i] * fp;
  return r;
}

// The strict-FP32 asinc with the exact derivative of what it evaluates (in
// FP64): the derivative of the float polynomial (coefficients as rounded) for
// |u| <= 1/4, of asin(u)/u above, where the value comes from the FP64 island.
inline DualF asinc_(const DualF& u) {
  const float x = u.v;
  const float f = asinc_(x);
  const double xd = (double)x;
  double fp;
  if ((x < 0.0f ? -x : x) <= 0.25f) {
    const double c[7] = {1.0, (double)(float)(1.0 / 6.0), (double)(float)(3.0 / 40.0), (double)(float)(5.0 / 112.0),
                         (double)(float)(35.0 / 1152.0), (double)(float)(63.0 / 2816.0),
                         (double)(float)(231.0 / 13312.0)};
    const double q = xd * xd;
    double acc = 6.0 * c[6];
    for (int k = 5; k >= 1; --k) acc = acc * q + (double)k * c[k];
    fp = 2.0 * xd * acc;
  } else {
    fp = (xd / std::sqrt((1.0 - xd) * (1.0 + xd)) - asin_f64(xd)) / (xd * xd);
  }
  DualF r(f);
  for (int i = 0; i < g_nd; ++i) r.d[i] = u.d[i] * fp;
  return r;
}

template <class T> inline double V(const T& x) { return Traits<T>::val(x); }
template <class T> inline T Sqrt(const T& x) { return Traits<T>::sqrt_(x); }

// ------------------------------------------------------------------ geometry
template <class S> struct Geo {
  int n_rows;
  S row_x[kMaxRows];
  S ca[kNSectorsPerSide][kNSectorsPerSide];  // rotation from sector a to sector b (mod 18)
  S sa[kNSectorsPerSide][kNSectorsPerSide];
  S kappa;
  S v_meas, c0, max_snp;
  // material along the path (off when mat = false): inverse radiation length,
  // minimum-ionising energy loss, squared mass of the particle (a pion)
  bool mat;
  S x0_inv, dedx, mass2, d_row;
  // field map Bz(r, z) = Bz0 (1 + c_r (r / 250)^2 + c_z (z / 250)^2) (off when field = false)
  bool field;
  S f_r, f_z;  // c_r / 250^2, c_z / 250^2 [1/cm^2]
  double inflate;  // inward restart from inflate * C_out (0: reset to C0)
};

// Rotation angle from sector a to b: m = (b - a) mod 18 taken in [-8, 9],
// dalpha = m * (w * pi / 180), cos / sin in FP64, then the constant type.
template <class S> void make_geo(Geo<S>& g, const double* row_x, int n_rows, double width_deg, double bz,
                                  double x0_cm = 0.0, double dedx = 0.0, double mass = 0.0, double d_row = 0.0,
                                  double c_r = 0.0, double c_z = 0.0) {
  g.n_rows = n_rows;
  for (int r = 0; r < n_rows; ++r) g.row_x[r] = (S)row_x[r];
  const double w_rad = width_deg * 3.14159265358979323846 / 180.0;
  for (int a = 0; a < kNSectorsPerSide; ++a)
    for (int b = 0; b < kNSectorsPerSide; ++b) {
      int m = ((b - a) % kNSectorsPerSide + kNSectorsPerSide) % kNSectorsPerSide;
      if (m > 9) m -= kNSectorsPerSide;
      const double da = (double)m * w_rad;
      g.ca[a][b] = (S)std::cos(da);
      g.sa[a][b] = (S)std::sin(da);
    }
  g.kappa = (S)(-0.00299792458 * bz);
  g.v_meas = (S)0.01;   // sigma_y = sigma_z = 0.1 cm
  g.c0 = (S)100.0;      // initial covariance diag(1e2)
  g.max_snp = (S)0.999;
  g.mat = x0_cm > 0.0 && std::isfinite(x0_cm);
  g.x0_inv = (S)(g.mat ? 1.0 / x0_cm : 0.0);
  g.dedx = (S)(g.mat ? dedx : 0.0);
  g.mass2 = (S)(mass * mass);
  g.d_row = (S)d_row;
  g.field = c_r != 0.0 || c_z != 0.0;
  g.f_r = (S)(c_r / (250.0 * 250.0));
  g.f_z = (S)(c_z / (250.0 * 250.0));
  g.inflate = 0.0;
}

// packed index of (i, j), i >= j
inline int P(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// ------------------------------------------------------------------ Jacobian
template <class T> struct Jac {
  bool rot;
  T yy, ys, yq, zy, zs, zt, zq, sy, ss, sq;
};

// ------------------------------------------------------------------ material
// A thin layer of material at every pad row (a uniform material budget per
// row), in the reading fixed for this project.  The state at a row is the one
// the track leaves it with.  The particle is a pion.  With the state at the
// row (s, t, q) the layer is crossed over l = d sqrt(1 + t^2) / c,
// c = sqrt(1 - s^2) (d its thickness at normal incidence); p^2 = (1 + t^2)/q^2,
// E^2 = p^2 + m^2, beta^2 = p^2 / E^2:
//  * energy loss: dE = dEdx_mip l / beta^2 (the 1/beta^2 rise, no logarithmic
//    term); E' = E - dir dE (dir = +1: crossed along the flight, which the
//    outward pass does on arriving at a row; -1: undone, which the inward pass
//    does before leaving a row against the flight); q' = q p / p'; the
//    Jacobian's q row is scaled by p / p' (its dependence on the state is
//    neglected);
//  * multiple scattering (Highland without its logarithmic term):
//    theta0^2 = 0.0136^2 l / X0 / (beta^2 p^2); two independent plane angles
//    th1 (bending plane), th2: ds = c / cos(lambda) th1, dt = (1 + t^2) th2,
//    dq = q' t th2, i.e. process noise Q = B B^T with
//    B = [theta0 c sqrt(1 + t^2) e_s | theta0 ((1 + t^2) e_t + q' t e_q)].
// A particle that would stop (E' <= m) makes the step impossible.
template <class T> struct Noise {
  T qq;        // p / p'
  T b_s;       // B: s entry of the first column
  T b_t, b_q;  // t and q entries of the second column
};

template <class T>
bool material_step(const Geo<typename Traits<T>::S>& g, T p[5], int dir, Noise<T>& N) {
  using S = typename Traits<T>::S;
  const S one = (S)1.0;
  const T& s = p[2];
  const T& t = p[3];
  const T q = p[4];
  const T q2 = q * q;
  if (!(V(q2) > 0.0)) {  // infinite momentum: no scattering, no loss
    N.qq = T(one);
    N.b_s = T((S)0.0);
    N.b_t = T((S)0.0);
    N.b_q = T((S)0.0);
    return true;
  }
  const T tt1 = one + t * t;
  const T c = Sqrt((one - s) * (one + s));
  const T st1 = Sqrt(tt1);
  const T ell = (g.d_row * st1) / c;
  const T p2 = tt1 / q2;
  const T e2 = p2 + g.mass2;
  const T th2 = (((S)(0.0136 * 0.0136) * ell) * g.x0_inv) * (e2 / (p2 * p2));
  const T de = (g.dedx * ell) * (e2 / p2);
  const T e = Sqrt(e2);
  const T en = dir > 0 ? e - de : e + de;
  const T pn2 = en * en - g.mass2;
  if (!(V(pn2) > 0.0)) return false;
  const T ratio = Sqrt(p2 / pn2);
  p[4] = q * ratio;
  const T th = Sqrt(th2);
  N.qq = ratio;
  N.b_s = (th * c) * st1;
  N.b_t = th * tt1;
  N.b_q = (th * p[4]) * t;
  return true;
}

// ------------------------------------------------------------------ one prediction step
// Moves state (p, x) in sector sec_from to pad row X in sector sec_to:
// optional rotation to the new sector's frame, then helix propagation to local
// x = X.  Returns false (state untouched) if the step is not possible.
//
// Field map (g.field): the step's curvature uses Bz at the step's midpoint,
// estimated by a straight half step from the start point (after the
// rotation): x_m = x1 + dx/2, y_m = y1 + (dx/2) s1/c1, z_m = z1 + (dx/2) t/c1,
// kappa_step = kappa (1 + f_r (x_m^2 + y_m^2) + f_z z_m^2).  The midpoint makes
// an arc's curvature the same in both directions.  The Jacobian treats
// kappa_step as a constant (its dependence on the state is neglected).
// (yo, zo): what to add to pin[0], pin[1] for absolute positions (residual form).
template <class T>
bool predict(const Geo<typename Traits<T>::S>& g, const T pin[5], const T& xin, int sec_from, int sec_to,
             typename Traits<T>::S X, T pout[5], T& xout, Jac<T>& J, const T& yo = T(0.0), const T& zo = T(0.0)) {
  using S = typename Traits<T>::S;
  const S one = (S)1.0, half = (S)0.5;
  T kappa = T(g.kappa);
  const double maxsnp = (double)g.max_snp;
  const int a = sec_from % kNSectorsPerSide, b = sec_to % kNSectorsPerSide;
  T x1 = xin, y1 = pin[0], s1 = pin[2];
  const T& t = pin[3];
  const T& q = pin[4];
  J.rot = (a != b);
  T cprev(0.0), crot(0.0);
  S ca = one, sa = (S)0.0;
  if (J.rot) {
    ca = g.ca[a][b];
    sa = g.sa[a][b];
    const T s = pin[2];
    const T c = Sqrt((one - s) * (one + s));
    const T xr = xin * ca + pin[0] * sa;
    const T yr = pin[0] * ca - xin * sa;
    const T sr = s * ca - c * sa;
    const T cr = c * ca + s * sa;
    if (!(V(cr) > 0.0)) return false;
    if (!(std::fabs(V(sr)) < maxsnp)) return false;
    x1 = xr; y1 = yr; s1 = sr; cprev = c; crot = cr;
  }
  const T dx = T(X) - x1;
  if (g.field) {
    const T c1f = Sqrt((one - s1) * (one + s1));
    const T hdx = dx * half;
    const T ym = (yo + y1) + hdx * (s1 / c1f);
    const T zm = (zo + pin[1]) + hdx * (t / c1f);
    const T xm = x1 + hdx;
    kappa = kappa * ((one + g.f_r * (xm * xm + ym * ym)) + g.f_z * (zm * zm));
  }
  const T k = q * kappa;
  const T kdx = k * dx;
  const T s2 = s1 + kdx;
  if (!(std::fabs(V(s2)) < maxsnp)) return false;
  const T c1 = Sqrt((one - s1) * (one + s1));
  const T c2 = Sqrt((one - s2) * (one + s2));
  const T Tm = (s1 + s2) / (c1 + c2);
  const T w = c1 + s1 * Tm;
  const T sig = kdx * w;
  const T dl = (dx * w) * asinc_(sig);
  pout[0] = y1 + dx * Tm;
  pout[1] = pin[1] + t * dl;
  pout[2] = s2;
  pout[3] = t;
  pout[4] = q;
  xout = T(X);
  // analytic Jacobian of the propagation at fixed dx
  const T ic1 = one / c1;
  const T ic2 = one / c2;
  const T tt = one + Tm * Tm;
  J.ys = (dx * tt) * ((ic1 + ic2) * half);
  J.yq = ((dx * kappa) * dx) * (tt * (ic2 * half));
  J.zs = (t * dx) * (Tm * (ic1 * ic2));
  J.zt = dl;
  T Lk;  // d(dl)/dk
  if (std::fabs(V(kdx)) < Traits<T>::kLkSeries) {
    const T i2 = ic1 * ic1;
    const T i3 = i2 * ic1;
    const T i5 = i3 * i2;
    const T i7 = i5 * i2;
    const T s1s = s1 * s1;
    const T a1 = (s1 * i3) * half;
    const T a2 = ((one + (S)2.0 * s1s) * i5) * (S)(1.0 / 3.0);
    const T a3 = ((s1 * ((S)3.0 + (S)2.0 * s1s)) * i7) * (S)0.125;
    Lk = (dx * dx) * (a1 + kdx * (a2 + kdx * a3));
  } else {
    Lk = (dx * ic2 - dl) / k;
  }
  J.zq = (t * kappa) * Lk;
  J.sq = dx * kappa;
  if (J.rot) {
    // chain rule through the rotated start point: x1 depends on the old y
    // (dx1/dy = sa), s1 on the old s (ds1/ds = c'/c)
    const T rr = crot / cprev;
    J.yy = T(ca) - sa * (s2 * ic2);
    J.zy = -(sa * (t * ic2));
    J.sy = -(sa * k);
    J.ss = rr;
    J.ys = J.ys * rr;
    J.zs = J.zs * rr;
  } else {
    J.yy = T(one); J.zy = T(0.0); J.sy = T(0.0); J.ss = T(one);
  }
  return true;
}

// ------------------------------------------------------------------ covariance transport
// C <- J C J^T with A = J C first (rows y, z, s; t and q rows are identity),
// then C'_ij = sum_k A_ik J_jk for i >= j, k ascending, structural zeros skipped.
template <class T> void transport(T C[15], const Jac<T>& J) {
  T M[5][5];
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) M[i][j] = C[P(i, j)];
  T A[5][5];
  for (int j = 0; j < 5; ++j) {
    if (!J.rot) {
      A[0][j] = (M[0][j] + J.ys * M[2][j]) + J.yq * M[4][j];
      A[1][j] = ((M[1][j] + J.zs * M[2][j]) + J.zt * M[3][j]) + J.zq * M[4][j];
      A[2][j] = M[2][j] + J.sq * M[4][j];
    } else {
      A[0][j] = (J.yy * M[0][j] + J.ys * M[2][j]) + J.yq * M[4][j];
      A[1][j] = (((J.zy * M[0][j] + M[1][j]) + J.zs * M[2][j]) + J.zt * M[3][j]) + J.zq * M[4][j];
      A[2][j] = (J.sy * M[0][j] + J.ss * M[2][j]) + J.sq * M[4][j];
    }
    A[3][j] = M[3][j];
    A[4][j] = M[4][j];
  }
  for (int i = 0; i < 5; ++i) {
    if (!J.rot) {
      C[P(i, 0)] = (A[i][0] + J.ys * A[i][2]) + J.yq * A[i][4];
      if (i >= 1) C[P(i, 1)] = ((A[i][1] + J.zs * A[i][2]) + J.zt * A[i][3]) + J.zq * A[i][4];
      if (i >= 2) C[P(i, 2)] = A[i][2] + J.sq * A[i][4];
    } else {
      C[P(i, 0)] = (J.yy * A[i][0] + J.ys * A[i][2]) + J.yq * A[i][4];
      if (i >= 1) C[P(i, 1)] = (((J.zy * A[i][0] + A[i][1]) + J.zs * A[i][2]) + J.zt * A[i][3]) + J.zq * A[i][4];
      if (i >= 2) C[P(i, 2)] = (J.sy * A[i][0] + J.ss * A[i][2]) + J.sq * A[i][4];
    }
    if (i >= 3) C[P(i, 3)] = A[i][3];
    if (i >= 4) C[P(i, 4)] = A[i][4];
  }
}

// ------------------------------------------------------------------ filter state
// Two algebraically identical forms of the same Kalman filter:
//  * covariance form (kSqrt = false): C packed lower-triangular, C <- J C J^T,
//    joint 2D update.  The FP64 reference and the gradient reference use it.
//  * square-root (Potter) form (kSqrt = true): C = L L^T with L a general 5x5
//    factor, L <- J L, and the 2D cluster processed as two scalar updates (y
//    then z; exact for the diagonal V).  The FP32 canonical sequence uses it:
//    it keeps C symmetric and positive semi-definite by construction and halves
//    the digits lost when a diffuse C0 meets a precise cluster (Potter 1963;
//    Bierman, "Factorization Methods for Discrete Sequential Estimation", 1977).
template <class T, bool kSqrt> struct Filter;

template <class T> struct Filter<T, false> {
  using S = typename Traits<T>::S;
  T C[15];
  void init(const Geo<S>& g) {
    for (int e = 0; e < 15; ++e) C[e] = T((S)0.0);
    for (int i = 0; i < 5; ++i) C[P(i, i)] = T(g.c0);
  }
  void transport_(const Jac<T>& J) { transport<T>(C, J); }
  void cov(T out[15]) const { for (int e = 0; e < 15; ++e) out[e] = C[e]; }
  void scale(double k) { for (int e = 0; e < 15; ++e) C[e] = C[e] * T((S)k); }
  // C <- D C D + B B^T, D = diag(1, 1, 1, 1, qq)
  void material_(const Noise<T>& N) {
    for (int j = 0; j < 4; ++j) C[P(4, j)] = C[P(4, j)] * N.qq;
    C[P(4, 4)] = (C[P(4, 4)] * N.qq) * N.qq;
    C[P(2, 2)] = C[P(2, 2)] + N.b_s * N.b_s;
    C[P(3, 3)] = C[P(3, 3)] + N.b_t * N.b_t;
    C[P(4, 3)] = C[P(4, 3)] + N.b_q * N.b_t;
    C[P(4, 4)] = C[P(4, 4)] + N.b_q * N.b_q;
  }

  // 2D measurement of (y, z), V = diag(v, v).  Gain from the 2x2 innovation
  // covariance S; chi2 increment r^T S^-1 r with the predicted residual r.
  // Afterwards the positive-definiteness guard: a diagonal element that is not
  // positive is set to 1e-12; an off-diagonal element with C_ij^2 above
  // (1 - 2^-10) C_ii C_jj (a check in the working precision) enters an FP64
  // island that clamps |C_ij| to (1 - 1e-6) sqrt(C_ii C_jj).
  bool update(const Geo<S>& g, T p[5], T& chi2, const T m[2]) {
    const S v = g.v_meas;
    const T S00 = C[0] + v;
    const T S10 = C[1];
    const T S11 = C[2] + v;
    const T det = S00 * S11 - S10 * S10;
    if (!(V(det) > 0.0)) return false;
    const T idet = T((S)1.0) / det;
    const T Si00 = S11 * idet;
    const T Si10 = -(S10 * idet);
    const T Si11 = S00 * idet;
    T K[5][2];
    for (int i = 0; i < 5; ++i) {
      const T& ci0 = C[P(i, 0)];
      const T& ci1 = C[P(i, 1)];
      K[i][0] = ci0 * Si00 + ci1 * Si10;
      K[i][1] = ci0 * Si10 + ci1 * Si11;
    }
    const T r0 = m[0] - p[0];
    const T r1 = m[1] - p[1];
    const T dchi2 = r0 * (Si00 * r0 + Si10 * r1) + r1 * (Si10 * r0 + Si11 * r1);
    chi2 = chi2 + dchi2;
    for (int i = 0; i < 5; ++i) p[i] = p[i] + (K[i][0] * r0 + K[i][1] * r1);
    T Cn[15];
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j <= i; ++j) Cn[P(i, j)] = C[P(i, j)] - (K[i][0] * C[P(0, j)] + K[i][1] * C[P(1, j)]);
    for (int e = 0; e < 15; ++e) C[e] = Cn[e];
    for (int i = 0; i < 5; ++i)
      if (!(V(C[P(i, i)]) > 0.0)) {
        C[P(i, i)] = T((S)1e-12);
        g_guard_hits.fetch_add(1, std::memory_order_relaxed);
      }
    const S thr = (S)(1.0 - 1.0 / 1024.0);
    for (int i = 1; i < 5; ++i)
      for (int j = 0; j < i; ++j) {
        const T cij = C[P(i, j)];
        const T lhs = cij * cij;
        const T rhs = thr * (C[P(i, i)] * C[P(j, j)]);
        if (V(lhs) > V(rhs)) {
          const double b = (1.0 - 1e-6) * std::sqrt(V(C[P(i, i)]) * V(C[P(j, j)]));
          if (std::fabs(V(cij)) > b) {
            C[P(i, j)] = T((S)(V(cij) > 0.0 ? b : -b));
            g_guard_hits.fetch_add(1, std::memory_order_relaxed);
          }
        }
      }
    return true;
  }
};

template <class T> struct Filter<T, true> {
  using S = typename Traits<T>::S;
  T L[5][5];  // C = L L^T
  void init(const Geo<S>& g) {
    const S l0 = (S)std::sqrt((double)g.c0);
    for (int i = 0; i < 5; ++i)
      for (int c = 0; c < 5; ++c) L[i][c] = T(i == c ? l0 : (S)0.0);
  }
  void scale(double k) {
    const S r = (S)std::sqrt(k);
    for (int i = 0; i < 5; ++i)
      for (int c = 0; c < 5; ++c) L[i][c] = L[i][c] * T(r);
  }
  // L <- J L: only rows y, z, s change (rows t, q of J are identity).
  void transport_(const Jac<T>& J) {
    for (int c = 0; c < 5; ++c) {
      T ny, nz, ns;
      if (!J.rot) {
        ny = (L[0][c] + J.ys * L[2][c]) + J.yq * L[4][c];
        nz = ((L[1][c] + J.zs * L[2][c]) + J.zt * L[3][c]) + J.zq * L[4][c];
        ns = L[2][c] + J.sq * L[4][c];
      } else {
        ny = (J.yy * L[0][c] + J.ys * L[2][c]) + J.yq * L[4][c];
        nz = (((J.zy * L[0][c] + L[1][c]) + J.zs * L[2][c]) + J.zt * L[3][c]) + J.zq * L[4][c];
        ns = (J.sy * L[0][c] + J.ss * L[2][c]) + J.sq * L[4][c];
      }
      L[0][c] = ny;
      L[1][c] = nz;
      L[2][c] = ns;
    }
  }
  // L <- D L, then the noise folded in: with X = [L^T; B^T] (7x5) and its
  // Householder QR X = Q R, L R^T R = L L^T + B B^T, so L <- R^T (lower
  // triangular).  Canonical sequence, column k = 0..4: |x|^2 of rows k..6 (row
  // ascending), alpha = -sign(x_k) |x|, v = x - alpha e_k, g = 1 / (alpha v_k);
  // every later column j (ascending): t = (v_k X_kj + sum_{r>k} X_rk X_rj) g,
  // X_kj += t v_k, X_rj += t X_rk (r ascending); then X_kk = alpha.
  void material_(const Noise<T>& N) {
    using SS = typename Traits<T>::S;
    for (int c = 0; c < 5; ++c) L[4][c] = L[4][c] * N.qq;
    T X[7][5];
    for (int r = 0; r < 5; ++r)
      for (int i = 0; i < 5; ++i) X[r][i] = L[i][r];
    for (int i = 0; i < 5; ++i) {
      X[5][i] = T((SS)0.0);
      X[6][i] = T((SS)0.0);
    }
    X[5][2] = N.b_s;
    X[6][3] = N.b_t;
    X[6][4] = N.b_q;
    for (int k = 0; k < 5; ++k) {
      T nrm2 = X[k][k] * X[k][k];
      for (int r = k + 1; r < 7; ++r) nrm2 = nrm2 + X[r][k] * X[r][k];
      const T nrm = Sqrt(nrm2);
      const T alpha = V(X[k][k]) > 0.0 ? T((SS)0.0) - nrm : nrm;
      const T v0 = X[k][k] - alpha;
      const T gk = T((SS)1.0) / (alpha * v0);
      for (int j = k + 1; j < 5; ++j) {
        T t = v0 * X[k][j];
        for (int r = k + 1; r < 7; ++r) t = t + X[r][k] * X[r][j];
        t = t * gk;
        X[k][j] = X[k][j] + t * v0;
        for (int r = k + 1; r < 7; ++r) X[r][j] = X[r][j] + t * X[r][k];
      }
      X[k][k] = alpha;
    }
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) L[i][j] = j <= i ? X[j][i] : T((SS)0.0);
  }
  // C_ij = sum_c L_ic L_jc, c ascending
  void cov(T out[15]) const {
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j <= i; ++j) {
        T acc = L[i][0] * L[j][0];
        for (int c = 1; c < 5; ++c) acc = acc + L[i][c] * L[j][c];
        out[P(i, j)] = acc;
      }
  }
  // Potter's scalar update for component h (0 = y, 1 = z) with value mv:
  //   a = L^T e_h (row h of L), s2 = v + a.a, alpha = 1/s2, K = alpha L a,
  //   p += K r, chi2 += r^2 alpha, beta = sqrt(alpha v), gamma = 1/(1 + beta),
  //   L <- L - gamma K a^T, whose row h equals beta a exactly (used as such).
  void scalar_update(const Geo<S>& g, T p[5], T& chi2, int h, const T& mv) {
    const S v = g.v_meas;
    T a[5];
    for (int c = 0; c < 5; ++c) a[c] = L[h][c];
    T s2 = T(v) + a[0] * a[0];
    for (int c = 1; c < 5; ++c) s2 = s2 + a[c] * a[c];
    const T alpha = T((S)1.0) / s2;
    const T r = mv - p[h];
    T K[5];
    for (int i = 0; i < 5; ++i) {
      T la = L[i][0] * a[0];
      for (int c = 1; c < 5; ++c) la = la + L[i][c] * a[c];
      K[i] = la * alpha;
    }
    for (int i = 0; i < 5; ++i) p[i] = p[i] + K[i] * r;
    chi2 = chi2 + (r * r) * alpha;
    const T beta = Sqrt(alpha * v);
    const T gamma = T((S)1.0) / (T((S)1.0) + beta);
    for (int i = 0; i < 5; ++i) {
      if (i == h) continue;
      const T gk = gamma * K[i];
      for (int c = 0; c < 5; ++c) L[i][c] = L[i][c] - gk * a[c];
    }
    for (int c = 0; c < 5; ++c) L[h][c] = a[c] * beta;
  }
  bool update(const Geo<S>& g, T p[5], T& chi2, const T m[2]) {
    scalar_update(g, p, chi2, 0, m[0]);
    scalar_update(g, p, chi2, 1, m[1]);
    return true;
  }
};

// ------------------------------------------------------------------ track fit
template <class T> struct HitView {
  const T* y;
  const T* z;
  const uint16_t* rowsec;
  const T* align;  // [36][152][2] or null
  int64_t begin;
  int n;
};

template <class T> inline int hit_row(const HitView<T>& h, int j) { return (int)(h.rowsec[h.begin + j] >> 6); }
template <class T> inline int hit_sec(const HitView<T>& h, int j) { return (int)(h.rowsec[h.begin + j] & 63); }

template <class T> void meas(const HitView<T>& h, int j, const T& yv, const T& zv, T m[2]) {
  if (h.align) {
    const int64_t key = ((int64_t)hit_sec(h, j) * 152 + hit_row(h, j)) * 2;
    m[0] = yv - h.align[key];
    m[1] = zv - h.align[key + 1];
  } else {
    m[0] = yv;
    m[1] = zv;
  }
}

struct FitResult {
  int ok;
  int n_used;
};

// Linearised variant (ref != null): every prediction is the affine map
// p' = f(ref_a) + J(ref_a) (p - ref_a) about the reference state of the hit the
// step starts from; with it the filter is exactly linear-Gaussian.
template <class T, bool kSqrt>
FitResult fit_track(const Geo<typename Traits<T>::S>& g, const HitView<T>& h, const T* yv, const T* zv,
                    const T seed[5], const double* ref /*[n][5] or null*/, T p_out[5], T C_out[15], T& chi2_out,
                    double* trace /*[n][2][22] or null*/, double* ptrace = nullptr /*[n][2][20] or null*/) {
  using S = typename Traits<T>::S;
  FitResult res{0, 0};
  const int n = h.n;
  if (n < 1) return res;
  T p[5];
  Filter<T, kSqrt> F;
  T x;
  T chi2(0.0);
  constexpr bool kRes = std::is_same<typename Traits<T>::S, float>::value;  // residual coordinates (see below)
  T my(0.0), mz(0.0);                                    // measurement of the current cluster
  auto record = [&](int pass, int j) {
    if (!trace) return;
    double* o = trace + ((size_t)j * 2 + pass) * 22;
    T C[15];
    F.cov(C);
    for (int i = 0; i < 5; ++i) o[i] = V(p[i]);
    if (kRes && !ref) {  // residual form: report positions
      o[0] = (double)(float)(V(my) + V(p[0]));
      o[1] = (double)(float)(V(mz) + V(p[1]));
    }
    for (int e = 0; e < 15; ++e) o[5 + e] = V(C[e]);
    o[20] = V(chi2);
    o[21] = V(x);
  };
  // predicted state (p, C) at hit j of a pass, before its update: the two
  // predictions of a hit are the inputs of the two-filter smoother
  auto precord = [&](int pass, int j) {
    if (!ptrace) return;
    double* o = ptrace + ((size_t)j * 2 + pass) * 20;
    T C[15];
    F.cov(C);
    for (int i = 0; i < 5; ++i) o[i] = V(p[i]);
    if (kRes && !ref) {
      o[0] = (double)(float)(V(my) + V(p[0]));
      o[1] = (double)(float)(V(mz) + V(p[1]));
    }
    for (int e = 0; e < 15; ++e) o[5 + e] = V(C[e]);
  };
  // FP32 sequence: y and z are carried as residuals from the measurement of the
  // current cluster (p[0] = y - m_y, p[1] = z - m_z), so that their rounding is
  // that of ~0.1 cm quantities instead of positions up to 250 cm.  The helix
  // step adds the exact difference of consecutive measurements; across a
  // sector rotation the absolute position is formed, rotated and re-referenced.
  // The FP64 and dual instantiations keep absolute coordinates.
  auto step = [&](int from, int to, int pass) -> bool {
    if (g.mat && pass == 1) {  // the layer of the row left against the flight, undone first
      Noise<T> N;
      if (!material_step<T>(g, p, -1, N)) return false;
      F.material_(N);
    }
    const int r = hit_row(h, to);
    if (r < 0 || r >= g.n_rows) return false;
    Jac<T> J;
    T pn[5];
    T xn;
    T mt[2];
    meas<T>(h, to, yv[to], zv[to], mt);
    if (!ref) {
      if (kRes) {
        const bool rot = (hit_sec(h, from) % kNSectorsPerSide) != (hit_sec(h, to) % kNSectorsPerSide);
        T pin[5];
        for (int i = 0; i < 5; ++i) pin[i] = p[i];
        if (rot) {
          pin[0] = my + p[0];
          pin[1] = mz + p[1];
        }
        const T zero((S)0.0);
        if (!predict<T>(g, pin, x, hit_sec(h, from), hit_sec(h, to), g.row_x[r], pn, xn, J, rot ? zero : my,
                        rot ? zero : mz))
          return false;
        if (rot) {
          pn[0] = pn[0] - mt[0];
          pn[1] = pn[1] - mt[1];
        } else {
          pn[0] = pn[0] + (my - mt[0]);
          pn[1] = pn[1] + (mz - mt[1]);
        }
      } else if (!predict<T>(g, p, x, hit_sec(h, from), hit_sec(h, to), g.row_x[r], pn, xn, J)) {
        return false;
      }
    } else {
      T pr[5];
      for (int i = 0; i < 5; ++i) pr[i] = T((S)ref[(size_t)from * 5 + i]);
      T xr = T(g.row_x[hit_row(h, from)]);
      T fr[5];
      if (!predict<T>(g, pr, xr, hit_sec(h, from), hit_sec(h, to), g.row_x[r], fr, xn, J)) return false;
      // p' = f(ref) + J (p - ref)
      T d[5];
      for (int i = 0; i < 5; ++i) d[i] = p[i] - pr[i];
      pn[0] = fr[0] + ((J.yy * d[0] + J.ys * d[2]) + J.yq * d[4]);
      pn[1] = fr[1] + ((((J.zy * d[0] + d[1]) + J.zs * d[2]) + J.zt * d[3]) + J.zq * d[4]);
      pn[2] = fr[2] + ((J.sy * d[0] + J.ss * d[2]) + J.sq * d[4]);
      pn[3] = fr[3] + d[3];
      pn[4] = fr[4] + d[4];
    }
    Noise<T> N;
    // the layer of the row arrived at, crossed along the flight (a particle
    // that stops there ends the pass with the state before the step)
    if (g.mat && pass == 0 && !material_step<T>(g, pn, 1, N)) return false;
    // the step is taken: state, position and (residual form) the reference
    // measurement move to the new cluster together
    for (int i = 0; i < 5; ++i) p[i] = pn[i];
    x = xn;
    if (kRes && !ref) {
      my = mt[0];
      mz = mt[1];
    }
    F.transport_(J);
    if (g.mat && pass == 0) F.material_(N);
    T m[2] = {mt[0], mt[1]};
    if (kRes && !ref) {
      m[0] = T((S)0.0);
      m[1] = T((S)0.0);
    }
    precord(pass, to);
    return F.update(g, p, chi2, m);
  };
  // ---- outward pass
  const int r0 = hit_row(h, 0);
  if (r0 < 0 || r0 >= g.n_rows) return res;
  for (int i = 0; i < 5; ++i) p[i] = seed[i];
  if (!(std::fabs(V(p[2])) < (double)g.max_snp)) return res;
  x = T(g.row_x[r0]);
  F.init(g);
  {
    T m[2];
    meas<T>(h, 0, yv[0], zv[0], m);
    if (kRes && !ref) {
      my = m[0];
      mz = m[1];
      p[0] = p[0] - my;
      p[1] = p[1] - mz;
      m[0] = T((S)0.0);
      m[1] = T((S)0.0);
    }
    precord(0, 0);
    if (!F.update(g, p, chi2, m)) return res;
  }
  record(0, 0);
  int last = 0;
  for (int j = 1; j < n; ++j) {
    if (!step(j - 1, j, 0)) break;  // the outward pass ends at the last good hit
    last = j;
    record(0, j);
  }
  // ---- inward refit
  if (g.inflate > 0.0) F.scale(g.inflate);  // test-only reading: an informative restart
  else F.init(g);
  chi2 = T((S)0.0);
  int used = 0;
  {
    T m[2];
    meas<T>(h, last, yv[last], zv[last], m);
    if (kRes && !ref) {
      m[0] = T((S)0.0);
      m[1] = T((S)0.0);
    }
    precord(1, last);
    if (!F.update(g, p, chi2, m)) return res;
  }
  ++used;
  record(1, last);
  for (int j = last - 1; j >= 0; --j) {
    if (!step(j + 1, j, 1)) return res;
    ++used;
    record(1, j);
  }
  if (used < 3) return res;
  for (int i = 0; i < 5; ++i) p_out[i] = p[i];
  if (kRes && !ref) {
    p_out[0] = my + p[0];
    p_out[1] = mz + p[1];
  }
  F.cov(C_out);
  chi2_out = chi2;
  res.ok = 1;
  res.n_used = used;
  return res;
}

struct OracleGeometry {
  const double* row_x;
  int32_t n_rows;
  int32_t n_sectors;
  double sector_width_deg;
  double x0_cm;        // radiation length of the material (<= 0: no material)
  double dedx_gev_cm;  // minimum-ionising energy loss
  double mass_gev;     // particle mass
  double row_cm;       // thickness of the material layer at each pad row (normal incidence)
  double field_cr;     // field map Bz(r, z) = Bz0 (1 + field_cr (r/250)^2 + field_cz (z/250)^2)
  double field_cz;
  // Test-only alternative reading of the inward restart (0: the product
  // reading, C reset to C0): the inward pass starts from the outward result
  // with C = inward_inflate * C_out, an informative prior instead of the
  // diffuse one.  It exists to show where the EKF's pull excess comes from.
  double inward_inflate;
};

int check_inputs(const OracleGeometry* geo, int32_t n_tracks, const int32_t* off) {
  if (!geo || !geo->row_x || geo->n_rows <= 0 || geo->n_rows > kMaxRows || geo->n_sectors != 36) return 1;
  if (n_tracks < 0) return 1;
  if (n_tracks > 0 && !off) return 1;
  for (int32_t i = 0; i < n_tracks; ++i)
    if (off[i + 1] < off[i]) return 1;
  return 0;
}

template <class T, bool kSqrt>
int fit_all(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const T* y, const T* z,
            const uint16_t* rowsec, const T* seeds, const T* align, const double* ref, T* params, T* cov, T* chi2,
            int32_t* ndf, double* trace, int32_t nthreads, double* ptrace = nullptr) {
  using S = typename Traits<T>::S;
  if (check_inputs(geo, n_tracks, off)) return 1;
  Geo<S> g;
  make_geo<S>(g, geo->row_x, geo->n_rows, geo->sector_width_deg, bz, geo->x0_cm, geo->dedx_gev_cm, geo->mass_gev, geo->row_cm,
               geo->field_cr, geo->field_cz);
  g.inflate = geo->inward_inflate;
  if ((g.mat || g.field) && ref) return 1;  // the linearised filter has neither material nor a field map
  const T nan = T((S)NAN);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
  for (int32_t i = 0; i < n_tracks; ++i) {
    HitView<T> h{y, z, rowsec, align, off[i], off[i + 1] - off[i]};
    T seed[5];
    for (int c = 0; c < 5; ++c) seed[c] = seeds[(size_t)c * n_tracks + i];
    T p[5], C[15], c2((S)0.0);
    const double* tref = ref ? ref + (size_t)off[i] * 5 : nullptr;
    double* ttr = trace ? trace + (size_t)off[i] * 2 * 22 : nullptr;
    if (ttr)
      for (int64_t e = 0; e < (int64_t)h.n * 2 * 22; ++e) ttr[e] = NAN;
    double* tpt = ptrace ? ptrace + (size_t)off[i] * 2 * 20 : nullptr;
    if (tpt)
      for (int64_t e = 0; e < (int64_t)h.n * 2 * 20; ++e) tpt[e] = NAN;
    FitResult r = fit_track<T, kSqrt>(g, h, y + off[i], z + off[i], seed, tref, p, C, c2, ttr, tpt);
    if (r.ok) {
      for (int c = 0; c < 5; ++c) params[(size_t)c * n_tracks + i] = p[c];
      for (int e = 0; e < 15; ++e) cov[(size_t)e * n_tracks + i] = C[e];
      chi2[i] = c2;
      ndf[i] = 2 * r.n_used - 5;
    } else {
      for (int c = 0; c < 5; ++c) params[(size_t)c * n_tracks + i] = nan;
      for (int e = 0; e < 15; ++e) cov[(size_t)e * n_tracks + i] = nan;
      chi2[i] = nan;
      ndf[i] = -1;
    }
  }
  return 0;
}

}  // namespace

extern "C" {

// Fit n_tracks tracks (FP64).  Arrays are host memory, SoA:
//   off[n+1] CSR offsets into the hit arrays y, z, rowsec (rowsec = row<<6 | sector);
//   seeds[5][n]; align[36][152][2] (or null); ref[H][5] reference states for the
//   linearised filter (or null); outputs params[5][n], cov[15][n], chi2[n], ndf[n];
//   trace[H][2][22] per-hit filtered (p, C, chi2, x) of both passes (or null).
int oracle_fit_f64(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const double* y,
                   const double* z, const uint16_t* rowsec, const double* seeds, const double* align,
                   const double* ref, double* params, double* cov, double* chi2, int32_t* ndf, double* trace,
                   int32_t nthreads) {
  return fit_all<double, false>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, ref, params, cov, chi2, ndf,
                                trace, nthreads);
}

// The FP64 fit with the predicted state (p, C) of every hit of both passes,
// before its update: ptrace[H][2][20] (NaN where a pass does not reach a hit).
// They are the inputs of the two-filter smoother (Fraser & Potter, 1969).
int oracle_fit_pred_f64(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const double* y,
                        const double* z, const uint16_t* rowsec, const double* seeds, const double* align,
                        const double* ref, double* params, double* cov, double* chi2, int32_t* ndf, double* ptrace,
                        int32_t nthreads) {
  return fit_all<double, false>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, ref, params, cov, chi2, ndf,
                                nullptr, nthreads, ptrace);
}

// The square-root (Potter) form in FP64: the pin that ties the FP32 canonical
// sequence's algebra to the covariance form.
int oracle_fit_sqrt_f64(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const double* y,
                        const double* z, const uint16_t* rowsec, const double* seeds, const double* align,
                        const double* ref, double* params, double* cov, double* chi2, int32_t* ndf, double* trace,
                        int32_t nthreads) {
  return fit_all<double, true>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, ref, params, cov, chi2, ndf,
                               trace, nthreads);
}

// The covariance form in strict FP32: shows why the FP32 sequence is the
// square-root form (diffuse C0 = 100 I loses up to 7 digits in C - K C_H).
int oracle_fit_cov_f32(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const float* y,
                       const float* z, const uint16_t* rowsec, const float* seeds, const float* align,
                       const double* ref, float* params, float* cov, float* chi2, int32_t* ndf, double* trace,
                       int32_t nthreads) {
  return fit_all<float, false>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, ref, params, cov, chi2, ndf,
                               trace, nthreads);
}

// Same, strict FP32 (the bit-exact reference of the deterministic GPU mode).
int oracle_fit_f32(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const float* y,
                   const float* z, const uint16_t* rowsec, const float* seeds, const float* align,
                   const double* ref, float* params, float* cov, float* chi2, int32_t* ndf, double* trace,
                   int32_t nthreads) {
  return fit_all<float, true>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, ref, params, cov, chi2, ndf,
                              trace, nthreads);
}

}  // extern "C"

namespace {
// Forward-mode gradient of L = sum_i w_i chi2_i for one dual type: D = Dual
// (FP64 values, covariance form) or DualF (strict-FP32 values, square-root form
// and residual coordinates: the float fit's own operation sequence).
template <class D, bool kSqrt, class VIn>
int grad_all(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const VIn* y, const VIn* z,
             const uint16_t* rowsec, const VIn* seeds, const VIn* align, const double* w, double* grad_meas,
             double* grad_seed, double* chi2, int32_t* ndf, int32_t nthreads) {
  using S = typename Traits<D>::S;
  if (check_inputs(geo, n_tracks, off)) return 1;
  for (int32_t i = 0; i < n_tracks; ++i)
    if (off[i + 1] - off[i] > 152) return 1;
  Geo<S> g;
  make_geo<S>(g, geo->row_x, geo->n_rows, geo->sector_width_deg, bz, geo->x0_cm, geo->dedx_gev_cm, geo->mass_gev,
              geo->row_cm, geo->field_cr, geo->field_cz);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
  for (int32_t i = 0; i < n_tracks; ++i) {
    const int n = off[i + 1] - off[i];
    g_nd = 2 * n + 5;
    std::vector<D> yv(n), zv(n);
    for (int j = 0; j < n; ++j) {
      yv[j] = D(y[off[i] + j]);
      yv[j].d[2 * j] = 1.0;
      zv[j] = D(z[off[i] + j]);
      zv[j].d[2 * j + 1] = 1.0;
    }
    D seed[5];
    for (int c = 0; c < 5; ++c) {
      seed[c] = D(seeds[(size_t)c * n_tracks + i]);
      seed[c].d[2 * n + c] = 1.0;
    }
    // alignment enters as a constant shift (the same subtraction as the fit's
    // measurement); the hit views index from 0
    HitView<D> h{yv.data(), zv.data(), rowsec + off[i], nullptr, 0, n};
    if (align) {
      for (int j = 0; j < n; ++j) {
        const int64_t key = ((int64_t)(rowsec[off[i] + j] & 63) * 152 + (rowsec[off[i] + j] >> 6)) * 2;
        yv[j] = yv[j] - D(align[key]);
        zv[j] = zv[j] - D(align[key + 1]);
      }
    }
    D p[5], C[15], c2((S)0.0);
    FitResult r = fit_track<D, kSqrt>(g, h, yv.data(), zv.data(), seed, nullptr, p, C, c2, nullptr);
    const double wi = w ? w[i] : 1.0;
    for (int j = 0; j < n; ++j) {
      grad_meas[(size_t)(off[i] + j) * 2] = r.ok ? wi * c2.d[2 * j] : 0.0;
      grad_meas[(size_t)(off[i] + j) * 2 + 1] = r.ok ? wi * c2.d[2 * j + 1] : 0.0;
    }
    for (int c = 0; c < 5; ++c) grad_seed[(size_t)c * n_tracks + i] = r.ok ? wi * c2.d[2 * n + c] : 0.0;
    chi2[i] = r.ok ? (double)c2.v : NAN;
    ndf[i] = r.ok ? 2 * r.n_used - 5 : -1;
  }
  return 0;
}
}  // namespace

extern "C" {

// Forward-mode FP64 gradient of L = sum_i w_i chi2_i.
//   grad_meas[H][2] = dL/dm (m = measured y, z after alignment subtraction),
//   grad_seed[5][n] = dL/dseed; chi2[n] and ndf[n] as in the fit.
// Tracks that fail get zero gradients.
int oracle_grad_f64(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const double* y,
                    const double* z, const uint16_t* rowsec, const double* seeds, const double* align,
                    const double* w, double* grad_meas, double* grad_seed, double* chi2, int32_t* ndf,
                    int32_t nthreads) {
  return grad_all<Dual, false, double>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, w, grad_meas, grad_seed,
                                       chi2, ndf, nthreads);
}

// The gradient of the strict-FP32 fit itself: the same L with every value
// computed by the float instantiation's operation sequence (chi2 and ndf are
// bit for bit those of oracle_fit_f32) and its exact derivative carried in
// FP64.  Inputs are float, as for oracle_fit_f32; outputs as for
// oracle_grad_f64.  A reverse-mode FP32 adjoint of that sequence differs from it
// only by the rounding of its own derivative arithmetic.
int oracle_grad_f32(const OracleGeometry* geo, double bz, int32_t n_tracks, const int32_t* off, const float* y,
                    const float* z, const uint16_t* rowsec, const float* seeds, const float* align, const double* w,
                    double* grad_meas, double* grad_seed, double* chi2, int32_t* ndf, int32_t nthreads) {
  return grad_all<DualF, true, float>(geo, bz, n_tracks, off, y, z, rowsec, seeds, align, w, grad_meas, grad_seed,
                                      chi2, ndf, nthreads);
}

// One prediction step in FP64 (for Jacobian tests): state p_in at local x_in in
// sector sec_in, moved to pad row row_out of sector sec_out.  J_out is the 5x5
// Jacobian d p_out / d p_in, row-major.  Returns 0 on success, 1 if the step fails.
int oracle_step_f64(const OracleGeometry* geo, double bz, const double* p_in, double x_in, int32_t sec_in,
                    int32_t row_out, int32_t sec_out, double* p_out, double* x_out, double* J_out) {
  if (!geo || row_out < 0 || row_out >= geo->n_rows) return 2;
  Geo<double> g;
  make_geo<double>(g, geo->row_x, geo->n_rows, geo->sector_width_deg, bz);
  Jac<double> J;
  double xo;
  if (!predict<double>(g, p_in, x_in, sec_in, sec_out, g.row_x[row_out], p_out, xo, J)) return 1;
  *x_out = xo;
  const double M[25] = {J.yy, 0.0, J.ys, 0.0, J.yq,  J.zy, 1.0, J.zs, J.zt, J.zq,  J.sy, 0.0, J.ss, 0.0, J.sq,
                        0.0,  0.0, 0.0,  1.0, 0.0,   0.0,  0.0, 0.0,  0.0,  1.0};
  std::memcpy(J_out, M, sizeof(M));
  return 0;
}

// One Kalman update in FP64 on packed C (for tests).  Returns 0 on success.
int oracle_update_f64(double* p, double* C, double* chi2, const double* m) {
  Geo<double> g;
  const double rx = 85.0;
  make_geo<double>(g, &rx, 1, 20.0, 0.5);
  Filter<double, false> F;
  for (int e = 0; e < 15; ++e) F.C[e] = C[e];
  const bool ok = F.update(g, p, *chi2, m);
  for (int e = 0; e < 15; ++e) C[e] = F.C[e];
  return ok ? 0 : 1;
}

// Transport C <- J C J^T for a given Jacobian (tests).  J is 5x5 row-major with
// the fit's sparsity (t and q rows identity).
int oracle_transport_f64(double* C, const double* Jm) {
  Jac<double> J;
  J.yy = Jm[0]; J.ys = Jm[2]; J.yq = Jm[4];
  J.zy = Jm[5]; J.zs = Jm[7]; J.zt = Jm[8]; J.zq = Jm[9];
  J.sy = Jm[10]; J.ss = Jm[12]; J.sq = Jm[14];
  J.rot = !(Jm[0] == 1.0 && Jm[5] == 0.0 && Jm[10] == 0.0 && Jm[12] == 1.0);
  transport<double>(C, J);
  return 0;
}

double oracle_asin_f64(double u) { return asin_f64(u); }
float oracle_asinc_f32(float u) { return asinc_(u); }
// The strict-FP32 asinc with the derivative its dual carries (tests).
float oracle_asinc_dual_f32(float u, double* deriv) {
  g_nd = 1;
  DualF x(u);
  x.d[0] = 1.0;
  const DualF r = asinc_(x);
  *deriv = r.d[0];
  return r.v;
}

long long oracle_guard_count(void) { return g_guard_hits.load(); }
void oracle_guard_reset(void) { g_guard_hits.store(0); }

}  // extern "C"
