"""The roofline's algorithmic operation counts (flops.py) against a count of
the formula lists (CPU).

Each piece of a fit step is written out once more below, in the order of its
formula list, on a scalar type that counts its operations (add, subtract,
multiply, divide, square root: one each; a fused multiply-add is a multiply
and an add).  The counts must equal the constants the benchmark divides by.
Only the algorithm's operations count: the residual-coordinate shift that the
FP32 code adds for accuracy, branch tests and copies do not."""
import pytest

from paper_2511_17018_gb300 import flops


class N:
    """A number that counts the arithmetic done on it."""
    ops = 0

    def __init__(self, v=0.5):
        self.v = float(v)

    @staticmethod
    def _v(x):
        return x.v if isinstance(x, N) else float(x)

    def _op(self, v):
        N.ops += 1
        return N(v)

    def __add__(self, o): return self._op(self.v + N._v(o))
    __radd__ = __add__
    def __sub__(self, o): return self._op(self.v - N._v(o))
    def __rsub__(self, o): return self._op(N._v(o) - self.v)
    def __mul__(self, o): return self._op(self.v * N._v(o))
    __rmul__ = __mul__
    def __truediv__(self, o): return self._op(self.v / N._v(o))
    def __rtruediv__(self, o): return self._op(N._v(o) / self.v)


def sqrt(x):
    N.ops += 1
    return N(abs(x.v) ** 0.5)


def count(fn):
    N.ops = 0
    fn()
    return N.ops


def prediction():
    """Rotation-free helix step with its Jacobian, d(path)/dk from the series."""
    X, x1, y1, z1, s1, t, q, kappa = (N(v) for v in (90.0, 89.0, 1.0, 2.0, 0.1, 0.3, 0.5, -0.0015))
    dx = X - x1
    k = q * kappa
    kdx = k * dx
    s2 = s1 + kdx
    c1 = sqrt((1.0 - s1) * (1.0 + s1)); ic1 = 1.0 / c1
    c2 = sqrt((1.0 - s2) * (1.0 + s2)); ic2 = 1.0 / c2
    den = c1 + c2
    Tm = (s1 + s2) / den
    w = c1 + s1 * Tm
    sig = kdx * w
    u2 = sig * sig                                   # asin(u)/u, degree-12 polynomial in u
    acc = N(231.0 / 13312.0)
    for c in (63.0 / 2816.0, 35.0 / 1152.0, 5.0 / 112.0, 3.0 / 40.0, 1.0 / 6.0, 1.0):
        acc = acc * u2 + c
    dl = (dx * w) * acc
    y2 = y1 + dx * Tm
    z2 = z1 + t * dl
    tt = 1.0 + Tm * Tm
    j_ys = (dx * tt) * ((ic1 + ic2) * 0.5)
    j_yq = ((dx * kappa) * dx) * (tt * (ic2 * 0.5))
    j_zs = (t * dx) * (Tm * (ic1 * ic2))
    i2 = ic1 * ic1; i3 = i2 * ic1; i5 = i3 * i2; i7 = i5 * i2
    s1s = s1 * s1
    a1 = (s1 * i3) * 0.5
    a2 = ((1.0 + 2.0 * s1s) * i5) * (1.0 / 3.0)
    a3 = ((s1 * (3.0 + 2.0 * s1s)) * i7) * 0.125
    lk = (dx * dx) * (a1 + kdx * (a2 + kdx * a3))
    j_zq = (t * kappa) * lk
    j_sq = dx * kappa
    return y2, z2, s2, j_ys, j_yq, j_zs, j_zq, j_sq


def transport():
    """L <- J L for the five columns of the square-root factor (rows t, q identity)."""
    L = [[N(0.1 * (i + c + 1)) for c in range(5)] for i in range(5)]
    ys, yq, zs, zt, zq, sq = (N(0.2) for _ in range(6))
    for c in range(5):
        ny = (L[0][c] + ys * L[2][c]) + yq * L[4][c]
        nz = ((L[1][c] + zs * L[2][c]) + zt * L[3][c]) + zq * L[4][c]
        ns = L[2][c] + sq * L[4][c]
        L[0][c], L[1][c], L[2][c] = ny, nz, ns


def scalar_update(H=0):
    """Potter update with one measured coordinate H (variance v)."""
    L = [[N(0.1 * (i + 2 * c + 1)) for c in range(5)] for i in range(5)]
    p = [N(0.3) for _ in range(5)]
    v, mv, chi2 = N(0.01), N(0.05), N(0.0)
    a = [L[H][c] for c in range(5)]
    s2 = v + a[0] * a[0]
    for c in range(1, 5):
        s2 = s2 + a[c] * a[c]
    alpha = 1.0 / s2
    beta = sqrt(alpha * v)
    gamma = 1.0 / (1.0 + beta)
    r = mv - p[H]
    K = []
    for i in range(5):
        la = L[i][0] * a[0]
        for c in range(1, 5):
            la = la + L[i][c] * a[c]
        K.append(la * alpha)
    for i in range(5):
        p[i] = p[i] + K[i] * r
    chi2 = chi2 + (r * r) * alpha
    for i in range(5):
        if i == H:
            continue
        gk = gamma * K[i]
        for c in range(5):
            L[i][c] = L[i][c] - gk * a[c]
    for c in range(5):
        L[H][c] = a[c] * beta


def alignment():
    y, z, dy, dz = N(), N(), N(), N()
    return y - dy, z - dz


def covariance_output():
    """C = L L^T, lower triangle (15 entries, 5-term dot products)."""
    L = [[N(0.1) for _ in range(5)] for _ in range(5)]
    for i in range(5):
        for j in range(i + 1):
            acc = L[i][0] * L[j][0]
            for c in range(1, 5):
                acc = acc + L[i][c] * L[j][c]


@pytest.mark.parametrize("fn,const", [(prediction, flops.PREDICT), (transport, flops.TRANSPORT),
                                      (scalar_update, flops.SCALAR_UPDATE), (alignment, flops.MEAS),
                                      (covariance_output, flops.OUTPUT)],
                         ids=["prediction", "transport", "scalar_update", "alignment", "covariance_output"])
def test_piece_counts(fn, const):
    assert count(fn) == const


def test_step_totals():
    assert flops.STEP == flops.PREDICT + flops.TRANSPORT + 2 * flops.SCALAR_UPDATE + flops.MEAS == 397
    assert flops.FIRST == 2 * flops.SCALAR_UPDATE + flops.MEAS
    # a track of n clusters: both passes of n - 1 full steps and one first step, and the output
    assert flops.fit_flops([10, 1, 0]) == 2 * (9 * 397 + 258) + 135 + 2 * 258 + 135
