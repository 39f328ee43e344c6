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
    def __neg__(self): return N(-self.v)   # a sign flip folds into the operation that uses it


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


def _ud(seed=0.1):
    u = [[N(seed * (i + 2 * j + 1)) if j > i else None for j in range(5)] for i in range(5)]
    d = [N(1.0 + 0.1 * j) for j in range(5)]
    return u, d


def transport_ud():
    """U <- J U without rotation (J unit upper triangular): the seven entries that change."""
    u, _ = _ud()
    ys, yq, zs, zt, zq, sq = (N(0.2) for _ in range(6))
    u[0][4] = (u[0][4] + ys * u[2][4]) + yq
    u[0][3] = u[0][3] + ys * u[2][3]
    u[0][2] = u[0][2] + ys
    u[1][4] = ((u[1][4] + zs * u[2][4]) + zt * u[3][4]) + zq
    u[1][3] = (u[1][3] + zs * u[2][3]) + zt
    u[1][2] = u[1][2] + zs
    u[2][4] = u[2][4] + sq


def bierman_update(H):
    """Bierman's scalar update of component H in residual coordinates (measured value 0)."""
    u, d = _ud()
    p = [N(0.3) for _ in range(5)]
    v, chi2 = N(0.01), N(0.0)
    K = [None] * 5
    ap, iap = v, None
    for j in range(H, 5):
        f = None if j == H else u[H][j]
        g = d[j] if j == H else d[j] * f
        a = ap + g if j == H else ap + f * g
        ia = 1.0 / a
        if j > H:
            lam = -(f * iap)
            for i in range(j):
                uo = u[i][j]
                u[i][j] = uo + lam * K[i]
                K[i] = K[i] + g * uo
        else:
            for i in range(j):
                K[i] = g * u[i][j]
        d[j] = d[j] * (ap * ia)
        K[j] = g
        ap, iap = a, ia
    r = -p[H]
    q = r * iap
    for i in range(5):
        p[i] = p[i] + K[i] * q
    chi2 = chi2 + r * q


def covariance_output_ud():
    """C = U D U^T, lower triangle: C_ij = sum over k >= i of u_ik d_k u_jk (u_kk = 1)."""
    u, d = _ud()
    for i in range(5):
        for j in range(i + 1):
            acc = d[i] if j == i else u[j][i] * d[i]
            for k in range(i + 1, 5):
                acc = acc + (u[i][k] * d[k]) * u[j][k]


def transport_ud_rev():
    """Reverse of transport_ud: the Jacobian's adjoint (started at zero) and the factor's."""
    u, _ = _ud()
    b = {k: N(0.3) for k in ("02", "03", "04", "12", "13", "14", "24")}
    ys, zs, zt = N(0.2), N(0.2), N(0.2)
    bJ_ys = (b["02"] + u[2][3] * b["03"]) + u[2][4] * b["04"]
    bJ_zs = (b["12"] + u[2][3] * b["13"]) + u[2][4] * b["14"]
    bJ_zt = b["13"] + u[3][4] * b["14"]
    bu23, bu24, bu34 = N(0.1), N(0.1), N(0.1)
    bu23 = bu23 + (ys * b["03"] + zs * b["13"])
    bu24 = bu24 + (ys * b["04"] + zs * b["14"])
    bu34 = bu34 + zt * b["14"]


def bierman_update_rev(H):
    """Reverse of bierman_update<H> with the partial gain sums recomputed in the
    forward's order; operations whose results are unused where j = H are left out."""
    u, d = _ud()
    bu = [[N(0.2) if j > i else None for j in range(5)] for i in range(5)]
    bd = [N(0.2) for _ in range(5)]
    bp = [N(0.2) for _ in range(5)]
    p = [N(0.3) for _ in range(5)]
    v, bchi = N(0.01), N(1.0)
    gv = [None if j < H else (d[j] if j == H else d[j] * u[H][j]) for j in range(5)]
    al, ial = [None] * 5, [None] * 5
    ap = v
    for j in range(H, 5):
        al[j] = ap + gv[j] if j == H else ap + u[H][j] * gv[j]
        ial[j] = 1.0 / al[j]
        ap = al[j]

    def k_before(i, j):
        acc = gv[i]
        for k in range(max(i + 1, H), j):
            acc = u[i][k] * gv[k] if acc is None else acc + u[i][k] * gv[k]
        return acc

    K = [k_before(i, 5) for i in range(5)]
    r = -p[H]
    q = r * ial[4]
    bK = [q * bp[i] for i in range(5)]
    bqo = r * bchi
    for i in range(5):
        if i != H:
            bqo = bqo + K[i] * bp[i]
    bq = bqo + K[H] * bp[H]
    ba = -(ial[4] * ial[4]) * (r * bq)
    bp[H] = (v * ial[4]) * bp[H] - (q * bchi + ial[4] * bqo)
    for j in range(4, H - 1, -1):
        g = gv[j]
        bg = bK[j]
        if j > H:
            f = u[H][j]
            iapj = ial[j - 1]
            lam = -(f * iapj)
            blam = None
            for i in range(j - 1, -1, -1):
                uo = u[i][j]
                kb = k_before(i, j)
                bv = bu[i][j]
                bg = bg + uo * bK[i] if bK[i] is not None else bg
                blam = kb * bv if blam is None else blam + kb * bv
                if kb is None:
                    pass
                bu[i][j] = bv + g * bK[i] if bK[i] is not None else bv
                bK[i] = lam * bv if bK[i] is None else bK[i] + lam * bv
            bf = -(blam * iapj)
            bap = -(lam * blam) * iapj
            rho = al[j - 1] * ial[j]
            bdn = bd[j]
            bap = bap + (d[j] * bdn) * ial[j]
            ba = ba - ((d[j] * rho) * bdn) * ial[j]
            bdj = bdn * rho
            bap = bap + ba
            bf = bf + g * ba
            bg = bg + f * ba
            bdj = bdj + f * bg
            bf = bf + d[j] * bg
            bd[j] = bdj
            bu[H][j] = bu[H][j] + bf
            ba = bap
        else:
            for i in range(j - 1, -1, -1):
                uo = u[i][j]
                bg = bg + uo * bK[i]
                bu[i][j] = bu[i][j] + g * bK[i]
            rho = v * ial[j]
            bdn = bd[j]
            ba = ba - ((d[j] * rho) * bdn) * ial[j]
            bdj = bdn * rho
            bg = bg + ba
            bd[j] = bdj + bg


@pytest.mark.parametrize("fn,const", [(transport_ud, flops.UD_TRANSPORT),
                                      (lambda: bierman_update(0), flops.UD_UPDATE[0]),
                                      (lambda: bierman_update(1), flops.UD_UPDATE[1]),
                                      (covariance_output_ud, flops.UD_OUTPUT),
                                      (transport_ud_rev, flops.UD_REV_TRANSPORT),
                                      (lambda: bierman_update_rev(0), flops.UD_REV_UPDATE[0]),
                                      (lambda: bierman_update_rev(1), flops.UD_REV_UPDATE[1])],
                         ids=["transport_ud", "bierman_y", "bierman_z", "covariance_output_ud",
                              "transport_ud_rev", "bierman_rev_y", "bierman_rev_z"])
def test_u_d_piece_counts(fn, const):
    assert count(fn) == const


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
    assert flops.UD_STEP == flops.PREDICT + flops.UD_TRANSPORT + sum(flops.UD_UPDATE) + flops.MEAS
    assert flops.fit_flops([10], form=1) == 2 * (9 * flops.UD_STEP + flops.UD_FIRST) + flops.UD_OUTPUT
