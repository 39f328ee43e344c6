"""Planted mistakes in the oracle are caught by its pins.

Each case copies the oracle source, plants one plausible mistake (a wrong sign,
a dropped term or factor, a transposed operand), builds it on the CPU and
checks that the pin aimed at that part of the fit fails on the mutant while it
passes on the unmodified oracle."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import build as obuild

SRC = obuild.SRC

MUTANTS = {
    "propagation_sign": ("  pout[0] = y1 + dx * Tm;", "  pout[0] = y1 - dx * Tm;"),
    "jacobian_dropped_factor": ("  J.yq = ((dx * kappa) * dx) * (tt * (ic2 * half));",
                                "  J.yq = ((dx * kappa) * dx) * (tt * half);"),
    "transport_dropped_term": ("      A[1][j] = ((M[1][j] + J.zs * M[2][j]) + J.zt * M[3][j]) + J.zq * M[4][j];",
                               "      A[1][j] = (M[1][j] + J.zs * M[2][j]) + J.zq * M[4][j];"),
    "gain_transposed_operand": ("      K[i][1] = ci0 * Si10 + ci1 * Si11;", "      K[i][1] = ci1 * Si10 + ci0 * Si11;"),
    "rotation_sign": ("    const T sr = s * ca - c * sa;", "    const T sr = s * ca + c * sa;"),
    "potter_wrong_factor": ("    for (int c = 0; c < 5; ++c) L[h][c] = a[c] * beta;",
                            "    for (int c = 0; c < 5; ++c) L[h][c] = a[c] * gamma;"),
    "dual_quotient_rule_sign": ("  for (int i = 0; i < g_nd; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;",
                                "  for (int i = 0; i < g_nd; ++i) r.d[i] = (a.d[i] + r.v * b.d[i]) * ib;"),
    "energy_loss_direction": ("  const T en = dir > 0 ? e - de : e + de;", "  const T en = dir > 0 ? e + de : e - de;"),
    "highland_momentum_power": ("  const T th2 = (((S)(0.0136 * 0.0136) * ell) * g.x0_inv) * (e2 / (p2 * p2));",
                                "  const T th2 = (((S)(0.0136 * 0.0136) * ell) * g.x0_inv) * (e2 / p2);"),
    "field_map_dropped_z_term": ("    kappa = kappa * ((one + g.f_r * (xm * xm + ym * ym)) + g.f_z * (zm * zm));",
                                 "    kappa = kappa * (one + g.f_r * (xm * xm + ym * ym));"),
    "fp32_dual_asinc_derivative": ("    for (int k = 5; k >= 1; --k) acc = acc * q + (double)k * c[k];",
                                   "    for (int k = 5; k >= 1; --k) acc = acc * q + c[k];"),
    "side_change_as_sector_change": (
        "        const bool rot = (hit_sec(h, from) % kNSectorsPerSide) != (hit_sec(h, to) % kNSectorsPerSide);",
        "        const bool rot = hit_sec(h, from) != hit_sec(h, to);"),
    "smoother_filtered_not_predicted": ("    precord(pass, to);\n    return F.update(g, p, chi2, m);",
                                        "    const bool ok_ = F.update(g, p, chi2, m);\n    precord(pass, to);\n"
                                        "    return ok_;"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    p = tmp_path / f"{name}.cpp"
    p.write_text(src.replace(old, new))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["g++", *obuild.FLAGS, str(p), "-o", str(lib)], check=True)
    return str(lib)


class _Swap:
    """Point the oracle wrapper at another build of the library."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        self.saved_lib, self.saved_build = oracle._lib, obuild.build
        oracle._lib = None
        obuild.build = lambda force=False: self.path
        oracle.lib()
        return self

    def __exit__(self, *a):
        oracle._lib, obuild.build = self.saved_lib, self.saved_build


# ---- the checks (small versions of the pins in test_oracle_pins.py)
def check_exact_helix(synth):
    from conftest import truth_trajectory
    fr = synth.generate(60, 21, smear=0.0)
    ref = truth_trajectory(oracle, fr)
    return np.abs(ref[:, 0] - fr.y64).max() < 1e-9 and np.abs(ref[:, 1] - fr.z64).max() < 1e-9


def check_jacobian_fd(synth):
    g = synth.default_geometry()
    rng = np.random.default_rng(1)
    for _ in range(30):
        p = np.array([rng.uniform(-10, 10), rng.uniform(-50, 50), rng.uniform(-0.6, 0.6), rng.uniform(-1, 1),
                      rng.uniform(-5, 5)])
        r0 = int(rng.integers(0, 140))
        res = oracle.step(g, 0.5, p, g.row_x[r0], 3, r0 + 3, 3)
        if res is None:
            continue
        J = res[2]
        for c in range(5):
            h = 1e-6 * max(1.0, abs(p[c]))
            pp, pm = p.copy(), p.copy()
            pp[c] += h
            pm[c] -= h
            fd = (oracle.step(g, 0.5, pp, g.row_x[r0], 3, r0 + 3, 3)[0] -
                  oracle.step(g, 0.5, pm, g.row_x[r0], 3, r0 + 3, 3)[0]) / (2 * h)
            if np.any(np.abs(J[:, c] - fd) > 1e-6 * np.maximum(1, np.abs(fd))):
                return False
    return True


def check_transport_dense(synth):
    rng = np.random.default_rng(5)
    for _ in range(10):
        A = rng.normal(size=(5, 5))
        Cm = A @ A.T
        J = np.eye(5)
        J[0, 2], J[0, 4], J[1, 2], J[1, 3], J[1, 4], J[2, 4] = rng.normal(size=6)
        out = oracle.unpack(oracle.transport(oracle.pack(Cm), J))
        if not np.allclose(out, J @ Cm @ J.T, rtol=1e-12, atol=1e-12):
            return False
    return True


def check_information_form(synth):
    rng = np.random.default_rng(4)
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    Vi = np.eye(2) / 0.01
    for _ in range(10):
        A = rng.normal(size=(5, 5))
        Cm = A @ A.T + 1e-3 * np.eye(5)
        p = rng.normal(size=5)
        m = p[:2] + rng.normal(size=2) * 0.3
        pu, Cu, _ = oracle.update(p, oracle.pack(Cm), m)
        Ci = np.linalg.inv(Cm)
        Cplus = np.linalg.inv(Ci + H.T @ Vi @ H)
        if not np.allclose(oracle.unpack(Cu), Cplus, rtol=1e-9, atol=1e-12):
            return False
        if not np.allclose(pu, Cplus @ (Ci @ p + H.T @ Vi @ m), rtol=1e-9, atol=1e-11):
            return False
    return True


def check_round_trip(synth):
    g = synth.default_geometry()
    rng = np.random.default_rng(3)
    for _ in range(40):
        p = np.array([rng.uniform(-5, 5), rng.uniform(-50, 50), rng.uniform(-0.5, 0.5), rng.uniform(-1, 1),
                      rng.uniform(-3, 3)])
        r0 = int(rng.integers(20, 130))
        s0 = int(rng.integers(0, 18))
        fw = oracle.step(g, 0.5, p, g.row_x[r0], s0, r0 + 2, (s0 + 1) % 18)
        if fw is None:
            continue
        bw = oracle.step(g, 0.5, fw[0], fw[1], (s0 + 1) % 18, r0, s0)
        if bw is None or not np.allclose(bw[0], p, atol=1e-10):
            return False
    return True


def check_sqrt_vs_cov(synth):
    fr = synth.generate(200, 2, drop_p=0.05, cap_lengths=True)
    a = oracle.fit(fr, "f64")
    b = oracle.fit(fr, "sqrt_f64")
    ok = a["ndf"] > 0
    sig = np.sqrt(a["cov"][[0, 2, 5, 9, 14]])
    return bool(np.nanmax(np.abs(a["params"] - b["params"])[:, ok] / sig[:, ok]) < 1e-7)


def check_gradient_fd(synth):
    fr = synth.generate(2, 27, drop_p=0.05, cap_lengths=True)
    gr = oracle.grad(fr)
    y = fr.y.astype(np.float64)
    j = fr.n_hits // 3
    ff = fr.subset(np.arange(fr.n_tracks))
    vals = []
    for sgn in (1, -1):
        yy = y.copy(); yy[j] += sgn * 1e-4
        ff.y64, ff.z64, ff.seeds64 = yy, fr.z.astype(np.float64), fr.seeds.astype(np.float64)
        vals.append(np.nansum(oracle.fit(ff, "f64", exact_inputs=True)["chi2"]))
    fd = (vals[0] - vals[1]) / 2e-4
    return abs(gr["grad_meas"][j, 0] - fd) < 1e-6 * max(1.0, abs(fd))


def check_energy_loss_refit(synth):
    from test_oracle_pins import _material_tracks
    fr, _ = _material_tracks(synth, 12, 3, scatter=False, smear=0.0)
    seeds = fr.seeds64.copy()
    for _ in range(4):
        r = oracle.fit(fr, "f64", exact_inputs=True, seeds=seeds)
        if not np.all(r["ndf"] > 0):
            return False
        seeds = r["params"].copy()
    return bool(np.abs(r["params"][:4] - fr.truth[:4]).max() < 1e-7 and
                (np.abs(r["params"][4] - fr.truth[4]) / np.abs(fr.truth[4])).max() < 1e-7)


def check_material_pulls(synth):
    from test_oracle_pins import _material_tracks
    fr, _ = _material_tracks(synth, 400, 1)
    r = oracle.fit(fr, "f64")
    ok = r["ndf"] > 0
    C = oracle.unpack(r["cov"][:, ok])
    sig = np.sqrt(np.stack([C[i, i] for i in range(5)]))
    w = ((r["params"][:, ok] - fr.truth[:, ok]) / sig).std(axis=1)
    return bool(np.all((w > 0.88) & (w < 1.12)))


def check_field_map_refit(synth):
    from test_oracle_pins import _field_tracks
    fr, _ = _field_tracks(synth, 10, 3, smear=0.0)
    seeds = fr.seeds64.copy()
    for _ in range(4):
        r = oracle.fit(fr, "f64", exact_inputs=True, seeds=seeds)
        if not np.all(r["ndf"] > 0):
            return False
        seeds = r["params"].copy()
    return bool(np.abs(r["params"][:4] - fr.truth[:4]).max() < 1e-6 and
                (np.abs(r["params"][4] - fr.truth[4]) / np.abs(fr.truth[4])).max() < 3e-6)


def check_smoother_leave_one_out(synth):
    # the residual of each cluster of a short track against the dense weighted
    # least-squares solve without that cluster (both passes' priors)
    from conftest import truth_trajectory
    from test_oracle_pins import _affine_chain, _short_tracks
    fr, _ = _short_tracks(synth, 11, n=8)
    ref = truth_trajectory(oracle, fr)
    s = oracle.smooth(fr, ref=ref, exact_inputs=True)
    r = oracle.fit(fr, "f64", ref=ref, trace=True, exact_inputs=True)
    m = np.stack([fr.y64, fr.z64], axis=1)
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    for i in range(fr.n_tracks):
        order, A, bb = _affine_chain(oracle, fr, ref, i, backward=False)
        p_out = r["trace"][order[-1], 0, :5]
        for k, h in enumerate(order):
            N = np.eye(5) / 100.0 + A[-1].T @ A[-1] / 100.0
            rhs = fr.seeds64[:, i] / 100.0 + A[-1].T @ (p_out - bb[-1]) / 100.0
            for kk, j in enumerate(order):
                if kk != k:
                    HA = H @ A[kk]
                    N += HA.T @ HA / 0.01
                    rhs += HA.T @ (m[j] - H @ bb[kk]) / 0.01
            xc = A[k] @ np.linalg.solve(N, rhs) + bb[k]
            if not np.allclose(s["resid"][h], m[h] - xc[:2], rtol=1e-7, atol=1e-10):
                return False
    return True


def check_side_change(synth):
    # tracks crossing z = 0, fitted with their sector labels and with every
    # label moved to the A side: the strict-FP32 fits agree bit for bit
    fr = synth.generate(1500, 24, drop_p=0.05)
    sec = fr.rowsec.astype(np.int64) & 63
    off = fr.offsets.astype(np.int64)
    cross = [i for i in range(fr.n_tracks)
             if (sec[off[i]:off[i + 1]] >= 18).any() and (sec[off[i]:off[i + 1]] < 18).any()]
    sub = fr.subset(np.array(cross))
    a_side = sub.subset(np.arange(sub.n_tracks))
    r = a_side.rowsec.astype(np.int64)
    a_side.rowsec = (((r >> 6) << 6) | ((r & 63) % 18)).astype(np.uint16)
    x, y = oracle.fit(sub, "f32"), oracle.fit(a_side, "f32")
    return all(np.array_equal(x[k], y[k]) for k in ("params", "cov", "chi2", "ndf"))


def check_fp32_dual_asinc(synth):
    for u in (0.05, -0.12, 0.2, 0.24):
        _, d = oracle.asinc_dual_f32(u)
        uf = float(np.float32(u))
        exact = (uf / math.sqrt(1.0 - uf * uf) - math.asin(uf)) / (uf * uf)
        if abs(d - exact) > 1e-7 * max(1.0, abs(exact)):
            return False
    return True


CASES = [
    ("propagation_sign", check_exact_helix),
    ("jacobian_dropped_factor", check_jacobian_fd),
    ("transport_dropped_term", check_transport_dense),
    ("gain_transposed_operand", check_information_form),
    ("rotation_sign", check_round_trip),
    ("potter_wrong_factor", check_sqrt_vs_cov),
    ("dual_quotient_rule_sign", check_gradient_fd),
    ("energy_loss_direction", check_energy_loss_refit),
    ("highland_momentum_power", check_material_pulls),
    ("field_map_dropped_z_term", check_field_map_refit),
    ("smoother_filtered_not_predicted", check_smoother_leave_one_out),
    ("side_change_as_sector_change", check_side_change),
    ("fp32_dual_asinc_derivative", check_fp32_dual_asinc),
]


@pytest.mark.parametrize("name,check", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(tmp_path, synth, name, check):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    assert check(synth), "the pin must pass on the unmodified oracle"
    with _Swap(_build_mutant(tmp_path, name)):
        try:
            caught = not check(synth)
        except (TypeError, ValueError, FloatingPointError):  # the pin's own inputs break: caught too
            caught = True
    assert caught, f"planted mistake '{name}' was not caught"
