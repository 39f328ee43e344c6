"""Pins of the CPU oracle against things other than itself.

Each test ties a part of the oracle to a closed form, an identity, a library
routine, brute force or statistics, so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from conftest import truth_trajectory


# ---------------------------------------------------------------- elementary routines
def test_asin_f64_matches_libm(oracle_mod):
    # own FP64 arcsin (Maclaurin series + half-angle identity) vs the C library
    for u in np.concatenate([np.linspace(-1, 1, 4001), [0.5, -0.5, 0.4999999, 0.5000001, 1e-300]]):
        ref = math.asin(u)
        assert abs(oracle_mod.asin_f64(u) - ref) <= 4e-16 * max(1.0, abs(ref)), u


def test_asinc_f32_close_to_exact(oracle_mod):
    # the FP32 asinc (polynomial for |u|<=1/4, FP64 island above) within 2 ulp
    for u in np.concatenate([np.linspace(-0.999, 0.999, 3001), [0.25, -0.25, 0.2500001, 1e-30, 0.0]]):
        uf = float(np.float32(u))
        exact = 1.0 if uf == 0.0 else math.asin(uf) / uf
        got = oracle_mod.asinc_f32(uf)
        assert abs(got - exact) <= 2 * np.spacing(np.float32(exact)), (u, got, exact)


# ---------------------------------------------------------------- propagation step
def _random_steps(rng, geometry, n):
    for trial in range(n):
        p = np.array([rng.uniform(-10, 10), rng.uniform(-50, 50), rng.uniform(-0.7, 0.7),
                      rng.uniform(-1, 1), rng.uniform(-5, 5)])
        row0 = int(rng.integers(0, 147))
        sec0 = int(rng.integers(0, 36))
        rot = trial % 3 == 0
        side = 18 if sec0 >= 18 else 0
        sec1 = ((sec0 % 18) + (int(rng.choice([-1, 1])) if rot else 0)) % 18 + side
        row1 = int(np.clip(row0 + int(rng.integers(1, 6)) * (1 if trial % 2 else -1), 0, 151))
        x0 = geometry.row_x[row0] + rng.uniform(-0.5, 0.5)
        yield p, x0, sec0, row1, sec1


def test_step_jacobian_matches_central_differences(oracle_mod, synth):
    g = synth.default_geometry()
    rng = np.random.default_rng(1)
    n_rot = 0
    for p, x0, sec0, row1, sec1 in _random_steps(rng, g, 300):
        res = oracle_mod.step(g, 0.5, p, x0, sec0, row1, sec1)
        if res is None:
            continue
        n_rot += (sec0 % 18) != (sec1 % 18)
        _, _, J = res
        Jfd = np.zeros((5, 5))
        for c in range(5):
            h = 1e-6 * max(1.0, abs(p[c]))
            pp = p.copy(); pp[c] += h
            pm = p.copy(); pm[c] -= h
            a = oracle_mod.step(g, 0.5, pp, x0, sec0, row1, sec1)
            b = oracle_mod.step(g, 0.5, pm, x0, sec0, row1, sec1)
            Jfd[:, c] = (a[0] - b[0]) / (2 * h)
        scale = np.maximum(1.0, np.abs(Jfd))
        assert np.all(np.abs(J - Jfd) <= 1e-6 * scale), (J, Jfd)
    assert n_rot > 50


def test_step_straight_line_closed_form(oracle_mod, synth):
    # q/pt = 0: straight line, y2 = y1 + dx s/c, z2 = z1 + t dx/c, s unchanged
    g = synth.default_geometry()
    rng = np.random.default_rng(2)
    for _ in range(100):
        p = np.array([rng.uniform(-10, 10), rng.uniform(-50, 50), rng.uniform(-0.9, 0.9),
                      rng.uniform(-1, 1), 0.0])
        r0, r1 = rng.integers(0, 152, 2)
        x0 = g.row_x[r0]
        po, xo, J = oracle_mod.step(g, 0.5, p, x0, 3, int(r1), 3)
        dx = g.row_x[r1] - x0
        c = math.sqrt(1 - p[2] ** 2)
        assert xo == g.row_x[r1]
        assert abs(po[0] - (p[0] + dx * p[2] / c)) < 1e-12
        assert abs(po[1] - (p[1] + p[3] * dx / c)) < 1e-12
        assert po[2] == p[2] and po[3] == p[3] and po[4] == 0.0
        # straight-line Jacobian: dy/ds = dx / c^3, dz/dt = dx / c, dz/ds = t dx s / c^3
        assert abs(J[0, 2] - dx / c ** 3) < 1e-10 * max(1, abs(dx / c ** 3))
        assert abs(J[1, 3] - dx / c) < 1e-12
        assert abs(J[1, 2] - p[3] * dx * p[2] / c ** 3) < 1e-10 * max(1, abs(dx / c ** 3))


def test_step_round_trip_and_inverse_jacobian(oracle_mod, synth):
    # rotate-and-propagate to another sector's row and back: identity map
    g = synth.default_geometry()
    rng = np.random.default_rng(3)
    done = 0
    for _ in range(200):
        p = np.array([rng.uniform(-5, 5), rng.uniform(-50, 50), rng.uniform(-0.5, 0.5),
                      rng.uniform(-1, 1), rng.uniform(-3, 3)])
        r0 = int(rng.integers(20, 130)); r1 = r0 + int(rng.integers(-8, 9))
        s0 = int(rng.integers(0, 18)); s1 = (s0 + int(rng.choice([-1, 0, 1]))) % 18
        fw = oracle_mod.step(g, 0.5, p, g.row_x[r0], s0, r1, s1)
        if fw is None:
            continue
        bw = oracle_mod.step(g, 0.5, fw[0], fw[1], s1, r0, s0)
        if bw is None:
            continue
        assert np.allclose(bw[0], p, rtol=0, atol=1e-10), (p, bw[0])
        assert np.allclose(bw[2] @ fw[2], np.eye(5), atol=1e-8)
        done += 1
    assert done > 100


def test_propagation_reproduces_exact_helix(oracle_mod, synth):
    # carry the true first-hit state through all rows (sector changes included)
    # and land on the noise-free hits made by the generator's circle-plane solve
    fr = synth.generate(300, 21, smear=0.0)
    ref = truth_trajectory(oracle_mod, fr)
    assert np.abs(ref[:, 0] - fr.y64).max() < 1e-9
    assert np.abs(ref[:, 1] - fr.z64).max() < 1e-9
    sec = (fr.rowsec & 63).astype(int) % 18
    assert np.count_nonzero(np.diff(sec)) > 50  # crossings were exercised


# ---------------------------------------------------------------- Kalman update
def test_update_equals_information_form(oracle_mod):
    # gain form vs information form: C+^-1 = C^-1 + H^T V^-1 H,
    # p+ = C+ (C^-1 p + H^T V^-1 m); dchi2 = min over p of the two-term objective
    rng = np.random.default_rng(4)
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    Vi = np.eye(2) / 0.01
    for _ in range(50):
        A = rng.normal(size=(5, 5)) * rng.uniform(0.01, 3, 5)
        Cm = A @ A.T + 1e-3 * np.eye(5)
        p = rng.normal(size=5)
        m = p[:2] + rng.normal(size=2) * 0.3
        res = oracle_mod.update(p, oracle_mod.pack(Cm), m)
        assert res is not None
        pu, Cu, dchi2 = res
        Ci = np.linalg.inv(Cm)
        Cplus = np.linalg.inv(Ci + H.T @ Vi @ H)
        pplus = Cplus @ (Ci @ p + H.T @ Vi @ m)
        obj = (pplus - p) @ Ci @ (pplus - p) + (m - H @ pplus) @ Vi @ (m - H @ pplus)
        assert np.allclose(oracle_mod.unpack(Cu), Cplus, rtol=1e-9, atol=1e-12)
        assert np.allclose(pu, pplus, rtol=1e-9, atol=1e-11)
        assert abs(dchi2 - obj) < 1e-9 * max(1, obj)


def test_transport_equals_dense_product(oracle_mod):
    # packed sparse J C J^T vs the dense matrix product (with and without the
    # rotation columns)
    rng = np.random.default_rng(5)
    for trial in range(50):
        A = rng.normal(size=(5, 5))
        Cm = A @ A.T
        J = np.eye(5)
        J[0, 2], J[0, 4], J[1, 2], J[1, 3], J[1, 4], J[2, 4] = rng.normal(size=6)
        if trial % 2:
            J[0, 0], J[1, 0], J[2, 0], J[2, 2] = rng.normal(size=4)
        out = oracle_mod.unpack(oracle_mod.transport(oracle_mod.pack(Cm), J))
        assert np.allclose(out, J @ Cm @ J.T, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- whole fit: closed forms
def test_noise_free_helix_returns_generating_parameters(oracle_mod, synth):
    # exact FP64 clusters, seeds perturbed (q/pt by 5%, sin phi by 0.01), refit
    # with the previous output as seed until converged: truth to 1e-10
    fr = synth.generate(400, 22, smear=0.0)
    seeds = fr.seeds64.copy()
    seeds[4] *= 1.05
    seeds[2] += 0.01
    for _ in range(3):
        r = oracle_mod.fit(fr, "f64", exact_inputs=True, seeds=seeds)
        assert np.all(r["ndf"] > 0)
        seeds = r["params"].copy()
    err = np.abs(r["params"] - fr.truth) / np.maximum(1.0, np.abs(fr.truth))
    assert err.max() < 1e-10, err.max(axis=1)
    assert r["chi2"].max() < 1e-16


def test_three_point_seed_is_exact_on_noise_free_clusters(synth):
    # The test inputs' seeds: a circle through the first, middle and last
    # cluster (Menger curvature), the direction at the first cluster from the
    # chord and the half angle, tan(lambda) from the arc.  On an exact helix
    # (noise-free FP64 clusters, sector crossings included) the construction
    # is exact, so it returns the generating state at the first cluster.
    fr = synth.generate(500, 23, smear=0.0)
    s = synth.three_point_seeds(fr, as_f64=True)
    rs = fr.rowsec.astype(np.int64)
    assert np.any((rs[fr.offsets[:-1]] & 63) != (rs[fr.offsets[1:] - 1] & 63))  # some tracks change sector
    err = np.abs(s - fr.truth) / np.maximum(np.abs(fr.truth), 1e-3)
    assert err.max() < 1e-9, err.max(axis=1)


def test_crossing_z_zero_changes_only_the_sector_label(oracle_mod, synth):
    # Sectors s and s + 18 share their azimuth: a track that crosses z = 0
    # changes the side of its sector label but not its frame, so no rotation
    # applies.  Without alignment offsets, labelling every cluster with its
    # A-side sector leaves the fit unchanged, bit for bit, in both precisions;
    # with offsets the label decides which offsets apply.
    fr = synth.generate(3000, 24, drop_p=0.05)
    rs = fr.rowsec.astype(np.int64)
    sec = rs & 63
    off = fr.offsets.astype(np.int64)
    cross = np.array([(sec[off[i]:off[i + 1]] >= 18).any() and (sec[off[i]:off[i + 1]] < 18).any()
                      for i in range(fr.n_tracks)])
    assert cross.sum() >= 20
    sub = fr.subset(np.flatnonzero(cross))
    a_side = sub.subset(np.arange(sub.n_tracks))
    r = a_side.rowsec.astype(np.int64)
    a_side.rowsec = (((r >> 6) << 6) | ((r & 63) % 18)).astype(np.uint16)
    for prec in ("f64", "f32"):
        x, y = oracle_mod.fit(sub, prec), oracle_mod.fit(a_side, prec)
        assert np.all(x["ndf"] > 0)
        for k in ("params", "cov", "chi2", "ndf"):
            assert np.array_equal(x[k], y[k]), (prec, k)
    d = synth.alignment_offsets(7)
    x = oracle_mod.fit(sub, "f64", align=d)
    y = oracle_mod.fit(a_side, "f64", align=d)
    assert not np.array_equal(x["chi2"], y["chi2"])


def test_noise_free_straight_tracks_give_zero_curvature(oracle_mod, synth):
    n = 200
    rng = np.random.default_rng(6)
    qpt = np.zeros(n)
    tanl = rng.uniform(-0.8, 0.8, n)
    phi0 = rng.uniform(0, 2 * math.pi, n)
    z0 = rng.normal(0, 5, n)
    fr, ok = synth.simulate(qpt, tanl, phi0, z0, synth.default_geometry(), 0.5, smear=0.0)
    seeds = fr.seeds64.copy()
    seeds[4] = 0.05
    for _ in range(3):
        r = oracle_mod.fit(fr, "f64", exact_inputs=True, seeds=seeds)
        seeds = r["params"].copy()
    assert np.abs(r["params"][4]).max() < 1e-10
    assert np.abs(r["params"] - fr.truth).max() < 1e-9


def _affine_chain(oracle_mod, fr, ref, i, backward):
    """x_j = A_j x_start + b_j for the linearised transitions of track i."""
    g = fr.geometry
    off = fr.offsets.astype(np.int64)
    rs = fr.rowsec.astype(np.int64)
    a, b = off[i], off[i + 1]
    order = list(range(a, b))[::-1] if backward else list(range(a, b))
    A = [np.eye(5)]
    bb = [np.zeros(5)]
    for k in range(1, len(order)):
        jf, jt = order[k - 1], order[k]
        f, _, J = oracle_mod.step(g, fr.bz, ref[jf], g.row_x[rs[jf] >> 6], rs[jf] & 63, rs[jt] >> 6, rs[jt] & 63)
        A.append(J @ A[-1])
        bb.append(f + J @ (bb[-1] - ref[jf]))
    return order, A, bb


def _gls(order, A, bb, m, prior, C0):
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    N = np.eye(5) / C0
    rhs = prior / C0
    for k, j in enumerate(order):
        HA = H @ A[k]
        N += HA.T @ HA / 0.01
        rhs += HA.T @ (m[j] - H @ bb[k]) / 0.01
    x0 = np.linalg.solve(N, rhs)
    obj = (x0 - prior) @ (x0 - prior) / C0
    for k, j in enumerate(order):
        res = m[j] - H @ (A[k] @ x0 + bb[k])
        obj += res @ res / 0.01
    return x0, obj, np.linalg.inv(N)


def _short_tracks(synth, seed, n=60):
    """A frame of n tracks cut to their first 3..8 hits."""
    rng = np.random.default_rng(seed)
    base = synth.generate(n, 23, drop_p=0.05)
    keep = [np.arange(o, o + int(rng.integers(3, 9))) for o in base.offsets[:-1]]
    fr = base.subset(np.arange(base.n_tracks))
    lens = np.array([len(k) for k in keep])
    idx = np.concatenate(keep)
    fr.y, fr.z, fr.rowsec = base.y[idx], base.z[idx], base.rowsec[idx]
    fr.y64, fr.z64 = base.y64[idx], base.z64[idx]
    fr.offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return fr, lens


def test_smoother_equals_leave_one_out_least_squares(oracle_mod, synth):
    # Linearised about the exact trajectory, the outward and inward steps are
    # exact inverses of each other and the model is linear-Gaussian.  The
    # smoothed residual of a cluster must then equal the dense weighted least-
    # squares solve without that cluster, under the two priors the passes use:
    # the seed (C0) on the first state and the outward result (C0) on the last.
    fr, lens = _short_tracks(synth, 11)
    ref = truth_trajectory(oracle_mod, fr)
    s = oracle_mod.smooth(fr, ref=ref, exact_inputs=True)
    r = oracle_mod.fit(fr, "f64", ref=ref, trace=True, exact_inputs=True)
    m = np.stack([fr.y64, fr.z64], axis=1)
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    checked = 0
    for i in range(fr.n_tracks):
        order, A, bb = _affine_chain(oracle_mod, fr, ref, i, backward=False)
        last = order[-1]
        p_out = r["trace"][last, 0, :5]
        for k, h in enumerate(order):
            N = np.eye(5) / 100.0
            rhs = fr.seeds64[:, i] / 100.0
            N += A[-1].T @ A[-1] / 100.0
            rhs += A[-1].T @ (p_out - bb[-1]) / 100.0
            for kk, j in enumerate(order):
                if kk == k:
                    continue
                HA = H @ A[kk]
                N += HA.T @ HA / 0.01
                rhs += HA.T @ (m[j] - H @ bb[kk]) / 0.01
            x0 = np.linalg.solve(N, rhs)
            P = np.linalg.inv(N)
            xc = A[k] @ x0 + bb[k]
            Rc = 0.01 * np.eye(2) + (A[k] @ P @ A[k].T)[:2, :2]
            rc = m[h] - xc[:2]
            assert np.allclose(s["resid"][h], rc, rtol=1e-7, atol=1e-10)
            assert np.allclose(s["rcov"][h], [Rc[0, 0], Rc[1, 0], Rc[1, 1]], rtol=1e-7, atol=1e-13)
            assert abs(s["chi2"][h] - rc @ np.linalg.solve(Rc, rc)) < 1e-7 * max(1.0, s["chi2"][h])
            checked += 1
    assert checked == lens.sum()


def test_smoothed_states_equal_least_squares(oracle_mod, synth):
    # Linearised about the exact trajectory: the smoothed state at every
    # cluster (all clusters of the track, both passes' priors) equals the
    # dense weighted least-squares solve mapped to that cluster, and its
    # covariance the solve's covariance mapped there.
    fr, lens = _short_tracks(synth, 12)
    ref = truth_trajectory(oracle_mod, fr)
    s = oracle_mod.smooth_states(fr, ref=ref, exact_inputs=True)
    r = oracle_mod.fit(fr, "f64", ref=ref, trace=True, exact_inputs=True)
    m = np.stack([fr.y64, fr.z64], axis=1)
    H = np.zeros((2, 5)); H[0, 0] = 1; H[1, 1] = 1
    checked = 0
    for i in range(fr.n_tracks):
        order, A, bb = _affine_chain(oracle_mod, fr, ref, i, backward=False)
        p_out = r["trace"][order[-1], 0, :5]
        N = np.eye(5) / 100.0 + A[-1].T @ A[-1] / 100.0
        rhs = fr.seeds64[:, i] / 100.0 + A[-1].T @ (p_out - bb[-1]) / 100.0
        for kk, j in enumerate(order):
            HA = H @ A[kk]
            N += HA.T @ HA / 0.01
            rhs += HA.T @ (m[j] - H @ bb[kk]) / 0.01
        x0 = np.linalg.solve(N, rhs)
        P = np.linalg.inv(N)
        for k, h in enumerate(order):
            xc = A[k] @ x0 + bb[k]
            Pc = A[k] @ P @ A[k].T
            assert np.allclose(s["state"][h], xc, rtol=1e-8, atol=1e-10)
            assert np.allclose(oracle_mod.unpack(s["state_cov"][h]), Pc, rtol=1e-7, atol=1e-14)
            checked += 1
    assert checked == lens.sum()


def test_smoothed_state_at_the_first_cluster_is_the_fit_with_the_seed_prior(oracle_mod, synth):
    # At the first cluster the outward pass holds only the seed prior (seed,
    # c0 I) and that cluster; the inward pass's prediction there holds every
    # other cluster, so with the linear (y, z) measurement the smoothed state
    # is the inward refit's output combined, in information form, with the
    # seed prior — on the real, non-linearised fit of full-length tracks.
    fr = synth.generate(400, 15, drop_p=0.05, cap_lengths=True)
    s = oracle_mod.smooth_states(fr)
    r = oracle_mod.fit(fr, "f64")
    ok = r["ndf"] > 0
    assert ok.mean() > 0.95
    first = fr.offsets[:-1][ok]
    If = np.linalg.inv(np.moveaxis(oracle_mod.unpack(r["cov"][:, ok]), -1, 0))
    Cs = np.linalg.inv(If + np.eye(5) / 100.0)
    xs = np.einsum("nij,nj->ni", Cs, np.einsum("nij,nj->ni", If, r["params"][:, ok].T) + fr.seeds[:, ok].T / 100.0)
    sig = np.sqrt(np.einsum("nii->ni", Cs))
    assert np.max(np.abs(s["state"][first] - xs) / np.maximum(np.abs(xs), sig)) < 1e-7
    Cg = np.moveaxis(oracle_mod.unpack(s["state_cov"][first].T), -1, 0)
    assert np.max(np.abs(Cg - Cs) / np.sqrt(np.einsum("nii->ni", Cs)[:, :, None] * np.einsum("nii->ni", Cs)[:, None, :])) < 1e-7
    # the seed prior matters for the short, poorly measured tracks only
    moved = np.abs(xs - r["params"][:, ok].T) / sig
    assert np.median(moved) < 1e-2


def test_smoother_flags_a_displaced_cluster(oracle_mod, synth):
    # a cluster moved by 1 cm (10 sigma) stands out: the largest chi2 of its
    # track, far beyond the 2-dof tail; the rest follow the 2-dof distribution
    fr = synth.generate(300, 31, drop_p=0.05, cap_lengths=True)
    off = fr.offsets
    moved = off[:-1] + np.diff(off) // 2
    fr.y = fr.y.copy()
    fr.y[moved] += np.float32(1.0)
    s = oracle_mod.smooth(fr)
    c2 = s["chi2"]
    for i in range(fr.n_tracks):
        if s["ndf"][i] <= 0:
            continue
        seg = c2[off[i]:off[i + 1]]
        assert np.nanargmax(seg) == moved[i] - off[i]
        assert seg[moved[i] - off[i]] > 40.0
    rest = np.delete(c2, moved)
    rest = rest[np.isfinite(rest)]
    assert abs(rest.mean() - 2.0) < 0.25


@pytest.mark.parametrize("form", ["f64", "sqrt_f64"])
def test_linearised_filter_equals_dense_least_squares(oracle_mod, synth, form):
    # with a fixed linearisation the filter is linear-Gaussian: each pass must
    # equal the brute-force weighted least-squares solve of the same model, and
    # the accumulated chi2 must equal the minimum of the objective (prior incl.)
    rng = np.random.default_rng(7)
    base = synth.generate(60, 23, drop_p=0.05)
    keep = [np.arange(o, o + int(rng.integers(3, 9))) for o in base.offsets[:-1]]
    fr = base.subset(np.arange(base.n_tracks))
    # cut each track to its first 3..8 hits
    lens = np.array([len(k) for k in keep])
    idx = np.concatenate(keep)
    fr.y, fr.z, fr.rowsec = base.y[idx], base.z[idx], base.rowsec[idx]
    fr.y64, fr.z64 = base.y64[idx], base.z64[idx]
    fr.offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ref = truth_trajectory(oracle_mod, fr)
    ref_pert = ref + rng.normal(size=ref.shape) * np.array([0.05, 0.05, 0.01, 0.01, 0.05])
    r = oracle_mod.fit(fr, form, ref=ref_pert, trace=True, exact_inputs=True)
    m = np.stack([fr.y64, fr.z64], axis=1)
    off = fr.offsets.astype(np.int64)
    for i in range(fr.n_tracks):
        assert r["ndf"][i] == 2 * lens[i] - 5
        # outward pass: prior = seed at the first hit
        order, A, bb = _affine_chain(oracle_mod, fr, ref_pert, i, backward=False)
        x0, obj, P = _gls(order, A, bb, m, fr.seeds64[:, i], 100.0)
        last = order[-1]
        t_out = r["trace"][last, 0]
        x_last = A[-1] @ x0 + bb[-1]
        assert np.allclose(t_out[:5], x_last, rtol=1e-9, atol=1e-9)
        assert abs(t_out[20] - obj) < 1e-8 * max(1.0, obj)
        C_last = A[-1] @ P @ A[-1].T
        assert np.allclose(oracle_mod.unpack(t_out[5:20]), C_last, rtol=1e-7, atol=1e-11)
        # inward pass: prior = outward result at the last hit, C reset to C0
        order, A, bb = _affine_chain(oracle_mod, fr, ref_pert, i, backward=True)
        xl, obj, P = _gls(order, A, bb, m, t_out[:5], 100.0)
        x_first = A[-1] @ xl + bb[-1]
        assert np.allclose(r["params"][:, i], x_first, rtol=1e-9, atol=1e-9)
        assert abs(r["chi2"][i] - obj) < 1e-8 * max(1.0, obj)
        assert np.allclose(oracle_mod.unpack(r["cov"][:, i]), A[-1] @ P @ A[-1].T, rtol=1e-7, atol=1e-11)
        assert off[i + 1] - off[i] == lens[i]


def test_straight_tracks_match_polynomial_regression(oracle_mod, synth):
    # q/pt -> 0 limit in one sector, tan(lambda) = 0.  Linearised about the true
    # straight trajectory the measurement model is exactly y = a + b dx + e dx^2
    # (b = tan(phi_ref) + (s - s_ref)/c^3, e = kappa q / (2 c^3)) and
    # z = z0 + t dx / c, so the filter must equal the textbook weighted
    # polynomial regressions (the prior C0 = 100 I is 1e-6 of the data weight).
    # The relinearising filter agrees to a small fraction of sigma (median below
    # 0.05; its linearisation points move during the first hits after the
    # diffuse start of each pass).
    n = 300
    rng = np.random.default_rng(8)
    g = synth.default_geometry()
    sec = rng.integers(0, 18, n)
    phi0 = (sec + 0.5) * math.radians(20) + rng.uniform(-0.05, 0.05, n)
    fr, ok = synth.simulate(np.zeros(n), np.zeros(n), phi0, np.abs(rng.normal(0, 5, n)) + 1.0, g, 0.5,
                            smear=0.1, streams={"smear": np.random.default_rng(9)})
    assert np.all((fr.rowsec & 63) % 18 == np.repeat(sec[ok] % 18, fr.lengths()))
    ref = truth_trajectory(oracle_mod, fr)
    lin = oracle_mod.fit(fr, "f64", ref=ref)
    ekf = oracle_mod.fit(fr, "f64")
    kappa = synth.KAPPA_PER_TESLA * fr.bz
    off = fr.offsets.astype(np.int64)
    sig = np.sqrt(lin["cov"][[0, 2, 5, 9, 14]])
    ekf_dev = []
    for i in range(fr.n_tracks):
        a, b = off[i], off[i + 1]
        X = g.row_x[fr.rowsec[a:b].astype(int) >> 6]
        dx = X - X[0]
        Y = fr.y[a:b].astype(np.float64)
        Z = fr.z[a:b].astype(np.float64)
        s_ref = fr.truth[2, i]
        c = math.sqrt(1 - s_ref ** 2)
        cy = np.polynomial.polynomial.polyfit(dx, Y, 2)
        cz = np.polynomial.polynomial.polyfit(dx / c, Z, 1)
        est = np.array([cy[0], cz[0], s_ref + c ** 3 * (cy[1] - s_ref / c), cz[1], 2 * c ** 3 * cy[2] / kappa])
        d = np.abs(lin["params"][:, i] - est) / sig[:, i]
        assert d.max() < 1e-4, (i, d)
        ekf_dev.append(np.abs(ekf["params"][:, i] - est) / sig[:, i])
    ekf_dev = np.array(ekf_dev)
    assert np.all(np.median(ekf_dev, axis=0) < 0.05), np.median(ekf_dev, axis=0)
    assert ekf_dev.max() < 1.0


# ---------------------------------------------------------------- statistics
def test_pulls_of_linearised_filter_are_standard_normal(oracle_mod, synth):
    fr = synth.generate(20000, 24, drop_p=0.05, cap_lengths=True)
    ref = truth_trajectory(oracle_mod, fr)
    r = oracle_mod.fit(fr, "f64", ref=ref)
    ok = r["ndf"] > 0
    assert ok.mean() > 0.999
    sig = np.sqrt(r["cov"][[0, 2, 5, 9, 14]])
    pull = ((r["params"] - fr.truth) / sig)[:, ok]
    assert np.all(np.abs(pull.mean(axis=1)) < 0.03), pull.mean(axis=1)
    assert np.all(np.abs(pull.std(axis=1) - 1) < 0.025), pull.std(axis=1)
    chi2n = r["chi2"][ok] / r["ndf"][ok]
    assert abs(chi2n.mean() - 1) < 0.01
    # chi2 probability is flat
    from scipy.stats import chi2 as chi2dist
    pv = chi2dist.sf(r["chi2"][ok], r["ndf"][ok])
    hist, _ = np.histogram(pv, bins=10, range=(0, 1))
    assert np.all(np.abs(hist / hist.mean() - 1) < 0.1), hist


PT_BINS = ((0.2, 0.3), (0.3, 0.5), (0.5, 2.0), (2.0, 10.0))


def _pull_widths(oracle_mod, fr, **kw):
    r = oracle_mod.fit(fr, "f64", **kw)
    ok = r["ndf"] > 0
    sig = np.sqrt(r["cov"][[0, 2, 5, 9, 14]])
    pull = ((r["params"] - fr.truth) / sig)[:, ok]
    pt = 1 / np.abs(fr.truth[4, ok])
    return pull, [pull[:, (pt >= lo) & (pt < hi)].std(axis=1) for lo, hi in PT_BINS]


def test_pulls_of_extended_filter(oracle_mod, synth):
    # the relinearising filter with the reset reading of the inward restart:
    # unbiased; widths per pt bin (columns y, z, sin phi, tan lambda, q/pt)
    # within these bounds, with the excess of sin phi and q/pt at low pt (see
    # the next pin for where it comes from).  About 2,000-8,000 tracks per bin:
    # the statistical error of a width is ~0.015.
    fr = synth.generate(20000, 25, drop_p=0.05, cap_lengths=True)
    pull, widths = _pull_widths(oracle_mod, fr)
    assert np.all(np.abs(pull.mean(axis=1)) < 0.03)
    bounds = ((0.03, 0.03, 0.08, 0.03, 0.13),    # pt 0.2-0.3 GeV/c: measured 1.00 0.98 1.06 1.00 1.10
              (0.03, 0.03, 0.05, 0.03, 0.08),    # pt 0.3-0.5: 1.00 0.99 1.03 1.00 1.06
              (0.035, 0.035, 0.035, 0.035, 0.035),
              (0.035, 0.035, 0.035, 0.035, 0.035))
    for (lo, hi), w, b in zip(PT_BINS, widths, bounds):
        assert np.all(np.abs(w - 1) < np.array(b)), (lo, hi, w)
    assert widths[0][4] > 1.06   # the low-pt excess is there


def test_pull_excess_comes_from_the_diffuse_restart(oracle_mod, synth):
    # The same tracks with the test-only informative restart of the inward
    # pass (C = 1e4 C_out instead of C0 = 100 I): the filter no longer
    # relinearises about the few-cluster estimate a diffuse prior jumps to, and
    # the low-pt widths return to 1 (the prior's double counting of the outward
    # information is 1e-4 of it); so the excess follows from the reset reading.
    fr = synth.generate(20000, 25, drop_p=0.05, cap_lengths=True)
    _, widths = _pull_widths(oracle_mod, fr, inward_inflate=1e4)
    for (lo, hi), w in zip(PT_BINS, widths):
        assert np.all(np.abs(w - 1) < 0.02), (lo, hi, w)
    # with only 10 C_out the restart counts the outward clusters once more, a
    # tenth of their weight: every width grows by about sqrt(1.1)
    _, w10 = _pull_widths(oracle_mod, fr, inward_inflate=10.0)
    assert all(np.all(w > 1.03) for w in w10)


# ---------------------------------------------------------------- forms and precisions
def test_square_root_form_equals_covariance_form_fp64(oracle_mod, frame_drop):
    a = oracle_mod.fit(frame_drop, "f64")
    b = oracle_mod.fit(frame_drop, "sqrt_f64")
    assert np.array_equal(a["ndf"], b["ndf"])
    ok = a["ndf"] > 0
    sig = np.sqrt(a["cov"][[0, 2, 5, 9, 14]])
    assert np.nanmax(np.abs(a["params"] - b["params"])[:, ok] / sig[:, ok]) < 1e-7
    assert np.nanmax(np.abs(a["chi2"] - b["chi2"])[ok] / a["chi2"][ok]) < 1e-8
    ii = [0, 2, 5, 9, 14]
    pairs = [(i, j) for i in range(5) for j in range(i + 1)]
    for e, (i, j) in enumerate(pairs):
        scale = np.sqrt(a["cov"][ii[i]] * a["cov"][ii[j]])
        assert np.nanmax(np.abs(a["cov"][e] - b["cov"][e])[ok] / scale[ok]) < 1e-7


def test_strict_fp32_within_fast_mode_tolerance(oracle_mod, frame_drop):
    # the FP32 sequence against the FP64 reference, with the tolerance reading
    # used for the fast GPU mode (relative to max(|p|, sigma)); see tolerance.py
    from paper_2511_17018_gb300 import tolerance
    a = oracle_mod.fit(frame_drop, "f64")
    b = oracle_mod.fit(frame_drop, "f32")
    rep = tolerance.compare_to_fp64(b, a)
    assert rep["ok"], rep


def test_failure_conventions(oracle_mod, synth):
    fr = synth.generate(50, 26)
    seeds = fr.seeds.copy()
    seeds[2, 0] = 0.9995          # |sin phi| >= 0.999: unusable seed
    short = fr.subset(np.arange(50))
    lens = short.lengths().copy()
    lens[1] = 2                   # two hits: fewer than 3 used
    idx = np.concatenate([np.arange(o, o + l) for o, l in zip(short.offsets[:-1], lens)])
    short.y, short.z, short.rowsec = short.y[idx], short.z[idx], short.rowsec[idx]
    short.offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    for prec in ("f64", "f32"):
        r = oracle_mod.fit(short, prec, seeds=seeds)
        assert r["ndf"][0] == -1 and r["ndf"][1] == -1
        assert np.all(np.isnan(r["params"][:, :2]))
        assert np.all(r["ndf"][2:] > 0)
    empty = short.subset(np.arange(0))
    r = oracle_mod.fit(empty, "f64")
    assert r["params"].shape == (5, 0)


# ---------------------------------------------------------------- gradient reference
def test_forward_mode_gradient_matches_central_differences(oracle_mod, synth):
    d_true = synth.alignment_offsets(3)
    fr = synth.generate(8, 27, drop_p=0.05, cap_lengths=True, d_true=d_true)
    rng = np.random.default_rng(10)
    w = rng.uniform(0.5, 2.0, fr.n_tracks)
    gr = oracle_mod.grad(fr, weights=w)
    y = fr.y.astype(np.float64); z = fr.z.astype(np.float64)

    def L(yv, zv, sd):
        ff = fr.subset(np.arange(fr.n_tracks))
        ff.y64, ff.z64, ff.seeds64 = yv, zv, sd
        return float((oracle_mod.fit(ff, "f64", exact_inputs=True)["chi2"] * w).sum())

    h = 1e-4
    gfd = np.zeros((fr.n_hits, 2))
    for j in range(fr.n_hits):
        for c, arr in ((0, y), (1, z)):
            ap = arr.copy(); ap[j] += h
            am = arr.copy(); am[j] -= h
            fp = L(ap, z, fr.seeds.astype(np.float64)) if c == 0 else L(y, ap, fr.seeds.astype(np.float64))
            fm = L(am, z, fr.seeds.astype(np.float64)) if c == 0 else L(y, am, fr.seeds.astype(np.float64))
            gfd[j, c] = (fp - fm) / (2 * h)
    assert np.linalg.norm(gr["grad_meas"] - gfd) / np.linalg.norm(gfd) < 1e-6
    # seeds: the fit hardly depends on them (diffuse prior); FD noise ~1e-6
    gs = np.zeros((5, fr.n_tracks))
    for c in range(5):
        for i in range(fr.n_tracks):
            sp = fr.seeds.astype(np.float64).copy(); sp[c, i] += 1e-5
            sm = fr.seeds.astype(np.float64).copy(); sm[c, i] -= 1e-5
            gs[c, i] = (L(y, z, sp) - L(y, z, sm)) / 2e-5
    assert np.abs(gr["grad_seed"] - gs).max() < 1e-5 * np.abs(gfd).max()
    assert np.linalg.norm(gr["grad_seed"] - gs) < 0.1 * np.linalg.norm(gs)


@pytest.mark.parametrize("phys", ["field", "gas", "field+gas"])
def test_forward_mode_gradient_with_field_map_and_material_matches_central_differences(oracle_mod, synth, phys):
    # the gradient reference through the midpoint curvature of the field map
    # (which moves with the state) and through the material layers (energy
    # loss and the process noise, which depend on the state)
    fr = synth.generate(5, 31, drop_p=0.05, cap_lengths=True)
    field = synth.FieldMap(0.3, -0.2) if "field" in phys else None
    mat = synth.TPC_GAS if "gas" in phys else None
    fr.field, fr.material = field, mat
    gr = oracle_mod.grad(fr)
    assert np.all(gr["ndf"] > 0)
    y = fr.y.astype(np.float64); z = fr.z.astype(np.float64); sd = fr.seeds.astype(np.float64)

    def L(yv, zv):
        ff = fr.subset(np.arange(fr.n_tracks))
        ff.y64, ff.z64, ff.seeds64 = yv, zv, sd
        ff.field, ff.material = field, mat
        return float(oracle_mod.fit(ff, "f64", exact_inputs=True)["chi2"].sum())

    h = 1e-4
    gfd = np.zeros((fr.n_hits, 2))
    for j in range(fr.n_hits):
        for c, arr in ((0, y), (1, z)):
            ap = arr.copy(); ap[j] += h
            am = arr.copy(); am[j] -= h
            fp = L(ap, z) if c == 0 else L(y, ap)
            fm = L(am, z) if c == 0 else L(y, am)
            gfd[j, c] = (fp - fm) / (2 * h)
    assert np.linalg.norm(gr["grad_meas"] - gfd) / np.linalg.norm(gfd) < 1e-6
    # and the physics matters: the gradient without it is far off
    fr.field = fr.material = None
    assert np.linalg.norm(oracle_mod.grad(fr)["grad_meas"] - gfd) / np.linalg.norm(gfd) > 1e-3


# ---------------------------------------------------------------- material (per-row layers)
def _material_tracks(synth, n, seed, **kw):
    """Tracks of 2-5 GeV/c near the centre of sector 0 (they stay in it)
    through thick layers (X0 = 300 cm, 0.2 MeV/cm per cm of layer)."""
    rng = np.random.default_rng(seed)
    qpt = rng.choice([-1, 1], n) / rng.uniform(2.0, 5.0, n)
    tanl = rng.uniform(-0.5, 0.5, n)
    phi0 = np.full(n, 0.5 * math.pi / 9) + rng.uniform(-0.03, 0.03, n)
    z0 = rng.normal(0, 5, n)
    mat = synth.Material(300.0, 2e-4)
    return synth.simulate_material(qpt, tanl, phi0, z0, synth.default_geometry(), 0.5, mat, rng=rng, **kw), mat


def test_material_pulls_are_standard_normal(oracle_mod, synth):
    # the generator scatters the direction by drawn angles and lowers the energy
    # row by row (not through the fit's covariance formulas); with the material
    # correction the fitted parameters scatter as their covariance says, without
    # it they do not
    fr, mat = _material_tracks(synth, 400, 1)
    pulls = {}
    for use in (True, False):
        fr.material = mat if use else None
        r = oracle_mod.fit(fr, "f64")
        ok = r["ndf"] > 0
        C = oracle_mod.unpack(r["cov"][:, ok])
        sig = np.sqrt(np.stack([C[i, i] for i in range(5)]))
        pulls[use] = (r["params"][:, ok] - fr.truth[:, ok]) / sig
    p = pulls[True]
    assert np.all(np.abs(p.mean(axis=1)) < 0.15), p.mean(axis=1)
    assert np.all((p.std(axis=1) > 0.88) & (p.std(axis=1) < 1.12)), p.std(axis=1)
    assert pulls[False].std(axis=1).max() > 2.0


def test_material_noise_free_energy_loss(oracle_mod, synth):
    # energy loss without scattering or smearing: the refit to convergence returns
    # the generating parameters (the inward pass undoes a layer with the momentum
    # after it, a second-order difference); without the correction q/pt is off
    fr, mat = _material_tracks(synth, 40, 3, scatter=False, smear=0.0)
    seeds = fr.seeds64.copy()
    for _ in range(4):
        r = oracle_mod.fit(fr, "f64", exact_inputs=True, seeds=seeds)
        seeds = r["params"].copy()
    assert np.all(r["ndf"] > 0)
    assert np.abs(r["params"][:4] - fr.truth[:4]).max() < 1e-7
    assert (np.abs(r["params"][4] - fr.truth[4]) / np.abs(fr.truth[4])).max() < 1e-7
    fr.material = None
    r0 = oracle_mod.fit(fr, "f64", exact_inputs=True, seeds=seeds)
    assert (np.abs(r0["params"][4] - fr.truth[4]) / np.abs(fr.truth[4])).max() > 1e-3


@pytest.mark.parametrize("thick", [False, True])
def test_material_square_root_form_equals_covariance_form(oracle_mod, synth, thick):
    # C <- D C D + B B^T (covariance form) against L <- R^T of the QR of
    # [(D L)^T; B^T] (square-root form), both in FP64
    fr = synth.generate(1000, 5, drop_p=0.05, cap_lengths=True)
    fr.material = synth.Material(300.0, 2e-4) if thick else synth.TPC_GAS
    a = oracle_mod.fit(fr, "f64")
    b = oracle_mod.fit(fr, "sqrt_f64")
    assert np.array_equal(a["ndf"], b["ndf"])
    ok = a["ndf"] > 0
    assert np.allclose(a["params"][:, ok], b["params"][:, ok], rtol=1e-8, atol=1e-10)
    assert np.allclose(a["cov"][:, ok], b["cov"][:, ok], rtol=1e-6, atol=1e-14)
    assert np.allclose(a["chi2"][ok], b["chi2"][ok], rtol=1e-8)


def test_material_strict_fp32_within_fast_mode_tolerance(oracle_mod, synth):
    from paper_2511_17018_gb300 import tolerance
    fr = synth.generate(3000, 6, drop_p=0.05, cap_lengths=True)
    fr.material = synth.TPC_GAS
    rep = tolerance.compare_to_fp64(oracle_mod.fit(fr, "f32"), oracle_mod.fit(fr, "f64"))
    assert rep["ok"], rep


# ---------------------------------------------------------------- field map
def _field_tracks(synth, n, seed, **kw):
    """Tracks of 2-5 GeV/c near the centre of sector 0 in the map
    Bz = 0.5 T (1 + 0.3 (r/250)^2 - 0.2 (z/250)^2), integrated by RK4."""
    rng = np.random.default_rng(seed)
    qpt = rng.choice([-1, 1], n) / rng.uniform(2.0, 5.0, n)
    tanl = rng.uniform(-0.5, 0.5, n)
    phi0 = np.full(n, 0.5 * math.pi / 9) + rng.uniform(-0.03, 0.03, n)
    z0 = rng.normal(0, 5, n)
    fm = synth.FieldMap(0.3, -0.2)
    return synth.simulate_field(qpt, tanl, phi0, z0, synth.default_geometry(), 0.5, fm, rng=rng, step_cm=0.5,
                                **kw), fm


def test_field_map_pulls_are_standard_normal(oracle_mod, synth):
    # the generator integrates the equation of motion in the map (Runge-Kutta),
    # the fit takes a helix per step with Bz at the step's midpoint; with the map
    # the parameters scatter as their covariance says, with a uniform field not
    fr, fm = _field_tracks(synth, 250, 1)
    widths = {}
    for use in (True, False):
        fr.field = fm if use else None
        r = oracle_mod.fit(fr, "f64")
        ok = r["ndf"] > 0
        C = oracle_mod.unpack(r["cov"][:, ok])
        sig = np.sqrt(np.stack([C[i, i] for i in range(5)]))
        pull = (r["params"][:, ok] - fr.truth[:, ok]) / sig
        widths[use] = pull.std(axis=1)
        if use:
            assert np.all(np.abs(pull.mean(axis=1)) < 0.15), pull.mean(axis=1)
    assert np.all((widths[True] > 0.85) & (widths[True] < 1.15)), widths[True]
    assert widths[False].max() > 3.0


def test_field_map_noise_free_refit(oracle_mod, synth):
    # exact clusters of Runge-Kutta tracks: the refit to convergence returns the
    # generating parameters (the midpoint helix differs from the exact path at
    # second order in the step)
    fr, fm = _field_tracks(synth, 30, 3, smear=0.0)
    seeds = fr.seeds64.copy()
    for _ in range(4):
        r = oracle_mod.fit(fr, "f64", exact_inputs=True, seeds=seeds)
        seeds = r["params"].copy()
    assert np.all(r["ndf"] > 0)
    assert np.abs(r["params"][:4] - fr.truth[:4]).max() < 1e-6
    assert (np.abs(r["params"][4] - fr.truth[4]) / np.abs(fr.truth[4])).max() < 3e-6


def test_field_map_forms_and_strict_fp32(oracle_mod, synth):
    from paper_2511_17018_gb300 import tolerance
    fr = synth.generate(1000, 5, drop_p=0.05, cap_lengths=True)
    fr.field = synth.FieldMap(0.3, -0.2)
    a = oracle_mod.fit(fr, "f64")
    b = oracle_mod.fit(fr, "sqrt_f64")
    ok = a["ndf"] > 0
    assert np.array_equal(a["ndf"], b["ndf"])
    assert np.allclose(a["params"][:, ok], b["params"][:, ok], rtol=1e-8, atol=1e-10)
    rep = tolerance.compare_to_fp64(oracle_mod.fit(fr, "f32"), a)
    assert rep["ok"], rep


def test_fp32_dual_asinc_derivative_matches_closed_form(oracle_mod):
    # d/du asin(u)/u = (u / sqrt(1 - u^2) - asin(u)) / u^2; the FP32 dual takes
    # the derivative of its polynomial for |u| <= 1/4 and of the FP64 island above
    for u in np.concatenate([np.linspace(-0.9, 0.9, 181), [1e-3, -1e-3, 0.2499, 0.2501, 0.01]]):
        v, d = oracle_mod.asinc_dual_f32(u)
        uf = float(np.float32(u))
        assert v == oracle_mod.asinc_f32(uf)
        if abs(uf) < 1e-6:
            continue
        exact = (uf / np.sqrt(1.0 - uf * uf) - np.arcsin(uf)) / (uf * uf)
        assert abs(d - exact) <= 1e-7 * max(1.0, abs(exact)), (u, d, exact)


def test_fp32_dual_gradient_follows_the_strict_fp32_fit(oracle_mod, synth):
    # the FP32-valued dual evaluates the strict-FP32 sequence itself: chi2 and
    # ndf bit for bit those of the float fit; its derivative (carried in FP64)
    # is that of the FP32 trajectory, so it sits within the FP32 forward's own
    # rounding (a few 1e-5 in norm) of the FP64 gradient, not at 1e-9
    d_true = synth.alignment_offsets(3)
    fr = synth.generate(300, 3, drop_p=0.05, cap_lengths=True, d_true=d_true)
    w = np.random.default_rng(5).uniform(0.5, 2.0, fr.n_tracks).astype(np.float32).astype(np.float64)
    g32 = oracle_mod.grad(fr, weights=w, align=d_true, precision="f32")
    g64 = oracle_mod.grad(fr, weights=w, align=d_true)
    f32 = oracle_mod.fit(fr, "f32", align=d_true)
    ok = f32["ndf"] > 0
    assert ok.mean() > 0.99
    assert np.array_equal(g32["ndf"], f32["ndf"])
    assert np.array_equal(g32["chi2"][ok].astype(np.float32).view(np.int32), f32["chi2"][ok].view(np.int32))
    a, b = g32["grad_meas"], g64["grad_meas"]
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert 1e-6 < rel < 2e-4, rel
    scale = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
    assert np.quantile(np.abs(a - b) / scale, 0.99) < 2e-3
    assert np.linalg.norm(g32["grad_seed"] - g64["grad_seed"]) < 3e-4 * np.linalg.norm(g64["grad_seed"])


@pytest.mark.parametrize("phys", ["field", "gas", "field+gas"])
def test_fp32_dual_follows_the_strict_fp32_fit_with_physics(oracle_mod, synth, phys):
    # the FP32-valued dual through the field map and the material layers: its
    # chi2 is bit for bit the strict-FP32 fit's, its gradient within the FP32
    # floor of the FP64 gradient
    fr = synth.generate(60, 31, drop_p=0.05, cap_lengths=True)
    fr.field = synth.FieldMap(0.3, -0.2) if "field" in phys else None
    fr.material = synth.TPC_GAS if "gas" in phys else None
    g32 = oracle_mod.grad(fr, precision="f32")
    g64 = oracle_mod.grad(fr)
    f32 = oracle_mod.fit(fr, "f32")
    ok = f32["ndf"] > 0
    assert ok.all() and np.array_equal(g32["ndf"], f32["ndf"])
    assert np.array_equal(g32["chi2"][ok].astype(np.float32).view(np.int32), f32["chi2"][ok].view(np.int32))
    a, b = g32["grad_meas"], g64["grad_meas"]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 3e-4
