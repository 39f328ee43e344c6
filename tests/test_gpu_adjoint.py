"""The hand-written adjoint against the oracle's forward-mode gradients and
FP64 central finite differences (run on a GB300 with -m gpu).  Gradients are
compared element by element: |g - g_ref| <= tol * max(|g_ref|, 1e-3 max|g_ref|)
(tolerance.gradient_errors).

Two references.  (1) The gradient of the strict-FP32 fit itself (oracle
precision 'f32': the same FP32 operation sequence as the deterministic kernels,
its derivative carried exactly in FP64).  The deterministic adjoint runs on
that very trajectory, so the two differ only by the FP32 rounding of the
reverse sweep's own arithmetic (measured on 2,500 and 3,000 tracks: cluster
gradients 1.4e-7 in norm, 99.9% of elements within 6e-6 to 1e-5, the worst
at 5e-5; alignment keys at most 8e-5).  DET_NORM = 1e-5 holds the norm to the
gradient accuracy asked of the method; DET_Q999 and DET_MAX hold the elements.
The seed gradient is ~1e-5 of the cluster gradient (the diffuse prior), so its
elements carry the cluster gradients' rounding relative to a far smaller
scale.  (2) The FP64 gradient.  No FP32 gradient can be closer to it than the
FP32 forward is to the FP64 forward -- cluster positions carry ~4e-6 cm of
rounding against ~0.1 cm residuals -- which shifts even the strict-FP32
trajectory's exact gradient by ~5e-5 in norm and by up to ~2e-2 in single
cluster elements and ~6e-2 in alignment keys whose clusters cancel
(measured); FP32_ELEM bounds that floor and the norm stays at 5e-4."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2511_17018_gb300 import synth, tolerance  # noqa: E402
from paper_2511_17018_gb300 import tpcfit as tf  # noqa: E402
from paper_2511_17018_gb300.autograd import fit_chi2  # noqa: E402

REL = 5e-4
DET_NORM = 1e-5
DET_Q999 = {"meas": 2e-5, "align": 1e-4}
DET_MAX = {"meas": 1e-4, "align": 2e-4, "seeds": 1e-2}
FP32_ELEM = 0.1


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _elem(got, ref):
    return tolerance.gradient_errors(got, ref)


@pytest.fixture(scope="module")
def case():
    d_true = synth.alignment_offsets(3)
    fr = synth.generate(3000, 3, drop_p=0.05, cap_lengths=True, d_true=d_true)
    w = np.random.default_rng(5).uniform(0.5, 2.0, fr.n_tracks).astype(np.float32)
    ref = oracle.grad(fr, weights=w.astype(np.float64), align=d_true)
    ref["f32"] = oracle.grad(fr, weights=w.astype(np.float64), align=d_true, precision="f32")
    return fr, d_true, w, ref


def _gpu_grad(fr, d_true, w, det, rps=4, warps=24, srt=True, bwd=12, form=1, fit_form=1):
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=det, rows_per_stage=rps, warps_per_block=warps,
                  sort_by_length=srt)
    f.set_backward_config(bwd)
    f.set_backward_form(form)
    f.set_fit_form(fit_form)
    try:
        f.set_alignment(torch.from_numpy(d_true).cuda())
        f.set_record(True)
        out = f.fit(dev)
        gm = torch.empty((fr.n_hits, 2), device="cuda")
        ga, gs = f.backward(dev, out, torch.from_numpy(w).cuda(), gm)
        torch.cuda.synchronize()
        return gm.cpu().numpy(), ga.cpu().numpy(), gs.cpu().numpy(), out["ndf"].cpu().numpy()
    finally:
        f.close()


@pytest.mark.parametrize("det,form", [(False, 1), (False, 0), (True, 0)], ids=["fast-ud", "fast-sqrt", "det"])
def test_adjoint_matches_forward_mode_oracle(case, det, form):
    # against the FP64 gradient: per element within the FP32 forward's floor
    fr, d_true, w, ref = case
    gm, ga, gs, ndf = _gpu_grad(fr, d_true, w, det, form=form, fit_form=form)
    assert np.array_equal(ndf, ref["ndf"])
    ga_ref = oracle.align_grad_from_meas(fr, ref["grad_meas"])
    for name, got, want in (("meas", gm, ref["grad_meas"]), ("align", ga, ga_ref), ("seeds", gs, ref["grad_seed"])):
        e = _elem(got, want)
        print(name, e)
        assert e["max"] < FP32_ELEM and e["norm"] < (10 * REL if name == "seeds" else REL), (name, e)


def test_fast_adjoint_factor_forms_agree(case):
    # the U-D and the square-root recomputation differentiate the same recorded
    # fast fit (square-root form): they differ by the FP32 rounding of the
    # reverse sweeps only, in every compiled block shape
    fr, d_true, w, _ = case
    base = _gpu_grad(fr, d_true, w, False, form=0, fit_form=0)
    for bwd in (4, 8, 10, 12):
        got = _gpu_grad(fr, d_true, w, False, bwd=bwd, form=1, fit_form=0)
        for name, a, b in zip(("meas", "align", "seeds"), got[:3], base[:3]):
            e = _elem(a, b)
            print(bwd, name, e)
            assert e["norm"] < 2e-5 and e["max"] < 1e-2, (bwd, name, e)


def test_deterministic_adjoint_matches_the_fp32_sequence_gradient(case):
    # the deterministic adjoint runs on the strict-FP32 trajectory: against that
    # trajectory's exact gradient only the reverse sweep's rounding remains
    fr, d_true, w, ref = case
    r32 = ref["f32"]
    gm, ga, gs, ndf = _gpu_grad(fr, d_true, w, True)
    assert np.array_equal(ndf, r32["ndf"])
    ga_ref = oracle.align_grad_from_meas(fr, r32["grad_meas"])
    for name, got, want in (("meas", gm, r32["grad_meas"]), ("align", ga, ga_ref), ("seeds", gs, r32["grad_seed"])):
        e = _elem(got, want)
        assert e["max"] <= DET_MAX[name], (name, e)
        if name != "seeds":
            assert e["norm"] <= DET_NORM and e["q999"] <= DET_Q999[name], (name, e)
        else:
            assert e["norm"] <= 1e-4, (name, e)


def test_deterministic_adjoint_is_bitwise_reproducible(case):
    fr, d_true, w, _ = case
    base = _gpu_grad(fr, d_true, w, True)
    for rps, warps, srt, bwd in ((4, 24, True, 8), (8, 8, False, 4), (16, 8, True, 12), (4, 12, True, 10)):
        got = _gpu_grad(fr, d_true, w, True, rps, warps, srt, bwd)
        for a, b in zip(got[:3], base[:3]):
            assert np.array_equal(a.view(np.int32), b.view(np.int32)), (rps, warps, srt, bwd)


def _det_reduce(fr, d_true, w, method, shapes=((4, 24, True, 8),)):
    """Deterministic per-cluster and alignment gradients with the given
    reduction, in each launch shape (rows per stage, warps, length order,
    backward warps)."""
    res = []
    for rps, warps, srt, bwd in shapes:
        dev = tf.frame_to_device(fr)
        f = tf.Fitter(fr.geometry, fr.bz, deterministic=True, rows_per_stage=rps, warps_per_block=warps,
                      sort_by_length=srt)
        try:
            f.set_backward_config(bwd)
            f.set_det_reduction(method)
            f.set_alignment(torch.from_numpy(d_true).cuda())
            f.set_record(True)
            out = f.fit(dev)
            gm = torch.empty((fr.n_hits, 2), device="cuda")
            ga, gs = f.backward(dev, out, torch.from_numpy(w).cuda(), gm)
            torch.cuda.synchronize()
            res.append((gm.cpu().numpy(), ga.cpu().numpy()))
        finally:
            f.close()
    return res


def _exact_key_sums(fr, gm):
    """-(sum over each (sector, row) of the per-cluster gradients), in FP64 with
    a compensated (math.fsum) sum per key."""
    import math
    rs = fr.rowsec.astype(np.int64)
    key = (rs & 63) * 152 + (rs >> 6)
    out = np.zeros((36 * 152, 2))
    mag = np.zeros((36 * 152, 2))
    order = np.argsort(key, kind="stable")
    ks = key[order]
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    ends = np.r_[starts[1:], ks.size]
    g = gm.astype(np.float64)[order]
    for b, e in zip(starts, ends):
        out[ks[b], 0] = -math.fsum(g[b:e, 0])
        out[ks[b], 1] = -math.fsum(g[b:e, 1])
        mag[ks[b]] = np.abs(g[b:e]).sum(axis=0)
    return out.reshape(36, 152, 2), mag.reshape(36, 152, 2)


def test_deterministic_fixed_point_sums_are_exact_sums_rounded_once(case):
    # the default reduction: each key's result is the exact sum of the FP32
    # per-cluster gradients to within one FP32 rounding of the result plus
    # the fixed-point unit per cluster (2^-S, S = 62 - ceil(log2(H+1)) -
    # exponent of the largest |g|); the sorted FP32 sums are within the
    # rounding of an FP32 summation of the same values
    fr, d_true, w, _ = case
    (gm, ga), = _det_reduce(fr, d_true, w, 0)
    exact, mag = _exact_key_sums(fr, gm)
    amax = np.abs(gm).max()
    e = np.frexp(amax)[1]
    cbits = int(np.ceil(np.log2(fr.n_hits + 1)))
    unit = 2.0 ** (-(62 - cbits - int(e)))
    n_key = np.bincount(((fr.rowsec.astype(np.int64) & 63) * 152 + (fr.rowsec.astype(np.int64) >> 6)),
                        minlength=36 * 152).reshape(36, 152, 1)
    bound = np.abs(exact) * 2.0 ** -23 + n_key * unit * 0.5 + 1e-45
    assert np.all(np.abs(ga.astype(np.float64) - exact) <= bound)
    (gm1, ga1), = _det_reduce(fr, d_true, w, 1)
    assert np.array_equal(gm1.view(np.int32), gm.view(np.int32))  # the reduction does not touch the clusters
    # an FP32 sum of n terms: within n 2^-24 of the sum of their magnitudes
    err = np.abs(ga1.astype(np.float64) - exact)
    assert np.all(err <= n_key * 2.0 ** -24 * mag + 1e-45), (err / np.maximum(mag, 1e-30)).max()


def test_both_deterministic_reductions_are_bitwise_reproducible(case):
    fr, d_true, w, _ = case
    shapes = ((4, 24, True, 8), (8, 8, False, 4), (16, 8, True, 12))
    for method in (0, 1):
        res = _det_reduce(fr, d_true, w, method, shapes) + _det_reduce(fr, d_true, w, method, shapes[:1])
        for gm, ga in res[1:]:
            assert np.array_equal(ga.view(np.int32), res[0][1].view(np.int32)), method
            assert np.array_equal(gm.view(np.int32), res[0][0].view(np.int32)), method


def test_det_reduction_setter_rejects_other_values():
    fr = synth.generate(20, 38)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        for bad in (-1, 2):
            with pytest.raises(tf.TpcfitError) as e:
                f.set_det_reduction(bad)
            assert e.value.status == tf.EINVAL
    finally:
        f.close()


def test_alignment_gradient_matches_fp64_finite_differences():
    # central differences of the FP64 oracle's weighted chi2 sum, step 1e-4 cm,
    # on a 200-track subset of the 100,000-track adjoint workload (its first
    # 200 tracks that the oracle fits), for 40 (sector, row, component) keys
    # the subset uses
    d_true = synth.alignment_offsets(3)
    whole = synth.adjoint_frame()
    head = whole.subset(np.arange(400))
    fitted = np.flatnonzero(oracle.fit(head, "f64", align=d_true)["ndf"] > 0)[:200]
    assert fitted.size == 200
    fr = head.subset(fitted)
    w = np.ones(fr.n_tracks, np.float32)
    _, ga, _, ndf = _gpu_grad(fr, d_true, w, False)
    assert np.all(ndf > 0)
    rs = fr.rowsec.astype(np.int64)
    keys = np.unique((rs & 63) * 152 + (rs >> 6))
    pick = np.random.default_rng(6).choice(keys, 40, replace=False)
    h = 1e-4
    fd, got = [], []
    for k in pick:
        for c in (0, 1):
            dp = d_true.astype(np.float64).copy().reshape(-1, 2)
            dm = dp.copy()
            dp[k, c] += h
            dm[k, c] -= h
            lp = np.nansum(oracle.fit(fr, "f64", align=dp.reshape(36, 152, 2))["chi2"])
            lm = np.nansum(oracle.fit(fr, "f64", align=dm.reshape(36, 152, 2))["chi2"])
            fd.append((lp - lm) / (2 * h))
            got.append(ga.reshape(-1, 2)[k, c])
    fd = np.array(fd)
    assert rel(got, fd) < REL
    # per component against the largest: the FP32 forward's floor (~5e-5 of each element)
    assert np.abs(np.array(got) - fd).max() <= 2e-4 * np.abs(fd).max()


def test_autograd_function_and_masking(case):
    fr, d_true, w, ref = case
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        align = torch.from_numpy(d_true).cuda().requires_grad_(True)
        seeds = dev["seeds"].clone().requires_grad_(True)
        chi2, params, ndf = fit_chi2(align, seeds, f, dev)
        ok = ndf > 0
        loss = (chi2[ok] * torch.from_numpy(w).cuda()[ok]).sum()
        loss.backward()
        ea = _elem(align.grad.cpu().numpy(), oracle.align_grad_from_meas(fr, ref["grad_meas"]))
        es = _elem(seeds.grad.cpu().numpy(), ref["grad_seed"])
        assert ea["max"] < FP32_ELEM and ea["norm"] < REL, ea
        assert es["max"] < FP32_ELEM and es["norm"] < 10 * REL, es
    finally:
        f.close()


def test_factor_form_setters_reject_other_values():
    fr = synth.generate(20, 37)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        for bad in (-1, 2):
            with pytest.raises(tf.TpcfitError) as e:
                f.set_fit_form(bad)
            assert e.value.status == tf.EINVAL
            with pytest.raises(tf.TpcfitError) as e:
                f.set_backward_form(bad)
            assert e.value.status == tf.EINVAL
        f.set_fit_form(0)
        f.set_backward_form(0)
    finally:
        f.close()


def test_square_root_reverse_refuses_a_u_d_recording():
    fr = synth.generate(200, 36)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        f.set_record(True)
        f.set_fit_form(1)
        out = f.fit(dev)
        f.set_backward_form(0)
        with pytest.raises(tf.TpcfitError) as e:
            f.backward(dev, out, torch.ones(fr.n_tracks, device="cuda"))
        assert e.value.status == tf.ESTATE
        f.set_backward_form(1)
        ga, gs = f.backward(dev, out, torch.ones(fr.n_tracks, device="cuda"))
        torch.cuda.synchronize()
        assert np.all(np.isfinite(ga.cpu().numpy()))
    finally:
        f.close()


def test_backward_requires_a_recorded_fit():
    fr = synth.generate(50, 34)
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        out = f.fit(dev)  # recording is off
        with pytest.raises(tf.TpcfitError) as e:
            f.backward(dev, out, torch.ones(fr.n_tracks, device="cuda"))
        assert e.value.status == tf.ESTATE
        f.set_record(True)
        out = f.fit(dev)
        f.set_mode(True)   # mode changed since the recording
        with pytest.raises(tf.TpcfitError):
            f.backward(dev, out, torch.ones(fr.n_tracks, device="cuda"))
    finally:
        f.close()


def test_failed_tracks_contribute_nothing():
    fr = synth.generate(64, 35)
    fr.seeds[2, :8] = 0.9995  # unusable seeds: these tracks fail
    dev = tf.frame_to_device(fr)
    f = tf.Fitter(fr.geometry, fr.bz)
    try:
        f.set_record(True)
        out = f.fit(dev)
        gm = torch.full((fr.n_hits, 2), 9.0, device="cuda")
        ga, gs = f.backward(dev, out, torch.ones(fr.n_tracks, device="cuda"), gm)
        torch.cuda.synchronize()
        assert np.all(out["ndf"].cpu().numpy()[:8] == -1)
        gm = gm.cpu().numpy()
        assert np.all(gm[: fr.offsets[8]] == 0)
        assert np.all(gs.cpu().numpy()[:, :8] == 0)
        assert np.all(np.isfinite(ga.cpu().numpy()))
    finally:
        f.close()


def test_fit_adjoint_host_pipelined_calls(case):
    # the host-buffer entry point equals the device calls bit for bit
    # (deterministic mode), and two calls issued back to back (the second's
    # copies overlapping the first's work) each return their own batch's results
    fr, d_true, w, _ = case
    parts = [fr.subset(np.arange(0, 1500)), fr.subset(np.arange(1500, fr.n_tracks))]
    f = tf.Fitter(fr.geometry, fr.bz, deterministic=True)
    try:
        f.set_alignment(torch.from_numpy(d_true).cuda())
        want = []
        for p in parts:
            dev = tf.frame_to_device(p)
            f.set_record(True)
            out = f.fit(dev)
            ga, gs = f.backward(dev, out, torch.from_numpy(w[:p.n_tracks]).cuda())
            torch.cuda.synchronize()
            want.append((out["chi2"].cpu().numpy(), out["ndf"].cpu().numpy(), ga.cpu().numpy(), gs.cpu().numpy()))
        f.set_record(False)
        pins = []
        for p in parts:
            pins.append([torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
                         (p.y, p.z, p.rowsec.view(np.int16), p.offsets, p.seeds, w[:p.n_tracks])])
        got = []
        for p, pn in zip(parts, pins):
            y, z, rs, off, sd, g = (t.numpy() for t in pn)
            got.append(tf.tpcfit_fit_adjoint_host(f.h, y, z, rs.view(np.uint16), off, sd, g))
        torch.cuda.synchronize()
    finally:
        f.close()
    for (chi2, ndf, ga, gs), o in zip(want, got):
        assert np.array_equal(o["ndf"], ndf)
        assert np.array_equal(o["chi2"].view(np.int32), chi2.view(np.int32))
        assert np.array_equal(o["grad_align"].view(np.int32), ga.view(np.int32))
        assert np.array_equal(o["grad_seeds"].view(np.int32), gs.view(np.int32))
