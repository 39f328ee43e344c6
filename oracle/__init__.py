"""CPU oracle of the batched TPC Kalman track fit -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is independent of the CUDA library
(no shared code, headers or tables); ``tpcfit_oracle.cpp`` holds the fit.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class _Geo(C.Structure):
    _fields_ = [("row_x", C.POINTER(C.c_double)), ("n_rows", C.c_int32), ("n_sectors", C.c_int32),
                ("sector_width_deg", C.c_double), ("x0_cm", C.c_double), ("dedx_gev_cm", C.c_double),
                ("mass_gev", C.c_double), ("row_cm", C.c_double), ("field_cr", C.c_double),
                ("field_cz", C.c_double), ("inward_inflate", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        for name in ("oracle_fit_f64", "oracle_fit_f32", "oracle_fit_sqrt_f64", "oracle_fit_cov_f32",
                     "oracle_fit_pred_f64"):
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = [C.POINTER(_Geo), C.c_double, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                          C.c_int32]
        for name in ("oracle_grad_f64", "oracle_grad_f32"):
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = [C.POINTER(_Geo), C.c_double, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                          C.c_int32]
        L.oracle_step_f64.restype = C.c_int
        L.oracle_step_f64.argtypes = [C.POINTER(_Geo), C.c_double, vp, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                      vp, vp, vp]
        L.oracle_update_f64.restype = C.c_int
        L.oracle_update_f64.argtypes = [vp, vp, vp, vp]
        L.oracle_transport_f64.restype = C.c_int
        L.oracle_transport_f64.argtypes = [vp, vp]
        L.oracle_asin_f64.restype = C.c_double
        L.oracle_asin_f64.argtypes = [C.c_double]
        L.oracle_asinc_f32.restype = C.c_float
        L.oracle_asinc_f32.argtypes = [C.c_float]
        L.oracle_asinc_dual_f32.restype = C.c_float
        L.oracle_asinc_dual_f32.argtypes = [C.c_float, C.POINTER(C.c_double)]
        L.oracle_guard_count.restype = C.c_longlong
        L.oracle_guard_reset.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _geo(geometry, material=None, field=None, inward_inflate=0.0):
    """ctypes geometry; material: object with x0_cm, dedx_gev_cm, mass_gev, row_cm (None: none);
    field: object with c_r, c_z of the field map (None: uniform); inward_inflate:
    the test-only informative restart of the inward pass (0: C reset to C0)."""
    rx = np.ascontiguousarray(geometry.row_x, dtype=np.float64)
    m = material
    g = _Geo(rx.ctypes.data_as(C.POINTER(C.c_double)), rx.shape[0], geometry.n_sectors,
             float(geometry.sector_width_deg), float(m.x0_cm) if m is not None else 0.0,
             float(m.dedx_gev_cm) if m is not None else 0.0, float(m.mass_gev) if m is not None else 0.0,
             float(m.row_cm) if m is not None else 0.0, float(field.c_r) if field is not None else 0.0,
             float(field.c_z) if field is not None else 0.0, float(inward_inflate))
    return g, rx


def default_threads() -> int:
    return max(1, min(os.cpu_count() or 1, 64))


def fit(frame, precision: str = "f64", align=None, ref=None, trace: bool = False, exact_inputs: bool = False,
        nthreads: int | None = None, seeds=None, inward_inflate: float = 0.0):
    """Run the oracle fit on a ``synth.Frame``.

    precision: 'f64' (FP64 reference, covariance form), 'f32' (strict FP32
    reference, square-root form), 'sqrt_f64' (square-root form in FP64) or
    'cov_f32' (covariance form in strict FP32).
    exact_inputs: feed the FP64 copies of hits / seeds (noise-free tests).
    inward_inflate > 0: test-only reading of the inward restart, from
    inward_inflate * C_out instead of C0 (0: the product reading).
    Returns dict(params[5,n], cov[15,n], chi2[n], ndf[n], trace[H,2,22] or None).
    """
    L = lib()
    dt = np.float64 if precision in ("f64", "sqrt_f64") else np.float32
    n = frame.n_tracks
    H = frame.n_hits
    if exact_inputs:
        y, z = frame.y64, frame.z64
        sd = frame.seeds64 if seeds is None else seeds
    else:
        y, z = frame.y, frame.z
        sd = frame.seeds if seeds is None else seeds
    y = np.ascontiguousarray(y, dtype=dt)
    z = np.ascontiguousarray(z, dtype=dt)
    sd = np.ascontiguousarray(sd, dtype=dt)
    rs = np.ascontiguousarray(frame.rowsec, dtype=np.uint16)
    off = np.ascontiguousarray(frame.offsets, dtype=np.int32)
    al = None if align is None else np.ascontiguousarray(align, dtype=dt).reshape(-1)
    rf = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    params = np.empty((5, n), dt); cov = np.empty((15, n), dt); chi2 = np.empty(n, dt)
    ndf = np.empty(n, np.int32)
    tr = np.empty((H, 2, 22), np.float64) if trace else None
    g, _keep = _geo(frame.geometry, getattr(frame, "material", None), getattr(frame, "field", None), inward_inflate)
    fn = {"f64": L.oracle_fit_f64, "f32": L.oracle_fit_f32, "sqrt_f64": L.oracle_fit_sqrt_f64,
          "cov_f32": L.oracle_fit_cov_f32}[precision]
    rc = fn(C.byref(g), float(frame.bz), n, _ptr(off), _ptr(y), _ptr(z), _ptr(rs), _ptr(sd), _ptr(al), _ptr(rf),
            _ptr(params), _ptr(cov), _ptr(chi2), _ptr(ndf), _ptr(tr), nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle fit rejected its inputs (rc={rc})")
    return dict(params=params, cov=cov, chi2=chi2, ndf=ndf, trace=tr)


def grad(frame, weights=None, align=None, nthreads: int | None = None, exact_inputs: bool = False,
         precision: str = "f64"):
    """Forward-mode gradient of L = sum_i w_i chi2_i.

    precision 'f64': FP64 values (covariance form), the gradient reference.
    precision 'f32': the strict-FP32 fit's own operation sequence (square-root
    form, residual coordinates; chi2 and ndf bit for bit those of
    ``fit(frame, 'f32')``) with its exact derivative carried in FP64 -- the
    reference for an FP32 reverse-mode adjoint of that sequence.
    Returns dict(grad_meas[H,2] = dL/dm, grad_seed[5,n], chi2[n], ndf[n]).
    dL/d(alignment offset of key (sector,row,c)) = -sum of grad_meas over hits with that key.
    """
    L = lib()
    n = frame.n_tracks
    H = frame.n_hits
    dt = {"f64": np.float64, "f32": np.float32}[precision]
    y = np.ascontiguousarray(frame.y64 if exact_inputs else frame.y, dtype=dt)
    z = np.ascontiguousarray(frame.z64 if exact_inputs else frame.z, dtype=dt)
    sd = np.ascontiguousarray(frame.seeds64 if exact_inputs else frame.seeds, dtype=dt)
    rs = np.ascontiguousarray(frame.rowsec, dtype=np.uint16)
    off = np.ascontiguousarray(frame.offsets, dtype=np.int32)
    al = None if align is None else np.ascontiguousarray(align, dtype=dt).reshape(-1)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    gm = np.zeros((H, 2)); gs = np.zeros((5, n)); chi2 = np.empty(n); ndf = np.empty(n, np.int32)
    g, _keep = _geo(frame.geometry, getattr(frame, "material", None), getattr(frame, "field", None))
    fn = L.oracle_grad_f64 if precision == "f64" else L.oracle_grad_f32
    rc = fn(C.byref(g), float(frame.bz), n, _ptr(off), _ptr(y), _ptr(z), _ptr(rs), _ptr(sd), _ptr(al), _ptr(w),
            _ptr(gm), _ptr(gs), _ptr(chi2), _ptr(ndf), nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle grad rejected its inputs (rc={rc})")
    return dict(grad_meas=gm, grad_seed=gs, chi2=chi2, ndf=ndf)


# Cluster variance of the fit: sigma_y = sigma_z = 0.1 cm.
V_MEAS = 0.01


def smooth(frame, align=None, ref=None, exact_inputs: bool = False, seeds=None, nthreads: int | None = None):
    """Two-filter smoother of the FP64 fit (Fraser & Potter, 1969): for every
    cluster, the estimate from all the other clusters is the information-
    weighted mean of the outward prediction (clusters before it, seed prior)
    and the inward prediction (clusters after it, the inward pass's prior):

        C_u = (C_out^-1 + C_in^-1)^-1,   x_u = C_u (C_out^-1 x_out + C_in^-1 x_in).

    Per cluster h: resid[h] = m_h - (y, z) of x_u (m = measured y, z minus the
    alignment offsets), rcov[h] = (R00, R10, R11) of R = V + H C_u H^T, and
    chi2[h] = resid^T R^-1 resid.  NaN for the clusters of unfitted tracks and
    for clusters the outward pass did not reach.
    Returns dict(resid[H,2], rcov[H,3], chi2[H], ndf[n]).
    """
    L = lib()
    n = frame.n_tracks
    H = frame.n_hits
    y = np.ascontiguousarray(frame.y64 if exact_inputs else frame.y, dtype=np.float64)
    z = np.ascontiguousarray(frame.z64 if exact_inputs else frame.z, dtype=np.float64)
    sd = frame.seeds64 if exact_inputs else frame.seeds
    sd = np.ascontiguousarray(sd if seeds is None else seeds, dtype=np.float64)
    rs = np.ascontiguousarray(frame.rowsec, dtype=np.uint16)
    off = np.ascontiguousarray(frame.offsets, dtype=np.int32)
    al = None if align is None else np.ascontiguousarray(align, dtype=np.float64).reshape(-1)
    rf = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    params = np.empty((5, n)); cov = np.empty((15, n)); chi2 = np.empty(n); ndf = np.empty(n, np.int32)
    pt = np.empty((H, 2, 20))
    g, _keep = _geo(frame.geometry, getattr(frame, "material", None), getattr(frame, "field", None))
    rc = L.oracle_fit_pred_f64(C.byref(g), float(frame.bz), n, _ptr(off), _ptr(y), _ptr(z), _ptr(rs), _ptr(sd),
                               _ptr(al), _ptr(rf), _ptr(params), _ptr(cov), _ptr(chi2), _ptr(ndf), _ptr(pt),
                               nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle fit rejected its inputs (rc={rc})")
    m = np.stack([y, z], axis=1)
    if al is not None:
        a = al.reshape(36 * 152, 2)
        key = (rs.astype(np.int64) & 63) * 152 + (rs.astype(np.int64) >> 6)
        m = m - a[key]
    fitted = np.repeat(ndf > 0, np.diff(off))
    ok = fitted & np.all(np.isfinite(pt.reshape(H, -1)), axis=1)
    resid = np.full((H, 2), np.nan)
    rcov = np.full((H, 3), np.nan)
    c2 = np.full(H, np.nan)
    if ok.any():
        x1, x2 = pt[ok, 0, :5], pt[ok, 1, :5]
        C1 = np.moveaxis(unpack(pt[ok, 0, 5:].T), -1, 0)
        C2 = np.moveaxis(unpack(pt[ok, 1, 5:].T), -1, 0)
        I1, I2 = np.linalg.inv(C1), np.linalg.inv(C2)
        Cu = np.linalg.inv(I1 + I2)
        xu = np.einsum("nij,nj->ni", Cu, np.einsum("nij,nj->ni", I1, x1) + np.einsum("nij,nj->ni", I2, x2))
        r = m[ok] - xu[:, :2]
        R = V_MEAS * np.eye(2) + Cu[:, :2, :2]
        resid[ok] = r
        rcov[ok] = np.stack([R[:, 0, 0], R[:, 1, 0], R[:, 1, 1]], axis=1)
        c2[ok] = np.einsum("ni,ni->n", r, np.linalg.solve(R, r[..., None])[..., 0])
    return dict(resid=resid, rcov=rcov, chi2=c2, ndf=ndf)


def smooth_states(frame, align=None, ref=None, exact_inputs: bool = False, seeds=None, nthreads: int | None = None):
    """Smoothed state at every cluster from all clusters of its track (FP64,
    two-filter form, Fraser & Potter 1969): the information-weighted mean of
    the outward pass's filtered state at the cluster (seed prior and clusters
    0..c) and the inward pass's prediction there (the inward prior and clusters
    c+1..last):
        C_s = (C_out^-1 + C_in^-1)^-1,   x_s = C_s (C_out^-1 x_out + C_in^-1 x_in).
    Positions are absolute, in the cluster's sector frame at its pad row.
    NaN for the clusters of unfitted tracks and for clusters the outward pass
    did not reach.  Returns dict(state[H,5], state_cov[H,15] (packed), ndf[n]).
    """
    L = lib()
    n = frame.n_tracks
    H = frame.n_hits
    y = np.ascontiguousarray(frame.y64 if exact_inputs else frame.y, dtype=np.float64)
    z = np.ascontiguousarray(frame.z64 if exact_inputs else frame.z, dtype=np.float64)
    sd = frame.seeds64 if exact_inputs else frame.seeds
    sd = np.ascontiguousarray(sd if seeds is None else seeds, dtype=np.float64)
    rs = np.ascontiguousarray(frame.rowsec, dtype=np.uint16)
    off = np.ascontiguousarray(frame.offsets, dtype=np.int32)
    al = None if align is None else np.ascontiguousarray(align, dtype=np.float64).reshape(-1)
    rf = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    params = np.empty((5, n)); cov = np.empty((15, n)); chi2 = np.empty(n); ndf = np.empty(n, np.int32)
    pt = np.empty((H, 2, 20))
    g, _keep = _geo(frame.geometry, getattr(frame, "material", None), getattr(frame, "field", None))
    rc = L.oracle_fit_pred_f64(C.byref(g), float(frame.bz), n, _ptr(off), _ptr(y), _ptr(z), _ptr(rs), _ptr(sd),
                               _ptr(al), _ptr(rf), _ptr(params), _ptr(cov), _ptr(chi2), _ptr(ndf), _ptr(pt),
                               nthreads or default_threads())
    if rc != 0:
        raise ValueError(f"oracle fit rejected its inputs (rc={rc})")
    tr = fit(frame, "f64", align=align, ref=ref, trace=True, exact_inputs=exact_inputs, nthreads=nthreads,
             seeds=seeds)["trace"]
    fitted = np.repeat(ndf > 0, np.diff(off))
    ok = fitted & np.all(np.isfinite(tr[:, 0, :20]), axis=1) & np.all(np.isfinite(pt[:, 1]), axis=1)
    state = np.full((H, 5), np.nan)
    scov = np.full((H, 15), np.nan)
    if ok.any():
        x1, x2 = tr[ok, 0, :5], pt[ok, 1, :5]
        C1 = np.moveaxis(unpack(tr[ok, 0, 5:20].T), -1, 0)
        C2 = np.moveaxis(unpack(pt[ok, 1, 5:].T), -1, 0)
        I1, I2 = np.linalg.inv(C1), np.linalg.inv(C2)
        Cs = np.linalg.inv(I1 + I2)
        xs = np.einsum("nij,nj->ni", Cs, np.einsum("nij,nj->ni", I1, x1) + np.einsum("nij,nj->ni", I2, x2))
        state[ok] = xs
        scov[ok] = pack(np.moveaxis(Cs, 0, -1)).T
    return dict(state=state, state_cov=scov, ndf=ndf)


def align_grad_from_meas(frame, grad_meas):
    """dL/d(offsets) [36,152,2] from dL/dm (m = raw - offset)."""
    rs = frame.rowsec.astype(np.int64)
    key = (rs & 63) * 152 + (rs >> 6)
    out = np.zeros((36 * 152, 2))
    np.add.at(out, key, -grad_meas)
    return out.reshape(36, 152, 2)


def step(geometry, bz, p, x, sec_in, row_out, sec_out):
    """One FP64 prediction step; returns (p_out[5], x_out, J[5,5]) or None if it fails."""
    L = lib()
    g, _keep = _geo(geometry)
    p = np.ascontiguousarray(p, np.float64)
    po = np.empty(5); xo = np.empty(1); J = np.empty(25)
    rc = L.oracle_step_f64(C.byref(g), float(bz), _ptr(p), float(x), int(sec_in), int(row_out), int(sec_out),
                           _ptr(po), _ptr(xo), _ptr(J))
    if rc != 0:
        return None
    return po, float(xo[0]), J.reshape(5, 5)


def update(p, Cp, m):
    """One FP64 Kalman update on packed covariance; returns (p, C, dchi2) or None."""
    L = lib()
    p = np.array(p, np.float64); Cp = np.array(Cp, np.float64); m = np.ascontiguousarray(m, np.float64)
    c2 = np.zeros(1)
    rc = L.oracle_update_f64(_ptr(p), _ptr(Cp), _ptr(c2), _ptr(m))
    return None if rc else (p, Cp, float(c2[0]))


def transport(Cp, J):
    L = lib()
    Cp = np.array(Cp, np.float64); J = np.ascontiguousarray(J, np.float64).reshape(-1)
    L.oracle_transport_f64(_ptr(Cp), _ptr(J))
    return Cp


def asin_f64(u: float) -> float:
    return lib().oracle_asin_f64(float(u))


def asinc_f32(u: float) -> float:
    return lib().oracle_asinc_f32(float(u))


def asinc_dual_f32(u: float):
    """(value, derivative) of the strict-FP32 asinc as its dual number carries them."""
    d = C.c_double()
    v = lib().oracle_asinc_dual_f32(float(u), C.byref(d))
    return float(v), float(d.value)


def guard_count() -> int:
    return int(lib().oracle_guard_count())


def guard_reset() -> None:
    lib().oracle_guard_reset()


PACKED = [(i, j) for i in range(5) for j in range(i + 1)]


def unpack(cp):
    """Packed lower-triangular [15,...] -> symmetric [5,5,...]."""
    cp = np.asarray(cp)
    M = np.zeros((5, 5) + cp.shape[1:], cp.dtype)
    for e, (i, j) in enumerate(PACKED):
        M[i, j] = cp[e]
        M[j, i] = cp[e]
    return M


def pack(M):
    return np.stack([M[i, j] for (i, j) in PACKED])
