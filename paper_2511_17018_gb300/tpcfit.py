"""Python binding of libtpcfit (include/tpcfit.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device arrays are
torch CUDA tensors (torch provides device memory and streams); every step of
the fit runs in the library's kernels.  There is no CPU fallback: if the
shared library is missing or fails to load, the functions raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpcfit.so")

OK, EINVAL, ECUDA, ENOMEM, EDEVICE, ETIMEOUT, ESTATE, ERTC = range(8)


class TpcfitError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class _Geometry(C.Structure):
    _fields_ = [("n_sectors", C.c_int32), ("n_rows", C.c_int32), ("row_x", C.POINTER(C.c_double)),
                ("sector_width_deg", C.c_double), ("z_max", C.c_double)]


class _Hits(C.Structure):
    _fields_ = [("y", C.c_void_p), ("z", C.c_void_p), ("rowsec", C.c_void_p), ("n_hits", C.c_int64)]


_lib = None


def load():
    """Load libtpcfit.so (built by paper_2511_17018_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtpcfit.so not built ({LIB_PATH}); run paper_2511_17018_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "tpcfit_create": (C.c_int, [C.POINTER(_Geometry), C.c_double, C.POINTER(vp)]),
        "tpcfit_destroy": (None, [vp]),
        "tpcfit_set_mode": (C.c_int, [vp, C.c_int]),
        "tpcfit_set_config": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int]),
        "tpcfit_set_alignment": (C.c_int, [vp, vp, vp]),
        "tpcfit_reserve": (C.c_int, [vp, i64, i64]),
        "tpcfit_fit": (C.c_int, [vp, C.POINTER(_Hits), vp, i32, vp, vp, vp, vp, vp, vp]),
        "tpcfit_fit_host": (C.c_int, [vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp]),
        "tpcfit_fit_adjoint_host": (C.c_int, [vp, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp, vp]),
        "tpcfit_get_status": (C.c_int, [vp, vp, C.POINTER(i32), C.POINTER(i64)]),
        "tpcfit_fit_noalloc": (C.c_int, [C.POINTER(_Geometry), C.c_double, vp, C.c_int, C.POINTER(_Hits), vp, i32, vp,
                                         vp, vp, vp, vp, vp]),
        "tpcfit_set_record": (C.c_int, [vp, C.c_int]),
        "tpcfit_set_backward_config": (C.c_int, [vp, C.c_int]),
        "tpcfit_set_backward_form": (C.c_int, [vp, C.c_int]),
        "tpcfit_set_det_reduction": (C.c_int, [vp, C.c_int]),
        "tpcfit_set_fit_form": (C.c_int, [vp, C.c_int]),
        "tpcfit_reject_outliers": (C.c_int, [vp, C.POINTER(_Hits), vp, C.c_int32, vp, C.c_float, vp, vp, vp, vp, vp]),
        "tpcfit_fit_frames": (C.c_int, [vp, C.POINTER(_Hits), vp, i32, vp, i32, vp, vp, i64, vp, vp, vp, vp, vp,
                                        vp]),
        "tpcfit_fit_backward": (C.c_int, [vp, C.POINTER(_Hits), vp, i32, vp, vp, vp, vp, vp, vp]),
        "tpcfit_smooth": (C.c_int, [vp, C.POINTER(_Hits), vp, i32, vp, vp, vp, vp, vp]),
        "tpcfit_smooth_states": (C.c_int, [vp, C.POINTER(_Hits), vp, i32, vp, vp, vp, vp]),
        "tpcfit_set_material": (C.c_int, [vp, C.c_double, C.c_double, C.c_double, C.c_double]),
        "tpcfit_set_field_map": (C.c_int, [vp, C.c_double, C.c_double]),
        "tpcfit_set_rtc": (C.c_int, [vp, C.c_int, C.c_char_p]),
        "tpcfit_rtc_build": (C.c_int, [C.POINTER(_Geometry), C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_char_p]),
        "tpcfit_rtc_available": (C.c_int, []),
        "tpcfit_rtc_compile_count": (C.c_longlong, []),
        "tpcfit_rtc_log": (C.c_char_p, []),
        "tpcfit_fp32_peak": (C.c_int, [C.c_int, i64, vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "tpcfit_status_string": (C.c_char_p, [C.c_int]),
        "tpcfit_version": (i32, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st: int, where: str):
    if st != OK:
        raise TpcfitError(st, where)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return t.data_ptr()


def _check_sizes(n, y, z, rowsec, seeds=None, params=None, cov=None, chi2=None, ndf=None):
    """The C entry points see only pointers: array sizes are checked here."""
    if z.numel() != y.numel() or rowsec.numel() != y.numel():
        raise ValueError("y, z and rowsec must have the same length")
    for name, t, per in (("seeds", seeds, 5), ("params", params, 5), ("cov", cov, 15), ("chi2", chi2, 1),
                         ("ndf", ndf, 1)):
        if t is not None and t.numel() != per * n:
            raise ValueError(f"{name} has {t.numel()} elements, {per * n} expected for {n} tracks")


def status_string(st: int) -> str:
    return load().tpcfit_status_string(int(st)).decode()


def tpcfit_fp32_peak(mode: int = 0, iterations: int = 200000, stream=None):
    """(FP32 flops executed, launch ms) of the FMA-chain microbenchmark."""
    fl, ms = C.c_double(), C.c_double()
    _check(load().tpcfit_fp32_peak(int(mode), int(iterations), _stream(stream), C.byref(fl), C.byref(ms)),
           "tpcfit_fp32_peak")
    return fl.value, ms.value


def tpcfit_version() -> int:
    return int(load().tpcfit_version())


def _geometry(geometry):
    """(ctypes geometry, the row array it points into)."""
    rx = np.ascontiguousarray(geometry.row_x, dtype=np.float64)
    g = _Geometry(int(geometry.n_sectors), int(rx.shape[0]), rx.ctypes.data_as(C.POINTER(C.c_double)),
                  float(geometry.sector_width_deg), float(getattr(geometry, "z_max", 250.0)))
    return g, rx


def tpcfit_create(geometry, bz: float):
    """geometry: object with row_x (float64 array), n_sectors, sector_width_deg, z_max."""
    L = load()
    g, rx = _geometry(geometry)
    h = C.c_void_p()
    _check(L.tpcfit_create(C.byref(g), float(bz), C.byref(h)), "tpcfit_create")
    return h


def tpcfit_set_material(h, x0_cm: float = 0.0, dedx_gev_cm: float = 0.0, mass_gev: float = 0.13957,
                        row_cm: float = 160.0 / 151.0) -> None:
    _check(load().tpcfit_set_material(h, float(x0_cm), float(dedx_gev_cm), float(mass_gev), float(row_cm)),
           "tpcfit_set_material")


def tpcfit_set_field_map(h, c_r: float = 0.0, c_z: float = 0.0) -> None:
    _check(load().tpcfit_set_field_map(h, float(c_r), float(c_z)), "tpcfit_set_field_map")


def tpcfit_set_rtc(h, enable: bool = True, cache_dir: str | None = None) -> None:
    _check(load().tpcfit_set_rtc(h, int(bool(enable)), cache_dir.encode() if cache_dir else None), "tpcfit_set_rtc")


def tpcfit_rtc_build(geometry, bz: float, deterministic: bool = False, rows_per_stage: int = 4,
                     warps_per_block: int = 24, record: bool = False, frames: bool = False,
                     cache_dir: str | None = None) -> None:
    g, rx = _geometry(geometry)
    st = load().tpcfit_rtc_build(C.byref(g), float(bz), int(bool(deterministic)), int(rows_per_stage),
                                 int(warps_per_block), int(bool(record)), int(bool(frames)),
                                 cache_dir.encode() if cache_dir else None)
    if st != OK:
        raise TpcfitError(st, "tpcfit_rtc_build: " + tpcfit_rtc_log()[-2000:])


def tpcfit_rtc_available() -> bool:
    return bool(load().tpcfit_rtc_available())


def tpcfit_rtc_compile_count() -> int:
    return int(load().tpcfit_rtc_compile_count())


def tpcfit_rtc_log() -> str:
    return (load().tpcfit_rtc_log() or b"").decode(errors="replace")


def tpcfit_destroy(h) -> None:
    load().tpcfit_destroy(h)


def tpcfit_set_mode(h, deterministic: bool) -> None:
    _check(load().tpcfit_set_mode(h, int(bool(deterministic))), "tpcfit_set_mode")


def tpcfit_set_config(h, lanes_per_track: int = 1, rows_per_stage: int = 4, warps_per_block: int = 24,
                      sort_by_length: bool = True) -> None:
    _check(load().tpcfit_set_config(h, int(lanes_per_track), int(rows_per_stage), int(warps_per_block),
                                    int(bool(sort_by_length))), "tpcfit_set_config")


def tpcfit_set_alignment(h, d=None, stream=None) -> None:
    import torch
    ptr = None
    if d is not None:
        if d.numel() != 36 * 152 * 2:
            raise ValueError("alignment must have 36*152*2 elements")
        ptr = _dev(d, torch.float32, "alignment")
    _check(load().tpcfit_set_alignment(h, ptr, _stream(stream)), "tpcfit_set_alignment")


def tpcfit_reserve(h, max_tracks: int, max_hits: int = 0) -> None:
    _check(load().tpcfit_reserve(h, int(max_tracks), int(max_hits)), "tpcfit_reserve")


def tpcfit_fit(h, y, z, rowsec, offsets, seeds, params, cov, chi2, ndf, stream=None) -> None:
    """Enqueue the fit of all tracks (device tensors; see include/tpcfit.h).

    rowsec is an int16 tensor holding the uint16 bits row << 6 | sector."""
    import torch
    n = int(offsets.numel()) - 1
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"),
                 int(y.numel()))
    _check_sizes(n, y, z, rowsec, seeds, params, cov, chi2, ndf)
    st = load().tpcfit_fit(h, C.byref(hits), _dev(offsets, torch.int32, "offsets"), n, _dev(seeds, torch.float32, "seeds"),
                           _dev(params, torch.float32, "params"), _dev(cov, torch.float32, "cov"),
                           _dev(chi2, torch.float32, "chi2"), _dev(ndf, torch.int32, "ndf"), _stream(stream))
    _check(st, "tpcfit_fit")


def tpcfit_fit_frames(h, y, z, rowsec, offsets, frame_base, seeds, params, cov, chi2, ndf, frame_alignment=None,
                      frame_ready=None, wait_timeout_ns: int = 0, stream=None) -> None:
    """Enqueue the fit of several concatenated time frames (see include/tpcfit.h)."""
    import torch
    n = int(offsets.numel()) - 1
    nf = int(frame_base.numel()) - 1
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"),
                 int(y.numel()))
    fa = None if frame_alignment is None else _dev(frame_alignment, torch.float32, "frame_alignment")
    fr = None if frame_ready is None else _dev(frame_ready, torch.int32, "frame_ready")
    if fa is not None and frame_alignment.numel() != nf * 36 * 152 * 2:
        raise ValueError("frame_alignment must be [n_frames, 36, 152, 2]")
    if fr is not None and frame_ready.numel() != nf:
        raise ValueError("frame_ready must have one flag per frame")
    _check_sizes(n, y, z, rowsec, seeds, params, cov, chi2, ndf)
    st = load().tpcfit_fit_frames(h, C.byref(hits), _dev(offsets, torch.int32, "offsets"), n,
                                  _dev(frame_base, torch.int64, "frame_base"), nf, fa, fr, int(wait_timeout_ns),
                                  _dev(seeds, torch.float32, "seeds"), _dev(params, torch.float32, "params"),
                                  _dev(cov, torch.float32, "cov"), _dev(chi2, torch.float32, "chi2"),
                                  _dev(ndf, torch.int32, "ndf"), _stream(stream))
    _check(st, "tpcfit_fit_frames")


def tpcfit_set_backward_config(h, warps_per_block: int = 8) -> None:
    _check(load().tpcfit_set_backward_config(h, int(warps_per_block)), "tpcfit_set_backward_config")


def tpcfit_set_det_reduction(h, method: int = 0) -> None:
    _check(load().tpcfit_set_det_reduction(h, int(method)), "tpcfit_set_det_reduction")


def tpcfit_set_fit_form(h, form: int = 1) -> None:
    _check(load().tpcfit_set_fit_form(h, int(form)), "tpcfit_set_fit_form")


def tpcfit_set_backward_form(h, form: int = 1) -> None:
    _check(load().tpcfit_set_backward_form(h, int(form)), "tpcfit_set_backward_form")


def tpcfit_set_record(h, record: bool) -> None:
    _check(load().tpcfit_set_record(h, int(bool(record))), "tpcfit_set_record")


def tpcfit_fit_backward(h, y, z, rowsec, offsets, ndf, grad_chi2, grad_align, grad_seeds, grad_meas=None,
                        stream=None) -> None:
    """Enqueue the adjoint of the last recorded fit (device tensors; see include/tpcfit.h)."""
    import torch
    n = int(offsets.numel()) - 1
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"),
                 int(y.numel()))
    if grad_align.numel() != 36 * 152 * 2 or grad_seeds.numel() != 5 * n or grad_chi2.numel() != n:
        raise ValueError("gradient sizes do not match")
    if grad_meas is not None and grad_meas.numel() != 2 * int(y.numel()):
        raise ValueError("grad_meas must have two elements per cluster")
    _check_sizes(n, y, z, rowsec, ndf=ndf)
    gm = None if grad_meas is None else _dev(grad_meas, torch.float32, "grad_meas")
    st = load().tpcfit_fit_backward(h, C.byref(hits), _dev(offsets, torch.int32, "offsets"), n,
                                    _dev(ndf, torch.int32, "ndf"), _dev(grad_chi2, torch.float32, "grad_chi2"),
                                    _dev(grad_align, torch.float32, "grad_align"),
                                    _dev(grad_seeds, torch.float32, "grad_seeds"), gm, _stream(stream))
    _check(st, "tpcfit_fit_backward")


def tpcfit_smooth(h, y, z, rowsec, offsets, ndf, resid, rcov, chi2, stream=None) -> None:
    """Enqueue the two-filter smoother of the last recorded fit (device tensors; see include/tpcfit.h)."""
    import torch
    n = int(offsets.numel()) - 1
    H = int(y.numel())
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"), H)
    if resid.numel() != 2 * H or rcov.numel() != 3 * H or chi2.numel() != H:
        raise ValueError("smoother output sizes do not match the clusters")
    _check_sizes(n, y, z, rowsec, ndf=ndf)
    st = load().tpcfit_smooth(h, C.byref(hits), _dev(offsets, torch.int32, "offsets"), n, _dev(ndf, torch.int32, "ndf"),
                              _dev(resid, torch.float32, "resid"), _dev(rcov, torch.float32, "rcov"),
                              _dev(chi2, torch.float32, "chi2"), _stream(stream))
    _check(st, "tpcfit_smooth")


def tpcfit_reject_outliers(h, y, z, rowsec, offsets, chi2, chi2_cut, y_out, z_out, rowsec_out, offsets_out,
                           stream=None) -> None:
    """Enqueue the outlier rejection: the clusters with chi2 above chi2_cut dropped (device tensors; see
    include/tpcfit.h)."""
    import torch
    n = int(offsets.numel()) - 1
    H = int(y.numel())
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"), H)
    _check_sizes(n, y, z, rowsec)
    if chi2.numel() != H:
        raise ValueError("chi2 must have one value per cluster")
    if y_out.numel() < H or z_out.numel() < H or rowsec_out.numel() < H:
        raise ValueError("the outputs must hold as many clusters as the input")
    if offsets_out.numel() != n + 1:
        raise ValueError("offsets_out must have n_tracks + 1 elements")
    st = load().tpcfit_reject_outliers(h, C.byref(hits), _dev(offsets, torch.int32, "offsets"), n,
                                       _dev(chi2, torch.float32, "chi2"), C.c_float(float(chi2_cut)),
                                       _dev(y_out, torch.float32, "y_out"), _dev(z_out, torch.float32, "z_out"),
                                       _dev(rowsec_out, torch.int16, "rowsec_out"),
                                       _dev(offsets_out, torch.int32, "offsets_out"), _stream(stream))
    _check(st, "tpcfit_reject_outliers")


def tpcfit_smooth_states(h, y, z, rowsec, offsets, ndf, state, state_cov, stream=None) -> None:
    """Enqueue the smoothed states of the last recorded fit (device tensors; see include/tpcfit.h)."""
    import torch
    n = int(offsets.numel()) - 1
    H = int(y.numel())
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"), H)
    if state.numel() != 5 * H or state_cov.numel() != 15 * H:
        raise ValueError("smoothed-state output sizes do not match the clusters")
    _check_sizes(n, y, z, rowsec, ndf=ndf)
    st = load().tpcfit_smooth_states(h, C.byref(hits), _dev(offsets, torch.int32, "offsets"), n,
                                     _dev(ndf, torch.int32, "ndf"), _dev(state, torch.float32, "state"),
                                     _dev(state_cov, torch.float32, "state_cov"), _stream(stream))
    _check(st, "tpcfit_smooth_states")


def tpcfit_fit_host(h, y, z, rowsec, offsets, seeds, stream=None, out=None):
    """Fit from host arrays (numpy or pinned CPU tensors); returns host outputs."""
    def arr(a, dt):
        if hasattr(a, "numpy"):
            a = a.numpy()
        a = np.asarray(a)
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"host array must be contiguous {dt}")
        return a
    y = arr(y, np.float32); z = arr(z, np.float32); rowsec = arr(rowsec, np.uint16)
    offsets = arr(offsets, np.int32); seeds = arr(seeds, np.float32)
    n = offsets.shape[0] - 1
    if out is None:
        out = dict(params=np.empty((5, n), np.float32), cov=np.empty((15, n), np.float32),
                   chi2=np.empty(n, np.float32), ndf=np.empty(n, np.int32))
    st = load().tpcfit_fit_host(h, y.ctypes.data, z.ctypes.data, rowsec.ctypes.data, y.shape[0], offsets.ctypes.data,
                                n, seeds.ctypes.data, out["params"].ctypes.data, out["cov"].ctypes.data,
                                out["chi2"].ctypes.data, out["ndf"].ctypes.data, _stream(stream))
    _check(st, "tpcfit_fit_host")
    return out


def tpcfit_fit_adjoint_host(h, y, z, rowsec, offsets, seeds, grad_chi2, out=None, stream=None):
    """Enqueue fit + adjoint from host arrays (pinned CPU tensors for overlap);
    the host outputs are valid once `stream` has passed the call."""
    def arr(a, dt):
        if hasattr(a, "numpy"):
            a = a.numpy()
        a = np.asarray(a)
        if a.dtype != dt or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"host array must be contiguous {dt}")
        return a
    y = arr(y, np.float32); z = arr(z, np.float32); rowsec = arr(rowsec, np.uint16)
    offsets = arr(offsets, np.int32); seeds = arr(seeds, np.float32); grad_chi2 = arr(grad_chi2, np.float32)
    n = offsets.shape[0] - 1
    if out is None:
        out = dict(chi2=np.empty(n, np.float32), ndf=np.empty(n, np.int32),
                   grad_align=np.empty((36, 152, 2), np.float32), grad_seeds=np.empty((5, n), np.float32))
    o = {}
    for k, dt, size in (("chi2", np.float32, n), ("ndf", np.int32, n), ("grad_align", np.float32, 36 * 152 * 2),
                        ("grad_seeds", np.float32, 5 * n)):
        o[k] = arr(out[k], dt)
        if o[k].size != size:
            raise TypeError(f"{k}: {size} elements expected")
    st = load().tpcfit_fit_adjoint_host(h, y.ctypes.data, z.ctypes.data, rowsec.ctypes.data, y.shape[0],
                                        offsets.ctypes.data, n, seeds.ctypes.data, grad_chi2.ctypes.data,
                                        o["chi2"].ctypes.data, o["ndf"].ctypes.data, o["grad_align"].ctypes.data,
                                        o["grad_seeds"].ctypes.data, _stream(stream))
    _check(st, "tpcfit_fit_adjoint_host")
    return out


NOALLOC_MAX_TRACKS = 1 << 20


def tpcfit_fit_noalloc(geometry, bz, alignment, deterministic, y, z, rowsec, offsets, seeds, params, cov, chi2, ndf,
                       stream=None) -> None:
    """Fit without a handle and without device allocation (see include/tpcfit.h)."""
    import torch
    n = int(offsets.numel()) - 1
    rx = np.ascontiguousarray(geometry.row_x, dtype=np.float64)
    g = _Geometry(int(geometry.n_sectors), int(rx.shape[0]), rx.ctypes.data_as(C.POINTER(C.c_double)),
                  float(geometry.sector_width_deg), float(getattr(geometry, "z_max", 250.0)))
    hits = _Hits(_dev(y, torch.float32, "y"), _dev(z, torch.float32, "z"), _dev(rowsec, torch.int16, "rowsec"),
                 int(y.numel()))
    al = None if alignment is None else _dev(alignment, torch.float32, "alignment")
    if alignment is not None and alignment.numel() != 36 * 152 * 2:
        raise ValueError("alignment must have 36*152*2 elements")
    _check_sizes(n, y, z, rowsec, seeds, params, cov, chi2, ndf)
    st = load().tpcfit_fit_noalloc(C.byref(g), float(bz), al, int(bool(deterministic)), C.byref(hits),
                                   _dev(offsets, torch.int32, "offsets"), n, _dev(seeds, torch.float32, "seeds"),
                                   _dev(params, torch.float32, "params"), _dev(cov, torch.float32, "cov"),
                                   _dev(chi2, torch.float32, "chi2"), _dev(ndf, torch.int32, "ndf"), _stream(stream))
    _check(st, "tpcfit_fit_noalloc")


def tpcfit_get_status(h, stream=None):
    """Returns (status, err_code, err_track) and clears the device error word."""
    code = C.c_int32(0)
    trk = C.c_int64(-1)
    st = load().tpcfit_get_status(h, _stream(stream), C.byref(code), C.byref(trk))
    if st not in (OK, EDEVICE, ETIMEOUT):
        _check(st, "tpcfit_get_status")
    return st, int(code.value), int(trk.value)


# ------------------------------------------------------------------ conveniences
def frame_to_device(frame, device="cuda"):
    """Copy a synth.Frame's inputs to device tensors (one H2D copy per array)."""
    import torch
    return dict(
        y=torch.from_numpy(frame.y).to(device), z=torch.from_numpy(frame.z).to(device),
        rowsec=torch.from_numpy(frame.rowsec.view(np.int16)).to(device),
        offsets=torch.from_numpy(frame.offsets).to(device),
        seeds=torch.from_numpy(np.ascontiguousarray(frame.seeds)).to(device),
    )


def empty_outputs(n: int, device="cuda"):
    import torch
    return dict(params=torch.empty((5, n), dtype=torch.float32, device=device),
                cov=torch.empty((15, n), dtype=torch.float32, device=device),
                chi2=torch.empty(n, dtype=torch.float32, device=device),
                ndf=torch.empty(n, dtype=torch.int32, device=device))


class Fitter:
    """Owns a tpcfit handle."""

    def __init__(self, geometry, bz: float, deterministic: bool = False, rows_per_stage: int = 4,
                 warps_per_block: int = 24, sort_by_length: bool = True):
        self.h = tpcfit_create(geometry, bz)
        tpcfit_set_mode(self.h, deterministic)
        tpcfit_set_config(self.h, 1, rows_per_stage, warps_per_block, sort_by_length)

    def close(self):
        if self.h is not None:
            tpcfit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, deterministic: bool):
        tpcfit_set_mode(self.h, deterministic)

    def set_material(self, material=None):
        """material: object with x0_cm, dedx_gev_cm, mass_gev, row_cm (synth.Material), or None for none."""
        if material is None:
            tpcfit_set_material(self.h, 0.0)
        else:
            tpcfit_set_material(self.h, material.x0_cm, material.dedx_gev_cm, material.mass_gev, material.row_cm)

    def set_field(self, field=None):
        """field: object with c_r, c_z (synth.FieldMap), or None for the uniform field."""
        tpcfit_set_field_map(self.h, 0.0 if field is None else field.c_r, 0.0 if field is None else field.c_z)

    def set_rtc(self, enable: bool = True, cache_dir: str | None = None):
        tpcfit_set_rtc(self.h, enable, cache_dir)

    def set_config(self, lanes_per_track=1, rows_per_stage=4, warps_per_block=24, sort_by_length=True):
        tpcfit_set_config(self.h, lanes_per_track, rows_per_stage, warps_per_block, sort_by_length)

    def set_alignment(self, d=None, stream=None):
        tpcfit_set_alignment(self.h, d, stream)

    def fit(self, dev: dict, out: dict | None = None, stream=None) -> dict:
        n = int(dev["offsets"].numel()) - 1
        out = out or empty_outputs(n, dev["y"].device)
        tpcfit_fit(self.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], dev["seeds"], out["params"],
                   out["cov"], out["chi2"], out["ndf"], stream)
        return out

    def status(self, stream=None):
        return tpcfit_get_status(self.h, stream)

    def set_backward_config(self, warps_per_block: int = 8):
        tpcfit_set_backward_config(self.h, warps_per_block)

    def set_det_reduction(self, method: int = 0):
        """Deterministic alignment-gradient sums: 0 fixed-point (default), 1 key sort + fixed-order FP32."""
        tpcfit_set_det_reduction(self.h, method)

    def set_fit_form(self, form: int = 1):
        """Factor of the fast fit without material: 1 U-D (default), 0 square root."""
        tpcfit_set_fit_form(self.h, form)

    def set_backward_form(self, form: int = 1):
        """Factor of the fast backward's recomputation: 1 U-D (default), 0 square root."""
        tpcfit_set_backward_form(self.h, form)

    def set_record(self, record: bool):
        tpcfit_set_record(self.h, record)

    def smooth(self, dev: dict, out: dict, stream=None) -> dict:
        """Per-cluster leave-one-out residuals of the last recorded fit."""
        import torch
        H = int(dev["y"].numel())
        d = dev["y"].device
        res = dict(resid=torch.empty((H, 2), dtype=torch.float32, device=d),
                   rcov=torch.empty((H, 3), dtype=torch.float32, device=d),
                   chi2=torch.empty(H, dtype=torch.float32, device=d))
        tpcfit_smooth(self.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"], res["resid"], res["rcov"],
                      res["chi2"], stream)
        return res

    def reject_outliers(self, dev: dict, chi2, chi2_cut: float, stream=None) -> dict:
        """A copy of the device frame without the clusters whose leave-one-out chi2 (from smooth) is above
        chi2_cut; the seeds are kept.  Waits for the kept count to size the arrays."""
        import torch
        H = int(dev["y"].numel())
        n = int(dev["offsets"].numel()) - 1
        d = dev["y"].device
        y = torch.empty(H, dtype=torch.float32, device=d)
        z = torch.empty(H, dtype=torch.float32, device=d)
        rs = torch.empty(H, dtype=torch.int16, device=d)
        off = torch.empty(n + 1, dtype=torch.int32, device=d)
        tpcfit_reject_outliers(self.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], chi2, chi2_cut, y, z, rs, off,
                               stream)
        if stream is not None:
            stream.synchronize()
        kept = int(off[-1].item())
        return dict(y=y[:kept], z=z[:kept], rowsec=rs[:kept], offsets=off, seeds=dev["seeds"])

    def smooth_states(self, dev: dict, out: dict, stream=None) -> dict:
        """Smoothed state and covariance at every cluster of the last recorded fit."""
        import torch
        H = int(dev["y"].numel())
        d = dev["y"].device
        res = dict(state=torch.empty((H, 5), dtype=torch.float32, device=d),
                   state_cov=torch.empty((H, 15), dtype=torch.float32, device=d))
        tpcfit_smooth_states(self.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"], res["state"],
                             res["state_cov"], stream)
        return res

    def backward(self, dev: dict, out: dict, grad_chi2, grad_meas=None, stream=None):
        """Gradients of sum_i grad_chi2[i] chi2_i for the last recorded fit."""
        import torch
        n = int(dev["offsets"].numel()) - 1
        ga = torch.empty(36 * 152 * 2, dtype=torch.float32, device=dev["y"].device)
        gs = torch.empty((5, n), dtype=torch.float32, device=dev["y"].device)
        tpcfit_fit_backward(self.h, dev["y"], dev["z"], dev["rowsec"], dev["offsets"], out["ndf"], grad_chi2, ga, gs,
                            grad_meas, stream)
        return ga.view(36, 152, 2), gs
