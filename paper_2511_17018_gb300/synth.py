"""Seeded synthetic time frames for the TPC track fit.

This module only makes inputs: it simulates exact helices through a planar
pad-row TPC, drops and smears clusters, and derives three-point seeds.  It
holds none of the fit's arithmetic (no propagation recursion, no Kalman
update) so that both the CUDA library and the CPU oracle can be fed from it.

Workload definitions (geometry, momentum / angle distributions, cluster
smearing, hit dropping, alignment offsets) follow the benchmark configurations
of the track-fit workload; the paper itself only states that TPC track
reconstruction propagates tracks through the magnetic field (Sec. 4) and that
processing is organised in time frames (Sec. 1).

Geometry, everything in cm / GeV/c / T:
  * 36 sectors of 20 deg, 0-17 on the A side (z >= 0), 18-35 on the C side;
    sector s has its centre at alpha = ((s mod 18) + 0.5) * 20 deg.
  * 152 planar pad rows at local x = X_r = 85 + r * 160/151.
  * local frame of a sector: x along (cos a, sin a), y along (-sin a, cos a).

Hits are generated by intersecting the exact circle (centre / radius form, in
global coordinates) with each pad-row plane, which is a different computation
from the incremental local-frame propagation used by the fit.

Random numbers: numpy ``Generator(Philox)`` (counter-based, Salmon et al.,
SC'11) with one independent stream per purpose derived from the config seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: curvature per unit charge/pt and field: k = KAPPA_PER_TESLA * Bz * q/pt  [1/cm]
#: (c = 0.299792458 m/ns -> 0.00299792458 cm^-1 per GeV/c per T); the sign
#: makes a positive charge bend clockwise seen from +z for Bz > 0.
KAPPA_PER_TESLA = -0.00299792458

N_SECTORS = 36
N_ROWS = 152
ROWSEC_SHIFT = 6  # rowsec = row << 6 | sector
CHUNK = 131072    # tracks simulated per vectorised chunk (fixed: part of the stream layout)


@dataclass
class Geometry:
    row_x: np.ndarray = field(default_factory=lambda: 85.0 + np.arange(N_ROWS) * (160.0 / 151.0))
    n_sectors: int = N_SECTORS
    sector_width_deg: float = 20.0
    z_max: float = 250.0

    @property
    def n_rows(self) -> int:
        return int(self.row_x.shape[0])


def default_geometry() -> Geometry:
    return Geometry()


@dataclass
class Material:
    """A thin material layer at every pad row: radiation length (cm) and
    minimum-ionising energy loss (GeV/cm) of the material, its thickness at
    normal incidence (cm) and the particle's mass (a pion)."""
    x0_cm: float
    dedx_gev_cm: float
    mass_gev: float = 0.13957
    row_cm: float = 160.0 / 151.0


# TPC drift gas (Ne-CO2-N2 90-10-5 at 1 atm): X0 ~ 3.1e4 cm, dE/dx_mip ~ 1.6 MeV/m;
# one row pitch of gas per row.
TPC_GAS = Material(3.1e4, 1.6e-5)


def sector_alpha(sector, width_deg: float = 20.0):
    """Azimuth of a sector's centre in radians (A and C side share alphas)."""
    return ((np.asarray(sector) % 18) + 0.5) * (width_deg * math.pi / 180.0)


def _streams(seed: int, names):
    ss = np.random.SeedSequence(int(seed))
    kids = ss.spawn(len(names))
    return {n: np.random.Generator(np.random.Philox(k)) for n, k in zip(names, kids)}


@dataclass
class Frame:
    """One time frame in the layout the fit consumes (SoA, CSR by track)."""
    geometry: Geometry
    bz: float
    y: np.ndarray          # float32 [H] local y (cm), alignment offset + smearing included
    z: np.ndarray          # float32 [H] z (cm)
    rowsec: np.ndarray     # uint16  [H] row << 6 | sector
    offsets: np.ndarray    # int32   [N+1]
    seeds: np.ndarray      # float32 [5, N] (y, z, sin phi, tan lambda, q/pt) at the first hit
    truth: np.ndarray      # float64 [5, N] exact state at the first hit
    d_true: np.ndarray | None = None  # float32 [36, 152, 2] injected alignment offsets
    y64: np.ndarray | None = None     # float64 copies of the hits (noise-free closed-form tests)
    z64: np.ndarray | None = None
    seeds64: np.ndarray | None = None
    material: Material | None = None  # material the tracks crossed (for the fit's material correction)

    @property
    def n_tracks(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_hits(self) -> int:
        return int(self.y.shape[0])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def subset(self, idx) -> "Frame":
        """Frame restricted to tracks ``idx`` (order kept)."""
        idx = np.asarray(idx, dtype=np.int64)
        off = self.offsets.astype(np.int64)
        lens = off[idx + 1] - off[idx]
        new_off = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=new_off[1:])
        gather = np.concatenate([np.arange(off[i], off[i + 1]) for i in idx]) if idx.size else np.zeros(0, np.int64)
        return Frame(self.geometry, self.bz, self.y[gather].copy(), self.z[gather].copy(),
                     self.rowsec[gather].copy(), new_off.astype(np.int32),
                     self.seeds[:, idx].copy(), self.truth[:, idx].copy(), self.d_true,
                     None if self.y64 is None else self.y64[gather].copy(),
                     None if self.z64 is None else self.z64[gather].copy(),
                     None if self.seeds64 is None else self.seeds64[:, idx].copy(), self.material)


def _wrap(a):
    return (a + math.pi) % (2.0 * math.pi) - math.pi


def simulate(qpt, tanl, phi0, z0, geometry: Geometry, bz: float, *, drop_p: float = 0.0,
             cap=None, smear: float = 0.1, d_true=None, streams=None, min_hits: int = 10,
             curl_cut: float = 0.99):
    """Simulate tracks with explicit parameters; returns (Frame, accepted_mask).

    ``cap``: None (natural length) or int array of maximal hit counts per track.
    ``streams``: dict with 'drop' and 'smear' generators (needed if drop_p>0 or smear>0).
    Tracks with fewer than ``min_hits`` hits are rejected (mask False).
    """
    qpt = np.asarray(qpt, np.float64); tanl = np.asarray(tanl, np.float64)
    phi0 = np.asarray(phi0, np.float64); z0 = np.asarray(z0, np.float64)
    n = qpt.shape[0]
    rows_x = geometry.row_x
    width = geometry.sector_width_deg * math.pi / 180.0
    half_tan = math.tan(0.5 * width)
    kappa = KAPPA_PER_TESLA * bz
    k = kappa * qpt
    straight = k == 0.0
    ks = np.where(straight, 1.0, k)
    inv_k = 1.0 / ks
    # circle centre (centre = start + (1/k) * left normal); unused for straight tracks
    xc = -np.sin(phi0) * inv_k
    yc = np.cos(phi0) * inv_k

    R = geometry.n_rows
    hy = np.zeros((R, n)); hz = np.zeros((R, n)); hsec = np.zeros((R, n), np.int16)
    keep = np.zeros((R, n), bool)
    truth_first = np.full((5, n), np.nan)
    have_first = np.zeros(n, bool)
    alive = np.ones(n, bool)
    l_prev = np.zeros(n)
    cand = np.floor(np.mod(phi0, 2 * math.pi) / width).astype(np.int64) % 18

    def intersect(sec18, xr):
        a = (sec18 + 0.5) * width
        ca, sa = np.cos(a), np.sin(a)
        # circle: sin(phi - a) = k (X_r - C.n); straight: phi stays phi0
        u_c = k * (xr - (xc * ca + yc * sa))
        u_s = np.sin(phi0 - a)
        u = np.where(straight, u_s, u_c)
        ok = np.abs(u) < curl_cut
        uu = np.clip(u, -0.999999, 0.999999)
        cphi = np.sqrt(1.0 - uu * uu)
        y_c = (-xc * sa + yc * ca) - cphi * inv_k
        # straight line from the origin: path l = X_r / cos(phi0 - a)
        cs = np.cos(phi0 - a)
        l_s = xr / np.where(cs > 1e-9, cs, 1e-9)
        y_s = l_s * u_s
        y = np.where(straight, y_s, y_c)
        theta = _wrap(a + np.arcsin(uu) - phi0)
        l_c = theta * inv_k
        l = np.where(straight, l_s, l_c)
        ok &= np.where(straight, cs > 1e-9, True)
        return u, y, l, ok

    for r in range(R):
        if not alive.any():
            break
        xr = rows_x[r]
        u, y, l, ok = intersect(cand, xr)
        out = np.abs(y) > xr * half_tan
        if out.any():
            nb = (cand + np.where(y > 0, 1, -1)) % 18
            u2, y2, l2, ok2 = intersect(nb, xr)
            u = np.where(out, u2, u); y = np.where(out, y2, y)
            l = np.where(out, l2, l); ok = np.where(out, ok2, ok)
            cand = np.where(out, nb, cand)
        zz = z0 + tanl * l
        ok &= np.abs(y) <= xr * half_tan
        ok &= (l > l_prev) & (np.abs(zz) <= geometry.z_max)
        alive &= ok
        l_prev = np.where(alive, l, l_prev)
        side = np.where(zz < 0.0, 18, 0)
        sec = cand + side
        if drop_p > 0.0:
            dropped = streams["drop"].random(n) < drop_p
        else:
            dropped = np.zeros(n, bool)
        kept = alive & ~dropped
        hy[r] = y; hz[r] = zz; hsec[r] = sec; keep[r] = kept
        newf = kept & ~have_first
        if newf.any():
            truth_first[0, newf] = y[newf]
            truth_first[1, newf] = zz[newf]
            truth_first[2, newf] = u[newf]
            truth_first[3, newf] = tanl[newf]
            truth_first[4, newf] = qpt[newf]
            have_first |= newf

    counts = keep.sum(axis=0)
    if cap is not None:
        cap = np.asarray(cap, np.int64)
        csum = np.cumsum(keep, axis=0)
        keep &= csum <= cap[None, :]
        counts = keep.sum(axis=0)
    accepted = counts >= min_hits
    keep &= accepted[None, :]
    counts = np.where(accepted, counts, 0)

    # CSR, track-major, rows ascending within a track
    kt = keep.T
    tr_idx, row_idx = np.nonzero(kt)
    y_h = hy.T[tr_idx, row_idx]
    z_h = hz.T[tr_idx, row_idx]
    s_h = hsec.T[tr_idx, row_idx].astype(np.int64)
    if d_true is not None:
        y_h = y_h + d_true[s_h, row_idx, 0].astype(np.float64)
        z_h = z_h + d_true[s_h, row_idx, 1].astype(np.float64)
    if smear > 0.0:
        y_h = y_h + streams["smear"].normal(0.0, smear, y_h.shape[0])
        z_h = z_h + streams["smear"].normal(0.0, smear, z_h.shape[0])
    rowsec = ((row_idx.astype(np.int64) << ROWSEC_SHIFT) | s_h).astype(np.uint16)
    acc_idx = np.nonzero(accepted)[0]
    off = np.zeros(acc_idx.shape[0] + 1, np.int64)
    np.cumsum(counts[acc_idx], out=off[1:])
    fr = Frame(geometry, bz, y_h.astype(np.float32), z_h.astype(np.float32), rowsec,
               off.astype(np.int32), np.zeros((5, acc_idx.shape[0]), np.float32),
               truth_first[:, acc_idx], None if d_true is None else np.asarray(d_true, np.float32))
    fr.y64, fr.z64 = y_h, z_h
    fr.seeds64 = three_point_seeds(fr, as_f64=True)
    fr.seeds = fr.seeds64.astype(np.float32)
    return fr, accepted


def global_xy(frame: Frame, idx, as_f64: bool = False):
    """Global (X, Y) of hits ``idx`` (float64)."""
    rs = frame.rowsec[idx].astype(np.int64)
    row = rs >> ROWSEC_SHIFT
    sec = rs & ((1 << ROWSEC_SHIFT) - 1)
    xr = frame.geometry.row_x[row]
    a = sector_alpha(sec, frame.geometry.sector_width_deg)
    y = (frame.y64 if as_f64 and frame.y64 is not None else frame.y)[idx].astype(np.float64)
    return xr * np.cos(a) - y * np.sin(a), xr * np.sin(a) + y * np.cos(a), a


def three_point_seeds(frame: Frame, as_f64: bool = False) -> np.ndarray:
    """Seed (y, z, sin phi, tan lambda, q/pt) at the first hit from a circle
    through the first, middle and last hit (Menger curvature), FP64 -> FP32."""
    off = frame.offsets.astype(np.int64)
    n = off.shape[0] - 1
    if n == 0:
        return np.zeros((5, 0), np.float32)
    first = off[:-1]; last = off[1:] - 1
    mid = first + (last - first) // 2
    x0, y0, a0 = global_xy(frame, first, as_f64)
    x1, y1, _ = global_xy(frame, mid, as_f64)
    x2, y2, _ = global_xy(frame, last, as_f64)
    d01x, d01y = x1 - x0, y1 - y0
    d12x, d12y = x2 - x1, y2 - y1
    d02x, d02y = x2 - x0, y2 - y0
    l01 = np.hypot(d01x, d01y); l12 = np.hypot(d12x, d12y); l02 = np.hypot(d02x, d02y)
    cross = d01x * d12y - d01y * d12x
    denom = l01 * l12 * l02
    k = np.where(denom > 0, 2.0 * cross / np.where(denom > 0, denom, 1.0), 0.0)
    kappa = KAPPA_PER_TESLA * frame.bz
    small = np.abs(k) < 1e-12
    sgn = np.where(cross >= 0, 1.0, -1.0)
    k = np.where(small, sgn * 1e-4 * abs(kappa), k)
    qpt = k / kappa
    beta = np.arctan2(d01y, d01x)
    phi0 = beta - np.arcsin(np.clip(k * l01 * 0.5, -1.0, 1.0))
    snp = np.sin(phi0 - a0)
    ak = np.abs(k)
    arc02 = 2.0 * np.arcsin(np.clip(ak * l02 * 0.5, 0.0, 1.0)) / ak
    zz = frame.z64 if as_f64 and frame.z64 is not None else frame.z
    yy = frame.y64 if as_f64 and frame.y64 is not None else frame.y
    z0 = zz[first].astype(np.float64)
    z2 = zz[last].astype(np.float64)
    tanl = (z2 - z0) / np.where(arc02 > 0, arc02, 1.0)
    seeds = np.stack([yy[first].astype(np.float64), z0, snp, tanl, qpt])
    return seeds if as_f64 else seeds.astype(np.float32)


def draw_track_params(rng, n, *, pt_min=0.2, pt_max=10.0, eta_max=0.9, z0_sigma=5.0):
    q = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    pt = np.exp(rng.uniform(math.log(pt_min), math.log(pt_max), n))
    eta = rng.uniform(-eta_max, eta_max, n)
    phi0 = rng.uniform(0.0, 2.0 * math.pi, n)
    z0 = rng.normal(0.0, z0_sigma, n)
    return q / pt, np.sinh(eta), phi0, z0


def generate(n_tracks: int, seed: int, *, drop_p: float = 0.0, cap_lengths: bool = False,
             smear: float = 0.1, d_true=None, bz: float = 0.5, geometry: Geometry | None = None,
             pt_min: float = 0.2, pt_max: float = 10.0, min_hits: int = 10) -> Frame:
    """Draw ``n_tracks`` accepted tracks (rejecting those with < ``min_hits`` hits)."""
    geometry = geometry or default_geometry()
    st = _streams(seed, ["params", "drop", "cap", "smear"])
    parts = []
    got = 0
    while got < n_tracks:
        m = min(CHUNK, int((n_tracks - got) * 1.05) + 64)
        qpt, tanl, phi0, z0 = draw_track_params(st["params"], m, pt_min=pt_min, pt_max=pt_max)
        cap = st["cap"].integers(10, N_ROWS + 1, m) if cap_lengths else None
        fr, _ = simulate(qpt, tanl, phi0, z0, geometry, bz, drop_p=drop_p, cap=cap, smear=smear,
                         d_true=d_true, streams=st, min_hits=min_hits)
        take = min(fr.n_tracks, n_tracks - got)
        parts.append(fr.subset(np.arange(take)) if take < fr.n_tracks else fr)
        got += take
    return concat(parts)


def concat(frames) -> Frame:
    """Concatenate frames (tracks appended in order)."""
    f0 = frames[0]
    if len(frames) == 1:
        return f0
    offs = [f0.offsets.astype(np.int64)]
    base = offs[0][-1]
    for f in frames[1:]:
        offs.append(f.offsets[1:].astype(np.int64) + base)
        base += f.offsets[-1]
    off = np.concatenate(offs)
    assert off[-1] < 2**31, "track offsets exceed int32"
    have64 = all(f.y64 is not None for f in frames)
    return Frame(f0.geometry, f0.bz, np.concatenate([f.y for f in frames]),
                 np.concatenate([f.z for f in frames]), np.concatenate([f.rowsec for f in frames]),
                 off.astype(np.int32), np.concatenate([f.seeds for f in frames], axis=1),
                 np.concatenate([f.truth for f in frames], axis=1), f0.d_true,
                 np.concatenate([f.y64 for f in frames]) if have64 else None,
                 np.concatenate([f.z64 for f in frames]) if have64 else None,
                 np.concatenate([f.seeds64 for f in frames], axis=1) if have64 else None)


def alignment_offsets(seed: int, sigma: float = 0.05) -> np.ndarray:
    """Injected per-(sector, row) offsets (dy, dz) ~ N(0, sigma), float32 [36, 152, 2]."""
    rng = _streams(seed, ["align"])["align"]
    return rng.normal(0.0, sigma, (N_SECTORS, N_ROWS, 2)).astype(np.float32)


# --- the benchmark workloads -----------------------------------------------------

def plain_frame(n_tracks: int = 1000) -> Frame:
    """Plain-fit frame (1,000 tracks by default): natural lengths, one cluster
    per crossed row, sigma 0.1 cm, no drops."""
    return generate(n_tracks, 1)


def time_frame(n_tracks: int = 400_000) -> Frame:
    """Time-frame-sized batch (400,000 tracks by default): 5% of hits dropped,
    lengths capped at U{10..152}."""
    return generate(n_tracks, 2, drop_p=0.05, cap_lengths=True)


def adjoint_frame(n_tracks: int = 100_000) -> Frame:
    """Adjoint workload (100,000 tracks by default): injected offsets
    N(0, 0.05 cm) on all 36 x 152 x 2 keys."""
    d = alignment_offsets(3)
    return generate(n_tracks, 3, drop_p=0.05, cap_lengths=True, d_true=d)


def alignment_frame(n_tracks: int = 2_000_000) -> Frame:
    """Alignment-recovery workload (2,000,000 tracks by default): as the
    adjoint workload, more tracks."""
    d = alignment_offsets(5)
    return generate(n_tracks, 5, drop_p=0.05, cap_lengths=True, d_true=d)


def frame_sizes_batched(seed: int = 4, n_frames: int = 256, lo: int = 1000, hi: int = 200_000):
    """Track counts of the batched workload: log-uniform on [lo, hi]."""
    rng = _streams(seed, ["frames"])["frames"]
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n_frames)).astype(np.int64)


def batched_frames(pool_tracks: int = 1_000_000, n_frames: int = 256, seed: int = 4):
    """Batched uneven frames: ``n_frames`` frames with track counts log-uniform
    on [1e3, 2e5] (256 frames: about 9.6M tracks on average, 8.99M for seed 4).
    Tracks are drawn (seeded, with replacement) from a simulated pool of
    ``pool_tracks`` distinct tracks with the time-frame batch's distributions;
    returns (pool Frame, per-frame track index arrays)."""
    pool = generate(pool_tracks, seed, drop_p=0.05, cap_lengths=True)
    sizes = frame_sizes_batched(seed, n_frames)
    rng = _streams(seed + 1000, ["pick"])["pick"]
    picks = [rng.integers(0, pool.n_tracks, int(s)) for s in sizes]
    return pool, picks


def simulate_material(qpt, tanl, phi0, z0, geometry: Geometry, bz: float, material: Material, *, rng=None,
                      scatter: bool = True, eloss: bool = True, smear: float = 0.1, sector: int = 0):
    """Tracks through thin material layers at the pad rows, row by row, in the
    local frame of one sector (the caller picks tracks that stay in it).
    Between two rows the track follows the exact circle through its current
    point and direction (centre form, as ``simulate``).  At a row it crosses the
    layer over l = d sqrt(1 + t^2) / cos(phi): the energy drops by
    dE = dEdx l / beta^2 and the direction turns by two independent plane
    angles drawn from N(0, theta0), theta0^2 = 0.0136^2 l / X0 / (beta p)^2
    (Highland without its logarithmic term; phi by th1 / cos(lambda), lambda by
    th2), before the cluster is recorded: the state at a cluster is the one the
    track leaves it with.  Tracks that leave the sector, curl or stop are cut
    there.  Returns a Frame (material attached) with truth at the first
    cluster."""
    rng = np.random.default_rng(0) if rng is None else rng
    kappa = KAPPA_PER_TESLA * bz
    width = geometry.sector_width_deg * math.pi / 180.0
    half_tan = math.tan(0.5 * width)
    alpha = (sector % 18 + 0.5) * width
    m2 = material.mass_gev ** 2
    ys, zs, secs, rows, offs, truth = [], [], [], [], [0], []
    for i in range(len(qpt)):
        q = float(qpt[i]); t = float(tanl[i]); phi = float(phi0[i]) - alpha
        # start: the vertex (0, 0, z0) in global = local (0, 0) for the sector frame
        x, y, z = 0.0, 0.0, float(z0[i])
        hy, hz, hr = [], [], []
        first = None
        for r in range(geometry.n_rows):
            X = float(geometry.row_x[r])
            k = kappa * q
            if abs(k) < 1e-15:
                if math.cos(phi) <= 1e-9:
                    break
                dxl = X - x
                y2 = y + dxl * math.tan(phi)
                lt = dxl / math.cos(phi)
                phi2 = phi
            else:
                xc = x - math.sin(phi) / k
                yc = y + math.cos(phi) / k
                u = k * (X - xc)
                if abs(u) >= 0.99:
                    break
                phi2 = math.asin(u)
                y2 = yc - math.cos(phi2) / k
                lt = (phi2 - phi) / k
            if lt <= 0.0 or abs(y2) > X * half_tan:
                break
            z2 = z + t * lt
            if abs(z2) > geometry.z_max:
                break
            x, y, z, phi = X, y2, z2, phi2
            # the row's material layer, crossed on arrival; the state recorded
            # at the row is the one the track leaves it with
            ell = material.row_cm * math.sqrt(1.0 + t * t) / math.cos(phi)
            p2 = (1.0 + t * t) / (q * q)
            e2 = p2 + m2
            if eloss:
                en = math.sqrt(e2) - material.dedx_gev_cm * ell * e2 / p2
                pn2 = en * en - m2
                if pn2 <= 0.0:
                    break
                q = math.copysign(math.sqrt((1.0 + t * t) / pn2), q)
            if scatter:
                th0 = math.sqrt(0.0136 ** 2 * ell / material.x0_cm * e2 / (p2 * p2))
                th1, th2 = rng.normal(0.0, th0, 2)
                lam = math.atan(t)
                phi += th1 / math.cos(lam)
                tn = math.tan(lam + th2)
                q = q * math.sqrt((1.0 + tn * tn) / (1.0 + t * t))  # |p| kept: pt follows the new dip
                t = tn
            hy.append(y); hz.append(z); hr.append(r)
            if first is None:
                first = (y, z, math.sin(phi), t, q)
        if len(hy) < 10:
            continue
        ys += hy; zs += hz; rows += hr; secs += [sector + (18 if zz < 0 else 0) for zz in hz]
        offs.append(offs[-1] + len(hy))
        truth.append(first)
    y64 = np.asarray(ys); z64 = np.asarray(zs)
    if smear > 0.0:
        y64 = y64 + rng.normal(0.0, smear, y64.shape[0])
        z64 = z64 + rng.normal(0.0, smear, z64.shape[0])
    rowsec = ((np.asarray(rows, np.int64) << ROWSEC_SHIFT) | np.asarray(secs, np.int64)).astype(np.uint16)
    n = len(truth)
    fr = Frame(geometry, bz, y64.astype(np.float32), z64.astype(np.float32), rowsec,
               np.asarray(offs, np.int32), np.zeros((5, n), np.float32), np.asarray(truth, np.float64).T.reshape(5, n),
               None, y64, z64, None, material)
    fr.seeds64 = three_point_seeds(fr, as_f64=True)
    fr.seeds = fr.seeds64.astype(np.float32)
    return fr


@dataclass
class FieldMap:
    """Analytic map Bz(r, z) = Bz0 (1 + c_r (r / 250 cm)^2 + c_z (z / 250 cm)^2)."""
    c_r: float
    c_z: float


def simulate_field(qpt, tanl, phi0, z0, geometry: Geometry, bz: float, field: FieldMap, *, rng=None,
                   smear: float = 0.1, step_cm: float = 0.2, sector: int = 0):
    """Tracks in a non-uniform Bz field, by Runge-Kutta (4th order) integration
    of the direction along the path, d u / ds = 0.00299792458 (q / p) u x B,
    in the local frame of one sector (the caller picks tracks that stay in it).
    A row plane crossed inside a step is reached by a last step of the exact
    remaining length, so hits sit on the planes.  Returns a Frame (field
    attached) with truth (y, z, sin phi, tan lambda, q/pt) at the first cluster;
    without material pt and tan lambda stay constant along the track."""
    rng = np.random.default_rng(0) if rng is None else rng
    width = geometry.sector_width_deg * math.pi / 180.0
    half_tan = math.tan(0.5 * width)
    alpha = (sector % 18 + 0.5) * width
    c = 0.00299792458
    fr2, fz2 = field.c_r / 250.0 ** 2, field.c_z / 250.0 ** 2

    def deriv(st, qp):
        x, y, z, ux, uy, uz = st
        b = bz * (1.0 + fr2 * (x * x + y * y) + fz2 * z * z)
        a = c * qp * b
        return np.array([ux, uy, uz, a * uy, -a * ux, 0.0])

    def rk4(st, h, qp):
        k1 = deriv(st, qp)
        k2 = deriv(st + 0.5 * h * k1, qp)
        k3 = deriv(st + 0.5 * h * k2, qp)
        k4 = deriv(st + h * k3, qp)
        return st + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)

    ys, zs, rows, secs, offs, truth = [], [], [], [], [0], []
    for i in range(len(qpt)):
        q = float(qpt[i]); t = float(tanl[i]); phi = float(phi0[i]) - alpha
        cl = 1.0 / math.sqrt(1.0 + t * t)
        p = 1.0 / (abs(q) * cl)                 # |p| = pt / cos(lambda)
        qp = math.copysign(1.0 / p, q)
        st = np.array([0.0, 0.0, float(z0[i]), math.cos(phi) * cl, math.sin(phi) * cl, t * cl])
        hy, hz, hr = [], [], []
        first = None
        r = 0
        for _ in range(200000):
            if r >= geometry.n_rows:
                break
            X = float(geometry.row_x[r])
            nxt = rk4(st, step_cm, qp)
            if nxt[0] < X:
                st = nxt
                if st[3] <= 0.0:
                    break
                continue
            # the plane is inside this step: shrink the step to reach it (two refinements)
            h = step_cm * (X - st[0]) / (nxt[0] - st[0])
            for _ in range(3):
                trial = rk4(st, h, qp)
                h = h + (X - trial[0]) / max(trial[3], 1e-9)
            st = rk4(st, h, qp)
            st[0] = X
            if abs(st[1]) > X * half_tan or abs(st[2]) > geometry.z_max:
                break
            hy.append(st[1]); hz.append(st[2]); hr.append(r)
            if first is None:
                upt = math.hypot(st[3], st[4])
                first = (st[1], st[2], st[4] / upt, st[5] / upt, qp / upt)
            r += 1
        if len(hy) < 10:
            continue
        ys += hy; zs += hz; rows += hr; secs += [sector + (18 if zz < 0 else 0) for zz in hz]
        offs.append(offs[-1] + len(hy))
        truth.append(first)
    y64 = np.asarray(ys); z64 = np.asarray(zs)
    if smear > 0.0:
        y64 = y64 + rng.normal(0.0, smear, y64.shape[0])
        z64 = z64 + rng.normal(0.0, smear, z64.shape[0])
    rowsec = ((np.asarray(rows, np.int64) << ROWSEC_SHIFT) | np.asarray(secs, np.int64)).astype(np.uint16)
    n = len(truth)
    fr = Frame(geometry, bz, y64.astype(np.float32), z64.astype(np.float32), rowsec, np.asarray(offs, np.int32),
               np.zeros((5, n), np.float32), np.asarray(truth, np.float64).T.reshape(5, n), None, y64, z64, None)
    fr.field = field
    fr.seeds64 = three_point_seeds(fr, as_f64=True)
    fr.seeds = fr.seeds64.astype(np.float32)
    return fr
