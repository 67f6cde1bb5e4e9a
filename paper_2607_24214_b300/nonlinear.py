"""The pair-beam instability past its linear stage at full scale, and the beam-trapping
saturation estimates of the paper's blazar discussion (the paragraphs after Eqs. 6-7).

Units throughout: lengths k_p^-1, times omega_p^-1, momenta m c, fields m c omega_p / e,
densities n_p, so that alpha = n_b / n_p is one species' beam density.

`run` advances one handle (normally the 512^2, 2048-slice pair beam) and records, every few
beam steps, the transverse rms of each field per xi segment of width 2 k_p^-1 (the averaging
of Fig. 2), the field energies, and the beam's rms momentum spreads per segment.  `summary`
reads the record at xi = 2 (filamentation, near the front) and xi = 20 (oblique two-stream,
downstream): the growth of the transverse magnetic and electric rms fields against the
asymptotic exponents of Eqs. 7 and 6, the growth rate at the end of the run against the
spatiotemporal rate, and the fractional field energy and transverse momentum spread beside
the trapping estimates.

    python -m paper_2607_24214_b300.nonlinear --steps 400 --every 6 --out run.npz
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import config

# ------------------------------------------------------------------ closed forms
SQ3 = math.sqrt(3.0)


def temporal_rate(k: float, species) -> float:
    """Gamma of Eq. 5 at transverse wavenumber k: (sum_s omega_bs^2 k^2/(k^2 + 1))^1/2 with
    omega_bs^2 = Z_s^2 alpha_s / (gamma_b M_s)."""
    wb2 = sum(s.Z ** 2 * s.alpha / (s.gamma_b * s.M) for s in species)
    return math.sqrt(wb2 * k * k / (k * k + 1.0))


def exponent_front(gamma_tau, xi):
    """Growth exponent near the front (Eq. 7): 2 (Gamma tau xi)^1/2 (1 - xi/(4 Gamma tau))."""
    gt = np.asarray(gamma_tau, dtype=float)
    return 2.0 * np.sqrt(gt * xi) * (1.0 - xi / (4.0 * gt))


def exponent_rear(gamma_tau, xi):
    """Growth exponent downstream (Eq. 6): (3 sqrt 3 / 4) (Gamma tau)^2/3 xi^1/3."""
    gt = np.asarray(gamma_tau, dtype=float)
    return 0.75 * SQ3 * gt ** (2.0 / 3.0) * xi ** (1.0 / 3.0)


def rate_front(Gamma, xi, tau):
    """Spatiotemporal filamentation rate d ln|Psi| / d tau near the front: (Gamma xi/tau)^1/2."""
    return np.sqrt(Gamma * xi / np.asarray(tau, dtype=float))


def rate_rear(Gamma, xi, tau):
    """Spatiotemporal oblique two-stream rate downstream: (sqrt 3/2) Gamma^2/3 (xi/tau)^1/3."""
    return 0.5 * SQ3 * Gamma ** (2.0 / 3.0) * (xi / np.asarray(tau, dtype=float)) ** (1.0 / 3.0)


def fractional_energy(mean_square, alpha, gamma_b):
    """A field's energy density over four times one species' beam kinetic energy density,
    F^2 / (4 n_b gamma_b m c^2), which in these units is <F^2> / (4 alpha gamma_b)."""
    return np.asarray(mean_square, dtype=float) / (4.0 * alpha * gamma_b)


def eps_bz_sat(xi, tau_sat, ky=1.0):
    """Magnetic energy fraction at trapping saturation near the front: the bounce frequency
    (k_y B_z / gamma_b)^1/2 equal to the spatiotemporal rate gives (xi / tau_sat)^2 / (4 k_y^2)."""
    return (xi / tau_sat) ** 2 / (4.0 * ky * ky)


def eps_ey_sat(xi, tau_sat, alpha, gamma_b, ky=1.0):
    """Electric energy fraction at trapping saturation downstream:
    9/(64 k_y^2) (alpha/gamma_b)^1/3 (xi/tau_sat)^4/3."""
    return 9.0 / (64.0 * ky * ky) * (alpha / gamma_b) ** (1.0 / 3.0) * (xi / tau_sat) ** (4.0 / 3.0)


def dpy_front(Gamma, xi, tau_sat, gamma_b, ky=1.0):
    """Transverse momentum spread at saturation near the front: gamma_b Gamma^st / k_y."""
    return gamma_b * rate_front(Gamma, xi, tau_sat) / ky


def dpy_rear(Gamma, xi, tau_sat, gamma_b, ky=1.0):
    """Transverse momentum spread at saturation downstream: gamma_b Gamma^st / k_y."""
    return gamma_b * rate_rear(Gamma, xi, tau_sat) / ky


def ex_wake_amplitude(rho_b, length, width):
    """Longitudinal wake field behind a current filament (the paper's E_x, E_z here), from the
    blazar paragraph: |2 rho_b sin(l/2)| (1 - exp(-w)), rho_b the filament's charge density,
    l its length, w its transverse size.  The first factor is the linear plasma wake behind a
    flat-top bunch of length l (Eq. 1 for a step-on, step-off source); the second is the
    on-axis share of a transversely finite source under the screened operator of Eq. 2, whose
    Green's function in the paper's 2D geometry is exp(-|y|)/2: a slab |y| < w keeps
    1 - exp(-w) of the field of an unbounded one.  w is read as the half-width."""
    return np.abs(2.0 * np.asarray(rho_b, dtype=float) * np.sin(0.5 * np.asarray(length))) \
        * (1.0 - np.exp(-np.asarray(width, dtype=float)))


def dpx_spread(rho_b, tau):
    """Longitudinal momentum spread the filament wakes build up in the beam, Delta p_x ~
    |rho_b| tau (blazar paragraph; Delta p_x is u_z here)."""
    return np.abs(np.asarray(rho_b, dtype=float)) * np.asarray(tau, dtype=float)


def filament_sizes(rho, dx, dy, dxi):
    """Sizes of the current filaments in a block of beam charge density rho[k, iy, ix] (xi
    slices k dxi of the front region, periodic transverse grid), from the fluctuation
    d = rho - <rho>_(x, y) of each slice and its transverse power spectrum P(k) summed over
    the slices, averaged over shells of |k| one box wavenumber wide:
      spacing: 2 pi / |k| at the peak of P (the distance between neighbouring filaments);
      width: the filament's full width at half maximum 2 sqrt(2 ln 2) s, with s from the
        roll-off of P above its peak: a Gaussian filament of standard deviation s has
        |F(k)|^2 ~ exp(-k^2 s^2), and the filaments' positions only multiply that by a
        structure factor that tends to 1 at large k (fitted where P is above 1e-4 of its
        peak, up to the grid's Nyquist wavenumber);
      length: twice the xi lag at which the longitudinal autocorrelation
        sum_k d_k d_(k+m) / sum_k d_k^2 (over the grid) first falls below 1/2; for filaments of
        a flat-top profile of length l it falls as 1 - m dxi / l, to 1/2 at l/2.
    Returns dict(spacing, width, length, rho_rms) with rho_rms the rms of d."""
    rho = np.asarray(rho, dtype=float)
    nk, ny, nx = rho.shape
    d = rho - rho.mean(axis=(1, 2), keepdims=True)
    P = (np.abs(np.fft.fft2(d, axes=(1, 2))) ** 2).sum(axis=0)
    P[0, 0] = 0.0
    KX, KY = np.meshgrid(2 * np.pi * np.fft.fftfreq(nx, d=dx), 2 * np.pi * np.fft.fftfreq(ny, d=dy))
    dk = 2 * np.pi / max(nx * dx, ny * dy)
    shell = np.rint(np.hypot(KX, KY) / dk).astype(int)
    cnt = np.bincount(shell.ravel())
    avg = np.bincount(shell.ravel(), weights=P.ravel()) / np.maximum(cnt, 1)
    kp = int(np.argmax(avg[1:])) + 1
    spacing = 2 * np.pi / (kp * dk)
    kk = np.arange(avg.size) * dk
    sel = ((np.arange(avg.size) >= kp) & (avg > 1e-4 * avg[kp]) &
           (kk <= np.pi / max(dx, dy)))
    slope = np.polyfit(kk[sel] ** 2, np.log(avg[sel]), 1)[0] if sel.sum() >= 2 else 0.0
    sd = math.sqrt(max(-slope, 0.0))

    def half_crossing(r, h):
        """Lag (in units of h) where the sequence r (r[0] = 1) first falls below 1/2."""
        for i in range(1, r.size):
            if r[i] < 0.5:
                return (i - 1 + (r[i - 1] - 0.5) / (r[i - 1] - r[i])) * h
        return r.size * h

    s2 = np.sum(d * d)
    r = np.array([1.0] + [np.sum(d[:-m] * d[m:]) / s2 for m in range(1, nk)])
    return {"spacing": float(spacing), "width": float(2.0 * math.sqrt(2.0 * math.log(2.0)) * sd),
            "length": float(2 * half_crossing(r, dxi)), "rho_rms": float(np.sqrt(s2 / d.size))}


# ------------------------------------------------------------------ the run
FIELD_NAMES = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")  # order of the rms columns of qsa_diag


def run(p: config.Params, steps: int, every: int, seg_width: float = 2.0, log=None,
        read=None, read_every: int = 0) -> dict:
    """Advance a fresh handle of `p` by `steps` beam steps, `every` at a time (one pipelined
    call each), and record after each call the diagnostics of its last sweep.  That sweep saw
    the beam after (sweeps - 1) pushes, so its time is tau = (sweeps - 1) dt.  With `read`
    (a function of the handle, p and the diagnostics), its result is recorded after every
    read_every-th call and after the last, under "reads" with their times "read_tau"."""
    from .qsa import QSA
    q = QSA(p)
    rec = {k: [] for k in ("tau", "rms_seg", "energy", "beam_rms_seg", "beam_lost", "ms")}
    reads, read_tau, calls = [], [], 0
    nseg = int(math.ceil(p.Lxi / seg_width - 1e-12))
    cell_seg = np.minimum((np.arange(p.nxi) * p.dxi / seg_width + 1e-12).astype(int), nseg - 1)
    done = 0
    while done < steps:
        n = min(every, steps - done)
        t = time.perf_counter()
        q.advance(n)
        d = q.diagnostics(seg_width)
        ms = 1e3 * (time.perf_counter() - t)
        done += n
        # weighted rms momentum spread per segment: sum w u^2 / sum w - (sum w u / sum w)^2
        m = d["beam_moments"]                                   # [species, cell, 7]
        bseg = np.zeros((m.shape[0], nseg, 3))
        for s in range(nseg):
            ms_ = m[:, cell_seg == s, :].sum(axis=1)            # [species, 7]
            w = np.maximum(ms_[:, :1], 1e-300)
            mean = ms_[:, 1:4] / w
            bseg[:, s] = np.sqrt(np.maximum(ms_[:, 4:7] / w - mean ** 2, 0.0))
        rec["tau"].append((d["sweeps"] - 1) * p.dt)
        rec["rms_seg"].append(d["rms_seg"])
        rec["energy"].append(d["energy"].sum(axis=0))
        rec["beam_rms_seg"].append(bseg)
        rec["beam_lost"].append(d["beam_lost"])
        rec["ms"].append(ms)
        calls += 1
        if read is not None and ((read_every and calls % read_every == 0) or done >= steps):
            reads.append(read(q, p, d))
            read_tau.append(rec["tau"][-1])
            if log:
                log(f"  read at tau {read_tau[-1]:.0f}: {json.dumps(reads[-1])}")
        if log:
            r = d["rms_seg"]
            log(f"step {done}/{steps} tau {rec['tau'][-1]:.0f}  rms B_perp(xi=2) "
                f"{math.hypot(r[1, 3], r[1, 4]):.3e}  rms E_perp(xi=20) "
                f"{math.hypot(r[10, 0], r[10, 1]):.3e}  {ms:.0f} ms")
    q.close()
    out = {k: np.asarray(v) for k, v in rec.items()}
    out["seg_width"] = np.float64(seg_width)
    if read is not None:
        out["reads"] = reads
        out["read_tau"] = np.asarray(read_tau)
    return out


def summary(rec: dict, p: config.Params, k_ref: float = 1.0) -> dict:
    """Growth and saturation near the front (xi = 2) and downstream (xi = 20), read from
    `run`'s record.

    The paper's geometry is 2D with the beam along x: its B_z (filamentation) and E_y (oblique
    two-stream) are the transverse magnetic and electric fields, here B_perp = (B_x, B_y) and
    E_perp = (E_x, E_y) of the 3D box, read as rms magnitudes.  Gamma is Eq. 5's rate at
    k_y = k_ref; the segment [xi, xi + 2) is read at its centre.
      growth_vs_exponent: slope of ln rms against the asymptotic exponent (Eq. 7 at the front,
        Eq. 6 downstream) over 2 <= Gamma tau <= 5; 1 where the field follows it;
      rate_ratio_end: the growth rate over the last recorded interval over the spatiotemporal
        rate Gamma^st there; well below 1 once the growth saturates (near the front a field
        that follows Eq. 7 exactly gives 1 + xi/(4 Gamma tau), from its correction factor);
      eps_end, eps_estimate_end: the fractional field energy at the end of the run, and the
        trapping estimate evaluated with tau_sat = that time;
      dpy_end, dpy_estimate_end: the beam's rms u_y spread in the segment (first species) and
        its trapping estimate gamma_b Gamma^st / k_y, likewise."""
    sp = p.species[0]
    Gamma = temporal_rate(k_ref, p.species)
    tau = rec["tau"]
    w = float(rec["seg_width"])
    rs = rec["rms_seg"]
    out = {"Gamma": Gamma, "Gamma_tau_end": float(Gamma * tau[-1]),
           "ms_per_step": float(np.sum(rec["ms"]) / max(tau[-1] / p.dt + 1.0, 1.0))}
    bperp = np.sqrt(rs[:, :, 3] ** 2 + rs[:, :, 4] ** 2)
    eperp = np.sqrt(rs[:, :, 0] ** 2 + rs[:, :, 1] ** 2)
    for name, xi0, F, expo, rate, eps, dpy in (
            ("front_Bperp", 2.0, bperp, exponent_front, rate_front,
             lambda x, ts: eps_bz_sat(x, ts, k_ref), dpy_front),
            ("rear_Eperp", 20.0, eperp, exponent_rear, rate_rear,
             lambda x, ts: eps_ey_sat(x, ts, sp.alpha, sp.gamma_b, k_ref), dpy_rear)):
        s = int(xi0 / w)
        xi = (s + 0.5) * w
        r = F[:, s]
        gt = Gamma * tau
        res = {"xi": xi}
        sel = (gt >= 2.0) & (gt <= 5.0) & (r > 0)
        if sel.sum() >= 3:
            res["growth_vs_exponent"] = float(np.polyfit(expo(gt[sel], xi), np.log(r[sel]), 1)[0])
        if len(tau) >= 2 and r[-2] > 0 and r[-1] > 0:
            local = math.log(r[-1] / r[-2]) / (tau[-1] - tau[-2])
            res["rate_ratio_end"] = float(local / rate(Gamma, xi, 0.5 * (tau[-1] + tau[-2])))
        te = float(tau[-1])
        res["eps_end"] = float(fractional_energy(r[-1] ** 2, sp.alpha, sp.gamma_b))
        res["eps_estimate_end"] = float(eps(xi, te))
        res["dpy_end"] = float(rec["beam_rms_seg"][-1, 0, s, 1])
        res["dpy_estimate_end"] = float(dpy(Gamma, xi, te, sp.gamma_b, k_ref))
        out[name] = res
    return out


def filament_reading(q, p: config.Params, d: dict, front: float = 10.0,
                     downstream=(12.0, 40.0)) -> dict:
    """The filaments of the beam front and their wakes, read from handle q after a run (d: its
    diagnostics).  The beam charge density rho_b = S_b + J_z (both species) on the slab nodes
    of xi < front gives filament_sizes; the filament charge density is read as the mean |rho_b
    - <rho_b>| over the cells where it exceeds half its maximum (the filament cores).  The
    wake estimate ex_wake_amplitude(rho_fil, length, width/2) (w read as the half-width of a
    filament of full width `width`) stands beside the measured E_z (the paper's E_x) downstream:
    sqrt 2 times its rms over the slices of `downstream` (the amplitude of a wave of that rms)."""
    n = int(round(front / p.dxi))
    rho = q.source("Sb", 0, n) + q.source("Jz", 0, n)
    sz = filament_sizes(rho, p.dx, p.dy, p.dxi)
    dev = np.abs(rho - rho.mean(axis=(1, 2), keepdims=True))
    core = dev > 0.5 * dev.max()
    rho_fil = float(dev[core].mean())
    est = float(ex_wake_amplitude(rho_fil, sz["length"], 0.5 * sz["width"]))
    xi = np.arange(p.nxi + 1) * p.dxi
    sel = (xi >= downstream[0]) & (xi < downstream[1])
    ez_amp = float(np.sqrt(2.0 * np.mean(d["rms"][sel, 2] ** 2)))
    return dict(sz, rho_fil=rho_fil, ex_wake_estimate=est, ez_downstream_amplitude=ez_amp,
                ratio=ez_amp / est if est > 0 else float("nan"))


def dpx_reading(rec: dict, p: config.Params, rho_fil: float, seg=(12.0, 40.0),
                last: float = 0.3) -> dict:
    """Growth of the beam's longitudinal momentum spread downstream over the last fraction
    `last` of the run (rms u_z of the first species over the segments of `seg`, averaged),
    as d(rms u_z)/d tau, beside the blazar paragraph's Delta p_x ~ |rho_b| tau: against one
    species' mean beam density alpha, and against the filament charge density rho_fil."""
    w = float(rec["seg_width"])
    s0, s1 = int(seg[0] / w), int(seg[1] / w)
    uz = rec["beam_rms_seg"][:, 0, s0:s1, 2].mean(axis=1)
    tau = rec["tau"]
    sel = tau >= tau[-1] * (1.0 - last)
    slope = float(np.polyfit(tau[sel], uz[sel], 1)[0]) if sel.sum() >= 3 else float("nan")
    alpha = p.species[0].alpha
    return {"duz_dtau": slope, "alpha": alpha, "ratio_alpha": slope / alpha,
            "rho_fil": rho_fil, "ratio_fil": slope / rho_fil if rho_fil else None}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c3", choices=["c3", "filaments"],
                    help="c3: the 512^2 pair beam (400 steps); filaments: the 256^2 pair beam "
                         "driven to Gamma tau = 20, with the filament and wake reading")
    ap.add_argument("--steps", type=int, default=0, help="beam steps (0: the workload's)")
    ap.add_argument("--every", type=int, default=6)
    ap.add_argument("--depth", type=int, default=0,
                    help="beam steps in flight per launch (0: 1 for the 512^2 pair beam, whose "
                         "slices fill the GPU alone, 16 for the 256^2 one)")
    ap.add_argument("--read-every", type=int, default=10)
    ap.add_argument("--out", default="nonlinear_run.npz")
    a = ap.parse_args()
    depth = a.depth or (1 if a.workload == "c3" else 16)
    p = (config.c3_pair_beam() if a.workload == "c3" else
         config.pair_beam_filaments()).with_(pipeline_depth=depth)
    steps = a.steps or p.steps
    read = filament_reading if a.workload == "filaments" else None
    rec = run(p, steps, a.every, log=lambda s: print(s, flush=True), read=read,
              read_every=a.read_every)
    np.savez_compressed(a.out, **{k: v for k, v in rec.items() if k != "reads"})
    out = summary(rec, p)
    if read is not None:
        out["filaments"] = {"tau": rec["read_tau"].tolist(), "reads": rec["reads"]}
        out["dpx"] = dpx_reading(rec, p, rec["reads"][-1]["rho_fil"])
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
