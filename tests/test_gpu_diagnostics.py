"""The per-slice diagnostics of the boundary (qsa_diag) against their definitions evaluated
on the FP64 oracle's state: Fourier amplitudes of requested modes, rms fields per slice and
per xi segment of width 2 k_p^-1, and the beam's momentum moments per xi cell.

Tolerances as the field parity: 1e-9 of each quantity's scale (FP64), 1e-4 (mixed)."""
import numpy as np
import pytest

from oracle import qspic
from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-4}
MODES = [(1, 0), (0, 2), (-1, 1), (2, -3), (3, 3), (-16, 5)]


@pytest.fixture(scope="module")
def Q(cuda_ok):
    from paper_2607_24214_b300.qsa import QSA
    return QSA


def fourier(F, mx, my):
    """F(k)/(nx ny) of a real grid F[ny, nx] at k = (mx, my) (numpy's forward sign)."""
    ny, nx = F.shape
    return np.fft.fft2(F)[my % ny, mx % nx] / (nx * ny)


def run_both(Q, prec, steps=1):
    p = config.c1_fp64_electron_beam().with_(precision=prec, diag_modes=MODES)
    beams = inputs.all_beams(p)
    q = Q(p)
    q.set_beam(0, beams[0])
    for _ in range(steps):
        q.sweep()
        q.beam_step()
    q.sweep()
    d = q.diagnostics()
    rb = [dict((k, v.copy()) for k, v in b.items()) for b in beams]
    for _ in range(steps):
        slab, _ = qspic.plasma_sweep(p, qspic.beam_sources(p, rb))
        qspic.beam_push(p, rb, slab)
    slab, rd = qspic.plasma_sweep(p, qspic.beam_sources(p, rb), return_psi=True)
    return p, q, d, slab, rd, rb


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mode_amplitudes(Q, prec):
    p, q, d, slab, rd, _ = run_both(Q, prec)
    psi = np.asarray(rd["psi"])
    Wx, Wy, Ez, Bx, By, Bz = (slab[:, c] for c in range(6))
    fields = [psi, Ez, Bx, By, Bz]
    got = d["mode_amp"][..., 0] + 1j * d["mode_amp"][..., 1]       # [nk, m, 5]
    for f, F in enumerate(fields):
        want = np.array([[fourier(F[j], mx, my) for (mx, my) in MODES]
                         for j in range(p.nxi + 1)])
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(got[:, :, f] - want).max() <= TOL[prec] * scale, f


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rms_per_slice_and_segment(Q, prec):
    p, q, d, slab, rd, _ = run_both(Q, prec)
    Wx, Wy, Ez, Bx, By, Bz = (slab[:, c] for c in range(6))
    F = np.stack([Wx + By, Wy - Bx, Ez, Bx, By, Bz], axis=1)
    ms = (F ** 2).mean(axis=(2, 3))                                 # [nk, 6]
    scale = np.sqrt(ms).max(axis=0)
    assert np.all(np.abs(d["rms"] - np.sqrt(ms)) <= TOL[prec] * scale)
    # segments of width 2 k_p^-1: slices j dxi in [2 s, 2 s + 2), slice nxi joins the last
    nseg = int(np.ceil(p.Lxi / 2.0))
    seg = np.minimum(np.floor(np.arange(p.nxi + 1) * p.dxi / 2.0 + 1e-12).astype(int),
                     nseg - 1)
    want = np.array([np.sqrt(ms[seg == s].mean(axis=0)) for s in range(nseg)])
    assert np.all(np.abs(d["rms_seg"] - want) <= TOL[prec] * want.max(axis=0))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_beam_moments(Q, prec):
    p, q, d, slab, rd, rb = run_both(Q, prec, steps=2)
    sp = p.species[0]
    b = rb[0]
    wbar = sp.alpha * p.dx * p.dy * p.dxi / (sp.ppc_x * sp.ppc_y * sp.ppc_xi)
    live = b["w"] > 0
    cell = np.floor(b["xi"][live] / p.dxi).astype(int)
    wr = b["w"][live] / wbar
    ux, uy = b["ux"][live], b["uy"][live]
    duz = b["uz"][live] - np.sqrt(sp.gamma_b ** 2 - 1.0)
    vals = [wr, wr * ux, wr * uy, wr * duz, wr * ux * ux, wr * uy * uy, wr * duz * duz]
    want = np.stack([np.bincount(cell, weights=v, minlength=p.nxi) for v in vals], axis=1)
    got = d["beam_moments"][0]
    for k in range(7):
        scale = max(np.abs(want[:, k]).max(), 1e-300)
        tol = TOL[prec] if k in (0, 1, 2, 4, 5) or prec == "fp64" else 1e-3
        assert np.abs(got[:, k] - want[:, k]).max() <= tol * scale, k
    # the binding's derived weighted rms spreads, against the same from the oracle's sums
    if prec == "fp64":
        mean = want[:, 1:4] / want[:, :1]
        rms = np.sqrt(np.maximum(want[:, 4:7] / want[:, :1] - mean ** 2, 0.0))
        np.testing.assert_allclose(d["beam_rms_u"][0], rms, rtol=1e-6, atol=1e-12)


def test_pipelined_diagnostics_match_sequential(Q):
    p = config.c1_fp64_electron_beam().with_(diag_modes=MODES)
    beams = inputs.all_beams(p)
    a = Q(p)
    a.set_beam(0, beams[0])
    for _ in range(3):
        a.sweep()
        a.beam_step()
    b = Q(p.with_(pipeline_depth=3))
    b.set_beam(0, beams[0])
    b.advance(3)
    da, db = a.diagnostics(), b.diagnostics()
    for k in ("mode_amp", "rms", "rms_seg", "beam_moments"):
        scale = max(np.abs(da[k]).max(), 1e-300)
        assert np.abs(da[k] - db[k]).max() <= 1e-10 * scale, k


def test_invalid_diag_modes_rejected(Q):
    from paper_2607_24214_b300.qsa import QsaError
    p = config.c1_fp64_electron_beam()
    for bad in ([(0, 0)], [(17, 0)], [(0, -17)]):
        with pytest.raises(QsaError):
            Q(p.with_(diag_modes=bad))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_field_energies(Q, prec):
    """Per-slice energies 1/2 sum F^2 dx dy dxi of E_x, E_y, E_z, B_x, B_y, B_z against the
    oracle's field_energy of its own slab (pinned to closed forms on the CPU)."""
    p, q, d, slab, rd, _ = run_both(Q, prec)
    want = qspic.field_energy(p, slab)
    scale = want.max(axis=0)
    assert np.all(np.abs(d["energy"] - want) <= 2 * TOL[prec] * scale)
