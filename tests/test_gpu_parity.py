"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: the FP64 path must match the oracle to 1e-9 relative over one beam step; the
mixed path to 1e-4 per field (error normalised by the field's largest magnitude in the slab:
fields are O(alpha) and several vanish near the beam front, so a pointwise relative error is
undefined there).  Index work (beam initialisation lattice, particle loss) is exact.
"""
import math

import numpy as np
import pytest

from oracle import linear_theory as lt
from oracle import qspic
from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-4}


@pytest.fixture(scope="module")
def Q(cuda_ok):
    from paper_2607_24214_b300.qsa import QSA
    return QSA


def field_err(a, b):
    """Per-field error of slabs [nk, 6, ny, nx]: max |a - b| / max |b| (absolute if b == 0)."""
    out = []
    for f in range(a.shape[1]):
        scale = np.abs(b[:, f]).max()
        d = np.abs(a[:, f] - b[:, f]).max()
        out.append(d / scale if scale > 0 else d)
    return np.array(out)


def gpu(Q, p, beams=None):
    q = Q(p)
    if beams is not None:
        for si, b in enumerate(beams):
            q.set_beam(si, b)
    return q


# ------------------------------------------------------------------ transverse solves
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny", [(32, 32), (9, 12), (1, 64), (96, 48), (256, 256), (256, 36),
                                   (36, 256), (1, 256)])
def test_field_solve(Q, prec, nx, ny):
    p = config.Params(nx=nx, ny=ny, nxi=4, Lx=0.3 * nx, Ly=0.25 * ny, Lxi=1.0, dt=1.0,
                      precision=prec)
    rng = np.random.default_rng(nx * 1000 + ny)
    S, Jx, Jy, Jz, Dx, Dy = (rng.normal(size=(ny, nx)) for _ in range(6))
    q = Q(p)
    out = q.field_solve(S, Jx, Jy, Jz, Dx, Dy, kappa2=0.7)
    G = qspic.Grid(p)
    psi, gx, gy = qspic.solve_psi(G, S)
    Ez, Bz = qspic.solve_ez_bz(G, Jx, Jy)
    Bx, By = qspic.solve_bperp(G, Jz, Dx, Dy, 0.7, np.zeros_like(S), np.zeros_like(S))
    tol = 1e-12 if prec == "fp64" else 3e-6
    for name, ref in (("psi", psi), ("gpx", gx), ("gpy", gy), ("Ez", Ez), ("Bz", Bz),
                      ("Bx", Bx), ("By", By)):
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(out[name] - ref).max() <= tol * scale + 1e-300, name


# ------------------------------------------------------------------ beam initial conditions
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_beam_init_matches_generator(Q, prec):
    p = config.c1_fp64_electron_beam().with_(precision=prec)
    q = Q(p)
    n = inputs.beam_count(p, 0)
    g = q.get_beam(0, n)
    ref = inputs.beam_arrays(p, 0)
    for k in ("x", "y", "xi"):
        np.testing.assert_allclose(g[k], ref[k], rtol=0, atol=1e-12)
    r = 1e-13 if prec == "fp64" else 1e-6
    for k in ("ux", "uy", "w"):
        np.testing.assert_allclose(g[k], ref[k], rtol=r, atol=r * np.abs(ref[k]).max())
    np.testing.assert_allclose(g["uz"], ref["uz"], rtol=1e-13)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_beam_sources(Q, prec):
    p = config.c1_fp64_electron_beam().with_(precision=prec)
    q = Q(p)
    src = np.stack([q.source(k) for k in range(4)])
    ref = qspic.beam_sources(p, inputs.all_beams(p))
    tol = 1e-12 if prec == "fp64" else 2e-6
    for k in range(4):
        assert np.abs(src[k] - ref[k]).max() <= tol * np.abs(ref[k]).max(), k


# ------------------------------------------------------------------ sweep parity
def _sweep_parity(Q, p, tol):
    beams = inputs.all_beams(p)
    q = gpu(Q, p, beams)
    q.sweep()
    d = q.diagnostics()
    slab = q.slab()
    ref, rd = qspic.plasma_sweep(p, qspic.beam_sources(p, beams))
    err = field_err(slab, ref)
    assert err.max() <= tol, err
    # k = 0 mode: relative to its own scale, or to the field scale where it is only roundoff
    # (a pair beam has no mean current)
    scale = max(np.abs(rd["psi0"]).max(), np.abs(ref).max())
    np.testing.assert_allclose(d["psi0"], rd["psi0"], rtol=tol, atol=tol * scale)
    scale = max(np.abs(rd["ez0"]).max(), np.abs(ref).max())
    np.testing.assert_allclose(d["ez0"], rd["ez0"], rtol=tol, atol=tol * scale)
    np.testing.assert_allclose(d["kappa2"], rd["kappa2"], rtol=tol)
    return q, d, rd


def test_sweep_c1_fp64(Q):
    p = config.c1_fp64_electron_beam()
    q, d, rd = _sweep_parity(Q, p, TOL["fp64"])
    assert d["invariant"].max() < 1e-12
    assert d["charge"].max() < 1e-12 * p.Lx * p.Ly
    assert d["n_floor"].sum() == 0
    np.testing.assert_allclose(d["opp_min"], rd["opp_min"], rtol=1e-9)
    np.testing.assert_allclose(d["pc_residual"], rd["pc_residual"], rtol=1e-6, atol=1e-12)


def test_sweep_c1_mixed(Q):
    p = config.c1_fp64_electron_beam().with_(precision="mixed")
    q, d, rd = _sweep_parity(Q, p, TOL["mixed"])
    assert d["charge"].max() < 1e-5 * p.Lx * p.Ly


@pytest.mark.parametrize("geom", ["2d3v", "odd", "radix3", "tiny", "ppc1_odd"])
def test_sweep_geometries_fp64(Q, geom):
    if geom == "ppc1_odd":
        # one plasma particle per cell on an odd grid: a deposit chunk of 9 particles is not
        # a multiple of 16 bytes, so its L2 prefetch is skipped
        p = config.c1_fp64_electron_beam().with_(nx=9, ny=12, Lx=9 * 0.2, Ly=12 * 0.2,
                                                 nxi=24, Lxi=3.0, ppc_plasma_x=1,
                                                 ppc_plasma_y=1)
    elif geom == "2d3v":
        p = config.v_pair_single_mode(Lxi=6.0, eps=1e-3)
    elif geom == "odd":
        p = config.c1_fp64_electron_beam().with_(nx=9, ny=12, Lx=9 * 0.2, Ly=12 * 0.2,
                                                 nxi=24, Lxi=3.0)
    elif geom == "radix3":
        p = config.c1_fp64_electron_beam().with_(nx=48, ny=24, Lx=48 * 0.2, Ly=24 * 0.2,
                                                 nxi=16, Lxi=2.0)
    else:
        p = config.c1_fp64_electron_beam().with_(nx=2, ny=3, Lx=0.4, Ly=0.6, nxi=8, Lxi=1.0)
    _sweep_parity(Q, p, TOL["fp64"])


def test_sweep_ppc1_odd_mixed(Q):
    p = config.c1_fp64_electron_beam().with_(nx=9, ny=12, Lx=9 * 0.2, Ly=12 * 0.2, nxi=24,
                                             Lxi=3.0, ppc_plasma_x=1, ppc_plasma_y=1,
                                             precision="mixed")
    _sweep_parity(Q, p, TOL["mixed"])


def test_sweep_without_beam(Q):
    """No beam: the plasma stays at rest and every field vanishes."""
    p = config.c1_fp64_electron_beam().with_(species=[])
    q = Q(p)
    q.sweep()
    assert np.abs(q.slab()).max() == 0.0
    assert q.diagnostics()["charge"].max() < 1e-12


# ------------------------------------------------------------------ per-warp transforms
# FP32 rows of 256 points and FP32 columns of 256 points take the per-warp transforms, each on
# its own: grids 256 wide but 36 tall (the last 8-row unit of the row phases holds 4 rows),
# and the reverse.
WARP_GRIDS = {"rows256": (256, 36), "cols256": (36, 256)}


def _warp_grid(geom, **kw):
    nx, ny = WARP_GRIDS[geom]
    return config.c1_fp64_electron_beam().with_(nx=nx, ny=ny, Lx=nx * 0.2, Ly=ny * 0.2, nxi=8,
                                                Lxi=1.0, precision="mixed", **kw)


@pytest.mark.parametrize("geom", sorted(WARP_GRIDS))
def test_sweep_warp_paths_mixed(Q, geom):
    _sweep_parity(Q, _warp_grid(geom), TOL["mixed"])


def test_sweep_2d3v_256_mixed(Q):
    """The paper's 2D3V geometry (nx = 1) on 256 rows: per-warp column transforms of a single
    half-spectrum column, block row transforms of one point."""
    _sweep_parity(Q, config.v_pair_single_mode(ny=256, Lxi=4.0, precision="mixed"),
                  TOL["mixed"])


@pytest.mark.parametrize("geom", sorted(WARP_GRIDS))
def test_pipelined_warp_paths_mixed(Q, geom):
    """Two beam steps as one pipelined launch of two slots, then a sweep, against the
    oracle's run."""
    p = _warp_grid(geom, pipeline_depth=2)
    beams = inputs.all_beams(p)
    q = gpu(Q, p, beams)
    q.advance(2)
    q.sweep()
    ref_slab, _, _ = qspic.run(p, beams, 2)
    err = field_err(q.slab(), ref_slab)
    assert err.max() <= TOL["mixed"], err


# ------------------------------------------------------------------ beam step parity
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_one_beam_step_c1(Q, prec):
    p = config.c1_fp64_electron_beam().with_(precision=prec)
    beams = inputs.all_beams(p)
    q = gpu(Q, p, beams)
    q.sweep()
    q.beam_step()
    q.sweep()
    slab = q.slab()
    g = q.get_beam(0, beams[0]["x"].size)
    ref_slab, diags, rb = qspic.run(p, [dict((k, v.copy()) for k, v in b.items()) for b in beams],
                                    1)
    err = field_err(slab, ref_slab)
    assert err.max() <= TOL[prec], err
    tol = 1e-12 if prec == "fp64" else 1e-6
    for k in ("x", "y", "xi"):
        d = np.abs(g[k] - rb[0][k])
        L = {"x": p.Lx, "y": p.Ly, "xi": p.Lxi}[k]
        d = np.minimum(d, L - d) if k != "xi" else d
        assert d.max() < tol * L, k
    for k in ("ux", "uy", "uz"):
        scale = np.abs(rb[0][k]).max()
        assert np.abs(g[k] - rb[0][k]).max() <= max(tol, 1e-9) * scale, k


def test_ten_steps_c1_fp64(Q):
    """The whole C1 run (10 beam steps, 11 sweeps) stays within 1e-9 of the oracle."""
    p = config.c1_fp64_electron_beam()
    beams = inputs.all_beams(p)
    q = gpu(Q, p, beams)
    for _ in range(p.steps):
        q.sweep()
        q.beam_step()
    q.sweep()
    ref_slab, _, _ = qspic.run(p, beams, p.steps)
    err = field_err(q.slab(), ref_slab)
    assert err.max() <= TOL["fp64"], err


def test_mixed_uz_deviation_tracks_fp64(Q):
    """The mixed path keeps u_z as one float of its deviation from u_zb.  A pair-beam-like
    beam (gamma_b = 1e4, 1 % energy spread, dt = 200: a float of u_z itself has a spacing of
    1e-3 there) over ten steps: the change of every live particle's u_z over the run agrees
    with the FP64 path's to 1e-3 of the changes' scale (the mixed fields' 1e-4 acting on the
    increments, not the storage), and that scale is hundreds of float spacings of u_z; u_x,
    u_y within 1e-4 of their scale."""
    base = config.c1_fp64_electron_beam().with_(nx=16, ny=16, Lx=3.2, Ly=3.2, nxi=16,
                                                Lxi=2.0, dt=200.0)
    base.species[0].gamma_b = 1e4
    base.species[0].gamma_spread_rel = 1e-2
    base.species[0].alpha = 1e-2
    out = {}
    for prec in ("fp64", "mixed"):
        p = base.with_(precision=prec)
        beams = inputs.all_beams(p)
        q = gpu(Q, p, beams)
        for _ in range(10):
            q.sweep()
            q.beam_step()
        out[prec] = q.get_beam(0, beams[0]["x"].size)
        q.close()
    uz0 = inputs.all_beams(base)[0]["uz"]
    a, b = out["fp64"], out["mixed"]
    live = a["w"] != 0
    assert np.array_equal(live, b["w"] != 0)
    da, db = a["uz"][live] - uz0[live], b["uz"][live] - uz0[live]
    scale = np.abs(da).max()
    assert scale > 100 * np.spacing(np.float32(1e4)), scale
    assert np.abs(db - da).max() <= 1e-3 * scale, (np.abs(db - da).max(), scale)
    for k in ("ux", "uy"):
        scale = np.abs(a[k][live]).max()
        assert np.abs(b[k][live] - a[k][live]).max() <= 1e-4 * scale, k


def test_lost_particles_exact(Q):
    """A slow beam (gamma_b = 2) slips back by dt/(2 gamma^2) per step: the particles that
    cross xi = Lxi are removed, the same ones as in the oracle."""
    p = config.c1_fp64_electron_beam().with_(dt=2.0)
    p.species[0].gamma_b = 2.0
    p.species[0].alpha = 1e-3
    beams = inputs.all_beams(p)
    q = gpu(Q, p, beams)
    q.sweep()
    q.beam_step()
    d = q.diagnostics()
    _, _, rb = qspic.run(p, [dict((k, v.copy()) for k, v in b.items()) for b in beams], 1)
    n_lost = int(np.count_nonzero(rb[0]["w"] == 0))
    assert n_lost > 1000
    assert d["beam_lost"] == n_lost
    g = q.get_beam(0, beams[0]["x"].size)
    np.testing.assert_array_equal(g["w"] == 0, rb[0]["w"] == 0)


def test_resume_from_host_state(Q):
    """run(4) equals run(2) + get_beam/set_beam + run(2)."""
    p = config.c1_fp64_electron_beam().with_(nxi=32, Lxi=4.0)
    beams = inputs.all_beams(p)
    a = gpu(Q, p, beams)
    for _ in range(4):
        a.sweep()
        a.beam_step()
    a.sweep()
    b = gpu(Q, p, beams)
    for _ in range(2):
        b.sweep()
        b.beam_step()
    st = b.get_beam(0, beams[0]["x"].size)
    c = gpu(Q, p, [st])
    for _ in range(2):
        c.sweep()
        c.beam_step()
    c.sweep()
    assert field_err(c.slab(), a.slab()).max() < 1e-11


def test_set_beam_rejects_live_particle_outside_window(Q):
    """A live particle with xi outside [0, Lxi) (or NaN) is rejected, and the beam on the
    device is left as it was; the same particle marked lost (w = 0) is accepted."""
    from paper_2607_24214_b300.qsa import QsaError
    p = config.c1_fp64_electron_beam().with_(nxi=16, Lxi=2.0)
    beams = inputs.all_beams(p)
    q = gpu(Q, p, beams)
    n = beams[0]["x"].size
    before = q.get_beam(0, n)
    for bad in (p.Lxi, -1e-9, float("nan")):
        b = {k: v.copy() for k, v in beams[0].items()}
        b["xi"][n // 2] = bad
        b["ux"][:] = 1.0  # would change the beam if it were taken
        with pytest.raises(QsaError):
            q.set_beam(0, b)
        after = q.get_beam(0, n)
        for k in before:
            np.testing.assert_array_equal(after[k], before[k])
    b["w"][n // 2] = 0.0
    q.set_beam(0, b)
    assert np.all(q.get_beam(0, n)["ux"][b["w"] != 0] == 1.0)


def test_timeout_is_reported_and_context_survives(Q):
    """spin_limit = 0 makes every grid-barrier wait give up at once: the sweep ends with
    QSA_ERR_TIMEOUT reported on the host and the CUDA context stays usable."""
    from paper_2607_24214_b300.qsa import QSA_ERR_TIMEOUT, QsaError
    p = config.c1_fp64_electron_beam().with_(spin_limit=0)
    q = Q(p)
    q.sweep()
    with pytest.raises(QsaError) as e:
        q.diagnostics()
    assert e.value.code == QSA_ERR_TIMEOUT
    q.close()
    r = Q(config.c1_fp64_electron_beam().with_(nxi=8, Lxi=1.0))
    r.sweep()
    assert r.diagnostics()["status"] == 0


# ------------------------------------------------------------------ linear growth on the GPU
@pytest.fixture(scope="module")
def growth(Q):
    """Linear growth of one seeded mode (paper's 2D3V geometry), both precisions."""
    out = {}
    for prec in ("fp64", "mixed"):
        p = config.v_pair_single_mode(precision=prec)
        my = p.modes[0].my
        k = 2 * math.pi * my / p.Ly
        q = Q(p)
        amps = []
        for n in range(p.steps + 1):
            q.sweep()
            Wy = q.field("Wy")[:, :, 0]
            amps.append(np.abs(np.fft.fft(Wy, axis=1)[:, my]) / k)
            if n < p.steps:
                q.beam_step()
        out[prec] = (p, k, np.array(amps))
    return out


@pytest.mark.parametrize("xi", [2.0, 20.0])
def test_growth_rates(growth, xi):
    p, k, a64 = growth["fp64"]
    _, _, a32 = growth["mixed"]
    G = lt.growth_rate(k, p.species)
    taus = np.arange(p.steps + 1) * p.dt
    sel = (G * taus >= 2.0) & (G * taus <= 5.0)
    j = int(round(xi / p.dxi))
    r64 = np.polyfit(taus[sel], np.log(a64[sel, j]), 1)[0]
    r32 = np.polyfit(taus[sel], np.log(a32[sel, j]), 1)[0]
    ex = np.array([abs(lt.psi_series(xi, G * t, 1.0, k)) for t in taus[sel]])
    rex = np.polyfit(taus[sel], np.log(ex), 1)[0]
    assert abs(r64 / rex - 1) < 0.03
    assert abs(r32 / r64 - 1) < 0.02


# ------------------------------------------------------------------ full-size C2, sampled
def test_c2_full_size_first_slices(Q):
    """C2 at full size (256^2, 1024 slices, 5.4e8 beam particles built on the device, mixed):
    the beam sources of the first nodes, the fields of the first K slices of the sweep and the
    beam sources after one beam step match the oracle run on exactly the particles that reach
    those nodes (the slice loop is sequential in xi, so the first slices depend on nothing
    behind them)."""
    K = 6
    p = config.c2_mixed_electron_beam()
    q = Q(p)
    per_layer = p.nx * p.ny * 8
    sub = inputs.beam_arrays(p, 0, 0, (K + 2) * per_layer)       # xi cells 0..K+1
    src_ref = qspic.beam_sources(p, [sub], n_nodes=K + 2)
    src = np.stack([q.source(k, 0, K + 2) for k in range(4)])
    for k in range(4):
        assert np.abs(src[k, :K + 1] - src_ref[k, :K + 1]).max() <= 2e-6 * np.abs(src_ref[k]).max()
    q.sweep()
    slab = q.slab(0, K)
    ref, rd = qspic.plasma_sweep(p, src_ref, n_slices=K)
    assert field_err(slab, ref[:K]).max() <= TOL["mixed"]
    # one beam step of the particles in xi cells 0..K-2, which gather nodes <= K-1
    q.beam_step()
    part = {k: v[: (K - 1) * per_layer].copy() for k, v in sub.items()}
    qspic.beam_push(p, [part], ref[:K])
    src2_ref = qspic.beam_sources(p, [part], n_nodes=K)
    src2 = np.stack([q.source(k, 0, K - 1) for k in range(4)])
    for k in range(4):
        scale = np.abs(src2_ref[k, :K - 1]).max()
        assert np.abs(src2[k] - src2_ref[k, :K - 1]).max() <= 2e-6 * scale, k
