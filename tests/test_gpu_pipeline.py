"""Pipelined beam steps (qsa_advance with pipeline_depth >= 2) against the same steps run one
after the other (qsa_plasma_sweep; qsa_beam_step), and against the FP64 oracle.

The pipelined launch reorders the work of consecutive beam steps (a wavefront in xi) but
computes the same thing; only the summation order of the atomic deposits differs.  So the
FP64 path must agree with the sequential path to rounding (1e-10 of each field's scale) and
with the oracle to the usual 1e-9; the mixed path to the mixed tolerance.  The schedule's
gates follow the beam's actual xi extent, which the drift cases below exercise: a slow beam
that slips several cells per step (and out of the window), and particles placed up to 2.5
cells ahead of and behind their lattice home.
"""
import numpy as np
import pytest

from oracle import qspic
from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module")
def Q(cuda_ok):
    from paper_2607_24214_b300.qsa import QSA
    return QSA


def field_err(a, b):
    out = []
    for f in range(a.shape[1]):
        scale = np.abs(b[:, f]).max()
        d = np.abs(a[:, f] - b[:, f]).max()
        out.append(d / scale if scale > 0 else d)
    return np.array(out)


def field_err_trans(a, b):
    """Errors of (W_x, W_y, E_z, B_x, B_y, B_z) with the transverse components against the
    transverse field magnitude (the largest of |W|, |B|) and E_z against its own scale: B_z
    of a nearly cold, round beam is small, and FP32 summation-order noise of the deposits is
    measured against the fields it perturbs, not against B_z alone (the same reading as the
    full-size pair-beam test)."""
    trans = max(np.abs(b[:, f]).max() for f in (0, 1, 3, 4, 5))
    scales = [trans, trans, np.abs(b[:, 2]).max(), trans, trans, trans]
    return np.array([np.abs(a[:, f] - b[:, f]).max() / scales[f] for f in range(6)])


def make(Q, p, beams):
    q = Q(p)
    for si, b in enumerate(beams):
        q.set_beam(si, b)
    return q


def compare(Q, p, beams, n, depth, tol, err=field_err):
    """advance(n) at `depth` vs n sequential steps; then one more sweep on both."""
    a = make(Q, p.with_(pipeline_depth=1), beams)
    for _ in range(n):
        a.sweep()
        a.beam_step()
    b = make(Q, p.with_(pipeline_depth=depth), beams)
    b.advance(n)
    da, db = a.diagnostics(), b.diagnostics()
    assert db["sweeps"] == n and da["beam_lost"] == db["beam_lost"]
    # the last sweep's slab (that of step n - 1) and its k = 0 mode
    assert err(b.slab(), a.slab()).max() <= tol
    for k in ("psi0", "ez0"):
        scale = max(np.abs(da[k]).max(), 1e-300)
        assert np.abs(db[k] - da[k]).max() <= tol * scale, k
    # the beam after n pushes, and the sources of the next sweep
    for si, bm in enumerate(beams):
        n_p = bm["x"].size
        ga, gb = a.get_beam(si, n_p), b.get_beam(si, n_p)
        np.testing.assert_array_equal(ga["w"] == 0, gb["w"] == 0)
        for key in ("x", "y", "xi", "ux", "uy", "uz"):
            scale = max(np.abs(ga[key]).max(), 1e-300)
            assert np.abs(ga[key] - gb[key]).max() <= tol * scale, (si, key)
    for k in range(4):
        sa, sb = a.source(k), b.source(k)
        assert np.abs(sa - sb).max() <= tol * max(np.abs(sa).max(), 1e-300), k
    # a single sweep after the pipelined launches reads the right sources
    a.sweep()
    b.sweep()
    assert err(b.slab(), a.slab()).max() <= tol
    return a, b


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("depth,n", [(4, 6), (3, 3), (16, 5), (2, 1)])
def test_pipelined_equals_sequential_c1(Q, prec, depth, n):
    p = config.c1_fp64_electron_beam().with_(precision=prec)
    compare(Q, p, inputs.all_beams(p), n, depth, TOL[prec])


def test_pipelined_c1_against_oracle(Q):
    """The whole C1 run (10 beam steps) pipelined, then a sweep: within 1e-9 of the oracle."""
    p = config.c1_fp64_electron_beam().with_(pipeline_depth=4)
    beams = inputs.all_beams(p)
    q = make(Q, p, beams)
    q.advance(p.steps)
    q.sweep()
    ref_slab, _, _ = qspic.run(p, beams, p.steps)
    assert field_err(q.slab(), ref_slab).max() <= 1e-9


def test_pipelined_slow_beam_drift_and_loss(Q):
    """gamma_b = 2: the beam slips about two xi cells per step and leaves the window; the
    gates must wait for the slab nodes that the drifted particles gather."""
    p = config.c1_fp64_electron_beam().with_(dt=2.0, nxi=32, Lxi=4.0)
    p.species[0].gamma_b = 2.0
    p.species[0].alpha = 1e-3
    beams = inputs.all_beams(p)
    a, b = compare(Q, p, beams, 6, 4, TOL["fp64"])
    assert b.diagnostics()["beam_lost"] > 1000


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pipelined_particles_off_home(Q, prec):
    """Particles up to 2.5 cells ahead of or behind their home layer (a state qsa_set_beam
    accepts); a particle ahead of its home deposits into nodes that an earlier layer also
    feeds, which the schedule covers with its margin.  The clipped ones sit just below the
    window's end, where FP32 rounds them onto it: their xi cell must still be the last one,
    or the schedule waits for a slab node that does not exist."""
    p = config.c1_fp64_electron_beam().with_(nxi=32, Lxi=4.0, precision=prec)
    beams = inputs.all_beams(p)
    rng = np.random.default_rng(7)
    b0 = beams[0]
    b0["xi"] = np.clip(b0["xi"] + rng.uniform(-2.5, 2.5, b0["xi"].size) * p.dxi, 0.0,
                       p.Lxi * (1 - 1e-12))
    compare(Q, p, beams, 5, 4, TOL[prec], field_err if prec == "fp64" else field_err_trans)


def test_pipelined_pair_beam_partial_window(Q):
    """Two species, the second filling only the middle half of the window (layers with
    particles of one species only, ring entries fed by two species)."""
    p = config.c1_fp64_electron_beam().with_(nxi=32, Lxi=4.0)
    e = p.species[0]
    pos = config.Species(Z=+1.0, M=1.0, alpha=e.alpha, gamma_b=e.gamma_b, ppc_x=2, ppc_y=2,
                         ppc_xi=1, uperp_spread=e.uperp_spread, noise_rel=e.noise_rel,
                         xi_front=1.0, xi_back=3.0)
    p = p.with_(species=[e, pos])
    compare(Q, p, inputs.all_beams(p), 4, 3, TOL["fp64"])


def test_advance_zero_steps_and_sequential_depth(Q):
    p = config.c1_fp64_electron_beam().with_(nxi=16, Lxi=2.0)
    beams = inputs.all_beams(p)
    q = make(Q, p.with_(pipeline_depth=4), beams)
    q.advance(0)
    assert q.diagnostics()["sweeps"] == 0
    # depth 1: advance is the sequential loop
    compare(Q, p, beams, 3, 1, 1e-12)


def scattered(p, seed=4):
    """The C1-like beam with every particle moved up to 6 cells from its lattice home in x
    and y (cells end up with uneven counts, some above the ppc slots a cell has), and 1 % of
    the particles marked lost."""
    rng = np.random.default_rng(seed)
    beams = inputs.all_beams(p)
    for b in beams:
        m = b["x"].size
        b["x"] = np.mod(b["x"] + rng.uniform(-6, 6, m) * p.dx, p.Lx)
        b["y"] = np.mod(b["y"] + rng.uniform(-6, 6, m) * p.dy, p.Ly)
        b["ux"] = b["ux"] + rng.normal(0, 0.05, m)
        b["w"][rng.random(m) < 0.01] = 0.0
    return beams


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rehome_keeps_every_particle_and_the_fields(Q, prec):
    """Re-homing moves particles between storage slots only: the host copy of the beam (each
    particle by its id) and the next sweep's fields are unchanged, to rounding."""
    p = config.c1_fp64_electron_beam().with_(nxi=24, Lxi=3.0, precision=prec)
    beams = scattered(p)
    a, b = make(Q, p, beams), make(Q, p, beams)
    n = beams[0]["x"].size
    before = b.get_beam(0, n)
    b.rehome()
    assert b.rehome_count() == 1
    after = b.get_beam(0, n)
    np.testing.assert_array_equal(before["w"], after["w"])
    ptol = 1e-12 if prec == "fp64" else 1e-6
    for key, L in (("x", p.Lx), ("y", p.Ly)):
        e = np.mod(after[key] - before[key] + 0.5 * L, L) - 0.5 * L
        assert np.abs(e).max() <= ptol * L, key
    for key in ("xi", "ux", "uy", "uz"):
        assert np.abs(after[key] - before[key]).max() <= ptol * np.abs(before[key]).max(), key
    a.sweep()
    b.sweep()
    assert field_err(b.slab(), a.slab()).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pipelined_run_rehomes_and_matches_sequential(Q, prec):
    """A pipelined run whose particles sit away from their homes re-homes the beam before
    its second launch (rehome_frac) and still matches the steps run one after the other."""
    p = config.c1_fp64_electron_beam().with_(nxi=24, Lxi=3.0, precision=prec, rehome_frac=0.05)
    a, b = compare(Q, p, scattered(p), 4, 2, TOL[prec])
    assert b.rehome_count() >= 1
