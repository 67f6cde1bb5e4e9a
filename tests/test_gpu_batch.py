"""Batched instances (qsa_advance_batch): several independent runs of different grids and
beams advanced together, one step of up to 16 of them per persistent launch.  Each instance
must end where its own steps, run one after the other, end (FP64: 1e-10 of each field's
scale; mixed: the mixed tolerance), whatever FFT unit shape the autotuner tries."""
import numpy as np
import pytest

from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-4}


@pytest.fixture(scope="module")
def qsa_mod(cuda_ok):
    from paper_2607_24214_b300 import qsa
    return qsa


def instances(n, prec):
    """Small instances of different grids, boxes, alpha and gamma_b (C1-like slices)."""
    grids = [(16, 16), (24, 24), (32, 32), (12, 18), (32, 16), (9, 12), (18, 18), (8, 24)]
    out = []
    for i in range(n):
        nx, ny = grids[i % len(grids)]
        p = config.c1_fp64_electron_beam().with_(
            nx=nx, ny=ny, Lx=nx * 0.2, Ly=ny * 0.25, nxi=32, Lxi=4.0, precision=prec,
            seed=i, dt=3.0 + i, diag_modes=[(1, 1)])
        p.species[0].alpha = 0.02 * (1 + i % 5)
        p.species[0].gamma_b = 50.0 + 40.0 * i
        out.append(p)
    return out


def field_err(a, b):
    out = []
    for f in range(a.shape[1]):
        scale = np.abs(b[:, f]).max()
        d = np.abs(a[:, f] - b[:, f]).max()
        out.append(d / scale if scale > 0 else d)
    return np.array(out)


def check_batch(qsa_mod, ps, steps, tol):
    seq = []
    for p in ps:
        q = qsa_mod.QSA(p)
        q.set_beam(0, inputs.all_beams(p)[0])
        for _ in range(steps):
            q.sweep()
            q.beam_step()
        seq.append(q)
    bat = []
    for p in ps:
        q = qsa_mod.QSA(p)
        q.set_beam(0, inputs.all_beams(p)[0])
        bat.append(q)
    qsa_mod.advance_batch(bat, steps)
    for a, b, p in zip(seq, bat, ps):
        da, db = a.diagnostics(), b.diagnostics()
        assert db["sweeps"] == steps and da["beam_lost"] == db["beam_lost"]
        assert field_err(b.slab(), a.slab()).max() <= tol
        n = inputs.all_beams(p)[0]["x"].size
        ga, gb = a.get_beam(0, n), b.get_beam(0, n)
        for key in ("x", "y", "xi", "ux", "uy", "uz"):
            scale = max(np.abs(ga[key]).max(), 1e-300)
            assert np.abs(ga[key] - gb[key]).max() <= tol * scale, key
        for k in ("mode_amp", "beam_moments"):
            scale = max(np.abs(da[k]).max(), 1e-300)
            assert np.abs(da[k] - db[k]).max() <= tol * scale, k
        # the next sweep of each batched instance reads the right sources
        a.sweep()
        b.sweep()
        assert field_err(b.slab(), a.slab()).max() <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_of_uneven_instances(qsa_mod, prec):
    check_batch(qsa_mod, instances(5, prec), 3, TOL[prec])


def test_batch_mixing_row_paths(qsa_mod):
    """Mixed precision, grids 256 wide (rows by warps: each row unit's pairs of fields are
    separate work items) in one launch with narrower grids (rows by block transforms): the
    slots' work items of every phase are laid end to end with different counts per unit."""
    ps = []
    for i, (nx, ny) in enumerate([(256, 16), (32, 32), (256, 8), (24, 24)]):
        p = config.c1_fp64_electron_beam().with_(
            nx=nx, ny=ny, Lx=nx * 0.05, Ly=ny * 0.25, nxi=24, Lxi=3.0, precision="mixed",
            seed=40 + i, dt=3.0 + i, diag_modes=[(1, 1)])
        p.species[0].alpha = 0.02 * (1 + i)
        p.species[0].gamma_b = 60.0 + 30.0 * i
        ps.append(p)
    check_batch(qsa_mod, ps, 3, TOL["mixed"])


def test_batch_larger_than_one_launch(qsa_mod):
    """18 instances: two launches per step (16 + 2)."""
    check_batch(qsa_mod, instances(18, "fp64"), 2, TOL["fp64"])


def test_batch_with_autotuned_shapes(qsa_mod):
    """8 steps: the first four run one FFT unit shape each, the rest the fastest."""
    check_batch(qsa_mod, instances(3, "fp64"), 8, TOL["fp64"])


def test_batch_rejects_mixed_precisions_and_duplicates(qsa_mod):
    a = qsa_mod.QSA(instances(1, "fp64")[0])
    b = qsa_mod.QSA(instances(1, "mixed")[0])
    with pytest.raises(qsa_mod.QsaError):
        qsa_mod.advance_batch([a, b], 1)
    with pytest.raises(qsa_mod.QsaError):
        qsa_mod.advance_batch([a, a], 1)


def test_c4_scan_instances_are_valid(qsa_mod):
    """The C4 workload's parameter draw builds on the device (two of its instances)."""
    ps = config.c4_parameter_scan(2)
    qs = [qsa_mod.QSA(p) for p in ps]
    qsa_mod.advance_batch(qs, 1)
    for q in qs:
        assert q.diagnostics()["status"] >= 0


def test_smaller_handle_created_later_does_not_break_larger(qsa_mod):
    """Kernel launch limits are per function, shared by all handles: a handle of a smaller
    grid created after a larger one must leave the larger one's launches valid."""
    big = qsa_mod.QSA(config.c1_fp64_electron_beam().with_(precision="mixed"))
    small = qsa_mod.QSA(config.c1_fp64_electron_beam().with_(nx=8, ny=8, Lx=1.6, Ly=1.6,
                                                              precision="mixed"))
    big.sweep()
    big.beam_step()
    big.sweep()
    small.sweep()
    assert big.diagnostics()["status"] >= 0 and small.diagnostics()["status"] >= 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_instances_match_the_oracle(qsa_mod, prec):
    """Four uneven instances (grids 16x16, 24x24, 32x32, 12x18; alpha, gamma_b and dt all
    different, like the scan over alpha_b and gamma_b after Fig. 2) advanced together by
    qsa_advance_batch for two steps, then swept: each instance's slab, beam and lost count
    against the FP64 oracle's run of the same beam (FP64 1e-9, mixed 1e-4 of each field's
    scale; lost particles exact)."""
    from oracle import qspic
    tol = {"fp64": 1e-9, "mixed": 1e-4}[prec]
    ps = instances(4, prec)
    qs = []
    for p in ps:
        q = qsa_mod.QSA(p)
        q.set_beam(0, inputs.all_beams(p)[0])
        qs.append(q)
    qsa_mod.advance_batch(qs, 2)
    for q, p in zip(qs, ps):
        q.sweep()
        d = q.diagnostics()
        assert d["status"] >= 0
        ref, _, rb = qspic.run(p, inputs.all_beams(p), 2)
        assert field_err(q.slab(), ref).max() <= tol
        n = rb[0]["x"].size
        gb = q.get_beam(0, n)
        assert np.array_equal(gb["w"] == 0, rb[0]["w"] == 0)
        live = rb[0]["w"] != 0
        for key in ("xi", "ux", "uy"):
            scale = max(np.abs(rb[0][key][live]).max(), 1e-300)
            assert np.abs(gb[key][live] - rb[0][key][live]).max() <= tol * scale, key
        for key, L, d in (("x", p.Lx, p.dx), ("y", p.Ly, p.dy)):     # periodic positions
            e = np.mod(gb[key][live] - rb[0][key][live] + 0.5 * L, L) - 0.5 * L
            assert np.abs(e).max() <= tol * d, key
        q.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_graphs_match_direct_launches(qsa_mod, prec):
    """The batched steps replayed as CUDA graphs (qsa_batch_graphs; 18 instances, so two
    launches per step, over five steps, so both ring phases of the sources are captured and
    replayed) against the same steps launched directly: the same fields, beams and
    diagnostics to rounding, and the graphs really ran.  The same kernels run in the same
    order; only the order of the atomic sums differs between any two runs: FP64 keeps that
    below 1e-12 of a field's scale over these steps (the check of the graph machinery),
    while FP32 sums, amplified by the growing modes, reach ~1e-5 after the last sweep and
    are held to the mixed path's tolerance."""
    ps = instances(18, prec)
    runs = []
    for graphs in (False, True):
        qs = []
        for p in ps:
            q = qsa_mod.QSA(p)
            q.set_beam(0, inputs.all_beams(p)[0])
            qs.append(q)
        qsa_mod.batch_graphs(qs[0], graphs)
        qsa_mod.advance_batch(qs, 5)
        n = qsa_mod.batch_graphs(qs[0])
        if graphs:
            assert n == 4, n  # the first step launches directly (it sets the launches up)
            lt = qs[0].launch_times()  # the replays' launches, timed by their own events
            assert len(lt) >= 2 and np.all(np.asarray(lt) > 0), lt
        else:
            assert n == -1, n
        runs.append(qs)
    tol = 1e-12 if prec == "fp64" else TOL["mixed"]
    for a, b, p in zip(runs[0], runs[1], ps):
        da, db = a.diagnostics(), b.diagnostics()
        assert da["sweeps"] == db["sweeps"] == 5 and da["beam_lost"] == db["beam_lost"]
        assert field_err(b.slab(), a.slab()).max() <= tol
        n = inputs.all_beams(p)[0]["x"].size
        ga, gb = a.get_beam(0, n), b.get_beam(0, n)
        for key in ("x", "y", "xi", "ux", "uy", "uz"):
            scale = max(np.abs(ga[key]).max(), 1e-300)
            assert np.abs(ga[key] - gb[key]).max() <= tol * scale, key
        a.sweep()
        b.sweep()
        assert field_err(b.slab(), a.slab()).max() <= tol
