"""The oracle's tolerance mode of the predictor-corrector (B_perp iterated until its relative
change falls below pc_tol, at most n_pc_iter solves) against the fixed-count loop it must
reduce to: a tolerance no solve can miss is one solve, a tolerance no solve can meet is the
fixed count, and on the first slice the count is the first n whose fixed-count run ends
with a change below the tolerance, with that run's fields."""
import numpy as np
import pytest

from oracle import qspic
from paper_2607_24214_b300 import config, inputs


@pytest.fixture(scope="module")
def case():
    p = config.c1_fp64_electron_beam().with_(nxi=8, Lxi=1.0)
    return p, qspic.beam_sources(p, inputs.all_beams(p))


def test_huge_tolerance_is_one_solve(case):
    p, src = case
    a, da = qspic.plasma_sweep(p.with_(n_pc_iter=4, pc_tol=1e9), src)
    b, db = qspic.plasma_sweep(p.with_(n_pc_iter=1), src)
    np.testing.assert_array_equal(a, b)
    assert np.all(da["pc_iters"] == 1) and np.all(db["pc_iters"] == 1)


def test_unreachable_tolerance_is_the_fixed_count(case):
    p, src = case
    a, da = qspic.plasma_sweep(p.with_(n_pc_iter=3, pc_tol=1e-300), src)
    b, db = qspic.plasma_sweep(p.with_(n_pc_iter=3), src)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(da["pc_residual"], db["pc_residual"])
    assert np.all(da["pc_iters"] == 3) and np.all(db["pc_iters"] == 3)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_first_slice_stops_at_first_converged_solve(case, tol):
    p, src = case
    runs = [qspic.plasma_sweep(p.with_(n_pc_iter=n), src, n_slices=1) for n in range(1, 7)]
    res = [d["pc_residual"][0] for _, d in runs]
    want = next(n for n in range(1, 7) if res[n - 1] < tol or n == 6)
    got, d = qspic.plasma_sweep(p.with_(n_pc_iter=6, pc_tol=tol), src, n_slices=1)
    assert d["pc_iters"][0] == want
    np.testing.assert_array_equal(got[0], runs[want - 1][0][0])
    # the changes shrink from solve to solve (the corrector contracts on this case)
    assert all(res[n + 1] < res[n] for n in range(len(res) - 1))
