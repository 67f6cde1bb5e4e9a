"""Gradients of a run with respect to the beam's seed (the discrete adjoint, qsa_grad_forward /
qsa_grad_backward, through the torch.autograd.Function).

The loss is 1/2 sum (B_x^2 + B_y^2) dx dy dxi of the final sweep; the parameters are the
seeded mode amplitudes a_m and the density ratio alpha (the paper's linear theory, Eqs. 3-5,
ties the growth of each transverse mode to both).  Checks:
- a small seeded run (16 x 16, 16 slices, three beam steps, checkpoints every two steps):
  the adjoint gradient against central differences of the GPU's own FP64 forward run and
  against central differences of the FP64 oracle's run of the same seeded beam;
- the seeded-mode workload (128 x 128, 256 slices, 16 modes, 50 steps, checkpoints every 10)
  against central differences (h = 1e-4) of the GPU forward run, to 1e-3, on a subset of the
  parameters.
"""
import copy
import math

import numpy as np
import pytest

from oracle import qspic
from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsa_mod(cuda_ok):
    from paper_2607_24214_b300 import qsa
    return qsa


def small_seeded(n_modes=4):
    """A scaled-down seeded-mode run: 16 x 16 cells (box pi), 16 slices over 2, electron beam
    alpha 1e-2, gamma_b 500, 8 ppc, the lowest n_modes modes of amplitude 1e-3, dt 20."""
    p = config.c5_seeded_modes()
    L = 16 * config.DX_DEFAULT
    return p.with_(nx=16, ny=16, Lx=L, Ly=L, nxi=16, Lxi=2.0, modes=p.modes[:n_modes],
                   precision="fp64")


def seeded(p, amps, alpha):
    q = copy.deepcopy(p)
    for m, a in zip(q.modes, amps):
        m.amplitude = a
    q.species[0].alpha = alpha
    return q


def gpu_loss(qsa_mod, p, steps):
    q = qsa_mod.QSA(p)
    v = q.grad_forward(steps, 100)
    q.close()
    return v


def oracle_loss(p, steps):
    slab, _, _ = qspic.run(p, inputs.all_beams(p), steps)
    return 0.5 * (slab[:, 3] ** 2 + slab[:, 4] ** 2).sum() * p.dx * p.dy * p.dxi


def adjoint(p, steps, ckpt):
    import torch
    from paper_2607_24214_b300.autograd import QSAFunction
    amps = torch.tensor([m.amplitude for m in p.modes], dtype=torch.float64, requires_grad=True)
    alphas = torch.tensor([s.alpha for s in p.species], dtype=torch.float64, requires_grad=True)
    loss = QSAFunction.apply(amps, alphas, p, steps, ckpt)
    loss.backward()
    return float(loss.detach()), amps.grad.numpy().copy(), alphas.grad.numpy().copy()


def fd(loss_fn, p, steps, rel):
    """Central differences of loss_fn over every mode amplitude and alpha (steps rel times
    the parameter)."""
    amps = [m.amplitude for m in p.modes]
    alpha = p.species[0].alpha
    out = []
    for k in range(len(amps) + 1):
        vals = []
        for sgn in (1, -1):
            a = list(amps)
            al = alpha
            if k < len(amps):
                h = rel * a[k]
                a[k] += sgn * h
            else:
                h = rel * alpha
                al += sgn * h
            vals.append(loss_fn(seeded(p, a, al), steps))
        out.append((vals[0] - vals[1]) / (2 * h))
    return np.array(out)


def test_adjoint_matches_finite_differences_small(qsa_mod):
    p = small_seeded()
    steps = 3
    loss, ga, gal = adjoint(p, steps, 2)
    assert loss > 0
    grad = np.concatenate([ga, gal])
    # the GPU's own FP64 forward, relative steps 1e-5 (the loss is smooth in the weights)
    fd_gpu = fd(lambda q, n: gpu_loss(qsa_mod, q, n), p, steps, 1e-5)
    scale = np.abs(fd_gpu).max()
    assert np.abs(grad - fd_gpu).max() <= 1e-6 * scale, (grad, fd_gpu)
    # the oracle's run of the same seeded beam, relative steps 1e-4
    fd_or = fd(oracle_loss, p, steps, 1e-4)
    assert abs(oracle_loss(p, steps) / loss - 1) < 1e-9
    assert np.abs(grad - fd_or).max() <= 1e-5 * scale, (grad, fd_or)


def test_adjoint_segments_do_not_change_the_gradient(qsa_mod):
    """Checkpoint intervals of 1, 2 and 10 steps give the same gradient (each segment is
    recomputed from its checkpoint)."""
    p = small_seeded(2)
    res = [adjoint(p, 3, k) for k in (1, 2, 10)]
    for loss, ga, gal in res[1:]:
        assert loss == pytest.approx(res[0][0], rel=1e-12)
        np.testing.assert_allclose(ga, res[0][1], rtol=1e-9, atol=1e-9 * np.abs(res[0][1]).max())
        np.testing.assert_allclose(gal, res[0][2], rtol=1e-9)


def test_adjoint_rejects_unsupported_runs(qsa_mod):
    p = small_seeded(2)
    q = qsa_mod.QSA(p.with_(precision="mixed"))
    with pytest.raises(qsa_mod.QsaError):
        q.grad_forward(1)
    q.close()
    q = qsa_mod.QSA(p)
    q.sweep()
    with pytest.raises(qsa_mod.QsaError):
        q.grad_forward(1)               # not a fresh handle
    with pytest.raises(qsa_mod.QsaError):
        q.grad_backward()               # nothing recorded
    q.close()


@pytest.mark.timeout(1800)
def test_adjoint_seeded_mode_workload(qsa_mod):
    """The 128 x 128, 256-slice, 16-mode workload, 50 steps, checkpoints every 10: the
    adjoint gradient against central differences (h = 1e-4) of the GPU forward run for three
    mode amplitudes and alpha, to 1e-3."""
    p = config.c5_seeded_modes().with_(precision="fp64")
    steps = p.steps
    loss, ga, gal = adjoint(p, steps, 10)
    picks = [0, 5, 15]
    for k in picks:
        vals = []
        for sgn in (1, -1):
            a = [m.amplitude for m in p.modes]
            a[k] += sgn * 1e-4
            vals.append(gpu_loss(qsa_mod, seeded(p, a, p.species[0].alpha), steps))
        d = (vals[0] - vals[1]) / 2e-4
        assert abs(ga[k] - d) <= 1e-3 * max(abs(d), 1e-3 * np.abs(ga).max()), (k, ga[k], d)
    vals = [gpu_loss(qsa_mod, seeded(p, [m.amplitude for m in p.modes],
                                     p.species[0].alpha + s * 1e-4), steps) for s in (1, -1)]
    d = (vals[0] - vals[1]) / 2e-4
    assert abs(gal[0] - d) <= 1e-3 * abs(d), (gal[0], d)
