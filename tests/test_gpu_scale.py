"""The pair-beam workload at its full size (512 x 512, 2048 slices, electrons and positrons,
4.3e9 beam macroparticles built on the device, mixed precision, ~180 GB of device memory):
its first slices, and the beam sources after one push, against the oracle run on exactly the
particles that reach those slices (the slice loop is sequential in xi, so the first slices
depend on nothing behind them).

Tolerances: fields 1e-4, as every mixed-path test, of their scale.  E_z against its own.
The transverse components W = E_perp - z x B and B against the transverse field magnitude,
the largest of |E_x|, |E_y|, |B_x|, |B_y|, |B_z|: at the pair-beam front the species' currents
cancel, B_z vanishes, and W is three orders below E_perp and B_perp, so a relative error of W
or B_z alone would measure roundoff against zero.  Beam sources
2e-6 of their scale, except S_b = Z n (1 - v_z): at gamma_b = 1e4 with a 1 % energy spread,
1 - v_z ~ 5e-9 and its deviation from the reference is ~50 times smaller than itself, so FP32
resolves S_b (~1e-15 in absolute terms, negligible in the fields) to ~1e-5 of its scale.
After the push, J_x and J_y come from the transverse momentum the push gives, driven by W,
which the field check holds to the transverse magnitude: relative to its own (tiny) scale W,
and so the new J_perp, carries ~1e-3."""
import numpy as np
import pytest

from oracle import qspic
from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-4
SRC_TOL = (1e-4, 2e-6, 2e-6, 2e-6)  # S_b, J_z, J_x, J_y
PUSHED_SRC_TOL = (1e-4, 2e-6, 1e-3, 1e-3)


def field_err(a, b):
    """Errors of the slab components (W_x, W_y, E_z, B_x, B_y, B_z) against the scales of the
    module docstring."""
    Wx, Wy, Ez, Bx, By, Bz = (b[:, f] for f in range(6))
    trans = max(np.abs(F).max() for F in (Wx + By, Wy - Bx, Bx, By, Bz))
    scales = [trans, trans, np.abs(Ez).max(), trans, trans, trans]
    return np.array([np.abs(a[:, f] - b[:, f]).max() / scales[f] for f in range(6)])


def test_pair_beam_full_size_first_slices(cuda_ok):
    import torch

    from paper_2607_24214_b300.qsa import QSA
    K = 3
    p = config.c3_pair_beam()
    q = QSA(p)
    per_layer = [p.nx * p.ny * s.ppc_x * s.ppc_y * s.ppc_xi for s in p.species]
    subs = [inputs.beam_arrays(p, si, 0, (K + 2) * per_layer[si]) for si in range(2)]
    src_ref = qspic.beam_sources(p, subs, n_nodes=K + 2)
    src = np.stack([q.source(k, 0, K + 2) for k in range(4)])
    for k in range(4):
        scale = np.abs(src_ref[k]).max()
        assert np.abs(src[k, :K + 1] - src_ref[k, :K + 1]).max() <= SRC_TOL[k] * scale, k
    q.sweep()
    slab = q.slab(0, K)
    ref, _ = qspic.plasma_sweep(p, src_ref, n_slices=K)
    err = field_err(slab, ref[:K])
    assert err.max() <= TOL, err
    d = q.diagnostics()
    assert d["status"] >= 0 and np.isfinite(d["energy"]).all()
    # one push of the particles in xi cells 0..K-2, which gather nodes <= K-1
    q.beam_step()
    parts = [{k: v[: (K - 1) * per_layer[si]].copy() for k, v in subs[si].items()}
             for si in range(2)]
    qspic.beam_push(p, parts, ref[:K])
    src2_ref = qspic.beam_sources(p, parts, n_nodes=K)
    src2 = np.stack([q.source(k, 0, K - 1) for k in range(4)])
    for k in range(4):
        scale = np.abs(src2_ref[k, :K - 1]).max()
        assert np.abs(src2[k] - src2_ref[k, :K - 1]).max() <= PUSHED_SRC_TOL[k] * scale, k
    q.close()
    del q
    torch.cuda.empty_cache()
