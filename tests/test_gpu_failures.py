"""Failure detection without a GPU fault: every failure here is made on the host.

- a NaN momentum in a host beam: the sweep's fields turn non-finite, the device status word
  latches it and the next synchronising call returns QSA_ERR_NONFINITE; the context stays
  usable;
- a psi floor above the lowest 1 + psi the plasma reaches: the floor is applied and counted,
  the status is the warning QSA_WARN_PSI_FLOOR, and the floored fields still match the
  oracle, which floors the same way;
- an allocator that refuses past a byte cap: qsa_init returns QSA_ERR_OOM, gives no handle,
  and has released everything it had allocated."""
import ctypes as ct

import numpy as np
import pytest

from oracle import qspic
from paper_2607_24214_b300 import config, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsa_mod(cuda_ok):
    from paper_2607_24214_b300 import qsa
    return qsa


def test_nan_momentum_is_reported_and_context_survives(qsa_mod):
    p = config.c1_fp64_electron_beam().with_(nxi=16, Lxi=2.0)
    b = inputs.all_beams(p)[0]
    b["ux"][b["ux"].size // 3] = np.nan
    q = qsa_mod.QSA(p)
    q.set_beam(0, b)
    q.sweep()
    with pytest.raises(qsa_mod.QsaError) as e:
        q.diagnostics()
    assert e.value.code == qsa_mod.QSA_ERR_NONFINITE
    q.close()
    r = qsa_mod.QSA(p)
    r.set_beam(0, inputs.all_beams(p)[0])
    r.sweep()
    assert r.diagnostics()["status"] == 0
    r.close()


def test_psi_floor_warning_and_floored_parity(qsa_mod):
    # a positron beam drives psi negative: 1 + psi reaches ~0.94 at alpha = 0.03, so a floor
    # of 0.95 is applied on some slices (an electron beam drives psi positive)
    p = config.c1_fp64_electron_beam().with_(psi_floor=0.95)
    p.species[0].Z = 1.0
    p.species[0].alpha = 0.03
    beams = inputs.all_beams(p)
    q = qsa_mod.QSA(p)
    q.set_beam(0, beams[0])
    q.sweep()
    d = q.diagnostics()
    assert d["status"] == qsa_mod.QSA_WARN_PSI_FLOOR
    ref, rd = qspic.plasma_sweep(p, qspic.beam_sources(p, beams))
    np.testing.assert_array_equal(d["n_floor"], rd["n_floor"])
    assert d["n_floor"].max() > 0
    slab = q.slab()
    for f in range(6):
        scale = np.abs(ref[:, f]).max()
        assert np.abs(slab[:, f] - ref[:, f]).max() <= 1e-9 * scale, f
    q.close()


def test_allocation_failure_returns_oom_and_releases_everything(qsa_mod):
    import torch
    dev = torch.cuda.current_device()
    live = {}
    cap = 4 << 20  # the handle needs far more than 4 MB

    def _alloc(nbytes, ctx, strm):
        if sum(live.values()) + nbytes > cap:
            return None
        ptr = torch.cuda.caching_allocator_alloc(nbytes, dev, strm)
        live[ptr] = nbytes
        return ptr

    def _free(ptr, nbytes, ctx, strm):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    alloc, free = qsa_mod.ALLOC_FN(_alloc), qsa_mod.FREE_FN(_free)
    lib = qsa_mod.load_library()
    cp = qsa_mod.to_c_params(config.c1_fp64_electron_beam())
    h = ct.c_void_p()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.qsa_init(ct.byref(cp), stream, alloc, free, None, ct.byref(h))
    torch.cuda.synchronize()
    assert rc == qsa_mod.QSA_ERR_OOM
    assert not h.value
    assert live == {}
