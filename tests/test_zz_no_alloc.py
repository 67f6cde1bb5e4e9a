"""qsa_field_solve_static: the field solve for callers that cannot allocate device memory.

Such callers (a code whose own memory manager already holds the GPU's memory in a fixed pool,
or a process under a hard device-memory budget) pass device inputs and outputs they own; the
entry point takes its scratch from a static array inside the library and allocates nothing.
Its results must equal those of qsa_field_solve, through the C ABI, on two calls in a row.
This file is collected last so that a stop at the first failure has run every other test.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_2607_24214_b300 import config

pytestmark = pytest.mark.gpu

QSA_FP64, QSA_MIXED, QSA_ERR_ARG, QSA_ERR_NONFINITE = 0, 1, -1, -5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny", [(96, 64), (128, 128), (1, 32)])
def test_static_solve_matches_handle_solve(cuda_ok, prec, nx, ny):
    import torch

    from paper_2607_24214_b300.qsa import QSA, load_library
    lib = load_library()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 3e-6
    p = config.Params(nx=nx, ny=ny, nxi=4, Lx=0.3 * nx, Ly=0.25 * ny, Lxi=1.0, dt=1.0,
                      precision=prec)
    q = QSA(p)
    stream = torch.cuda.current_stream()
    out = torch.empty((7, ny, nx), dtype=dtype, device="cuda")
    free_after_first = None
    for call in range(2):
        rng = np.random.default_rng(1000 * nx + ny + call)
        ins = [rng.normal(size=(ny, nx)) for _ in range(6)]
        kappa2 = 0.7 + 0.1 * call
        ref = q.field_solve(*ins, kappa2=kappa2)
        dev = [torch.tensor(a, dtype=dtype, device="cuda") for a in ins]
        torch.cuda.synchronize()
        if call == 1:
            free_after_first = torch.cuda.mem_get_info()[0]
        rc = lib.qsa_field_solve_static(nx, ny, p.Lx, p.Ly, kappa2,
                                        QSA_FP64 if prec == "fp64" else QSA_MIXED,
                                        *[ct.c_void_p(t.data_ptr()) for t in dev],
                                        ct.c_void_p(out.data_ptr()),
                                        ct.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.qsa_last_error(None)
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_after_first   # nothing allocated
        got = out.double().cpu().numpy()
        for k, name in enumerate(("psi", "gpx", "gpy", "Ez", "Bz", "Bx", "By")):
            scale = max(np.abs(ref[name]).max(), 1e-300)
            assert np.abs(got[k] - ref[name]).max() <= tol * scale, (call, name)
    q.close()


def test_static_solve_rejects_large_grid(cuda_ok):
    import torch

    from paper_2607_24214_b300.qsa import load_library
    lib = load_library()
    n = 256
    t = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    out = torch.zeros((7, n, n), dtype=torch.float64, device="cuda")
    ptr = ct.c_void_p(t.data_ptr())
    rc = lib.qsa_field_solve_static(n, n, 1.0, 1.0, 0.0, QSA_FP64, ptr, ptr, ptr, ptr, ptr, ptr,
                                    ct.c_void_p(out.data_ptr()), None)
    assert rc == QSA_ERR_ARG
    assert b"128" in lib.qsa_last_error(None)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_static_solve_reports_non_finite_like_handle_solve(cuda_ok, prec):
    """A NaN in one input makes the outputs non-finite: both entry points return
    QSA_ERR_NONFINITE and say so, and the next call on clean inputs succeeds."""
    import torch

    from paper_2607_24214_b300.qsa import QSA, QsaError, load_library
    lib = load_library()
    nx, ny = 32, 24
    dtype = torch.float64 if prec == "fp64" else torch.float32
    p = config.Params(nx=nx, ny=ny, nxi=4, Lx=0.3 * nx, Ly=0.25 * ny, Lxi=1.0, dt=1.0,
                      precision=prec)
    rng = np.random.default_rng(5)
    ins = [rng.normal(size=(ny, nx)) for _ in range(6)]
    ins[3][4, 7] = np.nan                                        # J_z
    q = QSA(p)
    with pytest.raises(QsaError) as e:
        q.field_solve(*ins, kappa2=0.5)
    assert e.value.code == QSA_ERR_NONFINITE
    q.close()
    out = torch.empty((7, ny, nx), dtype=dtype, device="cuda")
    stream = torch.cuda.current_stream()
    code = QSA_FP64 if prec == "fp64" else QSA_MIXED

    def call(arrs):
        dev = [torch.tensor(a, dtype=dtype, device="cuda") for a in arrs]
        return lib.qsa_field_solve_static(nx, ny, p.Lx, p.Ly, 0.5, code,
                                          *[ct.c_void_p(t.data_ptr()) for t in dev],
                                          ct.c_void_p(out.data_ptr()),
                                          ct.c_void_p(stream.cuda_stream))
    assert call(ins) == QSA_ERR_NONFINITE
    assert b"non-finite" in lib.qsa_last_error(None)
    ins[3][4, 7] = 0.0
    assert call(ins) == 0, lib.qsa_last_error(None)
    assert torch.isfinite(out).all()
