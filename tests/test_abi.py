"""The C-ABI library builds, loads and exports every entry point that include/qsa.h declares;
the ctypes mirror of the structs has the C layout (CPU only, no compute calls)."""
import ctypes as ct
import os
import re
import subprocess
import tempfile

import pytest

from paper_2607_24214_b300 import build, qsa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qsa.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ct.CDLL(build.LIB)


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|int64_t|const char\*)\s+(qsa_\w+)\(", text,
                                 re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(qsa.EXPORTS)


def test_struct_layout_matches_c():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "qsa.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(qsa_params),
         sizeof(qsa_species), sizeof(qsa_mode), sizeof(qsa_diag), offsetof(qsa_params, species),
         offsetof(qsa_params, modes), offsetof(qsa_params, diag_modes),
         offsetof(qsa_params, pc_tol), offsetof(qsa_diag, seg_width),
         offsetof(qsa_diag, beam_moments), offsetof(qsa_diag, pc_iters),
         offsetof(qsa_params, rehome_frac));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    want = [ct.sizeof(qsa.ParamsC), ct.sizeof(qsa.Species), ct.sizeof(qsa.Mode),
            ct.sizeof(qsa.Diag), qsa.ParamsC.species.offset, qsa.ParamsC.modes.offset,
            qsa.ParamsC.diag_modes.offset, qsa.ParamsC.pc_tol.offset, qsa.Diag.seg_width.offset,
            qsa.Diag.beam_moments.offset, qsa.Diag.pc_iters.offset,
            qsa.ParamsC.rehome_frac.offset]
    assert got == want


def test_init_without_gpu_fails_cleanly(lib):
    """With no usable device qsa_init returns an error code and a message, never crashes."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = qsa.load_library()
    from paper_2607_24214_b300 import config
    cp = qsa.to_c_params(config.c1_fp64_electron_beam())
    h = ct.c_void_p()
    rc = L.qsa_init(ct.byref(cp), None, qsa.ALLOC_FN(), qsa.FREE_FN(), None, ct.byref(h))
    assert rc in (qsa.QSA_ERR_CUDA, qsa.QSA_ERR_ARG)
    assert L.qsa_last_error(None)
    assert not h.value


def test_invalid_params_rejected(lib):
    """Parameter validation runs before any device call."""
    L = qsa.load_library()
    from paper_2607_24214_b300 import config
    for bad in (dict(nx=100), dict(ny=1024), dict(nxi=0), dict(n_pc_iter=0),
                dict(psi_floor=0.0), dict(dt=-1.0)):
        p = config.c1_fp64_electron_beam().with_(**bad)
        cp = qsa.to_c_params(p)
        h = ct.c_void_p()
        rc = L.qsa_init(ct.byref(cp), None, qsa.ALLOC_FN(), qsa.FREE_FN(), None, ct.byref(h))
        assert rc == qsa.QSA_ERR_ARG, bad
        assert not h.value
