"""The bounds-checked debug build (libqsa_bounds.so, -DQSA_DEBUG_BOUNDS) on cases that drive
every index path of the kernels: the sequential sweep and push, the pipelined launch with a
slipping beam that is lost off the window, particles placed cells away from their lattice
homes in x, y and xi, an odd grid with one plasma particle per cell, a batch of uneven
instances, the tolerance mode, and the allocation-free field solve (whose kernels are compiled
in a source file of their own, with their own counters).  Not one index check may fail.  The library runs in a
child process (one library per process); the release build reports its checks as absent.

This stands in for a memory checker, which is not available here: a failed check records
the source line and skips the access, so an out-of-range index shows up as a count instead
of as a write into a neighbouring buffer."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2607_24214_b300 import config, inputs, qsa
import torch

def run(p, n, move=None, depth=1):
    q = qsa.QSA(p.with_(pipeline_depth=depth))
    bs = inputs.all_beams(p)
    if move is not None:
        move(p, bs)
    for si, b in enumerate(bs):
        q.set_beam(si, b)
    if depth > 1:
        q.advance(n)
    else:
        for _ in range(n):
            q.sweep()
            q.beam_step()
    q.sweep()
    st = q.diagnostics()["status"]
    q.close()
    return st

def scatter(p, bs):
    rng = np.random.default_rng(1)
    for b in bs:
        m = b["x"].size
        b["x"] = np.mod(b["x"] + rng.uniform(-6, 6, m) * p.dx, p.Lx)
        b["y"] = np.mod(b["y"] + rng.uniform(-6, 6, m) * p.dy, p.Ly)
        b["xi"] = np.clip(b["xi"] + rng.uniform(-2.5, 2.5, m) * p.dxi, 0, p.Lxi * (1 - 1e-12))
        b["ux"] = b["ux"] + rng.normal(0, 0.3, m)

c1 = config.c1_fp64_electron_beam().with_(nxi=32, Lxi=4.0)
out = []
out.append(run(c1, 2))
out.append(run(c1.with_(precision="mixed"), 3, depth=4))
import copy
slow = copy.deepcopy(c1).with_(dt=2.0)
slow.species[0].gamma_b = 2.0
slow.species[0].alpha = 1e-3
out.append(run(slow, 6, depth=4))
out.append(run(c1.with_(precision="mixed"), 3, move=scatter, depth=3))
out.append(run(c1, 2, move=scatter))
odd = c1.with_(nx=9, ny=12, Lx=1.8, Ly=2.4, ppc_plasma_x=1, ppc_plasma_y=1, precision="mixed")
out.append(run(odd, 2))
out.append(run(c1.with_(pc_tol=6e-3, n_pc_iter=4, precision="mixed"), 3, depth=3))
ps = [c1.with_(nx=n, ny=n, Lx=n * 0.2, Ly=n * 0.2, seed=i, precision="mixed")
      for i, n in enumerate((16, 24, 12))]
qs = [qsa.QSA(pi) for pi in ps]
qsa.advance_batch(qs, 2)
out += [q.diagnostics()["status"] for q in qs]
# the allocation-free solve, whose kernels sit in another source file with its own counters
import ctypes as ct
lib = qsa.load_library()
for nx, ny in ((96, 64), (1, 32)):
    rng = np.random.default_rng(nx)
    ins = [torch.tensor(rng.normal(size=(ny, nx)), device="cuda") for _ in range(6)]
    o = torch.empty((7, ny, nx), dtype=torch.float64, device="cuda")
    out.append(lib.qsa_field_solve_static(nx, ny, 0.3 * nx, 0.25 * ny, 0.5, 0,
                                          *[ct.c_void_p(t.data_ptr()) for t in ins],
                                          ct.c_void_p(o.data_ptr()), None))
torch.cuda.synchronize()
enabled, first, count = qsa.bounds_check()
print(json.dumps({"status": out, "enabled": enabled, "first_line": first, "count": count}))
'''


@pytest.fixture(scope="module")
def bounds_lib(cuda_ok):
    from paper_2607_24214_b300 import build
    return build.build(bounds=True)


def test_release_build_has_no_checks(cuda_ok):
    from paper_2607_24214_b300 import qsa
    enabled, first, count = qsa.bounds_check()
    assert not enabled and first == 0 and count == 0


@pytest.mark.timeout(900)
def test_no_index_check_fails(bounds_lib):
    env = dict(os.environ, QSA_LIBRARY=bounds_lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CASES], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["enabled"]
    assert res["count"] == 0, res
    assert all(s >= 0 for s in res["status"]), res
