"""Seeded input generator: Philox-4x32-10 known-answer vectors (Salmon et al., SC'11, the
Random123 distribution's kat vectors) and the beam lattice layout."""
import numpy as np

from paper_2607_24214_b300 import config, inputs

KAT = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
       ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
       ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
        (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]


def test_philox_known_answers():
    for ctr, key, want in KAT:
        got = inputs.philox4x32_10(*[np.array([c], dtype=np.uint32) for c in ctr], *key)
        assert tuple(int(g[0]) for g in got) == want


def test_beam_lattice_and_weights():
    p = config.c1_fp64_electron_beam()
    b = inputs.beam_arrays(p, 0)
    s = p.species[0]
    assert b["x"].size == inputs.beam_count(p, 0) == 32 * 32 * 64 * 8
    # total weight = alpha * box volume (noise averages out)
    vol = p.Lx * p.Ly * p.Lxi
    assert abs(b["w"].sum() / (s.alpha * vol) - 1) < 1e-4
    assert np.all((b["x"] > 0) & (b["x"] < p.Lx) & (b["xi"] > 0) & (b["xi"] < p.Lxi))
    g = np.sqrt(1 + b["ux"] ** 2 + b["uy"] ** 2 + b["uz"] ** 2)
    np.testing.assert_allclose(g, 100.0, rtol=1e-12)
    assert abs(b["ux"].std() / 1e-3 - 1) < 0.01
    # a slice of ids equals the same ids of the full array
    part = inputs.beam_arrays(p, 0, 1000, 2000)
    for k in b:
        np.testing.assert_array_equal(part[k], b[k][1000:2000])
