"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test compares the oracle with something that is not the oracle: a closed form, an
independent integrator, a value the paper prints, a conservation law, or the exact lab-frame
Lorentz-force motion of one electron.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import linear_theory as lt
from oracle import qspic
from paper_2607_24214_b300 import config, inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _p(**kw):
    return config.Params(**kw)


# ------------------------------------------------------------------ transverse field solves
@pytest.mark.parametrize("n,mx,my", [(32, 3, 5), (96, 7, 48), (192, 95, 1), (16, 8, 8)])
def test_single_mode_solves(n, mx, my):
    """Source A cos(k.x) gives psi = A cos(k.x)/k^2 and the analogues for E_z, B_z, B_perp
    (spectral operators are exact for grid modes; i k vanishes at the Nyquist index)."""
    L = 2 * math.pi * 1.3
    p = _p(nx=n, ny=n, nxi=4, Lx=L, Ly=L, Lxi=1.0, dt=1.0)
    G = qspic.Grid(p)
    X, Y = np.meshgrid(np.arange(n) * p.dx, np.arange(n) * p.dy)
    kx, ky = 2 * math.pi * mx / L, 2 * math.pi * my / L
    kxd = 0.0 if 2 * mx == n else kx
    kyd = 0.0 if 2 * my == n else ky
    k2 = kx * kx + ky * ky
    ph = kx * X + ky * Y
    c, s = np.cos(ph), np.sin(ph)
    A = 0.37
    psi, gx, gy = qspic.solve_psi(G, A * c)
    np.testing.assert_allclose(psi, A * c / k2, atol=1e-13)
    np.testing.assert_allclose(gx, -A * kxd * s / k2, atol=1e-13)
    np.testing.assert_allclose(gy, -A * kyd * s / k2, atol=1e-13)
    # J_x = a cos, J_y = b cos: div J = -(a kx + b ky) sin -> E_z = (a kx + b ky) sin / k2
    a, b = 0.3, -0.8
    Ez, Bz = qspic.solve_ez_bz(G, a * c, b * c)
    np.testing.assert_allclose(Ez, (a * kxd + b * kyd) * s / k2, atol=1e-13)
    # curl J = d_x J_y - d_y J_x = (-b kx + a ky) sin ; lap B_z = -curl -> B_z = (-b kx + a ky) sin/k2
    np.testing.assert_allclose(Bz, (-b * kxd + a * kyd) * s / k2, atol=1e-13)
    # B_perp with a D source and kappa^2 = 0.7 (fixed point B_old = B)
    Jz, Dx, Dy = 0.5 * c, 0.2 * s, -0.4 * c
    rhs_x = 0.5 * kyd * s + 0.4 * c          # -d_y J_z - D_y
    rhs_y = -0.5 * kxd * s + 0.2 * s         # d_x J_z + D_x
    Bx_ex, By_ex = -rhs_x / k2, -rhs_y / k2  # lap -> -k^2 on a single mode
    Bx, By = qspic.solve_bperp(G, Jz, Dx, Dy)
    np.testing.assert_allclose(Bx, Bx_ex, atol=1e-13)
    np.testing.assert_allclose(By, By_ex, atol=1e-13)
    Bx2, By2 = qspic.solve_bperp(G, Jz, Dx, Dy, 0.7, Bx_ex, By_ex)
    np.testing.assert_allclose(Bx2, Bx_ex, atol=1e-13)
    np.testing.assert_allclose(By2, By_ex, atol=1e-13)


def test_deposit_gather_conservation():
    """CIC deposit conserves charge; gather of a linear-in-cell field is exact inside a cell."""
    rng = np.random.default_rng(3)
    p = _p(nx=12, ny=9, nxi=2, Lx=3.0, Ly=2.0, Lxi=1.0, dt=1.0)
    G = qspic.Grid(p)
    x, y, q = rng.uniform(0, 3, 500), rng.uniform(0, 2, 500), rng.normal(size=500)
    rho = qspic.deposit(G, x, y, q)
    assert abs(rho.sum() * p.dx * p.dy - q.sum()) < 1e-12
    # a single particle at a node puts all of its charge there
    r1 = qspic.deposit(G, np.array([4 * p.dx]), np.array([3 * p.dy]), np.array([1.0]))
    assert abs(r1[3, 4] * p.dx * p.dy - 1.0) < 1e-14


# ------------------------------------------------------------------ xi-push: exact orbits
def _potential_fields(t_xyz):
    """Analytic potentials of (x, y, xi) with xi = t - z, zero with zero xi-derivative at
    xi = 0 (unperturbed plasma ahead of fields that rise smoothly), and the fields they give: E = -grad phi - d_t A, B = curl A, with
    d_t = d_xi, d_z = -d_xi."""
    a, b, c, d = 0.03, 0.02, 0.015, 0.01

    def pot(x, y, xi):
        phi = a * math.cos(x) * math.sin(0.7 * xi) ** 2 + 0.02 * math.sin(0.5 * xi) ** 2
        Az = b * math.sin(y) * math.sin(0.6 * xi) ** 2
        Ax = c * math.sin(0.5 * xi) ** 2 * math.cos(y)
        Ay = d * math.cos(x) * math.sin(0.4 * xi) ** 2
        return phi, Ax, Ay, Az

    def fields(x, y, xi, h=1e-5):
        def dd(f, i):
            e = [0.0, 0.0, 0.0]
            e[i] = h
            return (np.array(pot(x + e[0], y + e[1], xi + e[2])) -
                    np.array(pot(x - e[0], y - e[1], xi - e[2]))) / (2 * h)
        dX, dY, dXI = dd(None, 0), dd(None, 1), dd(None, 2)     # d of (phi, Ax, Ay, Az)
        # d_z = -d_xi, d_t = d_xi
        Ex = -dX[0] - dXI[1]
        Ey = -dY[0] - dXI[2]
        Ez = dXI[0] - dXI[3]
        Bx = dY[3] + dXI[2]          # d_y A_z - d_z A_y
        By = -dXI[1] - dX[3]         # d_z A_x - d_x A_z
        Bz = dX[2] - dY[1]
        psi = pot(x, y, xi)[0] - pot(x, y, xi)[3]
        gpx, gpy = dX[0] - dX[3], dY[0] - dY[3]
        return (Ex, Ey, Ez), (Bx, By, Bz), psi, (gpx, gpy)
    return fields


def test_xi_push_matches_lab_frame_lorentz_motion():
    """An electron starting at rest ahead of the fields, integrated in lab time t with
    du/dt = -(E + v x B), must follow the xi-push of the quasistatic equations (signs of every
    term, the invariant gamma - u_z = 1 + psi, dx/dxi = u/(1+psi)); O(dxi^2) agreement."""
    fields = _potential_fields(None)

    def rhs(t, s):
        x, y, z, ux, uy, uz = s
        g = math.sqrt(1 + ux * ux + uy * uy + uz * uz)
        v = np.array([ux, uy, uz]) / g
        E, B, _, _ = fields(x, y, t - z)
        f = -(np.array(E) + np.cross(v, B))
        return [v[0], v[1], v[2], f[0], f[1], f[2]]

    x0, y0 = 0.4, -0.3
    xi_end = 6.0
    sol = solve_ivp(rhs, [0, 20.0], [x0, y0, 0.0, 0, 0, 0], rtol=1e-11, atol=1e-13,
                    dense_output=True, method="DOP853")
    # find t where xi = t - z reaches xi_end
    ts = np.linspace(0, 20, 20001)
    xis = ts - sol.sol(ts)[2]
    t_end = np.interp(xi_end, xis, ts)
    X = sol.sol(t_end)
    _, _, psi_end, _ = fields(X[0], X[1], xi_end)
    g_end = math.sqrt(1 + X[3] ** 2 + X[4] ** 2 + X[5] ** 2)
    assert abs(g_end - X[5] - (1 + psi_end)) < 1e-8          # invariant in the lab solution

    errs = []
    for nst in (300, 600):
        dxi = xi_end / nst
        x, y, ux, uy = np.array([x0]), np.array([y0]), np.zeros(1), np.zeros(1)
        psi_prev = np.zeros(1)
        for j in range(nst):
            _, B, psi, gp = fields(x[0], y[0], j * dxi)
            opp = np.array([1 + psi])
            opph = 1 + 0.5 * (3 * psi - psi_prev)
            uxh, uyh = qspic.push_xi(ux, uy, opp, np.array([gp[0]]), np.array([gp[1]]),
                                     np.array([B[0]]), np.array([B[1]]), np.array([B[2]]), dxi)
            x, y = x + dxi * uxh / opph, y + dxi * uyh / opph
            ux, uy, psi_prev = uxh, uyh, np.array([psi])
        # u^{N-1/2} vs u(xi_end - dxi/2) of the lab solution
        th = np.interp(xi_end - 0.5 * dxi, xis, ts)
        Xh = sol.sol(th)
        errs.append(max(abs(x[0] - X[0]), abs(y[0] - X[1]), abs(ux[0] - Xh[3]), abs(uy[0] - Xh[4])))
    assert errs[1] < 2e-5
    assert errs[0] / errs[1] > 3.0            # second order in dxi


def test_xi_push_uniform_fields():
    """B_z alone rotates u_perp counter-clockwise by exactly 2 atan(dxi B_z/(2(1+psi))) per
    slice with |u| conserved; B_x alone gives du_y/dxi = B_x exactly."""
    opp = np.array([1.3])
    u0 = np.array([0.2]), np.array([-0.1])
    Bz, dxi = 0.8, 0.1
    ux, uy = qspic.push_xi(u0[0], u0[1], opp, np.zeros(1), np.zeros(1), np.zeros(1),
                           np.zeros(1), np.array([Bz]), dxi)
    ang = math.atan2(uy[0], ux[0]) - math.atan2(u0[1][0], u0[0][0])
    assert abs(ang - 2 * math.atan(dxi * Bz / (2 * 1.3))) < 1e-14
    assert abs(math.hypot(ux[0], uy[0]) - math.hypot(0.2, -0.1)) < 1e-15
    ux, uy = qspic.push_xi(np.zeros(1), np.zeros(1), opp, np.zeros(1), np.zeros(1),
                           np.array([0.25]), np.zeros(1), np.zeros(1), dxi)
    assert ux[0] == 0.0 and abs(uy[0] - 0.25 * dxi) < 1e-16


def test_invariant_mass_shell():
    """gamma and u_z rebuilt from (u_perp, 1+psi) lie on the mass shell and satisfy
    gamma - u_z = 1 + psi (paper's QSA with psi = -Psi)."""
    rng = np.random.default_rng(0)
    ux, uy = rng.normal(0, 0.3, 1000), rng.normal(0, 0.3, 1000)
    opp = rng.uniform(0.2, 3.0, 1000)
    g = qspic.gamma_from_invariant(ux, uy, opp)
    uz = qspic.uz_from_invariant(ux, uy, opp)
    np.testing.assert_allclose(g * g - uz * uz - ux * ux - uy * uy, 1.0, rtol=1e-13)
    np.testing.assert_allclose(g - uz, opp, rtol=1e-13)
    # plasma electron in constant psi, no fields: stays at rest
    a, b = qspic.push_xi(np.zeros(3), np.zeros(3), opp[:3], np.zeros(3), np.zeros(3),
                         np.zeros(3), np.zeros(3), np.zeros(3), 0.1)
    assert not a.any() and not b.any()


# ------------------------------------------------------------------ beam push orbits
def _uniform_slab(p, **vals):
    slab = np.zeros((p.nxi + 1, 6, p.ny, p.nx))
    for i, name in enumerate(qspic.FIELD_NAMES):
        slab[:, i] = vals.get(name, 0.0)
    return slab


def _one_particle(p, **kw):
    b = dict(x=np.array([1.0]), y=np.array([1.0]), xi=np.array([0.5]), ux=np.zeros(1),
             uy=np.zeros(1), uz=np.array([100.0]), w=np.array([1.0]))
    b.update({k: np.array([v]) for k, v in kw.items()})
    return b


def test_beam_uniform_ez_exact():
    p = _p(nx=4, ny=4, nxi=8, Lx=4.0, Ly=4.0, Lxi=8.0, dt=7.0,
           species=[config.Species(Z=-1, M=1)])
    slab = _uniform_slab(p, Ez=0.01)
    b = [_one_particle(p)]
    for _ in range(5):
        qspic.beam_push(p, b, slab)
    assert abs(b[0]["uz"][0] - (100.0 - 5 * 7.0 * 0.01)) < 1e-12
    assert b[0]["ux"][0] == 0.0


def test_beam_uniform_bz_boris_angle():
    p = _p(nx=4, ny=4, nxi=8, Lx=4.0, Ly=4.0, Lxi=8.0, dt=3.0,
           species=[config.Species(Z=1, M=2.0)])
    slab = _uniform_slab(p, Bz=0.05)
    b = [_one_particle(p, ux=0.3, uz=20.0)]
    g = math.sqrt(1 + 0.09 + 400)
    qspic.beam_push(p, b, slab)
    ang = math.atan2(b[0]["uy"][0], b[0]["ux"][0])
    t = 0.5 * 1 * 3.0 / 2.0 * 0.05 / g
    assert abs(ang + 2 * math.atan(t)) < 1e-14            # clockwise for a positive charge
    assert abs(math.hypot(b[0]["ux"][0], b[0]["uy"][0]) - 0.3) < 1e-15


def test_beam_focusing_leapfrog_closed_form():
    """Small transverse oscillation in W_x = -A sin(k x) ~ -A k x: with u^{-1/2} = 0 the beam
    leapfrog is the recurrence x_{n+1} - 2 x_n + x_{n-1} = -(omega dt)^2 x_n, x_1 = x_0 (1 -
    (omega dt)^2), omega^2 = Z A k/(gamma M), whose closed form is
    x_n = x_0 [cos(n th) - (omega dt)^2 sin(n th) / (2 sin th)], cos th = 1 - (omega dt)^2/2."""
    L = 8.0
    p = _p(nx=64, ny=4, nxi=8, Lx=L, Ly=4.0, Lxi=8.0, dt=4.0, species=[config.Species(Z=1, M=1)])
    k = 2 * math.pi / L
    X = np.arange(p.nx) * p.dx
    slab = np.zeros((p.nxi + 1, 6, p.ny, p.nx))
    A = 1e-2
    slab[:, 0] = -A * np.sin(k * X)[None, None, :]
    gam0 = 1000.0
    x0 = 1e-4
    b = [_one_particle(p, x=x0, uz=gam0)]
    om = math.sqrt(A * k / gam0)
    c = (om * p.dt) ** 2
    th = math.acos(1 - c / 2)
    for n in range(1, 60):
        qspic.beam_push(p, b, slab)
        xs = b[0]["x"][0]
        xs = xs - L if xs > L / 2 else xs
        ex = x0 * (math.cos(n * th) - c * math.sin(n * th) / (2 * math.sin(th)))
        assert abs(xs - ex) < 1e-3 * x0


# ------------------------------------------------------------------ plasma sweep pins
def _uniform_beam(p):
    for s in p.species:
        s.noise_rel = 0.0
        s.uperp_spread = 0.0
        s.gamma_spread_rel = 0.0
    return inputs.all_beams(p)


def test_wake_1d_second_order():
    """Uniform electron beam: the k = 0 mode obeys psi'' = [(1+psi)^-2 - 1]/2 + n_b v_z; the
    mean psi0 converges to the high-order ODE solution at second order in dxi."""
    errs = []
    for nxi in (64, 128):
        p = config.c1_fp64_electron_beam().with_(nx=4, ny=4, Lx=math.pi / 4, Ly=math.pi / 4,
                                                 nxi=nxi)
        slab, d = qspic.plasma_sweep(p, qspic.beam_sources(p, _uniform_beam(p)))
        xs = np.arange(nxi + 1) * p.dxi
        vz = math.sqrt(1 - 1 / 100.0 ** 2)
        psi, ez = lt.wake_1d(xs, 0.1 * vz)
        errs.append(np.abs(psi - d["psi0"]).max())
        inner = slice(2, nxi - 1)
        assert np.abs(ez - d["ez0"])[inner].max() < 0.02 * 64 / nxi
    assert errs[1] < 1e-4
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_linear_wake_small_beam():
    """alpha -> 0: psi0 = alpha (1 - cos xi), E_z0 = alpha sin xi (Eq. 1 with k = 0)."""
    p = config.c1_fp64_electron_beam().with_(nx=4, ny=4, Lx=math.pi / 4, Ly=math.pi / 4, nxi=128)
    p.species[0].alpha = 1e-6
    slab, d = qspic.plasma_sweep(p, qspic.beam_sources(p, _uniform_beam(p)))
    xs = np.arange(p.nxi + 1) * p.dxi
    np.testing.assert_allclose(d["psi0"], 1e-6 * (1 - np.cos(xs)), atol=2e-9)   # O(dxi^2)


def test_single_mode_linear_response():
    """Frozen pair beam with the electron weights seeded by eps cos(k y): the plasma response is
    psi^ = -rho^_b1 (1 - cos xi)/(k^2+1) (Eqs. 1-2) and the screened beam field
    B^_x = i k_y J^_zb/(k^2+1)."""
    p = config.v_pair_single_mode(Lxi=12.0)
    k = 2 * math.pi * 2 / p.Ly
    eps, alpha = p.modes[0].amplitude, p.species[0].alpha
    slab, d = qspic.plasma_sweep(p, qspic.beam_sources(p, inputs.all_beams(p)))
    xs = np.arange(p.nxi + 1) * p.dxi
    Wy = np.fft.fft(slab[:, 1, :, 0], axis=1)[:, 2] / p.ny       # coefficient of e^{iky}
    Bx = np.fft.fft(slab[:, 3, :, 0], axis=1)[:, 2] / p.ny
    rho1 = -alpha * eps / 2                                       # electrons: Z = -1
    psi_ex = -rho1 * (1 - np.cos(xs)) / (k * k + 1)
    sel = slice(8, -1)            # the last node holds half a cell of beam
    # W_y = -i k psi
    np.testing.assert_allclose(Wy[sel], -1j * k * psi_ex[sel], rtol=5e-3, atol=1e-3 * k * abs(rho1))
    vz = math.sqrt(1 - 1 / 1e3 ** 2)
    np.testing.assert_allclose(Bx[sel], 1j * k * rho1 * vz / (k * k + 1), rtol=5e-3)


def test_sweep_invariants_c1():
    """C1 sweep: invariant to 1e-12 per slice, quasistatic charge conservation
    sum(rho - J_z)_e dx dy = -Lx Ly to 1e-13 relative, E_z = d_xi psi to O(dxi^2)."""
    p = config.c1_fp64_electron_beam()
    slab, d = qspic.plasma_sweep(p, qspic.beam_sources(p, inputs.all_beams(p)), return_psi=True)
    assert d["invariant"].max() < 1e-12
    assert d["charge"].max() < 1e-13 * p.Lx * p.Ly
    assert d["n_floor"].sum() == 0
    psi = d["psi"]
    dpsi = (psi[2:] - psi[:-2]) / (2 * p.dxi)
    ez = slab[1:-1, 2]
    err = np.abs(dpsi - ez)[4:-2].max()
    assert err < 0.01 * np.abs(ez).max()


def test_beam_deposit_conserves_charge():
    p = config.c1_fp64_electron_beam()
    beams = inputs.all_beams(p)
    src = qspic.beam_sources(p, beams)
    tot = (src[0] + src[1]).sum() * p.dx * p.dy * p.dxi       # rho = S_b + J_zb
    assert abs(tot - (-1) * beams[0]["w"].sum()) < 1e-12 * abs(tot)


# ------------------------------------------------------------------ linear theory
def test_gamma_worked_example():
    g = GOLDEN["gamma_fig1e"]
    sp = [config.Species(**s) for s in g["species"]]
    assert abs(lt.growth_rate(g["k"], sp) / g["value"] - 1) < g["rel_tol"]


def test_series_h1_is_step_wake_and_matches_march():
    xs = np.linspace(0, 20, 9)
    for x in xs:
        assert abs(lt.psi_series(x, 0.0) + (1 - math.cos(x)) / 2.0) < 1e-14
    G = 4e-3
    grid = np.linspace(0, 21, 21 * 128 + 1)
    m = lt.march_eq5(grid, 4.0 / G, 400, G, k=1.0)
    for x in (2.0, 10.0, 20.0):
        s = lt.psi_series(x, 4.0, k=1.0)
        assert abs(m[int(round(x * 128))] / s - 1) < 2e-4


def test_asymptotic_exponents():
    """Far from the front the local growth exponent of the exact Eq. 5 solution approaches
    Eq. 6; near the front it approaches Eq. 7 (asymptotic: 15%)."""
    for xi, expo, Gt1, Gt2 in ((40.0, lt.exponent_rear, 8.0, 10.0),
                               (2.0, lt.exponent_front, 30.0, 40.0)):
        d_exact = math.log(abs(lt.psi_series(xi, Gt2))) - math.log(abs(lt.psi_series(xi, Gt1)))
        d_asym = expo(Gt2, xi) - expo(Gt1, xi)
        assert abs(d_exact / d_asym - 1) < 0.15


def test_saturation_arithmetic_and_extent():
    g = GOLDEN["cfi_saturation_blazar"]
    sp = [config.Species(Z=-1, alpha=g["alpha"], gamma_b=g["gamma_b"]),
          config.Species(Z=1, alpha=g["alpha"], gamma_b=g["gamma_b"])]
    Gam = lt.growth_rate(g["k_y"], sp)
    gst = lt.local_rate_front(Gam, g["xi"], g["tau_sat"])
    eps_bz = (1 / g["k_y"]) ** 2 * (g["xi"] / g["tau_sat"]) ** 2 / 4
    assert abs(eps_bz / g["eps_Bz"] - 1) < g["rel_tol"]
    assert abs(g["gamma_b"] * gst / g["k_y"] / g["dpy"] - 1) < g["rel_tol"]
    o = GOLDEN["otsi_saturation_blazar"]
    gst = lt.local_rate_rear(Gam, o["xi"], o["tau_sat"])
    assert abs(o["gamma_b"] * gst / o["k_y"] / o["dpy"] - 1) < o["rel_tol"]
    e = (9 / (64 * o["k_y"] ** 2)) * (o["alpha"] / o["gamma_b"]) ** (1 / 3) \
        * (o["xi"] / o["tau_sat"]) ** (4 / 3)
    assert abs(e / o["eps_Ey"] - 1) < o["rel_tol"]
    c = GOLDEN["cfi_extent"]
    assert abs(lt.transition_xi(10.0) / 10.0 - c["value"]) < c["abs_tol"]


# ------------------------------------------------------------------ direct pins of helpers
def test_gather_exact_on_bilinear_fields_and_adjoint_to_deposit():
    """CIC gather reproduces a field that is bilinear in (x, y) exactly inside every cell
    (bilinear interpolation of a bilinear function), and it is the transpose of the deposit:
    sum over nodes deposit(q) F dx dy = sum over particles q gather(F)."""
    rng = np.random.default_rng(11)
    p = _p(nx=10, ny=7, nxi=2, Lx=2.5, Ly=1.4, Lxi=1.0, dt=1.0)
    G = qspic.Grid(p)
    X, Y = np.meshgrid(np.arange(p.nx) * p.dx, np.arange(p.ny) * p.dy)
    a, b, c, d = 0.3, -1.7, 2.2, 0.9
    F = a + b * X + c * Y + d * X * Y
    # points whose cell does not wrap (the bilinear function is not periodic)
    x = rng.uniform(0, (p.nx - 1) * p.dx, 400)
    y = rng.uniform(0, (p.ny - 1) * p.dy, 400)
    np.testing.assert_allclose(qspic.gather(G, F, x, y), a + b * x + c * y + d * x * y,
                               rtol=0, atol=1e-13)
    # adjointness on arbitrary (periodic) positions and a random field
    xs, ys = rng.uniform(0, p.Lx, 300), rng.uniform(0, p.Ly, 300)
    q = rng.normal(size=300)
    Fr = rng.normal(size=(p.ny, p.nx))
    lhs = (qspic.deposit(G, xs, ys, q) * Fr).sum() * p.dx * p.dy
    rhs = (q * qspic.gather(G, Fr, xs, ys)).sum()
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


def test_beam_source_slots_of_one_particle():
    """One beam particle on a node (x = i dx, y = j dy, xi = k dxi) puts its whole charge on
    that node: S_b = Z w (1 - v_z), J_z = Z w v_z, J_x = Z w v_x, J_y = Z w v_y, each divided
    by dx dy dxi, with v = u/gamma (the source terms of the field equations); 1 - v_z is
    compared with its value from u_z/gamma in 50-digit arithmetic."""
    import mpmath
    sp = config.Species(Z=-2.0, M=3.0)
    p = _p(nx=6, ny=5, nxi=8, Lx=3.0, Ly=2.5, Lxi=4.0, dt=1.0, species=[sp])
    i, j, k = 2, 3, 5
    ux, uy, uz, w = 0.7, -1.3, 40.0, 0.25
    b = [dict(x=np.array([i * p.dx]), y=np.array([j * p.dy]), xi=np.array([k * p.dxi]),
              ux=np.array([ux]), uy=np.array([uy]), uz=np.array([uz]), w=np.array([w]))]
    src = qspic.beam_sources(p, b)
    vol = p.dx * p.dy * p.dxi
    with mpmath.workdps(50):
        g = mpmath.sqrt(1 + mpmath.mpf(ux) ** 2 + mpmath.mpf(uy) ** 2 + mpmath.mpf(uz) ** 2)
        omv = float(1 - mpmath.mpf(uz) / g)
        gam = float(g)
    want = sp.Z * w / vol * np.array([omv, uz / gam, ux / gam, uy / gam])
    for s in range(4):
        assert abs(src[s, k, j, i] - want[s]) <= 1e-14 * abs(want[s]), s
        rest = src[s].copy()
        rest[k, j, i] = 0.0
        assert not rest.any(), s
    # a particle halfway between two xi nodes splits each slot evenly between them
    b[0]["xi"] = np.array([(k + 0.5) * p.dxi])
    src = qspic.beam_sources(p, b)
    np.testing.assert_allclose(src[2, k:k + 2, j, i], 0.5 * want[2], rtol=1e-13)


def test_gamma_otsi_is_the_maximum_temporal_rate():
    """The temporal oblique-two-stream rate quoted after Eq. 6 is the largest growth rate of
    the temporal dispersion relation of the beam-plasma system that Eq. 5 reduces: with the
    plasma operator left without the quasistatic approximation (d_t = d_xi + d_tau), a mode
    exp(-i k xi + sigma tau) obeys ((sigma - i k)^2 + 1) sigma^2 = Gamma^2.  Its roots are
    found with numpy (companion matrix) and maximised over k near the plasma resonance; the
    result tends to sqrt(3)/2^(4/3) Gamma^(2/3) as Gamma -> 0 (relative corrections
    O(Gamma^(2/3)))."""
    for G in (1e-6, 1e-5):
        best = 0.0
        for k in 1.0 + np.linspace(-0.05, 0.05, 2001) * G ** (2.0 / 3.0) * 20:
            # sigma^4 - 2 i k sigma^3 + (1 - k^2) sigma^2 - Gamma^2 = 0
            r = np.roots([1.0, -2j * k, 1.0 - k * k, 0.0, -G * G])
            best = max(best, r.real.max())
        assert abs(best / lt.gamma_otsi(G) - 1) < 3 * G ** (2.0 / 3.0) + 1e-4, (G, best)


def test_field_energy_of_single_modes():
    """Per-slice energies 1/2 sum F^2 dx dy dxi for fields whose energy is known in closed
    form: B_x = A cos(k.x) gives A^2 Lx Ly dxi / 4; W_x = a, B_y = b (so E_x = a + b) gives
    (a + b)^2 Lx Ly dxi / 2 in E_x and b^2 Lx Ly dxi / 2 in B_y; W_y = c, B_x = 0 gives E_y = c."""
    p = _p(nx=12, ny=8, nxi=3, Lx=3.0, Ly=2.0, Lxi=1.5, dt=1.0)
    X, Y = np.meshgrid(np.arange(p.nx) * p.dx, np.arange(p.ny) * p.dy)
    slab = np.zeros((p.nxi + 1, 6, p.ny, p.nx))
    A = 0.7
    slab[1, 3] = A * np.cos(2 * math.pi * (2 * X / p.Lx + 3 * Y / p.Ly))
    a, b, c = 0.2, -0.5, 0.3
    slab[2, 0], slab[2, 4], slab[2, 1] = a, b, c
    e = qspic.field_energy(p, slab)
    area = p.Lx * p.Ly
    want = np.zeros((p.nxi + 1, 6))
    want[1, 3] = A * A * area * p.dxi / 4          # B_x (and E_y = W_y - B_x = -B_x)
    want[1, 1] = A * A * area * p.dxi / 4
    want[2, 0] = (a + b) ** 2 * area * p.dxi / 2   # E_x = W_x + B_y
    want[2, 4] = b * b * area * p.dxi / 2
    want[2, 1] = c * c * area * p.dxi / 2          # E_y = W_y - B_x
    np.testing.assert_allclose(e, want, rtol=0, atol=1e-14)
