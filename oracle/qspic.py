"""FP64 CPU oracle of the quasistatic PIC (QS-PIC) hot path.  TEST INFRASTRUCTURE ONLY.

Only the tests, the graft entry's smoke() and the benchmark's CPU-baseline leg may import
this module.  It shares no code with the CUDA path and imports nothing from it: it takes a
parameter object (duck-typed: nx, ny, nxi, Lx, Ly, Lxi, dt, species, ppc_plasma_x/y,
n_pc_iter, psi_floor) and plain fp64 beam arrays.

What it computes
----------------
The paper (section "Quasistatic model") changes to comoving variables (xi, tau) = (ct - x, t)
and lets fields depend on xi faster than on tau; its QS-PIC runs (QuaSSis paragraph) use a
transversely periodic box and random macroparticle weights.  The paper prints only the
linearised system (Eqs. 1-5); the nonlinear equations below are Maxwell's equations in Lorenz
gauge and the cold-electron Lorentz force with d/dt = d/dxi, d/dz = -d/dxi, in normalised
units (z is the propagation axis, psi = phi - A_z = -Psi of the paper, Eq. 2):

  lap psi = -(rho - J_z)            E_x - B_y = -d_x psi,  E_y + B_x = -d_y psi
  lap E_z = div J_perp              E_z = d_xi psi
  lap B_z = -(d_x J_y - d_y J_x)
  lap B_x = -d_y J_z - d_xi J_y     lap B_y = d_x J_z + d_xi J_x        (lap = transverse)

Plasma electrons (charge -1, mass 1) obey, with the quasistatic invariant gamma - u_z = 1 + psi,

  du_x/dxi = gamma d_x psi/(1+psi) - B_y - u_y B_z/(1+psi)
  du_y/dxi = gamma d_y psi/(1+psi) + B_x + u_x B_z/(1+psi)
  dx_perp/dxi = u_perp/(1+psi),  gamma = (1 + u_perp^2 + (1+psi)^2) / (2(1+psi)),
  u_z = (1 + u_perp^2 - (1+psi)^2) / (2(1+psi)),

and a macroparticle of quasistatic weight w carries rho - J_z = -w, J = -w u/(1+psi).
Linearising this system gives back the paper's Eqs. 1 and 2 (a unit test checks it through the
simulated single-mode response).  The k_perp = 0 part of the fields obeys dE_z0/dxi = -<J_z>,
dpsi0/dxi = E_z0 with zero data ahead of the beam; mean transverse fields are zero.

Discrete scheme (the readings are listed in the design notes):
  * nodes at (i dx, j dy), periodic; CIC deposit/gather; grid density = sum q W / (dx dy);
  * transverse operators spectral (numpy.fft, forward unnormalised); i k zeroed at Nyquist;
    the k = 0 mode dropped from the transverse solves;
  * plasma re-initialised at xi = 0 on a quiet lattice, w = dx dy / ppc, u = 0;
  * xi leapfrog: x at slices j, u at half slices; Boris-type push (half kick, exact-angle
    rotation by B_z/(1+psi), half kick, gamma/(1+psi) of both kicks taken at the predicted
    pre-rotation momentum); x^{j+1} = x^j + dxi u^{j+1/2}/(1+psi^{j+1/2}) with
    1+psi^{j+1/2} extrapolated per particle as 1 + (3 psi_p^j - psi_p^{j-1})/2;
  * B_perp from a predictor-corrector of n_pc_iter field solves per slice, d_xi J_perp =
    (J_perp^{j+1/2} - J_perp^{j-1/2})/dxi, J_perp^{j+1/2} deposited at x^{j+1/2}; each solve is
    shifted by kappa^2 = <w/(1+psi_p)> / (Lx Ly): (k^2 + kappa^2) B_new = rhs + kappa^2 B_old;
    with pc_tol > 0 (the corrector iterated to convergence instead of a fixed count) the
    solves stop after the first whose change ||B_new - B_old|| / ||B_new|| (2-norms over the
    grid) is below pc_tol, or is zero, after n_pc_iter solves at most;
  * mean mode by leapfrog in xi (FP64 scalars);
  * beam: Boris in tau with step dt, fields trilinear from the slab of slices 0..nxi,
    lost when xi >= Lxi; beam sources deposited CIC x linear-in-xi with velocities u/gamma.
"""
from __future__ import annotations

import numpy as np

FIELD_NAMES = ("Wx", "Wy", "Ez", "Bx", "By", "Bz")   # Wx = E_x - B_y, Wy = E_y + B_x


# ----------------------------------------------------------------------------------------
# grid helpers
# ----------------------------------------------------------------------------------------
def wavenumbers(n, L):
    """Angular wavenumbers of an n-point periodic grid of length L (numpy.fft order), and the
    same array with the Nyquist entry zeroed (the first-derivative symbol)."""
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=L / n)
    kd = k.copy()
    if n % 2 == 0:
        kd[n // 2] = 0.0
    return k, kd


class Grid:
    def __init__(self, p):
        self.nx, self.ny = p.nx, p.ny
        self.dx, self.dy = p.Lx / p.nx, p.Ly / p.ny
        self.Lx, self.Ly = p.Lx, p.Ly
        kx, kxd = wavenumbers(p.nx, p.Lx)
        ky, kyd = wavenumbers(p.ny, p.Ly)
        self.KX, self.KY = np.meshgrid(kx, ky)          # [ny, nx]
        self.IKX, self.IKY = np.meshgrid(1j * kxd, 1j * kyd)
        self.K2 = self.KX ** 2 + self.KY ** 2
        self.zero = self.K2 == 0.0
        self.invK2 = np.where(self.zero, 0.0, 1.0 / np.where(self.zero, 1.0, self.K2))


def cic_1d(pos, n, d):
    """Cloud-in-cell nodes and weights along one periodic axis: node floor(pos/d) gets 1-f,
    the next node gets f."""
    g = pos / d
    i0 = np.floor(g)
    f = g - i0
    i0 = i0.astype(np.int64) % n
    return i0, (i0 + 1) % n, 1.0 - f, f


def deposit(G, x, y, q):
    """Grid density [ny, nx] of the charges q at (x, y): sum q W / (dx dy)."""
    ix0, ix1, wx0, wx1 = cic_1d(x, G.nx, G.dx)
    iy0, iy1, wy0, wy1 = cic_1d(y, G.ny, G.dy)
    out = np.zeros(G.ny * G.nx)
    for iy, wy in ((iy0, wy0), (iy1, wy1)):
        for ix, wx in ((ix0, wx0), (ix1, wx1)):
            out += np.bincount(iy * G.nx + ix, weights=q * wy * wx, minlength=G.ny * G.nx)
    return out.reshape(G.ny, G.nx) / (G.dx * G.dy)


def gather(G, F, x, y):
    """CIC interpolation of the grid field F [ny, nx] at (x, y)."""
    ix0, ix1, wx0, wx1 = cic_1d(x, G.nx, G.dx)
    iy0, iy1, wy0, wy1 = cic_1d(y, G.ny, G.dy)
    return (F[iy0, ix0] * wy0 * wx0 + F[iy0, ix1] * wy0 * wx1
            + F[iy1, ix0] * wy1 * wx0 + F[iy1, ix1] * wy1 * wx1)


def fwd(F):
    return np.fft.fft2(F)


def inv(Fh):
    return np.fft.ifft2(Fh).real


# ----------------------------------------------------------------------------------------
# transverse field solves (k != 0), spectral
# ----------------------------------------------------------------------------------------
def solve_psi(G, S):
    """lap psi = -S (S = rho - J_z total): psi^ = S^/k^2; returns psi, d_x psi, d_y psi."""
    Ph = fwd(S) * G.invK2
    return inv(Ph), inv(G.IKX * Ph), inv(G.IKY * Ph)


def solve_ez_bz(G, Jx, Jy):
    """lap E_z = div J_perp  ->  E_z^ = -(i k . J^)/k^2;
    lap B_z = -(d_x J_y - d_y J_x)  ->  B_z^ = (i k_x J_y^ - i k_y J_x^)/k^2."""
    Jxh, Jyh = fwd(Jx), fwd(Jy)
    Ez = inv(-(G.IKX * Jxh + G.IKY * Jyh) * G.invK2)
    Bz = inv((G.IKX * Jyh - G.IKY * Jxh) * G.invK2)
    return Ez, Bz


def solve_bperp(G, Jz, Dx, Dy, kappa2=0.0, Bx_old=None, By_old=None):
    """lap B_x = -d_y J_z - D_y,  lap B_y = d_x J_z + D_x  (D = d_xi J_perp), solved as
    (k^2 + kappa^2) B^ = rhs^ + kappa^2 B_old^ at k != 0; B^(0) = 0."""
    Jzh, Dxh, Dyh = fwd(Jz), fwd(Dx), fwd(Dy)
    rx = G.IKY * Jzh + Dyh
    ry = -(G.IKX * Jzh + Dxh)
    if kappa2 != 0.0:
        rx = rx + kappa2 * fwd(Bx_old)
        ry = ry + kappa2 * fwd(By_old)
    den = G.K2 + kappa2
    invden = np.where(G.zero, 0.0, 1.0 / np.where(G.zero, 1.0, den))
    return inv(rx * invden), inv(ry * invden)


# ----------------------------------------------------------------------------------------
# plasma electrons: xi push
# ----------------------------------------------------------------------------------------
def gamma_over_opp(ux, uy, opp):
    """gamma/(1+psi) from the quasistatic invariant."""
    return (1.0 + ux * ux + uy * uy + opp * opp) / (2.0 * opp * opp)


def uz_from_invariant(ux, uy, opp):
    return (1.0 + ux * ux + uy * uy - opp * opp) / (2.0 * opp)


def gamma_from_invariant(ux, uy, opp):
    return (1.0 + ux * ux + uy * uy + opp * opp) / (2.0 * opp)


def push_xi(ux, uy, opp, gx, gy, Bx, By, Bz, dxi):
    """u^{j-1/2} -> u^{j+1/2} with fields of slice j gathered at x^j.

    du/dxi = g(u) grad psi + (-B_y, B_x) + (B_z/(1+psi)) (-u_y, u_x),  g = gamma/(1+psi).
    Boris-type split: half kick, rotation of angle 2 atan(dxi B_z/(2(1+psi))) counter-clockwise,
    half kick.  The rotation keeps |u_perp|, so g is the same before and after it; both half
    kicks use g evaluated at the predicted pre-rotation momentum
    u^- ~ u^{j-1/2} + (dxi/2)(g(u^{j-1/2}) grad psi + (-B_y, B_x)), which makes the step
    second order."""
    h = 0.5 * dxi
    g0 = gamma_over_opp(ux, uy, opp)
    g = gamma_over_opp(ux + h * (g0 * gx - By), uy + h * (g0 * gy + Bx), opp)
    mx = ux + h * (g * gx - By)
    my = uy + h * (g * gy + Bx)
    t = h * Bz / opp
    s = 2.0 * t / (1.0 + t * t)
    px = mx - t * my
    py = my + t * mx
    qx = mx - s * py
    qy = my + s * px
    return qx + h * (g * gx - By), qy + h * (g * gy + Bx)


# ----------------------------------------------------------------------------------------
# beam sources and plasma sweep
# ----------------------------------------------------------------------------------------
def beam_sources(p, beams, n_nodes=None):
    """Slab [4, nxi+1, ny, nx] of beam S_b = Z n (1 - v_z), J_z, J_x, J_y at xi nodes k dxi:
    CIC in x, y, linear in xi, density = sum Z w W / (dx dy dxi).  Live particles have
    0 <= xi < Lxi, so both xi nodes lie in 0..nxi.  With n_nodes, only nodes 0..n_nodes-1 are
    kept (for runs on the first slices of a large window)."""
    G = Grid(p)
    nk = p.nxi + 1 if n_nodes is None else n_nodes
    dxi = p.Lxi / p.nxi
    src = np.zeros((4, nk * p.ny * p.nx))
    for sp, b in zip(p.species, beams):
        live = b["w"] != 0.0
        x, y, xi = b["x"][live], b["y"][live], b["xi"][live]
        ux, uy, uz, w = b["ux"][live], b["uy"][live], b["uz"][live], b["w"][live]
        gam = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
        omv = (1.0 + ux * ux + uy * uy) / (gam * (gam + uz))     # 1 - v_z, cancellation-free
        q = sp.Z * w / (dxi * G.dx * G.dy)
        vals = (q * omv, q * uz / gam, q * ux / gam, q * uy / gam)
        ix0, ix1, wx0, wx1 = cic_1d(x, G.nx, G.dx)
        iy0, iy1, wy0, wy1 = cic_1d(y, G.ny, G.dy)
        g = xi / dxi
        k0 = np.floor(g).astype(np.int64)
        f = g - k0
        for k, wk in ((k0, 1.0 - f), (k0 + 1, f)):
            keep = k < nk
            for iy, wy in ((iy0, wy0), (iy1, wy1)):
                for ix, wx in ((ix0, wx0), (ix1, wx1)):
                    idx = ((k * p.ny + iy) * p.nx + ix)[keep]
                    wt = (wk * wy * wx)[keep]
                    for slot in range(4):
                        src[slot] += np.bincount(idx, weights=vals[slot][keep] * wt,
                                                 minlength=src.shape[1])
    return src.reshape(4, nk, p.ny, p.nx)


def plasma_sweep(p, src, return_particles=False, return_psi=False, n_slices=None):
    """One sweep of the plasma through slices j = 0..nxi.  Returns the field slab
    [nxi+1, 6, ny, nx] (Wx, Wy, Ez, Bx, By, Bz) and per-slice diagnostics.  With n_slices the
    sweep stops after slices 0..n_slices-1 (the slice loop is sequential in xi, so these are
    exactly the first slices of the full sweep); src then needs nodes 0..n_slices."""
    G = Grid(p)
    dxi = p.Lxi / p.nxi
    nk = p.nxi + 1 if n_slices is None else n_slices
    nsrc = src.shape[1]
    floor = p.psi_floor
    pc_tol = getattr(p, "pc_tol", 0.0)
    cell = G.dx * G.dy
    # quiet lattice at xi = 0
    ppx, ppy = p.ppc_plasma_x, p.ppc_plasma_y
    ix, iy, sx, sy = np.meshgrid(np.arange(p.nx), np.arange(p.ny), np.arange(ppx),
                                 np.arange(ppy), indexing="ij")
    # particle order: ((iy*nx + ix)*ppc + sy*ppx + sx) -- the order does not change results
    order = np.lexsort((sx.ravel(), sy.ravel(), ix.ravel(), iy.ravel()))
    x = ((ix.ravel() + (sx.ravel() + 0.5) / ppx) * G.dx)[order]
    y = ((iy.ravel() + (sy.ravel() + 0.5) / ppy) * G.dy)[order]
    npart = x.size
    w = np.full(npart, cell / (ppx * ppy))
    ux = np.zeros(npart)
    uy = np.zeros(npart)
    psi_prev = np.zeros(npart)

    def src_at(slot, k):
        if 0 <= k < nsrc:
            return src[slot, k]
        return np.zeros((p.ny, p.nx))

    def jperp_half(xh, yh, uxh, uyh, opph, j):
        """Total J_perp at xi_{j+1/2}: plasma at x^{j+1/2} plus beam averaged over nodes."""
        jx = deposit(G, xh, yh, -w * uxh / opph) + 0.5 * (src_at(2, j) + src_at(2, j + 1))
        jy = deposit(G, xh, yh, -w * uyh / opph) + 0.5 * (src_at(3, j) + src_at(3, j + 1))
        return jx, jy

    slab = np.zeros((nk, 6, p.ny, p.nx))
    psi_slices = np.zeros((nk, p.ny, p.nx)) if return_psi else None
    diag = {k: np.zeros(nk) for k in ("kappa2", "psi0", "ez0", "jz_mean", "opp_min",
                                      "n_floor", "invariant", "charge", "pc_residual",
                                      "pc_iters")}
    # prologue: J_perp^{-1/2} (plasma at rest, beam half node 0), psi of slice 0
    Jx_prev, Jy_prev = 0.5 * src_at(2, 0), 0.5 * src_at(3, 0)
    psi0, ez0_half = 0.0, 0.0
    Se = deposit(G, x, y, -w)
    psi, gx_grid, gy_grid = solve_psi(G, Se + src_at(0, 0))
    Bx = np.zeros((p.ny, p.nx))
    By = np.zeros((p.ny, p.nx))
    Bz = np.zeros((p.ny, p.nx))
    for j in range(nk):
        diag["charge"][j] = abs(Se.sum() * cell + p.Lx * p.Ly)
        psi_p = psi0 + gather(G, psi, x, y)
        opp_raw = 1.0 + psi_p
        diag["opp_min"][j] = opp_raw.min()
        diag["n_floor"][j] = np.count_nonzero(opp_raw < floor)
        opp = np.maximum(opp_raw, floor)
        opph = np.maximum(1.0 + 0.5 * (3.0 * psi_p - psi_prev), floor)
        gx = gather(G, gx_grid, x, y)
        gy = gather(G, gy_grid, x, y)
        kappa2 = np.sum(w / opp) / (p.Lx * p.Ly)
        diag["kappa2"][j] = kappa2
        Bx_old = None
        for it in range(p.n_pc_iter):
            bx = gather(G, Bx, x, y)
            by = gather(G, By, x, y)
            bz = gather(G, Bz, x, y)
            uxh, uyh = push_xi(ux, uy, opp, gx, gy, bx, by, bz, dxi)
            uxj, uyj = 0.5 * (ux + uxh), 0.5 * (uy + uyh)
            uzj = uz_from_invariant(uxj, uyj, opp)
            Jx = deposit(G, x, y, -w * uxj / opp) + src_at(2, j)
            Jy = deposit(G, x, y, -w * uyj / opp) + src_at(3, j)
            Jz = deposit(G, x, y, -w * uzj / opp) + src_at(1, j)
            xh = x + 0.5 * dxi * uxh / opph
            yh = y + 0.5 * dxi * uyh / opph
            Jxh, Jyh = jperp_half(xh, yh, uxh, uyh, opph, j)
            Ez_fl, Bz = solve_ez_bz(G, Jx, Jy)
            Bx_old, By_old = Bx, By
            Bx, By = solve_bperp(G, Jz, (Jxh - Jx_prev) / dxi, (Jyh - Jy_prev) / dxi,
                                 kappa2, Bx, By)
            diag["pc_iters"][j] = it + 1
            if pc_tol > 0 and it + 1 < p.n_pc_iter:
                change = np.sqrt(np.sum((Bx - Bx_old) ** 2 + (By - By_old) ** 2))
                if change == 0 or change < pc_tol * np.sqrt(np.sum(Bx ** 2 + By ** 2)):
                    break
        num = np.sqrt(np.sum((Bx - Bx_old) ** 2 + (By - By_old) ** 2))
        den = np.sqrt(np.sum(Bx ** 2 + By ** 2))
        diag["pc_residual"][j] = num / den if den > 0 else 0.0
        gam = gamma_from_invariant(uxj, uyj, opp)
        diag["invariant"][j] = np.max(np.abs(gam - uzj - opp) / opp)
        # mean mode (k = 0), leapfrog in xi
        jz_mean = Jz.mean()
        ez0_next = ez0_half - dxi * jz_mean
        ez0 = 0.5 * (ez0_half + ez0_next)
        diag["jz_mean"][j], diag["psi0"][j], diag["ez0"][j] = jz_mean, psi0, ez0
        slab[j] = (-gx_grid, -gy_grid, ez0 + Ez_fl, Bx, By, Bz)
        if return_psi:
            psi_slices[j] = psi0 + psi
        # commit push with the final fields of slice j
        bx = gather(G, Bx, x, y)
        by = gather(G, By, x, y)
        bz = gather(G, Bz, x, y)
        uxh, uyh = push_xi(ux, uy, opp, gx, gy, bx, by, bz, dxi)
        xh = x + 0.5 * dxi * uxh / opph
        yh = y + 0.5 * dxi * uyh / opph
        Jx_prev, Jy_prev = jperp_half(xh, yh, uxh, uyh, opph, j)
        x = np.mod(x + dxi * uxh / opph, p.Lx)
        y = np.mod(y + dxi * uyh / opph, p.Ly)
        ux, uy = uxh, uyh
        psi_prev = psi_p
        psi0 = psi0 + dxi * ez0_next
        ez0_half = ez0_next
        if j + 1 < min(nk, p.nxi + 1):
            Se = deposit(G, x, y, -w)
            psi, gx_grid, gy_grid = solve_psi(G, Se + src_at(0, j + 1))
    if return_psi:
        diag["psi"] = psi_slices
    if return_particles:
        return slab, diag, dict(x=x, y=y, ux=ux, uy=uy)
    return slab, diag


# ----------------------------------------------------------------------------------------
# beam push in tau
# ----------------------------------------------------------------------------------------
def gather_slab(p, slab, x, y, xi):
    """Trilinear field values [6, n] at beam positions: CIC in x, y, linear in xi."""
    G = Grid(p)
    dxi = p.Lxi / p.nxi
    ix0, ix1, wx0, wx1 = cic_1d(x, G.nx, G.dx)
    iy0, iy1, wy0, wy1 = cic_1d(y, G.ny, G.dy)
    g = xi / dxi
    k0 = np.floor(g).astype(np.int64)
    f = g - k0
    out = np.zeros((6, x.size))
    for k, wk in ((k0, 1.0 - f), (k0 + 1, f)):
        for iy, wy in ((iy0, wy0), (iy1, wy1)):
            for ix, wx in ((ix0, wx0), (ix1, wx1)):
                out += slab[k, :, iy, ix].T * (wk * wy * wx)
    return out


def boris(ux, uy, uz, E, B, h):
    """Relativistic Boris step: half kick h E, rotation with t = h B/gamma, half kick."""
    mx, my, mz = ux + h * E[0], uy + h * E[1], uz + h * E[2]
    gm = np.sqrt(1.0 + mx * mx + my * my + mz * mz)
    tx, ty, tz = h * B[0] / gm, h * B[1] / gm, h * B[2] / gm
    px = mx + (my * tz - mz * ty)
    py = my + (mz * tx - mx * tz)
    pz = mz + (mx * ty - my * tx)
    s = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz)
    sx, sy, sz = s * tx, s * ty, s * tz
    qx = mx + (py * sz - pz * sy)
    qy = my + (pz * sx - px * sz)
    qz = mz + (px * sy - py * sx)
    return qx + h * E[0], qy + h * E[1], qz + h * E[2]


def beam_push(p, beams, slab):
    """Advance every live beam particle by dt through the field slab (in place)."""
    for sp, b in zip(p.species, beams):
        live = b["w"] != 0.0
        x, y, xi = b["x"][live], b["y"][live], b["xi"][live]
        F = gather_slab(p, slab, x, y, xi)
        Wx, Wy, Ez, Bx, By, Bz = F
        E = (Wx + By, Wy - Bx, Ez)
        B = (Bx, By, Bz)
        h = 0.5 * sp.Z * p.dt / sp.M
        ux, uy, uz = boris(b["ux"][live], b["uy"][live], b["uz"][live], E, B, h)
        gam = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
        omv = (1.0 + ux * ux + uy * uy) / (gam * (gam + uz))
        b["x"][live] = np.mod(x + p.dt * ux / gam, p.Lx)
        b["y"][live] = np.mod(y + p.dt * uy / gam, p.Ly)
        b["xi"][live] = xi + p.dt * omv
        b["ux"][live], b["uy"][live], b["uz"][live] = ux, uy, uz
        lost = b["xi"] >= p.Lxi
        b["w"][lost] = 0.0
    return beams


def run(p, beams, steps, diag_every=False):
    """steps x (sweep, beam push), then the final sweep.  Returns the final slab, the list of
    per-sweep diagnostics, and the beams (modified in place)."""
    diags = []
    for _ in range(steps):
        slab, d = plasma_sweep(p, beam_sources(p, beams))
        diags.append(d)
        beam_push(p, beams, slab)
    slab, d = plasma_sweep(p, beam_sources(p, beams))
    diags.append(d)
    return slab, diags, beams


def field_energy(p, slab):
    """Per-slice energies 1/2 sum F^2 dx dy dxi of E_x, E_y, E_z, B_x, B_y, B_z [nk, 6]."""
    dxi = p.Lxi / p.nxi
    Wx, Wy, Ez, Bx, By, Bz = (slab[:, c] for c in range(6))
    F = np.stack([Wx + By, Wy - Bx, Ez, Bx, By, Bz], axis=1)
    return 0.5 * (F ** 2).sum(axis=(2, 3)) * (p.Lx / p.nx) * (p.Ly / p.ny) * dxi
