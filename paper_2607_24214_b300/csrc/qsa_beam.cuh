// Beam macroparticles: device initialisation, relativistic Boris push in tau through the
// field slab (trilinear: CIC in x, y, linear in xi), loss at the back of the window, and the
// deposit of the beam sources S_b = Z n (1 - v_z), J_z, J_x, J_y of the next sweep.
//
// Storage per species, index s = ((k_xi * ny + iy) * ppc + sub) * nx + ix (a warp holds 32
// neighbouring cells of one sub-lattice position).  Positions are offsets, in cells, from
// the particle's lattice home; this keeps the slow transverse and longitudinal drifts of an
// ultrarelativistic beam (1e-6 cells per step) exact in FP32.  u_z is FP64 in the FP64 path
// and, in the mixed path, one float holding its deviation u_z - u_zb from the species'
// reference momentum u_zb = sqrt(gamma_b^2 - 1): the per-step increments of u_z are ~1e-6 of
// it, too small for a float of u_z itself, but the deviation is the energy spread (a few
// percent of u_zb at most), whose float resolves them.  A mixed-path particle is 28 bytes:
// three offsets, u_x, u_y, the u_z deviation and the weight deviation; the slot's canonical
// id (4 bytes more) is only kept once the beam has been re-homed.
// The weight is stored as its relative deviation dw = w / wbar - 1 from the species' nominal
// weight wbar = alpha dx dy dxi / ppc (dw = -1 marks a lost particle), and the beam sources
// are deposited as deviations from the reference beam (nominal weight, at home, u = (0, 0,
// sqrt(gamma_b^2 - 1))): the reference is uniform in x, y (k = 0 only) and is kept in FP64
// per node, so FP32 sums keep the 1e-4 density noise of the fluctuations.
#pragma once
#include <cmath>

#include "qsa_common.cuh"

namespace qsa {

// Storage type of u_z: FP64 (u_z itself), or in the mixed path a float of u_z - u_zb.
template <typename BR>
struct UzT {
  using T = double;
};
template <>
struct UzT<float> {
  using T = float;
};
// Stored u_z <-> its value, with uzb = sqrt(gamma_b^2 - 1) of the species (FP64).
__host__ __device__ __forceinline__ double uz_value(double v, double) { return v; }
__host__ __device__ __forceinline__ double uz_value(float v, double uzb) {
  return uzb + (double)v;
}
__host__ __device__ __forceinline__ void uz_store(double& d, double v, double) { d = v; }
__host__ __device__ __forceinline__ void uz_store(float& d, double v, double uzb) {
  d = (float)(v - uzb);
}

// id[s]: the canonical id of the particle slot s holds (see rehome_*), so that host copies
// keep every particle's identity; null until the beam is first re-homed (every slot then
// holds its own particle).
template <typename BR>
struct BeamArrays {
  BR *ox, *oy, *oxi, *ux, *uy, *dw;
  typename UzT<BR>::T* uz;
  unsigned* id;
  long long n;
};

struct SpeciesDev {
  double Z, M, alpha, gamma_b, gamma_spread_rel, uperp_spread, noise_rel;
  double wbar;   // nominal weight alpha dx dy dxi / ppc
  double qbar;   // Z wbar / (dx dy dxi): reference density per particle
  double omvbar; // 1 - v_z of the reference momentum
  double uzb;    // reference momentum sqrt(gamma_b^2 - 1)
  int ppx, ppy, ppxi, ppc;
  int k0, nkb;  // first xi cell and number of xi cells
  int seeded, index;
};

// Per-species constants of the push and deposit in the working precision, formed on the host
// in FP64 (no FP64 division in device code).
template <typename BR>
struct BeamConst {
  BR hdt;            // 0.5 Z dt / M
  BR cdx, cdy, cdk;  // dt/dx, dt/dy, dt/dxi
  BR refS, refJz;    // reference source weights qbar omvbar, qbar (1 - omvbar)
  BR qb, omvbar;     // qbar, 1 - v_z of the reference momentum
  BR uzb;            // sqrt(gamma_b^2 - 1), the reference momentum
  BR gamb, Db;       // gamma_b and gamma_b (gamma_b + u_zb) = 1 / omvbar
  BR inv_ppx, inv_ppy, inv_ppxi;  // 1 / sub-lattice counts
};
template <typename BR>
inline BeamConst<BR> beam_consts(const DevParams& p, const SpeciesDev& sp) {
  BeamConst<BR> c;
  c.hdt = BR(0.5 * sp.Z * p.dt / sp.M);
  c.cdx = BR(p.dt / p.dx);
  c.cdy = BR(p.dt / p.dy);
  c.cdk = BR(p.dt / p.dxi);
  c.refS = BR(sp.qbar * sp.omvbar);
  c.refJz = BR(sp.qbar * (1.0 - sp.omvbar));
  c.qb = BR(sp.qbar);
  c.omvbar = BR(sp.omvbar);
  c.gamb = BR(sp.gamma_b);
  c.Db = BR(1.0 / sp.omvbar);
  const double uzb = std::sqrt(sp.gamma_b * sp.gamma_b - 1.0);
  c.uzb = BR(uzb);
  c.inv_ppx = BR(1.0 / sp.ppx);
  c.inv_ppy = BR(1.0 / sp.ppy);
  c.inv_ppxi = BR(1.0 / sp.ppxi);
  return c;
}

struct ModesDev {
  int n;
  int mx[16], my[16];
  double amp[16], phase[16];
};

// Home of storage index s: cell (ix, iy, kxi) and sub-lattice (sx, sy, sxi).
struct Home {
  int ix, iy, kxi, sx, sy, sxi;
  long long id;  // canonical id ((kxi*ny + iy)*nx + ix)*ppc + sub
};
__device__ __forceinline__ Home home_of(long long s, int nx, int ny, const SpeciesDev& sp) {
  Home h;
  h.ix = (int)(s % nx);
  long long r = s / nx;
  const int sub = (int)(r % sp.ppc);
  r /= sp.ppc;
  h.iy = (int)(r % ny);
  h.kxi = (int)(r / ny);
  h.sx = sub % sp.ppx;
  h.sy = (sub / sp.ppx) % sp.ppy;
  h.sxi = sub / (sp.ppx * sp.ppy);
  h.id = (((long long)h.kxi * ny + h.iy) * nx + h.ix) * sp.ppc + sub;
  return h;
}

// ------------------------------------------------------------------ initialisation
template <typename BR>
__global__ void beam_init_kernel(BeamArrays<BR> b, DevParams p, SpeciesDev sp, ModesDev md,
                                 unsigned long long seed) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= b.n) return;
  const Home h = home_of(s, p.nx, p.ny, sp);
  const U4 r = philox4x32_10(U4{(uint32_t)(h.id & 0xFFFFFFFFull), (uint32_t)(h.id >> 32),
                                (uint32_t)sp.index, 0u},
                             (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const double a0 = sqrt(-2.0 * log(u01(r.a))), a1 = sqrt(-2.0 * log(u01(r.c)));
  double s1, c1, s3, c3;
  sincospi(2.0 * u01(r.b), &s1, &c1);
  sincospi(2.0 * u01(r.d), &s3, &c3);
  const double n0 = a0 * c1, n1 = a0 * s1, n2 = a1 * c3, n3 = a1 * s3;
  // w / wbar = (1 + noise n0) * (1 + sum_m a_m cos(k_m . x + phi_m)), stored minus one
  double mm = 0.0;  // mode factor minus one
  if (sp.seeded && md.n > 0) {
    const double x = (h.ix + (h.sx + 0.5) / sp.ppx) * p.dx;
    const double y = (h.iy + (h.sy + 0.5) / sp.ppy) * p.dy;
    for (int k = 0; k < md.n; ++k) {
      const double kx = 6.283185307179586476925 * md.mx[k] / p.Lx;
      const double ky = 6.283185307179586476925 * md.my[k] / p.Ly;
      mm += md.amp[k] * cos(kx * x + ky * y + md.phase[k]);
    }
  }
  const double dw = mm + sp.noise_rel * n0 * (1.0 + mm);
  const double ux = sp.uperp_spread * n1, uy = sp.uperp_spread * n2;
  const double gam = sp.gamma_b * (1.0 + sp.gamma_spread_rel * n3);
  b.ox[s] = BR(0);
  b.oy[s] = BR(0);
  b.oxi[s] = BR(0);
  b.ux[s] = BR(ux);
  b.uy[s] = BR(uy);
  uz_store(b.uz[s], sqrt(gam * gam - 1.0 - ux * ux - uy * uy), sp.uzb);
  b.dw[s] = BR(dw);
  if (b.id) b.id[s] = (unsigned)h.id;
}

// ------------------------------------------------------------------ deposit and push
// A block handles one group of a species: the ppc * nx particles whose home is xi cell k and
// row iy.  Their deposits land in a shared-memory tile of the nodes (k, k+1) x rows
// (iy-1 .. iy+2) x every x, field-major ([node][row][quantity][x]: the lanes of a warp, on
// consecutive columns, hit consecutive banks), which is flushed to the source slab with one
// vector atomic per touched node; a deposit outside the tile goes straight to global memory.

__device__ __forceinline__ void red4(float* a, float s, float z, float x, float y) {
  atomicAdd(reinterpret_cast<float4*>(a), make_float4(s, z, x, y));
}
__device__ __forceinline__ void red4(double* a, double s, double z, double x, double y) {
  atomicAdd(a, s);
  atomicAdd(a + 1, z);
  atomicAdd(a + 2, x);
  atomicAdd(a + 3, y);
}

template <typename BR>
struct Group {
  int kabs, iy;  // home xi node and row of the group
  BR* tile;      // [2][4][4][nx]: S_b, J_z, J_x, J_y deviations
  int* outer;    // bit dk * 4 + r set when a deposit landed in the outer tile row r (0 or 3)
};

// Trilinear weights W of the eight corners of the home cell at (h + d) and their differences
// dW = W - W(h) from the reference position h, both separable by axis: with a = h or 1 - h and
// d = +-offset per axis, W = (a1 + d1)(a2 + d2)(a3 + d3) and the difference telescopes as
// dW = d1 (a2 + d2)(a3 + d3) + a1 [d2 (a3 + d3) + a2 d3], free of cancellation.
template <typename BR>
__device__ __forceinline__ void home_weights(BR hx, BR hy, BR hk, BR ox, BR oy, BR oxi,
                                             BR (&W)[2][2][2], BR (&dW)[2][2][2]) {
#pragma unroll
  for (int ck = 0; ck < 2; ++ck) {
    const BR a3 = ck ? hk : BR(1) - hk, d3 = ck ? oxi : -oxi, K = a3 + d3;
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
      const BR a2 = cy ? hy : BR(1) - hy, d2 = cy ? oy : -oy;
      const BR YK = (a2 + d2) * K, T = d2 * K + a2 * d3;
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const BR a1 = cx ? hx : BR(1) - hx, d1 = cx ? ox : -ox;
        W[ck][cy][cx] = (a1 + d1) * YK;
        dW[ck][cy][cx] = d1 * YK + a1 * T;
      }
    }
  }
}

// Deposit, per source quantity, dev W(x) + ref (W(x) - W(home)) (ref = 0 for J_x, J_y) for a
// particle of home column ix, home sub-cell position (hx, hy, hk) and offsets (ox, oy, oxi) in
// cells.  In the home cell the trilinear weight differences come from the offsets without
// cancellation.  Out of it, home_ref = false leaves the -ref W(home) part to the caller.
template <typename BR>
__device__ __forceinline__ void deposit_particle(const Group<BR>& g, BR* src, const DevParams& p,
                                                 int ix, BR hx, BR hy, BR hk, BR ox, BR oy,
                                                 BR oxi, BR dS, BR dJz, BR jx, BR jy, BR refS,
                                                 BR refJz, bool home_ref = true) {
  const BR lx = hx + ox, ly = hy + oy, lk = hk + oxi;
  const int nx = p.nx;
  if (lx >= BR(0) && lx < BR(1) && ly >= BR(0) && ly < BR(1) && lk >= BR(0) && lk < BR(1)) {
    const int x1 = (ix + 1 == nx) ? 0 : ix + 1;
    BR Wc[2][2][2], dWc[2][2][2];
    home_weights(hx, hy, hk, ox, oy, oxi, Wc, dWc);
#pragma unroll
    for (int ck = 0; ck < 2; ++ck) {
      if (g.kabs + ck >= p.nk) continue;
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        BR* row = g.tile + (size_t)(ck * 4 + 1 + cy) * 4 * nx;
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const BR w = Wc[ck][cy][cx], dW = dWc[ck][cy][cx];
          BR* t = row + (cx ? x1 : ix);
          atomicAdd(t, dS * w + refS * dW);
          atomicAdd(t + nx, dJz * w + refJz * dW);
          atomicAdd(t + 2 * nx, jx * w);
          atomicAdd(t + 3 * nx, jy * w);
        }
      }
    }
    return;
  }
  // left the home cell: full weights at the new corners, minus the reference at home.  The
  // destination (tile row or global row) is settled once per (node, row); the row's two
  // corners share it
#pragma unroll 1
  for (int pass = 0; pass < (home_ref ? 2 : 1); ++pass) {
    const BR mx = pass ? hx : lx, my = pass ? hy : ly, mk = pass ? hk : lk;
    const BR fx = floor(mx), fy = floor(my), fk = floor(mk);
    const BR ex = mx - fx, ey = my - fy, ek = mk - fk;
    const int gx0 = wrap(ix + (int)fx, nx), gx1 = (gx0 + 1 == nx) ? 0 : gx0 + 1;
    const int gy = g.iy + (int)fy, gk = g.kabs + (int)fk;
    (void)QSA_IN(gx0 >= 0 && gx0 < nx && gx1 < nx);
    const BR s0 = pass ? -refS : dS + refS, z0 = pass ? -refJz : dJz + refJz;
    const BR x0v = pass ? BR(0) : jx, y0v = pass ? BR(0) : jy;
#pragma unroll
    for (int ck = 0; ck < 2; ++ck) {
      const int k = gk + ck, dk = k - g.kabs;
      if (k < 0 || k >= p.nk) continue;
      const BR wk = ck ? ek : BR(1) - ek;
#pragma unroll
      for (int cy = 0; cy < 2; ++cy) {
        const BR wy = wk * (cy ? ey : BR(1) - ey);
        const BR w0 = wy * (BR(1) - ex), w1 = wy * ex;
        const int r = gy + cy - (g.iy - 1);
        if (dk >= 0 && dk < 2 && r >= 0 && r < 4) {
          if (r == 0 || r == 3) atomicOr(g.outer, 1 << (dk * 4 + r));
          BR* t = g.tile + (size_t)(dk * 4 + r) * 4 * nx;
          atomicAdd(t + gx0, w0 * s0);
          atomicAdd(t + nx + gx0, w0 * z0);
          atomicAdd(t + 2 * nx + gx0, w0 * x0v);
          atomicAdd(t + 3 * nx + gx0, w0 * y0v);
          atomicAdd(t + gx1, w1 * s0);
          atomicAdd(t + nx + gx1, w1 * z0);
          atomicAdd(t + 2 * nx + gx1, w1 * x0v);
          atomicAdd(t + 3 * nx + gx1, w1 * y0v);
        } else {
          BR* e = src + ((size_t)k * p.ny + wrap(gy + cy, p.ny)) * nx * 4;
          red4(e + (size_t)gx0 * 4, w0 * s0, w0 * z0, w0 * x0v, w0 * y0v);
          red4(e + (size_t)gx1 * 4, w1 * s0, w1 * z0, w1 * x0v, w1 * y0v);
        }
      }
    }
  }
}

// FP32 quotient and square root through the hardware approximations (about 2 ulp): the mixed
// path's beam arithmetic carries errors far below its 1e-4 field tolerance.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fast_sqrt(float x) { return x * rsqrtf(x); }  // x > 0

// Source deviations of one particle with q = qbar (1 + dw): dS = q(1 - v_z) - qbar omvbar,
// dJz = q v_z - qbar (1 - omvbar); J_perp = q u_perp/gamma (reference zero).
__device__ __forceinline__ void beam_sources(double ux, double uy, double uz, double /*duz*/,
                                             double dw, const BeamConst<double>& c, double& dS,
                                             double& dJz, double& jx, double& jy) {
  const double up2 = ux * ux + uy * uy;
  const double g = sqrt(1.0 + up2 + uz * uz);
  const double omv = (1.0 + up2) / (g * (g + uz));
  const double q = c.qb * (1.0 + dw);
  dS = c.qb * (dw * omv + (omv - c.omvbar));
  dJz = c.qb * (dw * (1.0 - omv) - (omv - c.omvbar));
  jx = q * ux / g;
  jy = q * uy / g;
}
// The FP32 path forms (1 - v_z) - (1 - v_z)_ref from the small quantities u_perp^2 and
// duz = u_z - u_zb, without subtracting the two nearly equal values (at gamma_b = 1e4 they
// agree to ~2 % and are ~5e-9 each):  with A = 1 + u_perp^2, D = gamma (gamma + u_z) and
// D_b = gamma_b (gamma_b + u_zb),  A/D - 1/D_b = (u_perp^2 D_b + D_b - D) / (D D_b), where
// D_b - D = -s2 - dgamma u_z - gamma_b duz,  s2 = gamma^2 - gamma_b^2 = u_perp^2 +
// duz (u_z + u_zb),  dgamma = gamma - gamma_b = s2 / (gamma + gamma_b).
__device__ __forceinline__ void beam_sources(float ux, float uy, float uzf, float duz, float dw,
                                             const BeamConst<float>& c, float& dS, float& dJz,
                                             float& jx, float& jy) {
  const float up2 = ux * ux + uy * uy;
  const float d = fast_div(1.0f + up2, fast_sqrt(1.0f + up2 + uzf * uzf) + uzf);  // gamma - u_z
  const float g = uzf + d;
  const float ig = fast_div(1.0f, g);
  const float omv = d * ig;                                              // 1 - v_z
  const float s2 = up2 + duz * (uzf + c.uzb);
  const float dg = fast_div(s2, g + c.gamb);
  const float num = up2 * c.Db - s2 - dg * uzf - c.gamb * duz;
  const float domv = num * fast_div(1.0f, g * (g + uzf)) * c.omvbar;
  dS = c.qb * (dw * omv + domv);
  dJz = c.qb * (dw * (1.0f - omv) - domv);
  const float q = c.qb * (1.0f + dw) * ig;
  jx = q * ux;
  jy = q * uy;
}

// 1/gamma and 1 - v_z = (1 + u_perp^2)/(gamma (gamma + u_z)) of the pushed momentum.
__device__ __forceinline__ void drift_rates(double ux, double uy, double uz, double& ig,
                                            double& omv) {
  const double up2 = ux * ux + uy * uy;
  const double gg = sqrt(1.0 + up2 + uz * uz);
  ig = 1.0 / gg;
  omv = (1.0 + up2) / (gg * (gg + uz));
}
__device__ __forceinline__ void drift_rates(float ux, float uy, float uzf, float& ig,
                                            float& omv) {
  const float up2 = ux * ux + uy * uy;
  const float d = fast_div(1.0f + up2, fast_sqrt(1.0f + up2 + uzf * uzf) + uzf);  // gamma - u_z
  ig = fast_div(1.0f, uzf + d);
  omv = d * ig;
}

// Trilinear gather of the six slab fields (CIC in x, y, linear in xi) at unwrapped node
// (gk, gy, gx) + fractions (ek, ey, ex).
__device__ __forceinline__ void ldslab(const float* e, float v[6]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(e));
  const float2 b = __ldg(reinterpret_cast<const float2*>(e + 4));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
__device__ __forceinline__ void ldslab(const double* e, double v[6]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(e));
  const double2 b = __ldg(reinterpret_cast<const double2*>(e + 2));
  const double2 c = __ldg(reinterpret_cast<const double2*>(e + 4));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}
template <typename BR>
__device__ __forceinline__ void gather_slab(const BR* __restrict__ slab, const DevParams& p, int gk,
                                            int gy, int gx, BR ek, BR ey, BR ex, BR F[6]) {
#pragma unroll
  for (int f = 0; f < 6; ++f) F[f] = BR(0);
  const int y0 = wrap(gy, p.ny), y1 = wrap(gy + 1, p.ny);
  const int x0 = wrap(gx, p.nx), x1 = wrap(gx + 1, p.nx);
#pragma unroll
  for (int ck = 0; ck < 2; ++ck) {
    const int k = gk + ck;
    if (k < 0 || k >= p.nk) continue;
    const BR wk = ck ? ek : BR(1) - ek;
    (void)QSA_IN(y0 < p.ny && y1 < p.ny && x0 < p.nx && x1 < p.nx);
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
      const BR wy = wk * (cy ? ey : BR(1) - ey);
      const BR* row = slab + ((size_t)k * p.ny + (cy ? y1 : y0)) * p.nx * 8;
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const BR wt = wy * (cx ? ex : BR(1) - ex);
        BR v[6];
        ldslab(row + (size_t)(cx ? x1 : x0) * 8, v);
#pragma unroll
        for (int f = 0; f < 6; ++f) F[f] += wt * v[f];
      }
    }
  }
}

// Relativistic Boris (FP64): half kick h E, rotation t = h B/gamma^-, half kick.
__device__ __forceinline__ void boris(double& ux, double& uy, double& uz, const double F[6],
                                      double h) {
  const double Ex = F[0] + F[4], Ey = F[1] - F[3], Ez = F[2];
  const double Bx = F[3], By = F[4], Bz = F[5];
  const double mx = ux + h * Ex, my = uy + h * Ey, mz = uz + h * Ez;
  const double gm = sqrt(1.0 + mx * mx + my * my + mz * mz);
  const double tx = h * Bx / gm, ty = h * By / gm, tz = h * Bz / gm;
  const double px = mx + (my * tz - mz * ty), py = my + (mz * tx - mx * tz),
               pz = mz + (mx * ty - my * tx);
  const double s = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
  const double sx = s * tx, sy = s * ty, sz = s * tz;
  ux = mx + (py * sz - pz * sy) + h * Ex;
  uy = my + (pz * sx - px * sz) + h * Ey;
  uz = mz + (px * sy - py * sx) + h * Ez;
}

// The same Boris step with FP32 arithmetic, u_z kept as its deviation duz = u_z - u_zb (a
// float of the energy spread resolves the small per-step increments that a float of u_z
// would round away), written so that no step subtracts nearly equal terms: with W = E_perp -
// z x B (the slab's first two fields), E_x - v_z B_y = W_x + (1 - v_z) B_y, and 1 - v_z is
// formed from gamma - u_z = (1 + u_perp^2)/(gamma + u_z).  uzb: u_zb in FP32.
__device__ __forceinline__ void boris(float& ux, float& uy, float& duz, const float F[6],
                                      float h, float uzb) {
  const float Wx = F[0], Wy = F[1], Ez = F[2], Bx = F[3], By = F[4], Bz = F[5];
  const float mx = ux + h * (Wx + By), my = uy + h * (Wy - Bx);
  const float mzf = (uzb + duz) + h * Ez;
  const float mp2 = mx * mx + my * my;
  const float gm = fast_sqrt(1.0f + mp2 + mzf * mzf);
  const float dm = fast_div(1.0f + mp2, gm + mzf);  // gamma^- - m_z
  const float ig = fast_div(1.0f, gm);
  const float tx = h * Bx * ig, ty = h * By * ig, tz = h * Bz * ig;
  const float t2 = tx * tx + ty * ty + tz * tz;
  const float i1t2 = fast_div(1.0f, 1.0f + t2);
  const float sfac = 2.0f * i1t2;
  const float sx = sfac * tx, sy = sfac * ty, sz = sfac * tz;
  // u' = m + m x t, transverse parts without the m_z t cancellation
  const float pxp = ux + h * Wx + h * By * dm * ig + my * tz;
  const float pyp = uy + h * Wy - h * Bx * dm * ig - mx * tz;
  // eps = 1 - u'_z / (gamma^- (1 + t^2)), u'_z = m_z + m_x t_y - m_y t_x
  const float eps = (dm + gm * t2 - (mx * ty - my * tx)) * ig * i1t2;
  ux = ux + 2.0f * h * Wx + 2.0f * h * By * eps + pyp * sz;
  uy = uy + 2.0f * h * Wy - 2.0f * h * Bx * eps - pxp * sz;
  duz += 2.0f * h * Ez + pxp * sy - pyp * sx;
}

template <typename BR>
__device__ __forceinline__ bool in_cell(BR lx, BR ly, BR lk) {
  return lx >= BR(0) && lx < BR(1) && ly >= BR(0) && ly < BR(1) && lk >= BR(0) && lk < BR(1);
}

// Trilinear gather for the two particles of a thread, both inside their home cell (layer k,
// row iy, column ix; x1 the next column): the eight corner nodes are loaded once.
template <typename BR>
__device__ __forceinline__ void gather_cell(const BR* __restrict__ slab, const DevParams& p,
                                            int k, int iy, int ix, int x1, const BR hx[2],
                                            const BR hy[2], const BR hk[2], const BR ox[2],
                                            const BR oy[2], const BR oxi[2], BR F[2][6]) {
  const int y1 = (iy + 1 == p.ny) ? 0 : iy + 1;
  (void)QSA_IN(k >= 0 && k + 1 < p.nk && iy >= 0 && iy < p.ny && ix < p.nx && x1 < p.nx);
  BR lx[2], ly[2], lk[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    lx[u] = hx[u] + ox[u];
    ly[u] = hy[u] + oy[u];
    lk[u] = hk[u] + oxi[u];
#pragma unroll
    for (int f = 0; f < 6; ++f) F[u][f] = BR(0);
  }
#pragma unroll
  for (int ck = 0; ck < 2; ++ck) {
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
      const BR* row = slab + ((size_t)(k + ck) * p.ny + (cy ? y1 : iy)) * p.nx * 8;
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        BR v[6];
        ldslab(row + (size_t)(cx ? x1 : ix) * 8, v);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const BR wt = (ck ? lk[u] : BR(1) - lk[u]) * (cy ? ly[u] : BR(1) - ly[u]) *
                        (cx ? lx[u] : BR(1) - lx[u]);
#pragma unroll
          for (int f = 0; f < 6; ++f) F[u][f] += wt * v[f];
        }
      }
    }
  }
}

// Where the live particles of a group sit after its push (or now, without a push): the
// largest xi cell, max-reduced per home layer into cmax[layer] (a later push of the layer
// gathers slab nodes up to that cell + 1), and the smallest cell minus the home layer,
// min-reduced into dmin (a particle deposits at nodes >= its home layer + dmin).  Either
// pointer may be null.
struct Extent {
  int* cmax;
  int* dmin;
  double* mom;  // [nxi][7] beam moments of the species per xi cell (see qsa_diag), or null
  unsigned long long* away;  // live particles outside their slot's cell after the push, or null
};

// u_z - sqrt(gamma_b^2 - 1) (the stored deviation in the mixed path), and u_z (in FP32 there,
// for the derived quantities gamma and 1 - v_z)
__device__ __forceinline__ double uz_dev(double uz, const BeamConst<double>& c) {
  return uz - c.uzb;
}
__device__ __forceinline__ float uz_dev(float duz, const BeamConst<float>&) { return duz; }
__device__ __forceinline__ double uz_lead(double uz, const BeamConst<double>&) { return uz; }
__device__ __forceinline__ float uz_lead(float duz, const BeamConst<float>& c) {
  return c.uzb + duz;
}
// the Boris step of either precision with the stored u_z
__device__ __forceinline__ void boris_st(double& ux, double& uy, double& uz, const double F[6],
                                         const BeamConst<double>& c) {
  boris(ux, uy, uz, F, c.hdt);
}
__device__ __forceinline__ void boris_st(float& ux, float& uy, float& duz, const float F[6],
                                         const BeamConst<float>& c) {
  boris(ux, uy, duz, F, c.hdt, c.uzb);
}

// One group of a species: the ppc * nx particles whose home is xi cell (layer) k and row iy.
// PUSH = false: deposit the current beam (sources of the first sweep).  PUSH = true: push
// every live particle by dt through the slab, drop those with xi >= Lxi, and deposit the
// sources of the next sweep.  Called by every thread of the block; tile holds
// beam_smem_bytes(nx).
// The descriptors b, sp, bc come by value: the particle loop then reads them from registers,
// not again after each store through memory the compiler cannot prove distinct.
template <typename BR, bool PUSH>
__device__ void beam_group(const BeamArrays<BR> b, const DevParams& p, const SpeciesDev sp,
                           const BeamConst<BR> bc, const BR* __restrict__ slab, BR* src,
                           unsigned long long* lost, Extent ext, int grp, BR* tile) {
  using UZ = typename UzT<BR>::T;
  __shared__ int s_ext[2], s_outer;
  Group<BR> g;
  g.tile = tile;
  g.outer = &s_outer;
  g.iy = grp % p.ny;
  g.kabs = sp.k0 + grp / p.ny;
  const int nx = p.nx;
  const int tn = 2 * 4 * nx * 4;
  zero_block(g.tile, tn);
  __shared__ double s_mom[7];
  if (threadIdx.x == 0) {
    s_ext[0] = -1;
    s_ext[1] = 0;
    s_outer = 0;
    for (int k = 0; k < 7; ++k) s_mom[k] = 0.0;
  }
  __syncthreads();
  int cmax_t = -1, dmin_t = 0;
  BR mom_t[7] = {0, 0, 0, 0, 0, 0, 0};  // moments of the particles in the home layer
  // the aggregated deposit needs whole warps over consecutive columns
  const bool lane_agg = (nx % 32 == 0) && (blockDim.x % 32 == 0);
  const size_t base = (size_t)grp * sp.ppc * nx;
  const BR refS = bc.refS, refJz = bc.refJz;
  const BR cdx = bc.cdx, cdy = bc.cdy, cdk = bc.cdk;
  const int kleft = p.nxi - g.kabs;  // lost when the local xi position reaches this
  int my_lost = 0, my_away = 0;
  // two sub-lattice positions per thread per pass: particles (sub0, ix) and (sub0 + 1, ix);
  // the loads and gathers of both are issued before either particle's arithmetic
  for (int sub0 = 0; sub0 < sp.ppc; sub0 += 2) {
    BR hx[2], hy[2], hk[2];
    bool ok[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      ok[u] = sub0 + u < sp.ppc;
      const int sub = ok[u] ? sub0 + u : sub0;
      // sub = (sxi ppy + sy) ppx + sx, split with exact float quotients of small integers
      const int q1 = (int)((float(sub) + 0.5f) * float(bc.inv_ppx));
      const int sx = sub - q1 * sp.ppx;
      const int sxi = (int)((float(q1) + 0.5f) * float(bc.inv_ppy));
      const int sy = q1 - sxi * sp.ppy;
      hx[u] = (BR(sx) + BR(0.5)) * bc.inv_ppx;
      hy[u] = (BR(sy) + BR(0.5)) * bc.inv_ppy;
      hk[u] = (BR(sxi) + BR(0.5)) * bc.inv_ppxi;
    }
    for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
      size_t si[2];
      BR dw[2], ox[2], oy[2], oxi[2], ux[2], uy[2];
      UZ uz[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        si[u] = base + (size_t)(ok[u] ? sub0 + u : sub0) * nx + ix;
        if (!QSA_IN(si[u] < (size_t)b.n)) si[u] = 0;
        dw[u] = b.dw[si[u]];
        ox[u] = b.ox[si[u]];
        oy[u] = b.oy[si[u]];
        oxi[u] = b.oxi[si[u]];
        ux[u] = b.ux[si[u]];
        uy[u] = b.uy[si[u]];
        uz[u] = b.uz[si[u]];
      }
      const int x1 = (ix + 1 == nx) ? 0 : ix + 1;
      // pre-push positions in cells from the home cell's lower corner
      bool pre_home = true;
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (ok[u]) pre_home = pre_home && in_cell(hx[u] + ox[u], hy[u] + oy[u], hk[u] + oxi[u]);
      BR F[2][6];
      if (PUSH) {
        if (pre_home) {
          // both particles in the home cell: one gather of the cell's eight slab nodes
          gather_cell(slab, p, g.kabs, g.iy, ix, x1, hx, hy, hk, ox, oy, oxi, F);
        } else {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const BR lx = hx[u] + ox[u], ly = hy[u] + oy[u], lk = hk[u] + oxi[u];
            const BR fx = floor(lx), fy = floor(ly), fk = floor(lk);
            gather_slab(slab, p, g.kabs + (int)fk, g.iy + (int)fy, ix + (int)fx, lk - fk,
                        ly - fy, lx - fx, F[u]);
          }
        }
      }
      // push and loss; the deposit of each particle: values (dS, dJz, J_x, J_y) at offsets
      // (ox, oy, oxi) from home (a lost particle removes its reference: offsets 0)
      BR dv[2][4], dox[2], doy[2], doxi[2];
      bool post_home = true;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        dv[u][0] = dv[u][1] = dv[u][2] = dv[u][3] = BR(0);
        dox[u] = doy[u] = doxi[u] = BR(0);
        if (!ok[u]) continue;
        if (dw[u] == BR(-1)) {  // lost: only its reference, at home, is removed
          dv[u][0] = -refS;
          dv[u][1] = -refJz;
          continue;
        }
        if (PUSH) {
          boris_st(ux[u], uy[u], uz[u], F[u], bc);
          // dx/dt = u/gamma, dxi/dt = 1 - v_z = (1 + u_perp^2)/(gamma (gamma + u_z))
          BR ig, omv;
          drift_rates(ux[u], uy[u], uz_lead(uz[u], bc), ig, omv);
          ox[u] += cdx * ux[u] * ig;
          oy[u] += cdy * uy[u] * ig;
          oxi[u] += cdk * omv;
          const size_t s = si[u];
          b.ox[s] = ox[u];
          b.oy[s] = oy[u];
          b.oxi[s] = oxi[u];
          b.ux[s] = ux[u];
          b.uy[s] = uy[u];
          b.uz[s] = uz[u];
          if (hk[u] + oxi[u] >= BR(kleft)) {
            b.dw[s] = BR(-1);
            ++my_lost;
            dv[u][0] = -refS;
            dv[u][1] = -refJz;
            continue;
          }
        }
        {
          // xi cell relative to the home layer.  A live particle lies in [0, Lxi), so its cell
          // is at most the last one; a position given just below Lxi can round onto Lxi in the
          // working precision, and its cell must not name a slab node past the last one (the
          // pipelined schedule would wait for that node forever)
          const int cell = min((int)floor(hk[u] + oxi[u]), kleft - 1);
          cmax_t = max(cmax_t, g.kabs + cell);
          dmin_t = min(dmin_t, cell);
          if (ext.mom) {  // the moments, where asked for
            const BR wr = BR(1) + dw[u], duz = uz_dev(uz[u], bc);
            const BR mv[7] = {wr, wr * ux[u], wr * uy[u], wr * duz, wr * ux[u] * ux[u],
                              wr * uy[u] * uy[u], wr * duz * duz};
            if (cell == 0) {
#pragma unroll
              for (int k = 0; k < 7; ++k) mom_t[k] += mv[k];
            } else if (g.kabs + cell >= 0 && g.kabs + cell < p.nxi) {
              for (int k = 0; k < 7; ++k)
                atomicAdd(ext.mom + (size_t)(g.kabs + cell) * 7 + k, (double)mv[k]);
            }
          }
        }
        beam_sources(ux[u], uy[u], uz_lead(uz[u], bc), uz_dev(uz[u], bc), dw[u], bc, dv[u][0],
                     dv[u][1], dv[u][2], dv[u][3]);
        dox[u] = ox[u];
        doy[u] = oy[u];
        doxi[u] = oxi[u];
        post_home = post_home && in_cell(hx[u] + ox[u], hy[u] + oy[u], hk[u] + oxi[u]);
        // away from the slot's cell transversely (what re-homing within the layer can mend)
        if (ext.away) my_away += in_cell(hx[u] + ox[u], hy[u] + oy[u], BR(0)) ? 0 : 1;
      }
      if (lane_agg && __all_sync(0xffffffffu, post_home)) {
        // every particle of the warp's two sub-lattice positions is in its home cell: the two
        // particles of a thread share their eight corners, and the right corners of lane l
        // are the left corners of lane l + 1
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int ck = 0; ck < 2; ++ck) {
#pragma unroll
          for (int cy = 0; cy < 2; ++cy) {
            BR acc[2][4];
#pragma unroll
            for (int cx = 0; cx < 2; ++cx)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[cx][q] = BR(0);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              // the separable, telescoped weights of home_weights, one (ck, cy) row at a time
              const BR a3 = ck ? hk[u] : BR(1) - hk[u], d3 = ck ? doxi[u] : -doxi[u];
              const BR a2 = cy ? hy[u] : BR(1) - hy[u], d2 = cy ? doy[u] : -doy[u];
              const BR K = a3 + d3, YK = (a2 + d2) * K, T = d2 * K + a2 * d3;
#pragma unroll
              for (int cx = 0; cx < 2; ++cx) {
                const BR a1 = cx ? hx[u] : BR(1) - hx[u], d1 = cx ? dox[u] : -dox[u];
                const BR w = (a1 + d1) * YK, dW = d1 * YK + a1 * T;
                acc[cx][0] += dv[u][0] * w + refS * dW;
                acc[cx][1] += dv[u][1] * w + refJz * dW;
                acc[cx][2] += dv[u][2] * w;
                acc[cx][3] += dv[u][3] * w;
              }
            }
            BR* row = g.tile + (size_t)(ck * 4 + 1 + cy) * 4 * nx;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const BR from = __shfl_up_sync(0xffffffffu, acc[1][q], 1);
              atomicAdd(row + (size_t)q * nx + ix, acc[0][q] + (lane ? from : BR(0)));
              red_shared_if(lane == 31, row + (size_t)q * nx + x1, acc[1][q]);
            }
          }
        }
      } else {
        // the reference removed at home by the thread's particles that left the home cell:
        // summed per home corner over both particles, then one lane-aggregated deposit
        BR hw[2][2][2];
#pragma unroll
        for (int ck = 0; ck < 2; ++ck)
#pragma unroll
          for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx) hw[ck][cy][cx] = BR(0);
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (ok[u]) {
            const bool away = lane_agg && !in_cell(hx[u] + dox[u], hy[u] + doy[u], hk[u] + doxi[u]);
            deposit_particle(g, src, p, ix, hx[u], hy[u], hk[u], dox[u], doy[u], doxi[u],
                             dv[u][0], dv[u][1], dv[u][2], dv[u][3], refS, refJz, !away);
            if (away) {
#pragma unroll
              for (int ck = 0; ck < 2; ++ck)
#pragma unroll
                for (int cy = 0; cy < 2; ++cy)
#pragma unroll
                  for (int cx = 0; cx < 2; ++cx)
                    hw[ck][cy][cx] += (ck ? hk[u] : BR(1) - hk[u]) * (cy ? hy[u] : BR(1) - hy[u]) *
                                      (cx ? hx[u] : BR(1) - hx[u]);
            }
          }
        if (lane_agg) {
          const int lane = threadIdx.x & 31;
#pragma unroll
          for (int ck = 0; ck < 2; ++ck)
#pragma unroll
            for (int cy = 0; cy < 2; ++cy) {
              BR* row = g.tile + (size_t)(ck * 4 + 1 + cy) * 4 * nx;
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const BR rf = q ? -refJz : -refS;
                const BR lft = rf * hw[ck][cy][0], rgt = rf * hw[ck][cy][1];
                const BR from = __shfl_up_sync(0xffffffffu, rgt, 1);
                const BR v = lft + (lane ? from : BR(0));
                if (v != BR(0)) atomicAdd(row + (size_t)q * nx + ix, v);
                if (lane == 31 && rgt != BR(0)) atomicAdd(row + (size_t)q * nx + x1, rgt);
              }
            }
        }
      }
    }
  }
  cmax_t = warp_max(cmax_t);
  dmin_t = warp_min(dmin_t);
  if (ext.mom)
#pragma unroll
    for (int k = 0; k < 7; ++k) mom_t[k] = warp_sum(mom_t[k]);
  if ((threadIdx.x & 31) == 0) {
    if (cmax_t > s_ext[0]) atomicMax(&s_ext[0], cmax_t);
    if (dmin_t < 0) atomicMin(&s_ext[1], dmin_t);
    if (ext.mom)
      for (int k = 0; k < 7; ++k) atomicAdd(&s_mom[k], (double)mom_t[k]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ext.cmax && s_ext[0] >= 0) atomicMax(ext.cmax + g.kabs, s_ext[0]);
    if (ext.dmin && s_ext[1] < 0) atomicMin(ext.dmin, s_ext[1]);
    if (ext.mom && g.kabs < p.nxi)
      for (int k = 0; k < 7; ++k)
        if (s_mom[k] != 0.0) atomicAdd(ext.mom + (size_t)g.kabs * 7 + k, s_mom[k]);
  }
  const int outer = s_outer;  // final: every deposit preceded the barrier above
  for (int row = 0; row < 2 * 4; ++row) {  // node kabs + row / 4, grid row iy - 1 + row % 4
    const int k = g.kabs + (row >> 2);
    if (k >= p.nk) continue;
    // the outer rows hold something only where a deposit landed there
    if (((row & 3) == 0 || (row & 3) == 3) && !((outer >> row) & 1)) continue;
    BR* dst = src + ((size_t)k * p.ny + wrap(g.iy - 1 + (row & 3), p.ny)) * nx * 4;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const BR* t = g.tile + (size_t)row * 4 * nx + x;
      const BR t0 = t[0], t1 = t[nx], t2 = t[2 * nx], t3 = t[3 * nx];
      if (t0 != BR(0) || t1 != BR(0) || t2 != BR(0) || t3 != BR(0))
        red4(dst + (size_t)x * 4, t0, t1, t2, t3);
    }
  }
  if (my_lost && lost) atomicAdd(lost, (unsigned long long)my_lost);
  if (ext.away) {
    my_away = warp_sum(my_away);
    if ((threadIdx.x & 31) == 0 && my_away) atomicAdd(ext.away, (unsigned long long)my_away);
  }
  __syncthreads();  // the tile and s_ext are reused by the block's next group
}

// Grid: one block per (xi cell, row) group of the species.
template <typename BR, bool PUSH>
__global__ void __launch_bounds__(256, 2) beam_kernel(BeamArrays<BR> b, DevParams p, SpeciesDev sp,
                                                   BeamConst<BR> bc, const BR* __restrict__ slab,
                                                   BR* src, unsigned long long* lost, Extent ext) {
  extern __shared__ __align__(16) unsigned char smem[];
  beam_group<BR, PUSH>(b, p, sp, bc, slab, src, lost, ext, blockIdx.x,
                       reinterpret_cast<BR*>(smem));
}

template <typename BR>
__host__ __device__ inline size_t beam_smem_bytes(int nx) {
  return (size_t)2 * 4 * nx * 4 * sizeof(BR);
}

// Conversion between host fp64 arrays (canonical id order, absolute positions) and the
// device layout.
template <typename BR>
__global__ void beam_from_host_kernel(BeamArrays<BR> b, DevParams p, SpeciesDev sp,
                                      const double* x, const double* y, const double* xi,
                                      const double* ux, const double* uy, const double* uz,
                                      const double* w) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= b.n) return;
  const Home h = home_of(s, p.nx, p.ny, sp);
  const long long id = h.id;
  const double hx = h.ix + (h.sx + 0.5) / sp.ppx, hy = h.iy + (h.sy + 0.5) / sp.ppy;
  const double hk = sp.k0 + h.kxi + (h.sxi + 0.5) / sp.ppxi;
  // offsets from home, with the periodic image nearest to home; a lost particle (w = 0)
  // sits at home, whatever position it came with (it is never pushed or gathered for)
  const bool live = w[id] != 0.0;
  double ox = live ? x[id] / p.dx - hx : 0.0, oy = live ? y[id] / p.dy - hy : 0.0;
  ox -= p.nx * rint(ox / p.nx);
  oy -= p.ny * rint(oy / p.ny);
  b.ox[s] = BR(ox);
  b.oy[s] = BR(oy);
  b.oxi[s] = live ? BR(xi[id] / p.dxi - hk) : BR(0);
  b.ux[s] = BR(ux[id]);
  b.uy[s] = BR(uy[id]);
  uz_store(b.uz[s], uz[id], sp.uzb);
  b.dw[s] = (w[id] == 0.0) ? BR(-1) : BR(w[id] / sp.wbar - 1.0);
  if (b.id) b.id[s] = (unsigned)id;
}

template <typename BR>
__global__ void beam_to_host_kernel(BeamArrays<BR> b, DevParams p, SpeciesDev sp, double* x,
                                    double* y, double* xi, double* ux, double* uy, double* uz,
                                    double* w) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= b.n) return;
  const Home h = home_of(s, p.nx, p.ny, sp);
  // the particle in slot s (slot s's own until the beam has been re-homed)
  const long long id = b.id ? (long long)b.id[s] : h.id;
  const double hx = h.ix + (h.sx + 0.5) / sp.ppx, hy = h.iy + (h.sy + 0.5) / sp.ppy;
  const double hk = sp.k0 + h.kxi + (h.sxi + 0.5) / sp.ppxi;
  double xx = (hx + (double)b.ox[s]) * p.dx, yy = (hy + (double)b.oy[s]) * p.dy;
  xx -= p.Lx * floor(xx / p.Lx);
  yy -= p.Ly * floor(yy / p.Ly);
  x[id] = xx;
  y[id] = yy;
  xi[id] = (hk + (double)b.oxi[s]) * p.dxi;
  ux[id] = (double)b.ux[s];
  uy[id] = (double)b.uy[s];
  uz[id] = uz_value(b.uz[s], sp.uzb);
  w[id] = (b.dw[s] == BR(-1)) ? 0.0 : sp.wbar * (1.0 + (double)b.dw[s]);
}

}  // namespace qsa
