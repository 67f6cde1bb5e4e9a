// Plasma sweep: one persistent cooperative kernel that runs the whole xi-slice loop.
//
// Per slice j (notation of qsa.h; x at slices, u at half slices):
//   trial iterations it = 0..n_pc-1, each four phases separated by grid barriers
//     DEP : push every plasma particle from x^j with the current field guess, deposit
//           J^j (x, y, z) at x^j and J_perp^{j+1/2} at x^{j+1/2} into shared-memory tiles;
//     ROW : sum the tiles of each grid row, add the beam sources, real->half-spectrum FFT
//           along x (two real rows packed per complex transform);
//     COL : FFT along y per half-spectrum column, k-space solve of B_x, B_y (Helmholtz
//           shifted), B_z, E_z, inverse FFT along y;
//     IROW: half-spectrum->real inverse FFT along x; on the last iteration the slice's
//           fields go to the slab (E_x - B_y, E_y + B_x, E_z, B_x, B_y, B_z);
//   commit (four phases): push with the final fields, store x^{j+1}, u^{j+1/2}, deposit
//     S at x^{j+1} and J_perp^{j+1/2}, FFT, solve psi and its gradient for slice j+1.
// The k = 0 mode (psi0, E_z0) is integrated in FP64 registers by every block identically.
//
// Plasma particles are stored [home row iy][sub-lattice index][ix]: a warp holds 32
// neighbouring cells, and a block owns one home row (a "chunk") whose deposits land in a
// four-row shared-memory tile [iy-1, iy+2]; the tile goes to a per-chunk partial buffer that
// the row phase sums without atomics.  Particles that moved out of their tile deposit with
// global atomics into an overflow grid.
#pragma once
#include "qsa_common.cuh"
#include "qsa_fft.cuh"

namespace qsa {

constexpr int kNF = 5;  // deposit fields of a trial phase
constexpr int kTileRows = 4;

enum Diag : int {
  D_KAPPA = 0,  // sum 1/(1+psi) over particles -> kappa^2 after scaling
  D_JZ,         // <J_z> total
  D_PSI0,
  D_EZ0,
  D_CHARGE,     // sum over cells of the plasma (rho - J_z), times dx dy
  D_PCNUM,
  D_PCDEN,
  D_OPPMIN,     // ordered-key minimum of 1 + psi
  D_NFLOOR,
  D_INV,        // max invariant residual (non-negative double bits)
  D_E0,         // six energies D_E0..D_E0+5
  D_COUNT = D_E0 + 6
};

// Order-preserving map of a double to an unsigned key (min over keys = min over values).
__device__ __forceinline__ unsigned long long dkey(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

template <typename R>
struct SweepArgs {
  DevParams p;
  R *pox, *poy, *pux, *puy, *ppsi;          // plasma state (offsets in cells)
  R *psi, *gpx, *gpy, *bx, *by, *bz, *ez;   // real grids [ny][nx]
  R* part;                                  // [ny][4][nx][nf]
  R* ovf;                                   // [ny][nx][nf]
  C<R>* rspec;                              // [kNF][nxh][ny]
  C<R>* cspec;                              // [4][nxh][ny]
  C<R>* jprev;                              // [2][nxh][ny]  J_perp^{j-1/2} spectra
  C<R>* bold;                               // [2][nxh][ny]  B_perp spectra of the last solve
  const C<R>* twx;
  const C<R>* twy;
  const R* src;                             // [nk][ny][nx][4] beam S_b, J_z, J_x, J_y
  R* slab;                                  // [nk][ny][nx][8]
  double* diag;                             // [D_COUNT][nk]
  const double* bref;                       // [nk] beam J_z reference density per node
  Barrier bar;
};

// ------------------------------------------------------------------ particle helpers
template <typename R>
struct Cic {
  int x0, x1, y0, y1;  // wrapped nodes
  int ty;              // unwrapped lower row minus (chunk row - 1): tile row if in [0, 2]
  R fx, fy;
};

// CIC of a particle whose home cell is (ix, iy) at sub-cell position (lx, ly) in cells.
template <typename R>
__device__ __forceinline__ Cic<R> cic(int ix, int iy, R lx, R ly, int nx, int ny, int crow) {
  Cic<R> c;
  const R flx = floor(lx), fly = floor(ly);
  c.fx = lx - flx;
  c.fy = ly - fly;
  const int gx = ix + (int)flx, gy = iy + (int)fly;
  c.x0 = wrap(gx, nx);
  c.x1 = wrap(gx + 1, nx);
  c.y0 = wrap(gy, ny);
  c.y1 = wrap(gy + 1, ny);
  c.ty = gy - (crow - 1);
  return c;
}

template <typename R>
__device__ __forceinline__ R gather(const R* __restrict__ F, const Cic<R>& c, int nx) {
  const R a = F[c.y0 * nx + c.x0], b = F[c.y0 * nx + c.x1];
  const R d = F[c.y1 * nx + c.x0], e = F[c.y1 * nx + c.x1];
  const R gx = R(1) - c.fx, gy = R(1) - c.fy;
  return gy * (gx * a + c.fx * b) + c.fy * (gx * d + c.fx * e);
}

// Deposit v (already a density) at the four corners into the tile, or to the overflow grid
// when the rows fall outside the tile.
template <typename R>
__device__ __forceinline__ void deposit(R* tile, R* ovf, const Cic<R>& c, int f, int nf, int nx,
                                        R v) {
  const R gx = R(1) - c.fx, gy = R(1) - c.fy;
  const R w00 = gx * gy * v, w01 = c.fx * gy * v, w10 = gx * c.fy * v, w11 = c.fx * c.fy * v;
  if (c.ty >= 0 && c.ty <= kTileRows - 2) {
    R* r0 = tile + (size_t)c.ty * nx * nf;
    R* r1 = r0 + (size_t)nx * nf;
    atomicAdd(r0 + c.x0 * nf + f, w00);
    atomicAdd(r0 + c.x1 * nf + f, w01);
    atomicAdd(r1 + c.x0 * nf + f, w10);
    atomicAdd(r1 + c.x1 * nf + f, w11);
  } else {
    atomicAdd(ovf + ((size_t)c.y0 * nx + c.x0) * nf + f, w00);
    atomicAdd(ovf + ((size_t)c.y0 * nx + c.x1) * nf + f, w01);
    atomicAdd(ovf + ((size_t)c.y1 * nx + c.x0) * nf + f, w10);
    atomicAdd(ovf + ((size_t)c.y1 * nx + c.x1) * nf + f, w11);
  }
}

// Deposit v_dev W(x) + v_ref (W(x) - W(home)) for a particle of home cell (ix, crow), home
// sub-cell position (hx, hy) and offset (ox, oy) in cells.  v_ref W(home), summed over the
// quiet lattice, is uniform (k = 0 only) and is carried analytically by the caller; keeping
// it out of the grid sums lets FP32 accumulation resolve the fluctuations.  While the
// particle is in its home cell the weight differences are formed from the offsets without
// cancellation.
template <typename R>
__device__ __forceinline__ void deposit_ref(R* tile, R* ovf, int ix, int crow, R hx, R hy, R ox,
                                            R oy, int f, int nf, int nx, int ny, R v_dev,
                                            R v_ref) {
  const R lx = hx + ox, ly = hy + oy;
  if (lx >= R(0) && lx < R(1) && ly >= R(0) && ly < R(1)) {
    const R ax = R(1) - hx, ay = R(1) - hy;
    const R oxy = ox * oy;
    const R d00 = -ox * ay - oy * ax + oxy, d01 = ox * ay - hx * oy - oxy;
    const R d10 = ax * oy - ox * hy - oxy, d11 = hx * oy + ox * hy + oxy;
    const R w00 = (ax - ox) * (ay - oy), w01 = lx * (ay - oy), w10 = (ax - ox) * ly,
            w11 = lx * ly;
    const int x0 = ix, x1 = (ix + 1 == nx) ? 0 : ix + 1;
    R* r0 = tile + (size_t)1 * nx * nf;  // home row crow is tile row 1
    R* r1 = r0 + (size_t)nx * nf;
    atomicAdd(r0 + x0 * nf + f, v_dev * w00 + v_ref * d00);
    atomicAdd(r0 + x1 * nf + f, v_dev * w01 + v_ref * d01);
    atomicAdd(r1 + x0 * nf + f, v_dev * w10 + v_ref * d10);
    atomicAdd(r1 + x1 * nf + f, v_dev * w11 + v_ref * d11);
  } else {
    const Cic<R> c = cic<R>(ix, crow, lx, ly, nx, ny, crow);
    deposit(tile, ovf, c, f, nf, nx, v_dev + v_ref);
    const Cic<R> h = cic<R>(ix, crow, hx, hy, nx, ny, crow);
    deposit(tile, ovf, h, f, nf, nx, -v_ref);
  }
}

// gamma/(1+psi) from the quasistatic invariant gamma - u_z = 1 + psi.
template <typename R>
__device__ __forceinline__ R g_over_opp(R ux, R uy, R opp) {
  return (R(1) + ux * ux + uy * uy + opp * opp) / (R(2) * opp * opp);
}

// xi push u^{j-1/2} -> u^{j+1/2}: half kick, counter-clockwise rotation by
// 2 atan(dxi B_z/(2(1+psi))), half kick; gamma/(1+psi) of both kicks taken at the predicted
// pre-rotation momentum (the rotation keeps |u_perp|).
template <typename R>
__device__ __forceinline__ void push_xi(R& ux, R& uy, R opp, R gx, R gy, R bx, R by, R bz,
                                        R dxi) {
  const R h = R(0.5) * dxi;
  const R g0 = g_over_opp(ux, uy, opp);
  const R g = g_over_opp(ux + h * (g0 * gx - by), uy + h * (g0 * gy + bx), opp);
  const R kx = h * (g * gx - by), ky = h * (g * gy + bx);
  const R mx = ux + kx, my = uy + ky;
  const R t = h * bz / opp;
  const R s = R(2) * t / (R(1) + t * t);
  const R px = mx - t * my, py = my + t * mx;
  const R qx = mx - s * py, qy = my + s * px;
  ux = qx + kx;
  uy = qy + ky;
}

enum DepMode : int { DEP_INIT = 0, DEP_TRIAL = 1, DEP_COMMIT = 2 };

template <typename R>
__device__ void dep_phase(const SweepArgs<R>& a, R* tile, int mode, int j, double psi0,
                          bool first, bool last) {
  // reference state of the deposits: a particle at rest at its lattice home with psi = psi0
  // carries rho - J_z = -w and u_z/(1+psi) = c0 = -psi0 (2 + psi0) / (2 (1+psi0)^2)
  const double opp0d = 1.0 + psi0;
  const R opp0 = R(opp0d);
  const R c0 = R(-psi0 * (2.0 + psi0) / (2.0 * opp0d * opp0d));
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny;
  const int nf = (mode == DEP_TRIAL) ? kNF : 3;
  const int per_chunk = p.ppc * nx;
  const R wn = R(1) / R(p.ppc);  // w/(dx dy) of a plasma macroparticle
  const R dxi = R(p.dxi);
  const R idx = R(1) / R(p.dx), idy = R(1) / R(p.dy);
  const R floor_ = R(p.psi_floor);
  const int tile_elems = kTileRows * nx * nf;
  double kap = 0.0, inv = 0.0, omin = 1e300;
  unsigned long long nfloor = 0;
  __shared__ double red[32];

  for (int crow = blockIdx.x; crow < ny; crow += gridDim.x) {
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) tile[e] = R(0);
    __syncthreads();
    const size_t base = (size_t)crow * per_chunk;
    for (int t = threadIdx.x; t < per_chunk; t += blockDim.x) {
      const size_t i = base + t;
      const int sub = t / nx, ix = t - sub * nx;
      const int sx = sub % p.ppx, sy = sub / p.ppx;
      const R hx = (R(sx) + R(0.5)) / R(p.ppx), hy = (R(sy) + R(0.5)) / R(p.ppy);
      if (mode == DEP_INIT) {  // at home: rho - J_z equals its reference, nothing to add
        a.pox[i] = R(0);
        a.poy[i] = R(0);
        a.pux[i] = R(0);
        a.puy[i] = R(0);
        a.ppsi[i] = R(0);
        continue;
      }
      const R ox = a.pox[i], oy = a.poy[i];
      R ux = a.pux[i], uy = a.puy[i];
      const R pprev = a.ppsi[i];
      const Cic<R> c = cic<R>(ix, crow, hx + ox, hy + oy, nx, ny, crow);
      const R psi_fl = gather(a.psi, c, nx);
      const R psi_p = R(psi0 + (double)psi_fl);
      const R gxp = gather(a.gpx, c, nx), gyp = gather(a.gpy, c, nx);
      const R bxp = gather(a.bx, c, nx), byp = gather(a.by, c, nx), bzp = gather(a.bz, c, nx);
      const R opp_raw = R(1) + psi_p;
      const R opp = opp_raw < floor_ ? floor_ : opp_raw;
      R oph = R(1) + R(0.5) * (R(3) * psi_p - pprev);
      oph = oph < floor_ ? floor_ : oph;
      const R uxm = ux, uym = uy;
      push_xi(ux, uy, opp, gxp, gyp, bxp, byp, bzp, dxi);
      const R sh = R(0.5) * dxi / oph;
      const Cic<R> ch = cic<R>(ix, crow, hx + ox + sh * ux * idx, hy + oy + sh * uy * idy, nx, ny,
                               crow);
      const R jxh = -wn * ux / oph, jyh = -wn * uy / oph;
      if (mode == DEP_TRIAL) {
        const R uxj = R(0.5) * (uxm + ux), uyj = R(0.5) * (uym + uy);
        const R u2 = uxj * uxj + uyj * uyj;
        const R pe = opp - R(1);
        // u_z from gamma - u_z = 1 + psi without cancellation: (u^2 - psi (2 + psi)) / (2(1+psi))
        const R uzj = (u2 - pe * (R(2) + pe)) / (R(2) * opp);
        const R q = -wn / opp;
        // u_z/(1+psi) - c0 = u^2/(2 opp^2) + (1/opp^2 - 1/opp0^2)/2, the second term formed
        // from the psi fluctuation opp - opp0 without cancellation
        const R dpsi = (opp_raw < floor_) ? R((double)floor_ - opp0d) : psi_fl;
        const R iop2 = R(1) / (opp * opp);
        const R dz = R(0.5) * u2 * iop2 - R(0.5) * dpsi * (opp0 + opp) * iop2 / (opp0 * opp0);
        deposit(tile, a.ovf, c, 0, nf, nx, q * uxj);
        deposit(tile, a.ovf, c, 1, nf, nx, q * uyj);
        deposit_ref(tile, a.ovf, ix, crow, hx, hy, ox, oy, 2, nf, nx, ny, -wn * dz, -wn * c0);
        deposit(tile, a.ovf, ch, 3, nf, nx, jxh);
        deposit(tile, a.ovf, ch, 4, nf, nx, jyh);
        if (first) {
          kap += 1.0 / (double)opp;
          omin = fmin(omin, (double)opp_raw);
          if (opp_raw < floor_) ++nfloor;
        }
        if (last) {
          const R gam = (R(1) + u2 + opp * opp) / (R(2) * opp);
          inv = fmax(inv, (double)(fabs(gam - uzj - opp) / opp));
        }
      } else {  // commit
        const R sf = dxi / oph;
        a.pox[i] = ox + sf * ux * idx;
        a.poy[i] = oy + sf * uy * idy;
        a.pux[i] = ux;
        a.puy[i] = uy;
        a.ppsi[i] = psi_p;
        deposit_ref(tile, a.ovf, ix, crow, hx, hy, ox + sf * ux * idx, oy + sf * uy * idy, 0, nf,
                    nx, ny, R(0), -wn);
        deposit(tile, a.ovf, ch, 1, nf, nx, jxh);
        deposit(tile, a.ovf, ch, 2, nf, nx, jyh);
      }
    }
    __syncthreads();
    R* dst = a.part + (size_t)crow * tile_elems;
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) dst[e] = tile[e];
    __syncthreads();
  }
  if (mode == DEP_TRIAL && first) {
    double s = block_sum(kap, red);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(&a.diag[D_KAPPA * p.nk + j], s);
    double m = block_min(omin, red);
    if (threadIdx.x == 0 && m < 1e299) {
      atomicMin((unsigned long long*)&a.diag[D_OPPMIN * p.nk + j], dkey(m));
    }
    double nfl = block_sum((double)nfloor, red);
    if (threadIdx.x == 0 && nfl > 0) {
      atomicAdd(&a.diag[D_NFLOOR * p.nk + j], nfl);
      atomicOr(a.bar.status, ST_FLOOR);
    }
  }
  if (mode == DEP_TRIAL && last) {
    double m = block_max(inv, red);
    if (threadIdx.x == 0 && m > 0) atomic_max_nonneg(&a.diag[D_INV * p.nk + j], m);
  }
}

// ------------------------------------------------------------------ row phase (forward)
// mode DEP_TRIAL: fields Jx^j, Jy^j, Jz^j, Jx^{j+1/2}, Jy^{j+1/2} of slice j = jj.
// else: fields S, Jx^{jn-1/2}, Jy^{jn-1/2} of the new slice jn = jj.
template <typename R>
__device__ void row_phase(const SweepArgs<R>& a, C<R>* buf, int mode, int jj) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny, nxh = p.nxh, nk = p.nk;
  const int nf = (mode == DEP_TRIAL) ? kNF : 3;
  const int npair = (nf + 1) / 2;
  C<R>* A = buf;
  C<R>* B = buf + npair * nx;
  const int tile_elems = kTileRows * nx * nf;
  __shared__ double red[32];
  double charge = 0.0;
  for (int q = blockIdx.x; q < ny; q += gridDim.x) {
    for (int e = threadIdx.x; e < npair * nx; e += blockDim.x) {
      const int pr = e / nx, x = e - pr * nx;
      R v[2];
      for (int h = 0; h < 2; ++h) {
        const int f = 2 * pr + h;
        R s = R(0);
        if (f < nf) {
          for (int t = 0; t < kTileRows; ++t) {
            const int c = wrap(q + 1 - t, ny);
            s += a.part[(size_t)c * tile_elems + ((size_t)t * nx + x) * nf + f];
          }
          R* o = a.ovf + ((size_t)q * nx + x) * nf + f;
          s += *o;
          *o = R(0);
          // beam sources [nk][ny][nx][4]: 0 S_b, 1 J_z, 2 J_x, 3 J_y
          auto src = [&](int k, int comp) -> R {
            return (a.src != nullptr && k >= 0 && k < nk)
                       ? a.src[(((size_t)k * ny + q) * nx + x) * 4 + comp]
                       : R(0);
          };
          if (mode == DEP_TRIAL) {
            if (f == 0) s += src(jj, 2);
            else if (f == 1) s += src(jj, 3);
            else if (f == 2) s += src(jj, 1);
            else if (f == 3) s += R(0.5) * (src(jj, 2) + src(jj + 1, 2));
            else s += R(0.5) * (src(jj, 3) + src(jj + 1, 3));
          } else {
            if (f == 0) {
              charge += (double)s;
              s += src(jj, 0);
            } else if (f == 1) {
              s += R(0.5) * (src(jj - 1, 2) + src(jj, 2));
            } else {
              s += R(0.5) * (src(jj - 1, 3) + src(jj, 3));
            }
          }
        }
        v[h] = s;
      }
      A[pr * nx + x] = C<R>{v[0], v[1]};
    }
    __syncthreads();
    C<R>* Z = block_fft(A, B, npair, p.px, a.twx, -1);
    // unpack two real transforms: A_k = (Z_k + conj Z_{-k})/2, B_k = -i (Z_k - conj Z_{-k})/2
    for (int e = threadIdx.x; e < npair * nxh; e += blockDim.x) {
      const int pr = e / nxh, k = e - pr * nxh;
      const C<R> zk = Z[pr * nx + k];
      const C<R> zm = cconj(Z[pr * nx + (k == 0 ? 0 : nx - k)]);
      const C<R> fa = C<R>{R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y + zm.y)};
      const C<R> fb = C<R>{R(0.5) * (zk.y - zm.y), R(-0.5) * (zk.x - zm.x)};
      a.rspec[((size_t)(2 * pr) * nxh + k) * ny + q] = fa;
      if (2 * pr + 1 < nf) a.rspec[((size_t)(2 * pr + 1) * nxh + k) * ny + q] = fb;
    }
    __syncthreads();
  }
  if (mode != DEP_TRIAL) {
    double s = block_sum(charge, red);
    if (threadIdx.x == 0 && s != 0.0)
      atomicAdd(&a.diag[D_CHARGE * p.nk + jj], s * p.dx * p.dy);
  }
}

// Wavenumbers of half-spectrum column kx and row ky (derivative symbols zero at Nyquist).
struct Kv {
  double kx, ky, kxd, kyd, k2;
};
__device__ __forceinline__ Kv kvec(const DevParams& p, int kx, int ky) {
  Kv k;
  const int my = (ky <= p.ny / 2) ? ky : ky - p.ny;
  k.kx = 6.283185307179586476925 * kx / p.Lx;
  k.ky = 6.283185307179586476925 * my / p.Ly;
  k.kxd = ((p.nx % 2 == 0) && (2 * kx == p.nx)) ? 0.0 : k.kx;
  k.kyd = ((p.ny % 2 == 0) && (2 * ky == p.ny)) ? 0.0 : k.ky;
  k.k2 = k.kx * k.kx + k.ky * k.ky;
  return k;
}

// ------------------------------------------------------------------ column phase: B, E_z
// jz_ref: the uniform parts of J_z left out of the grid deposits (plasma reference state and
// beam reference density), added to <J_z> for the k = 0 mode.
template <typename R>
__device__ void col_phase_b(const SweepArgs<R>& a, C<R>* buf, int j, bool last, double jz_ref) {
  const DevParams& p = a.p;
  const int ny = p.ny, nxh = p.nxh;
  C<R>* A = buf;
  C<R>* B = buf + kNF * ny;
  const double kappa2 = a.diag[D_KAPPA * p.nk + j] / ((double)p.ppc * p.nx * p.ny);
  const R rdxi = R(1.0 / p.dxi);
  const R kap = R(kappa2);
  __shared__ double red[32];
  double num = 0.0, den = 0.0;
  for (int kx = blockIdx.x; kx < nxh; kx += gridDim.x) {
    for (int e = threadIdx.x; e < kNF * ny; e += blockDim.x) {
      const int f = e / ny, ky = e - f * ny;
      A[e] = a.rspec[((size_t)f * nxh + kx) * ny + ky];
    }
    __syncthreads();
    C<R>* Z = block_fft(A, B, kNF, p.py, a.twy, -1);
    C<R>* O = (Z == A) ? B : A;
    const double pw = (kx == 0 || ((p.nx % 2 == 0) && 2 * kx == p.nx)) ? 1.0 : 2.0;
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
      const C<R> Jx = Z[ky], Jy = Z[ny + ky], Jz = Z[2 * ny + ky];
      const C<R> Jxh = Z[3 * ny + ky], Jyh = Z[4 * ny + ky];
      const size_t ix0 = (size_t)kx * ny + ky, ix1 = ((size_t)nxh + kx) * ny + ky;
      if (kx == 0 && ky == 0)
        a.diag[D_JZ * p.nk + j] = (double)Jz.x / ((double)p.nx * p.ny) + jz_ref;
      const Kv k = kvec(p, kx, ky);
      C<R> obx{0, 0}, oby{0, 0}, obz{0, 0}, oez{0, 0};
      if (k.k2 > 0.0) {
        const R ik2 = R(1.0 / k.k2);
        const R kxd = R(k.kxd), kyd = R(k.kyd);
        const C<R> Jxp = a.jprev[ix0], Jyp = a.jprev[ix1];
        const C<R> Bxo = a.bold[ix0], Byo = a.bold[ix1];
        const C<R> Dx = cscale(csub(Jxh, Jxp), rdxi), Dy = cscale(csub(Jyh, Jyp), rdxi);
        // B_z = (i kx Jy - i ky Jx)/k^2 ; E_z = -(i kx Jx + i ky Jy)/k^2
        obz = cscale(cmuli(csub(cscale(Jy, kxd), cscale(Jx, kyd))), ik2);
        oez = cscale(cmuli(cadd(cscale(Jx, kxd), cscale(Jy, kyd))), -ik2);
        const R ih = R(1.0 / (k.k2 + kappa2));
        // (k^2 + kappa^2) B_x = i ky Jz + D_y + kappa^2 Bx_old
        obx = cscale(cadd(cadd(cmuli(cscale(Jz, kyd)), Dy), cscale(Bxo, kap)), ih);
        // (k^2 + kappa^2) B_y = -i kx Jz - D_x + kappa^2 By_old
        oby = cscale(csub(csub(cscale(Byo, kap), cmuli(cscale(Jz, kxd))), Dx), ih);
        if (last) {
          const double ex = (double)obx.x - Bxo.x, ey = (double)obx.y - Bxo.y;
          const double fx = (double)oby.x - Byo.x, fy = (double)oby.y - Byo.y;
          num += pw * (ex * ex + ey * ey + fx * fx + fy * fy);
          den += pw * ((double)obx.x * obx.x + (double)obx.y * obx.y + (double)oby.x * oby.x +
                       (double)oby.y * oby.y);
        }
      }
      a.bold[ix0] = obx;
      a.bold[ix1] = oby;
      O[ky] = obx;
      O[ny + ky] = oby;
      O[2 * ny + ky] = obz;
      O[3 * ny + ky] = oez;
    }
    __syncthreads();
    C<R>* W = block_fft(O, Z, 4, p.py, a.twy, +1);
    for (int e = threadIdx.x; e < 4 * ny; e += blockDim.x) {
      const int f = e / ny, ky = e - f * ny;
      a.cspec[((size_t)f * nxh + kx) * ny + ky] = W[e];
    }
    __syncthreads();
  }
  if (last) {
    double s = block_sum(num, red);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(&a.diag[D_PCNUM * p.nk + j], s);
    s = block_sum(den, red);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(&a.diag[D_PCDEN * p.nk + j], s);
  }
}

// ------------------------------------------------------------------ column phase: psi
template <typename R>
__device__ void col_phase_psi(const SweepArgs<R>& a, C<R>* buf) {
  const DevParams& p = a.p;
  const int ny = p.ny, nxh = p.nxh;
  C<R>* A = buf;
  C<R>* B = buf + 3 * ny;
  for (int kx = blockIdx.x; kx < nxh; kx += gridDim.x) {
    for (int e = threadIdx.x; e < 3 * ny; e += blockDim.x) {
      const int f = e / ny, ky = e - f * ny;
      A[e] = a.rspec[((size_t)f * nxh + kx) * ny + ky];
    }
    __syncthreads();
    C<R>* Z = block_fft(A, B, 3, p.py, a.twy, -1);
    C<R>* O = (Z == A) ? B : A;
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
      const size_t ix0 = (size_t)kx * ny + ky, ix1 = ((size_t)nxh + kx) * ny + ky;
      a.jprev[ix0] = Z[ny + ky];
      a.jprev[ix1] = Z[2 * ny + ky];
      const Kv k = kvec(p, kx, ky);
      C<R> ps{0, 0};
      if (k.k2 > 0.0) ps = cscale(Z[ky], R(1.0 / k.k2));
      O[ky] = ps;
      O[ny + ky] = cmuli(cscale(ps, R(k.kxd)));
      O[2 * ny + ky] = cmuli(cscale(ps, R(k.kyd)));
    }
    __syncthreads();
    C<R>* W = block_fft(O, Z, 3, p.py, a.twy, +1);
    for (int e = threadIdx.x; e < 3 * ny; e += blockDim.x) {
      const int f = e / ny, ky = e - f * ny;
      a.cspec[((size_t)f * nxh + kx) * ny + ky] = W[e];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ inverse row phase
// psi_mode: outputs psi, d_x psi, d_y psi.  Else: B_x, B_y, B_z, E_z; on the last trial
// iteration also the slab of slice j and the field energies.
template <typename R>
__device__ void irow_phase(const SweepArgs<R>& a, C<R>* buf, bool psi_mode, int j, bool last,
                           double ez0j) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny, nxh = p.nxh;
  const int nout = psi_mode ? 3 : 4;
  const int npair = (nout + 1) / 2;
  C<R>* A = buf;
  C<R>* B = buf + npair * nx;
  const R scale = R(1.0 / ((double)nx * ny));
  R* outs[4];
  if (psi_mode) {
    outs[0] = a.psi; outs[1] = a.gpx; outs[2] = a.gpy; outs[3] = nullptr;
  } else {
    outs[0] = a.bx; outs[1] = a.by; outs[2] = a.bz; outs[3] = a.ez;
  }
  __shared__ double red[32];
  double en[6] = {0, 0, 0, 0, 0, 0};
  bool bad = false;
  for (int q = blockIdx.x; q < ny; q += gridDim.x) {
    for (int e = threadIdx.x; e < npair * nx; e += blockDim.x) {
      const int pr = e / nx, k = e - pr * nx;
      const int f0 = 2 * pr, f1 = 2 * pr + 1;
      // full spectrum of z = a + i b from the half spectra of the real outputs a, b
      const int kk = (k < nxh) ? k : nx - k;
      C<R> fa = a.cspec[((size_t)f0 * nxh + kk) * ny + q];
      C<R> fb = (f1 < nout) ? a.cspec[((size_t)f1 * nxh + kk) * ny + q] : C<R>{0, 0};
      const bool selfconj = (kk == 0) || ((nx % 2 == 0) && 2 * kk == nx);
      if (selfconj) {
        fa.y = R(0);
        fb.y = R(0);
      }
      if (k >= nxh) {
        fa = cconj(fa);
        fb = cconj(fb);
      }
      A[pr * nx + k] = cadd(fa, cmuli(fb));
    }
    __syncthreads();
    C<R>* Z = block_fft(A, B, npair, p.px, a.twx, +1);
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      R v[4];
      for (int pr = 0; pr < npair; ++pr) {
        v[2 * pr] = Z[pr * nx + x].x * scale;
        if (2 * pr + 1 < 4) v[2 * pr + 1] = Z[pr * nx + x].y * scale;
      }
      const size_t g = (size_t)q * nx + x;
      for (int f = 0; f < nout; ++f) outs[f][g] = v[f];
      if (!psi_mode && last) {
        const R wx = -a.gpx[g], wy = -a.gpy[g];
        const R ez = R(ez0j + (double)v[3]);
        R* s = a.slab + (((size_t)j * ny + q) * nx + x) * 8;
        s[0] = wx;
        s[1] = wy;
        s[2] = ez;
        s[3] = v[0];
        s[4] = v[1];
        s[5] = v[2];
        s[6] = R(0);
        s[7] = R(0);
        const double Ex = (double)wx + v[1], Ey = (double)wy - v[0];
        en[0] += Ex * Ex;
        en[1] += Ey * Ey;
        en[2] += (double)ez * ez;
        en[3] += (double)v[0] * v[0];
        en[4] += (double)v[1] * v[1];
        en[5] += (double)v[2] * v[2];
        if (!(isfinite((double)wx) && isfinite((double)wy) && isfinite((double)ez) &&
              isfinite((double)v[0]) && isfinite((double)v[1]) && isfinite((double)v[2])))
          bad = true;
      }
    }
    __syncthreads();
  }
  if (!psi_mode && last) {
    const double cell = 0.5 * p.dx * p.dy * p.dxi;
    for (int f = 0; f < 6; ++f) {
      double s = block_sum(en[f], red);
      if (threadIdx.x == 0 && s != 0.0) atomicAdd(&a.diag[(D_E0 + f) * p.nk + j], s * cell);
    }
    if (bad) atomicOr(a.bar.status, ST_NONFINITE);
  }
}

// ------------------------------------------------------------------ the kernel
template <typename R>
__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* tile = reinterpret_cast<R*>(smem);
  C<R>* buf = reinterpret_cast<C<R>*>(smem);
  const DevParams& p = a.p;
  double psi0 = 0.0, ez0h = 0.0;

  dep_phase(a, tile, DEP_INIT, 0, 0.0, false, false);
  if (!grid_sync(a.bar)) return;
  row_phase(a, buf, DEP_INIT, 0);
  if (!grid_sync(a.bar)) return;
  col_phase_psi(a, buf);
  if (!grid_sync(a.bar)) return;
  irow_phase(a, buf, true, 0, false, 0.0);
  if (!grid_sync(a.bar)) return;

  for (int j = 0; j < p.nk; ++j) {
    double ez0n = ez0h, ez0j = ez0h;
    const double opp0 = 1.0 + psi0;
    const double jz_ref = psi0 * (2.0 + psi0) / (2.0 * opp0 * opp0) + (a.bref ? a.bref[j] : 0.0);
    for (int it = 0; it < p.n_pc; ++it) {
      const bool first = (it == 0), last = (it == p.n_pc - 1);
      dep_phase(a, tile, DEP_TRIAL, j, psi0, first, last);
      if (!grid_sync(a.bar)) return;
      row_phase(a, buf, DEP_TRIAL, j);
      if (!grid_sync(a.bar)) return;
      col_phase_b(a, buf, j, last, jz_ref);
      if (!grid_sync(a.bar)) return;
      if (last) {
        const double jz = *((volatile double*)&a.diag[D_JZ * p.nk + j]);
        ez0n = ez0h - p.dxi * jz;
        ez0j = 0.5 * (ez0h + ez0n);
      }
      irow_phase(a, buf, false, j, last, ez0j);
      if (!grid_sync(a.bar)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.diag[D_PSI0 * p.nk + j] = psi0;
      a.diag[D_EZ0 * p.nk + j] = ez0j;
    }
    if (j + 1 < p.nk) {
      dep_phase(a, tile, DEP_COMMIT, j, psi0, false, false);
      if (!grid_sync(a.bar)) return;
      row_phase(a, buf, DEP_COMMIT, j + 1);
      if (!grid_sync(a.bar)) return;
      col_phase_psi(a, buf);
      if (!grid_sync(a.bar)) return;
      irow_phase(a, buf, true, j + 1, false, 0.0);
      if (!grid_sync(a.bar)) return;
    }
    psi0 += p.dxi * ez0n;
    ez0h = ez0n;
  }
}

// Standalone transverse solve through the same phases: which = 0 solves B_x, B_y, B_z, E_z
// from the five trial fields placed in the overflow grid; which = 1 solves psi and its
// gradient from S placed in the overflow grid (field 0 of three).
template <typename R>
__global__ void __launch_bounds__(256) solve_kernel(SweepArgs<R> a, int which) {
  extern __shared__ __align__(16) unsigned char smem[];
  C<R>* buf = reinterpret_cast<C<R>*>(smem);
  if (which == 0) {
    row_phase(a, buf, DEP_TRIAL, 0);
    if (!grid_sync(a.bar)) return;
    col_phase_b(a, buf, 0, false, 0.0);
    if (!grid_sync(a.bar)) return;
    irow_phase(a, buf, false, 0, false, 0.0);
  } else {
    row_phase(a, buf, DEP_COMMIT, 0);
    if (!grid_sync(a.bar)) return;
    col_phase_psi(a, buf);
    if (!grid_sync(a.bar)) return;
    irow_phase(a, buf, true, 0, false, 0.0);
  }
}

}  // namespace qsa
