// Discrete adjoint of the QS-PIC step (FP64): the plasma sweep, the beam-source deposit and
// the beam push, differentiated exactly as the forward scheme computes them (the scheme the
// FP64 oracle states), so that the gradient of a loss of the final sweep's fields with respect
// to every beam macroparticle weight comes out of one backward pass.  The seeded mode
// amplitudes and the density ratio alpha of the paper's beam (section "Quasistatic model")
// enter the run only through these weights.
//
// Notation (forward, slice j of one sweep, as in the oracle's plasma_sweep): particle state
// x^j, u^{j-1/2}, psi_prev; psi_p = psi0 + <psi>(x^j), opp = 1 + psi_p,
// oph = 1 + (3 psi_p - psi_prev)/2, g = <grad psi>(x^j); kappa^2 = sum w/opp / (Lx Ly);
// for each of n_pc solves: b = <B guess>(x^j), u^{j+1/2} = push(u^{j-1/2}, opp, g, b),
// J^j deposited at x^j with u^j = (u^{j-1/2} + u^{j+1/2})/2, J_perp^{j+1/2} at
// x^{j+1/2} = x^j + dxi u^{j+1/2}/(2 oph), then E_z, B_z from J_perp^j and the shifted B_perp
// solve from J_z^j and D = (J_perp^{j+1/2} - J_perp^{j-1/2})/dxi; the commit pushes with the
// final fields, moves x^{j+1} = x^j + dxi u^{j+1/2}/oph, deposits J_perp^{j+1/2} and the
// charge at x^{j+1}, whose psi solve gives slice j+1's psi and grad psi.  The k = 0 mode:
// ez0n = ez0h - dxi <J_z>, E_z0^j = (ez0h + ez0n)/2, psi0 += dxi ez0n.
//
// The adjoint runs the slices backwards.  Adjoints of deposits are gathers of the adjoint
// grid (and of the weight function's gradient for the particle position); adjoints of gathers
// are deposits (atomics).  A spectral solve multiplies by a symbol sigma(k); its adjoint
// multiplies by conj(sigma(k)) (the forward transform unnormalised, the inverse divided by
// nx ny).  The psi floor is taken as inactive (the caller checks that no particle met it).
#pragma once
#include "qsa_beam.cuh"
#include "qsa_fft.cuh"
#include "qsa_sweep.cuh"

namespace qsa {

// ------------------------------------------------------------------ CIC with gradients
struct CicG {
  int x0, x1, y0, y1;
  double fx, fy;
};
__device__ __forceinline__ CicG cic_g(double x, double y, double idx, double idy, int nx,
                                      int ny) {
  CicG c;
  const double gx = x * idx, gy = y * idy;
  const double fx0 = floor(gx), fy0 = floor(gy);
  c.fx = gx - fx0;
  c.fy = gy - fy0;
  c.x0 = wrap((int)fx0, nx);
  c.x1 = wrap((int)fx0 + 1, nx);
  c.y0 = wrap((int)fy0, ny);
  c.y1 = wrap((int)fy0 + 1, ny);
  return c;
}
// Value of grid F (element stride `st`) at c and its x, y derivatives (per unit length).
__device__ __forceinline__ double gat(const double* F, const CicG& c, int nx, int st,
                                      double idx, double idy, double& dvx, double& dvy) {
  const double f00 = F[((size_t)c.y0 * nx + c.x0) * st], f01 = F[((size_t)c.y0 * nx + c.x1) * st];
  const double f10 = F[((size_t)c.y1 * nx + c.x0) * st], f11 = F[((size_t)c.y1 * nx + c.x1) * st];
  const double gx = 1.0 - c.fx, gy = 1.0 - c.fy;
  dvx = (gy * (f01 - f00) + c.fy * (f11 - f10)) * idx;
  dvy = (gx * (f10 - f00) + c.fx * (f11 - f01)) * idy;
  return gy * (gx * f00 + c.fx * f01) + c.fy * (gx * f10 + c.fx * f11);
}
__device__ __forceinline__ double gat0(const double* F, const CicG& c, int nx, int st) {
  const double gx = 1.0 - c.fx, gy = 1.0 - c.fy;
  return gy * (gx * F[((size_t)c.y0 * nx + c.x0) * st] + c.fx * F[((size_t)c.y0 * nx + c.x1) * st]) +
         c.fy * (gx * F[((size_t)c.y1 * nx + c.x0) * st] + c.fx * F[((size_t)c.y1 * nx + c.x1) * st]);
}
// Adjoint of a gather: F += W(x) v at the four corners.
__device__ __forceinline__ void scat(double* F, const CicG& c, int nx, double v) {
  if (v == 0.0) return;
  const double gx = 1.0 - c.fx, gy = 1.0 - c.fy;
  atomicAdd(F + (size_t)c.y0 * nx + c.x0, gy * gx * v);
  atomicAdd(F + (size_t)c.y0 * nx + c.x1, gy * c.fx * v);
  atomicAdd(F + (size_t)c.y1 * nx + c.x0, c.fy * gx * v);
  atomicAdd(F + (size_t)c.y1 * nx + c.x1, c.fy * c.fx * v);
}

// ------------------------------------------------------------------ xi push and its adjoint
// Forward of push_xi (the same operations as the sweep's push) with the intermediate values
// kept for the reverse pass.
struct PushT {
  double ux, uy, opp, gx, gy, bx, by, bz;  // inputs
  double h, g0, px0, py0, g, kx, ky, mx, my, t, s, px, py;
  double ox, oy;  // outputs
};
__device__ __forceinline__ void push_fwd(PushT& P, double dxi) {
  const double h = 0.5 * dxi, o2 = P.opp * P.opp;
  P.h = h;
  P.g0 = (1.0 + P.ux * P.ux + P.uy * P.uy + o2) / (2.0 * o2);
  P.px0 = P.ux + h * (P.g0 * P.gx - P.by);
  P.py0 = P.uy + h * (P.g0 * P.gy + P.bx);
  P.g = (1.0 + P.px0 * P.px0 + P.py0 * P.py0 + o2) / (2.0 * o2);
  P.kx = h * (P.g * P.gx - P.by);
  P.ky = h * (P.g * P.gy + P.bx);
  P.mx = P.ux + P.kx;
  P.my = P.uy + P.ky;
  P.t = h * P.bz / P.opp;
  P.s = 2.0 * P.t / (1.0 + P.t * P.t);
  P.px = P.mx - P.t * P.my;
  P.py = P.my + P.t * P.mx;
  P.ox = P.mx - P.s * P.py + P.kx;
  P.oy = P.my + P.s * P.px + P.ky;
}
// Reverse of push_fwd: given the adjoints (lox, loy) of the outputs, adds the adjoints of
// the inputs into l[8] = (ux, uy, opp, gx, gy, bx, by, bz).
__device__ __forceinline__ void push_adj(const PushT& P, double lox, double loy, double l[8]) {
  const double h = P.h, o2 = P.opp * P.opp, o3 = o2 * P.opp;
  // ox = qx + kx, qx = mx - s py ; oy = qy + ky, qy = my + s px
  double lkx = lox, lky = loy, lmx = lox, lmy = loy;
  double ls = -P.py * lox + P.px * loy;
  double lpy = -P.s * lox, lpx = P.s * loy;
  // px = mx - t my ; py = my + t mx
  lmx += lpx + P.t * lpy;
  lmy += lpy - P.t * lpx;
  double lt = -P.my * lpx + P.mx * lpy;
  // s = 2t/(1+t^2)
  const double tt = 1.0 + P.t * P.t;
  lt += ls * 2.0 * (1.0 - P.t * P.t) / (tt * tt);
  // t = h bz/opp
  l[7] += lt * h / P.opp;
  l[2] -= lt * P.t / P.opp;
  // mx = ux + kx ; my = uy + ky
  l[0] += lmx;
  l[1] += lmy;
  lkx += lmx;
  lky += lmy;
  // kx = h (g gx - by) ; ky = h (g gy + bx)
  double lg = h * (lkx * P.gx + lky * P.gy);
  l[3] += lkx * h * P.g;
  l[4] += lky * h * P.g;
  l[6] -= lkx * h;
  l[5] += lky * h;
  // g = (1 + px0^2 + py0^2 + opp^2)/(2 opp^2)
  const double lpx0 = lg * P.px0 / o2, lpy0 = lg * P.py0 / o2;
  l[2] -= lg * (1.0 + P.px0 * P.px0 + P.py0 * P.py0) / o3;
  // px0 = ux + h (g0 gx - by) ; py0 = uy + h (g0 gy + bx)
  l[0] += lpx0;
  l[1] += lpy0;
  const double lg0 = h * (lpx0 * P.gx + lpy0 * P.gy);
  l[3] += lpx0 * h * P.g0;
  l[4] += lpy0 * h * P.g0;
  l[6] -= lpx0 * h;
  l[5] += lpy0 * h;
  // g0 = (1 + ux^2 + uy^2 + opp^2)/(2 opp^2)
  l[0] += lg0 * P.ux / o2;
  l[1] += lg0 * P.uy / o2;
  l[2] -= lg0 * (1.0 + P.ux * P.ux + P.uy * P.uy) / o3;
}

// ------------------------------------------------------------------ arguments
struct AdjArgs {
  DevParams p;
  double w;              // plasma macroparticle weight dx dy / ppc
  double idx, idy;       // 1/dx, 1/dy
  double dv;             // 1/(dx dy): deposit normalisation
  double inv_LxLy;
  // the forward record of this sweep and its per-slice scalars
  Tape<double> tape;
  const double* psi0;    // [nk]
  const double* kappa2;  // [nk]
  // adjoint inputs and outputs
  const double* lslab;   // [nk][ny][nx][8]: adjoint of the slab (W_x, W_y, E_z, B_x, B_y, B_z)
  double* lsrc;          // [nk][ny][nx][4]: adjoint of the beam sources S_b, J_z, J_x, J_y
  // per-particle adjoints [np] (carried between slices, and per-slice accumulators)
  double *lx, *ly, *lux, *luy, *lpp, *lopp, *loph, *lgx, *lgy;
  // adjoint grids [ny][nx]
  double* lpsi[2][3];    // adjoint of (psi, d_x psi, d_y psi) of a slice (double buffer)
  double* lB[2][3];      // adjoint of a B field guess (B_x, B_y, B_z) (double buffer)
  double* ljp[2][2];     // adjoint of J_perp^{j-1/2} (x, y) (double buffer)
  double* lS;            // adjoint of the charge source of a psi solve
  double* lJ[5];         // J_x^j, J_y^j, J_z^j, J_x^{j+1/2}, J_y^{j+1/2} adjoints of a solve
  C<double>* zs;         // spectral scratch [8][ny][nx]
  C<double>* zt;         // spectral scratch [8][ny][nx]
  const C<double>* twx;
  const C<double>* twy;
  const double* ktab;    // wavenumbers (half spectrum along x; see kvec)
  double* part;          // [gridDim][4] per-block partial sums
  Barrier bar;
};

// Wavenumber and derivative symbol of full-spectrum index m along an axis whose half table
// holds nh = n/2 + 1 entries (k at [off + m], derivative symbol at [off + nh + m]... for x);
// the y table already covers every index.
__device__ __forceinline__ void kx_full(const double* kt, int nxh, int nx, int m, double& k,
                                        double& kd) {
  if (m < nxh) {
    k = kt[m];
    kd = kt[nxh + m];
  } else {
    k = -kt[nx - m];
    kd = -kt[nxh + nx - m];
  }
}

// ------------------------------------------------------------------ spectral operator
// One linear operator applied in k-space to nin real grids, giving nout real grids, in three
// grid-wide phases: forward row transforms, column transforms + pointwise map + inverse column
// transforms, inverse row transforms.  `op` maps the input spectra at (kx, ky) to the
// outputs; `out` receives every output value (cell, output index, value).
enum SpecOp : int { OP_PSI = 0, OP_SOLVE = 1 };

// Input f is the real grid in[f] with element stride ist[f] (null: zero).
__device__ void spec_rows_fwd(const AdjArgs& a, const double* const* in, const int* ist, int nin,
                              C<double>* buf, C<double>* tw) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny;
  load_tw(tw, a.twx, nx);
  __syncthreads();
  for (int u = blockIdx.x; u < nin * ny; u += gridDim.x) {
    const int f = u / ny, q = u - f * ny;
    const double* row = in[f];
    const int es = ist[f];
    for (int x = threadIdx.x; x < nx; x += blockDim.x)
      buf[x] = C<double>{row ? row[((size_t)q * nx + x) * es] : 0.0, 0.0};
    __syncthreads();
    C<double>* Z = block_fft(buf, buf + nx, 1, p.px, tw, -1);
    C<double>* dst = a.zs + ((size_t)f * ny + q) * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = Z[x];
    __syncthreads();
  }
}

__device__ void spec_cols(const AdjArgs& a, int op, int nin, int nout, double kap,
                          C<double>* buf, C<double>* tw) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny;
  load_tw(tw, a.twy, ny);
  __syncthreads();
  C<double>* A = buf;
  C<double>* B = buf + 8 * ny;
  for (int kx = blockIdx.x; kx < nx; kx += gridDim.x) {
    for (int e = threadIdx.x; e < nin * ny; e += blockDim.x) {
      const int f = e / ny, q = e - f * ny;
      A[e] = a.zs[((size_t)f * ny + q) * nx + kx];
    }
    __syncthreads();
    C<double>* Z = block_fft(A, B, nin, p.py, tw, -1);
    C<double>* O = (Z == A) ? B : A;
    double kxv, kxd;
    kx_full(a.ktab, p.nxh, nx, kx, kxv, kxd);
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
      const double kyv = a.ktab[2 * p.nxh + ky], kyd = a.ktab[2 * p.nxh + ny + ky];
      const double k2 = kxv * kxv + kyv * kyv;
      const double ik2 = k2 > 0.0 ? 1.0 / k2 : 0.0;
      if (op == OP_PSI) {
        // psi^ = S^/k^2, (d_x, d_y) psi^ = i k_d psi^: adjoint (L_psi - i kxd L_gx - i kyd L_gy)/k^2
        const C<double> lp = Z[ky], lgx = Z[ny + ky], lgy = Z[2 * ny + ky];
        C<double> r = csub(csub(lp, cscale(cmuli(lgx), kxd)), cscale(cmuli(lgy), kyd));
        O[ky] = cscale(r, ik2);
      } else {
        // inputs L_Bx, L_By, L_Bz, L_Ez; outputs L_Jx, L_Jy, L_Jz, L_Dx, L_Dy
        const C<double> lbx = Z[ky], lby = Z[ny + ky], lbz = Z[2 * ny + ky],
                        lez = Z[3 * ny + ky];
        const double hh = k2 > 0.0 ? 1.0 / (k2 + kap) : 0.0;
        // E_z^ = -i (kxd J_x + kyd J_y)/k^2, B_z^ = i (kxd J_y - kyd J_x)/k^2
        O[ky] = cscale(cadd(cscale(cmuli(lez), kxd), cscale(cmuli(lbz), kyd)), ik2);
        O[ny + ky] = cscale(csub(cscale(cmuli(lez), kyd), cscale(cmuli(lbz), kxd)), ik2);
        // B_x^ = H (i kyd J_z + D_y + kap B_x_old), B_y^ = H (-i kxd J_z - D_x + kap B_y_old)
        O[2 * ny + ky] = cscale(csub(cscale(cmuli(lby), kxd), cscale(cmuli(lbx), kyd)), hh);
        O[3 * ny + ky] = cscale(lby, -hh);
        O[4 * ny + ky] = cscale(lbx, hh);
      }
    }
    __syncthreads();
    C<double>* W = block_fft(O, Z, nout, p.py, tw, +1);
    for (int e = threadIdx.x; e < nout * ny; e += blockDim.x) {
      const int f = e / ny, q = e - f * ny;
      a.zt[((size_t)f * ny + q) * nx + kx] = W[e];
    }
    __syncthreads();
  }
}

// Inverse row transforms: output o of row q, scaled by 1/(nx ny), to `emit(cell, o, value)`.
template <typename Emit>
__device__ void spec_rows_inv(const AdjArgs& a, int nout, C<double>* buf, C<double>* tw,
                              Emit emit) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny;
  const double sc = 1.0 / ((double)nx * ny);
  load_tw(tw, a.twx, nx);
  __syncthreads();
  for (int u = blockIdx.x; u < nout * ny; u += gridDim.x) {
    const int o = u / ny, q = u - o * ny;
    const C<double>* srcr = a.zt + ((size_t)o * ny + q) * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) buf[x] = srcr[x];
    __syncthreads();
    C<double>* Z = block_fft(buf, buf + nx, 1, p.px, tw, +1);
    for (int x = threadIdx.x; x < nx; x += blockDim.x) emit((size_t)q * nx + x, o, Z[x].x * sc);
    __syncthreads();
  }
}

__host__ __device__ inline size_t adj_smem_bytes(int nx, int ny) {
  const size_t rows = (size_t)2 * nx * sizeof(C<double>);
  const size_t cols = (size_t)16 * ny * sizeof(C<double>);
  const size_t m = rows > cols ? rows : cols;
  return m + (size_t)(nx > ny ? nx : ny) * sizeof(C<double>) + 64;
}

// Sum over blocks of per-block partial `k` (read through L2), identical in every block;
// valid in thread 0.
__device__ double sum_parts(const AdjArgs& a, int k, double* red) {
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(a.part + (size_t)b * 4 + k);
  return block_sum_lo(v, red);
}

// ------------------------------------------------------------------ the adjoint sweep
// One cooperative launch runs the slices nk-1 .. 0 backwards.  Inputs: the tape of the
// forward sweep, its psi0 and kappa^2 per slice, and lslab; output: lsrc (accumulated; the
// caller zeroes it).  Every grid buffer of AdjArgs starts at zero (the caller clears them).
__global__ void __launch_bounds__(256, 1) adj_sweep_kernel(AdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  C<double>* tw = reinterpret_cast<C<double>*>(smem);
  C<double>* buf = tw + (a.p.nx > a.p.ny ? a.p.nx : a.p.ny);
  __shared__ double red[32];
  __shared__ double s_lez0, s_lez0n, s_ljz, s_lkap;
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny, nk = p.nk, n_pc = p.n_pc;
  const size_t g = (size_t)nx * ny, np = (size_t)p.np;
  const double dxi = p.dxi, w = a.w, dv = a.dv;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  unsigned epoch = 0;
  // carried scalars (identical in every block): adjoints of psi0 and ez0h of slice j + 1
  double lpsi0n = 0.0, lez0hn = 0.0;
  for (int j = nk - 1; j >= 0; --j) {
    const int cur = j & 1, nxt = cur ^ 1;  // lpsi[nxt]: slice j + 1's; lpsi[cur]: slice j's
    const double* tfg0 = a.tape.fg + (size_t)j * (n_pc + 1) * g * kFG;  // snap 0 of slice j
    const double* tpart = a.tape.part + (size_t)j * 5 * np;
    const double* slab = a.lslab + (size_t)j * g * 8;
    const double kap = a.kappa2[j], psi0 = a.psi0[j];
    // ---- P1: the psi solve of slice j + 1 (rows), and the slab's adjoint of slice j
    {
      double ez = 0.0;
      for (size_t c = t0; c < g; c += st) {
        const double* e = slab + c * 8;
        a.lpsi[cur][0][c] = 0.0;
        a.lpsi[cur][1][c] = -e[0];  // W_x = -d_x psi
        a.lpsi[cur][2][c] = -e[1];  // W_y = -d_y psi
        // the final B of slice j: carried guess adjoint of slice j + 1 (lB[0]) + slab
        a.lB[0][0][c] += e[3];
        a.lB[0][1][c] += e[4];
        a.lB[0][2][c] += e[5];
        a.ljp[cur][0][c] = 0.0;
        a.ljp[cur][1][c] = 0.0;
        ez += e[2];
      }
      const double s = block_sum_lo(ez, red);
      if (threadIdx.x == 0) a.part[(size_t)blockIdx.x * 4 + 0] = s;
      if (j + 1 < nk) {
        const double* ins[3] = {a.lpsi[nxt][0], a.lpsi[nxt][1], a.lpsi[nxt][2]};
        const int ist[3] = {1, 1, 1};
        spec_rows_fwd(a, ins, ist, 3, buf, tw);
      }
      if (!grid_sync(a.bar, epoch)) return;
    }
    // mean mode: ez0n = ez0h - dxi <J_z>, E_z0 = (ez0h + ez0n)/2, psi0' = psi0 + dxi ez0n
    if (threadIdx.x == 0) s_lez0 = 0.0;
    {
      const double lez0 = sum_parts(a, 0, red);
      if (threadIdx.x == 0) {
        s_lez0 = lez0;
        s_lez0n = lez0hn + dxi * lpsi0n + 0.5 * lez0;
        s_ljz = -dxi * s_lez0n;
      }
    }
    __syncthreads();
    if (j + 1 < nk) {
      spec_cols(a, OP_PSI, 3, 1, 0.0, buf, tw);
      if (!grid_sync(a.bar, epoch)) return;
      double* lsrc_next = a.lsrc + (size_t)(j + 1) * g * 4;
      spec_rows_inv(a, 1, buf, tw, [&](size_t c, int, double v) {
        a.lS[c] = v;
        lsrc_next[c * 4 + 0] += v;  // S = plasma deposit + S_b of node j + 1
      });
      if (!grid_sync(a.bar, epoch)) return;
    }
    // ---- P4: the commit (j + 1 < nk) and the per-particle accumulators of slice j
    {
      const double* tB = tfg0 + (size_t)n_pc * g * kFG;  // final fields of slice j
      double* lsrc_j = a.lsrc + (size_t)j * g * 4;
      if (j + 1 < nk) {
        // J_perp^{j+1/2} = deposit + (src_j + src_{j+1})/2 and its carried adjoint
        double* lsrc_n = a.lsrc + (size_t)(j + 1) * g * 4;
        for (size_t c = t0; c < g; c += st) {
          const double hx = 0.5 * a.ljp[nxt][0][c], hy = 0.5 * a.ljp[nxt][1][c];
          lsrc_j[c * 4 + 2] += hx;
          lsrc_j[c * 4 + 3] += hy;
          lsrc_n[c * 4 + 2] += hx;
          lsrc_n[c * 4 + 3] += hy;
        }
      }
      for (size_t i = t0; i < np; i += st) {
        const double x = tpart[i], y = tpart[np + i], ux = tpart[2 * np + i],
                     uy = tpart[3 * np + i], pprev = tpart[4 * np + i];
        const CicG c = cic_g(x, y, a.idx, a.idy, nx, ny);
        double lx = 0.0, ly = 0.0, lux = 0.0, luy = 0.0, lopp = 0.0, loph = 0.0, lgx = 0.0,
               lgy = 0.0;
        if (j + 1 < nk) {
          double d0, d1;
          const double psi_p = psi0 + gat(tfg0 + FG_PSI, c, nx, kFG, a.idx, a.idy, d0, d1);
          const double opp = 1.0 + psi_p, oph = 1.0 + 0.5 * (3.0 * psi_p - pprev);
          PushT P;
          P.ux = ux; P.uy = uy; P.opp = opp;
          P.gx = gat0(tfg0 + FG_GX, c, nx, kFG);
          P.gy = gat0(tfg0 + FG_GY, c, nx, kFG);
          P.bx = gat0(tB + FG_BX, c, nx, kFG);
          P.by = gat0(tB + FG_BY, c, nx, kFG);
          P.bz = gat0(tB + FG_BZ, c, nx, kFG);
          push_fwd(P, dxi);
          const double iop = 1.0 / oph;
          // carried adjoints of x^{j+1}, u^{j+1/2}
          double lxn = a.lx[i], lyn = a.ly[i];
          double luxh = a.lux[i], luyh = a.luy[i];
          // S at x^{j+1}: charge -w
          const double xn = x + dxi * P.ox * iop, yn = y + dxi * P.oy * iop;
          const CicG cn = cic_g(xn, yn, a.idx, a.idy, nx, ny);
          gat(a.lS, cn, nx, 1, a.idx, a.idy, d0, d1);
          lxn += -w * dv * d0;
          lyn += -w * dv * d1;
          // J_perp^{j+1/2} at x^{j+1/2}: value -w u/oph
          const double xh = x + 0.5 * dxi * P.ox * iop, yh = y + 0.5 * dxi * P.oy * iop;
          const CicG ch = cic_g(xh, yh, a.idx, a.idy, nx, ny);
          double ex0, ex1, ey0, ey1;
          const double gjx = gat(a.ljp[nxt][0], ch, nx, 1, a.idx, a.idy, ex0, ex1);
          const double gjy = gat(a.ljp[nxt][1], ch, nx, 1, a.idx, a.idy, ey0, ey1);
          const double vhx = -w * P.ox * iop, vhy = -w * P.oy * iop;
          double lxh = dv * (vhx * ex0 + vhy * ey0), lyh = dv * (vhx * ex1 + vhy * ey1);
          luxh += -w * iop * dv * gjx;
          luyh += -w * iop * dv * gjy;
          loph += w * iop * iop * dv * (P.ox * gjx + P.oy * gjy);
          // x^{j+1} = x + dxi u/oph, x^{j+1/2} = x + dxi u/(2 oph)
          lx += lxn + lxh;
          ly += lyn + lyh;
          luxh += dxi * iop * (lxn + 0.5 * lxh);
          luyh += dxi * iop * (lyn + 0.5 * lyh);
          loph -= dxi * iop * iop * (P.ox * (lxn + 0.5 * lxh) + P.oy * (lyn + 0.5 * lyh));
          double l8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
          push_adj(P, luxh, luyh, l8);
          lux += l8[0];
          luy += l8[1];
          lopp += l8[2];
          lgx += l8[3];
          lgy += l8[4];
          // gather of the final B at x^j
          double bx0, bx1;
          gat(tB + FG_BX, c, nx, kFG, a.idx, a.idy, bx0, bx1);
          lx += l8[5] * bx0;
          ly += l8[5] * bx1;
          gat(tB + FG_BY, c, nx, kFG, a.idx, a.idy, bx0, bx1);
          lx += l8[6] * bx0;
          ly += l8[6] * bx1;
          gat(tB + FG_BZ, c, nx, kFG, a.idx, a.idy, bx0, bx1);
          lx += l8[7] * bx0;
          ly += l8[7] * bx1;
          scat(a.lB[0][0], c, nx, l8[5]);
          scat(a.lB[0][1], c, nx, l8[6]);
          scat(a.lB[0][2], c, nx, l8[7]);
        }
        a.lx[i] = lx;
        a.ly[i] = ly;
        a.lux[i] = lux;
        a.luy[i] = luy;
        a.lopp[i] = lopp;
        a.loph[i] = loph;
        a.lgx[i] = lgx;
        a.lgy[i] = lgy;
      }
      if (threadIdx.x == 0) {
        a.part[(size_t)blockIdx.x * 4 + 1] = 0.0;  // kappa^2 adjoint partials
        a.part[(size_t)blockIdx.x * 4 + 2] = 0.0;  // psi0 adjoint partials
      }
      if (!grid_sync(a.bar, epoch)) return;
    }
    // ---- the n_pc field solves, last first; lB[bi]: adjoint of the solve's output B
    double kap_part = 0.0;
    int bi = 0;
    for (int it = n_pc - 1; it >= 0; --it) {
      const bool last = (it == n_pc - 1);
      const double* tBo = tfg0 + (size_t)it * g * kFG;        // B guess of this solve
      const double* tBn = tfg0 + (size_t)(it + 1) * g * kFG;  // its output
      {
        // E_z^j of the last solve enters the slab: its adjoint is the slab's E_z adjoint
        const double* ins[4] = {a.lB[bi][0], a.lB[bi][1], a.lB[bi][2], last ? slab + 2 : nullptr};
        const int ist[4] = {1, 1, 1, 8};
        spec_rows_fwd(a, ins, ist, 4, buf, tw);
        if (!grid_sync(a.bar, epoch)) return;
      }
      spec_cols(a, OP_SOLVE, 4, 5, kap, buf, tw);
      if (!grid_sync(a.bar, epoch)) return;
      {
        double* lsrc_j = a.lsrc + (size_t)j * g * 4;
        double* lsrc_n = (j + 1 < nk) ? a.lsrc + (size_t)(j + 1) * g * 4 : nullptr;
        const int bo = bi ^ 1;
        const double ljz = last ? s_ljz / (double)g : 0.0;
        const double rdxi = 1.0 / dxi;
        // outputs of one cell come from different units (possibly different blocks): the
        // source adjoints they share are added atomically
        spec_rows_inv(a, 5, buf, tw, [&](size_t c, int o, double v) {
          if (o == 0) {
            a.lJ[0][c] = v;
            atomicAdd(lsrc_j + c * 4 + 2, v);
          } else if (o == 1) {
            a.lJ[1][c] = v;
            atomicAdd(lsrc_j + c * 4 + 3, v);
          } else if (o == 2) {
            const double vz = v + ljz;  // <J_z> of the last solve feeds the k = 0 mode
            a.lJ[2][c] = vz;
            lsrc_j[c * 4 + 1] += vz;
          } else if (o == 3) {  // D_x = (J_x^{j+1/2} - J_x^{j-1/2})/dxi
            const double lh = v * rdxi;
            a.lJ[3][c] = lh;
            a.ljp[cur][0][c] -= lh;
            atomicAdd(lsrc_j + c * 4 + 2, 0.5 * lh);
            if (lsrc_n) lsrc_n[c * 4 + 2] += 0.5 * lh;
            a.lB[bo][1][c] = -kap * v;  // kap B_y_old enters B_y: adjoint kap L_By = -kap L_Dx
            kap_part -= v * (tBo[c * kFG + FG_BY] - tBn[c * kFG + FG_BY]);
          } else {
            const double lh = v * rdxi;
            a.lJ[4][c] = lh;
            a.ljp[cur][1][c] -= lh;
            atomicAdd(lsrc_j + c * 4 + 3, 0.5 * lh);
            if (lsrc_n) lsrc_n[c * 4 + 3] += 0.5 * lh;
            a.lB[bo][0][c] = kap * v;  // kap B_x_old enters B_x: adjoint kap L_Bx = kap L_Dy
            a.lB[bo][2][c] = 0.0;
            kap_part += v * (tBo[c * kFG + FG_BX] - tBn[c * kFG + FG_BX]);
          }
        });
        if (!grid_sync(a.bar, epoch)) return;
        // ---- the particles of this solve
        for (size_t i = t0; i < np; i += st) {
          const double x = tpart[i], y = tpart[np + i], ux = tpart[2 * np + i],
                       uy = tpart[3 * np + i], pprev = tpart[4 * np + i];
          const CicG c = cic_g(x, y, a.idx, a.idy, nx, ny);
          const double psi_p = psi0 + gat0(tfg0 + FG_PSI, c, nx, kFG);
          const double opp = 1.0 + psi_p, oph = 1.0 + 0.5 * (3.0 * psi_p - pprev);
          const double iopp = 1.0 / opp, ioph = 1.0 / oph;
          PushT P;
          P.ux = ux; P.uy = uy; P.opp = opp;
          P.gx = gat0(tfg0 + FG_GX, c, nx, kFG);
          P.gy = gat0(tfg0 + FG_GY, c, nx, kFG);
          P.bx = gat0(tBo + FG_BX, c, nx, kFG);
          P.by = gat0(tBo + FG_BY, c, nx, kFG);
          P.bz = gat0(tBo + FG_BZ, c, nx, kFG);
          push_fwd(P, dxi);
          const double uxj = 0.5 * (ux + P.ox), uyj = 0.5 * (uy + P.oy);
          const double u2 = uxj * uxj + uyj * uyj;
          const double uzj = (1.0 + u2 - opp * opp) / (2.0 * opp);
          // J^j at x^j: values -w (u_x, u_y, u_z)/opp
          double d0, d1, e0, e1, f0, f1;
          const double gJx = gat(a.lJ[0], c, nx, 1, a.idx, a.idy, d0, d1);
          const double gJy = gat(a.lJ[1], c, nx, 1, a.idx, a.idy, e0, e1);
          const double gJz = gat(a.lJ[2], c, nx, 1, a.idx, a.idy, f0, f1);
          const double vx = -w * uxj * iopp, vy = -w * uyj * iopp, vz = -w * uzj * iopp;
          double lx = dv * (vx * d0 + vy * e0 + vz * f0), ly = dv * (vx * d1 + vy * e1 + vz * f1);
          double luxj = -w * iopp * dv * gJx, luyj = -w * iopp * dv * gJy;
          const double luzj = -w * iopp * dv * gJz;
          double lopp = w * iopp * iopp * dv * (uxj * gJx + uyj * gJy + uzj * gJz);
          // u_z = (1 + u^2 - opp^2)/(2 opp)
          luxj += luzj * uxj * iopp;
          luyj += luzj * uyj * iopp;
          lopp += luzj * (-(1.0 + u2) * 0.5 * iopp * iopp - 0.5);
          // J_perp^{j+1/2} at x^{j+1/2}: values -w u^{j+1/2}/oph
          const double xh = x + 0.5 * dxi * P.ox * ioph, yh = y + 0.5 * dxi * P.oy * ioph;
          const CicG ch = cic_g(xh, yh, a.idx, a.idy, nx, ny);
          const double gHx = gat(a.lJ[3], ch, nx, 1, a.idx, a.idy, d0, d1);
          const double gHy = gat(a.lJ[4], ch, nx, 1, a.idx, a.idy, e0, e1);
          const double vhx = -w * P.ox * ioph, vhy = -w * P.oy * ioph;
          const double lxh = dv * (vhx * d0 + vhy * e0), lyh = dv * (vhx * d1 + vhy * e1);
          double luxh = -w * ioph * dv * gHx + 0.5 * luxj, luyh = -w * ioph * dv * gHy + 0.5 * luyj;
          double loph = w * ioph * ioph * dv * (P.ox * gHx + P.oy * gHy);
          lx += lxh;
          ly += lyh;
          luxh += 0.5 * dxi * ioph * lxh;
          luyh += 0.5 * dxi * ioph * lyh;
          loph -= 0.5 * dxi * ioph * ioph * (P.ox * lxh + P.oy * lyh);
          double l8[8] = {0.5 * luxj, 0.5 * luyj, lopp, 0, 0, 0, 0, 0};
          push_adj(P, luxh, luyh, l8);
          double b0, b1;
          gat(tBo + FG_BX, c, nx, kFG, a.idx, a.idy, b0, b1);
          lx += l8[5] * b0;
          ly += l8[5] * b1;
          gat(tBo + FG_BY, c, nx, kFG, a.idx, a.idy, b0, b1);
          lx += l8[6] * b0;
          ly += l8[6] * b1;
          gat(tBo + FG_BZ, c, nx, kFG, a.idx, a.idy, b0, b1);
          lx += l8[7] * b0;
          ly += l8[7] * b1;
          scat(a.lB[bo][0], c, nx, l8[5]);
          scat(a.lB[bo][1], c, nx, l8[6]);
          scat(a.lB[bo][2], c, nx, l8[7]);
          a.lx[i] += lx;
          a.ly[i] += ly;
          a.lux[i] += l8[0];
          a.luy[i] += l8[1];
          a.lopp[i] += l8[2];
          a.loph[i] += loph;
          a.lgx[i] += l8[3];
          a.lgy[i] += l8[4];
        }
        bi = bo;
      }
      if (it == 0) {
        const double s = block_sum_lo(kap_part, red);
        if (threadIdx.x == 0) a.part[(size_t)blockIdx.x * 4 + 1] = s;
      }
      // every block's deposits into lB[bi] are complete before the next solve reads it
      if (!grid_sync(a.bar, epoch)) return;
    }
    // ---- P9: psi_p, opp, oph, grad psi at x^j, and kappa^2
    {
      const double lk = sum_parts(a, 1, red);
      if (threadIdx.x == 0) s_lkap = lk;
      __syncthreads();
      const double lkap = s_lkap;
      double lps = 0.0;
      for (size_t i = t0; i < np; i += st) {
        const double x = tpart[i], y = tpart[np + i];
        const CicG c = cic_g(x, y, a.idx, a.idy, nx, ny);
        double p0, p1, g0x, g0y, g1x, g1y;
        const double psi_p = psi0 + gat(tfg0 + FG_PSI, c, nx, kFG, a.idx, a.idy, p0, p1);
        gat(tfg0 + FG_GX, c, nx, kFG, a.idx, a.idy, g0x, g0y);
        gat(tfg0 + FG_GY, c, nx, kFG, a.idx, a.idy, g1x, g1y);
        const double opp = 1.0 + psi_p;
        const double lopp = a.lopp[i] - w * a.inv_LxLy / (opp * opp) * lkap;
        const double loph = a.loph[i];
        const double lpsip = lopp + 1.5 * loph + a.lpp[i];
        a.lpp[i] = -0.5 * loph;  // adjoint of psi_prev: the previous slice's psi_p
        lps += lpsip;
        const double lgx = a.lgx[i], lgy = a.lgy[i];
        a.lx[i] += lpsip * p0 + lgx * g0x + lgy * g1x;
        a.ly[i] += lpsip * p1 + lgx * g0y + lgy * g1y;
        scat(a.lpsi[cur][0], c, nx, lpsip);
        scat(a.lpsi[cur][1], c, nx, lgx);
        scat(a.lpsi[cur][2], c, nx, lgy);
      }
      const double s = block_sum_lo(lps, red);
      if (threadIdx.x == 0) a.part[(size_t)blockIdx.x * 4 + 2] = s;
      // the B guess of slice j (the final B of slice j - 1) has its adjoint in lB[bi]: move it
      // to lB[0] for the next slice
      if (bi != 0)
        for (size_t c = t0; c < g; c += st) {
          a.lB[0][0][c] = a.lB[1][0][c];
          a.lB[0][1][c] = a.lB[1][1][c];
          a.lB[0][2][c] = a.lB[1][2][c];
        }
      if (!grid_sync(a.bar, epoch)) return;
      const double lp = sum_parts(a, 2, red);
      if (threadIdx.x == 0) s_lkap = lp;
      __syncthreads();
      lpsi0n = lpsi0n + s_lkap;        // adjoint of psi0 of slice j
      lez0hn = s_lez0n + 0.5 * s_lez0;  // adjoint of ez0h of slice j
    }
  }
  // ---- prologue: slice 0's psi solve (charge of the plasma at rest + S_b of node 0) and
  // J_perp^{-1/2} = (beam node 0)/2
  {
    const double* ins[3] = {a.lpsi[0][0], a.lpsi[0][1], a.lpsi[0][2]};
    const int ist[3] = {1, 1, 1};
    for (size_t c = t0; c < g; c += st) {
      a.lsrc[c * 4 + 2] += 0.5 * a.ljp[0][0][c];
      a.lsrc[c * 4 + 3] += 0.5 * a.ljp[0][1][c];
    }
    spec_rows_fwd(a, ins, ist, 3, buf, tw);
    if (!grid_sync(a.bar, epoch)) return;
    spec_cols(a, OP_PSI, 3, 1, 0.0, buf, tw);
    if (!grid_sync(a.bar, epoch)) return;
    spec_rows_inv(a, 1, buf, tw, [&](size_t c, int, double v) { a.lsrc[c * 4 + 0] += v; });
  }
}

// ------------------------------------------------------------------ beam adjoints
// Trilinear weights (CIC in x, y; linear in xi) of a beam particle at absolute (x, y, xi),
// with the gradient of the weights.
struct Tri {
  int k0, y0, y1, x0, x1;
  double fk, fy, fx;
};
__device__ __forceinline__ Tri tri(const DevParams& p, double x, double y, double xi) {
  Tri t;
  const double gx = x / p.dx, gy = y / p.dy, gk = xi / p.dxi;
  const double ix = floor(gx), iy = floor(gy), k = floor(gk);
  t.fx = gx - ix;
  t.fy = gy - iy;
  t.fk = gk - k;
  t.x0 = wrap((int)ix, p.nx);
  t.x1 = wrap((int)ix + 1, p.nx);
  t.y0 = wrap((int)iy, p.ny);
  t.y1 = wrap((int)iy + 1, p.ny);
  t.k0 = (int)k;
  return t;
}
// Value and (x, y, xi) gradient of component comp of a [nk][ny][nx][stride] slab at t.
__device__ __forceinline__ double tri_gat(const double* S, const DevParams& p, const Tri& t,
                                          int stride, int comp, double d[3]) {
  double v = 0.0;
  d[0] = d[1] = d[2] = 0.0;
  for (int ck = 0; ck < 2; ++ck) {
    const int k = t.k0 + ck;
    if (k < 0 || k >= p.nk) continue;
    const double wk = ck ? t.fk : 1.0 - t.fk, dk = ck ? 1.0 : -1.0;
    for (int cy = 0; cy < 2; ++cy) {
      const double wy = cy ? t.fy : 1.0 - t.fy, dy = cy ? 1.0 : -1.0;
      for (int cx = 0; cx < 2; ++cx) {
        const double wx = cx ? t.fx : 1.0 - t.fx, dx = cx ? 1.0 : -1.0;
        const double f = S[(((size_t)k * p.ny + (cy ? t.y1 : t.y0)) * p.nx + (cx ? t.x1 : t.x0)) *
                               stride + comp];
        v += wk * wy * wx * f;
        d[0] += wk * wy * dx * f;
        d[1] += wk * dy * wx * f;
        d[2] += dk * wy * wx * f;
      }
    }
  }
  d[0] /= p.dx;
  d[1] /= p.dy;
  d[2] /= p.dxi;
  return v;
}
__device__ __forceinline__ void tri_scat(double* S, const DevParams& p, const Tri& t, int stride,
                                         int comp, double v) {
  if (v == 0.0) return;
  for (int ck = 0; ck < 2; ++ck) {
    const int k = t.k0 + ck;
    if (k < 0 || k >= p.nk) continue;
    const double wk = ck ? t.fk : 1.0 - t.fk;
    for (int cy = 0; cy < 2; ++cy) {
      const double wy = cy ? t.fy : 1.0 - t.fy;
      for (int cx = 0; cx < 2; ++cx) {
        const double wx = cx ? t.fx : 1.0 - t.fx;
        atomicAdd(S + (((size_t)k * p.ny + (cy ? t.y1 : t.y0)) * p.nx + (cx ? t.x1 : t.x0)) *
                          stride + comp,
                  wk * wy * wx * v);
      }
    }
  }
}

// Per-particle beam adjoints: positions (absolute units), momenta and weight.
struct BeamAdj {
  double *lx, *ly, *lxi, *lux, *luy, *luz, *lw;
};

__device__ __forceinline__ void beam_abs(const BeamArrays<double>& b, const DevParams& p,
                                         const SpeciesDev& sp, long long s, double& x, double& y,
                                         double& xi) {
  const Home h = home_of(s, p.nx, p.ny, sp);
  x = (h.ix + (h.sx + 0.5) / sp.ppx + b.ox[s]) * p.dx;
  y = (h.iy + (h.sy + 0.5) / sp.ppy + b.oy[s]) * p.dy;
  xi = (sp.k0 + h.kxi + (h.sxi + 0.5) / sp.ppxi + b.oxi[s]) * p.dxi;
}

// Adjoint of the beam-source deposit of the beam state b: sources S_b = q (1 - v_z),
// J_z = q v_z, J_x = q v_x, J_y = q v_y with q = Z w/(dx dy dxi), trilinear.  Adds to L.
__global__ void beam_src_adj_kernel(BeamArrays<double> b, DevParams p, SpeciesDev sp,
                                    const double* __restrict__ lsrc, BeamAdj L) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= b.n || b.dw[s] == -1.0) return;
  double x, y, xi;
  beam_abs(b, p, sp, s, x, y, xi);
  const double ux = b.ux[s], uy = b.uy[s], uz = b.uz[s];
  const double wgt = sp.wbar * (1.0 + b.dw[s]);
  const double up2 = ux * ux + uy * uy, gm = sqrt(1.0 + up2 + uz * uz), ig = 1.0 / gm;
  const double omv = (1.0 + up2) / (gm * (gm + uz));
  const double qn = sp.Z / (p.dx * p.dy * p.dxi);  // q / w
  const Tri t = tri(p, x, y, xi);
  double d[4][3], lv[4];
  for (int k = 0; k < 4; ++k) lv[k] = tri_gat(lsrc, p, t, 4, k, d[k]);
  const double f[4] = {omv, uz * ig, ux * ig, uy * ig};
  double lwq = 0.0, lp[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k) {
    lwq += lv[k] * f[k];
    for (int a = 0; a < 3; ++a) lp[a] += qn * wgt * f[k] * d[k][a];
  }
  // derivatives of u_a/gamma and of 1 - v_z = 1 - u_z/gamma (written without cancellation)
  const double ig3 = ig * ig * ig;
  const double lvx = qn * wgt * lv[2], lvy = qn * wgt * lv[3], lvz = qn * wgt * (lv[1] - lv[0]);
  // d(u_a/g)/du_b = delta_ab/g - u_a u_b/g^3
  const double lux = lvx * (ig - ux * ux * ig3) - lvy * ux * uy * ig3 - lvz * uz * ux * ig3;
  const double luy = -lvx * ux * uy * ig3 + lvy * (ig - uy * uy * ig3) - lvz * uz * uy * ig3;
  const double luz = -lvx * ux * uz * ig3 - lvy * uy * uz * ig3 + lvz * (1.0 + up2) * ig3;
  L.lx[s] += lp[0];
  L.ly[s] += lp[1];
  L.lxi[s] += lp[2];
  L.lux[s] += lux;
  L.luy[s] += luy;
  L.luz[s] += luz;
  L.lw[s] += qn * lwq;
}

// Adjoint of the beam push of state b through slab (both before the push): L holds the
// adjoints of the pushed state and is overwritten by those of the state before the push;
// the slab's adjoint is added to lslab [nk][ny][nx][8].  Particles lost in this push (xi
// reaches Lxi) or before it carry no adjoint.
__global__ void beam_push_adj_kernel(BeamArrays<double> b, DevParams p, SpeciesDev sp,
                                     const double* __restrict__ slab, double* lslab, BeamAdj L) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= b.n) return;
  if (b.dw[s] == -1.0) {
    L.lx[s] = L.ly[s] = L.lxi[s] = L.lux[s] = L.luy[s] = L.luz[s] = 0.0;
    return;
  }
  double x, y, xi;
  beam_abs(b, p, sp, s, x, y, xi);
  const Tri t = tri(p, x, y, xi);
  double F[6], dF[6][3];
  for (int k = 0; k < 6; ++k) F[k] = tri_gat(slab, p, t, 8, k, dF[k]);
  const double h = 0.5 * sp.Z * p.dt / sp.M, dt = p.dt;
  // forward Boris (the FP64 beam push)
  const double Ex = F[0] + F[4], Ey = F[1] - F[3], Ez = F[2];
  const double Bv[3] = {F[3], F[4], F[5]};
  const double m[3] = {b.ux[s] + h * Ex, b.uy[s] + h * Ey, b.uz[s] + h * Ez};
  const double gm = sqrt(1.0 + m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  const double tv[3] = {h * Bv[0] / gm, h * Bv[1] / gm, h * Bv[2] / gm};
  const double pv[3] = {m[0] + (m[1] * tv[2] - m[2] * tv[1]), m[1] + (m[2] * tv[0] - m[0] * tv[2]),
                        m[2] + (m[0] * tv[1] - m[1] * tv[0])};
  const double t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
  const double sf = 2.0 / (1.0 + t2);
  const double r[3] = {sf * tv[0], sf * tv[1], sf * tv[2]};
  const double un[3] = {m[0] + (pv[1] * r[2] - pv[2] * r[1]) + h * Ex,
                        m[1] + (pv[2] * r[0] - pv[0] * r[2]) + h * Ey,
                        m[2] + (pv[0] * r[1] - pv[1] * r[0]) + h * Ez};
  const double up2 = un[0] * un[0] + un[1] * un[1];
  const double gn = sqrt(1.0 + up2 + un[2] * un[2]), ign = 1.0 / gn;
  const double omv = (1.0 + up2) / (gn * (gn + un[2]));
  if (xi + dt * omv >= p.Lxi) {  // lost in this push
    L.lx[s] = L.ly[s] = L.lxi[s] = L.lux[s] = L.luy[s] = L.luz[s] = 0.0;
    return;
  }
  // adjoints of the pushed state
  const double lxn = L.lx[s], lyn = L.ly[s], lxin = L.lxi[s];
  double lu[3] = {L.lux[s], L.luy[s], L.luz[s]};
  // x' = x + dt u_x/g, y' = y + dt u_y/g, xi' = xi + dt (1 - u_z/g)
  const double ig3 = ign * ign * ign;
  {
    const double ax = dt * lxn, ay = dt * lyn, az = -dt * lxin;  // adjoints of v_x, v_y, v_z
    lu[0] += ax * (ign - un[0] * un[0] * ig3) - ay * un[0] * un[1] * ig3 - az * un[2] * un[0] * ig3;
    lu[1] += -ax * un[0] * un[1] * ig3 + ay * (ign - un[1] * un[1] * ig3) - az * un[2] * un[1] * ig3;
    lu[2] += -ax * un[0] * un[2] * ig3 - ay * un[1] * un[2] * ig3 + az * (ign - un[2] * un[2] * ig3);
  }
  // reverse Boris: u' = m + p x r + h E
  double lE[3] = {h * lu[0], h * lu[1], h * lu[2]};
  double lm[3] = {lu[0], lu[1], lu[2]};
  // p x r: lp += r x lu ; lr += lu x p
  double lp[3] = {r[1] * lu[2] - r[2] * lu[1], r[2] * lu[0] - r[0] * lu[2], r[0] * lu[1] - r[1] * lu[0]};
  const double lr[3] = {lu[1] * pv[2] - lu[2] * pv[1], lu[2] * pv[0] - lu[0] * pv[2],
                        lu[0] * pv[1] - lu[1] * pv[0]};
  // r = sf t, sf = 2/(1 + t^2)
  const double lsf = lr[0] * tv[0] + lr[1] * tv[1] + lr[2] * tv[2];
  double lt[3] = {sf * lr[0], sf * lr[1], sf * lr[2]};
  const double dsf = -4.0 / ((1.0 + t2) * (1.0 + t2));
  for (int a = 0; a < 3; ++a) lt[a] += lsf * dsf * tv[a];
  // p = m + m x t: lm += lp + t x lp ; lt += lp x m
  lm[0] += lp[0] + (tv[1] * lp[2] - tv[2] * lp[1]);
  lm[1] += lp[1] + (tv[2] * lp[0] - tv[0] * lp[2]);
  lm[2] += lp[2] + (tv[0] * lp[1] - tv[1] * lp[0]);
  lt[0] += lp[1] * m[2] - lp[2] * m[1];
  lt[1] += lp[2] * m[0] - lp[0] * m[2];
  lt[2] += lp[0] * m[1] - lp[1] * m[0];
  // t = h B/gm
  double lB[3] = {h / gm * lt[0], h / gm * lt[1], h / gm * lt[2]};
  const double lgm = -(tv[0] * lt[0] + tv[1] * lt[1] + tv[2] * lt[2]) / gm;
  for (int a = 0; a < 3; ++a) lm[a] += lgm * m[a] / gm;
  // m = u + h E
  for (int a = 0; a < 3; ++a) lE[a] += h * lm[a];
  // E = (W_x + B_y, W_y - B_x, E_z), B = (B_x, B_y, B_z)
  const double lF[6] = {lE[0], lE[1], lE[2], lB[0] - lE[1], lB[1] + lE[0], lB[2]};
  double lpos[3] = {lxn, lyn, lxin};
  for (int k = 0; k < 6; ++k) {
    tri_scat(lslab, p, t, 8, k, lF[k]);
    for (int a = 0; a < 3; ++a) lpos[a] += lF[k] * dF[k][a];
  }
  L.lx[s] = lpos[0];
  L.ly[s] = lpos[1];
  L.lxi[s] = lpos[2];
  L.lux[s] = lm[0];
  L.luy[s] = lm[1];
  L.luz[s] = lm[2];
}

// dL/d(mode amplitude m) and dL/d(alpha) from the weight adjoints: the initial weight of a
// seeded species is wbar (1 + noise n) (1 + sum_m a_m cos(k_m . x0 + phi_m)) with x0 the
// particle's lattice home, and wbar is proportional to alpha.  out[0..nm-1] += dL/da_m,
// out[nm] += dL/dalpha.  w0 holds the initial weights (the dw of the first beam state).
__global__ void weight_grad_kernel(const double* __restrict__ dw0, long long n, DevParams p,
                                   SpeciesDev sp, ModesDev md, const double* __restrict__ lw,
                                   double* out) {
  __shared__ double red[32];
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double acc[17];
  for (int k = 0; k < 17; ++k) acc[k] = 0.0;
  if (s < n && dw0[s] != -1.0) {
    const double w0 = sp.wbar * (1.0 + dw0[s]);
    const double lwv = lw[s];
    acc[md.n] = lwv * w0 / sp.alpha;
    if (sp.seeded && md.n > 0) {
      const Home hm = home_of(s, p.nx, p.ny, sp);
      const double x = (hm.ix + (hm.sx + 0.5) / sp.ppx) * p.dx;
      const double y = (hm.iy + (hm.sy + 0.5) / sp.ppy) * p.dy;
      double c[16], mm = 0.0;
      for (int k = 0; k < md.n; ++k) {
        const double kx = 6.283185307179586476925 * md.mx[k] / p.Lx;
        const double ky = 6.283185307179586476925 * md.my[k] / p.Ly;
        c[k] = cos(kx * x + ky * y + md.phase[k]);
        mm += md.amp[k] * c[k];
      }
      for (int k = 0; k < md.n; ++k) acc[k] = lwv * w0 * c[k] / (1.0 + mm);
    }
  }
  for (int k = 0; k <= md.n; ++k) {
    const double v = block_sum(acc[k], red);
    if (threadIdx.x == 0 && v != 0.0) atomicAdd(out + k, v);
    __syncthreads();
  }
}

// Loss of the final sweep: 1/2 sum over slices and cells of (B_x^2 + B_y^2) dx dy dxi, and
// its adjoint slab (B_x, B_y) dx dy dxi times `scale`.
__global__ void bperp_loss_kernel(const double* __restrict__ slab, size_t ncell, double vol,
                                  double scale, double* lslab, double* loss) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < ncell;
       c += (size_t)gridDim.x * blockDim.x) {
    const double bx = slab[c * 8 + 3], by = slab[c * 8 + 4];
    acc += 0.5 * (bx * bx + by * by) * vol;
    if (lslab) {
      for (int k = 0; k < 8; ++k) lslab[c * 8 + k] = 0.0;
      lslab[c * 8 + 3] = scale * bx * vol;
      lslab[c * 8 + 4] = scale * by * vol;
    }
  }
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, v);
}

}  // namespace qsa
