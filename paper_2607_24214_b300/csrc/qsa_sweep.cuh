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
// Layouts: plasma particles [home row iy][sub-lattice index][ix] (a warp holds 32 neighbouring
// cells); real-space fields interleaved per node, fg[iy][ix][8] = (psi, d_x psi, d_y psi, B_x,
// B_y, B_z, E_z, -) so that a CIC gather is two 16-byte loads per corner; deposit tiles,
// per-chunk partials and the overflow grid field-major; spectra [field][kx][ky] after the row
// phase and [field][ky][kx] after the column phase, so that every transpose is a strided
// write followed by contiguous reads.  A block owns one home row (a chunk) of particles whose
// deposits land in a four-row shared-memory tile [iy-1, iy+2]; the tile goes to a per-chunk
// partial buffer that the row phase sums without atomics; particles that left their tile
// deposit with global atomics into the overflow grid.
#pragma once
#include "qsa_common.cuh"
#include "qsa_fft.cuh"

namespace qsa {

constexpr int kNF = 5;  // deposit fields of a trial phase
constexpr int kTileRows = 4;
constexpr int kFG = 8;  // components of the interleaved field grid
enum FgComp : int { FG_PSI = 0, FG_GX, FG_GY, FG_BX, FG_BY, FG_BZ, FG_EZ };
// Phase timing of the first slices: for slice j < kTimedSlices and phase ph < kTimedPhases
// (trial iteration it, step k: ph = 4 it + k; commit: ph = 4 n_pc + k), the globaltimer of
// the last block's arrival at the barrier and of block 0's exit from it.
constexpr int kTimedSlices = 8;
constexpr int kTimedPhases = 32;

enum Diag : int {
  D_KAPPA = 0,  // sum 1/(1+psi) over particles -> kappa^2 after scaling
  D_JZ,         // <J_z> total
  D_PSI0,
  D_EZ0,
  D_CHARGE,     // sum over cells of the plasma (rho - J_z) deviation, times dx dy
  D_PCNUM,
  D_PCDEN,
  D_OPPMIN,     // ordered-key minimum of 1 + psi
  D_NFLOOR,
  D_INV,        // max invariant residual (non-negative double bits)
  D_NPC,        // field solves of the predictor-corrector at the slice
  D_E0,         // six energies D_E0..D_E0+5
  D_COUNT = D_E0 + 6
};

// Per-block partial diagnostics, written without atomics by thread 0 of every block into
// dpart[(j * gridDim.x + block) * P_COUNT + field] and reduced after the sweep.
enum Part : int {
  P_OPPMIN = 0,  // min
  P_NFLOOR,      // sum
  P_INV,         // max
  P_CHARGE,      // sum
  P_PCNUM,       // sum
  P_PCDEN,       // sum
  P_E0,          // six sums P_E0..P_E0+5
  P_COUNT = P_E0 + 6
};
__device__ __forceinline__ double* pslot(double* dpart, int j, int field) {
  return dpart + ((size_t)j * gridDim.x + blockIdx.x) * P_COUNT + field;
}

// Order-preserving map of a double to an unsigned key (min over keys = min over values).
__device__ __forceinline__ unsigned long long dkey(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Grid constants in the working precision, formed on the host in FP64 once: device code
// needs no FP64 division per phase (every thread of every block would repeat it, and FP64
// issue is scarce on this part).
template <typename R>
struct SweepConst {
  R dxi, rdxi;     // slice step and its inverse
  R idx, idy;      // inverse cell sizes
  R wn;            // w / (dx dy) of a plasma macroparticle = 1 / ppc
  R floor_;        // psi_floor
  R inv_npc;       // 1 / (ppc nx ny): kappa^2 from the sum of 1/(1+psi)
  R scale;         // 1 / (nx ny): inverse FFT normalisation
  R inv_ppx, inv_ppy;  // 1 / plasma sub-lattice counts
};
template <typename R>
inline SweepConst<R> sweep_consts(const DevParams& p) {
  SweepConst<R> k;
  k.dxi = R(p.dxi);
  k.rdxi = R(1.0 / p.dxi);
  k.idx = R(1.0 / p.dx);
  k.idy = R(1.0 / p.dy);
  k.wn = R(1.0 / p.ppc);
  k.floor_ = R(p.psi_floor);
  k.inv_npc = R(1.0 / ((double)p.ppc * p.nx * p.ny));
  k.scale = R(1.0 / ((double)p.nx * p.ny));
  k.inv_ppx = R(1.0 / p.ppx);
  k.inv_ppy = R(1.0 / p.ppy);
  return k;
}

// Record of one sweep for its adjoint (all pointers null: nothing recorded).  Per slice j:
//   part[j][5][np]: x, y (absolute, in units of length, unwrapped), u_x, u_y (u^{j-1/2}) and
//     the previous slice's psi_p of every plasma particle as the slice starts;
//   fg[j][s][ny][nx][8]: the interleaved field grid as the slice starts (s = 0: psi, grad psi
//     of slice j and the B guess, the previous slice's final fields) and after each of its
//     n_pc field solves (s = 1..n_pc);
//   jprev[j][2][nxh][ny]: the spectra of the total J_perp^{j-1/2}.
template <typename R>
struct Tape {
  R* part;
  R* fg;
  C<R>* jprev;
};

template <typename R>
struct SweepArgs {
  DevParams p;
  SweepConst<R> k;
  R *pox, *poy, *pux, *puy, *ppsi;          // plasma state (offsets in cells)
  R* fg;                                    // [ny][nx][8] real-space fields
  R* part;                                  // [ny chunks][nf][4][nx]
  R* ovf;                                   // [kNF][ny][nx]
  int* cflag;                               // [ny chunks] outer tile rows used (bits 0, 1)
  int* odirty;                              // [ny] overflow row holds deposits
  C<R>* rspec;                              // [kNF][nxh][ny]
  C<R>* cspec;                              // [4][ny][nxh]
  C<R>* jprev;                              // [2][nxh][ny]  J_perp^{j-1/2} spectra
  C<R>* bold;                               // [2][nxh][ny]  B_perp spectra of the last solve
  const C<R>* twx;
  const C<R>* twy;
  const R* src;                             // [nk][ny][nx][4] beam S_b, J_z, J_x, J_y deviations
  R* slab;                                  // [nk][ny][nx][8]
  R* mode_out;                              // [nk][nmodes][5][2] or null (diagnosed modes)
  double* diag;                             // [D_COUNT][nk]
  double* dpart;                            // [nk][gridDim.x][P_COUNT] partials
  const R* ktab;                            // wavenumber table, see kvec
  const double* bref;                       // [nk] beam J_z reference density per node
  unsigned long long* ptimes;               // [kTimedSlices][kTimedPhases][2] or null
  Barrier bar;
  Tape<R> tape;                             // recording for the adjoint, or all null
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

// Store one slab node (six fields and two zero pads) with 16-byte stores.
__device__ __forceinline__ void st8(float* s, float a, float b, float c, float d, float e,
                                    float f) {
  reinterpret_cast<float4*>(s)[0] = make_float4(a, b, c, d);
  reinterpret_cast<float4*>(s)[1] = make_float4(e, f, 0.f, 0.f);
}
__device__ __forceinline__ void st8(double* s, double a, double b, double c, double d, double e,
                                    double f) {
  reinterpret_cast<double2*>(s)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(s)[1] = make_double2(c, d);
  reinterpret_cast<double2*>(s)[2] = make_double2(e, f);
  reinterpret_cast<double2*>(s)[3] = make_double2(0.0, 0.0);
}

// Bilinear gather from the interleaved field grid.  The xi push needs the first kGP
// components of a node (psi, its gradient, B_x, B_y, B_z): one 16-byte and one 8-byte load
// per node (FP32).
constexpr int kGP = 6;
__device__ __forceinline__ void ld6(const float* p, float v[6]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  const float2 r = *reinterpret_cast<const float2*>(p + 4);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w; v[4] = r.x; v[5] = r.y;
}
__device__ __forceinline__ void ld6(const double* p, double v[6]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  const double2 c = *reinterpret_cast<const double2*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

template <typename R>
__device__ __forceinline__ void gather6(const R* __restrict__ fg, const Cic<R>& c, int nx,
                                        R out[kGP]) {
  R a[kGP], b[kGP], d[kGP], e[kGP];
  (void)QSA_IN(c.x0 >= 0 && c.x0 < nx && c.x1 >= 0 && c.x1 < nx && c.y0 >= 0 && c.y1 >= 0);
  ld6(fg + ((size_t)c.y0 * nx + c.x0) * kFG, a);
  ld6(fg + ((size_t)c.y0 * nx + c.x1) * kFG, b);
  ld6(fg + ((size_t)c.y1 * nx + c.x0) * kFG, d);
  ld6(fg + ((size_t)c.y1 * nx + c.x1) * kFG, e);
  const R gx = R(1) - c.fx, gy = R(1) - c.fy;
#pragma unroll
  for (int k = 0; k < kGP; ++k)
    out[k] = gy * (gx * a[k] + c.fx * b[k]) + c.fy * (gx * d[k] + c.fx * e[k]);
}

// The same gather for the two particles of a thread when both sit in their home cell
// (column ix, row iy; x1, y1 the next ones): the four corner nodes are loaded once.
template <typename R>
__device__ __forceinline__ void gather6_pair(const R* __restrict__ fg, int ix, int x1, int iy,
                                             int y1, int nx, const Cic<R> (&c)[2],
                                             R (&out)[2][kGP]) {
  R a[kGP], b[kGP], d[kGP], e[kGP];
  ld6(fg + ((size_t)iy * nx + ix) * kFG, a);
  ld6(fg + ((size_t)iy * nx + x1) * kFG, b);
  ld6(fg + ((size_t)y1 * nx + ix) * kFG, d);
  ld6(fg + ((size_t)y1 * nx + x1) * kFG, e);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const R gx = R(1) - c[u].fx, gy = R(1) - c[u].fy;
#pragma unroll
    for (int k = 0; k < kGP; ++k)
      out[u][k] = gy * (gx * a[k] + c[u].fx * b[k]) + c[u].fy * (gx * d[k] + c[u].fx * e[k]);
  }
}

// Deposit v (already a density) at the four corners into the field-major tile [nf][4][nx],
// or into the overflow grid [kNF][ny][nx] when the rows fall outside the tile.
// Deposits outside the two home rows of the tile are rare (a particle that left its home
// row); they are flagged so that the row phase reads the outer tile rows (cflag bit 0: tile
// row 0, bit 1: tile row 3) and the overflow rows (odirty) only where something landed.
struct DepFlags {
  int* tile;    // shared flag word of the chunk
  int* odirty;  // [ny] overflow rows
};
__device__ __forceinline__ void flag_rows(const DepFlags& fl, int ty) {
  if (ty == 0) atomicOr(fl.tile, 1);
  else if (ty == kTileRows - 2) atomicOr(fl.tile, 2);
}
__device__ __forceinline__ void flag_ovf(const DepFlags& fl, int y0, int y1) {
  atomicOr(fl.odirty + y0, 1);
  atomicOr(fl.odirty + y1, 1);
}

template <typename R>
__device__ __forceinline__ void deposit(R* tile, R* ovf, const DepFlags& fl, const Cic<R>& c,
                                        int f, int nx, int ny, R v) {
  const R gx = R(1) - c.fx, gy = R(1) - c.fy;
  const R w00 = gx * gy * v, w01 = c.fx * gy * v, w10 = gx * c.fy * v, w11 = c.fx * c.fy * v;
  if (!QSA_IN(c.x0 < nx && c.x1 < nx && c.y0 < ny && c.y1 < ny && f < kNF)) return;
  if (c.ty >= 0 && c.ty <= kTileRows - 2) {
    if (c.ty != 1) flag_rows(fl, c.ty);
    R* r0 = tile + ((size_t)f * kTileRows + c.ty) * nx;
    R* r1 = r0 + nx;
    atomicAdd(r0 + c.x0, w00);
    atomicAdd(r0 + c.x1, w01);
    atomicAdd(r1 + c.x0, w10);
    atomicAdd(r1 + c.x1, w11);
  } else {
    flag_ovf(fl, c.y0, c.y1);
    R* o = ovf + (size_t)f * ny * nx;
    atomicAdd(o + (size_t)c.y0 * nx + c.x0, w00);
    atomicAdd(o + (size_t)c.y0 * nx + c.x1, w01);
    atomicAdd(o + (size_t)c.y1 * nx + c.x0, w10);
    atomicAdd(o + (size_t)c.y1 * nx + c.x1, w11);
  }
}

// Deposit v_dev W(x) + v_ref (W(x) - W(home)) for a particle of home cell (ix, crow), home
// sub-cell position (hx, hy) and offset (ox, oy) in cells.  v_ref W(home), summed over the
// quiet lattice, is uniform (k = 0 only) and is carried analytically by the caller; keeping
// it out of the grid sums lets FP32 accumulation resolve the fluctuations.  While the
// particle is in its home cell the weight differences are formed from the offsets without
// cancellation.
template <typename R>
__device__ __forceinline__ void deposit_ref(R* tile, R* ovf, const DepFlags& fl, int ix, int crow,
                                            R hx, R hy, R ox, R oy, int f, int nx, int ny,
                                            R v_dev, R v_ref) {
  const R lx = hx + ox, ly = hy + oy;
  if (lx >= R(0) && lx < R(1) && ly >= R(0) && ly < R(1)) {
    const R ax = R(1) - hx, ay = R(1) - hy;
    const R oxy = ox * oy;
    const R d00 = -ox * ay - oy * ax + oxy, d01 = ox * ay - hx * oy - oxy;
    const R d10 = ax * oy - ox * hy - oxy, d11 = hx * oy + ox * hy + oxy;
    const R w00 = (ax - ox) * (ay - oy), w01 = lx * (ay - oy), w10 = (ax - ox) * ly,
            w11 = lx * ly;
    const int x0 = ix, x1 = (ix + 1 == nx) ? 0 : ix + 1;
    R* r0 = tile + ((size_t)f * kTileRows + 1) * nx;  // home row crow is tile row 1
    R* r1 = r0 + nx;
    atomicAdd(r0 + x0, v_dev * w00 + v_ref * d00);
    atomicAdd(r0 + x1, v_dev * w01 + v_ref * d01);
    atomicAdd(r1 + x0, v_dev * w10 + v_ref * d10);
    atomicAdd(r1 + x1, v_dev * w11 + v_ref * d11);
  } else {
    const Cic<R> c = cic<R>(ix, crow, lx, ly, nx, ny, crow);
    deposit(tile, ovf, fl, c, f, nx, ny, v_dev + v_ref);
    const Cic<R> h = cic<R>(ix, crow, hx, hy, nx, ny, crow);
    deposit(tile, ovf, fl, h, f, nx, ny, -v_ref);
  }
}

// Reciprocal: the FP32 path uses the fast hardware approximation (about 2 ulp), FP64 is exact.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// xi push u^{j-1/2} -> u^{j+1/2}: half kick, counter-clockwise rotation by
// 2 atan(dxi B_z/(2(1+psi))), half kick; gamma/(1+psi) of both kicks taken at the predicted
// pre-rotation momentum (the rotation keeps |u_perp|).  From the quasistatic invariant
// gamma - u_z = 1 + psi: gamma/(1+psi) = (1 + u^2 + (1+psi)^2) / (2 (1+psi)^2).
template <typename R>
__device__ __forceinline__ void push_xi(R& ux, R& uy, R opp, R iopp, R gx, R gy, R bx, R by,
                                        R bz, R dxi) {
  const R h = R(0.5) * dxi;
  const R hi2 = R(0.5) * iopp * iopp;
  const R g0 = (R(1) + ux * ux + uy * uy + opp * opp) * hi2;
  const R px0 = ux + h * (g0 * gx - by), py0 = uy + h * (g0 * gy + bx);
  const R g = (R(1) + px0 * px0 + py0 * py0 + opp * opp) * hi2;
  const R kx = h * (g * gx - by), ky = h * (g * gy + bx);
  const R mx = ux + kx, my = uy + ky;
  const R t = h * bz * iopp;
  const R s = R(2) * t * rcp(R(1) + t * t);
  const R px = mx - t * my, py = my + t * mx;
  const R qx = mx - s * py, qy = my + s * px;
  ux = qx + kx;
  uy = qy + ky;
}

enum DepMode : int { DEP_INIT = 0, DEP_TRIAL = 1, DEP_COMMIT = 2 };



template <typename R>
struct W4 {
  R w00, w01, w10, w11;
};
template <typename R>
__device__ __forceinline__ W4<R> cic_w(const Cic<R>& c) {
  const R gx = R(1) - c.fx, gy = R(1) - c.fy;
  return W4<R>{gx * gy, c.fx * gy, gx * c.fy, c.fx * c.fy};
}

// Deposit N values v[k] into fields f0 + k at the four corners of c (shared weights w), in
// the field-major tile or, outside it, in the overflow grid.
template <typename R, int N>
__device__ __forceinline__ void deposit_n(R* tile, R* ovf, const DepFlags& fl, const Cic<R>& c,
                                          const W4<R>& w, int f0, int nx, int ny,
                                          const R (&v)[N]) {
  if (!QSA_IN(c.x0 < nx && c.x1 < nx && c.y0 < ny && c.y1 < ny && f0 + N <= kNF)) return;
  if (c.ty >= 0 && c.ty <= kTileRows - 2) {
    if (c.ty != 1) flag_rows(fl, c.ty);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      R* r0 = tile + ((size_t)(f0 + k) * kTileRows + c.ty) * nx;
      R* r1 = r0 + nx;
      atomicAdd(r0 + c.x0, w.w00 * v[k]);
      atomicAdd(r0 + c.x1, w.w01 * v[k]);
      atomicAdd(r1 + c.x0, w.w10 * v[k]);
      atomicAdd(r1 + c.x1, w.w11 * v[k]);
    }
  } else {
    flag_ovf(fl, c.y0, c.y1);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      R* o = ovf + (size_t)(f0 + k) * ny * nx;
      atomicAdd(o + (size_t)c.y0 * nx + c.x0, w.w00 * v[k]);
      atomicAdd(o + (size_t)c.y0 * nx + c.x1, w.w01 * v[k]);
      atomicAdd(o + (size_t)c.y1 * nx + c.x0, w.w10 * v[k]);
      atomicAdd(o + (size_t)c.y1 * nx + c.x1, w.w11 * v[k]);
    }
  }
}

// Weight differences W(x) - W(home) at the four corners of the home cell, from the offsets
// (ox, oy) and the home sub-cell position (hx, hy), without cancellation.
template <typename R>
__device__ __forceinline__ W4<R> cic_dw(R hx, R hy, R ox, R oy) {
  const R ax = R(1) - hx, ay = R(1) - hy, oxy = ox * oy;
  return W4<R>{-ox * ay - oy * ax + oxy, ox * ay - hx * oy - oxy, ax * oy - ox * hy - oxy,
                hx * oy + ox * hy + oxy};
}

// Every phase takes its work units (grid rows, or half-spectrum columns) u0, u0 + G, ... so
// that one launch can spread the units of several sweeps over its blocks; a single sweep
// passes (blockIdx.x, gridDim.x).  The per-block diagnostic partials are written by every
// block that calls the phase, with or without units.
template <typename R>
__device__ void dep_phase(const SweepArgs<R>& a, R* tile, int mode, int j, double psi0,
                          bool first, bool last, int u0, int G) {
  // reference state of the deposits: a particle at rest at its lattice home with psi = psi0
  // carries rho - J_z = -w and u_z/(1+psi) = c0 = -psi0 (2 + psi0) / (2 (1+psi0)^2); formed
  // in the working precision (psi0 is O(alpha), no cancellation)
  const DevParams& p = a.p;
  // the fields the particle loop reads, held in registers (a reference into shared or global
  // memory would be re-read after every store the compiler cannot separate from it)
  const int ppc = p.ppc, ppx = p.ppx, np = p.np;
  const R inv_ppx = a.k.inv_ppx, inv_ppy = a.k.inv_ppy;
  const R* __restrict__ fgp = a.fg;
  R* const ovf = a.ovf;
  const R psi0r = R(psi0);
  const R opp0 = R(1) + psi0r;
  const R iopp02 = R(1) / (opp0 * opp0);
  const R c0 = R(-0.5) * psi0r * (R(2) + psi0r) * iopp02;
  const R floor_ = a.k.floor_;
  const R dfloor = floor_ - opp0;  // psi fluctuation of a floored particle
  const int nx = p.nx, ny = p.ny;
  const int nf = (mode == DEP_TRIAL) ? kNF : 3;
  const int per_chunk = ppc * nx;
  const R wn = a.k.wn;
  const R dxi = a.k.dxi;
  const R idx = a.k.idx, idy = a.k.idy;
  const int tile_elems = kTileRows * nx * nf;
  // the aggregated deposit needs whole warps over consecutive columns
  const bool lane_agg = (nx % 32 == 0) && (blockDim.x % 32 == 0);
  // the tile goes out in 16-byte pieces when rows are whole quads (FP32) and the block's
  // threads cover whole rows of quads
  const int nx4 = nx >> 2;
  const bool cp4 = sizeof(R) == 4 && (nx & 3) == 0 && nx4 <= (int)blockDim.x &&
                   blockDim.x % nx4 == 0;
  const int r0_t = cp4 ? (int)threadIdx.x / nx4 : 0, x4_t = cp4 ? (int)threadIdx.x % nx4 : 0;
  const int rstep = cp4 ? (int)blockDim.x / nx4 : 1;
  // per-thread diagnostics accumulate in R; the block reductions below finish in FP64
  R kap = R(0), inv = R(0), omin = R(1e30), nfloor = R(0);
  __shared__ double red[32];
  __shared__ int s_flag;
  if (u0 >= ny) {  // no unit in this block: identity partials, no reductions
    if (threadIdx.x == 0 && mode == DEP_TRIAL) {
      if (first) {
        *pslot(a.dpart, j, P_OPPMIN) = 1e30;
        *pslot(a.dpart, j, P_NFLOOR) = 0.0;
      }
      if (last) *pslot(a.dpart, j, P_INV) = 0.0;
    }
    return;
  }
  const DepFlags fl{&s_flag, a.odirty};
  R* __restrict__ pox = a.pox;
  R* __restrict__ poy = a.poy;
  R* __restrict__ pux = a.pux;
  R* __restrict__ puy = a.puy;
  R* __restrict__ pps = a.ppsi;

  for (int crow = u0; crow < ny; crow += G) {
    // (a bulk prefetch wants 16-byte multiples: chunks of other sizes go without)
    if (threadIdx.x == 0 && mode != DEP_INIT && (per_chunk * sizeof(R)) % 16 == 0) {
      // the plasma state of this chunk (first pass only) and of the block's next chunk into
      // L2: the state was last touched a tick ago and has usually left the cache
      const unsigned nbts = (unsigned)(per_chunk * sizeof(R));
      for (int c2 = (crow == u0 ? crow : crow + G); c2 <= crow + G && c2 < ny; c2 += G) {
        const size_t b2 = (size_t)c2 * per_chunk;
        l2_prefetch(pox + b2, nbts);
        l2_prefetch(poy + b2, nbts);
        l2_prefetch(pux + b2, nbts);
        l2_prefetch(puy + b2, nbts);
        l2_prefetch(pps + b2, nbts);
      }
    }
    zero_block(tile, tile_elems);
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    const int base = crow * per_chunk;  // particle indices fit in int (np < 2^31)
    if (mode == DEP_INIT) {  // at home: rho - J_z equals its reference, nothing to add
      for (int t = threadIdx.x; t < per_chunk; t += blockDim.x) {
        const int i = base + t;
        pox[i] = R(0);
        poy[i] = R(0);
        pux[i] = R(0);
        puy[i] = R(0);
        pps[i] = R(0);
      }
    } else {
      // two sub-lattice positions per thread per pass, (sub0, ix) and (sub0 + 1, ix): the
      // loads and gathers of both are issued before either particle's arithmetic
      for (int sub0 = 0; sub0 < ppc; sub0 += 2) {
        R hx[2], hy[2];
        bool ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          ok[u] = sub0 + u < ppc;
          const int sub = ok[u] ? sub0 + u : sub0;
          // sub = sy ppx + sx, split with an exact float quotient of small integers
          const int sy = (int)((float(sub) + 0.5f) * float(inv_ppx));
          hx[u] = (R(sub - sy * ppx) + R(0.5)) * inv_ppx;
          hy[u] = (R(sy) + R(0.5)) * inv_ppy;
        }
        for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
          int ii[2];
          R ox[2], oy[2], uxs[2], uys[2], pprev[2];
          Cic<R> c[2];
          R F[2][kGP];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            ii[u] = base + (ok[u] ? sub0 + u : sub0) * nx + ix;
            if (!QSA_IN(ii[u] >= 0 && ii[u] < np)) ii[u] = 0;
            ox[u] = pox[ii[u]];
            oy[u] = poy[ii[u]];
            uxs[u] = pux[ii[u]];
            uys[u] = puy[ii[u]];
            pprev[u] = pps[ii[u]];
          }
          bool pair_home = true;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const R lx = hx[u] + ox[u], ly = hy[u] + oy[u];
            if (ok[u]) pair_home = pair_home && lx >= R(0) && lx < R(1) && ly >= R(0) && ly < R(1);
          }
          if (pair_home) {
            // both in the home cell: shared corners (ix, crow) .. (ix + 1, crow + 1)
            const int gx1 = (ix + 1 == nx) ? 0 : ix + 1, gy1 = (crow + 1 == ny) ? 0 : crow + 1;
#pragma unroll
            for (int u = 0; u < 2; ++u)
              c[u] = Cic<R>{ix, gx1, crow, gy1, 1, hx[u] + ox[u], hy[u] + oy[u]};
            gather6_pair(fgp, ix, gx1, crow, gy1, nx, c, F);
          } else {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              c[u] = cic<R>(ix, crow, hx[u] + ox[u], hy[u] + oy[u], nx, ny, crow);
              gather6(fgp, c[u], nx, F[u]);
            }
          }
          // arithmetic of both particles; their deposit values are kept for the deposit step
          bool home[2] = {false, false}, homeh[2] = {false, false};
          R vx[2] = {0, 0}, vy[2] = {0, 0}, vdev[2] = {0, 0};
          R jhx[2] = {0, 0}, jhy[2] = {0, 0}, nox[2] = {0, 0}, noy[2] = {0, 0};
          R lxh[2] = {0, 0}, lyh[2] = {0, 0};  // sub-cell position at x^{j+1/2}
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (!ok[u]) continue;
            const int i = ii[u];
            R ux = uxs[u], uy = uys[u];
            const R psi_fl = F[u][FG_PSI];
            const R psi_p = psi0r + psi_fl;
            const R opp_raw = R(1) + psi_p;
            const R opp = opp_raw < floor_ ? floor_ : opp_raw;
            const R iopp = rcp(opp);
            R oph = R(1) + R(0.5) * (R(3) * psi_p - pprev[u]);
            oph = oph < floor_ ? floor_ : oph;
            const R ioph = rcp(oph);
            const R uxm = ux, uym = uy;
            push_xi(ux, uy, opp, iopp, F[u][FG_GX], F[u][FG_GY], F[u][FG_BX], F[u][FG_BY],
                    F[u][FG_BZ], dxi);
            const R sh = R(0.5) * dxi * ioph;
            lxh[u] = hx[u] + ox[u] + sh * ux * idx;
            lyh[u] = hy[u] + oy[u] + sh * uy * idy;
            homeh[u] = lxh[u] >= R(0) && lxh[u] < R(1) && lyh[u] >= R(0) && lyh[u] < R(1);
            jhx[u] = -wn * ux * ioph;
            jhy[u] = -wn * uy * ioph;
            if (mode == DEP_TRIAL) {
              const R uxj = R(0.5) * (uxm + ux), uyj = R(0.5) * (uym + uy);
              const R u2 = uxj * uxj + uyj * uyj;
              const R pe = opp - R(1);
              // u_z from gamma - u_z = 1 + psi without cancellation: (u^2 - psi (2 + psi)) /
              // (2 (1+psi))
              const R uzj = (u2 - pe * (R(2) + pe)) * R(0.5) * iopp;
              const R q = -wn * iopp;
              // u_z/(1+psi) - c0 = u^2/(2 opp^2) + (1/opp^2 - 1/opp0^2)/2, the second term
              // formed from the psi fluctuation opp - opp0 without cancellation
              const R dpsi = (opp_raw < floor_) ? dfloor : psi_fl;
              const R iop2 = iopp * iopp;
              const R dz = R(0.5) * u2 * iop2 - R(0.5) * dpsi * (opp0 + opp) * iop2 * iopp02;
              vx[u] = q * uxj;
              vy[u] = q * uyj;
              vdev[u] = -wn * dz;
              const R lx = hx[u] + ox[u], ly = hy[u] + oy[u];
              home[u] = lx >= R(0) && lx < R(1) && ly >= R(0) && ly < R(1);
              if (first) {
                kap += iopp;
                omin = opp_raw < omin ? opp_raw : omin;
                if (opp_raw < floor_) nfloor += R(1);
              }
              if (last) {
                const R gam = (R(1) + u2 + opp * opp) * R(0.5) * iopp;
                const R r = fabs(gam - uzj - opp) * iopp;
                inv = r > inv ? r : inv;
              }
            } else {  // commit
              const R sf = dxi * ioph;
              nox[u] = ox[u] + sf * ux * idx;
              noy[u] = oy[u] + sf * uy * idy;
              pox[i] = nox[u];
              poy[i] = noy[u];
              pux[i] = ux;
              puy[i] = uy;
              pps[i] = psi_p;
              const R lx = hx[u] + nox[u], ly = hy[u] + noy[u];
              home[u] = lx >= R(0) && lx < R(1) && ly >= R(0) && ly < R(1);
            }
          }
          const R vref = (mode == DEP_TRIAL) ? -wn * c0 : -wn;
          const int x1 = (ix + 1 == nx) ? 0 : ix + 1;
          // Aggregated deposit: when every particle of the warp's two sub-lattice positions
          // sits in its home cell (at x^j or x^{j+1} and at x^{j+1/2}), the two particles of a
          // thread share their four corners, and the right corners of lane l are the left
          // corners of lane l + 1: one atomic per node and row instead of four per particle.
          const bool agg = ok[1] && home[0] && home[1] && homeh[0] && homeh[1];
          if (lane_agg && __all_sync(0xffffffffu, agg)) {
            const int lane = threadIdx.x & 31;
            auto put = [&](int f, R a00, R a01, R a10, R a11) {
              R* r0 = tile + ((size_t)f * kTileRows + 1) * nx;  // tile rows 1, 2: home rows
#pragma unroll
              for (int r = 0; r < 2; ++r) {
                const R lft = r ? a10 : a00, rgt = r ? a11 : a01;
                const R from = __shfl_up_sync(0xffffffffu, rgt, 1);
                atomicAdd(r0 + r * nx + ix, lft + (lane ? from : R(0)));
                red_shared_if(lane == 31, r0 + r * nx + x1, rgt);
              }
            };
            W4<R> w[2], d[2], wh[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              w[u] = cic_w(Cic<R>{0, 0, 0, 0, 0, hx[u] + (mode == DEP_TRIAL ? ox[u] : nox[u]),
                                  hy[u] + (mode == DEP_TRIAL ? oy[u] : noy[u])});
              d[u] = (mode == DEP_TRIAL) ? cic_dw(hx[u], hy[u], ox[u], oy[u])
                                         : cic_dw(hx[u], hy[u], nox[u], noy[u]);
              wh[u] = cic_w(Cic<R>{0, 0, 0, 0, 0, lxh[u], lyh[u]});
            }
            const int fh = (mode == DEP_TRIAL) ? 3 : 1;
            if (mode == DEP_TRIAL) {
              put(0, w[0].w00 * vx[0] + w[1].w00 * vx[1], w[0].w01 * vx[0] + w[1].w01 * vx[1],
                  w[0].w10 * vx[0] + w[1].w10 * vx[1], w[0].w11 * vx[0] + w[1].w11 * vx[1]);
              put(1, w[0].w00 * vy[0] + w[1].w00 * vy[1], w[0].w01 * vy[0] + w[1].w01 * vy[1],
                  w[0].w10 * vy[0] + w[1].w10 * vy[1], w[0].w11 * vy[0] + w[1].w11 * vy[1]);
              put(2, w[0].w00 * vdev[0] + w[1].w00 * vdev[1] + (d[0].w00 + d[1].w00) * vref,
                  w[0].w01 * vdev[0] + w[1].w01 * vdev[1] + (d[0].w01 + d[1].w01) * vref,
                  w[0].w10 * vdev[0] + w[1].w10 * vdev[1] + (d[0].w10 + d[1].w10) * vref,
                  w[0].w11 * vdev[0] + w[1].w11 * vdev[1] + (d[0].w11 + d[1].w11) * vref);
            } else {
              put(0, (d[0].w00 + d[1].w00) * vref, (d[0].w01 + d[1].w01) * vref,
                  (d[0].w10 + d[1].w10) * vref, (d[0].w11 + d[1].w11) * vref);
            }
            put(fh, wh[0].w00 * jhx[0] + wh[1].w00 * jhx[1], wh[0].w01 * jhx[0] + wh[1].w01 * jhx[1],
                wh[0].w10 * jhx[0] + wh[1].w10 * jhx[1], wh[0].w11 * jhx[0] + wh[1].w11 * jhx[1]);
            put(fh + 1, wh[0].w00 * jhy[0] + wh[1].w00 * jhy[1],
                wh[0].w01 * jhy[0] + wh[1].w01 * jhy[1], wh[0].w10 * jhy[0] + wh[1].w10 * jhy[1],
                wh[0].w11 * jhy[0] + wh[1].w11 * jhy[1]);
          } else {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if (!ok[u]) continue;
              const R jh[2] = {jhx[u], jhy[u]};
              if (mode == DEP_TRIAL) {
                const W4<R> w = cic_w(c[u]);
                if (home[u]) {
                  // home cell: J_x, J_y, and J_z minus its reference share the four corners
                  const W4<R> d = cic_dw(hx[u], hy[u], ox[u], oy[u]);
                  R* t0 = tile + (size_t)1 * nx;  // field 0, tile row 1 (home row)
                  const size_t fs = (size_t)kTileRows * nx;
                  atomicAdd(t0 + ix, w.w00 * vx[u]);
                  atomicAdd(t0 + x1, w.w01 * vx[u]);
                  atomicAdd(t0 + nx + ix, w.w10 * vx[u]);
                  atomicAdd(t0 + nx + x1, w.w11 * vx[u]);
                  atomicAdd(t0 + fs + ix, w.w00 * vy[u]);
                  atomicAdd(t0 + fs + x1, w.w01 * vy[u]);
                  atomicAdd(t0 + fs + nx + ix, w.w10 * vy[u]);
                  atomicAdd(t0 + fs + nx + x1, w.w11 * vy[u]);
                  atomicAdd(t0 + 2 * fs + ix, w.w00 * vdev[u] + d.w00 * vref);
                  atomicAdd(t0 + 2 * fs + x1, w.w01 * vdev[u] + d.w01 * vref);
                  atomicAdd(t0 + 2 * fs + nx + ix, w.w10 * vdev[u] + d.w10 * vref);
                  atomicAdd(t0 + 2 * fs + nx + x1, w.w11 * vdev[u] + d.w11 * vref);
                } else {
                  const R v3[3] = {vx[u], vy[u], vdev[u] + vref};
                  deposit_n(tile, ovf, fl, c[u], w, 0, nx, ny, v3);
                  const Cic<R> hc = cic<R>(ix, crow, hx[u], hy[u], nx, ny, crow);
                  deposit(tile, ovf, fl, hc, 2, nx, ny, -vref);
                }
                const Cic<R> ch = cic<R>(ix, crow, lxh[u], lyh[u], nx, ny, crow);
                deposit_n(tile, ovf, fl, ch, cic_w(ch), 3, nx, ny, jh);
              } else {
                deposit_ref(tile, ovf, fl, ix, crow, hx[u], hy[u], nox[u], noy[u], 0, nx, ny,
                            R(0), vref);
                const Cic<R> ch = cic<R>(ix, crow, lxh[u], lyh[u], nx, ny, crow);
                deposit_n(tile, ovf, fl, ch, cic_w(ch), 1, nx, ny, jh);
              }
            }
          }
        }
      }
    }
    __syncthreads();
    R* dst = a.part + (size_t)crow * tile_elems;
    {
      // the outer tile rows go out only when a deposit landed there (the row phase reads
      // them only then)
      const int fl = s_flag;
      if (cp4) {
        // 16-byte copies: thread t moves column quad t % nx4 of rows t / nx4 + k rstep
        const float4* t4 = reinterpret_cast<const float4*>(tile);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int row = r0_t; row < nf * kTileRows; row += rstep) {
          const int r = row & (kTileRows - 1);
          if ((r == 0 && !(fl & 1)) || (r == kTileRows - 1 && !(fl & 2))) continue;
          d4[row * nx4 + x4_t] = t4[row * nx4 + x4_t];
        }
      } else {
        for (int row = 0; row < nf * kTileRows; ++row) {
          const int r = row & (kTileRows - 1);
          if ((r == 0 && !(fl & 1)) || (r == kTileRows - 1 && !(fl & 2))) continue;
          for (int x = threadIdx.x; x < nx; x += blockDim.x)
            dst[(size_t)row * nx + x] = tile[(size_t)row * nx + x];
        }
      }
    }
    if (threadIdx.x == 0) a.cflag[crow] = s_flag;
    __syncthreads();
  }
  if (mode == DEP_TRIAL && first) {
    // the three partials of the first solve in one block pass: the sums of 1/(1+psi) and of
    // floored particles, and the minimum of 1 + psi (warps' values summed in warp order)
    const R ks = warp_sum(kap), nfs = warp_sum(nfloor), om = warp_min(omin);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
      red[w] = (double)ks;
      red[nw + w] = (double)nfs;
      red[2 * nw + w] = (double)om;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sk = 0.0, nfl = 0.0, m = red[2 * nw];
      for (int k = 0; k < nw; ++k) {
        sk += red[k];
        nfl += red[nw + k];
        m = fmin(m, red[2 * nw + k]);
      }
      if (sk != 0.0) atomicAdd(&a.diag[D_KAPPA * p.nk + j], sk);
      *pslot(a.dpart, j, P_OPPMIN) = m;
      *pslot(a.dpart, j, P_NFLOOR) = nfl;
      if (nfl > 0) atomicOr(a.bar.status, ST_FLOOR);
    }
  }
  if (mode == DEP_TRIAL && last) {
    double m = block_max_lo(inv, red);
    if (threadIdx.x == 0) *pslot(a.dpart, j, P_INV) = m;
  }
}

// Copy a twiddle table into shared memory (visible after the next __syncthreads).
template <typename R>
__device__ __forceinline__ void load_tw(C<R>* dst, const C<R>* src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// ------------------------------------------------------------------ rows by warps
// FP32 grids 256 points wide take the transforms along x one per warp (warp_fft256): a unit of
// the row phases is kWarpRows grid rows, one per warp of the 256-thread block, and warp w keeps
// its kWarpFftBuf values of the phase buffer at w * kWarpRowStride (a stride that puts the
// block's reads across the rows on distinct banks).  Every kernel that runs these phases
// launches blocks of 256 threads.
constexpr int kWarpRows = 8, kWarpRowStride = kWarpFftBuf + 2;
template <typename R>
__host__ __device__ inline bool warp_rows(const DevParams& p) {
  return sizeof(R) == 4 && p.nx == 256;
}
// Units of the row and inverse-row phases when the other path takes nb rows per unit.
template <typename R>
__host__ __device__ inline int row_units(const DevParams& p, int nb) {
  return warp_rows<R>(p) ? (p.ny + kWarpRows - 1) / kWarpRows : (p.ny + nb - 1) / nb;
}
// Work items of the forward row phase: with rows by warps, one per unit and pair of fields
// (three pairs of a trial phase's five fields, two of the commit's three), so that a block
// takes the pairs of a unit apart and the phase's items spread over more blocks.
template <typename R>
__host__ __device__ inline int row_tasks(const DevParams& p, int nb, int mode) {
  const int u = row_units<R>(p, nb);
  return warp_rows<R>(p) ? u * (mode == DEP_TRIAL ? 3 : 2) : u;
}
// Work items of the inverse row phase: with rows by warps, one per unit and pair of output
// fields.
template <typename R>
__host__ __device__ inline int irow_tasks(const DevParams& p, int nb) {
  const int u = row_units<R>(p, nb);
  return warp_rows<R>(p) ? 2 * u : u;
}

// The same for the column phases of FP32 grids 256 points tall: a unit is one half-spectrum
// column; the forward transforms along y of its fields run one per warp into the block's
// column buffer ([field][k_y], in front of the warps' transform buffers), the k-space solve
// runs one k_y per thread, and the inverse transforms again one per warp.
template <typename R>
__host__ __device__ inline bool warp_cols(const DevParams& p) {
  return sizeof(R) == 4 && p.ny == 256;
}
template <typename R>
__host__ __device__ inline int col_units(const DevParams& p, int nb) {
  return warp_cols<R>(p) ? p.nxh : (p.nxh + nb - 1) / nb;
}
// Forward transform along y, by warp w, of column kx of field w of the row phase's spectra
// into the column buffer.
template <typename R>
__device__ __forceinline__ void col_forward_w(const SweepArgs<R>& a, C<R>* buf, const C<R>* tw,
                                              int kx) {
  constexpr int ny = 256;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C<R>* F = buf + kNF * ny + w * kWarpRowStride;
  const C<R>* col = a.rspec + ((size_t)w * a.p.nxh + kx) * ny;
  C<R> z[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) z[m] = col[lane + 32 * m];
  warp_fft256(z, F, tw, -1);
#pragma unroll
  for (int d = 0; d < 8; ++d) buf[w * ny + lane + 32 * d] = z[d];
}
// Inverse transform along y, by warp w, of output field w of the column buffer into the
// spectra the inverse row phase reads ([field][y][k_x]).
template <typename R>
__device__ __forceinline__ void col_inverse_w(const SweepArgs<R>& a, C<R>* buf, const C<R>* tw,
                                              int kx) {
  constexpr int ny = 256;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nxh = a.p.nxh;
  C<R>* F = buf + kNF * ny + w * kWarpRowStride;
  C<R> z[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) z[m] = buf[w * ny + lane + 32 * m];
  warp_fft256(z, F, tw, +1);
#pragma unroll
  for (int d = 0; d < 8; ++d) a.cspec[((size_t)w * ny + lane + 32 * d) * nxh + kx] = z[d];
}

// One item of the forward row phase by warps: pair pr of fields (2 pr, 2 pr + 1) of rows
// qb .. qb + 7 (those below ny).  Warp w forms the packed pair of row qb + w (the same sums as
// row_phase), transforms it, and leaves the spectrum in its buffer; the block then writes the
// half spectra of its rows, eight consecutive k_y per (field, k_x).  k0: the first
// beam-source node read.  The pairs of a unit are separate items (row_tasks).
template <typename R>
__device__ void row_unit_w(const SweepArgs<R>& a, C<R>* buf, const C<R>* tw, int mode, int k0,
                           int qb, int pr, R& charge) {
  const DevParams& p = a.p;
  constexpr int nx = 256;
  const int ny = p.ny, nxh = p.nxh, nk = p.nk;
  const int nf = (mode == DEP_TRIAL) ? kNF : 3;
  const int npair = (nf + 1) / 2;
  const int tile_elems = kTileRows * nx * nf;
  const int nr = min(kWarpRows, ny - qb);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = qb + w;
  const bool act = w < nr;
  const R* __restrict__ part = a.part;
  R* __restrict__ ovf = a.ovf;
  const R* __restrict__ src = a.src;
  C<R>* F = buf + w * kWarpRowStride;
  const bool s0ok = src != nullptr && k0 >= 0 && k0 < nk;
  const bool s1ok = src != nullptr && k0 + 1 < nk;
  if (threadIdx.x == 0 && src != nullptr) {
    // the unit's rows of the two beam-source nodes into L2 while the partials are read
    const unsigned nbts = (unsigned)((size_t)nr * nx * 4 * sizeof(R));
    if (s0ok) l2_prefetch(src + ((size_t)k0 * ny + qb) * nx * 4, nbts);
    if (s1ok) l2_prefetch(src + ((size_t)(k0 + 1) * ny + qb) * nx * 4, nbts);
  }
  // grid row q collects tile row t of chunk q + 1 - t; rows 1, 2 always, rows 0, 3 and the
  // overflow row only where a deposit landed
  bool use0 = false, use3 = false, od = false;
  const R *p0 = part, *p1 = part, *p2 = part, *p3 = part;
  if (act) {
    use0 = a.cflag[wrap(q + 1, ny)] & 1;
    use3 = a.cflag[wrap(q - 2, ny)] & 2;
    od = a.odirty[q] != 0;
    p0 = part + (size_t)wrap(q + 1, ny) * tile_elems;
    p1 = part + (size_t)q * tile_elems + nx;
    p2 = part + (size_t)wrap(q - 1, ny) * tile_elems + 2 * nx;
    p3 = part + (size_t)wrap(q - 2, ny) * tile_elems + 3 * nx;
  }
  {
    const int f0 = 2 * pr, f1 = 2 * pr + 1;
    if (act) {
      C<R> z[8];
      // the two home tile rows and the beam sources, four columns at a time with every load
      // issued before the sums (the loads are independent; one at a time they would wait on
      // L2 one after the other)
      const size_t fo0 = (size_t)f0 * kTileRows * nx, fo1 = (size_t)f1 * kTileRows * nx;
      const R* e0 = src + ((size_t)k0 * ny + q) * nx * 4;
      const R* e1 = src + ((size_t)(k0 + 1) * ny + q) * nx * 4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        R a0[4], a1[4], b0[4], b1[4], sa[4], sb[4], sc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int x = lane + 32 * (4 * h + i);
          a0[i] = p1[fo0 + x];
          b0[i] = p2[fo0 + x];
          a1[i] = (f1 < nf) ? p1[fo1 + x] : R(0);
          b1[i] = (f1 < nf) ? p2[fo1 + x] : R(0);
          // the source components this pair adds (S_b 0, J_z 1, J_x 2, J_y 3 of nodes k0, k0+1)
          sa[i] = sb[i] = sc[i] = R(0);
          if (mode == DEP_TRIAL) {
            if (pr == 0) {
              if (s0ok) sa[i] = e0[4 * x + 2], sb[i] = e0[4 * x + 3];
            } else if (pr == 1) {
              if (s0ok) sa[i] = e0[4 * x + 1], sb[i] = e0[4 * x + 2];
              if (s1ok) sc[i] = e1[4 * x + 2];
            } else {
              if (s0ok) sa[i] = e0[4 * x + 3];
              if (s1ok) sb[i] = e1[4 * x + 3];
            }
          } else if (pr == 0) {
            if (s1ok) sa[i] = e1[4 * x], sc[i] = e1[4 * x + 2];
            if (s0ok) sb[i] = e0[4 * x + 2];
          } else {
            if (s0ok) sa[i] = e0[4 * x + 3];
            if (s1ok) sb[i] = e1[4 * x + 3];
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          R v0 = a0[i] + b0[i], v1 = a1[i] + b1[i];
          if (mode == DEP_TRIAL) {
            if (pr == 0) {
              v0 += sa[i];
              v1 += sb[i];
            } else if (pr == 1) {
              v0 += sa[i];
              v1 += R(0.5) * (sb[i] + sc[i]);
            } else {
              v0 += R(0.5) * (sa[i] + sb[i]);
            }
          } else if (pr == 0) {
            charge += v0;  // the plasma charge (the rare rows below add to it too)
            v0 += sa[i];
            v1 += R(0.5) * (sb[i] + sc[i]);
          } else {
            v0 += R(0.5) * (sa[i] + sb[i]);
          }
          z[4 * h + i] = C<R>{v0, v1};
        }
      }
      // rare: the outer tile rows and the overflow row, where a deposit landed; four
      // columns at a time, loads first, then the overflow entries zeroed
      if (use0 || use3 || od) {
        R* o0 = ovf + ((size_t)f0 * ny + q) * nx;
        R* o1 = ovf + ((size_t)f1 * ny + q) * nx;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          R v0[4], v1[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int x = lane + 32 * (4 * h + i);
            v0[i] = v1[i] = R(0);
            if (use0) {
              v0[i] += p0[fo0 + x];
              if (f1 < nf) v1[i] += p0[fo1 + x];
            }
            if (use3) {
              v0[i] += p3[fo0 + x];
              if (f1 < nf) v1[i] += p3[fo1 + x];
            }
            if (od) {
              v0[i] += o0[x];
              if (f1 < nf) v1[i] += o1[x];
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int m = 4 * h + i, x = lane + 32 * m;
            if (od) {
              o0[x] = R(0);
              if (f1 < nf) o1[x] = R(0);
            }
            if (mode != DEP_TRIAL && pr == 0) charge += v0[i];
            z[m].x += v0[i];
            z[m].y += v1[i];
          }
        }
      }
      warp_fft256(z, F, tw, -1);
#pragma unroll
      for (int d = 0; d < 8; ++d) F[lane + 32 * d] = z[d];
    }
    __syncthreads();
    // unpack two real transforms: A_k = (Z_k + conj Z_{-k})/2, B_k = -i (Z_k - conj Z_{-k})/2
    for (int e = threadIdx.x; e < kWarpRows * nxh; e += blockDim.x) {
      const int r = e & (kWarpRows - 1), k = e >> 3;
      if (r >= nr) continue;
      const C<R>* Zr = buf + r * kWarpRowStride;
      const C<R> zk = Zr[k];
      const C<R> zm = cconj(Zr[k == 0 ? 0 : nx - k]);
      const C<R> fa = C<R>{R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y + zm.y)};
      const C<R> fb = C<R>{R(0.5) * (zk.y - zm.y), R(-0.5) * (zk.x - zm.x)};
      a.rspec[((size_t)f0 * nxh + k) * ny + qb + r] = fa;
      if (f1 < nf) a.rspec[((size_t)f1 * nxh + k) * ny + qb + r] = fb;
    }
    __syncthreads();
  }
  // the overflow row flags stay set: the unit's other pairs may still read them in other
  // blocks; the column phase that follows clears them (clear_odirty)
}

// Clear the overflow-row flags that the forward row phase by warps has consumed (it cannot
// clear them itself: the pairs of a row are read by different blocks).  Rows u0, u0 + G, ...
template <typename R>
__device__ __forceinline__ void clear_odirty(const SweepArgs<R>& a, int u0, int G) {
  if (!warp_rows<R>(a.p)) return;
  for (int q = u0 * (int)blockDim.x + (int)threadIdx.x; q < a.p.ny; q += G * (int)blockDim.x)
    a.odirty[q] = 0;
}

// One item of the inverse row phase by warps (see irow_phase): warp w transforms row qb + w
// of one packed pair of output fields (pr = 0: psi, d_x psi or B_x, B_y; pr = 1: d_y psi or
// B_z, E_z), read row-contiguous from the column phase's spectra, and writes the field grid,
// and on the last solve its components of the slab, for the 8 columns x = lane + 32 d.  The
// two pairs of a row are independent, so they may run in different blocks.
template <typename R>
__device__ void irow_unit_w(const SweepArgs<R>& a, C<R>* buf, const C<R>* tw, bool psi_mode,
                            int j, bool last, R ez0r, int qb, int pr, R (&en)[6], bool& bad) {
  const DevParams& p = a.p;
  constexpr int nx = 256;
  const int ny = p.ny, nxh = p.nxh;
  const int nout = psi_mode ? 3 : 4;
  const int nr = min(kWarpRows, ny - qb);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w >= nr) return;
  const int q = qb + w;
  const R scale = a.k.scale;
  const C<R>* __restrict__ cspec = a.cspec;
  R* __restrict__ fg = a.fg;
  C<R>* F = buf + w * kWarpRowStride;
  const bool slab = !psi_mode && last;
  // the slab's W = -grad psi comes from the field grid, written one slice earlier and by
  // now often out of L2: fetch the row while the transform runs
  if (slab && pr == 0 && lane == 0)
    l2_prefetch(fg + (size_t)q * nx * kFG, (unsigned)((size_t)nx * kFG * sizeof(R)));
  const C<R>* r0 = cspec + (size_t)q * nxh;  // field f's row: r0 + f * ny * nxh
  const size_t fs = (size_t)ny * nxh;
  const int f0 = 2 * pr, f1 = 2 * pr + 1;
  C<R> z[8];
  // full spectrum of z = a + i b from the half spectra of the real outputs a, b; four
  // columns at a time with the loads issued first
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    C<R> fa[4], fb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = lane + 32 * (4 * h + i);
      const int kk = (k < nxh) ? k : nx - k;
      fa[i] = r0[f0 * fs + kk];
      fb[i] = (f1 < nout) ? r0[f1 * fs + kk] : C<R>{0, 0};
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = lane + 32 * (4 * h + i);
      const int kk = (k < nxh) ? k : nx - k;
      if (kk == 0 || 2 * kk == nx) {  // self-conjugate columns
        fa[i].y = R(0);
        fb[i].y = R(0);
      }
      if (k >= nxh) {
        fa[i] = cconj(fa[i]);
        fb[i] = cconj(fb[i]);
      }
      z[4 * h + i] = cadd(fa[i], cmuli(fb[i]));
    }
  }
  warp_fft256(z, F, tw, +1);
  if (!slab) {
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      R* node = fg + ((size_t)q * nx + lane + 32 * d) * kFG;
      const R va = z[d].x * scale, vb = z[d].y * scale;
      if (pr == 0) {
        node[psi_mode ? FG_PSI : FG_BX] = va;
        node[psi_mode ? FG_GX : FG_BY] = vb;
      } else if (psi_mode) {
        node[FG_GY] = va;
      } else {
        node[FG_BZ] = va;
        node[FG_EZ] = vb;
      }
    }
    return;
  }
  // the last solve: the field grid, this pair's components of the slab node (W_x, W_y, B_x,
  // B_y from the first; E_z and B_z, with the node's two pads, from the second), their
  // energies and the finiteness check
  if (pr == 0) {
    // W = -grad psi from the field grid, four columns at a time with the loads issued first
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      R gx[4], gy[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const R* node = fg + ((size_t)q * nx + lane + 32 * (4 * h + i)) * kFG;
        gx[i] = node[FG_GX];
        gy[i] = node[FG_GY];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int d = 4 * h + i, x = lane + 32 * d;
        R* node = fg + ((size_t)q * nx + x) * kFG;
        const R bx = z[d].x * scale, by = z[d].y * scale;
        node[FG_BX] = bx;
        node[FG_BY] = by;
        const R wx = -gx[i], wy = -gy[i];
        R* sl = a.slab + (((size_t)j * ny + q) * nx + x) * 8;
        sl[0] = wx;
        sl[1] = wy;
        sl[3] = bx;
        sl[4] = by;
        const R Ex = wx + by, Ey = wy - bx;
        en[0] += Ex * Ex;
        en[1] += Ey * Ey;
        en[3] += bx * bx;
        en[4] += by * by;
        if (!(isfinite(Ex) && isfinite(Ey))) bad = true;
      }
    }
  } else {
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int x = lane + 32 * d;
      R* node = fg + ((size_t)q * nx + x) * kFG;
      const R va = z[d].x * scale, vb = z[d].y * scale;
      node[FG_BZ] = va;
      node[FG_EZ] = vb;
      const R ez = ez0r + vb;
      R* sl = a.slab + (((size_t)j * ny + q) * nx + x) * 8;
      sl[2] = ez;
      sl[5] = va;
      sl[6] = R(0);
      sl[7] = R(0);
      en[2] += ez * ez;
      en[5] += va * va;
      if (!(isfinite(ez) && isfinite(va))) bad = true;
    }
  }
}

// ------------------------------------------------------------------ row phase (forward)
// mode DEP_TRIAL: fields Jx^j, Jy^j, Jz^j, Jx^{j+1/2}, Jy^{j+1/2} of slice j = jj.
// else: fields S, Jx^{jn-1/2}, Jy^{jn-1/2} of the new slice jn = jj.
// A unit of the FFT phases is nb consecutive rows (or half-spectrum columns): their
// transforms run in one block_fft call (more butterflies per thread between the stage
// barriers) and the transposed writes of neighbouring rows (columns) land next to each other.
// With rows by warps (FP32, 256 wide) a unit is kWarpRows rows and its pairs of fields are
// dealt as separate items (row_tasks, irow_tasks).
template <typename R>
__device__ void row_phase(const SweepArgs<R>& a, C<R>* buf, C<R>* tw, int mode, int jj, int u0,
                          int G, int nb) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny, nxh = p.nxh, nk = p.nk;
  const int nf = (mode == DEP_TRIAL) ? kNF : 3;
  const int npair = (nf + 1) / 2;
  C<R>* A = buf;
  C<R>* B = buf + 3 * nx * nb;
  const int tile_elems = kTileRows * nx * nf;
  const R* __restrict__ part = a.part;
  R* __restrict__ ovf = a.ovf;
  const R* __restrict__ src = a.src;
  __shared__ double red[32];
  const bool wr = warp_rows<R>(p);
  const int ntask = row_tasks<R>(p, nb, mode);
  if (wr ? u0 >= ntask : u0 * nb >= ny) {  // no unit in this block
    if (threadIdx.x == 0 && mode != DEP_TRIAL) *pslot(a.dpart, jj, P_CHARGE) = 0.0;
    return;
  }
  R charge = R(0);
  load_tw(tw, a.twx, nx);
  const int k0 = (mode == DEP_TRIAL) ? jj : jj - 1;  // beam-source nodes k0, k0 + 1
  if (wr) {
    __syncthreads();
    for (int t = u0; t < ntask; t += G)
      row_unit_w(a, buf, tw, mode, k0, (t / npair) * kWarpRows, t % npair, charge);
  }
  for (int u = u0; !wr && u * nb < ny; u += G) {
    const int qb = u * nb, nr = min(nb, ny - qb);
    if (threadIdx.x == 0 && src != nullptr) {
      // the unit's rows of the two beam-source nodes into L2 while the partials are read
      const unsigned nbts = (unsigned)((size_t)nr * nx * 4 * sizeof(R));
      if (k0 >= 0 && k0 < nk) l2_prefetch(src + ((size_t)k0 * ny + qb) * nx * 4, nbts);
      if (k0 + 1 < nk) l2_prefetch(src + ((size_t)(k0 + 1) * ny + qb) * nx * 4, nbts);
    }
    for (int r = 0; r < nr; ++r) {
    const int q = qb + r;
    // grid row q collects tile row t of chunk q + 1 - t; rows 1, 2 always, rows 0, 3 and the
    // overflow row only where a deposit landed
    const bool use0 = a.cflag[wrap(q + 1, ny)] & 1, use3 = a.cflag[wrap(q - 2, ny)] & 2;
    const bool od = a.odirty[q] != 0;
    const R* p0 = part + (size_t)wrap(q + 1, ny) * tile_elems;
    const R* p1 = part + (size_t)q * tile_elems + nx;
    const R* p2 = part + (size_t)wrap(q - 1, ny) * tile_elems + 2 * nx;
    const R* p3 = part + (size_t)wrap(q - 2, ny) * tile_elems + 3 * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      R v[kNF];
#pragma unroll
      for (int f = 0; f < kNF; ++f) {
        if (f < nf) {
          const size_t fo = (size_t)f * kTileRows * nx + x;
          R s = p1[fo] + p2[fo];
          if (use0) s += p0[fo];
          if (use3) s += p3[fo];
          if (od) s += ovf[((size_t)f * ny + q) * nx + x];
          v[f] = s;
        } else {
          v[f] = R(0);
        }
      }
      // beam sources [nk][ny][nx][4]: 0 S_b, 1 J_z, 2 J_x, 3 J_y (deviations)
      R s0[4] = {0, 0, 0, 0}, s1[4] = {0, 0, 0, 0};
      if (src != nullptr) {
        if (k0 >= 0 && k0 < nk) {
          const R* e = src + (((size_t)k0 * ny + q) * nx + x) * 4;
#pragma unroll
          for (int k = 0; k < 4; ++k) s0[k] = e[k];
        }
        if (k0 + 1 < nk) {
          const R* e = src + (((size_t)(k0 + 1) * ny + q) * nx + x) * 4;
#pragma unroll
          for (int k = 0; k < 4; ++k) s1[k] = e[k];
        }
      }
      if (od)
        for (int f = 0; f < nf; ++f) ovf[((size_t)f * ny + q) * nx + x] = R(0);
      if (mode == DEP_TRIAL) {
        v[0] += s0[2];
        v[1] += s0[3];
        v[2] += s0[1];
        v[3] += R(0.5) * (s0[2] + s1[2]);
        v[4] += R(0.5) * (s0[3] + s1[3]);
      } else {
        charge += v[0];
        v[0] += s1[0];
        v[1] += R(0.5) * (s0[2] + s1[2]);
        v[2] += R(0.5) * (s0[3] + s1[3]);
      }
#pragma unroll
      for (int pr = 0; pr < 3; ++pr)
        if (pr < npair)
          A[(r * npair + pr) * nx + x] =
              C<R>{v[2 * pr], (2 * pr + 1 < kNF) ? v[2 * pr + 1] : R(0)};
    }
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int r = 0; r < nr; ++r) a.odirty[qb + r] = 0;  // consumed (read before the barrier)
    C<R>* Z = block_fft(A, B, nr * npair, p.px, tw, -1);
    // unpack two real transforms: A_k = (Z_k + conj Z_{-k})/2, B_k = -i (Z_k - conj Z_{-k})/2
    for (int e = threadIdx.x; e < npair * nxh * nr; e += blockDim.x) {
      const int t = div_small(e, nr), r = e - t * nr, pr = div_by(t, p.fd_nxh);
      const int k = t - pr * nxh, q = qb + r;
      const C<R>* zr = Z + (r * npair + pr) * nx;
      const C<R> zk = zr[k];
      const C<R> zm = cconj(zr[k == 0 ? 0 : nx - k]);
      const C<R> fa = C<R>{R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y + zm.y)};
      const C<R> fb = C<R>{R(0.5) * (zk.y - zm.y), R(-0.5) * (zk.x - zm.x)};
      a.rspec[((size_t)(2 * pr) * nxh + k) * ny + q] = fa;
      if (2 * pr + 1 < nf) a.rspec[((size_t)(2 * pr + 1) * nxh + k) * ny + q] = fb;
    }
    __syncthreads();
  }
  if (mode != DEP_TRIAL) {
    double s = block_sum_lo(charge, red);
    if (threadIdx.x == 0) *pslot(a.dpart, jj, P_CHARGE) = s * p.dx * p.dy;
  }
}

// Wavenumbers of half-spectrum column kx and row ky from the table built on the host in FP64,
// ktab = [k_x (nxh)][k_x derivative symbol (nxh)][k_y (ny)][k_y derivative symbol (ny)], the
// derivative symbols zero at the Nyquist index.
template <typename R>
struct Kv {
  R kxd, kyd, k2;
};
template <typename R>
__device__ __forceinline__ Kv<R> kvec(const R* __restrict__ ktab, int nxh, int ny, int kx,
                                      int ky) {
  Kv<R> k;
  const R kxv = ktab[kx], kyv = ktab[2 * nxh + ky];
  k.kxd = ktab[nxh + kx];
  k.kyd = ktab[2 * nxh + ny + ky];
  k.k2 = kxv * kxv + kyv * kyv;
  return k;
}

// Record the diagnosed modes that live in columns kb .. kb + nc - 1 of the column buffer O
// (per column nf spectra of ny rows, in the order given by fields[]: output field index of
// each spectrum, -1 to skip) as F(k)/(nx ny) of slice j.  Reads O only, before the inverse
// transform's first stage barrier.
template <typename R>
__device__ __forceinline__ void record_modes(const SweepArgs<R>& a, const C<R>* O, int kb,
                                             int nc, int nf, const int* fields, int j) {
  const DevParams& p = a.p;
  if (a.mode_out == nullptr || j < 0) return;
  for (int m = threadIdx.x; m < p.nmodes; m += blockDim.x) {
    const int c = p.mkx[m] - kb;
    if (c < 0 || c >= nc) continue;
    const R sg = p.mconj[m] ? R(-1) : R(1);
    R* o = a.mode_out + ((size_t)j * p.nmodes + m) * 10;
    for (int f = 0; f < nf; ++f) {
      if (fields[f] < 0) continue;
      const C<R> v = O[((size_t)c * nf + f) * p.ny + p.mky[m]];
      o[2 * fields[f]] = v.x * a.k.scale;
      o[2 * fields[f] + 1] = sg * v.y * a.k.scale;
    }
  }
}

// ------------------------------------------------------------------ column phase: B, E_z
// psi0: the k = 0 potential of the slice, which fixes the plasma reference state of the
// deposits (needed for <J_z>, the source of the k = 0 mode).
template <typename R>
__device__ void col_phase_b(const SweepArgs<R>& a, C<R>* buf, C<R>* tw, int j, bool last,
                            double psi0, int u0, int G, int nb) {
  const DevParams& p = a.p;
  const int ny = p.ny, nxh = p.nxh;
  C<R>* A = buf;
  C<R>* B = buf + kNF * ny * nb;
  __shared__ R s_kap;
  clear_odirty(a, u0, G);
  if (u0 * (warp_cols<R>(p) ? 1 : nb) >= nxh) {  // no unit in this block
    if (threadIdx.x == 0 && last) {
      *pslot(a.dpart, j, P_PCNUM) = 0.0;
      *pslot(a.dpart, j, P_PCDEN) = 0.0;
    }
    return;
  }
  if (threadIdx.x == 0) s_kap = R(a.diag[D_KAPPA * p.nk + j]) * a.k.inv_npc;
  const R rdxi = a.k.rdxi;
  const C<R>* __restrict__ rspec = a.rspec;
  C<R>* __restrict__ bold = a.bold;
  const C<R>* __restrict__ jprev = a.jprev;
  __shared__ double red[32];
  R num = R(0), den = R(0);
  load_tw(tw, a.twy, ny);
  const bool wc = warp_cols<R>(p);
  if (wc) __syncthreads();  // the table and s_kap
  for (int kx = u0; wc && kx < nxh; kx += G) {
    const int w = threadIdx.x >> 5;
    if (w < kNF) col_forward_w(a, buf, tw, kx);
    __syncthreads();
    {
      // the solve at k_y = threadIdx.x, in place: outputs B_x, B_y, B_z, E_z over fields 0..3
      const int ky = threadIdx.x;
      const R kap = s_kap;
      const R pw = (kx == 0 || ((p.nx % 2 == 0) && 2 * kx == p.nx)) ? R(1) : R(2);
      const size_t ix0 = (size_t)kx * ny + ky, ix1 = ((size_t)nxh + kx) * ny + ky;
      const C<R> Jxp = jprev[ix0], Jyp = jprev[ix1];
      const C<R> Bxo = bold[ix0], Byo = bold[ix1];
      const C<R> Jx = buf[ky], Jy = buf[ny + ky], Jz = buf[2 * ny + ky];
      const C<R> Jxh = buf[3 * ny + ky], Jyh = buf[4 * ny + ky];
      if (kx == 0 && ky == 0) {
        const double opp0 = 1.0 + psi0;
        const double jz_ref =
            psi0 * (2.0 + psi0) / (2.0 * opp0 * opp0) + (a.bref ? a.bref[j] : 0.0);
        a.diag[D_JZ * p.nk + j] = (double)Jz.x / ((double)p.nx * p.ny) + jz_ref;
      }
      const Kv<R> k = kvec(a.ktab, nxh, ny, kx, ky);
      C<R> obx{0, 0}, oby{0, 0}, obz{0, 0}, oez{0, 0};
      if (k.k2 > R(0)) {
        const R ik2 = R(1) / k.k2;
        const R kxd = k.kxd, kyd = k.kyd;
        const C<R> Dx = cscale(csub(Jxh, Jxp), rdxi), Dy = cscale(csub(Jyh, Jyp), rdxi);
        obz = cscale(cmuli(csub(cscale(Jy, kxd), cscale(Jx, kyd))), ik2);
        oez = cscale(cmuli(cadd(cscale(Jx, kxd), cscale(Jy, kyd))), -ik2);
        const R ih = R(1) / (k.k2 + kap);
        obx = cscale(cadd(cadd(cmuli(cscale(Jz, kyd)), Dy), cscale(Bxo, kap)), ih);
        oby = cscale(csub(csub(cscale(Byo, kap), cmuli(cscale(Jz, kxd))), Dx), ih);
        if (last) {
          const R ex = obx.x - Bxo.x, ey = obx.y - Bxo.y;
          const R fx = oby.x - Byo.x, fy = oby.y - Byo.y;
          num += pw * (ex * ex + ey * ey + fx * fx + fy * fy);
          den += pw * (obx.x * obx.x + obx.y * obx.y + oby.x * oby.x + oby.y * oby.y);
        }
      }
      bold[ix0] = obx;
      bold[ix1] = oby;
      buf[ky] = obx;
      buf[ny + ky] = oby;
      buf[2 * ny + ky] = obz;
      buf[3 * ny + ky] = oez;
    }
    __syncthreads();
    if (last) {
      const int fields[4] = {2, 3, 4, 1};  // B_x, B_y, B_z, E_z
      record_modes(a, buf, kx, 1, 4, fields, j);
    }
    if (w < 4) col_inverse_w(a, buf, tw, kx);
    __syncthreads();  // the column buffer is the next unit's
  }
  for (int u = u0; !wc && u * nb < nxh; u += G) {
    const int kb = u * nb, nc = min(nb, nxh - kb);
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
      const int c = div_by(e, p.fd_ny), ky = e - c * ny, kx = kb + c;
      C<R> v[kNF];
#pragma unroll
      for (int f = 0; f < kNF; ++f) v[f] = rspec[((size_t)f * nxh + kx) * ny + ky];
#pragma unroll
      for (int f = 0; f < kNF; ++f) A[(c * kNF + f) * ny + ky] = v[f];
    }
    __syncthreads();
    const R kap = s_kap;
    C<R>* Z = block_fft(A, B, nc * kNF, p.py, tw, -1);
    C<R>* O = (Z == A) ? B : A;
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
      const int c = div_by(e, p.fd_ny), ky = e - c * ny, kx = kb + c;
      const R pw = (kx == 0 || ((p.nx % 2 == 0) && 2 * kx == p.nx)) ? R(1) : R(2);
      const C<R>* Zc = Z + c * kNF * ny;
      C<R>* Oc = O + c * 4 * ny;
      const size_t ix0 = (size_t)kx * ny + ky, ix1 = ((size_t)nxh + kx) * ny + ky;
      const C<R> Jxp = jprev[ix0], Jyp = jprev[ix1];
      const C<R> Bxo = bold[ix0], Byo = bold[ix1];
      const C<R> Jx = Zc[ky], Jy = Zc[ny + ky], Jz = Zc[2 * ny + ky];
      const C<R> Jxh = Zc[3 * ny + ky], Jyh = Zc[4 * ny + ky];
      if (kx == 0 && ky == 0) {
        // <J_z> for the k = 0 mode: the grid mean plus the uniform parts left out of the grid
        // deposits (plasma reference state and beam reference density)
        const double opp0 = 1.0 + psi0;
        const double jz_ref =
            psi0 * (2.0 + psi0) / (2.0 * opp0 * opp0) + (a.bref ? a.bref[j] : 0.0);
        a.diag[D_JZ * p.nk + j] = (double)Jz.x / ((double)p.nx * p.ny) + jz_ref;
      }
      const Kv<R> k = kvec(a.ktab, nxh, ny, kx, ky);
      C<R> obx{0, 0}, oby{0, 0}, obz{0, 0}, oez{0, 0};
      if (k.k2 > R(0)) {
        const R ik2 = R(1) / k.k2;
        const R kxd = k.kxd, kyd = k.kyd;
        const C<R> Dx = cscale(csub(Jxh, Jxp), rdxi), Dy = cscale(csub(Jyh, Jyp), rdxi);
        // B_z = (i kx Jy - i ky Jx)/k^2 ; E_z = -(i kx Jx + i ky Jy)/k^2
        obz = cscale(cmuli(csub(cscale(Jy, kxd), cscale(Jx, kyd))), ik2);
        oez = cscale(cmuli(cadd(cscale(Jx, kxd), cscale(Jy, kyd))), -ik2);
        const R ih = R(1) / (k.k2 + kap);
        // (k^2 + kappa^2) B_x = i ky Jz + D_y + kappa^2 Bx_old
        obx = cscale(cadd(cadd(cmuli(cscale(Jz, kyd)), Dy), cscale(Bxo, kap)), ih);
        // (k^2 + kappa^2) B_y = -i kx Jz - D_x + kappa^2 By_old
        oby = cscale(csub(csub(cscale(Byo, kap), cmuli(cscale(Jz, kxd))), Dx), ih);
        if (last) {
          const R ex = obx.x - Bxo.x, ey = obx.y - Bxo.y;
          const R fx = oby.x - Byo.x, fy = oby.y - Byo.y;
          num += pw * (ex * ex + ey * ey + fx * fx + fy * fy);
          den += pw * (obx.x * obx.x + obx.y * obx.y + oby.x * oby.x + oby.y * oby.y);
        }
      }
      bold[ix0] = obx;
      bold[ix1] = oby;
      Oc[ky] = obx;
      Oc[ny + ky] = oby;
      Oc[2 * ny + ky] = obz;
      Oc[3 * ny + ky] = oez;
    }
    __syncthreads();
    if (last) {
      const int fields[4] = {2, 3, 4, 1};  // B_x, B_y, B_z, E_z
      record_modes(a, O, kb, nc, 4, fields, j);
    }
    C<R>* W = block_fft(O, Z, nc * 4, p.py, tw, +1);
    for (int e = threadIdx.x; e < 4 * ny * nc; e += blockDim.x) {
      const int t = div_small(e, nc), c = e - t * nc, f = div_by(t, p.fd_ny), ky = t - f * ny;
      a.cspec[((size_t)f * ny + ky) * nxh + kb + c] = W[(c * 4 + f) * ny + ky];
    }
    __syncthreads();
  }
  if (last) {
    double s = block_sum_lo(num, red);
    if (threadIdx.x == 0) *pslot(a.dpart, j, P_PCNUM) = s;
    s = block_sum_lo(den, red);
    if (threadIdx.x == 0) *pslot(a.dpart, j, P_PCDEN) = s;
  }
}

// ------------------------------------------------------------------ column phase: psi
template <typename R>
__device__ void col_phase_psi(const SweepArgs<R>& a, C<R>* buf, C<R>* tw, int u0, int G,
                              int nb, int jn) {
  const DevParams& p = a.p;
  const int ny = p.ny, nxh = p.nxh;
  C<R>* A = buf;
  C<R>* B = buf + kNF * ny * nb;
  const C<R>* __restrict__ rspec = a.rspec;
  const bool wc = warp_cols<R>(p);
  clear_odirty(a, u0, G);
  if (u0 * (wc ? 1 : nb) >= nxh) return;  // no unit in this block
  load_tw(tw, a.twy, ny);
  if (wc) __syncthreads();  // the table
  for (int kx = u0; wc && kx < nxh; kx += G) {
    const int w = threadIdx.x >> 5;
    if (w < 3) col_forward_w(a, buf, tw, kx);
    __syncthreads();
    {
      // psi and its gradient at k_y = threadIdx.x, in place over fields 0..2; the spectra of
      // J_perp^{j-1/2} are kept for the next slice's B_perp solves
      const int ky = threadIdx.x;
      const size_t ix0 = (size_t)kx * ny + ky, ix1 = ((size_t)nxh + kx) * ny + ky;
      a.jprev[ix0] = buf[ny + ky];
      a.jprev[ix1] = buf[2 * ny + ky];
      const Kv<R> k = kvec(a.ktab, nxh, ny, kx, ky);
      C<R> ps{0, 0};
      if (k.k2 > R(0)) ps = cscale(buf[ky], R(1) / k.k2);
      buf[ky] = ps;
      buf[ny + ky] = cmuli(cscale(ps, k.kxd));
      buf[2 * ny + ky] = cmuli(cscale(ps, k.kyd));
    }
    __syncthreads();
    {
      const int fields[3] = {0, -1, -1};  // psi
      record_modes(a, buf, kx, 1, 3, fields, jn);
    }
    if (w < 3) col_inverse_w(a, buf, tw, kx);
    __syncthreads();  // the column buffer is the next unit's
  }
  for (int u = u0; !wc && u * nb < nxh; u += G) {
    const int kb = u * nb, nc = min(nb, nxh - kb);
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
      const int c = div_by(e, p.fd_ny), ky = e - c * ny, kx = kb + c;
      C<R> v[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) v[f] = rspec[((size_t)f * nxh + kx) * ny + ky];
#pragma unroll
      for (int f = 0; f < 3; ++f) A[(c * 3 + f) * ny + ky] = v[f];
    }
    __syncthreads();
    C<R>* Z = block_fft(A, B, nc * 3, p.py, tw, -1);
    C<R>* O = (Z == A) ? B : A;
    for (int e = threadIdx.x; e < nc * ny; e += blockDim.x) {
      const int c = div_by(e, p.fd_ny), ky = e - c * ny, kx = kb + c;
      const C<R>* Zc = Z + c * 3 * ny;
      C<R>* Oc = O + c * 3 * ny;
      const size_t ix0 = (size_t)kx * ny + ky, ix1 = ((size_t)nxh + kx) * ny + ky;
      a.jprev[ix0] = Zc[ny + ky];
      a.jprev[ix1] = Zc[2 * ny + ky];
      const Kv<R> k = kvec(a.ktab, nxh, ny, kx, ky);
      C<R> ps{0, 0};
      if (k.k2 > R(0)) ps = cscale(Zc[ky], R(1) / k.k2);
      Oc[ky] = ps;
      Oc[ny + ky] = cmuli(cscale(ps, k.kxd));
      Oc[2 * ny + ky] = cmuli(cscale(ps, k.kyd));
    }
    __syncthreads();
    {
      const int fields[3] = {0, -1, -1};  // psi
      record_modes(a, O, kb, nc, 3, fields, jn);
    }
    C<R>* W = block_fft(O, Z, nc * 3, p.py, tw, +1);
    for (int e = threadIdx.x; e < 3 * ny * nc; e += blockDim.x) {
      const int t = div_small(e, nc), c = e - t * nc, f = div_by(t, p.fd_ny), ky = t - f * ny;
      a.cspec[((size_t)f * ny + ky) * nxh + kb + c] = W[(c * 3 + f) * ny + ky];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ inverse row phase
// psi_mode: outputs psi, d_x psi, d_y psi.  Else: B_x, B_y, B_z, E_z; on the last trial
// iteration also the slab of slice j and the field energies.
template <typename R>
__device__ void irow_phase(const SweepArgs<R>& a, C<R>* buf, C<R>* tw, bool psi_mode, int j,
                           bool last, double ez0j, int u0, int G, int nb) {
  const DevParams& p = a.p;
  const int nx = p.nx, ny = p.ny, nxh = p.nxh;
  const int nout = psi_mode ? 3 : 4;
  const int npair = 2;
  C<R>* A = buf;
  C<R>* B = buf + 3 * nx * nb;
  const R scale = a.k.scale;
  const R ez0r = R(ez0j);
  const C<R>* __restrict__ cspec = a.cspec;
  R* __restrict__ fg = a.fg;
  __shared__ double red[64];
  const bool wr = warp_rows<R>(p);
  const int ntask = irow_tasks<R>(p, nb);
  if (wr ? u0 >= ntask : u0 * nb >= ny) {  // no unit in this block
    if (threadIdx.x == 0 && !psi_mode && last)
      for (int f = 0; f < 6; ++f) *pslot(a.dpart, j, P_E0 + f) = 0.0;
    return;
  }
  R en[6] = {0, 0, 0, 0, 0, 0};
  bool bad = false;
  load_tw(tw, a.twx, nx);
  if (wr) {
    __syncthreads();
    for (int t = u0; t < ntask; t += G)
      irow_unit_w(a, buf, tw, psi_mode, j, last, ez0r, (t >> 1) * kWarpRows, t & 1, en, bad);
    __syncthreads();  // the buffers and the table are reused by the block's next phase
  }
  for (int u = u0; !wr && u * nb < ny; u += G) {
    const int qb = u * nb, nr = min(nb, ny - qb);
    // the slab of the last solve adds W = -grad psi from the field grid, written one slice
    // earlier and by now often out of L2: fetch the unit's rows while the transforms run
    if (!psi_mode && last && threadIdx.x == 0)
      l2_prefetch(fg + (size_t)qb * nx * kFG, (unsigned)((size_t)nr * nx * kFG * sizeof(R)));
    for (int e = threadIdx.x; e < nr * npair * nx; e += blockDim.x) {
      const int rp = div_by(e, p.fd_nx), k = e - rp * nx, r = rp >> 1, pr = rp - 2 * r,
                q = qb + r;  // npair = 2
      const int f0 = 2 * pr, f1 = 2 * pr + 1;
      // full spectrum of z = a + i b from the half spectra of the real outputs a, b
      const int kk = (k < nxh) ? k : nx - k;
      C<R> fa = cspec[((size_t)f0 * ny + q) * nxh + kk];
      C<R> fb = (f1 < nout) ? cspec[((size_t)f1 * ny + q) * nxh + kk] : C<R>{0, 0};
      const bool selfconj = (kk == 0) || ((nx % 2 == 0) && 2 * kk == nx);
      if (selfconj) {
        fa.y = R(0);
        fb.y = R(0);
      }
      if (k >= nxh) {
        fa = cconj(fa);
        fb = cconj(fb);
      }
      A[rp * nx + k] = cadd(fa, cmuli(fb));
    }
    __syncthreads();
    C<R>* Z = block_fft(A, B, nr * npair, p.px, tw, +1);
    for (int e = threadIdx.x; e < nr * nx; e += blockDim.x) {
      const int r = div_by(e, p.fd_nx), x = e - r * nx, q = qb + r;
      const C<R>* Zr = Z + r * npair * nx;
      R v[4];
      v[0] = Zr[x].x * scale;
      v[1] = Zr[x].y * scale;
      v[2] = Zr[nx + x].x * scale;
      v[3] = Zr[nx + x].y * scale;
      const size_t g = (size_t)q * nx + x;
      R* node = fg + g * kFG;
      if (psi_mode) {
        node[FG_PSI] = v[0];
        node[FG_GX] = v[1];
        node[FG_GY] = v[2];
      } else {
        node[FG_BX] = v[0];
        node[FG_BY] = v[1];
        node[FG_BZ] = v[2];
        node[FG_EZ] = v[3];
      }
      if (!psi_mode && last) {
        const R wx = -node[FG_GX], wy = -node[FG_GY];
        const R ez = ez0r + v[3];
        st8(a.slab + (((size_t)j * ny + q) * nx + x) * 8, wx, wy, ez, v[0], v[1], v[2]);
        const R Ex = wx + v[1], Ey = wy - v[0];
        en[0] += Ex * Ex;
        en[1] += Ey * Ey;
        en[2] += ez * ez;
        en[3] += v[0] * v[0];
        en[4] += v[1] * v[1];
        en[5] += v[2] * v[2];
        if (!(isfinite(Ex) && isfinite(Ey) && isfinite(ez) && isfinite(v[2]))) bad = true;
      }
    }
    __syncthreads();
  }
  if (!psi_mode && last) {
    const double cell = 0.5 * p.dx * p.dy * p.dxi;
    double tot[6];
    block_sum_lo_n<6>(en, tot, red);
    if (threadIdx.x == 0)
      for (int f = 0; f < 6; ++f)
        *pslot(a.dpart, j, P_E0 + f) = tot[f] * cell;
    if (bad) atomicOr(a.bar.status, ST_NONFINITE);
  }
}

// Shared-memory layout of the persistent kernels: the phase buffer (deposit tile or FFT
// buffers) followed by a twiddle table.
template <typename R>
__host__ __device__ inline size_t phase_smem_bytes(int nx, int ny, int nbr = 1, int nbc = 1) {
  size_t tile = (size_t)kTileRows * nx * kNF * sizeof(R);
  size_t row = (size_t)2 * 3 * nx * nbr * sizeof(C<R>);
  size_t col = (size_t)2 * kNF * ny * nbc * sizeof(C<R>);
  size_t m = tile > row ? tile : row;
  m = m > col ? m : col;
  // the per-warp paths (grids 256 wide or tall); a multi-slot launch sizes its buffer for
  // its largest grid, so every size from 256 up covers them
  if (sizeof(R) == 4 && nx >= 256) {  // per-warp row transforms
    const size_t wr = (size_t)kWarpRows * kWarpRowStride * sizeof(C<R>);
    m = m > wr ? m : wr;
  }
  if (sizeof(R) == 4 && ny >= 256) {  // column buffer and five per-warp transform buffers
    const size_t wc = ((size_t)kNF * 256 + kNF * kWarpRowStride) * sizeof(C<R>);
    m = m > wc ? m : wc;
  }
  return (m + 15) & ~size_t(15);
}
template <typename R>
__host__ __device__ inline size_t sweep_smem_bytes(int nx, int ny, int nbr = 1, int nbc = 1) {
  return phase_smem_bytes<R>(nx, ny, nbr, nbc) + (size_t)(nx > ny ? nx : ny) * sizeof(C<R>);
}

// ------------------------------------------------------------------ the kernel
// Tolerance mode of the predictor-corrector: has the last B_perp solve of slice j changed
// B_perp by less than pc_tol (relative, in the 2-norm over the grid)?  The solve's squared
// change and squared norm are in the per-block partial slots of slice j (written by every
// block before the barrier that precedes this call); each block sums all of them in the same
// order, so every block reaches the same answer.  Called by all threads of the block.
template <typename R>
__device__ bool pc_converged(const SweepArgs<R>& a, int j) {
  __shared__ double red[32];
  __shared__ int s_conv;
  double num = 0.0, den = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double* e = a.dpart + ((size_t)j * gridDim.x + b) * P_COUNT;
    num += __ldcg(e + P_PCNUM);  // through L2: earlier iterations left these slots in L1
    den += __ldcg(e + P_PCDEN);
  }
  const double N = block_sum_lo(num, red);
  const double D = block_sum_lo(den, red);
  // a zero field has converged; a non-finite sum never does
  if (threadIdx.x == 0) s_conv = (N < a.p.pc_tol2 * D) || (N == 0.0);
  __syncthreads();
  return s_conv != 0;
}

// Copies into the tape (see Tape): snap 0 at the start of slice j also takes the particle
// state and the J_perp^{j-1/2} spectra.  All blocks share the copy (grid-stride); it only
// reads buffers that no phase writes before the next grid barrier but one.
template <typename R>
__device__ void record_tape(const SweepArgs<R>& a, int j, int snap) {
  const DevParams& p = a.p;
  const size_t g = (size_t)p.nx * p.ny;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  R* fdst = a.tape.fg + ((size_t)j * (p.n_pc + 1) + snap) * g * kFG;
  for (size_t e = t0; e < g * kFG; e += st) fdst[e] = a.fg[e];
  if (snap != 0) return;
  const size_t np = (size_t)p.np;
  R* pd = a.tape.part + (size_t)j * 5 * np;
  const int per_chunk = p.ppc * p.nx;
  for (size_t i = t0; i < np; i += st) {
    const int crow = (int)(i / per_chunk);
    const int rem = (int)(i - (size_t)crow * per_chunk);
    const int sub = rem / p.nx, ix = rem - sub * p.nx;
    const int sy = sub / p.ppx, sx = sub - sy * p.ppx;
    const R hx = (R(sx) + R(0.5)) * a.k.inv_ppx, hy = (R(sy) + R(0.5)) * a.k.inv_ppy;
    pd[i] = (R(ix) + hx + a.pox[i]) * R(p.dx);
    pd[np + i] = (R(crow) + hy + a.poy[i]) * R(p.dy);
    pd[2 * np + i] = a.pux[i];
    pd[3 * np + i] = a.puy[i];
    pd[4 * np + i] = a.ppsi[i];
  }
  const size_t spec = (size_t)p.nxh * p.ny;
  C<R>* jd = a.tape.jprev + (size_t)j * 2 * spec;
  for (size_t e = t0; e < 2 * spec; e += st) jd[e] = a.jprev[e];
}

template <typename R>
__global__ void __launch_bounds__(256, 2) sweep_kernel(SweepArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevParams& p = a.p;
  R* tile = reinterpret_cast<R*>(smem);
  C<R>* buf = reinterpret_cast<C<R>*>(smem);
  C<R>* tw = reinterpret_cast<C<R>*>(smem + phase_smem_bytes<R>(p.nx, p.ny));
  unsigned epoch = 0;
  // barrier with phase timing of the first slices
  auto sync = [&](int j, int ph) -> bool {
    const bool timed = a.ptimes != nullptr && j >= 0 && j < kTimedSlices && ph < kTimedPhases;
    unsigned long long* slot = timed ? a.ptimes + ((size_t)j * kTimedPhases + ph) * 2 : nullptr;
    if (!grid_sync(a.bar, epoch, slot)) return false;
    if (timed && blockIdx.x == 0 && threadIdx.x == 0) slot[1] = globaltimer();
    return true;
  };
  double psi0 = 0.0, ez0h = 0.0;

  const int u0 = blockIdx.x, G = gridDim.x;
  dep_phase(a, tile, DEP_INIT, 0, 0.0, false, false, u0, G);
  if (!sync(-1, 0)) return;
  row_phase(a, buf, tw, DEP_INIT, 0, u0, G, 1);
  if (!sync(-1, 1)) return;
  col_phase_psi(a, buf, tw, u0, G, 1, 0);
  if (!sync(-1, 2)) return;
  irow_phase(a, buf, tw, true, 0, false, 0.0, u0, G, 1);
  if (!sync(-1, 3)) return;

  // tolerance mode: every solve may be the last, so each one completes the slice's outputs
  // (slab, diagnostics), and the loop stops after the first that has converged
  const bool tol = p.pc_tol2 > 0.0;
  const bool rec = a.tape.part != nullptr;
  for (int j = 0; j < p.nk; ++j) {
    double ez0n = ez0h, ez0j = ez0h;
    int nsolve = p.n_pc;
    if (rec) record_tape(a, j, 0);
    for (int it = 0; it < p.n_pc; ++it) {
      const bool first = (it == 0), last = tol || (it == p.n_pc - 1);
      if (rec && it > 0) record_tape(a, j, it);
      dep_phase(a, tile, DEP_TRIAL, j, psi0, first, last, u0, G);
      if (!sync(j, 4 * it + 0)) return;
      row_phase(a, buf, tw, DEP_TRIAL, j, u0, G, 1);
      if (!sync(j, 4 * it + 1)) return;
      col_phase_b(a, buf, tw, j, last, psi0, u0, G, 1);
      if (!sync(j, 4 * it + 2)) return;
      if (last) {
        const double jz = *((volatile double*)&a.diag[D_JZ * p.nk + j]);
        ez0n = ez0h - p.dxi * jz;
        ez0j = 0.5 * (ez0h + ez0n);
      }
      irow_phase(a, buf, tw, false, j, last, ez0j, u0, G, 1);
      if (!sync(j, 4 * it + 3)) return;
      if (tol && it + 1 < p.n_pc && pc_converged(a, j)) {
        nsolve = it + 1;
        break;
      }
    }
    if (rec) record_tape(a, j, p.n_pc);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.diag[D_PSI0 * p.nk + j] = psi0;
      a.diag[D_EZ0 * p.nk + j] = ez0j;
      a.diag[D_NPC * p.nk + j] = (double)nsolve;
    }
    if (j + 1 < p.nk) {
      const int pc = 4 * p.n_pc;
      dep_phase(a, tile, DEP_COMMIT, j, psi0, false, false, u0, G);
      if (!sync(j, pc + 0)) return;
      row_phase(a, buf, tw, DEP_COMMIT, j + 1, u0, G, 1);
      if (!sync(j, pc + 1)) return;
      col_phase_psi(a, buf, tw, u0, G, 1, j + 1);
      if (!sync(j, pc + 2)) return;
      irow_phase(a, buf, tw, true, j + 1, false, 0.0, u0, G, 1);
      if (!sync(j, pc + 3)) return;
    }
    psi0 += p.dxi * ez0n;
    ez0h = ez0n;
  }
}

// Standalone transverse solve through the same phases: which = 0 solves B_x, B_y, B_z, E_z
// from the five trial fields placed in the overflow grid; which = 1 solves psi and its
// gradient from S placed in the overflow grid (field 0 of three).
template <typename R>
__global__ void __launch_bounds__(256, 2) solve_kernel(SweepArgs<R> a, int which) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevParams& p = a.p;
  C<R>* buf = reinterpret_cast<C<R>*>(smem);
  C<R>* tw = reinterpret_cast<C<R>*>(smem + phase_smem_bytes<R>(p.nx, p.ny));
  unsigned epoch = 0;
  const int u0 = blockIdx.x, G = gridDim.x;
  if (which == 0) {
    row_phase(a, buf, tw, DEP_TRIAL, 0, u0, G, 1);
    if (!grid_sync(a.bar, epoch)) return;
    col_phase_b(a, buf, tw, 0, false, 0.0, u0, G, 1);
    if (!grid_sync(a.bar, epoch)) return;
    irow_phase(a, buf, tw, false, 0, false, 0.0, u0, G, 1);
  } else {
    row_phase(a, buf, tw, DEP_COMMIT, 0, u0, G, 1);
    if (!grid_sync(a.bar, epoch)) return;
    col_phase_psi(a, buf, tw, u0, G, 1, -1);
    if (!grid_sync(a.bar, epoch)) return;
    irow_phase(a, buf, tw, true, 0, false, 0.0, u0, G, 1);
  }
}

}  // namespace qsa
