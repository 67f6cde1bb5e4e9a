// Re-homing the beam: moving every particle into a storage slot of the cell it now occupies.
//
// A beam slot s has a fixed lattice site (its home: cell (ix, iy) of xi layer k and a
// sub-lattice position); the particle it holds is stored as an offset from that site.  The
// push's fast paths (one gather of a cell's slab nodes for a thread's two particles,
// warp-aggregated deposits into the group's shared-memory tile) need the particle inside the
// home cell.  As the beam filaments, particles move tens of cells away from their sites.
// Re-homing permutes the particles of each xi layer among the layer's slots:
//   1. every live particle in a cell that holds at most ppc of them takes one of that cell's
//      own slots;
//   2. the excess particles of crowded cells fill the free slots of the other cells, matched
//      in row-major cell order (the k-th excess particle of the layer takes the k-th free
//      slot), so that an excess particle lands near where it is;
//   3. lost particles (dw = -1) fill the slots left over.
// Every slot still holds one particle, so the deposits' reference state (one reference
// particle per slot, at the slot's site) is unchanged, and the deposit of a particle of
// reference weight at its slot's site plus its deviation is the same quantity wherever it is
// stored: the sweep sees the same sources up to the order of the sums.  Each particle keeps its
// canonical id (BeamArrays::id), so host copies are unchanged.  The layer (xi cell of the
// slot) never changes: the beam barely slips in xi.
#pragma once
#include "qsa_beam.cuh"

namespace qsa {

constexpr int kRehomeThreads = 1024;

// Canonical ids of a beam that has not been re-homed yet: every slot its own particle.
template <typename BR>
__global__ void beam_id_init_kernel(BeamArrays<BR> b, DevParams p, SpeciesDev sp) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= b.n) return;
  b.id[s] = (unsigned)home_of(s, p.nx, p.ny, sp).id;
}

// Cell (within the layer) of every particle of layers [k0, k0 + nl), and the particle count of
// each cell; lost particles are counted apart (key -1).
template <typename BR>
__global__ void rehome_count_kernel(BeamArrays<BR> b, DevParams p, SpeciesDev sp, int k0, int nl,
                                    int* __restrict__ key, int* __restrict__ cnt) {
  const long long L = (long long)p.nx * p.ny * sp.ppc;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nl * L) return;
  const long long s = (long long)k0 * L + i;
  if (b.dw[s] == BR(-1)) {
    key[i] = -1;
    return;
  }
  const Home h = home_of(s, p.nx, p.ny, sp);
  const double x = h.ix + (h.sx + 0.5) / sp.ppx + (double)b.ox[s];
  const double y = h.iy + (h.sy + 0.5) / sp.ppy + (double)b.oy[s];
  const int cx = wrap((int)floor(x), p.nx), cy = wrap((int)floor(y), p.ny);
  const int c = (int)(i / L) * p.nx * p.ny + cy * p.nx + cx;
  key[i] = c;
  atomicAdd(cnt + c, 1);
}

// Per layer (one block each): exclusive prefix sums, in row-major cell order, of the excess
// particles max(cnt - ppc, 0) and of the free slots max(ppc - cnt, 0); zeroes the cursors.
__global__ void __launch_bounds__(kRehomeThreads) rehome_scan_kernel(
    DevParams p, int ppc, const int* __restrict__ cnt, int* __restrict__ exc0,
    int* __restrict__ vac0, int* __restrict__ cur) {
  __shared__ int se[kRehomeThreads], sv[kRehomeThreads];
  const int ncell = p.nx * p.ny;
  const size_t base = (size_t)blockIdx.x * ncell;
  const int per = (ncell + blockDim.x - 1) / blockDim.x;
  const int c0 = threadIdx.x * per, c1 = min(ncell, c0 + per);
  int e = 0, v = 0;
  for (int c = c0; c < c1; ++c) {
    const int n = cnt[base + c];
    e += max(n - ppc, 0);
    v += max(ppc - n, 0);
  }
  se[threadIdx.x] = e;
  sv[threadIdx.x] = v;
  __syncthreads();
  // inclusive scan of the per-thread sums (Hillis-Steele)
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    const int ae = threadIdx.x >= o ? se[threadIdx.x - o] : 0;
    const int av = threadIdx.x >= o ? sv[threadIdx.x - o] : 0;
    __syncthreads();
    se[threadIdx.x] += ae;
    sv[threadIdx.x] += av;
    __syncthreads();
  }
  e = se[threadIdx.x] - e;
  v = sv[threadIdx.x] - v;
  for (int c = c0; c < c1; ++c) {
    const int n = cnt[base + c];
    exc0[base + c] = e;
    vac0[base + c] = v;
    cur[base + c] = 0;
    e += max(n - ppc, 0);
    v += max(ppc - n, 0);
  }
}

// The new slot (within the layer) of every particle of layers [k0, k0 + nl); the record goes to
// the staging arrays t at that slot, with its offsets taken from the new slot's site.
template <typename BR>
__global__ void rehome_scatter_kernel(BeamArrays<BR> b, BeamArrays<BR> t, DevParams p,
                                      SpeciesDev sp, int k0, int nl, const int* __restrict__ key,
                                      const int* __restrict__ cnt, const int* __restrict__ exc0,
                                      const int* __restrict__ vac0, int* __restrict__ cur,
                                      int* __restrict__ dead_cur) {
  const int ncell = p.nx * p.ny, ppc = sp.ppc;
  const long long L = (long long)ncell * ppc;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nl * L) return;
  const int layer = (int)(i / L);
  const size_t lb = (size_t)layer * ncell;
  const long long s = (long long)k0 * L + i;
  const int kc = key[i];
  int cell, sub;
  if (kc >= 0) {
    const int c = kc - layer * ncell;
    const int r = atomicAdd(cur + lb + c, 1);
    if (r < ppc) {  // one of its own cell's slots
      cell = c;
      sub = r;
    } else {  // the (exc0 + r - ppc)-th excess particle takes the free slot of that rank
      const int rank = exc0[lb + c] + (r - ppc);
      int lo = 0, hi = ncell - 1;  // last cell whose free-slot prefix is <= rank
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vac0[lb + mid] <= rank) lo = mid;
        else hi = mid - 1;
      }
      // the free slots of cell lo are its subs cnt .. ppc - 1 (cnt < ppc there)
      cell = lo;
      sub = cnt[lb + lo] + (rank - vac0[lb + lo]);
    }
  } else {
    // lost particles take what is left: after the free slots the excess particles used,
    // in row-major order
    const int d = atomicAdd(dead_cur + layer, 1);
    // total excess of the layer = its free slots used; the leftover free slots follow them
    const int used = exc0[lb + ncell - 1] + max(cnt[lb + ncell - 1] - ppc, 0);
    const int rank = used + d;
    int lo = 0, hi = ncell - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (vac0[lb + mid] <= rank) lo = mid;
      else hi = mid - 1;
    }
    cell = lo;
    sub = cnt[lb + lo] + (rank - vac0[lb + lo]);
  }
  // storage index of (layer, cell, sub): ((k * ny + iy) * ppc + sub) * nx + ix
  const int cy = cell / p.nx, cx = cell - cy * p.nx;
  const long long k = (long long)k0 + layer;
  const long long d = ((k * p.ny + cy) * ppc + sub) * p.nx + cx;
  const long long di = d - (long long)k0 * L;
  const Home ho = home_of(s, p.nx, p.ny, sp), hn = home_of(d, p.nx, p.ny, sp);
  // the same position, as offsets from the new site (nearest periodic image), in FP64; a lost
  // particle keeps its last position too (nothing reads it but the host copy)
  double ox = ho.ix + (ho.sx + 0.5) / sp.ppx + (double)b.ox[s] - (hn.ix + (hn.sx + 0.5) / sp.ppx);
  double oy = ho.iy + (ho.sy + 0.5) / sp.ppy + (double)b.oy[s] - (hn.iy + (hn.sy + 0.5) / sp.ppy);
  ox -= p.nx * rint(ox / p.nx);
  oy -= p.ny * rint(oy / p.ny);
  const double oxi = (ho.sxi + 0.5) / sp.ppxi + (double)b.oxi[s] - (hn.sxi + 0.5) / sp.ppxi;
  t.ox[di] = BR(ox);
  t.oy[di] = BR(oy);
  t.oxi[di] = BR(oxi);
  t.ux[di] = b.ux[s];
  t.uy[di] = b.uy[s];
  t.uz[di] = b.uz[s];
  t.dw[di] = b.dw[s];
  t.id[di] = b.id[s];
}

}  // namespace qsa
