// Pipelined beam steps: one persistent cooperative launch advances up to kMaxPipe beam steps
// (plasma sweep + beam push each) as a wavefront in xi.
//
// Why it is exact.  The sweep of step n at slice j reads the beam sources of nodes j and j+1
// only, and a beam particle only moves backwards in the window (d xi / d tau = 1 - v_z > 0).
// So the sources of step n at node j are complete once every home layer c <= j (+ margin, see
// below) has been pushed by step n-1; and the push of layer c by step n-1 needs the slab of
// step n-1 only up to node cmax[c] + 1, cmax[c] being the largest xi cell that a live particle
// of layer c occupies.  Step n can therefore run a few slices behind step n-1 instead of
// after it, and every block works on all steps in flight in each phase: the same arithmetic
// in a different order (summation order of the atomics aside).
//
// Schedule.  The launch proceeds in ticks.  In a tick each step in flight whose inputs are
// ready processes one slice (the n_pc trial iterations and the commit, the same 4 (n_pc + 1)
// grid-wide phases as the single sweep, each phase covering the units of all steps), and
// pushes the layers whose slab nodes are complete (commit slot).  Gates, evaluated by every
// block on identical data after a grid barrier:
//   step s processes slice j (j = -1: the initial psi solve)  iff  s is the first step of the
//     launch, or step s-1 has pushed layers 0 .. min(nxi, j + 2 + m) - 1, where m >= 0 is the
//     largest distance by which a live particle sits ahead of its home layer (set at the last
//     deposit of the sources; pushes only increase xi);
//   step s pushes layer c (layers in order, at most max_push per tick)  iff  step s-1 (if in
//     this launch) has pushed it and the slab of step s holds nodes 0 .. cmax_s[c] + 1 by the
//     commit slot of this tick.
// With no drift (cmax[c] = c) consecutive steps run three slices apart.
//
// Buffers.  Step i of the launch (global step g0 + i) uses sweep slot i (plasma state,
// scratch, slab, diagnostics) and reads the source buffer (g0 + i) mod (S + 1) of a ring of
// S + 1; its push writes buffer (g0 + i + 1) mod (S + 1) and the extent ring entry of the same
// index.  The host zeroes the buffers written by the launch before it starts.
#pragma once
#include "qsa_beam.cuh"
#include "qsa_sweep.cuh"

namespace qsa {

constexpr int kMaxPipe = 16;
constexpr int kMaxSpecies = 4;
// rows (half-spectrum columns) per unit of the FFT phases, and resident blocks per SM
constexpr int kPipeRowBatch = 2;
constexpr int kPipeColBatch = 1;
constexpr int kPipeBlocksPerSM = 4;

template <typename R>
struct PipeTable {
  SweepArgs<R> st[kMaxPipe];    // sweep slots (src is taken from the ring)
  R* srcbuf[kMaxPipe + 1];      // source ring [nk][ny][nx][4]
  int* cmaxbuf[kMaxPipe + 1];   // extent ring: largest live xi cell per home layer [nxi]
  double* mombuf[kMaxPipe + 1]; // beam-moment ring [nspecies][nxi][7]
  int nslot;                    // S: slots in use; the rings hold S + 1 entries
  int nspecies;
  int max_push;                 // layers a step pushes per tick at most
  BeamArrays<R> beam[kMaxSpecies];
  SpeciesDev sp[kMaxSpecies];
  BeamConst<R> bc[kMaxSpecies];
  const int* dmin;              // min over live particles of (xi cell - home layer), <= 0
  unsigned long long* lost;
};

// First unit of this block among U units of the k-th active step, the units of all active
// steps laid end to end and dealt round-robin to the G blocks.
__device__ __forceinline__ int unit0(int k, int U, int G) {
  int r = ((int)blockIdx.x - k * U) % G;
  return r < 0 ? r + G : r;
}

template <typename R>
__global__ void __launch_bounds__(256, kPipeBlocksPerSM)
    pipe_kernel(const PipeTable<R>* __restrict__ T, int r0, int nsteps, Barrier bar) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SweepArgs<R> sa[kMaxPipe];
  __shared__ BeamArrays<R> sb[kMaxSpecies];
  __shared__ SpeciesDev ssp[kMaxSpecies];
  __shared__ BeamConst<R> sbc[kMaxSpecies];
  __shared__ int js[kMaxPipe], pf[kMaxPipe], npush[kMaxPipe], adv[kMaxPipe];
  __shared__ double psi0[kMaxPipe], ez0h[kMaxPipe], ez0n[kMaxPipe], ez0j[kMaxPipe];
  __shared__ int act_t[kMaxPipe], act_c[kMaxPipe];
  __shared__ int n_t, n_c, stop, margin;
  const int tid = threadIdx.x, G = gridDim.x;
  {
    const int nw = (int)(nsteps * sizeof(SweepArgs<R>) / 4);
    const int* srcw = reinterpret_cast<const int*>(T->st);
    int* dstw = reinterpret_cast<int*>(sa);
    for (int i = tid; i < nw; i += blockDim.x) dstw[i] = srcw[i];
  }
  const int S1 = T->nslot + 1;
  if (tid == 0) {
    for (int i = 0; i < nsteps; ++i) {
      js[i] = -1;
      pf[i] = 0;
      psi0[i] = ez0h[i] = ez0n[i] = ez0j[i] = 0.0;
    }
    for (int k = 0; k < T->nspecies; ++k) {
      sb[k] = T->beam[k];
      ssp[k] = T->sp[k];
      sbc[k] = T->bc[k];
    }
    const int dm = *((volatile const int*)T->dmin);
    margin = dm < 0 ? -dm : 0;
  }
  __syncthreads();
  if (tid < nsteps) sa[tid].src = T->srcbuf[(r0 + tid) % S1];
  __syncthreads();

  const DevParams& p = sa[0].p;
  const int nx = p.nx, ny = p.ny, nxh = p.nxh, nk = p.nk, nxi = p.nxi;
  const int nspec = T->nspecies, max_push = T->max_push;
  R* tile = reinterpret_cast<R*>(smem);
  C<R>* buf = reinterpret_cast<C<R>*>(smem);
  constexpr int nbr = kPipeRowBatch, nbc = kPipeColBatch;
  const int ur = (ny + nbr - 1) / nbr, uc = (nxh + nbc - 1) / nbc;  // FFT units per step
  C<R>* tw = reinterpret_cast<C<R>*>(smem + phase_smem_bytes<R>(nx, ny, nbr, nbc));
  unsigned epoch = 0;
  // every tick processes at least one slice or one layer, so this bound is never reached by
  // a correct schedule; it keeps a scheduling fault from spinning forever
  const long long max_ticks = (long long)(nk + 1 + 3 * nsteps) * (nsteps + 1) + 2LL * nxi + 64;

  for (long long tick = 0;; ++tick) {
    if (tid == 0) {
      // plan of this tick (identical in every block)
      const int m = margin;
      int nt = 0, nc = 0, all_done = 1;
      for (int s = 0; s < nsteps; ++s) {
        int a = 0;
        if (js[s] < nk) {
          if (s == 0) {
            a = 1;
          } else {
            const int need = min(nxi, js[s] + 2 + m);
            a = pf[s - 1] >= need;
          }
        }
        adv[s] = a;
        if (a && js[s] >= 0) act_t[nt++] = s;
        if (a && js[s] < nk - 1) act_c[nc++] = s;
        // slab nodes 0 .. ready - 1 of step s are complete at the commit slot of this tick
        const int ready = js[s] + ((a && js[s] >= 0) ? 1 : 0);
        const volatile int* cm = T->cmaxbuf[(r0 + s) % S1];
        int c = pf[s], n = 0;
        while (c < nxi && n < max_push) {
          if (s > 0 && c >= pf[s - 1]) break;
          if (cm[c] + 2 > ready) break;
          ++c;
          ++n;
        }
        npush[s] = n;
        if (js[s] < nk || pf[s] < nxi) all_done = 0;
      }
      n_t = nt;
      n_c = nc;
      stop = all_done ? 1 : (tick >= max_ticks ? 2 : 0);
      if (stop == 2 && blockIdx.x == 0) atomicOr(bar.status, ST_TIMEOUT);
    }
    __syncthreads();
    if (stop) break;

    // ---- trial iterations of the steps that process a slice
    const int nt = n_t;
    if (nt > 0) {
      for (int it = 0; it < p.n_pc; ++it) {
        const bool first = (it == 0), last = (it == p.n_pc - 1);
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          dep_phase(sa[s], tile, DEP_TRIAL, js[s], psi0[s], first, last, unit0(k, ny, G), G);
        }
        if (!grid_sync(bar, epoch)) return;
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          row_phase(sa[s], buf, tw, DEP_TRIAL, js[s], unit0(k, ur, G), G, nbr);
        }
        if (!grid_sync(bar, epoch)) return;
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          col_phase_b(sa[s], buf, tw, js[s], last, psi0[s], unit0(k, uc, G), G, nbc);
        }
        if (!grid_sync(bar, epoch)) return;
        if (last) {
          if (tid == 0) {
            for (int k = 0; k < nt; ++k) {
              const int s = act_t[k], j = js[s];
              const double jz = *((volatile double*)&sa[s].diag[D_JZ * nk + j]);
              ez0n[s] = ez0h[s] - p.dxi * jz;
              ez0j[s] = 0.5 * (ez0h[s] + ez0n[s]);
              if (blockIdx.x == 0) {
                sa[s].diag[D_PSI0 * nk + j] = psi0[s];
                sa[s].diag[D_EZ0 * nk + j] = ez0j[s];
              }
            }
          }
          __syncthreads();
        }
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          irow_phase(sa[s], buf, tw, false, js[s], last, ez0j[s], unit0(k, ur, G), G, nbr);
        }
        if (!grid_sync(bar, epoch)) return;
      }
    }

    // ---- commit slot: commit (or initial) deposits, and the beam pushes
    const int nc = n_c;
    for (int k = 0; k < nc; ++k) {
      const int s = act_c[k];
      if (js[s] < 0)
        dep_phase(sa[s], tile, DEP_INIT, 0, 0.0, false, false, unit0(k, ny, G), G);
      else
        dep_phase(sa[s], tile, DEP_COMMIT, js[s], psi0[s], false, false, unit0(k, ny, G), G);
    }
    {
      int base = nc * ny;
      for (int s = 0; s < nsteps; ++s) {
        const int n = npush[s];
        if (n == 0) continue;
        R* src_next = T->srcbuf[(r0 + s + 1) % S1];
        int* cmax_next = T->cmaxbuf[(r0 + s + 1) % S1];
        double* mom_next = T->mombuf[(r0 + s + 1) % S1];
        const R* slab = sa[s].slab;
        for (int c = pf[s]; c < pf[s] + n; ++c) {
          for (int si = 0; si < nspec; ++si) {
            const SpeciesDev& sp = ssp[si];
            if (c < sp.k0 || c >= sp.k0 + sp.nkb) continue;
            int q0 = ((int)blockIdx.x - base) % G;
            if (q0 < 0) q0 += G;
            for (int q = q0; q < ny; q += G)
              beam_group<R, true>(sb[si], p, sp, sbc[si], slab, src_next, T->lost,
                                  Extent{cmax_next, nullptr, mom_next + (size_t)si * nxi * 7},
                                  (c - sp.k0) * ny + q, tile);
            base += ny;
          }
        }
      }
    }
    if (!grid_sync(bar, epoch)) return;
    if (nc > 0) {
      for (int k = 0; k < nc; ++k) {
        const int s = act_c[k];
        row_phase(sa[s], buf, tw, js[s] < 0 ? DEP_INIT : DEP_COMMIT, js[s] + 1,
                  unit0(k, ur, G), G, nbr);
      }
      if (!grid_sync(bar, epoch)) return;
      for (int k = 0; k < nc; ++k) {
        const int s = act_c[k];
        col_phase_psi(sa[s], buf, tw, unit0(k, uc, G), G, nbc, js[s] + 1);
      }
      if (!grid_sync(bar, epoch)) return;
      for (int k = 0; k < nc; ++k) {
        const int s = act_c[k];
        irow_phase(sa[s], buf, tw, true, js[s] + 1, false, 0.0, unit0(k, ur, G), G, nbr);
      }
      if (!grid_sync(bar, epoch)) return;
    }
    // ---- advance the per-step state
    if (tid == 0) {
      for (int s = 0; s < nsteps; ++s) {
        if (adv[s]) {
          if (js[s] >= 0) {
            psi0[s] += p.dxi * ez0n[s];
            ez0h[s] = ez0n[s];
          }
          ++js[s];
        }
        pf[s] += npush[s];
      }
    }
    // the next tick's plan (thread 0) is followed by a __syncthreads before any use
  }
}

template <typename R>
__host__ __device__ inline size_t pipe_smem_bytes(int nx, int ny) {
  const size_t a = sweep_smem_bytes<R>(nx, ny, kPipeRowBatch, kPipeColBatch),
               b = beam_smem_bytes<R>(nx);
  return a > b ? a : b;
}

}  // namespace qsa
