// Persistent multi-slot launch: up to kMaxPipe plasma sweeps, each followed by its beam push,
// advance together, every grid-wide phase covering the work units of all of them.  A slot is
// one sweep + push with its own grid, plasma state, scratch, slab, beam and source buffers.
// Two uses:
//   chained: the slots are consecutive beam steps of one instance (qsa_advance), run as a
//     wavefront in xi;
//   independent: the slots are separate instances, possibly of different grid sizes
//     (qsa_advance_batch), each advancing by one step.
//
// Why the chained wavefront is exact.  The sweep of step n at slice j reads the beam sources
// of nodes j and j+1 only, and a beam particle only moves backwards in the window
// (d xi / d tau = 1 - v_z > 0).  So the sources of step n at node j are complete once every
// home layer c <= j (+ margin, see below) has been pushed by step n-1; and the push of layer c
// by step n-1 needs the slab of step n-1 only up to node cmax[c] + 1, cmax[c] being the
// largest xi cell that a live particle of layer c occupies.  Step n can therefore run a few
// slices behind step n-1 instead of after it: the same arithmetic in a different order
// (summation order of the atomics aside).
//
// Schedule.  The launch proceeds in ticks.  In a tick each slot whose inputs are ready
// processes one slice (the n_pc trial iterations and the commit: the same 4 (n_pc + 1)
// grid-wide phases as the single sweep), and pushes the layers whose slab nodes are complete
// (commit slot).  Gates, evaluated by every block on identical data after a grid barrier:
//   slot s processes slice j (j = -1: the initial psi solve)  iff  the slots are independent,
//     or s is the first slot, or slot s-1 has pushed layers 0 .. min(nxi, j + 2 + m) - 1,
//     where m >= 0 is the largest distance by which a live particle sits ahead of its home
//     layer (set at the last deposit of the sources; pushes only increase xi);
//   slot s pushes layer c (layers in order, at most max_push per tick)  iff  (chained and
//     s > 0) slot s-1 has pushed it, and the slab of slot s holds nodes 0 .. cmax_s[c] + 1 by
//     the commit slot of this tick.
// With no drift (cmax[c] = c) consecutive chained steps run three slices apart.
//
// The work units of the slots of a phase are laid end to end and dealt round-robin to the
// blocks; FFT units hold nbr rows / nbc half-spectrum columns (a launch parameter: the
// autotuner of the batched path picks it).
#pragma once
#include "qsa_beam.cuh"
#include "qsa_sweep.cuh"

namespace qsa {

constexpr int kMaxPipe = 16;
constexpr int kMaxSpecies = 4;
// resident blocks per SM the register budget is set for (a build setting for tuning): three
// (85 registers a thread) run the late, filamented beam faster than four (64), at the same
// linear-stage speed
#ifndef QSA_PIPE_BLOCKS_PER_SM
#define QSA_PIPE_BLOCKS_PER_SM 3
#endif
constexpr int kPipeBlocksPerSM = QSA_PIPE_BLOCKS_PER_SM;

// The beam side of one slot: its push reads cmax_in and the slot's slab, and writes the
// sources of the next sweep (src_next), the extents cmax_out and the beam moments mom_out.
template <typename R>
struct PipeSlot {
  R* src_next;
  const int* cmax_in;   // [nxi]
  int* cmax_out;        // [nxi]
  double* mom_out;      // [nspecies][nxi][7], or null (moments not needed)
  const int* dmin;      // min over live particles of (xi cell - home layer), <= 0
  unsigned long long* lost;
  unsigned long long* away;  // live particles outside their slots' cells after the pushes, or null
  int nspecies;
  BeamArrays<R> beam[kMaxSpecies];
  SpeciesDev sp[kMaxSpecies];
  BeamConst<R> bc[kMaxSpecies];
};

template <typename R>
struct PipeTable {
  SweepArgs<R> st[kMaxPipe];  // sweep of each slot (src: the sources it reads)
  PipeSlot<R> slot[kMaxPipe];
  int chained;                // 1: consecutive steps of one instance
  int max_push;               // layers a slot pushes per tick at most
  int nbr, nbc;               // rows / half-spectrum columns per FFT unit
  int nx_max, ny_max;         // largest grid of the slots (shared-memory layout)
};

template <typename R>
__host__ __device__ inline size_t pipe_smem_bytes(int nx_max, int ny_max, int nbr, int nbc) {
  const size_t a = sweep_smem_bytes<R>(nx_max, ny_max, nbr, nbc), b = beam_smem_bytes<R>(nx_max);
  return a > b ? a : b;
}

// First unit of this block when units off .. off + U - 1 of a phase belong to one slot and
// all units are dealt round-robin to the G blocks.
__device__ __forceinline__ int unit0(int off, int G) {
  int r = ((int)blockIdx.x - off) % G;
  return r < 0 ? r + G : r;
}

template <typename R>
__global__ void __launch_bounds__(256, kPipeBlocksPerSM)
    pipe_kernel(const PipeTable<R>* __restrict__ T, int nslots, Barrier bar) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SweepArgs<R> sa[kMaxPipe];
  __shared__ int js[kMaxPipe], pf[kMaxPipe], npush[kMaxPipe], adv[kMaxPipe], margin[kMaxPipe];
  __shared__ double psi0[kMaxPipe], ez0h[kMaxPipe], ez0n[kMaxPipe], ez0j[kMaxPipe];
  // active slots of the trial phases (t) and of the commit slot (c), with the offsets of
  // their first work item in each phase (deposit rows; inverse-row items (row); FFT columns;
  // forward-row items (rowf); beam groups)
  __shared__ int act_t[kMaxPipe], act_c[kMaxPipe];
  __shared__ int ot_dep[kMaxPipe], ot_row[kMaxPipe], ot_col[kMaxPipe], ot_rowf[kMaxPipe];
  __shared__ int oc_dep[kMaxPipe], oc_row[kMaxPipe], oc_col[kMaxPipe], oc_rowf[kMaxPipe];
  __shared__ int o_push[kMaxPipe];
  __shared__ int ngrp[kMaxPipe];  // beam groups each slot pushes in this tick
  __shared__ int pcdone[kMaxPipe];  // tolerance mode: the slot's slice has converged
  __shared__ int n_t, n_c, stop;
  const int tid = threadIdx.x, G = gridDim.x;
  {
    const int nw = (int)(nslots * sizeof(SweepArgs<R>) / 4);
    const int* srcw = reinterpret_cast<const int*>(T->st);
    int* dstw = reinterpret_cast<int*>(sa);
    for (int i = tid; i < nw; i += blockDim.x) dstw[i] = srcw[i];
  }
  const int chained = T->chained, max_push = T->max_push, nbr = T->nbr, nbc = T->nbc;
  if (tid == 0) {
    for (int i = 0; i < nslots; ++i) {
      js[i] = -1;
      pf[i] = 0;
      psi0[i] = ez0h[i] = ez0n[i] = ez0j[i] = 0.0;
      const int dm = *((volatile const int*)T->slot[i].dmin);
      margin[i] = dm < 0 ? -dm : 0;
    }
  }
  __syncthreads();

  R* tile = reinterpret_cast<R*>(smem);
  C<R>* buf = reinterpret_cast<C<R>*>(smem);
  C<R>* tw = reinterpret_cast<C<R>*>(smem + phase_smem_bytes<R>(T->nx_max, T->ny_max, nbr, nbc));
  const int n_pc = sa[0].p.n_pc;  // the same in every slot
  const bool tol = sa[0].p.pc_tol2 > 0.0;  // so is the predictor-corrector tolerance
  unsigned epoch = 0;
  // every tick processes at least one slice or one layer, so this bound is never reached by
  // a correct schedule; it keeps a scheduling fault from spinning forever
  long long max_ticks = 64;
  for (int i = 0; i < nslots; ++i) max_ticks += 2LL * sa[i].p.nk + 3 + 2LL * sa[i].p.nxi;
  max_ticks *= chained ? nslots : 1;

  for (long long tick = 0;; ++tick) {
    __syncthreads();  // the state thread 0 advanced at the end of the previous tick
    if (tid < nslots) {
      // per-slot part of the plan, one thread per slot: slot s reads only what the previous
      // tick left (its own state and slot s - 1's pf), so the slots are independent
      const int s = tid;
      const DevParams& p = sa[s].p;
      const int nk = p.nk, nxi = p.nxi;
      int a = 0;
      if (js[s] < nk) {
        if (!chained || s == 0) {
          a = 1;
        } else {
          const int need = min(nxi, js[s] + 2 + margin[s]);
          a = pf[s - 1] >= need;
        }
      }
      adv[s] = a;
      // slab nodes 0 .. ready - 1 of slot s are complete at the commit slot of this tick
      const int ready = js[s] + ((a && js[s] >= 0) ? 1 : 0);
      const volatile int* cm = T->slot[s].cmax_in;
      int c = pf[s], n = 0;
      while (c < nxi && n < max_push) {
        if (chained && s > 0 && c >= pf[s - 1]) break;
        if (cm[c] + 2 > ready) break;
        ++c;
        ++n;
      }
      npush[s] = n;
      // beam groups of the layers pushed: ny per layer and species present there
      const PipeSlot<R>& ps = T->slot[s];
      int ng = 0;
      for (int l = pf[s]; l < pf[s] + n; ++l)
        for (int si = 0; si < ps.nspecies; ++si)
          if (l >= ps.sp[si].k0 && l < ps.sp[si].k0 + ps.sp[si].nkb) ng += p.ny;
      ngrp[s] = ng;
    }
    __syncthreads();
    if (tid == 0) {
      // offsets of each slot's units in the phases of this tick (identical in every block)
      int nt = 0, nc = 0, all_done = 1;
      int udep = 0, urow = 0, ucol = 0, cdep = 0, crow = 0, ccol = 0, urowf = 0, crowf = 0;
      for (int s = 0; s < nslots; ++s) {
        const DevParams& p = sa[s].p;
        const int nk = p.nk, a = adv[s];
        const int uc = col_units<R>(p, nbc);
        if (a && js[s] >= 0) {
          ot_dep[nt] = udep;
          ot_row[nt] = urow;
          ot_col[nt] = ucol;
          ot_rowf[nt] = urowf;
          udep += p.ny;
          urow += irow_tasks<R>(p, nbr);
          ucol += uc;
          urowf += row_tasks<R>(p, nbr, DEP_TRIAL);
          act_t[nt++] = s;
        }
        pcdone[s] = 0;
        if (a && js[s] < nk - 1) {
          oc_dep[nc] = cdep;
          oc_row[nc] = crow;
          oc_col[nc] = ccol;
          oc_rowf[nc] = crowf;
          cdep += p.ny;
          crow += irow_tasks<R>(p, nbr);
          ccol += uc;
          crowf += row_tasks<R>(p, nbr, DEP_COMMIT);
          act_c[nc++] = s;
        }
        if (js[s] < nk || pf[s] < p.nxi) all_done = 0;
      }
      // beam groups of the commit slot follow its deposit units
      int up = cdep;
      for (int s = 0; s < nslots; ++s) {
        o_push[s] = up;
        up += ngrp[s];
      }
      n_t = nt;
      n_c = nc;
      stop = all_done ? 1 : (tick >= max_ticks ? 2 : 0);
      if (stop == 2 && blockIdx.x == 0) atomicOr(bar.status, ST_TIMEOUT);
    }
    __syncthreads();
    if (stop) break;

    // ---- trial iterations of the slots that process a slice
    const int nt = n_t;
    if (nt > 0) {
      // tolerance mode: every solve may be a slot's last, so each completes the slice's
      // outputs; a slot whose B_perp has converged skips the remaining solves (its units
      // idle), and the loop ends once every slot has
      for (int it = 0; it < n_pc; ++it) {
        const bool first = (it == 0), last = tol || (it == n_pc - 1);
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          if (pcdone[s]) continue;
          dep_phase(sa[s], tile, DEP_TRIAL, js[s], psi0[s], first, last, unit0(ot_dep[k], G), G);
        }
        if (!grid_sync(bar, epoch)) return;
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          if (pcdone[s]) continue;
          row_phase(sa[s], buf, tw, DEP_TRIAL, js[s], unit0(ot_rowf[k], G), G, nbr);
        }
        if (!grid_sync(bar, epoch)) return;
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          if (pcdone[s]) continue;
          col_phase_b(sa[s], buf, tw, js[s], last, psi0[s], unit0(ot_col[k], G), G, nbc);
        }
        if (!grid_sync(bar, epoch)) return;
        if (last) {
          // one thread per active slot (distinct slots: no two threads share an entry)
          if (tid < nt && !pcdone[act_t[tid]]) {
            const int s = act_t[tid], j = js[s], nk = sa[s].p.nk;
            const double jz = *((volatile double*)&sa[s].diag[D_JZ * nk + j]);
            ez0n[s] = ez0h[s] - sa[s].p.dxi * jz;
            ez0j[s] = 0.5 * (ez0h[s] + ez0n[s]);
            if (blockIdx.x == 0) {
              sa[s].diag[D_PSI0 * nk + j] = psi0[s];
              sa[s].diag[D_EZ0 * nk + j] = ez0j[s];
              sa[s].diag[D_NPC * nk + j] = (double)(it + 1);
            }
          }
          __syncthreads();
        }
        for (int k = 0; k < nt; ++k) {
          const int s = act_t[k];
          if (pcdone[s]) continue;
          irow_phase(sa[s], buf, tw, false, js[s], last, ez0j[s], unit0(ot_row[k], G), G, nbr);
        }
        if (!grid_sync(bar, epoch)) return;
        if (tol && it + 1 < n_pc) {
          int left = 0;
          for (int k = 0; k < nt; ++k) {
            const int s = act_t[k];
            if (pcdone[s]) continue;
            if (pc_converged(sa[s], js[s])) {
              if (tid == 0) pcdone[s] = 1;
            } else {
              ++left;
            }
          }
          __syncthreads();
          if (left == 0) break;
        }
      }
    }

    // ---- commit slot: commit (or initial) deposits, and the beam pushes
    const int nc = n_c;
    for (int k = 0; k < nc; ++k) {
      const int s = act_c[k];
      if (js[s] < 0)
        dep_phase(sa[s], tile, DEP_INIT, 0, 0.0, false, false, unit0(oc_dep[k], G), G);
      else
        dep_phase(sa[s], tile, DEP_COMMIT, js[s], psi0[s], false, false, unit0(oc_dep[k], G),
                  G);
    }
    for (int s = 0; s < nslots; ++s) {
      const int n = npush[s];
      if (n == 0) continue;
      const PipeSlot<R>& ps = T->slot[s];
      const DevParams& p = sa[s].p;
      int base = o_push[s];
      for (int c = pf[s]; c < pf[s] + n; ++c) {
        for (int si = 0; si < ps.nspecies; ++si) {
          const SpeciesDev& sp = ps.sp[si];
          if (c < sp.k0 || c >= sp.k0 + sp.nkb) continue;
          for (int q = unit0(base, G); q < p.ny; q += G)
            beam_group<R, true>(ps.beam[si], p, sp, ps.bc[si], sa[s].slab, ps.src_next,
                                ps.lost,
                                Extent{ps.cmax_out, nullptr,
                                       ps.mom_out ? ps.mom_out + (size_t)si * p.nxi * 7
                                                  : nullptr,
                                       ps.away},
                                (c - sp.k0) * p.ny + q, tile);
          base += p.ny;
        }
      }
    }
    if (!grid_sync(bar, epoch)) return;
    if (nc > 0) {
      for (int k = 0; k < nc; ++k) {
        const int s = act_c[k];
        row_phase(sa[s], buf, tw, js[s] < 0 ? DEP_INIT : DEP_COMMIT, js[s] + 1,
                  unit0(oc_rowf[k], G), G, nbr);
      }
      if (!grid_sync(bar, epoch)) return;
      for (int k = 0; k < nc; ++k) {
        const int s = act_c[k];
        col_phase_psi(sa[s], buf, tw, unit0(oc_col[k], G), G, nbc, js[s] + 1);
      }
      if (!grid_sync(bar, epoch)) return;
      for (int k = 0; k < nc; ++k) {
        const int s = act_c[k];
        irow_phase(sa[s], buf, tw, true, js[s] + 1, false, 0.0, unit0(oc_row[k], G), G, nbr);
      }
      if (!grid_sync(bar, epoch)) return;
    }
    // ---- advance the per-slot state
    if (tid == 0) {
      for (int s = 0; s < nslots; ++s) {
        if (adv[s]) {
          if (js[s] >= 0) {
            psi0[s] += sa[s].p.dxi * ez0n[s];
            ez0h[s] = ez0n[s];
          }
          ++js[s];
        }
        pf[s] += npush[s];
      }
    }
  }
}

}  // namespace qsa
